"""GPU parity of the hand-written adjoint against the oracle's analytic FP64
gradient (itself pinned to central finite differences), on the
differentiation workload: the 4,096-Gaussian uniform scene restricted to a
1,024-Gaussian, 16-direction subset (16,384 rays), L = sum_r w_r T_r with
w_r ~ U(0,1), T_min = 0.  Bar: 1e-3 relative (vector norm per parameter
group), and per component 1e-3 relative plus 2e-5 of the group's largest
component (see _check)."""
import numpy as np
import pytest
import torch

import scenes
from conftest import check_flagged_bounds

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def case(orc):
    sc = scenes.uniform_scene(4096, 4)
    sub = {k: v[:1024].copy() for k, v in sc.items()}
    dirs = scenes.fibonacci_sphere(16)
    R = 1024 * 16
    ids = np.arange(R, dtype=np.int64)
    o, d, s = orc.dir_rays(sub["mean"], dirs, ids)
    w = scenes.loss_weights(R, 41).astype(np.float64)
    ref = orc.trace(sub, o, d, s, t_min=0.0)
    w[ref["flags"] != 0] = 0.0  # rays at a threshold are excluded on both sides
    g = orc.trace_grad(sub, o, d, s, w, t_min=0.0, with_origin=True)
    # rays start at mu_src + eps d: their origin gradient belongs to the source mean
    gm = g["mean"].copy()
    np.add.at(gm, s, g["ray_o"])
    return sub, dirs, w, {"mean": gm, "scale": g["scale"], "quat": g["quat"], "opacity": g["opacity"]}, ref


def _check(got, want, name):
    """1e-3 relative as a vector norm per parameter group, and per component
    |got - want| <= 1e-3 |want| + 2e-5 max|want| for every component.  The
    absolute term is the float32 evaluation of the chain rule: each
    component is a sum over hits of terms computed with ~1e-6 relative
    error, some of them as large as the group's largest component, and a
    mean component also collects the origin gradients of its own rays, which
    largely cancel its hit terms; the float64-exact (fixed-point) summation
    shows the same error, so it is not the atomics' order."""
    got = np.asarray(got, np.float64)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < 1e-3, (name, rel)
    tol = 1e-3 * np.abs(want) + 2e-5 * np.abs(want).max()
    err = np.abs(got - want)
    assert np.all(err <= tol), (name, float((err / tol).max()))


@pytest.mark.parametrize("use_log", [True, False])
def test_backward_matches_oracle(case, use_log):
    from paper_2311_16043_gb300 import rt
    sub, dirs, w, want, ref = case
    dv = {k: _dev(v) for k, v in sub.items()}
    bvh = rt.rt_build_bvh(dv["mean"], dv["scale"], dv["quat"], dv["opacity"], rt.params(t_min=0.0))
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
    R = 1024 * 16
    hit_ids = torch.empty((R, 64), dtype=torch.int32, device="cuda") if use_log else None
    hit_cnt = torch.empty(R, dtype=torch.int32, device="cuda") if use_log else None
    T = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(hit_ids=hit_ids, hit_count=hit_cnt))
    g = rt.rt_trace_visibility_backward(bvh, rs, dv["mean"], dv["scale"], dv["quat"], dv["opacity"], T,
                                        _dev(w.astype(np.float32)), hit_ids, hit_cnt)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    assert np.abs(T.cpu().numpy() - ref["T"])[ref["flags"] == 0].max() < 1e-5
    check_flagged_bounds(T.cpu().numpy(), ref, 1e-5, t_min=0.0)
    for k in ("opacity", "mean", "scale", "quat"):
        _check(g[k].cpu().numpy(), want[k], k)


def test_partial_log_replays_and_recomputes(case):
    """A log too small for some rays: those rays are re-traversed, the rest
    replayed; the gradient is the same."""
    from paper_2311_16043_gb300 import rt
    sub, dirs, w, want, _ = case
    dv = {k: _dev(v) for k, v in sub.items()}
    bvh = rt.rt_build_bvh(dv["mean"], dv["scale"], dv["quat"], dv["opacity"], rt.params(t_min=0.0))
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
    R = 1024 * 16
    hit_ids = torch.empty((R, 2), dtype=torch.int32, device="cuda")
    hit_cnt = torch.empty(R, dtype=torch.int32, device="cuda")
    T = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(hit_ids=hit_ids, hit_count=hit_cnt))
    g = rt.rt_trace_visibility_backward(bvh, rs, dv["mean"], dv["scale"], dv["quat"], dv["opacity"], T,
                                        _dev(w.astype(np.float32)), hit_ids, hit_cnt)
    torch.cuda.synchronize()
    assert (hit_cnt > 2).any().item() and (hit_cnt <= 2).any().item()
    for k in ("opacity", "mean", "scale", "quat"):
        _check(g[k].cpu().numpy(), want[k], k)


def test_autograd_function_log_scale(case):
    """torch.autograd.Function with a log-scale parameterisation."""
    from paper_2311_16043_gb300 import autograd, rt
    sub, dirs, w, want, _ = case
    mean = _dev(sub["mean"]).requires_grad_()
    log_s = _dev(np.log(sub["scale"])).requires_grad_()
    quat = _dev(sub["quat"]).requires_grad_()
    opac = _dev(sub["opacity"]).requires_grad_()
    for budget in (1 << 30, 0):  # with a hit log, then recompute only
        for t in (mean, log_s, quat, opac):
            t.grad = None
        T = autograd.visibility(mean, log_s.exp(), quat, opac, _dev(dirs), rt.params(t_min=0.0),
                                log_budget_bytes=budget)
        L = (T.reshape(-1) * _dev(w.astype(np.float32))).sum()
        L.backward()
        torch.cuda.synchronize()
        _check(opac.grad.cpu().numpy(), want["opacity"], "opacity")
        _check(mean.grad.cpu().numpy(), want["mean"], "mean")
        _check(quat.grad.cpu().numpy(), want["quat"], "quat")
        _check(log_s.grad.cpu().numpy(), want["scale"] * sub["scale"].astype(np.float64), "log_scale")


def test_deterministic_adjoint(case):
    """params deterministic: 64-bit fixed-point accumulation.  The gradient
    meets the oracle at the same bar, stays within 1e-5 (relative norm) of the
    float32-atomic accumulation, and is bit-identical when the same rays
    arrive in another order (the set's rays as an explicit list, permuted)."""
    from paper_2311_16043_gb300 import rt
    sub, dirs, w, want, _ = case
    dv = {k: _dev(v) for k, v in sub.items()}
    args = (dv["mean"], dv["scale"], dv["quat"], dv["opacity"])
    R = 1024 * 16
    wd = _dev(w.astype(np.float32))
    bvh_f = rt.rt_build_bvh(*args, rt.params(t_min=0.0))
    bvh_d = rt.rt_build_bvh(*args, rt.params(t_min=0.0, deterministic=True))
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
    T = rt.rt_trace_visibility(bvh_d, rs)
    g_d = rt.rt_trace_visibility_backward(bvh_d, rs, *args, T, wd)
    g_f = rt.rt_trace_visibility_backward(bvh_f, rs, *args, T, wd)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    for k in ("opacity", "mean", "scale", "quat"):
        _check(g_d[k].cpu().numpy(), want[k], k)
        a, b = g_d[k].double(), g_f[k].double()
        assert float((a - b).norm() / b.norm()) < 1e-5, k
    # the same rays as an explicit list, in order and permuted
    o, d, s = rt.rt_materialize_rays(bvh_d, rs, torch.arange(R, dtype=torch.int64, device="cuda"))
    perm = torch.from_numpy(np.random.default_rng(3).permutation(R)).cuda()
    grads = []
    for idx in (torch.arange(R, device="cuda"), perm):
        ex = rt.rayspec(rt.RT_RAYS_EXPLICIT, ray_o=o[idx].contiguous(), ray_d=d[idx].contiguous(),
                        ray_src=s[idx].contiguous())
        Te = rt.rt_trace_visibility(bvh_d, ex)
        grads.append(rt.rt_trace_visibility_backward(bvh_d, ex, *args, Te, wd[idx].contiguous()))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    for k in ("opacity", "mean", "scale", "quat"):
        assert torch.equal(grads[0][k], grads[1][k]), k
        assert float(grads[0][k].abs().max()) > 0.0


def test_deterministic_adjoint_range_error():
    """A gradient component beyond the fixed-point range (|sum| >= 2^31) is
    reported as RT_ERR_RANGE through the status word, not wrapped silently."""
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(256, 8)
    dv = {k: _dev(v) for k, v in sc.items()}
    args = (dv["mean"], dv["scale"], dv["quat"], dv["opacity"])
    bvh = rt.rt_build_bvh(*args, rt.params(t_min=0.0, deterministic=True))
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(scenes.fibonacci_sphere(16)))
    T = rt.rt_trace_visibility(bvh, rs)
    huge = torch.full((256 * 16,), 1e12, dtype=torch.float32, device="cuda")
    rt.rt_trace_visibility_backward(bvh, rs, *args, T, huge)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 9  # RT_ERR_RANGE
    rt.rt_status_clear()
    assert rt.rt_status_last() == 0
