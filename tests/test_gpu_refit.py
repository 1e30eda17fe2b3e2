"""GPU parity of the refit-only rebuild (topology kept, boxes recomputed):
refitting with the build's inputs reproduces the tree and T bit for bit; after
the Gaussians move, every internal box contains the exact FP64 supports of
the moved Gaussians under the build's topology (and is no more than the
stated margin larger), and traced visibility of every ray matches the oracle
on the moved scene for all traversals; refit inside a gradient loop with the
adjoint."""
import numpy as np
import pytest
import torch

import scenes
from conftest import check_flagged_bounds

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _build(sc, **kw):
    from paper_2311_16043_gb300 import rt
    d = {k: _dev(v) for k, v in sc.items()}
    return rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], rt.params(**kw))


def _refit(bvh, sc):
    from paper_2311_16043_gb300 import rt
    d = {k: _dev(v) for k, v in sc.items()}
    rt.rt_bvh_refit(bvh, d["mean"], d["scale"], d["quat"], d["opacity"])
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0


def _trace_all(bvh, dirs, kernels=(1, 2, 3, 4)):
    from paper_2311_16043_gb300 import rt
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
    out = {}
    for k in kernels:
        out[k] = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=k)).cpu().numpy()
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    return out


def _moved(sc, seed, amount=0.01):
    rng = np.random.default_rng(seed)
    n = sc["mean"].shape[0]
    q = sc["quat"].astype(np.float64) + rng.normal(0, 0.2, (n, 4))
    return {"mean": (sc["mean"] + rng.normal(0, amount, (n, 3))).astype(np.float32),
            "scale": (sc["scale"] * rng.uniform(0.8, 1.25, (n, 3))).astype(np.float32),
            "quat": (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32),
            "opacity": np.clip(sc["opacity"] * rng.uniform(0.7, 1.3, n), 0.0, 0.999).astype(np.float32)}


def test_refit_with_build_inputs_is_bit_identical():
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(20_000, 5)
    dirs = scenes.fibonacci_sphere(16)
    bvh = _build(sc)
    ex0 = {k: v.cpu().numpy() for k, v in rt.rt_bvh_export(bvh).items()}
    T0 = _trace_all(bvh, dirs)
    _refit(bvh, sc)
    _refit(bvh, sc)  # twice: the links are made once, the counters cleared each time
    ex1 = {k: v.cpu().numpy() for k, v in rt.rt_bvh_export(bvh).items()}
    T1 = _trace_all(bvh, dirs)
    for k in ex0:
        np.testing.assert_array_equal(ex0[k], ex1[k])
    for k in T0:
        np.testing.assert_array_equal(T0[k], T1[k])


def _exact_node_boxes(orc, mean_build, leaf, n):
    ref = orc.lbvh(mean_build)
    left = ref["left"].astype(np.int64) & 0xFFFFFFFF
    right = ref["right"].astype(np.int64) & 0xFFFFFFFF
    perm = (ref["keys"] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    box = np.zeros((n - 1, 6))
    order, stack = [], [0]
    while stack:
        i = stack.pop()
        order.append(i)
        for c in (left[i], right[i]):
            if not c & 0x80000000:
                stack.append(c)

    def child(c):
        return leaf[perm[c & 0x7FFFFFFF]] if c & 0x80000000 else box[c]
    for i in reversed(order):
        a, b = child(left[i]), child(right[i])
        box[i] = np.concatenate([np.minimum(a[:3], b[:3]), np.maximum(a[3:], b[3:])])
    return [np.array([child(c) for c in refs]) for refs in (left, right)]


def test_refit_boxes_contain_moved_supports(orc):
    from paper_2311_16043_gb300 import rt
    n = 4096
    sc = scenes.uniform_scene(n, 1)
    mv = _moved(sc, 3)
    bvh = _build(sc)
    _refit(bvh, mv)
    g = rt.rt_bvh_export(bvh)["boxes"].cpu().numpy().astype(np.float64)
    exact = _exact_node_boxes(orc, sc["mean"], orc.leaf_boxes(mv), n)
    for side in (0, 1):
        b = g[:, 6 * side:6 * side + 6]
        e = exact[side]
        ext = e[:, 3:] - e[:, :3]
        assert np.all(b[:, :3] <= e[:, :3]) and np.all(b[:, 3:] >= e[:, 3:])
        slack = np.maximum(e[:, :3] - b[:, :3], b[:, 3:] - e[:, 3:])
        assert np.all(slack <= 2e-4 * ext + 1e-5)


@pytest.mark.parametrize("amount", [0.01, 1.0])
def test_refit_trace_matches_oracle_on_moved_scene(orc, amount):
    """Small motion (the optimisation case) and motion of the scene's size
    (stale Morton order: slower traversal, same result); every ray, every
    traversal, against the oracle on the moved scene."""
    n = 4096
    sc = scenes.uniform_scene(n, 1)
    mv = _moved(sc, 4, amount)
    dirs = scenes.fibonacci_sphere(32)
    bvh = _build(sc)
    _refit(bvh, mv)
    T = _trace_all(bvh, dirs)
    o, d, s = orc.dir_rays(mv["mean"], dirs, np.arange(n * 32))
    ref = orc.BvhTracer(mv).trace(o, d, s)
    ok = ref["flags"] == 0
    assert ok.mean() > 0.99
    for k, t in T.items():
        err = np.abs(t.astype(np.float64) - ref["T"])
        assert err[ok].max() <= TOL, (k, err[ok].max())
        check_flagged_bounds(t, ref, TOL)


def test_refit_tiny_scenes():
    from paper_2311_16043_gb300 import rt
    for n in (0, 1, 2, 5):
        sc = scenes.uniform_scene(n, 9)
        bvh = _build(sc)
        _refit(bvh, _moved(sc, 1) if n else sc)
    bvh = _build(scenes.uniform_scene(10, 9))
    with pytest.raises(ValueError):
        sc = scenes.uniform_scene(11, 9)
        d = {k: _dev(v) for k, v in sc.items()}
        rt.rt_bvh_refit(bvh, d["mean"], d["scale"], d["quat"], d["opacity"])


def test_refit_in_a_gradient_loop(orc):
    """Outer loop of differentiable visibility: signed ascent steps on
    L = sum w T over the means and opacities with the hand-written adjoint,
    refitting the tree each step; the GPU gradient matches the oracle's at
    every step and L rises."""
    from paper_2311_16043_gb300 import rt
    n, K = 512, 8
    sc = scenes.uniform_scene(n, 4, lo=-0.3, hi=0.3)
    dirs = scenes.fibonacci_sphere(K)
    w = scenes.loss_weights(n * K, 41)
    prm = rt.params(t_min=0.0)
    d = {k: _dev(v) for k, v in sc.items()}
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], prm)
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
    ids = np.arange(n * K)
    losses = []
    cur = {k: v.copy() for k, v in sc.items()}
    for step in range(4):
        d = {k: _dev(v) for k, v in cur.items()}
        if step:
            rt.rt_bvh_refit(bvh, d["mean"], d["scale"], d["quat"], d["opacity"])
        T = rt.rt_trace_visibility(bvh, rs)
        torch.cuda.synchronize()
        assert rt.rt_status_last() == 0
        o, dd, s = orc.dir_rays(cur["mean"], dirs, ids)
        ww = w.astype(np.float64)
        ww[orc.trace(cur, o, dd, s, t_min=0.0)["flags"] != 0] = 0.0  # threshold rays: excluded
        ref = orc.trace_grad(cur, o, dd, s, ww, t_min=0.0, with_origin=True)
        np.add.at(ref["mean"], s, ref["ray_o"])  # origins ride on the source means
        g = rt.rt_trace_visibility_backward(bvh, rs, d["mean"], d["scale"], d["quat"], d["opacity"], T,
                                            _dev(ww.astype(np.float32)))
        torch.cuda.synchronize()
        for name in ("mean", "opacity"):
            got = g[name].cpu().numpy().astype(np.float64)
            rel = np.linalg.norm(got - ref[name]) / max(np.linalg.norm(ref[name]), 1e-30)
            assert rel < 1e-3, (step, name, rel)
        losses.append(float((T.double() * _dev(w).double()).sum()))
        # ascend L (more visibility): signed steps on opacities and means
        cur["opacity"] = np.clip(cur["opacity"] + 0.05 * np.sign(ref["opacity"]), 0.01, 0.99).astype(np.float32)
        cur["mean"] = (cur["mean"] + 0.002 * np.sign(ref["mean"])).astype(np.float32)
    assert losses[-1] > losses[0]
