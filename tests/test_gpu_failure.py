"""Failure handling on the GPU without a fault: a bounded wait that nothing
completes reports RT_ERR_TIMEOUT through the status word and the context stays
usable; invalid ray ids are reported the same way."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_2311_16043_gb300 import rt
    rt.rt_status_clear()
    L = rt.lib()
    assert L.rt_selftest_wait_timeout(2_000_000, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 6  # RT_ERR_TIMEOUT
    rt.rt_status_clear()
    assert rt.rt_status_last() == 0
    # the context still works
    x = torch.arange(10, device="cuda").sum().item()
    assert x == 45


def test_invalid_ray_ids_are_reported():
    from paper_2311_16043_gb300 import rt
    rt.rt_status_clear()
    sc = scenes.uniform_scene(100, 1)
    d = {k: torch.from_numpy(v).cuda() for k, v in sc.items()}
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])
    dirs = torch.from_numpy(scenes.fibonacci_sphere(4)).cuda()
    ids = torch.tensor([0, 5, 400, -3, 399], dtype=torch.int64, device="cuda")  # 400 and -3 are outside
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs, ray_ids=ids)
    T = rt.rt_trace_visibility(bvh, rs)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 1  # RT_ERR_INVALID_ARG
    T = T.cpu().numpy()
    assert np.isnan(T[2]) and np.isnan(T[3]) and np.all(np.isfinite(T[[0, 1, 4]]))
    rt.rt_status_clear()


def test_surrogate_waits_give_up_together_and_context_survives():
    """The surrogate kernels' own bounded waits (on their MMA commits) made
    to give up at once (a 1-cycle bound): inference and training report
    RT_ERR_TIMEOUT, leave only after their MMAs finished, and the next calls
    with the default bound give the same results as before."""
    from paper_2311_16043_gb300 import rt
    rng = np.random.default_rng(3)
    m = 4000  # several tiles and warpgroups, the last tile ragged
    pos = torch.from_numpy(rng.uniform(-1, 1, (m, 3)).astype(np.float32)).cuda()
    d = rng.standard_normal((m, 3))
    d = torch.from_numpy((d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.uniform(0, 1, m).astype(np.float32)).cuda()
    s = rt.rt_surrogate_create(rt.mlp_cfg(batch=1024), seed=4)
    p0 = rt.rt_surrogate_forward(s, pos, d)
    loss0, g0 = rt.rt_surrogate_loss_grad(s, pos, d, y)
    torch.cuda.synchronize()
    rt.rt_status_clear()
    try:
        rt.rt_set_wait_limit(1)
        rt.rt_surrogate_forward(s, pos, d)
        torch.cuda.synchronize()
        assert rt.rt_status_last() == 6  # RT_ERR_TIMEOUT
        rt.rt_status_clear()
        rt.rt_surrogate_loss_grad(s, pos, d, y)
        torch.cuda.synchronize()
        assert rt.rt_status_last() == 6
    finally:
        rt.rt_set_wait_limit(0)
        rt.rt_status_clear()
    p1 = rt.rt_surrogate_forward(s, pos, d)
    loss1, g1 = rt.rt_surrogate_loss_grad(s, pos, d, y)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    assert torch.equal(p0, p1)
    assert torch.equal(loss1, loss0) and torch.equal(g1, g0)  # fixed-order sums
    with pytest.raises(rt.RTError):
        rt.rt_set_wait_limit(-1)
