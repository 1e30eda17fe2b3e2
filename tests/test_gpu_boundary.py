"""GPU checks of the boundary's host-facing contracts: the caller's
allocator (torch's caching allocator through rt_set_allocator), the device
check of Gaussian inputs (synchronous error from the build, status word from
the refit) and the one-call precompute from host buffers."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu


def _dev(sc):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in sc.items()}


def test_torch_caching_allocator():
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(20_000, 3)
    d = _dev(sc)
    dirs = torch.from_numpy(scenes.fibonacci_sphere(16)).cuda()
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])
    ref = rt.rt_trace_visibility_dirs(bvh, dirs)
    torch.cuda.synchronize()
    bvh.destroy()
    rt.use_torch_allocator(True)
    try:
        before = torch.cuda.memory_allocated()
        bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])
        torch.cuda.synchronize()
        held = torch.cuda.memory_allocated() - before
        assert held >= bvh.info()["device_bytes"]   # the tree lives in torch's pool
        got = rt.rt_trace_visibility_dirs(bvh, dirs)  # per-call scratch goes through it too
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        del got
        bvh.destroy()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        rt.use_torch_allocator(False)
    assert rt.rt_status_last() == 0


@pytest.mark.parametrize("field,index,value", [("mean", (5, 1), np.nan), ("scale", (7, 0), 0.0),
                                               ("scale", (7, 2), -1.0), ("quat", (3,), 0.0),
                                               ("opacity", (9,), 1.5), ("opacity", (9,), np.inf)])
def test_build_rejects_bad_inputs(field, index, value):
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(1000, 4)
    sc[field] = sc[field].copy()
    sc[field][index] = value
    d = _dev(sc)
    with pytest.raises(rt.RTError) as e:
        rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])
    assert e.value.code == 1  # RT_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0


def test_build_accepts_edge_values():
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(1000, 4)
    sc["opacity"][:3] = [0.0, 1.0, 1.0]
    d = _dev(sc)
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])
    T = rt.rt_trace_visibility_dirs(bvh, torch.from_numpy(scenes.fibonacci_sphere(8)).cuda())
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0 and bool(torch.all((T >= 0) & (T <= 1)))


def test_refit_reports_bad_inputs_through_the_status_word():
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(1000, 5)
    d = _dev(sc)
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])
    bad = d["scale"].clone()
    bad[11, 1] = float("nan")
    rt.rt_bvh_refit(bvh, d["mean"], bad, d["quat"], d["opacity"])
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 1
    rt.rt_status_clear()
    rt.rt_bvh_refit(bvh, d["mean"], d["scale"], d["quat"], d["opacity"])
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0


@pytest.mark.parametrize("pinned,K", [(True, 32), (False, 32), (True, 100), (True, 128), (False, 128)])
def test_precompute_from_host_buffers(pinned, K):
    """rt_visibility_dirs_host (copies in, build, trace, copy out) gives the
    device path's table bit for bit, from page-locked or pageable memory,
    with the library's pool and with the caller's allocator, for direction
    counts that are and are not multiples of the warp width."""
    from paper_2311_16043_gb300 import rt
    sc = scenes.object_scene(30_000, 4)
    dirs_np = scenes.fibonacci_sphere(K)
    d = _dev(sc)
    bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])
    ref = rt.rt_trace_visibility_dirs(bvh, torch.from_numpy(dirs_np).cuda()).cpu()
    bvh.destroy()
    host = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in sc.items()}
    hdirs = torch.from_numpy(dirs_np)
    if pinned:
        host = {k: v.pin_memory() for k, v in host.items()}
        hdirs = hdirs.pin_memory()
    for torch_alloc in (False, True):
        rt.use_torch_allocator(torch_alloc)
        try:
            hT = torch.full((30_000, K), -1.0, pin_memory=pinned)
            out = rt.rt_visibility_dirs_host(host["mean"], host["scale"], host["quat"], host["opacity"], hdirs, hT)
            torch.cuda.synchronize()
        finally:
            rt.use_torch_allocator(False)
        assert out is hT
        assert rt.rt_status_last() == 0
        assert torch.equal(hT, ref)


def test_precompute_from_host_buffers_edges():
    from paper_2311_16043_gb300 import rt
    sc = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in scenes.uniform_scene(200, 5).items()}
    dirs = torch.from_numpy(scenes.fibonacci_sphere(4))
    empty = {k: v[:0] for k, v in sc.items()}
    T = rt.rt_visibility_dirs_host(empty["mean"], empty["scale"], empty["quat"], empty["opacity"], dirs)
    assert T.shape == (0, 4)
    T = rt.rt_visibility_dirs_host(sc["mean"], sc["scale"], sc["quat"], sc["opacity"], dirs[:0])
    assert T.shape == (200, 0)
    with pytest.raises(TypeError):  # device tensors are not host buffers
        rt.rt_visibility_dirs_host(sc["mean"].cuda(), sc["scale"], sc["quat"], sc["opacity"], dirs)
    bad = sc["scale"].clone()
    bad[7, 1] = 0.0
    with pytest.raises(rt.RTError):  # the build's input check
        rt.rt_visibility_dirs_host(sc["mean"], bad, sc["quat"], sc["opacity"], dirs)
    torch.cuda.synchronize()
    rt.rt_status_clear()


def test_pool_keeps_blocks_until_trimmed():
    """The library's pool keeps freed blocks mapped across calls (no driver
    remapping per call); rt_memory_trim hands them back."""
    from paper_2311_16043_gb300 import rt
    sc = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in scenes.uniform_scene(200_000, 6).items()}
    dirs = torch.from_numpy(scenes.fibonacci_sphere(32))
    T = rt.rt_visibility_dirs_host(sc["mean"], sc["scale"], sc["quat"], sc["opacity"], dirs)
    torch.cuda.synchronize()
    held = torch.cuda.mem_get_info()[0]
    rt.rt_memory_trim(0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] > held  # the T scratch (25.6 MB) and tree came back
    T2 = rt.rt_visibility_dirs_host(sc["mean"], sc["scale"], sc["quat"], sc["opacity"], dirs)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0 and torch.equal(T, T2)
    with pytest.raises(rt.RTError):
        rt.rt_memory_trim(-1)
