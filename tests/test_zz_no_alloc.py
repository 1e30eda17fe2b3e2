"""The allocation-free surrogate inference (for callers that may not let the
library allocate device memory during a call) against the allocating entry
point, through the C ABI, on two calls in a row.  Kept in its own file, named
to be collected last."""
import ctypes
import math

import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

NP = 60033


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _params(seed):
    # random weights spread the predictions over (0, 1), so many rays fall back
    rng = np.random.default_rng(seed)
    P = np.zeros(NP, np.float32)
    P[:10240] = rng.uniform(-1, 1, 10240) * math.sqrt(6.0 / 80)
    off = 10240 + 128
    for _ in range(3):
        P[off:off + 16384] = rng.uniform(-1, 1, 16384) * math.sqrt(6.0 / 128)
        off += 16384 + 128
    P[59904:60032] = rng.uniform(-1, 1, 128) * 0.3
    return P


def test_noalloc_matches_allocating_infer():
    from paper_2311_16043_gb300 import rt
    L = rt.lib()
    sc = scenes.object_scene(100_000, 2)
    dv = {k: _dev(v) for k, v in sc.items()}
    bvh = rt.rt_build_bvh(dv["mean"], dv["scale"], dv["quat"], dv["opacity"])
    s = rt.rt_surrogate_create(rt.mlp_cfg(batch=4096), seed=1)
    rt.rt_surrogate_set_params(s, _dev(_params(7)))
    info = bvh.info()
    rt.rt_surrogate_set_bounds(s, info["lo"], info["hi"])
    dirs = _dev(scenes.fibonacci_sphere(16))
    ids = _dev(scenes.sample_ray_ids(100_000 * 16, 300_000, 5))
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs, ray_ids=ids)
    m = ids.numel()
    band = 0.3
    ref = torch.empty(m, dtype=torch.float32, device="cuda")
    nref = torch.zeros(1, dtype=torch.int64, device="cuda")
    rt.rt_surrogate_infer(s, bvh, rs, band=band, T_out=ref, n_fallback=nref)
    torch.cuda.synchronize()
    assert 0 < int(nref.item()) < m  # both paths of the fallback are exercised
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full((m,), -1.0, dtype=torch.float32, device="cuda")
        nfb = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        code = L.rt_surrogate_infer_noalloc(s.handle, bvh.handle, ctypes.byref(rs), band, out.data_ptr(),
                                            nfb.data_ptr(), stream)
        assert code == 0, call
        torch.cuda.synchronize()
        assert rt.rt_status_last() == 0
        assert int(nfb.item()) == int(nref.item()), call
        assert torch.allclose(out, ref, rtol=0, atol=1e-6), call
        assert torch.equal(out, ref), call
    # more rays than the fixed scratch holds: rejected before any work
    big = _dev(np.arange(2 ** 20 + 1, dtype=np.int64))
    rs_big = rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs, ray_ids=big)
    out = torch.empty(2 ** 20 + 1, dtype=torch.float32, device="cuda")
    assert L.rt_surrogate_infer_noalloc(s.handle, bvh.handle, ctypes.byref(rs_big), band, out.data_ptr(),
                                        None, stream) == 1
