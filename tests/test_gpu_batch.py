"""Batched multi-scene launch and the autotuner: scenes of uneven size, each
with Fibonacci-direction rays and environment-map shadow rays, traced in one
persistent graph-captured launch, must give exactly the per-scene results
(the traversal visits each ray's Gaussians in the same order either way), and
the per-scene results match the oracle on sampled rays."""
import numpy as np
import pytest
import torch

import scenes
from conftest import check_flagged_bounds

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("autotune", [True, False])
def test_batch_equals_single_launches(orc, autotune):
    """Without tuning the env-map jobs run with lane refill (the batch's
    per-ray slot queue) and the direction sets, all over fewer than 2^19
    Gaussians here, with the per-ray 4-wide walk, as the single-scene AUTO."""
    from paper_2311_16043_gb300 import rt
    sizes = [700, 9000, 31, 2500, 20000]
    env = scenes.envmap(399)
    E = rt.rt_envmap_create(env["radiance"], env["solid_angle"], env["corners"])
    dirs = _dev(scenes.fibonacci_sphere(16))
    jobs, refs, scs = [], [], []
    for s, n in enumerate(sizes):
        sc = scenes.batch_scenes([n], seed_base=300 + 10 * s)[0]
        dv = {k: _dev(v) for k, v in sc.items()}
        bvh = rt.rt_build_bvh(dv["mean"], dv["scale"], dv["quat"], dv["opacity"])
        for rs in (rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs),
                   rt.rayspec(rt.RT_RAYS_ENV, env=E, n_samples=24, seed=399 + s)):
            R = rt.rt_rayspec_count(bvh, rs)
            T = torch.full((R,), -1.0, device="cuda")
            jobs.append((bvh, rs, T))
        scs.append((sc, bvh))
    batch = rt.rt_batch_create(jobs, autotune=autotune)
    info = batch.info()
    if not autotune:
        assert info["kernel"] == [rt.RT_KERNEL_RAY_WIDE, rt.RT_KERNEL_RAY_REFILL] * len(sizes)
    # single launches with each job's chosen strategy give the same T bit for bit
    for (bvh, rs, T), kernel in zip(jobs, info["kernel"]):
        refs.append(rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=kernel)))
    for rep in range(2):  # the captured graph replays
        for _, _, T in jobs:
            T.fill_(-1.0)
        batch.run()
        torch.cuda.synchronize()
        assert rt.rt_status_last() == 0
        for (bvh, rs, T), ref in zip(jobs, refs):
            assert torch.equal(T, ref)
    assert info["n_rays"] == sum(T.numel() for _, _, T in jobs)
    assert set(info["kernel"]) <= {1, 2, 3, 4, 5}
    # oracle on sampled rays of the largest scene
    sc, bvh = scs[4]
    sel = scenes.sample_ray_ids(20000 * 16, 2000, 5)
    o, d, s = orc.dir_rays(sc["mean"], scenes.fibonacci_sphere(16), sel)
    ref = orc.trace(sc, o, d, s)
    got = jobs[8][2].cpu().numpy().astype(np.float64)[sel]
    ok = ref["flags"] == 0
    assert np.abs(got - ref["T"])[ok].max() <= 1e-5
    check_flagged_bounds(got, ref)
    batch.destroy()
    E.destroy()


@pytest.mark.parametrize("n,kind", [(50_000, "dirs"), (100, "dirs"), (20_000, "env"), (200_000, "env")])
def test_autotune_picks_a_valid_shape(n, kind):
    """One block of all tiles (small scenes) or four blocks over the Morton
    range (large ones); the chosen shape gives the per-ray result."""
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(n, 3)
    dv = {k: _dev(v) for k, v in sc.items()}
    bvh = rt.rt_build_bvh(dv["mean"], dv["scale"], dv["quat"], dv["opacity"])
    E = None
    if kind == "dirs":
        rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(scenes.fibonacci_sphere(32)))
    else:
        env = scenes.envmap(399)
        E = rt.rt_envmap_create(env["radiance"], env["solid_angle"], env["corners"])
        rs = rt.rayspec(rt.RT_RAYS_ENV, env=E, n_samples=64, seed=3)
    T = torch.empty(rt.rt_rayspec_count(bvh, rs), device="cuda")
    o = rt.rt_trace_autotune(bvh, rs, T)
    assert o.kernel in (1, 2, 3, 4, 5) and o.order_block in (1, 16, 128, 1024)
    a = rt.rt_trace_visibility(bvh, rs, opts=o)
    b = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=1))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    assert (a - b).abs().max().item() <= 1e-6
    if E is not None:
        E.destroy()
