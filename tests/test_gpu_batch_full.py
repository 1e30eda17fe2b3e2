"""The batched multi-scene workloads at full size, in the launch
configuration the benchmark times: 16 scenes (uniform, or object-scale) of
log-uniform sizes in [50k, 2M] (about 8M Gaussians), 128 Fibonacci directions
and 512 environment-map shadow rays per Gaussian (about 5.12G rays),
autotuned and replayed as one captured graph.  Every job's outputs lie in [0, 1] and are all written; sampled rays of
every job match the CPU BVH oracle (itself pinned against brute force) within
the tracer's tolerance."""
import numpy as np
import pytest
import torch

import scenes
from conftest import check_flagged_bounds

pytestmark = pytest.mark.gpu
TOL = 1e-5
DIRS, ENV_SAMPLES, SAMPLES_PER_JOB = 128, 512, 96


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("kind", ["uniform", "objects"])
def test_batch_workload_sampled(orc, kind):
    from paper_2311_16043_gb300 import rt
    gen = scenes.batch_scenes if kind == "uniform" else scenes.batch_object_scenes
    scs = gen(scenes.batch_scene_sizes(16, 8_000_000, 300), seed_base=300)
    env = scenes.envmap(399)
    E = rt.rt_envmap_create(env["radiance"], env["solid_angle"], env["corners"])
    dirs_np = scenes.fibonacci_sphere(DIRS)
    dirs = _dev(dirs_np)
    jobs, bvhs = [], []
    for s, sc in enumerate(scs):
        d = {k: _dev(v) for k, v in sc.items()}
        bvh = rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], rt.params())
        bvhs.append(bvh)
        for rs in (rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs),
                   rt.rayspec(rt.RT_RAYS_ENV, env=E, n_samples=ENV_SAMPLES, seed=399 + s)):
            jobs.append((bvh, rs, torch.full((rt.rt_rayspec_count(bvh, rs),), -1.0, device="cuda")))
    batch = rt.rt_batch_create(jobs, autotune=True)
    info = batch.info()
    assert info["n_rays"] == sum(T.numel() for _, _, T in jobs)
    assert info["n_rays"] == sum(sc["mean"].shape[0] for sc in scs) * (DIRS + ENV_SAMPLES)
    batch.run()
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    for _, _, T in jobs:
        assert float(T.min()) >= 0.0 and float(T.max()) <= 1.0  # every output written, in range
    checked = excluded = 0
    worst = 0.0
    for s, sc in enumerate(scs):
        tracer = orc.BvhTracer(sc)
        for j, rays in enumerate(("dirs", "env")):
            T = jobs[2 * s + j][2]
            sel = scenes.sample_ray_ids(T.numel(), SAMPLES_PER_JOB, 17 + 2 * s + j)
            if rays == "dirs":
                o, d, src = orc.dir_rays(sc["mean"], dirs_np, sel)
            else:
                o, d, src = orc.env_rays(sc["mean"], env, 399 + s, ENV_SAMPLES, sel)
            ref = tracer.trace(o, d, src)
            got = T[_dev(sel)].cpu().numpy().astype(np.float64)
            ok = ref["flags"] == 0
            err = np.abs(got - ref["T"])
            bad = np.nonzero(ok & (err > TOL))[0]
            assert bad.size == 0, (s, rays, sel[bad[:5]], got[bad[:5]], ref["T"][bad[:5]])
            check_flagged_bounds(got, ref, TOL)
            checked += int(ok.sum())
            excluded += int((~ok).sum())
            if ok.any():
                worst = max(worst, float(err[ok].max()))
        tracer.close()
    # flattened object-scale Gaussians put more rays within the m^2 rounding
    # band of some candidate's 3-sigma support; those are held to the
    # oracle's bounds over that candidate, and counted
    assert excluded <= (0.02 if kind == "uniform" else 0.08) * (checked + excluded), excluded
    print(f"{kind} batch workload: {checked} sampled rays within {worst:.2e}, {excluded} in a rounding band")
    batch.destroy()
    for bvh in bvhs:
        bvh.destroy()
    E.destroy()
