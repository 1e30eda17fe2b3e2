"""GPU parity of the visibility trace against the FP64 brute-force oracle.

Bar: |T_gpu - T_oracle| <= 1e-5 on every ray the oracle does not flag.  A
flagged ray has a candidate inside a rounding band of a threshold (m^2 = K^2,
alpha = 1/255, t* = 0) or T_exact near T = T_min, where a float32 evaluation
may decide either way: its T must lie within 1e-5 of the oracle's bounds
[T_lo, T_hi] over taking or leaving each such candidate (or be 0 where the
bounds reach below T_min).  Flagged rays are counted and must stay rare.  The per-ray and packet traversals of the binary tree visit each
ray's accepted Gaussians in the same order, so they agree bit for bit; the
4-wide traversal visits them in another order (same factors, another product
rounding).
"""
import numpy as np
import pytest
import torch

import scenes
from conftest import check_flagged_bounds

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def build(sc, **kw):
    from paper_2311_16043_gb300 import rt
    return rt.rt_build_bvh(_dev(sc["mean"]), _dev(sc["scale"]), _dev(sc["quat"]), _dev(sc["opacity"]),
                           rt.params(**kw))


def trace_dirs(bvh, dirs, kernel=0, **opt):
    from paper_2311_16043_gb300 import rt
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
    T = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=kernel, **opt))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    return T.cpu().numpy().astype(np.float64)


def compare(T_gpu, ref, max_excluded=0.002, t_min=1e-4):
    ok = ref["flags"] == 0
    err = np.abs(T_gpu - ref["T"])
    bad = np.nonzero(ok & (err > TOL))[0]
    assert bad.size == 0, (bad[:10], err[bad[:10]], T_gpu[bad[:10]], ref["T"][bad[:10]])
    check_flagged_bounds(T_gpu, ref, TOL, t_min)  # flagged rays: within the oracle's bounds
    assert (~ok).mean() <= max_excluded, (~ok).sum()
    return err[ok].max(), int((~ok).sum())


@pytest.fixture(scope="module")
def small(orc):
    """Uniform scene: 4,096 Gaussians x 32 Fibonacci directions (131,072 rays),
    every ray checked."""
    sc = scenes.uniform_scene(4096, 1)
    dirs = scenes.fibonacci_sphere(32)
    ids = np.arange(4096 * 32, dtype=np.int64)
    o, d, s = orc.dir_rays(sc["mean"], dirs, ids)
    ref = orc.trace(sc, o, d, s)
    return sc, dirs, ref


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6])
def test_small_scene_all_rays(small, kernel):
    sc, dirs, ref = small
    bvh = build(sc)
    T = trace_dirs(bvh, dirs, kernel=kernel).reshape(-1)
    maxerr, excl = compare(T, ref)
    assert maxerr < TOL
    assert (ref["T"] < 1).mean() > 0.3 and (ref["T"] == 0).any() or (ref["hits"] > 3).any()


def test_kernels_agree(small):
    sc, dirs, _ = small
    bvh = build(sc)
    a = trace_dirs(bvh, dirs, kernel=1)
    b = trace_dirs(bvh, dirs, kernel=2)
    c = trace_dirs(bvh, dirs, kernel=3)
    e = trace_dirs(bvh, dirs, kernel=4)
    f = trace_dirs(bvh, dirs, kernel=5)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_allclose(c, a, atol=1e-6, rtol=0)
    np.testing.assert_allclose(e, a, atol=1e-6, rtol=0)
    # lane refill runs each ray's visits of the per-ray 4-wide loop in order
    np.testing.assert_allclose(f, e, atol=1e-6, rtol=0)
    # one warp per ray: the same accepted set, another product order
    w = trace_dirs(bvh, dirs, kernel=6)
    np.testing.assert_allclose(w, e, atol=1e-6, rtol=0)


def test_wide_tree_counts(small):
    """The 4-wide traversal tests the same leaves as the binary one (every
    Gaussian whose box the ray enters) and accepts the same hits."""
    from paper_2311_16043_gb300 import rt
    sc, dirs, _ = small
    bvh = build(sc)
    cnts = []
    for kernel in (1, 3):
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
        rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=kernel, counters=cnt))
        torch.cuda.synchronize()
        cnts.append(cnt.cpu().numpy())
    assert cnts[0][3] == cnts[1][3] == 4096 * 32
    # early termination can stop the two orders at different points: compare
    # with T_min = 0 below; here only the ray count and a sane ratio
    assert 0.5 < cnts[1][0] / cnts[0][0] < 3.0


def test_wide_tree_same_hits_without_early_exit(small):
    from paper_2311_16043_gb300 import rt
    sc, dirs, _ = small
    bvh = build(sc, t_min=0.0)
    R = 4096 * 32
    out = []
    for kernel in (1, 3, 4):
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        hc = torch.zeros(R, dtype=torch.int32, device="cuda")
        ids = torch.zeros((R, 4), dtype=torch.int32, device="cuda")
        rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
        rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=kernel, counters=cnt, hit_ids=ids, hit_count=hc))
        torch.cuda.synchronize()
        out.append((cnt.cpu().numpy(), hc.cpu().numpy()))
    for k in (1, 2):
        np.testing.assert_array_equal(out[0][1], out[k][1])  # same accepted hits per ray
        assert out[0][0][1] == out[k][0][1]  # same Gaussian tests (the leaves whose box a ray enters)
        assert out[0][0][2] == out[k][0][2]


@pytest.mark.parametrize("order_block", [1, 7, 1000])
def test_work_order_does_not_change_results(small, order_block):
    sc, dirs, _ = small
    bvh = build(sc)
    a = trace_dirs(bvh, dirs, kernel=2)
    b = trace_dirs(bvh, dirs, kernel=2, order_block=order_block)
    np.testing.assert_array_equal(a, b)


def test_box_mode_1_same_results(small):
    sc, dirs, _ = small
    a = trace_dirs(build(sc), dirs, kernel=1)
    b = trace_dirs(build(sc, box_mode=1), dirs, kernel=1)
    np.testing.assert_array_equal(a, b)


def test_no_early_termination(orc, small):
    sc, dirs, _ = small
    ids = np.arange(0, 4096 * 32, 7, dtype=np.int64)
    o, d, s = orc.dir_rays(sc["mean"], dirs, ids)
    ref = orc.trace(sc, o, d, s, t_min=0.0)
    T = trace_dirs(build(sc, t_min=0.0), dirs).reshape(-1)[ids]
    compare(T, ref)
    assert (ref["T"] < 1e-4).any()  # exercises products below the snap threshold


def test_explicit_rays_and_counters(orc):
    """Rays from the input generator (origins in and around the cube, random
    directions, some with a source to skip); per-ray work counts must be the
    same for both traversal strategies."""
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(4096, 1)
    rng = np.random.default_rng(17)
    R = 20000
    ro = rng.uniform(-1.5, 1.5, (R, 3)).astype(np.float32)
    rd = rng.standard_normal((R, 3))
    rd /= np.linalg.norm(rd, axis=1, keepdims=True)
    rd = rd.astype(np.float32)
    rd[:50] = np.array([1, 0, 0], np.float32)  # axis-aligned directions
    rd[50:100] = np.array([0, 0, -1], np.float32)
    src = np.where(rng.random(R) < 0.5, rng.integers(0, 4096, R), -1).astype(np.int32)
    ref = orc.trace(sc, ro, rd, src)
    bvh = build(sc)
    outs, cnts = [], []
    for kernel in (1, 2, 3, 4, 6):
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        rs = rt.rayspec(rt.RT_RAYS_EXPLICIT, ray_o=_dev(ro), ray_d=_dev(rd), ray_src=_dev(src))
        T = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=kernel, counters=cnt))
        torch.cuda.synchronize()
        outs.append(T.cpu().numpy().astype(np.float64))
        cnts.append(cnt.cpu().numpy())
    compare(outs[0], ref)
    compare(outs[2], ref)
    compare(outs[3], ref)
    compare(outs[4], ref)  # one warp per ray
    assert cnts[4][3] == R
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(cnts[0], cnts[1])
    assert cnts[0][3] == R
    assert cnts[0][2] == int(ref["hits"][ref["T"] > 0].sum()) or cnts[0][2] <= int(ref["hits"].sum())


def test_hit_log_matches_oracle(orc, small):
    from paper_2311_16043_gb300 import rt
    sc, dirs, _ = small
    bvh = build(sc, t_min=0.0)
    R = 4096 * 32
    cap = 16
    ids = torch.full((R, cap), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(R, dtype=torch.int32, device="cuda")
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
    rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(hit_ids=ids, hit_count=cnt))
    torch.cuda.synchronize()
    ids, cnt = ids.cpu().numpy(), cnt.cpu().numpy()
    sel = np.arange(0, R, 13, dtype=np.int64)
    o, d, s = orc.dir_rays(sc["mean"], dirs, sel)
    ref = orc.trace(sc, o, d, s, t_min=0.0)
    rid, rcnt = orc.trace_hits(sc, o, d, s, cap=64)
    ok = ref["flags"] == 0
    np.testing.assert_array_equal(cnt[sel][ok], rcnt[ok])
    assert (cnt > cap).any()  # some rays overflow the log and say so
    for j in np.nonzero(ok & (rcnt <= cap))[0][:2000]:
        r = sel[j]
        assert set(ids[r, :cnt[r]]) == set(rid[j, :rcnt[j]])
    # a flagged ray: each borderline candidate may go either way, so the
    # count and the listed set differ from the exact ones by at most that many
    nb = ref["n_border"]
    assert np.all(np.abs(cnt[sel] - rcnt) <= nb)
    for j in np.nonzero(~ok & (rcnt <= cap) & (cnt[sel] <= cap))[0][:2000]:
        r = sel[j]
        assert len(set(ids[r, :cnt[r]]) ^ set(rid[j, :rcnt[j]])) <= nb[j]


def test_id_subset_matches_full_trace(small):
    from paper_2311_16043_gb300 import rt
    sc, dirs, _ = small
    bvh = build(sc)
    full = trace_dirs(bvh, dirs, kernel=6).reshape(-1)  # id lists up to 2^22 rays: one warp per ray
    sel = scenes.sample_ray_ids(4096 * 32, 5000, 3)
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs), ray_ids=_dev(sel))
    T = rt.rt_trace_visibility(bvh, rs)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(T.cpu().numpy().astype(np.float64), full[sel])


def test_warp_per_ray_id_subset(small):
    """One warp per ray on an id list, including an invalid id (NaN output,
    status set): the same values as the full trace with that kernel."""
    from paper_2311_16043_gb300 import rt
    sc, dirs, _ = small
    bvh = build(sc)
    full = trace_dirs(bvh, dirs, kernel=6).reshape(-1)
    sel = scenes.sample_ray_ids(4096 * 32, 777, 9)
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs), ray_ids=_dev(sel))
    T = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=6))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    np.testing.assert_array_equal(T.cpu().numpy().astype(np.float64), full[sel])
    bad = sel.copy()
    bad[5] = 4096 * 32
    T = rt.rt_trace_visibility(bvh, rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs), ray_ids=_dev(bad)),
                               opts=rt.trace_opts(kernel=6))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 1 and np.isnan(T[5].item())
    rt.rt_status_clear()


@pytest.mark.parametrize("kind", ["dirs", "hemi"])
def test_long_id_list_sorted_trace(orc, kind):
    """AUTO on an id list longer than 2^22 rays traces it sorted by
    (direction, the tree's order) and writes each T back to its place: the
    same values, bit for bit, as the per-ray traversal of the list in the
    caller's order; an invalid id among them gives NaN at its place and sets
    the status.  300k object scene x 32 directions, 5M of its 9.6M rays in
    random order; 256 of them against the oracle's CPU BVH tracer."""
    from paper_2311_16043_gb300 import rt
    sc = scenes.object_scene(300_000, 2)
    bvh = build(sc)
    K = 32
    if kind == "dirs":
        dirs = scenes.fibonacci_sphere(K)
        rs_kw = dict(dirs=_dev(dirs))
        rkind = rt.RT_RAYS_DIRS
    else:
        nrm = scenes.shortest_axis_normals(sc["scale"], sc["quat"])
        rs_kw = dict(dirs=_dev(scenes.fibonacci_hemisphere(K)), normals=_dev(nrm))
        rkind = rt.RT_RAYS_HEMI
    rng = np.random.default_rng(21)
    sel = rng.permutation(300_000 * K)[:5_000_000].astype(np.int64)
    rs = rt.rayspec(rkind, ray_ids=_dev(sel), **rs_kw)
    T_auto = rt.rt_trace_visibility(bvh, rs)
    T_ray = rt.rt_trace_visibility(bvh, rs, opts=rt.trace_opts(kernel=rt.RT_KERNEL_RAY_WIDE))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    assert torch.equal(T_auto, T_ray)
    if kind == "dirs":
        pick = rng.choice(sel.size, 256, replace=False)
        ref = orc.BvhTracer(sc).trace_dirs(dirs, ids=sel[pick])
        compare(T_auto.cpu().numpy()[pick].astype(np.float64), ref, max_excluded=0.05)
    bad = sel.copy()
    bad[123_456] = 300_000 * K
    T_bad = rt.rt_trace_visibility(bvh, rt.rayspec(rkind, ray_ids=_dev(bad), **rs_kw))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 1
    rt.rt_status_clear()
    Tb = T_bad.cpu().numpy()
    assert np.isnan(Tb[123_456]) and np.isfinite(np.delete(Tb, 123_456)).all()
    assert np.array_equal(np.delete(Tb, 123_456), np.delete(T_ray.cpu().numpy(), 123_456))


def test_materialized_rays_bit_exact(orc, small):
    from paper_2311_16043_gb300 import rt
    sc, dirs, _ = small
    bvh = build(sc)
    sel = scenes.sample_ray_ids(4096 * 32, 3000, 4)
    rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
    o, d, s = rt.rt_materialize_rays(bvh, rs, _dev(sel))
    torch.cuda.synchronize()
    ro, rd, rsrc = orc.dir_rays(sc["mean"], dirs, sel)
    np.testing.assert_array_equal(o.cpu().numpy(), ro)
    np.testing.assert_array_equal(d.cpu().numpy(), rd)
    np.testing.assert_array_equal(s.cpu().numpy(), rsrc)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 33])
def test_tiny_scenes(orc, n):
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(max(n, 1), 5, log_scale_mean=np.log(0.3))
    sc = {k: v[:n] for k, v in sc.items()}
    dirs = scenes.fibonacci_sphere(16)
    bvh = build(sc)
    if n == 0:
        rs = rt.rayspec(rt.RT_RAYS_DIRS, dirs=_dev(dirs))
        assert rt.rt_rayspec_count(bvh, rs) == 0
        rng = np.random.default_rng(0)
        ro = _dev(rng.uniform(-1, 1, (10, 3)).astype(np.float32))
        rd = _dev(np.tile(np.array([[0, 0, 1]], np.float32), (10, 1)))
        T = rt.rt_trace_visibility(bvh, rt.rayspec(rt.RT_RAYS_EXPLICIT, ray_o=ro, ray_d=rd))
        torch.cuda.synchronize()
        assert torch.all(T == 1)
        return
    ids = np.arange(n * 16, dtype=np.int64)
    o, d, s = orc.dir_rays(sc["mean"], dirs, ids)
    ref = orc.trace(sc, o, d, s)
    for kernel in (1, 2, 3, 4, 5, 6):
        compare(trace_dirs(bvh, dirs, kernel=kernel).reshape(-1), ref, max_excluded=1.0)


def test_object_scene_300k_sample(orc):
    """Object-scale scene, 300k flattened Gaussians x 128 directions
    (38.4M rays); 4,096 sampled rays checked against brute force."""
    sc = scenes.object_scene(300_000, 2)
    dirs = scenes.fibonacci_sphere(128)
    bvh = build(sc)
    sel = scenes.sample_ray_ids(300_000 * 128, 4096, 7)
    o, d, s = orc.dir_rays(sc["mean"], dirs, sel)
    ref = orc.trace(sc, o, d, s)
    for kernel in (1, 3, 4, 5):
        T = trace_dirs(bvh, dirs, kernel=kernel).reshape(-1)
        compare(T[sel], ref, max_excluded=0.01)
        assert np.all((T >= 0) & (T <= 1))


def test_object_scene_300k_every_ray(orc):
    """Object-scale scene, 300k Gaussians x 128 directions: every one of the
    38.4M rays, traced in the default launch configuration, against the
    oracle's CPU BVH tracer (the brute-force T through the LBVH twin)."""
    sc = scenes.object_scene(300_000, 2)
    dirs = scenes.fibonacci_sphere(128)
    T = trace_dirs(build(sc), dirs).reshape(-1)
    B = orc.BvhTracer(sc)
    ref = B.trace_dirs(dirs)
    B.close()
    maxerr, excluded = compare(T, ref, max_excluded=0.01)
    print(f"300k scene, every ray: max |dT| {maxerr:.2e} over {T.size - excluded} rays, "
          f"{excluded} in a rounding band, {(ref['T'] == 0).mean():.3f} occluded")
    assert T.size == 300_000 * 128


def test_bench_workload_bvh_oracle_sample(orc):
    """The 2M-Gaussian bench scene: 262,144 sampled rays against the oracle's
    CPU BVH tracer (many more than brute force can take)."""
    sc = scenes.object_scene(2_000_000, 2)
    dirs = scenes.fibonacci_sphere(128)
    T = trace_dirs(build(sc), dirs).reshape(-1)
    sel = scenes.sample_ray_ids(2_000_000 * 128, 262_144, 13)
    B = orc.BvhTracer(sc)
    ref = B.trace_dirs(dirs, sel)
    B.close()
    maxerr, excluded = compare(T[sel], ref, max_excluded=0.06)
    print(f"2M scene: max |dT| {maxerr:.2e} over {sel.size - excluded} rays, {excluded} in a rounding band")


def test_env_rays_every_ray(orc):
    """Every env-map shadow ray (64 per Gaussian) of the 4,096-Gaussian scene,
    the rays made by the oracle's own generator, against the CPU BVH tracer."""
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(4096, 1)
    env = scenes.envmap(399)
    E = rt.rt_envmap_create(env["radiance"], env["solid_angle"], env["corners"])
    S = 64
    rs = rt.rayspec(rt.RT_RAYS_ENV, env=E, n_samples=S, seed=777)
    T = rt.rt_trace_visibility(build(sc), rs)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    T = T.cpu().numpy().astype(np.float64)
    ids = np.arange(4096 * S, dtype=np.int64)
    ro, rd, rsrc = orc.env_rays(sc["mean"], env, 777, S, ids)
    ref = orc.BvhTracer(sc).trace(ro, rd, rsrc)
    compare(T, ref)
    E.destroy()


def test_env_rays(orc):
    """Shadow rays importance-sampled from the 64x32 environment map: the
    materialised directions equal the oracle's float32 rays bit for bit, and
    the traced T matches brute force."""
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(4096, 1)
    env = scenes.envmap(399)
    E = rt.rt_envmap_create(env["radiance"], env["solid_angle"], env["corners"])
    S = 64
    bvh = build(sc)
    rs = rt.rayspec(rt.RT_RAYS_ENV, env=E, n_samples=S, seed=12345)
    T = rt.rt_trace_visibility(bvh, rs)
    torch.cuda.synchronize()
    T = T.cpu().numpy().astype(np.float64)
    sel = scenes.sample_ray_ids(4096 * S, 8192, 8)
    o, d, s = rt.rt_materialize_rays(bvh, rs, _dev(sel))
    ro, rd, rsrc = orc.env_rays(sc["mean"], env, 12345, S, sel)
    np.testing.assert_array_equal(d.cpu().numpy(), rd)
    np.testing.assert_array_equal(o.cpu().numpy(), ro)
    ref = orc.trace(sc, ro, rd, rsrc)
    compare(T[sel], ref)
    E.destroy()


def test_bench_workload_sampled(orc):
    """The bench workload at full size (2M object-scale Gaussians x 128
    directions, 256M rays) in the launch configuration bench.py times (default
    strategy, persistent grid): 512 sampled rays against brute force."""
    sc = scenes.object_scene(2_000_000, 2)
    dirs = scenes.fibonacci_sphere(128)
    bvh = build(sc)
    T = trace_dirs(bvh, dirs).reshape(-1)
    sel = scenes.sample_ray_ids(2_000_000 * 128, 512, 11)
    o, d, s = orc.dir_rays(sc["mean"], dirs, sel)
    ref = orc.trace(sc, o, d, s)
    # ~170 candidate Gaussians per ray here, so a few % of rays have one within
    # the m^2 rounding band of the 3-sigma support; those are held to the
    # oracle's bounds over that candidate, and counted
    maxerr, flagged = compare(T[sel], ref, max_excluded=0.06)
    print(f"2M scene: max |dT| {maxerr:.2e} over {512 - flagged} rays, {flagged} in a rounding band (bounded)")
    assert np.all((T >= 0) & (T <= 1))


def test_empty_ray_sets():
    """Zero rays in every form (explicit, id list, surrogate batch, PBR and AO
    over an empty scene) with every traversal: nothing written, no error."""
    from paper_2311_16043_gb300 import rt
    sc = scenes.uniform_scene(500, 2)
    bvh = build(sc)
    dirs = _dev(scenes.fibonacci_sphere(8))
    empty_f = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    empty_i = torch.empty(0, dtype=torch.int64, device="cuda")
    for kernel in range(7):
        T = rt.rt_trace_visibility(bvh, rt.rayspec(rt.RT_RAYS_EXPLICIT, ray_o=empty_f, ray_d=empty_f),
                                   opts=rt.trace_opts(kernel=kernel))
        assert T.numel() == 0
        T = rt.rt_trace_visibility(bvh, rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs, ray_ids=empty_i),
                                   opts=rt.trace_opts(kernel=kernel))
        assert T.numel() == 0
    s = rt.rt_surrogate_create(rt.mlp_cfg(batch=1024), seed=1)
    nfb = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    p = rt.rt_surrogate_infer(s, bvh, rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs, ray_ids=empty_i), band=0.3,
                              n_fallback=nfb)
    assert p.numel() == 0 and int(nfb.item()) == 0
    none = {k: v[:0] for k, v in sc.items()}
    b0 = build(none)
    assert rt.rt_trace_visibility_dirs(b0, dirs).numel() == 0
    assert rt.rt_trace_ao(b0, rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs)).numel() == 0
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
