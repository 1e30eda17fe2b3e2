"""GPU parity of composed scenes (two-level BVH over rigidly placed object
instances, Sec. 4.3) against the oracle's composed-scene tracer, every ray
(rays in a rounding band within the oracle's bounds);
a single identity instance against the plain per-ray trace; instance
updates (top level rebuilt) and refitted objects."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import scenes
from conftest import check_flagged_bounds

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _build(sc):
    from paper_2311_16043_gb300 import rt
    d = {k: _dev(v) for k, v in sc.items()}
    return rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"])


def _xforms(n, seed, spread=0.5):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        R = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        out.append(np.concatenate([R, rng.uniform(-spread, spread, (3, 1))], 1).astype(np.float32))
    return out


def _check(orc, objects, xforms, dirs, T):
    o, d, si, sl = orc.instance_world_rays(objects, xforms, dirs)
    ref = orc.trace_instances(objects, xforms, o, d, si, sl)
    ok = ref["flags"] == 0
    assert ok.mean() > 0.99, (~ok).sum()
    err = np.abs(T.reshape(-1).astype(np.float64) - ref["T"])
    assert err[ok].max() <= TOL, err[ok].max()
    check_flagged_bounds(T.reshape(-1), ref, TOL)
    return ref


@pytest.mark.parametrize("n_inst", [1, 2, 7])
def test_composed_scene_every_ray(orc, n_inst):
    from paper_2311_16043_gb300 import rt
    objs = [scenes.uniform_scene(3000, 41, lo=-0.5, hi=0.5), scenes.object_scene(5000, 42),
            scenes.uniform_scene(33, 43, lo=-0.2, hi=0.2)]
    bvhs = [_build(s) for s in objs]
    pick = [i % 3 for i in range(n_inst)]
    xf = _xforms(n_inst, 5)
    dirs = scenes.fibonacci_sphere(16)
    scene = rt.rt_scene_create([bvhs[i] for i in pick], xf)
    T = rt.rt_scene_trace_dirs(scene, _dev(dirs))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    ref = _check(orc, [objs[i] for i in pick], xf, dirs, T.cpu().numpy())
    if n_inst > 1:
        assert (ref["T"] < 0.9).mean() > 0.1


def test_identity_instance_equals_plain_trace():
    from paper_2311_16043_gb300 import rt
    sc = scenes.object_scene(20_000, 2)
    bvh = _build(sc)
    dirs = _dev(scenes.fibonacci_sphere(32))
    eye = np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32)
    scene = rt.rt_scene_create([bvh], [eye])
    a = rt.rt_scene_trace_dirs(scene, dirs)
    b = rt.rt_trace_visibility_dirs(bvh, dirs, opts=rt.trace_opts(kernel=rt.RT_KERNEL_RAY_WIDE))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    assert (a.view(-1) - b.view(-1)).abs().max().item() <= 1e-6


def test_update_and_refit(orc):
    """Moving instances rebuilds only the top level; refitting an object and
    updating the scene re-reads its box; both match the oracle."""
    from paper_2311_16043_gb300 import rt
    objs = [scenes.uniform_scene(2000, 51, lo=-0.5, hi=0.5), scenes.uniform_scene(1500, 52, lo=-0.5, hi=0.5)]
    bvhs = [_build(s) for s in objs]
    dirs = scenes.fibonacci_sphere(8)
    xf = _xforms(4, 6)
    pick = [0, 1, 0, 1]
    scene = rt.rt_scene_create([bvhs[i] for i in pick], xf)
    xf2 = _xforms(4, 7, spread=1.0)
    rt.rt_scene_update(scene, xf2)
    T = rt.rt_scene_trace_dirs(scene, _dev(dirs))
    torch.cuda.synchronize()
    _check(orc, [objs[i] for i in pick], xf2, dirs, T.cpu().numpy())
    moved = {k: v.copy() for k, v in objs[1].items()}
    moved["mean"] = (moved["mean"] * np.float32(1.5)).astype(np.float32)  # the object grows
    d = {k: _dev(v) for k, v in moved.items()}
    rt.rt_bvh_refit(bvhs[1], d["mean"], d["scale"], d["quat"], d["opacity"])
    rt.rt_scene_update(scene, xf2)
    T = rt.rt_scene_trace_dirs(scene, _dev(dirs))
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    _check(orc, [objs[0], moved, objs[0], moved], xf2, dirs, T.cpu().numpy())


def test_scene_argument_errors():
    from paper_2311_16043_gb300 import rt
    a = _build(scenes.uniform_scene(100, 1))
    b = rt.rt_build_bvh(*(_dev(v) for v in (lambda s: (s["mean"], s["scale"], s["quat"], s["opacity"]))(
        scenes.uniform_scene(100, 2))), rt.params(k_sigma=2.5))
    eye = np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32)
    with pytest.raises(rt.RTError):   # differing params
        rt.rt_scene_create([a, b], [eye, eye])
    bad = eye.copy()
    bad[0, 3] = np.nan
    with pytest.raises(rt.RTError):
        rt.rt_scene_create([a], [bad])


def test_composed_workload_sampled(orc):
    """The composed-scene workload at full size in the launch configuration
    the benchmark times: 4 object-scale objects (125k Gaussians each) as 16
    overlapping instances, one top-level rebuild and the trace of every
    Gaussian of every instance along 128 directions (256M rays); all 128 rays
    of 8 sampled Gaussians per instance against the oracle's composed-scene
    tracer."""
    from paper_2311_16043_gb300 import rt
    objs, pick, xf = scenes.composed_objects()
    bvhs = [_build(s) for s in objs]
    dirs = scenes.fibonacci_sphere(128)
    scene = rt.rt_scene_create([bvhs[i] for i in pick], xf)
    T = torch.full((scene.n_total, dirs.shape[0]), -1.0, device="cuda")
    rt.rt_scene_update(scene, xf)
    rt.rt_scene_trace_dirs(scene, _dev(dirs), T)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    assert float(T.min()) >= 0.0 and float(T.max()) <= 1.0
    inst = [objs[i] for i in pick]
    rng = np.random.default_rng(9)
    rows, o_all, d_all, si_all, sl_all = [], [], [], [], []
    off = 0
    for j, sc in enumerate(inst):
        n = sc["mean"].shape[0]
        g = np.sort(rng.choice(n, 8, replace=False))
        o, d, _, sl = orc.instance_world_rays([{"mean": sc["mean"][g]}], [xf[j]], dirs)
        o_all.append(o)
        d_all.append(d)
        si_all.append(np.full(o.shape[0], j, np.int32))
        sl_all.append(g[sl].astype(np.int32))
        rows.append(off + g)
        off += n
    ref = orc.trace_instances(inst, xf, np.concatenate(o_all), np.concatenate(d_all),
                              np.concatenate(si_all), np.concatenate(sl_all))
    got = T[_dev(np.concatenate(rows))].reshape(-1).cpu().numpy().astype(np.float64)
    ok = ref["flags"] == 0
    assert ok.mean() > 0.97, (~ok).sum()
    err = np.abs(got - ref["T"])
    assert err[ok].max() <= TOL, err[ok].max()
    check_flagged_bounds(got, ref, TOL)
    assert (ref["T"] < 0.5).mean() > 0.1  # the instances occlude one another
    scene.destroy()


@pytest.mark.parametrize("kind", ["hemi", "env"])
def test_composed_scene_hemi_env_every_ray(orc, kind):
    """Sec. 4.3 relighting of a composed scene: the hemisphere sets about
    each Gaussian's world-frame normal (Sec. 3.3) and env-map shadow rays,
    traced through a 4-instance scene; every ray against the oracle's
    composed-scene tracer on the oracle's own rays."""
    from paper_2311_16043_gb300 import rt
    objs = [scenes.object_scene(3000, 51), scenes.uniform_scene(2000, 52, lo=-0.4, hi=0.4)]
    bvhs = [_build(s) for s in objs]
    pick = [0, 1, 0, 1]
    xf = _xforms(4, 9)
    objects = [objs[i] for i in pick]
    scene = rt.rt_scene_create([bvhs[i] for i in pick], xf)
    n_total = sum(o["mean"].shape[0] for o in objects)
    m = orc.instance_world_means(objects, xf)
    K = 16
    ids = np.arange(n_total * K, dtype=np.int64)
    E = None
    if kind == "hemi":
        hemi = scenes.fibonacci_hemisphere(K)
        nw = np.concatenate([scenes.shortest_axis_normals(o["scale"], o["quat"]).astype(np.float64) @ X[:, :3].T
                             for o, X in zip(objects, xf)])
        nw = (nw / np.linalg.norm(nw, axis=1, keepdims=True)).astype(np.float32)
        rs = rt.rayspec(rt.RT_RAYS_HEMI, dirs=_dev(hemi), normals=_dev(nw))
        o, d, s = orc.hemi_rays(m, nw, hemi, ids)
    else:
        env = scenes.envmap(399)
        E = rt.rt_envmap_create(env["radiance"], env["solid_angle"], env["corners"])
        rs = rt.rayspec(rt.RT_RAYS_ENV, env=E, n_samples=K, seed=123)
        o, d, s = orc.env_rays(m, env, 123, K, ids)
    T = rt.rt_scene_trace(scene, rs)
    torch.cuda.synchronize()
    assert rt.rt_status_last() == 0
    assert T.shape == (n_total, K)
    si, sl = orc.instance_rows(objects, s)
    ref = orc.trace_instances(objects, xf, o, d, si, sl)
    ok = ref["flags"] == 0
    assert ok.mean() > 0.99, (~ok).sum()
    got = T.cpu().numpy().reshape(-1).astype(np.float64)
    err = np.abs(got - ref["T"])
    assert err[ok].max() <= TOL, err[ok].max()
    check_flagged_bounds(got, ref, TOL)
    assert (ref["T"] < 0.9).mean() > 0.05  # the instances shadow each other
    # DIRS through the general entry point = rt_scene_trace_dirs
    dirs = _dev(scenes.fibonacci_sphere(8))
    a = rt.rt_scene_trace(scene, rt.rayspec(rt.RT_RAYS_DIRS, dirs=dirs))
    b = rt.rt_scene_trace_dirs(scene, dirs)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    if E is not None:
        E.destroy()
    scene.destroy()
