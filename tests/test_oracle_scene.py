"""Pins of the oracle's composed-scene tracer (CPU only): one instance under
the identity map is the plain object; a composition equals the union scene
(every Gaussian moved to the world in FP64, brute force), bounds included;
and a rigid motion of the whole composition (instances and directions)
leaves T unchanged."""
import numpy as np
from scipy.spatial.transform import Rotation

import scenes

TOL = 1e-5


def _xform(R, t):
    return np.concatenate([np.asarray(R, np.float64), np.asarray(t, np.float64)[:, None]], 1).astype(np.float32)


def _composition(seed=0, n_inst=4):
    rng = np.random.default_rng(seed)
    objs = [scenes.uniform_scene(600, 31, lo=-0.5, hi=0.5), scenes.uniform_scene(400, 32, lo=-0.4, hi=0.4)]
    objects, xforms = [], []
    for i in range(n_inst):
        R = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        objects.append(objs[i % 2])
        xforms.append(_xform(R, rng.uniform(-0.4, 0.4, 3)))
    return objects, xforms


def _world_union(objects, xforms):
    """Every Gaussian moved into the world in FP64: mean R mu + t, rotation
    R R_q (so Sigma_w = R Sigma R^T)."""
    out = {"mean": [], "scale": [], "quat": [], "opacity": []}
    for sc, xf in zip(objects, xforms):
        X = xf.astype(np.float64)
        R, t = X[:, :3], X[:, 3]
        out["mean"].append(sc["mean"].astype(np.float64) @ R.T + t)
        q = sc["quat"].astype(np.float64)
        rq = Rotation.from_matrix(R) * Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1))
        xyzw = rq.as_quat()
        out["quat"].append(np.concatenate([xyzw[:, 3:], xyzw[:, :3]], 1))
        out["scale"].append(sc["scale"].astype(np.float64))
        out["opacity"].append(sc["opacity"].astype(np.float64))
    return {k: np.concatenate(v) for k, v in out.items()}


def test_identity_instance_is_the_object(orc):
    sc = scenes.uniform_scene(2000, 5)
    dirs = scenes.fibonacci_sphere(16)
    eye = _xform(np.eye(3), np.zeros(3))
    o, d, si, sl = orc.instance_world_rays([sc], [eye], dirs)
    got = orc.trace_instances([sc], [eye], o, d, si, sl)
    ref = orc.BvhTracer(sc).trace_dirs(dirs, t_min=1e-4)
    o2, d2, s2 = orc.dir_rays(sc["mean"], dirs, np.arange(2000 * 16))
    np.testing.assert_array_equal(o, o2)
    np.testing.assert_array_equal(sl, s2)
    full = ref["T"] > 0
    np.testing.assert_allclose(got["T"], ref["T"], atol=1e-14)
    np.testing.assert_array_equal(got["flags"][full], ref["flags"][full])
    # a walk that ran to the end (T > 0) gives the plain tracer's bounds
    np.testing.assert_allclose(got["T_lo"][full], ref["T_lo"][full], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got["T_hi"][full], ref["T_hi"][full], rtol=1e-12, atol=0)


def test_composition_is_the_union_scene(orc):
    objects, xforms = _composition()
    dirs = scenes.fibonacci_sphere(8)
    o, d, si, sl = orc.instance_world_rays(objects, xforms, dirs)
    got = orc.trace_instances(objects, xforms, o, d, si, sl)
    world = _world_union(objects, xforms)
    base = np.cumsum([0] + [sc["mean"].shape[0] for sc in objects])[:-1]
    src = (base[si] + sl).astype(np.int32)
    ref = orc.trace(world, o, d, src)
    ok = (ref["flags"] == 0) & (got["flags"] == 0)
    assert ok.mean() > 0.99
    assert np.abs(got["T"] - ref["T"])[ok].max() <= TOL
    assert (got["T"] < 0.5).mean() > 0.2  # the instances do shadow each other
    # the bounds: they bracket T_exact, close on it without a borderline
    # candidate, and equal the union scene's where both flag the same tests
    cand = orc.FLAG_M2 | orc.FLAG_ALPHA | orc.FLAG_T
    assert np.all(got["T_lo"] <= got["T_exact"] * (1 + 1e-12))
    assert np.all(got["T_exact"] <= got["T_hi"] * (1 + 1e-12))
    plain = (got["flags"] & cand) == 0
    assert np.array_equal(got["T_lo"][plain], got["T_exact"][plain])
    assert np.array_equal(got["T_hi"][plain], got["T_exact"][plain])
    same = got["flags"] == ref["flags"]
    assert same.mean() > 0.99 and (same & ~plain).sum() >= 5
    assert np.abs(got["T_lo"] - ref["T_lo"])[same].max() <= TOL
    assert np.abs(got["T_hi"] - ref["T_hi"])[same].max() <= TOL
    wide = ~plain & (got["T_hi"] > 1e-3)
    assert np.all(got["T_lo"][wide] < got["T_hi"][wide])


def test_rigid_motion_of_the_composition(orc):
    objects, xforms = _composition(1)
    dirs = scenes.fibonacci_sphere(8)
    o, d, si, sl = orc.instance_world_rays(objects, xforms, dirs)
    a = orc.trace_instances(objects, xforms, o, d, si, sl)
    G = Rotation.random(random_state=7).as_matrix()
    g = np.array([0.3, -1.2, 2.0])
    moved = [_xform(G @ x[:, :3].astype(np.float64), G @ x[:, 3].astype(np.float64) + g) for x in xforms]
    dirs2 = (dirs.astype(np.float64) @ G.T).astype(np.float32)
    o2, d2, si2, sl2 = orc.instance_world_rays(objects, moved, dirs2)
    b = orc.trace_instances(objects, moved, o2, d2, si2, sl2)
    ok = (a["flags"] == 0) & (b["flags"] == 0)
    assert ok.mean() > 0.99
    assert np.abs(a["T"] - b["T"])[ok].max() <= TOL


def test_world_means_and_rows(orc):
    """The world means are the origins the direction rays start from (less
    the offset along d), row by row in scene order; rows map back to their
    instance and local index."""
    objs = [scenes.uniform_scene(50, 3), scenes.uniform_scene(20, 4)]
    xf = [np.concatenate([np.eye(3), [[0.5], [0.0], [-1.0]]], 1).astype(np.float32),
          np.concatenate([np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]), [[0.0], [2.0], [0.0]]], 1).astype(np.float32)]
    m = orc.instance_world_means(objs, xf)
    assert m.dtype == np.float32 and m.shape == (70, 3)
    np.testing.assert_array_equal(m[:50], (objs[0]["mean"] + np.float32([0.5, 0.0, -1.0])).astype(np.float32))
    mu = objs[1]["mean"]
    np.testing.assert_allclose(m[50:], np.stack([-mu[:, 1], mu[:, 0] + 2.0, mu[:, 2]], 1), rtol=0, atol=1e-6)
    dirs = scenes.fibonacci_sphere(4)
    o, d, si, sl = orc.instance_world_rays(objs, xf, dirs, eps=0.0)
    np.testing.assert_array_equal(o[::4], m)
    inst, loc = orc.instance_rows(objs, np.arange(70))
    np.testing.assert_array_equal(inst, si[::4])
    np.testing.assert_array_equal(loc, sl[::4])
