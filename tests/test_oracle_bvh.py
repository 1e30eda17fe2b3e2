"""Pins of the oracle's CPU BVH tracer (CPU only) against the oracle's brute
force, which is pinned by closed forms and invariants elsewhere.  The tracer
walks the LBVH twin (Sec. 4.1) with boxes that cover every candidate the brute
force accepts or flags, so: T equal up to the order of the product, the same
hit counts, band flags a subset of brute force's (equal when nothing stops
early), and every ray flagged only by brute force has T = 0."""
import numpy as np
import pytest

import scenes


def _check(ref, got, tol=1e-12, expect_equal_flags=False):
    assert np.abs(got["T"] - ref["T"]).max() <= tol
    assert np.all((got["flags"] & ~ref["flags"]) == 0), "flag not raised by brute force"
    only_bf = (ref["flags"] != 0) & (got["flags"] == 0)
    assert np.all(got["T"][only_bf] == 0.0)
    if expect_equal_flags:
        np.testing.assert_array_equal(got["flags"], ref["flags"])
    live = ref["T"] > 0
    np.testing.assert_array_equal(got["hits"][live], ref["hits"][live])
    assert np.abs(got["T_exact"][live] - ref["T_exact"][live]).max(initial=0.0) <= tol


def test_uniform_all_rays(orc):
    """4,096-Gaussian uniform scene x 32 directions, every ray, both entry
    points (explicit rays and the direction set)."""
    sc = scenes.uniform_scene(4096, 1)
    dirs = scenes.fibonacci_sphere(32)
    ids = np.arange(4096 * 32, dtype=np.int64)
    o, d, s = orc.dir_rays(sc["mean"], dirs, ids)
    ref = orc.trace(sc, o, d, s)
    B = orc.BvhTracer(sc)
    a = B.trace(o, d, s)
    b = B.trace_dirs(dirs)
    _check(ref, a)
    _check(ref, b)
    for k in ("T", "T_exact", "hits", "flags"):
        np.testing.assert_array_equal(a[k], b[k])
    # the tree prunes: far fewer Gaussian tests than brute force
    assert a["counts"][1] < 0.05 * 4096 * len(ids)


def test_dense_object_scene_early_stop(orc):
    """Object-scale scene where most rays end occluded: the walk stops early
    and still agrees with brute force on a seeded ray sample."""
    sc = scenes.object_scene(150_000, 2)
    dirs = scenes.fibonacci_sphere(128)
    ids = scenes.sample_ray_ids(150_000 * 128, 1200, 7)
    o, d, s = orc.dir_rays(sc["mean"], dirs, ids)
    ref = orc.trace(sc, o, d, s)
    B = orc.BvhTracer(sc)
    got = B.trace_dirs(dirs, ids)
    _check(ref, got)
    assert (ref["T"] == 0).mean() > 0.3  # the stop path is exercised
    # without early termination nothing stops: identical flags
    ref0 = orc.trace(sc, o, d, s, t_min=0.0)
    got0 = B.trace_dirs(dirs, ids, t_min=0.0)
    _check(ref0, got0, expect_equal_flags=True)


def test_axis_directions_and_degenerate_scenes(orc):
    """Directions with zero components (slab NaN cases), rays without a
    source, origins on box faces, and the 0- and 1-Gaussian scenes."""
    rng = np.random.default_rng(3)
    sc = scenes.uniform_scene(512, 5)
    axes = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, 0, 0], [0, -1, 0], [0, 0, -1],
                     [0.6, 0.8, 0], [0, -0.6, 0.8]], np.float32)
    m = 4000
    o = rng.uniform(-1.2, 1.2, (m, 3)).astype(np.float32)
    o[:64] = sc["mean"][:64]                # origins at Gaussian centres
    o[64:128, 0] = sc["mean"][:64, 0]       # origins sharing a coordinate with a centre
    d = axes[rng.integers(0, len(axes), m)]
    B = orc.BvhTracer(sc)
    ref = orc.trace(sc, o, d)
    got = B.trace(o, d)
    _check(ref, got)
    assert (ref["hits"] > 0).mean() > 0.2

    empty = {k: v[:0] for k, v in sc.items()}
    got = orc.BvhTracer(empty).trace(o[:10], d[:10])
    assert np.all(got["T"] == 1.0) and np.all(got["hits"] == 0)

    one = {k: v[:1] for k, v in sc.items()}
    mu = one["mean"][0]
    o1 = np.array([mu - [0, 0, 0.5], mu + [0, 0, 0.5]], np.float32)
    d1 = np.array([[0, 0, 1], [0, 0, 1]], np.float32)
    ref = orc.trace(one, o1, d1)
    got = orc.BvhTracer(one).trace(o1, d1)
    _check(ref, got)
    assert got["hits"][0] == 1 and got["hits"][1] == 0


@pytest.mark.parametrize("band_m2", [0.0, 1e-3])
def test_band_width_is_honoured(orc, band_m2):
    """The boxes follow the m^2 band: a wider band flags (and so visits) more
    candidates, and the subset relation still holds."""
    sc = scenes.object_scene(20_000, 2)
    dirs = scenes.fibonacci_sphere(64)
    ids = scenes.sample_ray_ids(20_000 * 64, 3000, 11)
    o, d, s = orc.dir_rays(sc["mean"], dirs, ids)
    bands = dict(orc.DEFAULT_BANDS, band_m2=band_m2)
    ref = orc.trace(sc, o, d, s, bands=bands)
    got = orc.BvhTracer(sc, bands=bands).trace_dirs(dirs, ids)
    _check(ref, got)


def test_candidates_just_outside_the_support_are_reached(orc):
    """A ray passing a Gaussian at m^2 = 9 + 5e-5 (outside the 3-sigma
    support, inside the m^2 band) is flagged by brute force, so the tracer's
    boxes must reach it although the plain 3-sigma box would not."""
    sig = 0.1
    sc = {"mean": np.zeros((1, 3), np.float32), "scale": np.full((1, 3), sig, np.float32),
          "quat": np.array([[1, 0, 0, 0]], np.float32), "opacity": np.array([0.9], np.float32)}
    ys = sig * np.sqrt(np.array([9 + 5e-5, 9 - 5e-5, 9 + 5e-3]))
    o = np.stack([np.full(3, -1.0), ys, np.zeros(3)], 1).astype(np.float32)
    d = np.tile(np.array([[1, 0, 0]], np.float32), (3, 1))
    ref = orc.trace(sc, o, d)
    assert list(ref["flags"]) == [orc.FLAG_M2, orc.FLAG_M2, 0]
    assert list(ref["hits"]) == [0, 1, 0]
    got = orc.BvhTracer(sc).trace(o, d)
    _check(ref, got, expect_equal_flags=True)
