"""Pins of the FP64 brute-force visibility oracle (CPU only).

Each test fixes the oracle against something other than itself: a closed form
of Eq. 13-15, an invariant stated in Sec. 4.1 (order independence), a library
routine (scipy rotations, numpy matrix inverse, scipy scalar minimisation) or
the threshold readings (3-sigma support, alpha >= 1/255, t* > 0, T_min snap).
"""
import math

import numpy as np
import pytest

AMIN = 1.0 / 255.0


def scene(mu, s, q=None, o=None):
    mu = np.asarray(mu, np.float64).reshape(-1, 3)
    n = mu.shape[0]
    s = np.broadcast_to(np.asarray(s, np.float64), (n, 3)).copy()
    q = np.tile([1.0, 0, 0, 0], (n, 1)) if q is None else np.asarray(q, np.float64).reshape(n, 4)
    o = np.full(n, 0.5) if o is None else np.broadcast_to(np.asarray(o, np.float64), (n,)).copy()
    return {"mean": mu, "scale": s, "quat": q, "opacity": o}


def ray(o, d):
    return np.asarray(o, np.float64).reshape(1, 3), np.asarray(d, np.float64).reshape(1, 3)


def T1(orc, sc, o, d, src=None, **kw):
    ro, rd = ray(o, d)
    return orc.trace(sc, ro, rd, None if src is None else np.array([src], np.int32), **kw)["T"][0]


def test_rotation_matches_scipy(orc):
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.standard_normal(4) * rng.uniform(0.1, 3.0)
        R = orc.rotation(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-12)


def test_head_on_isotropic(orc):
    # m = 0 at the peak, so alpha = o and T = 1 - o
    for o in (0.05, 0.5, 0.93):
        sc = scene([0, 0, 5], 0.1, o=o)
        assert T1(orc, sc, [0, 0, 0], [0, 0, 1]) == pytest.approx(1 - o, abs=1e-15)


@pytest.mark.parametrize("b", [0.0, 0.05, 0.1, 0.2, 0.25, 0.29])
def test_offset_isotropic(orc, b):
    sig, o = 0.1, 0.8
    sc = scene([0, 0, 2], sig, o=o)
    alpha = o * math.exp(-b * b / (2 * sig * sig))
    assert T1(orc, sc, [b, 0, -1], [0, 0, 1]) == pytest.approx(1 - alpha, abs=1e-14)


def test_axis_aligned_anisotropic(orc):
    s = np.array([0.3, 0.05, 0.1])
    sc = scene([1, 0, 0], s, o=0.9)
    for y, z in [(0.0, 0.0), (0.04, 0.0), (0.0, 0.12), (0.03, 0.08), (-0.06, 0.1)]:
        m2 = y * y / s[1] ** 2 + z * z / s[2] ** 2
        want = 1 - 0.9 * math.exp(-m2 / 2) if m2 <= 9 and 0.9 * math.exp(-m2 / 2) >= AMIN else 1.0
        assert T1(orc, sc, [-2, y, z], [1, 0, 0]) == pytest.approx(want, abs=1e-14)


def test_rotated_anisotropic_orientation(orc):
    # 90 degrees about +z maps local x to world +y and local y to world -x.
    c = math.cos(math.pi / 4)
    sc = scene([0, 0, 0], [0.5, 0.05, 0.05], q=[c, 0, 0, c], o=0.9)
    b = 0.4  # offset along world y = local x (scale 0.5)
    want = 1 - 0.9 * math.exp(-(b / 0.5) ** 2 / 2)
    assert T1(orc, sc, [-3, b, 0], [1, 0, 0]) == pytest.approx(want, abs=1e-12)
    b = 0.08  # offset along world x = local -y (scale 0.05)
    want = 1 - 0.9 * math.exp(-(b / 0.05) ** 2 / 2)
    assert T1(orc, sc, [b, -3, 0], [0, 1, 0]) == pytest.approx(want, abs=1e-12)


def _sigma_inv(q, s):
    from scipy.spatial.transform import Rotation
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    return np.linalg.inv(R @ np.diag(np.asarray(s) ** 2) @ R.T)


def test_peak_is_minimiser_of_mahalanobis(orc):
    """Eq. 13-14 (read with Sigma^-1): r_x is where G peaks along the ray."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(1)
    for _ in range(40):
        q = rng.standard_normal(4)
        s = np.exp(rng.uniform(np.log(0.05), np.log(0.4), 3))
        mu = rng.uniform(-1, 1, 3)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        # origin placed so the peak is at t ~ 2 in front, with a small offset
        o = mu - 2.0 * d + rng.normal(0, 0.3 * s.min(), 3)
        Si = _sigma_inv(q, s)

        def maha(t):
            e = o + t * d - mu
            return e @ Si @ e
        res = minimize_scalar(maha, bracket=(0.0, 2.0, 4.0), tol=1e-12)
        m2 = res.fun
        sc = scene(mu, s, q=q, o=0.99)
        T = T1(orc, sc, o, d, t_min=0.0)
        alpha = 0.99 * math.exp(-m2 / 2)
        want = 1 - alpha if (m2 <= 9 and alpha >= AMIN) else 1.0
        assert T == pytest.approx(want, abs=1e-9)


def _numpy_trace(sc, ro, rd, src, t_min=1e-4):
    """Independent formulation: world-space Sigma^-1 from numpy.linalg.inv and
    scipy rotations; t* = (mu - o)^T Sigma^-1 d / d^T Sigma^-1 d."""
    n = sc["mean"].shape[0]
    Sis = [_sigma_inv(sc["quat"][j], sc["scale"][j]) for j in range(n)]
    out = np.ones(ro.shape[0])
    for r in range(ro.shape[0]):
        T = 1.0
        for j in range(n):
            if j == src[r]:
                continue
            Si = Sis[j]
            t = (sc["mean"][j] - ro[r]) @ Si @ rd[r] / (rd[r] @ Si @ rd[r])
            e = ro[r] + t * rd[r] - sc["mean"][j]
            m2 = e @ Si @ e
            a = sc["opacity"][j] * math.exp(-m2 / 2)
            if t > 0 and m2 <= 9 and a >= AMIN:
                T *= 1 - a
        out[r] = 0.0 if T < t_min else T
    return out


def test_matches_independent_numpy_formulation(orc):
    import scenes
    sc = scenes.uniform_scene(40, 11, log_scale_mean=math.log(0.15))
    sc = {k: v.astype(np.float64) for k, v in sc.items()}
    dirs = scenes.fibonacci_sphere(8)
    ids = np.arange(40 * 8, dtype=np.int64)
    ro, rd, src = orc.dir_rays(sc["mean"].astype(np.float32), dirs, ids)
    res = orc.trace(sc, ro, rd, src)
    want = _numpy_trace(sc, ro.astype(np.float64), rd.astype(np.float64), src)
    ok = res["flags"] == 0
    assert ok.mean() > 0.95
    np.testing.assert_allclose(res["T"][ok], want[ok], atol=1e-10)
    assert (res["hits"] > 0).mean() > 0.3  # the case exercises real hits


def test_miss_and_empty(orc):
    sc = scene([0, 0, 5], 0.1, o=0.9)
    assert T1(orc, sc, [0, 0, 0], [0, 0, -1]) == 1.0  # peak behind the origin
    assert T1(orc, sc, [1, 0, 0], [0, 0, 1]) == 1.0   # passes 10 sigma away
    empty = scene(np.zeros((0, 3)), 0.1)
    ro = np.zeros((3, 3))
    rd = np.tile([0.0, 0, 1], (3, 1))
    np.testing.assert_array_equal(orc.trace(empty, ro, rd)["T"], 1.0)


@pytest.mark.parametrize("k,o", [(1, 0.3), (4, 0.3), (7, 0.6), (12, 0.5), (20, 0.4)])
def test_k_identical_on_ray(orc, k, o):
    mu = np.stack([np.zeros(k), np.zeros(k), 1.0 + np.arange(k)], 1)
    sc = scene(mu, 0.05, o=o)
    want = (1 - o) ** k
    got = T1(orc, sc, [0, 0, 0], [0, 0, 1])
    assert got == (0.0 if want < 1e-4 else pytest.approx(want, rel=1e-13))
    assert T1(orc, sc, [0, 0, 0], [0, 0, 1], t_min=0.0) == pytest.approx(want, rel=1e-13)


def _dir_scene(orc, n, seed, k=16, log_s=math.log(0.08)):
    import scenes
    sc = scenes.uniform_scene(n, seed, log_scale_mean=log_s)
    dirs = scenes.fibonacci_sphere(k)
    ids = np.arange(n * k, dtype=np.int64)
    ro, rd, src = orc.dir_rays(sc["mean"], dirs, ids)
    return {kk: v.astype(np.float64) for kk, v in sc.items()}, ro, rd, src


def test_order_independence(orc):
    """Sec. 4.1: the order of the alpha_j does not change T."""
    sc, ro, rd, src = _dir_scene(orc, 300, 3)
    base = orc.trace(sc, ro, rd, src, t_min=0.0)
    perm = np.random.default_rng(5).permutation(300)
    inv = np.argsort(perm)
    sc2 = {k: v[perm] for k, v in sc.items()}
    got = orc.trace(sc2, ro, rd, inv[src].astype(np.int32), t_min=0.0)
    np.testing.assert_allclose(got["T"], base["T"], rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(got["hits"], base["hits"])
    assert base["hits"].mean() > 1.0


def test_bounds_and_monotone_in_opacity(orc):
    sc, ro, rd, src = _dir_scene(orc, 300, 4)
    base = orc.trace(sc, ro, rd, src, t_min=0.0)["T"]
    assert np.all((base >= 0) & (base <= 1))
    rng = np.random.default_rng(6)
    sc2 = dict(sc)
    o2 = sc["opacity"].copy()
    pick = rng.random(300) < 0.3
    o2[pick] = np.minimum(o2[pick] * 1.5 + 0.01, 0.999)
    sc2["opacity"] = o2
    up = orc.trace(sc2, ro, rd, src, t_min=0.0)["T"]
    assert np.all(up <= base + 1e-15)
    assert np.any(up < base - 1e-6)


def test_scale_invariance(orc):
    sc, ro, rd, src = _dir_scene(orc, 200, 7)
    base = orc.trace(sc, ro, rd, src)
    for c in (2.0, 0.25):  # powers of two: every operation scales exactly
        sc2 = dict(sc, mean=sc["mean"] * c, scale=sc["scale"] * c)
        got = orc.trace(sc2, ro.astype(np.float64) * c, rd, src)
        np.testing.assert_array_equal(got["T"], base["T"])
    sc3 = dict(sc, mean=sc["mean"] * 3.7, scale=sc["scale"] * 3.7)
    got = orc.trace(sc3, ro.astype(np.float64) * 3.7, rd, src)
    ok = (base["flags"] == 0) & (got["flags"] == 0)
    np.testing.assert_allclose(got["T"][ok], base["T"][ok], atol=1e-10)


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b.T
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)


def test_rigid_motion_invariance(orc):
    from scipy.spatial.transform import Rotation
    sc, ro, rd, src = _dir_scene(orc, 200, 8)
    base = orc.trace(sc, ro, rd, src)
    rng = np.random.default_rng(9)
    qr = rng.standard_normal(4)
    qr /= np.linalg.norm(qr)
    Q = Rotation.from_quat([qr[1], qr[2], qr[3], qr[0]]).as_matrix()
    tvec = rng.uniform(-5, 5, 3)
    sc2 = dict(sc, mean=sc["mean"] @ Q.T + tvec, quat=_qmul(qr, sc["quat"]))
    got = orc.trace(sc2, ro.astype(np.float64) @ Q.T + tvec, rd.astype(np.float64) @ Q.T, src)
    ok = (base["flags"] == 0) & (got["flags"] == 0)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(got["T"][ok], base["T"][ok], atol=1e-10)


def test_threshold_readings(orc):
    sig = 0.1
    # 3-sigma support: accepted at m = 3(1 - 1e-6), rejected at 3(1 + 1e-6)
    sc = scene([0, 0, 2], sig, o=0.99)
    b_in, b_out = 3 * sig * (1 - 1e-6), 3 * sig * (1 + 1e-6)
    a_in = 0.99 * math.exp(-((b_in / sig) ** 2) / 2)
    assert T1(orc, sc, [b_in, 0, 0], [0, 0, 1]) == pytest.approx(1 - a_in, abs=1e-14)
    assert T1(orc, sc, [b_out, 0, 0], [0, 0, 1]) == 1.0
    # alpha cutoff: a head-on hit has alpha = o
    assert T1(orc, scene([0, 0, 2], sig, o=AMIN), [0, 0, 0], [0, 0, 1]) == pytest.approx(1 - AMIN)
    assert T1(orc, scene([0, 0, 2], sig, o=AMIN * (1 - 1e-9)), [0, 0, 0], [0, 0, 1]) == 1.0
    # t* > 0: a Gaussian whose peak is just behind the origin does not count
    assert T1(orc, scene([0, 0, -1e-3], 0.5, o=0.5), [0, 0, 0], [0, 0, 1]) == 1.0
    assert T1(orc, scene([0, 0, 1e-3], 0.5, o=0.5), [0, 0, 0], [0, 0, 1]) == pytest.approx(0.5)
    # T_min snap: (1-o)^2 just above and just below 1e-4
    for o, snapped in ((1 - 1.0001e-2, False), (1 - 0.9999e-2, True)):
        sc2 = scene([[0, 0, 1], [0, 0, 2]], 0.05, o=o)
        want = (1 - o) ** 2
        got = T1(orc, sc2, [0, 0, 0], [0, 0, 1])
        assert got == (0.0 if snapped else pytest.approx(want, rel=1e-12))
    # self exclusion by index
    sc3 = scene([[0, 0, 1e-4], [0, 0, 1]], 0.05, o=[0.9, 0.5])
    assert T1(orc, sc3, [0, 0, 0], [0, 0, 1], src=0) == pytest.approx(0.5)
    assert T1(orc, sc3, [0, 0, 0], [0, 0, 1], src=1) == pytest.approx(0.1)


def test_band_flags(orc):
    sig = 0.1
    sc = scene([0, 0, 2], sig, o=0.99)
    ro, rd = ray([3 * sig * (1 + 1e-7), 0, 0], [0, 0, 1])
    assert orc.trace(sc, ro, rd)["flags"][0] & orc.FLAG_M2
    ro, rd = ray([0, 0, 0], [0, 0, 1])
    r = orc.trace(scene([0, 0, 2], sig, o=AMIN + 1e-8), ro, rd)
    assert r["flags"][0] & orc.FLAG_ALPHA
    r = orc.trace(scene([0, 0, 1e-8], 0.5, o=0.5), ro, rd)
    assert r["flags"][0] & orc.FLAG_T
    o = 1 - math.sqrt(1e-4 + 1e-9)
    r = orc.trace(scene([[0, 0, 1], [0, 0, 2]], 0.05, o=o), ro, rd)
    assert r["flags"][0] & orc.FLAG_TMIN
    r = orc.trace(scene([0, 0, 2], sig, o=0.5), ro, rd)
    assert r["flags"][0] == 0


def test_borderline_bounds(orc):
    """T_lo / T_hi: a candidate inside a band is taken in T_lo and left out of
    T_hi whichever way the exact test went; the other candidates count as in
    T_exact; no band bit -> T_lo = T_hi = T_exact."""
    sig = 0.1
    sure = scene([0, 0, 5], sig, o=0.3)  # head on: alpha = 0.3, far from every band
    ro, rd = ray([0, 0, 0], [0, 0, 1])
    for b, took in ((3 * sig * (1 - 1e-7), True), (3 * sig * (1 + 1e-7), False)):
        # a second Gaussian the ray passes at m = 3 (1 -/+ 1e-7): in the m^2 band
        sc = {k: np.concatenate([sure[k], scene([-b, 0, 2], sig, o=0.99)[k]]) for k in sure}
        r = orc.trace(sc, ro, rd)
        a = 0.99 * math.exp(-((b / sig) ** 2) / 2)
        assert r["flags"][0] & orc.FLAG_M2
        assert r["T_hi"][0] == pytest.approx(0.7, rel=1e-14)
        assert r["T_lo"][0] == pytest.approx(0.7 * (1 - a), rel=1e-14)
        assert r["T_exact"][0] == pytest.approx(0.7 * (1 - a) if took else 0.7, rel=1e-14)
        assert r["n_border"][0] == 1 and r["hits"][0] == (2 if took else 1)
    # two borderline candidates, one either side of 3 sigma
    b1, b2 = 3 * sig * (1 - 1e-7), 3 * sig * (1 + 1e-7)
    sc = {k: np.concatenate([sure[k], scene([-b1, 0, 2], sig, o=0.99)[k], scene([0, b2, 3], sig, o=0.99)[k]])
          for k in sure}
    r = orc.trace(sc, ro, rd)
    a1, a2 = (0.99 * math.exp(-((b / sig) ** 2) / 2) for b in (b1, b2))
    assert r["n_border"][0] == 2 and r["hits"][0] == 2
    assert r["T_lo"][0] == pytest.approx(0.7 * (1 - a1) * (1 - a2), rel=1e-14)
    assert r["T_hi"][0] == pytest.approx(0.7, rel=1e-14)
    r = orc.trace(sure, ro, rd)
    assert r["flags"][0] == 0 and r["T_lo"][0] == r["T_hi"][0] == r["T_exact"][0] and r["n_border"][0] == 0
    # a scene of many rays: the bounds bracket T_exact, equal it without a
    # candidate bit, and the tree walk gives the brute force's bounds
    sc, ro2, rd2, src = _dir_scene(orc, 300, 12)
    res = orc.trace(sc, ro2, rd2, src, t_min=0.0)
    cand = (res["flags"] & (orc.FLAG_M2 | orc.FLAG_ALPHA | orc.FLAG_T)) != 0
    assert np.all(res["T_lo"] <= res["T_exact"] * (1 + 1e-12)) and np.all(res["T_exact"] <= res["T_hi"] * (1 + 1e-12))
    assert np.array_equal(res["T_lo"][~cand], res["T_exact"][~cand]) and np.array_equal(res["T_hi"][~cand],
                                                                                          res["T_exact"][~cand])
    assert np.array_equal(res["n_border"] > 0, cand) and cand.any()
    tb = orc.BvhTracer(sc).trace(ro2, rd2, src, t_min=0.0)
    np.testing.assert_allclose(tb["T_lo"], res["T_lo"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tb["T_hi"], res["T_hi"], rtol=1e-12, atol=0)


def test_hit_lists_agree_with_trace(orc):
    sc, ro, rd, src = _dir_scene(orc, 300, 12)
    res = orc.trace(sc, ro, rd, src, t_min=0.0)
    ids, cnt = orc.trace_hits(sc, ro, rd, src, cap=64)
    np.testing.assert_array_equal(cnt, res["hits"])
    # recompute T from the listed ids with the single-Gaussian oracle
    for r in range(0, ro.shape[0], 97):
        T = 1.0
        for j in ids[r, :cnt[r]]:
            one = {k: v[j:j + 1] for k, v in sc.items()}
            T *= orc.trace(one, ro[r:r + 1], rd[r:r + 1], None, t_min=0.0)["T"][0]
        assert T == pytest.approx(res["T"][r], rel=1e-12)
