"""Pins of the oracle's hemisphere direction sets and per-Gaussian PBR colour
(Sec. 3.3, Eq. 8-10), CPU only: frame orthonormality and handedness, the
closed-form poles of the frame construction, GGX normalisation, the microfacet
change of variables (which fixes the factor 4 of Eq. 9), Fresnel and Smith
limits, reciprocity, SH orthonormality and the addition theorem, bilinear
environment lookup at pixel centres and across the azimuth seam, closed
forms of the Eq. 10 sum (the Fibonacci midpoint rule integrates cos exactly),
and its monotonicity in each visibility."""
import math

import numpy as np
import pytest

import scenes


def _frames(orc, normals, hemi):
    n = normals.shape[0]
    K = hemi.shape[0]
    mean = np.zeros((n, 3), np.float32)
    _, d, s = orc.hemi_rays(mean, normals, hemi, np.arange(n * K))
    assert np.array_equal(s, np.repeat(np.arange(n), K))
    return d.reshape(n, K, 3).astype(np.float64)


def test_hemisphere_frame_is_a_rotation(orc):
    rng = np.random.default_rng(1)
    nrm = rng.standard_normal((500, 3)).astype(np.float32)
    nrm[:4] = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1e-3, -1]]
    hemi = scenes.fibonacci_hemisphere(16)
    d = _frames(orc, nrm, hemi)
    H = hemi.astype(np.float64)
    nhat = nrm / np.linalg.norm(nrm.astype(np.float64), axis=1, keepdims=True)
    for g in range(nrm.shape[0]):
        # D = H F^T with F = [t1 t2 n]: solve for F and check it is a proper rotation
        F = np.linalg.lstsq(H, d[g], rcond=None)[0].T
        np.testing.assert_allclose(F.T @ F, np.eye(3), atol=2e-6)
        assert abs(np.linalg.det(F) - 1.0) < 2e-6
        np.testing.assert_allclose(F[:, 2], nhat[g], atol=2e-7)   # local z is the normal
    # every direction lies on the normal's side
    assert np.all(np.einsum("gkc,gc->gk", d, nhat) > 0)


def test_hemisphere_frame_poles(orc):
    hemi = scenes.fibonacci_hemisphere(32)
    d = _frames(orc, np.array([[0, 0, 1], [0, 0, -1]], np.float32), hemi)
    np.testing.assert_array_equal(d[0], hemi)                        # identity frame
    np.testing.assert_array_equal(d[1], hemi * np.array([1, -1, -1]))  # rotation by pi about x


def test_hemisphere_origins(orc):
    rng = np.random.default_rng(2)
    mean = rng.uniform(-1, 1, (50, 3)).astype(np.float32)
    nrm = rng.standard_normal((50, 3)).astype(np.float32)
    hemi = scenes.fibonacci_hemisphere(8)
    o, d, s = orc.hemi_rays(mean, nrm, hemi, np.arange(400), eps=1e-4)
    want = (mean[s] + (np.float32(1e-4) * d).astype(np.float32)).astype(np.float32)
    np.testing.assert_array_equal(o, want)


def _dirs_at(theta, phi=0.3):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], -1)


@pytest.mark.parametrize("r", [0.2, 0.5, 1.0])
def test_ggx_normalisation(orc, r):
    """int D(h) (n.h) d omega_h = 1 over the hemisphere (wi = wo = h makes h
    the queried half vector)."""
    th = np.linspace(0.0, math.pi / 2, 200001)
    h = _dirs_at(th)
    n = np.tile([0.0, 0.0, 1.0], (th.size, 1))
    _, terms = orc.brdf_spec(n, h, h, r)
    f = terms[:, 0] * np.cos(th) * np.sin(th) * 2 * math.pi
    assert abs(np.trapezoid(f, th) - 1.0) < 1e-4


@pytest.mark.parametrize("r", [0.25, 0.35])
def test_microfacet_change_of_variables(orc, r):
    """With wo = n, int f_s (n.wi) [(n.wo)(n.h) / ((wo.h) F G)] d omega_i
    = int D (n.h) d omega_h (Jacobian 1/(4 wo.h)) over the half vectors whose
    wi is above the horizon, theta_h <= 45 deg; the GGX distribution puts
    tan^2 / (alpha^2 + tan^2) of its mass there, so the integral is
    1 / (1 + alpha^2).  A missing or doubled factor 4 fails by 4x."""
    nt, nph = 4000, 64
    th = (np.arange(nt) + 0.5) * (math.pi / 2) / nt
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    wi = _dirs_at(T.ravel(), P.ravel())
    m = wi.shape[0]
    n = np.tile([0.0, 0.0, 1.0], (m, 1))
    fs, terms = orc.brdf_spec(n, wi, n, r)
    h = wi + n
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    nh = h[:, 2]
    vh = h[:, 2]
    q = fs * wi[:, 2] * (1.0 * nh) / (vh * terms[:, 1] * terms[:, 2])
    dA = np.sin(T.ravel()) * (math.pi / 2 / nt) * (2 * math.pi / nph)
    assert abs((q * dA).sum() - 1.0 / (1.0 + r ** 4)) < 2e-4


def test_fresnel_smith_reciprocity(orc):
    rng = np.random.default_rng(4)
    n = np.tile([0.0, 0.0, 1.0], (1000, 1))
    wi = rng.standard_normal((1000, 3))
    wi[:, 2] = np.abs(wi[:, 2])
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    wo = rng.standard_normal((1000, 3))
    wo[:, 2] = np.abs(wo[:, 2])
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    r = rng.uniform(0.05, 1.0, 1000)
    a, ta = orc.brdf_spec(n, wi, wo, r)
    b, tb = orc.brdf_spec(n, wo, wi, r)
    np.testing.assert_allclose(a, b, rtol=1e-12)                   # reciprocity
    assert np.all((ta[:, 1] >= 0.04 - 1e-15) & (ta[:, 1] <= 1.0))  # F between F0 and 1
    assert np.all((ta[:, 2] > 0) & (ta[:, 2] <= 1.0))              # G in (0, 1]
    z = np.array([[0.0, 0.0, 1.0]])
    _, t = orc.brdf_spec(z, z, z, 0.5)
    assert t[0, 1] == pytest.approx(0.04, abs=1e-15)               # normal incidence: F0
    assert t[0, 2] == pytest.approx(1.0, abs=1e-15)                # G1(1) = 1
    wo_g = np.array([[1.0, 0.0, 1e-6]]) / np.linalg.norm([1.0, 0.0, 1e-6])
    wi_g = wo_g * np.array([-1.0, 1.0, 1.0])                        # h = n, wo.h = 1e-6
    _, t = orc.brdf_spec(z, wi_g, wo_g, 0.5)
    assert t[0, 1] > 0.9999                                         # grazing: F -> 1
    fs, _ = orc.brdf_spec(z, z, -z, 0.5)                            # wi = -wo: no half vector
    assert fs[0] == 0.0


def test_sh_orthonormal_and_addition_theorem(orc):
    x, wx = np.polynomial.legendre.leggauss(16)       # cos(theta) nodes: exact to degree 31
    nph = 32
    ph = np.arange(nph) * 2 * math.pi / nph
    C, P = np.meshgrid(x, ph, indexing="ij")
    s = np.sqrt(1 - C ** 2)
    w = np.stack([s * np.cos(P), s * np.sin(P), C], -1).reshape(-1, 3)
    wt = (wx[:, None] * np.full(nph, 2 * math.pi / nph)[None, :]).ravel()
    Y = orc.sh_basis(w)
    G = (Y * wt[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(9), atol=1e-12)
    for l, sl in ((0, slice(0, 1)), (1, slice(1, 4)), (2, slice(4, 9))):
        np.testing.assert_allclose((Y[:, sl] ** 2).sum(1), (2 * l + 1) / (4 * math.pi), rtol=1e-12)


def test_env_lookup(orc):
    h, w = 16, 32
    rng = np.random.default_rng(5)
    env = rng.uniform(0.5, 2.0, (h, w, 3))
    th = (np.arange(h) + 0.5) * math.pi / h
    ph = (np.arange(w) + 0.5) * 2 * math.pi / w
    T, P = np.meshgrid(th, ph, indexing="ij")
    L = orc.env_lookup(env, _dirs_at(T.ravel(), P.ravel()))
    np.testing.assert_allclose(L, env.reshape(-1, 3), rtol=1e-12)     # pixel centres
    const = np.full((h, w, 3), 1.7)
    d = rng.standard_normal((1000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    np.testing.assert_allclose(orc.env_lookup(const, d), 1.7, rtol=1e-14)
    # azimuth seam: halfway between the last column's centre and the first's
    lin = np.zeros((h, w, 3))
    lin[:, -1] = 1.0
    L = orc.env_lookup(lin, _dirs_at(np.array([th[5]]), np.array([0.0])))
    np.testing.assert_allclose(L, 0.5, rtol=1e-12)
    # poles clamp to the first / last row
    L = orc.env_lookup(env, np.array([[0, 0, 1.0], [0, 0, -1.0]]))
    assert np.all((L[0] >= env[0].min(0) - 1e-12) & (L[0] <= env[0].max(0) + 1e-12))
    assert np.all((L[1] >= env[-1].min(0) - 1e-12) & (L[1] <= env[-1].max(0) + 1e-12))


def _pbr_case(orc, n=64, K=64, seed=7):
    sc = scenes.uniform_scene(n, seed)
    nrm = scenes.shortest_axis_normals(sc["scale"], sc["quat"])
    hemi = scenes.fibonacci_hemisphere(K)
    mat = scenes.pbr_material(n, seed)
    return sc, nrm, hemi, mat


def test_pbr_diffuse_is_the_albedo(orc):
    """V = 1, unit environment, no indirect light: the diffuse part of Eq. 10
    is b (the Fibonacci heights are the midpoint rule, exact for cos), so
    c'(b) - c'(0) = b."""
    sc, nrm, hemi, mat = _pbr_case(orc)
    n, K = nrm.shape[0], hemi.shape[0]
    V = np.ones((n, K))
    env = np.ones((16, 32, 3))
    cam = np.array([3.0, -2.0, 5.0])
    m1 = dict(mat, sh=None)
    m0 = dict(m1, albedo=np.zeros_like(mat["albedo"]))
    diff = orc.pbr(sc, nrm, m1, hemi, V, env, cam) - orc.pbr(sc, nrm, m0, hemi, V, env, cam)
    np.testing.assert_allclose(diff, mat["albedo"], atol=2e-6)


def test_pbr_linear_in_light_and_visibility(orc):
    sc, nrm, hemi, mat = _pbr_case(orc)
    n, K = nrm.shape[0], hemi.shape[0]
    rng = np.random.default_rng(8)
    V = rng.uniform(0, 1, (n, K))
    env = scenes.light_envmap(3).astype(np.float64)
    cam = np.array([0.5, 4.0, 1.0])
    m = dict(mat, sh=None)
    c = orc.pbr(sc, nrm, m, hemi, V, env, cam)
    np.testing.assert_allclose(orc.pbr(sc, nrm, m, hemi, V, 2 * env, cam), 2 * c, rtol=1e-13)
    np.testing.assert_allclose(orc.pbr(sc, nrm, m, hemi, 0.5 * V, env, cam), 0.5 * c, rtol=1e-13)
    assert np.all(orc.pbr(sc, nrm, m, hemi, 0 * V, env, cam) == 0)
    assert np.all(c >= 0)
    # indirect light only, constant SH band 0: c' = s0 * Y0 * c'(V=1, unit env)
    sh = np.zeros((n, 9, 3), np.float32)
    sh[:, 0, :] = 0.3
    ci = orc.pbr(sc, nrm, dict(mat, sh=sh), hemi, 0 * V, env, cam)
    cu = orc.pbr(sc, nrm, m, hemi, np.ones((n, K)), np.ones((16, 32, 3)), cam)
    np.testing.assert_allclose(ci, float(np.float32(0.3)) * 0.5 / math.sqrt(math.pi) * cu, rtol=1e-12)
    # a negative indirect radiance is clamped to 0
    assert np.all(orc.pbr(sc, nrm, dict(mat, sh=-sh), hemi, 0 * V, env, cam) == 0)


def test_pbr_monotone_in_visibility(orc):
    """Eq. 10 with indirect light: raising any V[g, k] changes only Gaussian
    g's colour and never lowers it (non-negative BRDF, direct light and
    cosine), which is what lets a consumer of a flagged ray's visibility be
    bounded by the colours of its visibility bounds."""
    sc, nrm, hemi, mat = _pbr_case(orc)
    n, K = nrm.shape[0], hemi.shape[0]
    rng = np.random.default_rng(11)
    V = rng.uniform(0, 1, (n, K))
    env = scenes.light_envmap(3).astype(np.float64)
    cam = np.array([0.5, 4.0, 1.0])
    assert mat["sh"] is not None
    c = orc.pbr(sc, nrm, mat, hemi, V, env, cam)
    V2 = V + rng.uniform(0, 1, (n, K)) * (1 - V)
    c2 = orc.pbr(sc, nrm, mat, hemi, V2, env, cam)
    assert np.all(c2 >= c * (1 - 1e-13)) and np.any(c2 > c)
    V3 = V.copy()
    V3[3, 5] = 1.0
    c3 = orc.pbr(sc, nrm, mat, hemi, V3, env, cam)
    assert np.array_equal(np.delete(c3, 3, 0), np.delete(c, 3, 0)) and np.all(c3[3] >= c[3])


def test_pbr_view_from_behind_is_finite(orc):
    sc, nrm, hemi, mat = _pbr_case(orc, n=8)
    cam = sc["mean"][0].astype(np.float64) - 10.0 * nrm[0]   # behind Gaussian 0's surface
    c = orc.pbr(sc, nrm, mat, hemi, np.ones((8, 64)), np.ones((16, 32, 3)), cam)
    assert np.all(np.isfinite(c)) and np.all(c >= 0)
