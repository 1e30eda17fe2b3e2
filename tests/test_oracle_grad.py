"""Pins of the oracle's analytic adjoint (CPU only): closed forms for a single
Gaussian, FP64 central finite differences of the oracle forward (h = 1e-6),
and the scale invariance of the quaternion parameterisation."""
import math

import numpy as np
import pytest

from test_oracle_trace import scene


def _loss(orc, sc, ro, rd, src, w):
    return float(np.dot(w, orc.trace(sc, ro, rd, src, t_min=0.0)["T"]))


def test_closed_form_single_gaussian(orc):
    sig, o, b = 0.1, 0.7, 0.13
    sc = scene([0.02, 0, 2], sig, o=o)
    ro = np.array([[b, 0, 0.0]])
    rd = np.array([[0, 0, 1.0]])
    g = orc.trace_grad(sc, ro, rd, None, np.ones(1), with_origin=True)
    dx = b - 0.02
    ex = math.exp(-dx * dx / (2 * sig * sig))
    # T = 1 - o exp(-(b - mu_x)^2 / 2 sigma^2)
    assert g["opacity"][0] == pytest.approx(-ex, rel=1e-12)
    assert g["mean"][0, 0] == pytest.approx(-o * ex * dx / sig ** 2, rel=1e-12)
    assert g["mean"][0, 2] == pytest.approx(0.0, abs=1e-12)
    assert g["scale"][0, 0] == pytest.approx(-o * ex * dx * dx / sig ** 3, rel=1e-12)
    assert g["scale"][0, 2] == pytest.approx(0.0, abs=1e-12)
    assert g["ray_o"][0, 0] == pytest.approx(o * ex * dx / sig ** 2, rel=1e-12)
    # head-on: dT/do = -1
    g0 = orc.trace_grad(scene([0, 0, 2], sig, o=o), np.zeros((1, 3)), rd, None, np.ones(1))
    assert g0["opacity"][0] == pytest.approx(-1.0, rel=1e-14)


def _fd_case(orc, seed):
    import scenes
    sc = scenes.uniform_scene(24, seed, lo=-0.4, hi=0.4, log_scale_mean=math.log(0.12))
    sc = {k: v.astype(np.float64) for k, v in sc.items()}
    dirs = scenes.fibonacci_sphere(8)
    ids = np.arange(24 * 8, dtype=np.int64)
    ro, rd, src = orc.dir_rays(sc["mean"].astype(np.float32), dirs, ids)
    w = np.random.default_rng(seed).uniform(0, 1, ro.shape[0])
    return sc, ro.astype(np.float64), rd.astype(np.float64), src, w


@pytest.mark.parametrize("seed", [21, 22])
def test_finite_differences(orc, seed):
    sc, ro, rd, src, w = _fd_case(orc, seed)
    g = orc.trace_grad(sc, ro, rd, src, w, with_origin=True)
    base_hits = orc.trace(sc, ro, rd, src, t_min=0.0)["hits"]
    h = 1e-6
    checked = skipped = 0
    for name, shape in (("mean", 3), ("scale", 3), ("quat", 4), ("opacity", 1)):
        for j in range(24):
            for c in range(shape):
                vals = []
                same = True
                for sgn in (1, -1):
                    sc2 = {k: v.copy() for k, v in sc.items()}
                    if shape == 1:
                        sc2[name][j] += sgn * h
                    else:
                        sc2[name][j, c] += sgn * h
                    r = orc.trace(sc2, ro, rd, src, t_min=0.0)
                    same &= np.array_equal(r["hits"], base_hits)
                    vals.append(float(np.dot(w, r["T"])))
                if not same:  # the stencil crosses a truncation: excluded
                    skipped += 1
                    continue
                fd = (vals[0] - vals[1]) / (2 * h)
                an = g[name][j] if shape == 1 else g[name][j, c]
                assert an == pytest.approx(fd, rel=1e-5, abs=1e-8), (name, j, c)
                checked += 1
    assert checked > 200 and skipped < checked / 10
    # ray origins
    for r_ in range(0, ro.shape[0], 5):
        for c in range(3):
            vals = []
            for sgn in (1, -1):
                ro2 = ro.copy()
                ro2[r_, c] += sgn * h
                vals.append(_loss(orc, sc, ro2, rd, src, w))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g["ray_o"][r_, c] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_quaternion_gradient_is_tangent(orc):
    """R depends on q/|q| only, so dL/dq is orthogonal to q."""
    sc, ro, rd, src, w = _fd_case(orc, 23)
    g = orc.trace_grad(sc, ro, rd, src, w)
    dots = np.sum(g["quat"] * sc["quat"], axis=1)
    assert np.max(np.abs(dots)) < 1e-10 * max(1.0, np.abs(g["quat"]).max())
    assert np.abs(g["quat"]).max() > 1e-3


def test_snapped_rays_have_zero_gradient(orc):
    k, o = 6, 0.9  # (0.1)^6 < 1e-4: snapped to 0
    mu = np.stack([np.zeros(k), np.zeros(k), 1.0 + np.arange(k)], 1)
    sc = scene(mu, 0.05, o=o)
    g = orc.trace_grad(sc, np.zeros((1, 3)), np.array([[0, 0, 1.0]]), None, np.ones(1), t_min=1e-4)
    assert np.all(g["opacity"] == 0)
    g = orc.trace_grad(sc, np.zeros((1, 3)), np.array([[0, 0, 1.0]]), None, np.ones(1), t_min=0.0)
    np.testing.assert_allclose(g["opacity"], -(1 - o) ** (k - 1), rtol=1e-12)
