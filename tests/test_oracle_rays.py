"""Pins of the oracle's ray sets (CPU only): the Philox4x64-10 generator
against numpy's own Philox bit generator, the float32 origin rule of the
direction set, and the environment-map sampler's distribution and geometry."""
import math

import numpy as np
import pytest

import scenes


@pytest.mark.parametrize("ctr,key", [([0, 0, 0, 0], [0, 0]), ([5, 1, 2, 3], [7, 9]),
                                     ([2 ** 64 - 2, 0, 0, 0], [2 ** 63, 12345])])
def test_philox_matches_numpy(orc, ctr, key):
    # numpy increments the counter before producing a block
    bg = np.random.Philox(counter=np.array(ctr, np.uint64), key=np.array(key, np.uint64))
    want = bg.random_raw(4)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2 ** 64
    if c[0] == 0:
        c[1] += 1
    got = orc.philox(np.array(c, np.uint64), np.array(key, np.uint64))
    np.testing.assert_array_equal(got, want)


def test_dir_rays(orc):
    sc = scenes.uniform_scene(50, 1)
    d = scenes.fibonacci_sphere(7)
    ids = np.array([0, 6, 7, 100, 349], np.int64)
    o, dd, s = orc.dir_rays(sc["mean"], d, ids, eps=1e-4)
    np.testing.assert_array_equal(s, ids // 7)
    np.testing.assert_array_equal(dd, d[ids % 7])
    want = sc["mean"][ids // 7] + (np.float32(1e-4) * d[ids % 7]).astype(np.float32)
    np.testing.assert_array_equal(o, want.astype(np.float32))


def test_fibonacci_set():
    d = scenes.fibonacci_sphere(128).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1, atol=1e-7)
    assert np.abs(d.mean(0)).max() < 0.02  # balanced over the sphere
    z = 1 - (2 * np.arange(128) + 1) / 128
    np.testing.assert_allclose(d[:, 2], z, atol=1e-7)


def test_env_rays_distribution(orc):
    env = scenes.envmap(399)
    h, w = env["radiance"].shape
    S = 512
    n = 400
    mean = np.zeros((n, 3), np.float32)
    ids = np.arange(n * S, dtype=np.int64)
    o, d, s = orc.env_rays(mean, env, 77, S, ids)
    np.testing.assert_array_equal(s, ids // S)
    np.testing.assert_allclose(np.linalg.norm(d.astype(np.float64), axis=1), 1, atol=2e-7)
    # azimuth is exact: the blend of two meridians stays between them
    phi = np.mod(np.arctan2(d[:, 1].astype(np.float64), d[:, 0]), 2 * math.pi)
    col = np.minimum((phi / (2 * math.pi / w)).astype(int), w - 1)
    wts = env["radiance"] * env["solid_angle"]
    p_col = wts.sum(0) / wts.sum()
    cnt = np.bincount(col, minlength=w)
    chi2 = np.sum((cnt - p_col * len(col)) ** 2 / (p_col * len(col)))
    assert chi2 < w + 6 * math.sqrt(2 * w)  # ~6 sigma of a chi^2 with w dof
    # polar angle: inside the pixel row up to the chord bulge of a 64-wide pixel
    theta = np.arccos(np.clip(d[:, 2].astype(np.float64), -1, 1))
    row = np.minimum((theta / (math.pi / h)).astype(int), h - 1)
    p_row = wts.sum(1) / wts.sum()
    cnt = np.bincount(row, minlength=h)
    assert np.max(np.abs(cnt / len(row) - p_row)) < 0.01
    # determinism: the same ids give the same rays
    o2, d2, _ = orc.env_rays(mean, env, 77, S, ids[:1000])
    np.testing.assert_array_equal(d2, d[:1000])
