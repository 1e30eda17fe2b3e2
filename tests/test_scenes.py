"""The seeded input generators follow the stated workload recipes: value
ranges and distribution moments of the uniform and object-scale scenes, the
object-scale geometry (flattened along the surface normal, local z on the
normal), the batch sizes, the environment map's solid angles and the
direction tables.  CPU only."""
import math

import numpy as np
import pytest

import scenes


def _rot(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                     2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                     2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1).reshape(-1, 3, 3)


def test_uniform_scene_recipe():
    n = 200_000
    sc = scenes.uniform_scene(n, 1)
    for k, shape in (("mean", (n, 3)), ("scale", (n, 3)), ("quat", (n, 4)), ("opacity", (n,))):
        assert sc[k].shape == shape and sc[k].dtype == np.float32
    assert sc["mean"].min() >= -1.0 and sc["mean"].max() <= 1.0
    ls = np.log(sc["scale"].astype(np.float64))
    assert abs(ls.mean() - math.log(0.02)) < 0.01 and abs(ls.std() - 0.5) < 0.01
    np.testing.assert_allclose(np.linalg.norm(sc["quat"], axis=1), 1.0, atol=1e-6)
    # Haar-uniform rotations: each entry of R has mean 0 and variance 1/3
    R = _rot(sc["quat"])
    assert np.abs(R.mean(0)).max() < 0.01 and np.abs(R.var(0) - 1 / 3).max() < 0.01
    o = sc["opacity"].astype(np.float64)  # Beta(2,2): mean 1/2, variance 1/20
    assert abs(o.mean() - 0.5) < 0.005 and abs(o.var() - 0.05) < 0.002
    assert o.min() > 0.0 and o.max() < 1.0


def test_uniform_scene_is_seeded():
    a, b, c = scenes.uniform_scene(1000, 3), scenes.uniform_scene(1000, 3), scenes.uniform_scene(1000, 4)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(a["mean"], c["mean"])


def test_object_scene_recipe():
    n = 100_000
    sc = scenes.object_scene(n, 2)
    s = sc["scale"].astype(np.float64)
    lt = np.log(s[:, :2])
    assert abs(lt.mean() - math.log(0.01)) < 0.01 and abs(lt.std() - 0.3) < 0.01
    # the normal-axis scale is 0.1 sqrt(s_t1 s_t2) (float32 rounding apart)
    np.testing.assert_allclose(s[:, 2], 0.1 * np.sqrt(s[:, 0] * s[:, 1]), rtol=1e-6)
    o = sc["opacity"].astype(np.float64)  # Beta(5,1): mean 5/6, all below 1
    assert abs(o.mean() - 5 / 6) < 0.005 and o.max() < 1.0
    # ground plane z = -1 over [-1.5, 1.5]^2, means jittered by N(0, 0.005^2):
    # its Gaussians' local z (the flattened axis) is the plane normal
    R = _rot(sc["quat"])
    ground = (np.abs(sc["mean"][:, 2] + 1.0) < 0.03) & (np.abs(sc["mean"][:, :2]).max(1) <= 1.52)
    assert ground.mean() > 0.2
    nz = R[ground][:, :, 2]  # third column: local z in world coordinates
    assert np.quantile(np.abs(nz[:, 2]), 0.01) > 0.999
    jitter = sc["mean"][ground, 2].astype(np.float64) + 1.0
    assert abs(jitter.std() - 0.005) < 0.0005


def test_batch_sizes_recipe():
    sizes = scenes.batch_scene_sizes(16, 8_000_000, 300)
    assert len(sizes) == 16 and all(50_000 <= s <= 2_000_000 for s in sizes)
    assert abs(sum(sizes) - 8_000_000) < 0.05 * 8_000_000
    assert max(sizes) / min(sizes) > 5  # uneven


def test_envmap_recipe():
    env = scenes.envmap(399)
    assert env["radiance"].shape == (32, 64) and env["corners"].shape == (33, 65, 3)
    np.testing.assert_allclose(env["solid_angle"].sum(), 4 * math.pi, rtol=1e-12)
    z = np.log(env["radiance"]) / 1.5  # log-normal radiance, sigma 1.5
    assert abs(z.mean()) < 0.1 and abs(z.std() - 1.0) < 0.1
    np.testing.assert_allclose(np.linalg.norm(env["corners"].astype(np.float64), axis=2), 1.0, atol=1e-6)


@pytest.mark.parametrize("k", [1, 32, 128])
def test_fibonacci_sets(k):
    d = scenes.fibonacci_sphere(k).astype(np.float64)
    assert d.shape == (k, 3)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    np.testing.assert_allclose(d[:, 2], 1.0 - (2 * np.arange(k) + 1) / k, atol=1e-6)
    h = scenes.fibonacci_hemisphere(k).astype(np.float64)
    assert np.all(h[:, 2] > 0)
    np.testing.assert_allclose(h[:, 2], 1.0 - (np.arange(k) + 0.5) / k, atol=1e-6)


def test_stratified_ray_ids():
    for n, m in ((1000, 1000), (1000, 7), (256_000_000, 1 << 20), (10, 3)):
        ids = scenes.stratified_ray_ids(n, m, 5)
        assert ids.dtype == np.int64 and ids.shape == (m,)
        assert np.all(np.diff(ids) > 0) and ids[0] >= 0 and ids[-1] < n
        j = np.arange(m)
        assert np.all(ids >= (j * n) // m) and np.all(ids < ((j + 1) * n) // m)
    assert scenes.stratified_ray_ids(5, 0, 1).size == 0
    np.testing.assert_array_equal(scenes.stratified_ray_ids(1 << 20, 1000, 9),
                                  scenes.stratified_ray_ids(1 << 20, 1000, 9))
