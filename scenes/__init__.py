"""Seeded synthetic inputs for point-based Gaussian ray tracing.

This module only *draws* inputs: Gaussian parameters {mu, s, q, o}, direction
tables, environment-map radiance and loss weights.  It contains none of the
visibility arithmetic (no intersection, no transmittance, no BVH), so both the
FP64 oracle and the CUDA path can consume the same arrays without sharing any
of the method's code.

Conventions (shared by every consumer, stated once here):
  * mean[N,3], scale[N,3] (linear standard deviations along the local axes),
    quat[N,4] as (w, x, y, z) (not necessarily unit length), opacity[N] in [0,1).
    All float32, C-contiguous.
  * The local axes of Gaussian i are the columns of R(q_i); Sigma = R S S^T R^T
    (Sec. 3.1 parameterisation of the covariance by q and s).
  * Direction tables are float32 [K,3], computed in float64 and rounded once.

Workload recipes (Sec. 4.2 visibility precompute, Sec. 5.1 N_s directions):
  uniform_scene   -- means U[-1,1]^3, log-scales N(log 0.02, 0.5), Haar-uniform
                     rotations, opacity Beta(2,2).  4,096 Gaussians x 32
                     directions is the small parity workload.
  object_scene    -- Gaussians on the surfaces of 2 spheres, a torus, a box and a
                     ground plane, flattened along the surface normal, opacity
                     Beta(5,1); 300k or 2M Gaussians x 128 directions.
  batch_scenes    -- 16 uniform scenes of uneven size (log-uniform counts).
  envmap          -- 64x32 equirectangular log-normal radiance map (sigma 1.5)
                     and its pixel-corner direction table.
  composed_objects -- 4 object-scale scenes (125k each) placed as 16 instances
                     by seeded rigid maps (Sec. 4.3 composition).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "fibonacci_sphere", "rotated_fibonacci", "uniform_scene", "object_scene",
    "batch_scene_sizes", "batch_scenes", "envmap", "loss_weights", "sample_ray_ids",
    "batch_object_scenes", "composed_objects", "fibonacci_hemisphere", "shortest_axis_normals",
    "pbr_material", "light_envmap",
]


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def fibonacci_sphere(k: int) -> np.ndarray:
    """K directions on the full unit sphere by Fibonacci (golden-angle) spacing.

    z_k = 1 - (2k+1)/K, phi_k = k * pi * (3 - sqrt 5); evaluated in float64,
    normalised, rounded to float32 once.  Sec. 3.3 samples the incident
    directions of each Gaussian with a Fibonacci lattice; here the full sphere
    is used.
    """
    kk = np.arange(k, dtype=np.float64)
    z = 1.0 - (2.0 * kk + 1.0) / k
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = kk * math.pi * (3.0 - math.sqrt(5.0))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return _f32(d)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def rotated_fibonacci(k: int, seed: int) -> np.ndarray:
    """The Fibonacci set under one seeded random rotation (held-out directions)."""
    kk = np.arange(k, dtype=np.float64)
    z = 1.0 - (2.0 * kk + 1.0) / k
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = kk * math.pi * (3.0 - math.sqrt(5.0))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    rot = _random_rotation(np.random.default_rng(seed))
    d = d @ rot.T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return _f32(d)


def uniform_scene(n: int, seed: int, lo: float = -1.0, hi: float = 1.0,
                  offset=(0.0, 0.0, 0.0), log_scale_mean: float = math.log(0.02),
                  log_scale_std: float = 0.5) -> dict:
    """Gaussians with means U[lo,hi]^3 (+offset), log-scales N(m, sd) per axis,
    Haar-uniform rotations (normalised N(0,1)^4) and opacity Beta(2,2).

    Draw order from numpy's PCG64 generator: means, log-scales, quaternions,
    opacity.
    """
    rng = np.random.default_rng(seed)
    mean = rng.uniform(lo, hi, size=(n, 3)) + np.asarray(offset, dtype=np.float64)
    log_s = rng.normal(log_scale_mean, log_scale_std, size=(n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    o = rng.beta(2.0, 2.0, size=n)
    return {"mean": _f32(mean), "scale": _f32(np.exp(log_s)), "quat": _f32(q),
            "opacity": _f32(o)}


def _frame_to_quat(t1, t2, nrm):
    """Unit quaternions (w,x,y,z) of rotations whose columns are (t1, t2, n)."""
    from scipy.spatial.transform import Rotation
    mats = np.stack([t1, t2, nrm], axis=2)  # columns
    xyzw = Rotation.from_matrix(mats).as_quat()
    return np.concatenate([xyzw[:, 3:4], xyzw[:, 0:3]], axis=1)


def object_scene(n: int, seed: int) -> dict:
    """Object-scale scene: Gaussians on 2 spheres (r~U[0.2,0.5]), a torus
    (R=0.4, r=0.1, axis +z), an axis-aligned box (sides U[0.3,0.6]) and the
    ground plane z=-1 over [-1.5,1.5]^2.  Object centres U[-0.6,0.6]^2 x
    U[-0.5,0.3].  Points are area-proportional over all surfaces; means are the
    surface point plus N(0, 0.005^2) isotropic jitter; tangent log-scales
    N(log 0.01, 0.3); normal scale 0.1*sqrt(s_t1*s_t2); local z maps to the
    surface normal with a uniform random twist; opacity Beta(5,1).
    """
    rng = np.random.default_rng(seed)
    centres = np.stack([rng.uniform(-0.6, 0.6, 4), rng.uniform(-0.6, 0.6, 4),
                        rng.uniform(-0.5, 0.3, 4)], axis=1)
    r_sph = rng.uniform(0.2, 0.5, 2)
    box = rng.uniform(0.3, 0.6, 3)
    R_t, r_t = 0.4, 0.1
    areas = np.array([
        4 * math.pi * r_sph[0] ** 2, 4 * math.pi * r_sph[1] ** 2,
        4 * math.pi ** 2 * R_t * r_t,
        2 * (box[0] * box[1] + box[1] * box[2] + box[0] * box[2]),
        9.0,
    ])
    counts = rng.multinomial(n, areas / areas.sum())
    pts, nrms = [], []
    # spheres
    for s in range(2):
        v = rng.standard_normal((counts[s], 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        pts.append(centres[s] + r_sph[s] * v)
        nrms.append(v)
    # torus, rejection-sampled so the density is uniform in area
    m = counts[2]
    uu = np.empty(0)
    vv = np.empty(0)
    while uu.size < m:
        u = rng.uniform(0, 2 * math.pi, 2 * m + 16)
        v = rng.uniform(0, 2 * math.pi, 2 * m + 16)
        acc = rng.uniform(0, 1, 2 * m + 16) < (R_t + r_t * np.cos(v)) / (R_t + r_t)
        uu = np.concatenate([uu, u[acc]])
        vv = np.concatenate([vv, v[acc]])
    uu, vv = uu[:m], vv[:m]
    ring = R_t + r_t * np.cos(vv)
    pts.append(centres[2] + np.stack([ring * np.cos(uu), ring * np.sin(uu), r_t * np.sin(vv)], 1))
    nrms.append(np.stack([np.cos(vv) * np.cos(uu), np.cos(vv) * np.sin(uu), np.sin(vv)], 1))
    # box: pick a face by area, then a uniform point on it
    m = counts[3]
    a, b, c = box
    face_area = np.array([b * c, b * c, a * c, a * c, a * b, a * b])
    face = rng.choice(6, size=m, p=face_area / face_area.sum())
    uv = rng.uniform(-0.5, 0.5, size=(m, 2))
    p = np.zeros((m, 3))
    nr = np.zeros((m, 3))
    half = box / 2
    for f in range(6):
        sel = face == f
        ax = f // 2
        sign = 1.0 if f % 2 == 0 else -1.0
        others = [i for i in range(3) if i != ax]
        p[sel, ax] = sign * half[ax]
        p[sel, others[0]] = uv[sel, 0] * box[others[0]]
        p[sel, others[1]] = uv[sel, 1] * box[others[1]]
        nr[sel, ax] = sign
    pts.append(centres[3] + p)
    nrms.append(nr)
    # ground plane
    m = counts[4]
    xy = rng.uniform(-1.5, 1.5, size=(m, 2))
    pts.append(np.concatenate([xy, np.full((m, 1), -1.0)], 1))
    nrms.append(np.tile(np.array([[0.0, 0.0, 1.0]]), (m, 1)))

    pts = np.concatenate(pts)
    nrm = np.concatenate(nrms)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    mean = pts + rng.normal(0.0, 0.005, size=pts.shape)
    st = np.exp(rng.normal(math.log(0.01), 0.3, size=(n, 2)))
    sn = 0.1 * np.sqrt(st[:, 0] * st[:, 1])
    # tangent frame: any unit vector orthogonal to n, then a uniform twist
    helper = np.where(np.abs(nrm[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    t1 = np.cross(nrm, helper)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(nrm, t1)
    psi = rng.uniform(0, 2 * math.pi, size=(n, 1))
    a1 = np.cos(psi) * t1 + np.sin(psi) * t2
    a2 = np.cross(nrm, a1)
    quat = _frame_to_quat(a1, a2, nrm)
    o = rng.beta(5.0, 1.0, size=n)
    # Beta(5,1) can round to 1.0 in float32; opacity must stay below 1.
    o = np.minimum(o, 1.0 - 2.0 ** -20)
    return {"mean": _f32(mean), "scale": _f32(np.stack([st[:, 0], st[:, 1], sn], 1)),
            "quat": _f32(quat), "opacity": _f32(o)}


def batch_scene_sizes(n_scenes: int = 16, total: int = 8_000_000, seed: int = 300,
                      lo: int = 50_000, hi: int = 2_000_000) -> list[int]:
    """Uneven scene sizes: log-uniform in [lo, hi], rescaled so the sum is about
    `total` (each size kept in [lo, hi])."""
    rng = np.random.default_rng(seed)
    c = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_scenes))
    c = c * (total / c.sum())
    return [int(x) for x in np.clip(np.round(c), lo, hi)]


def batch_scenes(sizes, seed_base: int = 300) -> list[dict]:
    """One uniform scene per size, seed seed_base+s, placed in a seeded box:
    side U[1.5, 2.5], translated by an offset U[-4,4]^3."""
    out = []
    for s, n in enumerate(sizes):
        rng = np.random.default_rng(seed_base + 1000 + s)
        side = rng.uniform(1.5, 2.5)
        off = rng.uniform(-4.0, 4.0, size=3)
        out.append(uniform_scene(int(n), seed_base + s, lo=-side / 2, hi=side / 2, offset=off))
    return out


def fibonacci_hemisphere(k: int) -> np.ndarray:
    """k local directions on the hemisphere z > 0 (Fibonacci sampling):
    z_i = 1 - (i + 1/2)/k, phi_i = i*pi*(3 - sqrt(5)); float64, rounded once."""
    i = np.arange(k, dtype=np.float64)
    z = 1.0 - (i + 0.5) / k
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return _f32(np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1))


def shortest_axis_normals(scale, quat) -> np.ndarray:
    """Per-Gaussian normal: the rotation's column of the smallest scale (the
    flattened axis), float64 then rounded once."""
    q = np.asarray(quat, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)], 1)
    ax = np.argmin(np.asarray(scale), axis=1)
    return _f32(R[np.arange(len(ax)), :, ax])


def pbr_material(n: int, seed: int, with_sh: bool = True) -> dict:
    """Per-Gaussian BRDF and indirect light: albedo U[0,1]^3, roughness
    U[0,1], SH coefficients (9 per channel) N(0, 0.1^2) with the constant term
    U[0, 0.5] (float32)."""
    rng = np.random.default_rng(seed)
    out = {"albedo": _f32(rng.uniform(0.0, 1.0, (n, 3))), "roughness": _f32(rng.uniform(0.0, 1.0, n)),
           "sh": None}
    if with_sh:
        sh = rng.normal(0.0, 0.1, (n, 9, 3))
        sh[:, 0, :] = rng.uniform(0.0, 0.5, (n, 3))
        out["sh"] = _f32(sh)
    return out


def light_envmap(seed: int = 499, h: int = 16, w: int = 32, sigma: float = 1.0) -> np.ndarray:
    """The direct light of the PBR colour: an h x w RGB equirectangular map,
    log-normal radiance exp(sigma z), z ~ N(0,1) per pixel and channel
    (float32, [h, w, 3])."""
    rng = np.random.default_rng(seed)
    return _f32(np.exp(sigma * rng.standard_normal((h, w, 3))))


def batch_object_scenes(sizes, seed_base: int = 300) -> list[dict]:
    """One object-scale scene (``object_scene``) per size, seed seed_base+s,
    translated by a seeded offset U[-4,4]^3."""
    out = []
    for s, n in enumerate(sizes):
        rng = np.random.default_rng(seed_base + 2000 + s)
        off = rng.uniform(-4.0, 4.0, size=3)
        sc = object_scene(int(n), seed_base + s)
        sc["mean"] = _f32(sc["mean"].astype(np.float64) + off)
        out.append(sc)
    return out


def composed_objects(seed: int = 60, n_obj: int = 4, n_inst: int = 16, per_obj: int = 125_000):
    """Objects (``object_scene``, seeds seed..seed+n_obj-1) and n_inst seeded
    rigid maps [R | t] (float32 3x4): R uniform over rotations, t U[-3,3]^3,
    so instances overlap.  Instance j places object j mod n_obj.  Returns
    (objects, pick, xforms)."""
    from scipy.spatial.transform import Rotation
    objs = [object_scene(per_obj, seed + i) for i in range(n_obj)]
    rng = np.random.default_rng(3)
    xf = []
    for _ in range(n_inst):
        R = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        xf.append(np.concatenate([R, rng.uniform(-3, 3, (3, 1))], 1).astype(np.float32))
    return objs, [i % n_obj for i in range(n_inst)], xf


def envmap(seed: int = 399, h: int = 32, w: int = 64, sigma: float = 1.5) -> dict:
    """Equirectangular HDR environment map with log-normal radiance.

    radiance[h, w] = exp(sigma * z), z ~ N(0,1) (float64).  Row i spans polar
    angles [i*pi/h, (i+1)*pi/h] from +z; column j spans azimuths
    [2*pi*j/w, 2*pi*(j+1)/w].  `corners[h+1, w+1, 3]` (float32) are the unit
    directions of the pixel corners and `z_edges[h+1]` (float64) the cosines of
    the row edges; `solid_angle[h, w]` (float64) is each pixel's solid angle.
    """
    rng = np.random.default_rng(seed)
    rad = np.exp(sigma * rng.standard_normal((h, w)))
    theta = np.arange(h + 1, dtype=np.float64) * math.pi / h
    phi = np.arange(w + 1, dtype=np.float64) * 2.0 * math.pi / w
    st, ct = np.sin(theta)[:, None], np.cos(theta)[:, None]
    corners = np.stack([st * np.cos(phi)[None, :], st * np.sin(phi)[None, :],
                        np.broadcast_to(ct, (h + 1, w + 1))], axis=2)
    z_edges = np.cos(theta)
    solid = (z_edges[:-1] - z_edges[1:])[:, None] * np.full((1, w), 2.0 * math.pi / w)
    return {"radiance": rad, "corners": _f32(corners), "z_edges": z_edges,
            "solid_angle": solid}


def loss_weights(n_rays: int, seed: int) -> np.ndarray:
    """w_r ~ U(0,1), float32: weights of the loss L = sum_r w_r T_r."""
    return _f32(np.random.default_rng(seed).uniform(0.0, 1.0, size=n_rays))


def stratified_ray_ids(n_rays: int, m: int, seed: int) -> np.ndarray:
    """A seeded sorted sample of m distinct ray ids spread over the whole of
    [0, n_rays): the range is cut into m strata [floor(j n/m), floor((j+1) n/m))
    and one id is drawn uniformly from each (int64).  O(m), for samples too
    large for sample_ray_ids."""
    m = min(m, n_rays)
    if m <= 0:
        return np.zeros(0, np.int64)
    j = np.arange(m + 1, dtype=np.int64)
    edges = (j * n_rays) // m
    lo, width = edges[:-1], edges[1:] - edges[:-1]
    u = np.random.default_rng(seed).random(m)
    return lo + np.minimum((u * width).astype(np.int64), width - 1)


def sample_ray_ids(n_rays: int, m: int, seed: int) -> np.ndarray:
    """A seeded sorted sample of m distinct ray ids in [0, n_rays) (int64)."""
    rng = np.random.default_rng(seed)
    m = min(m, n_rays)
    return np.sort(rng.choice(n_rays, size=m, replace=False)).astype(np.int64)
