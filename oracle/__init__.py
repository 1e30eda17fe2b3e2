"""FP64 CPU oracle for point-based Gaussian ray tracing -- TEST INFRASTRUCTURE.

Only tests/, the CUDA-path smoke check (``__graft_entry__.smoke``) and the CPU
baseline of ``bench.py`` may import this package.  It is a plain, slow,
obviously-correct restatement of the method (see ``rt_oracle.c`` for the
passage each function follows) and shares no code with the CUDA library.

``build()`` compiles ``rt_oracle.c`` with gcc (OpenMP, ``-ffp-contract=off``)
into ``oracle/_build/``; the numpy wrappers below call it through ctypes.

Parity status: every function here is pinned by tests/test_oracle_*.py
(closed forms, invariants, brute force, an independent numpy formulation,
finite differences, library routines), except the surrogate's visibility MAE,
which has no reference value (parity unpinned: the bar is MAE <= 0.01 against
the tracer).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "rt_oracle.c")
_lock = threading.Lock()
_lib = None

# band flag bits of oracle_trace
FLAG_M2, FLAG_ALPHA, FLAG_T, FLAG_TMIN = 1, 2, 4, 8
# default band widths: m^2 within 1e-4 of K^2 (FP32 m^2 error of flattened
# Gaussians seen from far away), alpha within 1e-6 of the cutoff, t* within
# 1e-6 of 0, T within 1e-7 of T_min.
DEFAULT_BANDS = dict(band_m2=1e-4, band_alpha=1e-6, band_t=1e-6, band_T=1e-7)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-D_GNU_SOURCE", "-O2", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = C.CDLL(path)
        P = C.c_void_p
        i64, i32, u32, f32, f64 = C.c_int64, C.c_int32, C.c_uint32, C.c_float, C.c_double
        sig = {
            "oracle_rotation": (None, [P, P]),
            "oracle_trace": (None, [i64, P, P, P, P, i64, P, P, P, f64, f64, f64,
                                    f64, f64, f64, f64, P, P, P, P, P, P, P]),
            "oracle_trace_hits": (None, [i64, P, P, P, P, i64, P, P, P, f64, f64, i32, P, P]),
            "oracle_trace_grad": (None, [i64, P, P, P, P, i64, P, P, P, f64, f64, f64,
                                         P, P, P, P, P, P]),
            "oracle_dir_rays": (None, [i64, P, i32, P, f32, P, i64, P, P, P]),
            "oracle_philox": (None, [P, P, P]),
            "oracle_env_rays": (None, [i64, P, i32, i32, P, P, P, u32, i32, f32, P, i64, P, P, P]),
            "oracle_morton": (None, [i64, P, P, P, P]),
            "oracle_lbvh": (None, [i64, P, P, P, P, P]),
            "oracle_leaf_boxes": (None, [i64, P, P, P, P, f64, f64, i32, P]),
            "oracle_bvh_create": (P, [i64, P, P, P, P, f64, f64]),
            "oracle_bvh_destroy": (None, [P]),
            "oracle_bvh_trace": (None, [P, i64, P, P, P, f64, f64, f64, f64, f64, P, P, P, P, P, P, P]),
            "oracle_bvh_trace_dirs": (None, [P, i32, P, f32, P, i64, f64, f64, f64, f64, f64,
                                             P, P, P, P, P, P, P]),
            "oracle_hemi_rays": (None, [i64, P, P, i32, P, f32, P, i64, P, P, P]),
            "oracle_brdf_spec": (None, [i64, P, P, P, P, P, P]),
            "oracle_sh_basis": (None, [i64, P, P]),
            "oracle_env_lookup": (None, [i32, i32, P, i64, P, P]),
            "oracle_pbr": (None, [i64, P, P, P, P, P, i32, P, P, i32, i32, P, P, P]),
            "oracle_bf16_round": (None, [i64, P, P]),
            "oracle_mlp_encode": (None, [i64, P, P, P, P, P]),
            "oracle_mlp_nparam": (i64, []),
            "oracle_mlp_set_bf16": (None, [i32]),
            "oracle_mlp_forward": (None, [P, i64, P, P, P]),
            "oracle_mlp_loss_grad": (f64, [P, i64, P, P, f64, P]),
            "oracle_mlp_visibility": (None, [P, i64, P, f64, P]),
            "oracle_adam_step": (None, [i64, P, P, P, P, i64, f64, f64, f64, f64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(np.asarray(a, dtype=dt))


def _scene(sc):
    """Scene arrays widened to float64 (exact for float32 inputs)."""
    return (_c(sc["mean"], np.float64), _c(sc["scale"], np.float64),
            _c(sc["quat"], np.float64), _c(sc["opacity"], np.float64))


def rotation(q) -> np.ndarray:
    q = _c(q, np.float64)
    R = np.empty(9, np.float64)
    _load().oracle_rotation(_p(q), _p(R))
    return R.reshape(3, 3)


def trace(scene, ray_o, ray_d, ray_src=None, k_sigma=3.0, alpha_min=1.0 / 255.0,
          t_min=1e-4, bands=None):
    """Brute-force visibility.  Returns dict(T, T_exact, hits, flags, T_lo,
    T_hi, n_border): T_lo / T_hi bound the unsnapped product over any choice
    of the flagged (borderline) candidates; both equal T_exact when no
    candidate set a band bit; n_border counts those candidates."""
    mean, scale, quat, opac = _scene(scene)
    ray_o = _c(ray_o, np.float64).reshape(-1, 3)
    ray_d = _c(ray_d, np.float64).reshape(-1, 3)
    R = ray_o.shape[0]
    src = None if ray_src is None else _c(ray_src, np.int32)
    b = dict(DEFAULT_BANDS)
    if bands:
        b.update(bands)
    T = np.empty(R, np.float64)
    Te = np.empty(R, np.float64)
    hits = np.empty(R, np.int32)
    flags = np.empty(R, np.uint32)
    lo, hi = np.empty(R, np.float64), np.empty(R, np.float64)
    nb = np.empty(R, np.int32)
    _load().oracle_trace(mean.shape[0], _p(mean), _p(scale), _p(quat), _p(opac), R, _p(ray_o),
                         _p(ray_d), _p(src), k_sigma, alpha_min, t_min, b["band_m2"],
                         b["band_alpha"], b["band_t"], b["band_T"], _p(T), _p(Te), _p(hits),
                         _p(flags), _p(lo), _p(hi), _p(nb))
    return {"T": T, "T_exact": Te, "hits": hits, "flags": flags, "T_lo": lo, "T_hi": hi, "n_border": nb}


def trace_hits(scene, ray_o, ray_d, ray_src=None, k_sigma=3.0, alpha_min=1.0 / 255.0, cap=256):
    """Accepted Gaussian ids per ray: (ids[R, cap] int32, count[R] int32)."""
    mean, scale, quat, opac = _scene(scene)
    ray_o = _c(ray_o, np.float64).reshape(-1, 3)
    ray_d = _c(ray_d, np.float64).reshape(-1, 3)
    R = ray_o.shape[0]
    src = None if ray_src is None else _c(ray_src, np.int32)
    ids = np.full((R, cap), -1, np.int32)
    cnt = np.empty(R, np.int32)
    _load().oracle_trace_hits(mean.shape[0], _p(mean), _p(scale), _p(quat), _p(opac), R,
                              _p(ray_o), _p(ray_d), _p(src), k_sigma, alpha_min, cap, _p(ids),
                              _p(cnt))
    return ids, cnt


def trace_grad(scene, ray_o, ray_d, ray_src, dL_dT, k_sigma=3.0, alpha_min=1.0 / 255.0,
               t_min=0.0, with_origin=False):
    """Analytic FP64 gradient of L = sum_r dL_dT[r] T[r]."""
    mean, scale, quat, opac = _scene(scene)
    ray_o = _c(ray_o, np.float64).reshape(-1, 3)
    ray_d = _c(ray_d, np.float64).reshape(-1, 3)
    R = ray_o.shape[0]
    n = mean.shape[0]
    src = None if ray_src is None else _c(ray_src, np.int32)
    g = _c(dL_dT, np.float64)
    out = {"mean": np.empty((n, 3)), "scale": np.empty((n, 3)), "quat": np.empty((n, 4)),
           "opacity": np.empty(n)}
    dro = np.empty((R, 3)) if with_origin else None
    _load().oracle_trace_grad(n, _p(mean), _p(scale), _p(quat), _p(opac), R, _p(ray_o),
                              _p(ray_d), _p(src), k_sigma, alpha_min, t_min, _p(g),
                              _p(out["mean"]), _p(out["scale"]), _p(out["quat"]),
                              _p(out["opacity"]), _p(dro))
    if with_origin:
        out["ray_o"] = dro
    return out


def dir_rays(mean, dirs, ids, eps=1e-4):
    """Float32 rays (o, d, src) for ray ids r = g*K + k (Sec. 4.2 ray set)."""
    mean = _c(mean, np.float32)
    dirs = _c(dirs, np.float32)
    ids = _c(ids, np.int64)
    m = ids.shape[0]
    o = np.empty((m, 3), np.float32)
    d = np.empty((m, 3), np.float32)
    s = np.empty(m, np.int32)
    _load().oracle_dir_rays(mean.shape[0], _p(mean), dirs.shape[0], _p(dirs), eps, _p(ids), m,
                            _p(o), _p(d), _p(s))
    return o, d, s


def philox(counter, key) -> np.ndarray:
    """Philox4x64-10 block: 4 uint64 outputs of counter[4], key[2]."""
    c = _c(counter, np.uint64)
    k = _c(key, np.uint64)
    out = np.empty(4, np.uint64)
    _load().oracle_philox(_p(c), _p(k), _p(out))
    return out


def env_rays(mean, env, seed, samples_per_gaussian, ids, eps=1e-4):
    """Float32 shadow rays importance-sampled from env (scenes.envmap dict)."""
    mean = _c(mean, np.float32)
    rad = _c(env["radiance"], np.float64)
    sa = _c(env["solid_angle"], np.float64)
    cor = _c(env["corners"], np.float32)
    h, w = rad.shape
    ids = _c(ids, np.int64)
    m = ids.shape[0]
    o = np.empty((m, 3), np.float32)
    d = np.empty((m, 3), np.float32)
    s = np.empty(m, np.int32)
    _load().oracle_env_rays(mean.shape[0], _p(mean), h, w, _p(rad), _p(sa), _p(cor), seed,
                            samples_per_gaussian, eps, _p(ids), m, _p(o), _p(d), _p(s))
    return o, d, s


def morton(mean):
    mean = _c(mean, np.float32)
    n = mean.shape[0]
    codes = np.empty(n, np.uint32)
    lo = np.empty(3, np.float32)
    hi = np.empty(3, np.float32)
    _load().oracle_morton(n, _p(mean), _p(codes), _p(lo), _p(hi))
    return codes, lo, hi


def lbvh(mean):
    """CPU twin of the LBVH topology: dict(keys, left, right, parent)."""
    mean = _c(mean, np.float32)
    n = mean.shape[0]
    keys = np.empty(max(n, 1), np.uint64)[:n]
    left = np.empty(max(n - 1, 1), np.int32)[:max(n - 1, 0)]
    right = np.empty(max(n - 1, 1), np.int32)[:max(n - 1, 0)]
    parent = np.empty(max(2 * n - 1, 1), np.int32)[:max(2 * n - 1, 0)]
    _load().oracle_lbvh(n, _p(mean), _p(keys), _p(left), _p(right), _p(parent))
    return {"keys": keys, "left": left, "right": right, "parent": parent}


def leaf_boxes(scene, k_sigma=3.0, alpha_min=1.0 / 255.0, box_mode=0):
    mean, scale, quat, opac = _scene(scene)
    n = mean.shape[0]
    box = np.empty((n, 6), np.float64)
    _load().oracle_leaf_boxes(n, _p(mean), _p(scale), _p(quat), _p(opac), k_sigma, alpha_min,
                              box_mode, _p(box))
    return box


class BvhTracer:
    """The brute-force visibility of ``trace`` found through the LBVH twin
    (``rt_oracle.c``, oracle_bvh_*): same T up to the order of the product,
    flags a subset of ``trace``'s, and a ray flagged only by ``trace`` has
    T = 0 (the walk stops once T is certain to snap to 0).  Fast enough to
    cover every ray of the 300k-Gaussian scene on the host cores."""

    def __init__(self, scene, k_sigma=3.0, bands=None):
        self._arrs = _scene(scene)
        mean, scale, quat, opac = self._arrs
        self.n = mean.shape[0]
        self.bands = dict(DEFAULT_BANDS)
        if bands:
            self.bands.update(bands)
        self._h = _load().oracle_bvh_create(self.n, _p(mean), _p(scale), _p(quat), _p(opac), k_sigma,
                                            self.bands["band_m2"])
        if not self._h:
            raise MemoryError("oracle_bvh_create")

    def close(self):
        if self._h:
            _load().oracle_bvh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, m):
        return {"T": np.empty(m), "T_exact": np.empty(m), "hits": np.empty(m, np.int32),
                "flags": np.empty(m, np.uint32), "counts": np.zeros(2, np.int64),
                "T_lo": np.empty(m), "T_hi": np.empty(m)}

    def trace(self, ray_o, ray_d, ray_src=None, alpha_min=1.0 / 255.0, t_min=1e-4):
        ray_o = _c(ray_o, np.float64).reshape(-1, 3)
        ray_d = _c(ray_d, np.float64).reshape(-1, 3)
        src = None if ray_src is None else _c(ray_src, np.int32)
        m = ray_o.shape[0]
        o, b = self._out(m), self.bands
        _load().oracle_bvh_trace(self._h, m, _p(ray_o), _p(ray_d), _p(src), alpha_min, t_min,
                                 b["band_alpha"], b["band_t"], b["band_T"], _p(o["T"]), _p(o["T_exact"]),
                                 _p(o["hits"]), _p(o["flags"]), _p(o["counts"]), _p(o["T_lo"]),
                                 _p(o["T_hi"]))
        return o

    def trace_dirs(self, dirs, ids=None, eps=1e-4, alpha_min=1.0 / 255.0, t_min=1e-4):
        """Rays r = g*K + k of the direction set (``dir_rays``); ids=None
        traces all n*K in id order."""
        dirs = _c(dirs, np.float32)
        K = dirs.shape[0]
        ids = None if ids is None else _c(ids, np.int64)
        m = self.n * K if ids is None else ids.shape[0]
        o, b = self._out(m), self.bands
        _load().oracle_bvh_trace_dirs(self._h, K, _p(dirs), eps, _p(ids), m, alpha_min, t_min,
                                      b["band_alpha"], b["band_t"], b["band_T"], _p(o["T"]),
                                      _p(o["T_exact"]), _p(o["hits"]), _p(o["flags"]), _p(o["counts"]),
                                      _p(o["T_lo"]), _p(o["T_hi"]))
        return o


def hemi_rays(mean, normals, hemi, ids, eps=1e-4):
    """Float32 rays (o, d, src) of the hemisphere sets about each Gaussian's
    normal: ray r = g*K + k uses the local direction hemi[k] (Sec. 3.3)."""
    mean = _c(mean, np.float32)
    normals = _c(normals, np.float32)
    hemi = _c(hemi, np.float32)
    ids = _c(ids, np.int64)
    m = ids.shape[0]
    o = np.empty((m, 3), np.float32)
    d = np.empty((m, 3), np.float32)
    s = np.empty(m, np.int32)
    _load().oracle_hemi_rays(mean.shape[0], _p(mean), _p(normals), hemi.shape[0], _p(hemi), eps, _p(ids), m,
                             _p(o), _p(d), _p(s))
    return o, d, s


def brdf_spec(n, wi, wo, rough):
    """Specular term f_s of Eq. 9 and its (D, F, G) for unit vectors (FP64)."""
    n = _c(n, np.float64).reshape(-1, 3)
    wi = _c(wi, np.float64).reshape(-1, 3)
    wo = _c(wo, np.float64).reshape(-1, 3)
    rough = _c(np.broadcast_to(rough, (n.shape[0],)), np.float64)
    fs = np.empty(n.shape[0])
    terms = np.empty((n.shape[0], 3))
    _load().oracle_brdf_spec(n.shape[0], _p(n), _p(wi), _p(wo), _p(rough), _p(fs), _p(terms))
    return fs, terms


def sh_basis(w):
    w = _c(w, np.float64).reshape(-1, 3)
    Y = np.empty((w.shape[0], 9))
    _load().oracle_sh_basis(w.shape[0], _p(w), _p(Y))
    return Y


def env_lookup(env_rgb, dirs):
    """Bilinear lookup of an equirectangular RGB map env_rgb[h, w, 3]."""
    env = _c(env_rgb, np.float64)
    h, w = env.shape[:2]
    dirs = _c(dirs, np.float64).reshape(-1, 3)
    L = np.empty((dirs.shape[0], 3))
    _load().oracle_env_lookup(h, w, _p(env), dirs.shape[0], _p(dirs), _p(L))
    return L


def pbr(scene, normals, material, hemi, V, env_rgb, cam):
    """Per-Gaussian PBR colour of Eq. 10 from the visibility V[n, K] of the
    hemisphere rays; material = dict(albedo[n,3], roughness[n], sh[n,9,3] or
    None).  Returns rgb[n, 3] (FP64)."""
    mean = _c(scene["mean"], np.float32)
    n = mean.shape[0]
    normals = _c(normals, np.float32)
    alb = _c(material["albedo"], np.float32)
    rough = _c(material["roughness"], np.float32)
    sh = None if material.get("sh") is None else _c(material["sh"], np.float32)
    hemi = _c(hemi, np.float32)
    V = _c(V, np.float64).reshape(n, hemi.shape[0])
    env = _c(env_rgb, np.float64)
    cam = _c(cam, np.float64)
    rgb = np.empty((n, 3))
    _load().oracle_pbr(n, _p(mean), _p(normals), _p(alb), _p(rough), _p(sh), hemi.shape[0], _p(hemi), _p(V),
                       env.shape[0], env.shape[1], _p(env), _p(cam), _p(rgb))
    return rgb


def _rows(R, v, c):
    """((R[0,c] v0 + R[1,c] v1) + R[2,c] v2) in float32, each operation rounded."""
    return (R[0, c] * v[:, 0] + R[1, c] * v[:, 1]) + R[2, c] * v[:, 2]


def instance_world_means(objects, xforms):
    """World means of a composed scene's Gaussians in scene order (instance
    by instance, each object's Gaussians in their original order): instance
    j places objects[j] by xforms[j] = [R | t] (3x4, world = R local + t),
    m_c = fl(((R_c0 x + R_c1 y) + R_c2 z) + t_c) in float32."""
    out = []
    for sc, xf in zip(objects, xforms):
        X = np.asarray(xf, np.float32).reshape(3, 4)
        R, t = X[:, :3], X[:, 3]
        mu = _c(sc["mean"], np.float32)
        out.append(np.stack([((R[c, 0] * mu[:, 0] + R[c, 1] * mu[:, 1]) + R[c, 2] * mu[:, 2]) + t[c]
                             for c in range(3)], 1).astype(np.float32))
    return np.concatenate(out)


def instance_rows(objects, rows):
    """(instance, local index) of scene rows (scene order as above)."""
    base = np.cumsum([0] + [sc["mean"].shape[0] for sc in objects])
    rows = np.asarray(rows, np.int64)
    inst = np.searchsorted(base, rows, side="right") - 1
    return inst.astype(np.int32), (rows - base[inst]).astype(np.int32)


def instance_world_rays(objects, xforms, dirs, eps=1e-4):
    """World rays of a composed scene (Sec. 4.3).  Instance j places object
    objects[j] by xforms[j] = [R | t] (3x4, world = R local + t); the ray from
    its Gaussian g (original order) along dirs[k] starts at
    fl(m + fl(eps d)) with m_c = fl(((R_c0 x + R_c1 y) + R_c2 z) + t_c) in
    float32.  Order: instance by instance, then g, then k.  Returns
    (o, d, src_inst, src_local)."""
    dirs = _c(dirs, np.float32)
    K = dirs.shape[0]
    eps = np.float32(eps)
    o_all, d_all, si, sl = [], [], [], []
    for j, (sc, xf) in enumerate(zip(objects, xforms)):
        X = np.asarray(xf, np.float32).reshape(3, 4)
        R, t = X[:, :3], X[:, 3]
        mu = _c(sc["mean"], np.float32)
        n = mu.shape[0]
        m = np.stack([((R[c, 0] * mu[:, 0] + R[c, 1] * mu[:, 1]) + R[c, 2] * mu[:, 2]) + t[c] for c in range(3)], 1)
        d = np.tile(dirs, (n, 1))
        o = np.repeat(m, K, axis=0) + eps * d
        o_all.append(o.astype(np.float32))
        d_all.append(d)
        si.append(np.full(n * K, j, np.int32))
        sl.append(np.repeat(np.arange(n, dtype=np.int32), K))
    return np.concatenate(o_all), np.concatenate(d_all), np.concatenate(si), np.concatenate(sl)


def trace_instances(objects, xforms, ray_o, ray_d, src_inst, src_local, alpha_min=1.0 / 255.0, t_min=1e-4,
                    bands=None):
    """Visibility through a composed scene: for every instance i the ray is
    taken into i's frame, o_i = fl(R_i^T fl(o - t_i)), d_i = fl(R_i^T d)
    (component c = ((R_0c v0 + R_1c v1) + R_2c v2), float32), and meets
    object i's Gaussians under Eq. 13-15 (CPU BVH tracer, no early stop),
    skipping the ray's own Gaussian; T_exact is the product over all
    instances, band flags are or-ed, and T is snapped to 0 below t_min.
    T_lo / T_hi are the products of the instances' bounds (every borderline
    candidate taken / left out; each factor lies in (0, 1], so the product
    is monotone in each and the bounds multiply).
    Returns dict(T, T_exact, flags, T_lo, T_hi)."""
    b = dict(DEFAULT_BANDS)
    if bands:
        b.update(bands)
    ray_o = _c(ray_o, np.float32)
    ray_d = _c(ray_d, np.float32)
    R_ = ray_o.shape[0]
    te = np.ones(R_)
    lo = np.ones(R_)
    hi = np.ones(R_)
    fl = np.zeros(R_, np.uint32)
    tracers = {}
    for i, (sc, xf) in enumerate(zip(objects, xforms)):
        if id(sc) not in tracers:
            tracers[id(sc)] = BvhTracer(sc, bands=b)
        X = np.asarray(xf, np.float32).reshape(3, 4)
        R, t = X[:, :3], X[:, 3]
        x = ray_o - t
        ol = np.stack([_rows(R, x, c) for c in range(3)], 1)
        dl = np.stack([_rows(R, ray_d, c) for c in range(3)], 1)
        src = np.where(src_inst == i, src_local, -1).astype(np.int32)
        r = tracers[id(sc)].trace(ol, dl, src, alpha_min=alpha_min, t_min=0.0)
        te *= r["T_exact"]
        lo *= r["T_lo"]
        hi *= r["T_hi"]
        fl |= r["flags"]
    if t_min > 0.0:
        fl[np.abs(te - t_min) <= b["band_T"]] |= FLAG_TMIN
    T = np.where(te < t_min, 0.0, te)
    return {"T": T, "T_exact": te, "flags": fl, "T_lo": lo, "T_hi": hi}


def bf16_round(x) -> np.ndarray:
    x = _c(x, np.float64)
    y = np.empty_like(x)
    _load().oracle_bf16_round(x.size, _p(x), _p(y))
    return y


MLP_IN, MLP_H = 80, 128


def mlp_set_bf16(on: bool) -> None:
    """Switch bf16 emulation (default on); off gives an exact FP64 MLP."""
    _load().oracle_mlp_set_bf16(1 if on else 0)


def mlp_nparam() -> int:
    return int(_load().oracle_mlp_nparam())


def mlp_encode(pos, dirs, lo, hi) -> np.ndarray:
    pos = _c(pos, np.float32).reshape(-1, 3)
    dirs = _c(dirs, np.float32).reshape(-1, 3)
    lo = _c(lo, np.float32)
    hi = _c(hi, np.float32)
    m = pos.shape[0]
    feat = np.empty((m, MLP_IN), np.float64)
    _load().oracle_mlp_encode(m, _p(pos), _p(dirs), _p(lo), _p(hi), _p(feat))
    return feat


def mlp_forward(params, feat):
    params = _c(params, np.float32)
    feat = _c(feat, np.float64)
    m = feat.shape[0]
    p = np.empty(m)
    z = np.empty(m)
    _load().oracle_mlp_forward(_p(params), m, _p(feat), _p(p), _p(z))
    return p, z


def mlp_loss_grad(params, feat, y, pos_weight=1.0):
    """Mean BCE against soft targets y with weight pos_weight on the lit
    term, and its gradient (parameter-block layout)."""
    params = _c(params, np.float32)
    feat = _c(feat, np.float64)
    y = _c(y, np.float64)
    g = np.empty(params.shape[0], np.float64)
    loss = _load().oracle_mlp_loss_grad(_p(params), feat.shape[0], _p(feat), _p(y), float(pos_weight), _p(g))
    return float(loss), g


def mlp_visibility(params, feat, pos_weight=1.0):
    """Visibility estimate 1 / (1 + w e^-z) of a network trained with weight
    w = pos_weight on the lit term (= the sigmoid output for w = 1)."""
    params = _c(params, np.float32)
    feat = _c(feat, np.float64)
    T = np.empty(feat.shape[0])
    _load().oracle_mlp_visibility(_p(params), feat.shape[0], _p(feat), float(pos_weight), _p(T))
    return T


def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place FP64 Adam step on numpy arrays w, m, v."""
    g = _c(g, np.float64)
    _load().oracle_adam_step(w.size, _p(w), _p(g), _p(m), _p(v), t, lr, b1, b2, eps)
