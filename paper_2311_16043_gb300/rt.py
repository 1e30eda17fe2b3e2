"""Thin Python binding of ``include/rt3dg.h`` (argument marshalling only).

Every function here keeps the C entry point's name and converts torch CUDA
tensors to device pointers and the current torch stream to a ``cudaStream_t``;
all computation runs in the sm_103a kernels of ``librt3dg.so``.  There is no
CPU fallback: if the library cannot be loaded, or a tensor is not a
contiguous CUDA tensor of the required dtype, the call raises.
"""
from __future__ import annotations

import ctypes as C
import threading

import torch

from . import _build

_lock = threading.Lock()
_LIB = None

RT_OK = 0
STATUS_NAMES = {0: "RT_OK", 1: "RT_ERR_INVALID_ARG", 2: "RT_ERR_OOM", 3: "RT_ERR_CUDA",
                4: "RT_ERR_STACK_OVERFLOW", 5: "RT_ERR_HITLOG_OVERFLOW", 6: "RT_ERR_TIMEOUT",
                7: "RT_ERR_NOT_TRAINED", 8: "RT_ERR_UNSUPPORTED", 9: "RT_ERR_RANGE"}
RT_RAYS_EXPLICIT, RT_RAYS_DIRS, RT_RAYS_ENV, RT_RAYS_HEMI = 0, 1, 2, 3
(RT_KERNEL_AUTO, RT_KERNEL_RAY, RT_KERNEL_PACKET, RT_KERNEL_WIDE, RT_KERNEL_RAY_WIDE, RT_KERNEL_RAY_REFILL,
 RT_KERNEL_WARP_RAY) = 0, 1, 2, 3, 4, 5, 6


class RTError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")


class rt_params(C.Structure):
    _fields_ = [("k_sigma", C.c_float), ("alpha_min", C.c_float), ("t_min", C.c_float),
                ("origin_eps", C.c_float), ("box_mode", C.c_int32), ("deterministic", C.c_int32)]


class rt_rayspec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_dirs", C.c_int32), ("n_rays", C.c_int64),
                ("ray_o", C.c_void_p), ("ray_d", C.c_void_p), ("ray_src", C.c_void_p),
                ("dirs", C.c_void_p), ("env", C.c_void_p), ("seed", C.c_uint64),
                ("ray_ids", C.c_void_p), ("n_ids", C.c_int64), ("normals", C.c_void_p)]


class rt_trace_opts(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("order_block", C.c_int32), ("block_threads", C.c_int32),
                ("hit_cap", C.c_int32), ("counters", C.c_void_p), ("hit_ids", C.c_void_p),
                ("hit_count", C.c_void_p)]


class rt_pbr_inputs(C.Structure):
    _fields_ = [("albedo", C.c_void_p), ("roughness", C.c_void_p), ("sh", C.c_void_p), ("env", C.c_void_p),
                ("env_h", C.c_int32), ("env_w", C.c_int32), ("cam", C.c_float * 3), ("kernel", C.c_int32)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class rt_allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


class rt_instance(C.Structure):
    _fields_ = [("bvh", C.c_void_p), ("xform", C.c_float * 12)]


class rt_batch_job(C.Structure):
    _fields_ = [("bvh", C.c_void_p), ("rays", rt_rayspec), ("T_out", C.c_void_p)]


class rt_mlp_cfg(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("batch", C.c_int32), ("pos_weight", C.c_float)]


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_U64 = C.c_uint64
_F32 = C.c_float
_SIGS = {
    "rt_params_default": (None, [_P]),
    "rt_status_string": (C.c_char_p, [_I32]),
    "rt_status_last": (_I32, []),
    "rt_status_clear": (_I32, []),
    "rt_selftest_wait_timeout": (_I32, [_I64, _P]),
    "rt_set_wait_limit": (_I32, [_I64]),
    "rt_set_allocator": (_I32, [_P]),
    "rt_build_bvh": (_I32, [_P, _P, _P, _P, _I64, _P, _P, _P]),
    "rt_bvh_destroy": (_I32, [_P, _P]),
    "rt_bvh_refit": (_I32, [_P, _P, _P, _P, _P, _P]),
    "rt_bvh_info": (_I32, [_P, _P, _P, _P, _P]),
    "rt_bvh_export": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "rt_envmap_create": (_I32, [_P, _P, _P, _I32, _I32, _P, _P]),
    "rt_envmap_destroy": (_I32, [_P, _P]),
    "rt_rayspec_count": (_I64, [_P, _P]),
    "rt_materialize_rays": (_I32, [_P, _P, _P, _I64, _P, _P, _P, _P]),
    "rt_trace_visibility": (_I32, [_P, _P, _P, _P, _P]),
    "rt_trace_visibility_dirs": (_I32, [_P, _P, _I32, _P, _P, _P]),
    "rt_visibility_dirs_host": (_I32, [_P, _P, _P, _P, _I64, _P, _I32, _P, _P, _P, _P]),
    "rt_memory_trim": (_I32, [_I64]),
    "rt_trace_visibility_backward": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I32,
                                            _P, _P, _P, _P, _P, _P]),
    "rt_mlp_cfg_default": (None, [_P]),
    "rt_surrogate_param_count": (_I64, []),
    "rt_surrogate_create": (_I32, [_P, _U64, _P, _P]),
    "rt_surrogate_destroy": (_I32, [_P, _P]),
    "rt_surrogate_set_params": (_I32, [_P, _P, _P]),
    "rt_surrogate_get_params": (_I32, [_P, _P, _P]),
    "rt_surrogate_get_state": (_I32, [_P, _P, _P]),
    "rt_surrogate_set_state": (_I32, [_P, _P, _P]),
    "rt_surrogate_set_bounds": (_I32, [_P, _P, _P]),
    "rt_surrogate_forward": (_I32, [_P, _P, _P, _I64, _P, _P]),
    "rt_surrogate_loss_grad": (_I32, [_P, _P, _P, _P, _I64, _P, _P, _P]),
    "rt_surrogate_train": (_I32, [_P, _P, _P, _P, _I32, _U64, _P, _P]),
    "rt_surrogate_infer": (_I32, [_P, _P, _P, _F32, _P, _P, _P]),
    "rt_surrogate_infer_noalloc": (_I32, [_P, _P, _P, _F32, _P, _P, _P]),
    "rt_trace_autotune": (_I32, [_P, _P, _P, _P, _P]),
    "rt_pbr_shade": (_I32, [_P, _P, _P, _P, _P, _P]),
    "rt_scene_create": (_I32, [_P, _I32, _P, _P]),
    "rt_scene_update": (_I32, [_P, _P, _I32, _P]),
    "rt_scene_info": (_I32, [_P, _P, _P]),
    "rt_scene_trace_dirs": (_I32, [_P, _P, _I32, _P, _P]),
    "rt_scene_trace": (_I32, [_P, _P, _P, _P]),
    "rt_scene_destroy": (_I32, [_P, _P]),
    "rt_trace_ao": (_I32, [_P, _P, _P, _P, _P]),
    "rt_batch_create": (_I32, [_P, _I32, _I32, _P, _P]),
    "rt_batch_run": (_I32, [_P, _P]),
    "rt_batch_info": (_I32, [_P, _P, _P, _P, _P]),
    "rt_batch_destroy": (_I32, [_P, _P]),
}


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def lib():
    """Load (building first if stale) librt3dg.so; raises if it cannot."""
    global _LIB
    with _lock:
        if _LIB is None:
            path = _build.build()
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def _check(code: int, where: str):
    if code != RT_OK:
        raise RTError(code, where)


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr() if t.numel() > 0 else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def params(k_sigma=3.0, alpha_min=1.0 / 255.0, t_min=1e-4, origin_eps=1e-4, box_mode=0,
           deterministic=False) -> rt_params:
    p = rt_params()
    lib().rt_params_default(C.byref(p))
    p.k_sigma, p.alpha_min, p.t_min, p.origin_eps, p.box_mode = k_sigma, alpha_min, t_min, origin_eps, box_mode
    p.deterministic = int(bool(deterministic))
    return p


def rt_status_last() -> int:
    return int(lib().rt_status_last())


def rt_status_clear() -> None:
    _check(lib().rt_status_clear(), "rt_status_clear")


def rt_set_wait_limit(max_cycles: int) -> None:
    """Bound (SM cycles) of the surrogate kernels' waits; 0 restores ~2 s."""
    _check(lib().rt_set_wait_limit(int(max_cycles)), "rt_set_wait_limit")


class Bvh:
    """Owning wrapper of an ``rt_bvh*`` handle."""

    def __init__(self, handle, n, prm):
        self.handle = handle
        self.n = n
        self.params = prm

    def info(self):
        n = C.c_int64()
        lo = (C.c_float * 3)()
        hi = (C.c_float * 3)()
        nb = C.c_int64()
        _check(lib().rt_bvh_info(self.handle, C.byref(n), lo, hi, C.byref(nb)), "rt_bvh_info")
        return {"n": n.value, "lo": list(lo), "hi": list(hi), "device_bytes": nb.value}

    def destroy(self, stream=None):
        if self.handle:
            _check(lib().rt_bvh_destroy(self.handle, _stream(stream)), "rt_bvh_destroy")
            self.handle = None

    def __del__(self):
        try:
            if self.handle and _LIB is not None and torch.cuda.is_initialized():
                _LIB.rt_bvh_destroy(self.handle, _stream())
                self.handle = None
        except Exception:
            pass


def rt_build_bvh(mean, scale, quat, opacity, prm: rt_params | None = None, stream=None) -> Bvh:
    n = mean.shape[0] if mean.dim() > 0 else 0
    for t, w, nm in ((mean, 3, "mean"), (scale, 3, "scale"), (quat, 4, "quat")):
        if t.numel() != n * w:
            raise ValueError(f"{nm} must have {w} values per Gaussian")
    if opacity.numel() != n:
        raise ValueError("opacity must have one value per Gaussian")
    prm = prm or params()
    h = C.c_void_p()
    _check(lib().rt_build_bvh(_ptr(mean, torch.float32, "mean"), _ptr(scale, torch.float32, "scale"),
                              _ptr(quat, torch.float32, "quat"), _ptr(opacity, torch.float32, "opacity"),
                              n, C.byref(prm), _stream(stream), C.byref(h)), "rt_build_bvh")
    return Bvh(h, n, prm)


def rt_bvh_refit(bvh: Bvh, mean, scale, quat, opacity, stream=None) -> Bvh:
    """Refit-only rebuild: new parameters of the same Gaussians, same tree
    topology, every box recomputed."""
    n = bvh.n
    for name, t, w in (("mean", mean, 3), ("scale", scale, 3), ("quat", quat, 4), ("opacity", opacity, 1)):
        if t.numel() != n * w:
            raise ValueError(f"{name} must hold {n} x {w} values")
    _check(lib().rt_bvh_refit(bvh.handle, _ptr(mean, torch.float32, "mean"), _ptr(scale, torch.float32, "scale"),
                              _ptr(quat, torch.float32, "quat"), _ptr(opacity, torch.float32, "opacity"),
                              _stream(stream)), "rt_bvh_refit")
    return bvh


def rt_bvh_export(bvh: Bvh, stream=None) -> dict:
    n = bvh.n
    dev = torch.device("cuda")
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    m = max(n - 1, 0)
    left = torch.empty(m, dtype=torch.int32, device=dev)
    right = torch.empty(m, dtype=torch.int32, device=dev)
    parent = torch.empty(max(2 * n - 1, 0), dtype=torch.int32, device=dev)
    boxes = torch.empty((m, 12), dtype=torch.float32, device=dev)
    _check(lib().rt_bvh_export(bvh.handle, _ptr(keys), _ptr(left), _ptr(right), _ptr(parent), _ptr(boxes),
                               _stream(stream)), "rt_bvh_export")
    return {"keys": keys, "left": left, "right": right, "parent": parent, "boxes": boxes}


class Envmap:
    def __init__(self, handle):
        self.handle = handle

    def destroy(self, stream=None):
        if self.handle:
            _check(lib().rt_envmap_destroy(self.handle, _stream(stream)), "rt_envmap_destroy")
            self.handle = None


def rt_envmap_create(radiance, solid_angle, corners, stream=None) -> Envmap:
    """Host numpy inputs: radiance[h,w] float64, solid_angle[h,w] float64,
    corners[h+1,w+1,3] float32."""
    import numpy as np
    rad = np.ascontiguousarray(radiance, dtype=np.float64)
    sa = np.ascontiguousarray(solid_angle, dtype=np.float64)
    cor = np.ascontiguousarray(corners, dtype=np.float32)
    h, w = rad.shape
    if sa.shape != (h, w) or cor.shape != (h + 1, w + 1, 3):
        raise ValueError("envmap shapes do not match")
    out = C.c_void_p()
    _check(lib().rt_envmap_create(rad.ctypes.data, sa.ctypes.data, cor.ctypes.data, h, w, _stream(stream),
                                  C.byref(out)), "rt_envmap_create")
    return Envmap(out)


def rayspec(kind=RT_RAYS_DIRS, *, dirs=None, ray_o=None, ray_d=None, ray_src=None, env=None,
            n_samples=0, seed=0, ray_ids=None, normals=None) -> rt_rayspec:
    rs = rt_rayspec()
    rs.kind = kind
    if kind == RT_RAYS_EXPLICIT:
        rs.n_rays = ray_o.shape[0]
        rs.ray_o = _ptr(ray_o, torch.float32, "ray_o")
        rs.ray_d = _ptr(ray_d, torch.float32, "ray_d")
        rs.ray_src = _ptr(ray_src, torch.int32, "ray_src")
    elif kind == RT_RAYS_DIRS:
        rs.n_dirs = dirs.shape[0]
        rs.dirs = _ptr(dirs, torch.float32, "dirs")
    elif kind == RT_RAYS_ENV:
        rs.n_dirs = n_samples
        rs.env = env.handle
        rs.seed = seed
    elif kind == RT_RAYS_HEMI:
        rs.n_dirs = dirs.shape[0]
        rs.dirs = _ptr(dirs, torch.float32, "dirs")
        rs.normals = _ptr(normals, torch.float32, "normals")
    if ray_ids is not None:
        rs.ray_ids = _ptr(ray_ids, torch.int64, "ray_ids")
        rs.n_ids = ray_ids.numel()
        if rs.n_ids == 0:  # an empty subset: a non-null list of length 0 (null means every ray)
            rs.ray_ids = _empty_list_ptr()
    rs._keep = (dirs, ray_o, ray_d, ray_src, env, ray_ids, normals)  # keep the tensors alive
    return rs


_EMPTY_LIST = None


def _empty_list_ptr():
    global _EMPTY_LIST
    if _EMPTY_LIST is None:
        _EMPTY_LIST = torch.zeros(1, dtype=torch.int64, device="cuda")
    return _EMPTY_LIST.data_ptr()


def rt_rayspec_count(bvh: Bvh, rs: rt_rayspec) -> int:
    return int(lib().rt_rayspec_count(bvh.handle, C.byref(rs)))


def trace_opts(kernel=RT_KERNEL_AUTO, order_block=0, counters=None, hit_ids=None, hit_count=None) -> rt_trace_opts:
    o = rt_trace_opts()
    o.kernel = kernel
    o.order_block = order_block
    o.counters = _ptr(counters, torch.int64, "counters")
    o.hit_ids = _ptr(hit_ids, torch.int32, "hit_ids")
    o.hit_count = _ptr(hit_count, torch.int32, "hit_count")
    o.hit_cap = hit_ids.shape[1] if hit_ids is not None else 0
    return o


def rt_trace_visibility(bvh: Bvh, rs: rt_rayspec, T_out=None, opts: rt_trace_opts | None = None, stream=None):
    R = rt_rayspec_count(bvh, rs)
    if R < 0:
        raise RTError(1, "rt_rayspec_count")
    if T_out is None:
        T_out = torch.empty(R, dtype=torch.float32, device="cuda")
    elif T_out.numel() != R:
        raise ValueError(f"T_out must have {R} elements")
    _check(lib().rt_trace_visibility(bvh.handle, C.byref(rs), _ptr(T_out, torch.float32, "T_out"),
                                     C.byref(opts) if opts is not None else None, _stream(stream)),
           "rt_trace_visibility")
    return T_out


def rt_trace_visibility_dirs(bvh: Bvh, dirs, T_out=None, opts: rt_trace_opts | None = None, stream=None):
    K = dirs.shape[0]
    if T_out is None:
        T_out = torch.empty((bvh.n, K), dtype=torch.float32, device="cuda")
    elif T_out.numel() != bvh.n * K:
        raise ValueError("T_out must have n*K elements")
    _check(lib().rt_trace_visibility_dirs(bvh.handle, _ptr(dirs, torch.float32, "dirs"), K,
                                          _ptr(T_out, torch.float32, "T_out"),
                                          C.byref(opts) if opts is not None else None, _stream(stream)),
           "rt_trace_visibility_dirs")
    return T_out


def _host_ptr(t, dtype, name):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr() if t.numel() > 0 else None


def rt_visibility_dirs_host(mean, scale, quat, opacity, dirs, T_host=None, prm: rt_params | None = None,
                            opts: rt_trace_opts | None = None, stream=None):
    """The whole precompute from host tensors (pin them for asynchronous
    copies): build + trace of every (Gaussian, direction) ray, T copied back
    to T_host [n, K].  Valid once the stream is synchronised."""
    n = mean.shape[0] if mean.dim() > 0 else 0
    for t, w, nm in ((mean, 3, "mean"), (scale, 3, "scale"), (quat, 4, "quat"), (opacity, 1, "opacity")):
        if t.numel() != n * w:
            raise ValueError(f"{nm} must have {w} values per Gaussian")
    K = dirs.shape[0]
    if T_host is None:
        T_host = torch.empty((n, K), dtype=torch.float32, pin_memory=torch.cuda.is_available())
    elif T_host.numel() != n * K:
        raise ValueError("T_host must have n*K elements")
    prm = prm or params()
    _check(lib().rt_visibility_dirs_host(_host_ptr(mean, torch.float32, "mean"),
                                         _host_ptr(scale, torch.float32, "scale"),
                                         _host_ptr(quat, torch.float32, "quat"),
                                         _host_ptr(opacity, torch.float32, "opacity"), n,
                                         _host_ptr(dirs, torch.float32, "dirs"), K, C.byref(prm),
                                         C.byref(opts) if opts is not None else None,
                                         _host_ptr(T_host, torch.float32, "T_host"), _stream(stream)),
           "rt_visibility_dirs_host")
    return T_host


def pbr_inputs(albedo, roughness, env, cam, sh=None, kernel=RT_KERNEL_AUTO) -> rt_pbr_inputs:
    """Material and light of the PBR colour: albedo[n,3], roughness[n],
    sh[n,9,3] or None, env[h,w,3] (device float32), cam (3 floats)."""
    p = rt_pbr_inputs()
    p.albedo = _ptr(albedo, torch.float32, "albedo")
    p.roughness = _ptr(roughness, torch.float32, "roughness")
    p.sh = _ptr(sh, torch.float32, "sh")
    p.env = _ptr(env, torch.float32, "env")
    p.env_h, p.env_w = int(env.shape[0]), int(env.shape[1])
    for i in range(3):
        p.cam[i] = float(cam[i])
    p.kernel = kernel
    p._keep = (albedo, roughness, sh, env)
    return p


def rt_pbr_shade(bvh: Bvh, rs: rt_rayspec, inputs: rt_pbr_inputs, V=None, rgb=None, stream=None):
    """Per-Gaussian PBR colour (Eq. 10) of the hemisphere set rs: from the
    visibility table V[n*K] or, with V=None, tracing the rays in the same
    kernel.  Returns rgb[n, 3]."""
    if rgb is None:
        rgb = torch.empty((bvh.n, 3), dtype=torch.float32, device="cuda")
    _check(lib().rt_pbr_shade(bvh.handle, C.byref(rs), _ptr(V, torch.float32, "V"), C.byref(inputs),
                              _ptr(rgb, torch.float32, "rgb"), _stream(stream)), "rt_pbr_shade")
    return rgb


def rt_trace_ao(bvh: Bvh, rs: rt_rayspec, ao=None, opts: rt_trace_opts | None = None, stream=None):
    """Mean visibility of each Gaussian over a full DIRS or HEMI ray set."""
    if ao is None:
        ao = torch.empty(bvh.n, dtype=torch.float32, device="cuda")
    _check(lib().rt_trace_ao(bvh.handle, C.byref(rs), C.byref(opts) if opts is not None else None,
                             _ptr(ao, torch.float32, "ao"), _stream(stream)), "rt_trace_ao")
    return ao


_ALLOCATOR = None  # keeps the ctypes callbacks alive while installed


def rt_memory_trim(keep_bytes: int = 0) -> None:
    """Return the library pool's unused device memory to the driver."""
    _check(lib().rt_memory_trim(int(keep_bytes)), "rt_memory_trim")


def use_torch_allocator(on: bool = True) -> None:
    """Route the library's device allocations through torch's caching
    allocator (on=True) or back to the stream-ordered CUDA pool (on=False).
    Switch while no library handle exists."""
    global _ALLOCATOR
    if not on:
        _check(lib().rt_set_allocator(None), "rt_set_allocator")
        _ALLOCATOR = None
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a = rt_allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)
    _check(lib().rt_set_allocator(C.byref(a)), "rt_set_allocator")
    _ALLOCATOR = a


class Scene:
    """A composed scene: object trees placed by rigid maps (two-level BVH)."""

    def __init__(self, handle, bvhs):
        self.handle = handle
        self.bvhs = list(bvhs)  # the trees must outlive the scene
        n_total = C.c_int64()
        _check(lib().rt_scene_info(handle, C.byref(n_total), None), "rt_scene_info")
        self.n_total = int(n_total.value)

    def destroy(self):
        if self.handle:
            lib().rt_scene_destroy(self.handle, None)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _instances(bvhs, xforms):
    import numpy as np
    arr = (rt_instance * len(bvhs))()
    for i, (b, x) in enumerate(zip(bvhs, xforms)):
        x = np.asarray(x, dtype=np.float32).reshape(3, 4)
        arr[i].bvh = b.handle
        for q in range(12):
            arr[i].xform[q] = float(x.flat[q])
    return arr


def rt_scene_create(bvhs, xforms, stream=None) -> Scene:
    """bvhs: list of Bvh (may repeat); xforms: list of 3x4 [R | t] (world =
    R local + t)."""
    if len(bvhs) != len(xforms) or not bvhs:
        raise ValueError("one transform per instance")
    h = C.c_void_p()
    _check(lib().rt_scene_create(_instances(bvhs, xforms), len(bvhs), _stream(stream), C.byref(h)),
           "rt_scene_create")
    return Scene(h, bvhs)


def rt_scene_update(scene: Scene, xforms, stream=None) -> Scene:
    _check(lib().rt_scene_update(scene.handle, _instances(scene.bvhs, xforms), len(scene.bvhs), _stream(stream)),
           "rt_scene_update")
    return scene


def rt_scene_trace_dirs(scene: Scene, dirs, T_out=None, stream=None):
    """Visibility of every Gaussian of every instance along dirs[K]:
    T[n_total, K], instances in order."""
    K = dirs.shape[0]
    if T_out is None:
        T_out = torch.empty((scene.n_total, K), dtype=torch.float32, device="cuda")
    _check(lib().rt_scene_trace_dirs(scene.handle, _ptr(dirs, torch.float32, "dirs"), K,
                                     _ptr(T_out, torch.float32, "T_out"), _stream(stream)), "rt_scene_trace_dirs")
    return T_out


def rt_scene_trace(scene: Scene, rs: rt_rayspec, T_out=None, stream=None):
    """Visibility of an implicit ray set (DIRS, HEMI with world-frame normals
    per scene row, or ENV) over every Gaussian of every instance:
    T[n_total, K], instances in order."""
    K = int(rs.n_dirs)
    if T_out is None:
        T_out = torch.empty((scene.n_total, K), dtype=torch.float32, device="cuda")
    _check(lib().rt_scene_trace(scene.handle, C.byref(rs), _ptr(T_out, torch.float32, "T_out"), _stream(stream)),
           "rt_scene_trace")
    return T_out


def rt_materialize_rays(bvh: Bvh, rs: rt_rayspec, ray_ids, stream=None):
    m = ray_ids.numel()
    dev = torch.device("cuda")
    o = torch.empty((m, 3), dtype=torch.float32, device=dev)
    d = torch.empty((m, 3), dtype=torch.float32, device=dev)
    s = torch.empty(m, dtype=torch.int32, device=dev)
    _check(lib().rt_materialize_rays(bvh.handle, C.byref(rs), _ptr(ray_ids, torch.int64, "ray_ids"), m,
                                     _ptr(o), _ptr(d), _ptr(s), _stream(stream)), "rt_materialize_rays")
    return o, d, s


def rt_trace_visibility_backward(bvh: Bvh, rs: rt_rayspec, mean, scale, quat, opacity, T, dL_dT,
                                 hit_ids=None, hit_count=None, d_mean=None, d_scale=None, d_quat=None,
                                 d_opacity=None, d_ray_o=None, stream=None):
    n = bvh.n
    dev = torch.device("cuda")
    d_mean = torch.zeros((n, 3), dtype=torch.float32, device=dev) if d_mean is None else d_mean
    d_scale = torch.zeros((n, 3), dtype=torch.float32, device=dev) if d_scale is None else d_scale
    d_quat = torch.zeros((n, 4), dtype=torch.float32, device=dev) if d_quat is None else d_quat
    d_opacity = torch.zeros(n, dtype=torch.float32, device=dev) if d_opacity is None else d_opacity
    cap = hit_ids.shape[1] if hit_ids is not None else 0
    _check(lib().rt_trace_visibility_backward(
        bvh.handle, C.byref(rs), _ptr(mean, torch.float32, "mean"), _ptr(scale, torch.float32, "scale"),
        _ptr(quat, torch.float32, "quat"), _ptr(opacity, torch.float32, "opacity"),
        _ptr(T, torch.float32, "T"), _ptr(dL_dT, torch.float32, "dL_dT"),
        _ptr(hit_ids, torch.int32, "hit_ids"), _ptr(hit_count, torch.int32, "hit_count"), cap,
        _ptr(d_mean, torch.float32, "d_mean"), _ptr(d_scale, torch.float32, "d_scale"),
        _ptr(d_quat, torch.float32, "d_quat"), _ptr(d_opacity, torch.float32, "d_opacity"),
        _ptr(d_ray_o, torch.float32, "d_ray_o"), _stream(stream)), "rt_trace_visibility_backward")
    return {"mean": d_mean, "scale": d_scale, "quat": d_quat, "opacity": d_opacity, "ray_o": d_ray_o}


# ---------------------------------------------------------------------------
# Learned visibility surrogate
# ---------------------------------------------------------------------------
def mlp_cfg(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, batch=262144, pos_weight=1.0) -> rt_mlp_cfg:
    c = rt_mlp_cfg()
    lib().rt_mlp_cfg_default(C.byref(c))
    c.lr, c.beta1, c.beta2, c.eps, c.batch, c.pos_weight = lr, beta1, beta2, eps, batch, pos_weight
    return c


def rt_surrogate_param_count() -> int:
    return int(lib().rt_surrogate_param_count())


class Surrogate:
    """Owning wrapper of an ``rt_surrogate*`` handle."""

    def __init__(self, handle):
        self.handle = handle

    def destroy(self, stream=None):
        if self.handle:
            _check(lib().rt_surrogate_destroy(self.handle, _stream(stream)), "rt_surrogate_destroy")
            self.handle = None

    def __del__(self):
        try:
            if self.handle and _LIB is not None and torch.cuda.is_initialized():
                _LIB.rt_surrogate_destroy(self.handle, _stream())
                self.handle = None
        except Exception:
            pass


def rt_surrogate_create(cfg: rt_mlp_cfg | None = None, seed: int = 0, stream=None) -> Surrogate:
    h = C.c_void_p()
    _check(lib().rt_surrogate_create(C.byref(cfg) if cfg is not None else None, seed, _stream(stream),
                                     C.byref(h)), "rt_surrogate_create")
    return Surrogate(h)


def rt_surrogate_set_params(s: Surrogate, params, stream=None):
    if params.numel() != rt_surrogate_param_count():
        raise ValueError("wrong parameter count")
    _check(lib().rt_surrogate_set_params(s.handle, _ptr(params, torch.float32, "params"), _stream(stream)),
           "rt_surrogate_set_params")


def rt_surrogate_get_params(s: Surrogate, stream=None):
    out = torch.empty(rt_surrogate_param_count(), dtype=torch.float32, device="cuda")
    _check(lib().rt_surrogate_get_params(s.handle, _ptr(out), _stream(stream)), "rt_surrogate_get_params")
    return out


def rt_surrogate_get_state(s: Surrogate, stream=None):
    out = torch.empty(3 * rt_surrogate_param_count() + 1, dtype=torch.float32, device="cuda")
    _check(lib().rt_surrogate_get_state(s.handle, _ptr(out), _stream(stream)), "rt_surrogate_get_state")
    return out


def rt_surrogate_set_state(s: Surrogate, state, stream=None):
    if state.numel() != 3 * rt_surrogate_param_count() + 1:
        raise ValueError("wrong state size")
    _check(lib().rt_surrogate_set_state(s.handle, _ptr(state, torch.float32, "state"), _stream(stream)),
           "rt_surrogate_set_state")


def rt_surrogate_set_bounds(s: Surrogate, lo, hi):
    lo_a = (C.c_float * 3)(*[float(x) for x in lo])
    hi_a = (C.c_float * 3)(*[float(x) for x in hi])
    _check(lib().rt_surrogate_set_bounds(s.handle, lo_a, hi_a), "rt_surrogate_set_bounds")


def rt_surrogate_forward(s: Surrogate, pos, dirs, p_out=None, stream=None):
    m = pos.shape[0]
    if p_out is None:
        p_out = torch.empty(m, dtype=torch.float32, device="cuda")
    _check(lib().rt_surrogate_forward(s.handle, _ptr(pos, torch.float32, "pos"), _ptr(dirs, torch.float32, "dir"),
                                      m, _ptr(p_out, torch.float32, "p_out"), _stream(stream)),
           "rt_surrogate_forward")
    return p_out


def rt_surrogate_loss_grad(s: Surrogate, pos, dirs, y, stream=None):
    m = pos.shape[0]
    g = torch.empty(rt_surrogate_param_count(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(lib().rt_surrogate_loss_grad(s.handle, _ptr(pos, torch.float32, "pos"), _ptr(dirs, torch.float32, "dir"),
                                        _ptr(y, torch.float32, "y"), m, _ptr(g), _ptr(loss), _stream(stream)),
           "rt_surrogate_loss_grad")
    return loss, g


def rt_surrogate_train(s: Surrogate, bvh: Bvh, rs: rt_rayspec, T_target, steps: int, seed: int = 0,
                       loss_curve=None, stream=None):
    if loss_curve is None:
        loss_curve = torch.empty(max(steps, 1), dtype=torch.float32, device="cuda")
    _check(lib().rt_surrogate_train(s.handle, bvh.handle, C.byref(rs), _ptr(T_target, torch.float32, "T_target"),
                                    steps, seed, _ptr(loss_curve, torch.float32, "loss_curve"), _stream(stream)),
           "rt_surrogate_train")
    return loss_curve


def rt_surrogate_infer(s: Surrogate, bvh: Bvh, rs: rt_rayspec, band: float = 0.3, T_out=None, n_fallback=None,
                       stream=None):
    R = rt_rayspec_count(bvh, rs)
    if T_out is None:
        T_out = torch.empty(R, dtype=torch.float32, device="cuda")
    _check(lib().rt_surrogate_infer(s.handle, bvh.handle, C.byref(rs), band, _ptr(T_out, torch.float32, "T_out"),
                                    _ptr(n_fallback, torch.int64, "n_fallback"), _stream(stream)),
           "rt_surrogate_infer")
    return T_out


# ---------------------------------------------------------------------------
# Autotuning and multi-scene batches
# ---------------------------------------------------------------------------
def rt_trace_autotune(bvh: Bvh, rs: rt_rayspec, T_scratch, opts: rt_trace_opts | None = None, stream=None):
    opts = opts if opts is not None else trace_opts()
    _check(lib().rt_trace_autotune(bvh.handle, C.byref(rs), _ptr(T_scratch, torch.float32, "T_scratch"),
                                   C.byref(opts), _stream(stream)), "rt_trace_autotune")
    return opts


class Batch:
    """Owning wrapper of an ``rt_batch*`` (keeps its jobs' objects alive)."""

    def __init__(self, handle, n_jobs, keep):
        self.handle = handle
        self.n_jobs = n_jobs
        self._keep = keep

    def run(self, stream=None):
        _check(lib().rt_batch_run(self.handle, _stream(stream)), "rt_batch_run")

    def info(self):
        nr, ni = C.c_int64(), C.c_int64()
        k = (C.c_int32 * self.n_jobs)()
        b = (C.c_int32 * self.n_jobs)()
        _check(lib().rt_batch_info(self.handle, C.byref(nr), C.byref(ni), k, b), "rt_batch_info")
        return {"n_rays": nr.value, "n_items": ni.value, "kernel": list(k), "order_block": list(b)}

    def destroy(self, stream=None):
        if self.handle:
            _check(lib().rt_batch_destroy(self.handle, _stream(stream)), "rt_batch_destroy")
            self.handle = None


def rt_batch_create(jobs, autotune: bool = True, stream=None) -> Batch:
    """jobs: list of (Bvh, rt_rayspec, T_out tensor)."""
    arr = (rt_batch_job * len(jobs))()
    for i, (bvh, rs, T) in enumerate(jobs):
        if T.numel() != rt_rayspec_count(bvh, rs):
            raise ValueError(f"job {i}: T_out has the wrong size")
        arr[i].bvh = bvh.handle
        arr[i].rays = rs
        arr[i].T_out = _ptr(T, torch.float32, "T_out")
    h = C.c_void_p()
    _check(lib().rt_batch_create(arr, len(jobs), 1 if autotune else 0, _stream(stream), C.byref(h)),
           "rt_batch_create")
    return Batch(h, len(jobs), [j for j in jobs])


def rt_surrogate_infer_noalloc(s: Surrogate, bvh: Bvh, rs: rt_rayspec, band: float, T_out, n_fallback=None,
                               stream=None):
    """rt_surrogate_infer without device allocation in the library: the
    caller provides T_out (and n_fallback); at most 2**20 rays per call."""
    _check(lib().rt_surrogate_infer_noalloc(s.handle, bvh.handle, C.byref(rs), band,
                                            _ptr(T_out, torch.float32, "T_out"),
                                            _ptr(n_fallback, torch.int64, "n_fallback"), _stream(stream)),
           "rt_surrogate_infer_noalloc")
    return T_out
