"""Thin Python binding of libkerr (include/kerr.h): argument marshalling only.

Every step of the integration runs in the CUDA library; this module converts
torch tensors / numpy arrays to pointers and back.  It never computes a
geodesic itself, and it raises if libkerr.so is missing (no CPU fallback).

Names follow the C ABI: ``kerr_init``, ``kerr_trace_rays``,
``kerr_trace_camera``, ``kerr_trace_particles``, ``kerr_get_stats``,
``kerr_autotune``.  Array arguments are [4][n] planes (component-major); a
torch tensor of shape (4, n) or a numpy array of that shape is accepted, on
the GPU or on the host.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libkerr.so")

FP64, FP32_KAHAN = 0, 1
ZONE_FP64, ZONE_F32X2 = 0, 1
ESCAPED, CAPTURED, ENDTIME, MAXSTEPS, TIMEOUT, NONFINITE, INVALID_IC = 1, 2, 3, 4, 5, 6, 7
STATUS_NAMES = {1: "escaped", 2: "captured", 3: "endtime", 4: "maxsteps", 5: "timeout",
                6: "nonfinite", 7: "invalid_ic"}


class KerrError(RuntimeError):
    pass


class Opts(ctypes.Structure):
    """kerr_opts (see include/kerr.h for the meaning of every field)."""
    _fields_ = [("prec", ctypes.c_int32), ("renorm_every", ctypes.c_int32),
                ("tol", ctypes.c_double), ("h0", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("r_escape", ctypes.c_double),
                ("t_end", ctypes.c_double), ("fp64_zone", ctypes.c_double),
                ("clip_maxit", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("budget_ns", ctypes.c_uint64), ("zone_prec", ctypes.c_int32),
                ("zone_variant", ctypes.c_int32), ("zone_quantum", ctypes.c_int32)]


class Camera(ctypes.Structure):
    """kerr_camera."""
    _fields_ = [("a", ctypes.c_double), ("incl", ctypes.c_double), ("r_obs", ctypes.c_double),
                ("half_width", ctypes.c_double), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32)]


class Stats(ctypes.Structure):
    """kerr_stats."""
    _fields_ = [("geodesics", ctypes.c_int64), ("attempts", ctypes.c_int64),
                ("accepted", ctypes.c_int64), ("rhs_fp32", ctypes.c_int64),
                ("rhs_fp64", ctypes.c_int64), ("attempts_fp64", ctypes.c_int64),
                ("deferred", ctypes.c_int64),
                ("status_count", ctypes.c_int64 * 8), ("kernel_ms", ctypes.c_float),
                ("variant", ctypes.c_int32), ("phase_ms", ctypes.c_float * 4),
                ("requeued", ctypes.c_int64), ("queue_errors", ctypes.c_int64),
                ("rhs_fp32_zone_phase", ctypes.c_int64),
                ("attempts_fp32_zone_phase", ctypes.c_int64),
                ("clips", ctypes.c_int64), ("clip_rhs", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_
             if f not in ("status_count", "phase_ms")}
        d["status_count"] = list(self.status_count)
        d["phase_ms"] = list(self.phase_ms)
        return d


class Tuning(ctypes.Structure):
    """kerr_tuning."""
    _fields_ = [("variant", ctypes.c_int32), ("zone_variant", ctypes.c_int32),
                ("ms", ctypes.c_float), ("from_cache", ctypes.c_int32),
                ("timed", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libkerr.so; raises KerrError when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise KerrError(f"libkerr.so not found at {LIB_PATH}; build it with "
                            "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        c = ctypes
        vp, i64, i32 = c.c_void_p, c.c_int64, c.c_int32
        L.kerr_opts_default.argtypes = [c.POINTER(Opts)]
        L.kerr_opts_default.restype = None
        L.kerr_init.argtypes = [c.c_double, c.POINTER(vp)]
        L.kerr_destroy.argtypes = [vp]
        L.kerr_trace_rays.argtypes = [vp, vp, vp, i64, c.POINTER(Opts), vp, vp, vp, vp, vp, vp,
                                      vp]
        L.kerr_trace_particles.argtypes = [vp, vp, vp, vp, i64, c.POINTER(Opts), vp, vp, vp, vp,
                                           vp, vp, vp]
        L.kerr_trace_camera.argtypes = [vp, c.POINTER(Camera), i32, c.POINTER(Opts), vp, vp, vp,
                                        vp, vp, vp, vp]
        L.kerr_trace_camera_static.argtypes = [c.POINTER(Camera), i32, c.POINTER(Opts), vp, vp,
                                               vp, vp, vp, vp, vp]
        L.kerr_get_stats.argtypes = [vp, c.POINTER(Stats)]
        L.kerr_trace_points.argtypes = [vp, vp, i64, c.c_double, c.POINTER(Opts), vp, vp, vp, vp,
                                        vp, vp, vp]
        L.kerr_surrogate_num_params.argtypes = []
        L.kerr_surrogate_num_params.restype = i64
        L.kerr_surrogate_create.argtypes = [vp, c.POINTER(vp)]
        L.kerr_surrogate_destroy.argtypes = [vp]
        L.kerr_surrogate_get_params.argtypes = [vp, vp]
        L.kerr_surrogate_get_grad.argtypes = [vp, vp]
        L.kerr_surrogate_targets.argtypes = [vp, vp, i64, c.c_double, c.POINTER(Opts), vp, vp, vp,
                                             vp]
        L.kerr_surrogate_forward.argtypes = [vp, vp, i64, vp, vp]
        L.kerr_surrogate_forward_impl.argtypes = [vp, vp, i64, vp, i32, vp]
        L.kerr_surrogate_grad.argtypes = [vp, vp, vp, vp, i64, c.POINTER(c.c_float), vp]
        L.kerr_surrogate_train.argtypes = [vp, vp, vp, vp, i64, i32, i32, c.c_float, vp, vp]
        L.kerr_surrogate_grad_impl.argtypes = [vp, vp, vp, vp, i64, c.POINTER(c.c_float), i32,
                                               vp]
        L.kerr_surrogate_train_impl.argtypes = [vp, vp, vp, vp, i64, i32, i32, c.c_float, vp,
                                                i32, vp]
        L.kerr_surrogate_render.argtypes = [vp, vp, c.POINTER(Camera), c.POINTER(Opts), c.c_float,
                                            c.c_float, c.c_float, vp, vp, c.POINTER(i64), vp]
        L.kerr_num_variants.argtypes = []
        L.kerr_variant_info.argtypes = [c.c_int, c.POINTER(i32), c.POINTER(i32)]
        L.kerr_variant_shape.argtypes = [c.c_int, c.POINTER(i32), c.POINTER(i32),
                                         c.POINTER(i32), c.POINTER(i32)]
        L.kerr_num_zone_variants.argtypes = []
        L.kerr_zone_variant_info.argtypes = [c.c_int, c.POINTER(i32), c.POINTER(i32)]
        L.kerr_autotune.argtypes = [vp, c.POINTER(Camera), c.POINTER(Opts), i64, c.POINTER(i32), vp]
        L.kerr_check_fp64_math.argtypes = [vp, i64, vp, vp]
        L.kerr_rk4_fixed.argtypes = [c.c_double, i32, i32, vp, i64, i32, c.c_double, vp]
        L.kerr_trace_coordtime.argtypes = [vp, vp, vp, vp, i64, c.POINTER(Opts), vp, vp, vp, vp,
                                           vp]
        L.kerr_rk4_fixed_bl.argtypes = [c.c_double, i32, i32, vp, i64, i32, c.c_double, vp]
        L.kerr_bl_camera_states.argtypes = [c.POINTER(Camera), i32, i32, vp, vp]
        L.kerr_trace_rays_dense.argtypes = [vp, vp, vp, i64, c.POINTER(Opts), i32, vp, vp, vp,
                                            vp, vp, vp, vp]
        L.kerr_dense_find_time.argtypes = [c.c_double, vp, i32, vp, i64, vp, vp, vp, vp, vp]
        L.kerr_fma_chain.argtypes = [i32, i64, i32, vp, c.POINTER(c.c_double), vp]
        L.kerr_trace_camera_pixels.argtypes = [vp, c.POINTER(Camera), vp, i64, c.POINTER(Opts),
                                               vp, vp, vp, vp, vp, vp, vp]
        L.kerr_abort_flag.argtypes = [vp, c.POINTER(c.POINTER(i32))]
        L.kerr_debug_fail_alloc.argtypes = [i32]
        L.kerr_params_write.argtypes = [c.c_char_p, vp, i64]
        L.kerr_params_read.argtypes = [c.c_char_p, vp, i64]
        L.kerr_surrogate_save.argtypes = [vp, c.c_char_p]
        L.kerr_surrogate_load.argtypes = [c.c_char_p, c.POINTER(vp)]
        L.kerr_autotune_cameras.argtypes = [vp, c.POINTER(Camera), i32, c.POINTER(Opts), i64,
                                            c.c_char_p, c.POINTER(Tuning), vp]
        L.kerr_autotune_particles.argtypes = [vp, vp, vp, vp, i64, c.POINTER(Opts), i64,
                                              c.c_char_p, c.POINTER(Tuning), vp]
        L.kerr_tune_key_cameras.argtypes = [c.POINTER(Camera), i32, c.POINTER(Opts), c.c_char_p,
                                            i32]
        L.kerr_tune_key_particles.argtypes = [i64, c.POINTER(Opts), c.c_char_p, i32]
        L.kerr_tune_cache_lookup.argtypes = [c.c_char_p, c.c_char_p, c.c_char_p,
                                             c.POINTER(Tuning)]
        L.kerr_tune_cache_store.argtypes = [c.c_char_p, c.c_char_p, c.c_char_p,
                                            c.POINTER(Tuning)]
        L.kerr_last_error.restype = c.c_char_p
        for name in ("kerr_init", "kerr_destroy", "kerr_trace_rays", "kerr_trace_particles",
                     "kerr_trace_camera", "kerr_trace_camera_static", "kerr_get_stats",
                     "kerr_num_variants",
                     "kerr_variant_info", "kerr_autotune", "kerr_num_zone_variants",
                     "kerr_zone_variant_info", "kerr_trace_points", "kerr_surrogate_create",
                     "kerr_surrogate_destroy", "kerr_surrogate_get_params",
                     "kerr_surrogate_get_grad", "kerr_surrogate_targets",
                     "kerr_surrogate_forward", "kerr_surrogate_grad", "kerr_surrogate_train",
                     "kerr_surrogate_render", "kerr_check_fp64_math",
                     "kerr_surrogate_forward_impl", "kerr_rk4_fixed",
                     "kerr_trace_coordtime", "kerr_rk4_fixed_bl",
                     "kerr_bl_camera_states", "kerr_trace_rays_dense",
                     "kerr_dense_find_time", "kerr_fma_chain", "kerr_abort_flag",
                     "kerr_debug_fail_alloc", "kerr_params_write", "kerr_params_read",
                     "kerr_surrogate_save", "kerr_surrogate_load", "kerr_autotune_cameras",
                     "kerr_autotune_particles", "kerr_tune_key_cameras",
                     "kerr_tune_key_particles", "kerr_tune_cache_lookup",
                     "kerr_tune_cache_store", "kerr_trace_camera_pixels",
                     "kerr_surrogate_grad_impl", "kerr_surrogate_train_impl"):
            getattr(L, name).restype = c.c_int
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise KerrError(f"{what} failed ({rc}): {lib().kerr_last_error().decode()}")


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().kerr_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def camera(a: float, incl: float, r_obs: float, half_width: float, nx: int, ny: int) -> Camera:
    return Camera(a, incl, r_obs, half_width, nx, ny)


# ---------------------------------------------------------------------------
# pointer marshalling
# ---------------------------------------------------------------------------
def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):            # torch tensor
        if not x.is_contiguous():
            raise KerrError("tensors must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise KerrError("arrays must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_ptr(stream, *bufs):
    if stream is not None:
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    for b in bufs:
        if hasattr(b, "is_cuda") and b.is_cuda:
            import torch
            return int(torch.cuda.current_stream(b.device).cuda_stream)
    return None


@dataclass
class TraceOut:
    x: object        # (4, n) float64: end events
    k: object        # (4, n) float64: end momenta
    status: object   # (n,) int32
    steps: object    # (n,) int32 attempted steps
    diag: object     # (4, n) float32 (E, L_z, Q, u^2) or None
    cross: object = None   # (5, n) float32 (r1, phi1, r2, phi2, g1) or None

    @property
    def n(self) -> int:
        return int(self.status.shape[0])


def alloc_out(n: int, device=None, diag: bool = True, pinned: bool = False,
              cross: bool = False) -> TraceOut:
    """Output buffers: torch tensors on `device` (a CUDA device, or "cpu" with
    optional pinned memory), or numpy arrays when device is None."""
    if device is None:
        return TraceOut(np.empty((4, n)), np.empty((4, n)), np.empty(n, np.int32),
                        np.empty(n, np.int32), np.empty((4, n), np.float32) if diag else None,
                        np.empty((5, n), np.float32) if cross else None)
    import torch
    kw = dict(device=device)
    if pinned:
        kw = dict(device="cpu", pin_memory=True)
    return TraceOut(torch.empty((4, n), dtype=torch.float64, **kw),
                    torch.empty((4, n), dtype=torch.float64, **kw),
                    torch.empty(n, dtype=torch.int32, **kw),
                    torch.empty(n, dtype=torch.int32, **kw),
                    torch.empty((4, n), dtype=torch.float32, **kw) if diag else None,
                    torch.empty((5, n), dtype=torch.float32, **kw) if cross else None)


# ---------------------------------------------------------------------------
# the C entry points
# ---------------------------------------------------------------------------
class Context:
    """Owns a kerr_ctx (kerr_init / kerr_destroy)."""

    def __init__(self, a: float):
        h = ctypes.c_void_p()
        _check(lib().kerr_init(float(a), ctypes.byref(h)), "kerr_init")
        self.handle = h
        self.a = float(a)

    def close(self):
        if self.handle:
            lib().kerr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kerr_init(a: float) -> Context:
    return Context(a)


def kerr_destroy(ctx: Context):
    ctx.close()


def kerr_trace_rays(ctx: Context, x0, k0, opts: Opts | None = None, out: TraceOut | None = None,
                    stream=None) -> TraceOut:
    n = int(x0.shape[-1])
    if tuple(x0.shape) != (4, n) or tuple(k0.shape) != (4, n):
        raise KerrError("x0 and k0 must have shape (4, n)")
    opts = opts or default_opts()
    if out is None:
        out = alloc_out(n, x0.device if hasattr(x0, "device") else None)
    _check(lib().kerr_trace_rays(ctx.handle, _ptr(x0), _ptr(k0), n, ctypes.byref(opts),
                                 _ptr(out.x), _ptr(out.k), _ptr(out.status), _ptr(out.steps),
                                 _ptr(out.diag), _ptr(out.cross), _stream_ptr(stream, x0, out.x)),
           "kerr_trace_rays")
    return out


def kerr_trace_particles(ctx: Context, x0, v0, t_end=None, opts: Opts | None = None,
                         out: TraceOut | None = None, stream=None) -> TraceOut:
    n = int(x0.shape[-1])
    if tuple(x0.shape) != (4, n) or tuple(v0.shape) != (3, n):
        raise KerrError("x0 must have shape (4, n) and v0 shape (3, n)")
    if t_end is not None and tuple(t_end.shape) != (n,):
        raise KerrError("t_end must have shape (n,)")
    opts = opts or default_opts()
    if out is None:
        out = alloc_out(n, x0.device if hasattr(x0, "device") else None)
    _check(lib().kerr_trace_particles(ctx.handle, _ptr(x0), _ptr(v0), _ptr(t_end), n,
                                      ctypes.byref(opts),
                                      _ptr(out.x), _ptr(out.k), _ptr(out.status),
                                      _ptr(out.steps), _ptr(out.diag), _ptr(out.cross),
                                      _stream_ptr(stream, x0, out.x)),
           "kerr_trace_particles")
    return out


def camera_rays(cams) -> int:
    return sum(c.nx * c.ny for c in cams)


def kerr_trace_camera(ctx: Context, cams, opts: Opts | None = None, out: TraceOut | None = None,
                      stream=None, device=None) -> TraceOut:
    if isinstance(cams, Camera):
        cams = [cams]
    arr = (Camera * len(cams))(*cams)
    n = camera_rays(cams)
    opts = opts or default_opts()
    if out is None:
        out = alloc_out(n, device)
    _check(lib().kerr_trace_camera(ctx.handle, arr, len(cams), ctypes.byref(opts), _ptr(out.x),
                                   _ptr(out.k), _ptr(out.status), _ptr(out.steps),
                                   _ptr(out.diag), _ptr(out.cross), _stream_ptr(stream, out.x)),
           "kerr_trace_camera")
    return out


def kerr_trace_camera_pixels(ctx: Context, cam: Camera, index, opts: Opts | None = None,
                             out: TraceOut | None = None, stream=None) -> TraceOut:
    """Trace the pixels `index` (device int64 tensor of flat indices) of one
    camera; entry i of the outputs belongs to pixel index[i]."""
    n = int(index.numel())
    opts = opts or default_opts()
    if out is None:
        out = alloc_out(n, index.device)
    _check(lib().kerr_trace_camera_pixels(ctx.handle, ctypes.byref(cam), _ptr(index), n,
                                          ctypes.byref(opts), _ptr(out.x), _ptr(out.k),
                                          _ptr(out.status), _ptr(out.steps), _ptr(out.diag),
                                          _ptr(out.cross), _stream_ptr(stream, index)),
           "kerr_trace_camera_pixels")
    return out


STATIC_MAX_GEODESICS = 131072
STATIC_MAX_CAMERAS = 64


def kerr_trace_camera_static(cams, opts: Opts | None = None, out: TraceOut | None = None,
                             stream=None, device=None) -> TraceOut:
    """Allocation-free camera tracing (kerr_trace_camera_static): no context,
    outputs must be device tensors, at most STATIC_MAX_GEODESICS rays."""
    if isinstance(cams, Camera):
        cams = [cams]
    arr = (Camera * len(cams))(*cams)
    n = camera_rays(cams)
    opts = opts or default_opts()
    if out is None:
        out = alloc_out(n, device)
    _check(lib().kerr_trace_camera_static(arr, len(cams), ctypes.byref(opts), _ptr(out.x),
                                          _ptr(out.k), _ptr(out.status), _ptr(out.steps),
                                          _ptr(out.diag), _ptr(out.cross),
                                          _stream_ptr(stream, out.x)),
           "kerr_trace_camera_static")
    return out


def kerr_get_stats(ctx: Context) -> Stats:
    s = Stats()
    _check(lib().kerr_get_stats(ctx.handle, ctypes.byref(s)), "kerr_get_stats")
    return s


def kerr_num_variants() -> int:
    return lib().kerr_num_variants()


def kerr_variant_info(v: int) -> tuple[int, int]:
    b, m = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().kerr_variant_info(v, ctypes.byref(b), ctypes.byref(m)), "kerr_variant_info")
    return b.value, m.value


def kerr_variant_shape(v: int) -> tuple[int, int, int, int]:
    """(threads per block, minimum blocks per SM, geodesics per thread,
    right-hand-side mode of the FP32 steps) of stepping variant v."""
    b, m, r, h = (ctypes.c_int32() for _ in range(4))
    _check(lib().kerr_variant_shape(v, ctypes.byref(b), ctypes.byref(m), ctypes.byref(r),
                                    ctypes.byref(h)), "kerr_variant_shape")
    return b.value, m.value, r.value, h.value


def kerr_num_zone_variants() -> int:
    return lib().kerr_num_zone_variants()


def kerr_zone_variant_info(v: int) -> tuple[int, int]:
    b, m = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().kerr_zone_variant_info(v, ctypes.byref(b), ctypes.byref(m)),
           "kerr_zone_variant_info")
    return b.value, m.value


def kerr_autotune(ctx: Context, cam: Camera, opts: Opts | None = None, sample: int = 65536,
                  stream=None) -> int:
    best = ctypes.c_int32()
    opts = opts or default_opts()
    _check(lib().kerr_autotune(ctx.handle, ctypes.byref(cam), ctypes.byref(opts), sample,
                               ctypes.byref(best), _stream_ptr(stream)), "kerr_autotune")
    return best.value


# ---------------------------------------------------------------------------
# image points and the learned surrogate
# ---------------------------------------------------------------------------
SURR_INPUT_SCALE = 25.0
SURR_OUTPUTS = 8


def kerr_trace_points(ctx: Context, points, r_obs: float, opts: Opts | None = None,
                      out: TraceOut | None = None, stream=None) -> TraceOut:
    """points: (n, 4) float64 rows (alpha, beta, a, inclination)."""
    n = int(points.shape[0])
    if tuple(points.shape) != (n, 4):
        raise KerrError("points must have shape (n, 4)")
    opts = opts or default_opts()
    if out is None:
        out = alloc_out(n, points.device if hasattr(points, "device") else None, cross=True)
    _check(lib().kerr_trace_points(ctx.handle, _ptr(points), n, float(r_obs), ctypes.byref(opts),
                                   _ptr(out.x), _ptr(out.k), _ptr(out.status), _ptr(out.steps),
                                   _ptr(out.diag), _ptr(out.cross),
                                   _stream_ptr(stream, points, out.x)), "kerr_trace_points")
    return out


def kerr_surrogate_num_params() -> int:
    return int(lib().kerr_surrogate_num_params())


class Surrogate:
    """Owns a kerr_surrogate (kerr_surrogate_create / kerr_surrogate_destroy)."""

    def __init__(self, init_params: np.ndarray):
        p = np.ascontiguousarray(init_params, dtype=np.float32)
        if p.size != kerr_surrogate_num_params():
            raise KerrError("init_params has the wrong size")
        h = ctypes.c_void_p()
        _check(lib().kerr_surrogate_create(p.ctypes.data, ctypes.byref(h)),
               "kerr_surrogate_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().kerr_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(kerr_surrogate_num_params(), np.float32)
        _check(lib().kerr_surrogate_get_params(self.handle, out.ctypes.data),
               "kerr_surrogate_get_params")
        return out

    def grad(self) -> np.ndarray:
        out = np.empty(kerr_surrogate_num_params(), np.float32)
        _check(lib().kerr_surrogate_get_grad(self.handle, out.ctypes.data),
               "kerr_surrogate_get_grad")
        return out


def kerr_surrogate_targets(ctx: Context, points, r_obs: float, opts: Opts | None = None,
                           stream=None):
    """(in, targets, mask) device tensors from (n, 4) device points."""
    import torch
    n = int(points.shape[0])
    dev = points.device
    inp = torch.empty((n, 4), dtype=torch.float32, device=dev)
    tgt = torch.empty((n, 8), dtype=torch.float32, device=dev)
    msk = torch.empty((n, 8), dtype=torch.float32, device=dev)
    opts = opts or default_opts()
    _check(lib().kerr_surrogate_targets(ctx.handle, _ptr(points), n, float(r_obs),
                                        ctypes.byref(opts), _ptr(inp), _ptr(tgt), _ptr(msk),
                                        _stream_ptr(stream, points)), "kerr_surrogate_targets")
    return inp, tgt, msk


SURR_FWD_TENSOR_CORE, SURR_FWD_GEMM = 0, 1


def kerr_surrogate_forward(s: Surrogate, inp, out=None, stream=None, impl=None):
    """(n, 8) network outputs; impl None = the fused tensor-core kernel."""
    import torch
    n = int(inp.shape[0])
    if out is None:
        out = torch.empty((n, 8), dtype=torch.float32, device=inp.device)
    if impl is None:
        _check(lib().kerr_surrogate_forward(s.handle, _ptr(inp), n, _ptr(out),
                                            _stream_ptr(stream, inp)), "kerr_surrogate_forward")
    else:
        _check(lib().kerr_surrogate_forward_impl(s.handle, _ptr(inp), n, _ptr(out), int(impl),
                                                 _stream_ptr(stream, inp)),
               "kerr_surrogate_forward_impl")
    return out


SURR_TRAIN_FUSED, SURR_TRAIN_GEMM = 0, 1


def kerr_surrogate_grad(s: Surrogate, inp, tgt, msk, stream=None, impl=None) -> float:
    """Batch loss; the gradient stays in the surrogate (Surrogate.grad()).
    impl None = the fused training kernels."""
    loss = ctypes.c_float()
    if impl is None:
        _check(lib().kerr_surrogate_grad(s.handle, _ptr(inp), _ptr(tgt), _ptr(msk),
                                         int(inp.shape[0]), ctypes.byref(loss),
                                         _stream_ptr(stream, inp)), "kerr_surrogate_grad")
    else:
        _check(lib().kerr_surrogate_grad_impl(s.handle, _ptr(inp), _ptr(tgt), _ptr(msk),
                                              int(inp.shape[0]), ctypes.byref(loss), int(impl),
                                              _stream_ptr(stream, inp)),
               "kerr_surrogate_grad_impl")
    return loss.value


def kerr_surrogate_train(s: Surrogate, inp, tgt, msk, epochs: int, batch: int, lr: float,
                         stream=None, impl=None) -> np.ndarray:
    """Mean batch loss per epoch; impl None = the fused training kernels."""
    losses = np.zeros(epochs, np.float32)
    if impl is None:
        _check(lib().kerr_surrogate_train(s.handle, _ptr(inp), _ptr(tgt), _ptr(msk),
                                          int(inp.shape[0]), int(epochs), int(batch), float(lr),
                                          losses.ctypes.data, _stream_ptr(stream, inp)),
               "kerr_surrogate_train")
    else:
        _check(lib().kerr_surrogate_train_impl(s.handle, _ptr(inp), _ptr(tgt), _ptr(msk),
                                               int(inp.shape[0]), int(epochs), int(batch),
                                               float(lr), losses.ctypes.data, int(impl),
                                               _stream_ptr(stream, inp)),
               "kerr_surrogate_train_impl")
    return losses


def kerr_surrogate_render(ctx: Context, s: Surrogate, cam: Camera, opts: Opts | None = None,
                          p_lo: float = 0.05, p_hi: float = 0.95, crit_dist: float = 0.5,
                          device="cuda", stream=None):
    """Returns (out (6, n) float32, fallback (n,) uint8, n_fallback)."""
    import torch
    n = cam.nx * cam.ny
    out = torch.empty((6, n), dtype=torch.float32, device=device)
    fb = torch.empty(n, dtype=torch.uint8, device=device)
    nfb = ctypes.c_int64()
    opts = opts or default_opts()
    _check(lib().kerr_surrogate_render(ctx.handle, s.handle, ctypes.byref(cam),
                                       ctypes.byref(opts), p_lo, p_hi, crit_dist, _ptr(out),
                                       _ptr(fb), ctypes.byref(nfb), _stream_ptr(stream, out)),
           "kerr_surrogate_render")
    return out, fb, nfb.value


def kerr_check_fp64_math(x, stream=None):
    """(3, n) device tensor: the integrator's FP64 1/x, 1/sqrt(x), sqrt(x)."""
    import torch
    n = int(x.numel())
    out = torch.empty((3, n), dtype=torch.float64, device=x.device)
    _check(lib().kerr_check_fp64_math(_ptr(x), n, _ptr(out), _stream_ptr(stream, x)),
           "kerr_check_fp64_math")
    return out


LAYOUT_SOA, LAYOUT_AOS = 0, 1
FIXED_FP32, FIXED_FP64, FIXED_FP32X2 = 0, 1, 2


def kerr_rk4_fixed(a: float, state, nsteps: int, h: float, layout: int = LAYOUT_SOA,
                   stream=None, coords: str = "ks", paired: bool = False):
    """Paper-mode fixed-step RK4 in place on a device tensor: float32 or
    float64, shape (8, n) for LAYOUT_SOA or (n, 8) for LAYOUT_AOS; coords
    "ks" (Cartesian Kerr-Schild, (x, k)) or "bl" (Boyer-Lindquist, (x, p)).
    paired: float32 KS only, two geodesics per thread on packed f32x2
    instructions (KERR_FIXED_FP32X2)."""
    import torch
    if state.dtype not in (torch.float32, torch.float64):
        raise KerrError("state must be float32 or float64")
    if coords not in ("ks", "bl"):
        raise KerrError("coords must be 'ks' or 'bl'")
    n = int(state.shape[1] if layout == LAYOUT_SOA else state.shape[0])
    fn = lib().kerr_rk4_fixed if coords == "ks" else lib().kerr_rk4_fixed_bl
    prec = FIXED_FP64 if state.dtype == torch.float64 else FIXED_FP32
    if paired:
        if prec != FIXED_FP32:
            raise KerrError("paired steps are FP32 only")
        prec = FIXED_FP32X2
    _check(fn(float(a), int(prec), int(layout), _ptr(state), n,
              int(nsteps), float(h), _stream_ptr(stream, state)), "kerr_rk4_fixed")
    return state


def kerr_bl_camera_states(cam: Camera, dtype=None, layout: int = LAYOUT_SOA, device="cuda",
                          stream=None):
    """BL start states (t, r, th, ph, p_t, p_r, p_th, p_ph) of a camera's rays."""
    import torch
    dtype = dtype or torch.float64
    n = cam.nx * cam.ny
    shape = (8, n) if layout == LAYOUT_SOA else (n, 8)
    st = torch.empty(shape, dtype=dtype, device=device)
    _check(lib().kerr_bl_camera_states(ctypes.byref(cam), int(dtype == torch.float64),
                                       int(layout), _ptr(st), _stream_ptr(stream, st)),
           "kerr_bl_camera_states")
    return st


@dataclass
class CoordTimeOut:
    x: object            # (4, n) end events (t, x, y, z)
    v: object            # (3, n) end velocities dx/dt
    status: object
    steps: object


def kerr_trace_coordtime(ctx: Context, x0, v0, t_end=None, opts: Opts | None = None,
                         stream=None) -> CoordTimeOut:
    """Coordinate-time integration of device tensors x0 (4, n), v0 (3, n)
    (float64) to t_end ((n,) tensor, or opts.t_end)."""
    import torch
    n = int(x0.shape[1])
    if tuple(x0.shape) != (4, n) or tuple(v0.shape) != (3, n):
        raise KerrError("x0 must have shape (4, n) and v0 shape (3, n)")
    opts = opts or default_opts()
    dev = x0.device
    out = CoordTimeOut(torch.empty((4, n), dtype=torch.float64, device=dev),
                       torch.empty((3, n), dtype=torch.float64, device=dev),
                       torch.empty(n, dtype=torch.int32, device=dev),
                       torch.empty(n, dtype=torch.int32, device=dev))
    _check(lib().kerr_trace_coordtime(ctx.handle, _ptr(x0), _ptr(v0), _ptr(t_end), n,
                                      ctypes.byref(opts), _ptr(out.x), _ptr(out.v),
                                      _ptr(out.status), _ptr(out.steps),
                                      _stream_ptr(stream, x0)), "kerr_trace_coordtime")
    return out


def kerr_trace_rays_dense(ctx: Context, x0, k0, cap: int, opts: Opts | None = None,
                          stream=None):
    """FP64 trace of device tensors x0, k0 (4, n) that also stores the solution.
    Returns (TraceOut, traj (n, cap, 9), traj_count (n,))."""
    import torch
    n = int(x0.shape[1])
    opts = opts or default_opts(prec=FP64)
    dev = x0.device
    out = alloc_out(n, dev, diag=False)
    traj = torch.empty((n, cap, 9), dtype=torch.float64, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    _check(lib().kerr_trace_rays_dense(ctx.handle, _ptr(x0), _ptr(k0), n, ctypes.byref(opts),
                                       int(cap), _ptr(traj), _ptr(cnt), _ptr(out.x), _ptr(out.k),
                                       _ptr(out.status), _ptr(out.steps),
                                       _stream_ptr(stream, x0)), "kerr_trace_rays_dense")
    return out, traj, cnt


def kerr_dense_find_time(a: float, traj, traj_count, t_target, stream=None):
    """(y (8, n), lam (n,), found (n,)) at t = t_target on stored solutions."""
    import torch
    n, cap = int(traj.shape[0]), int(traj.shape[1])
    dev = traj.device
    y = torch.empty((8, n), dtype=torch.float64, device=dev)
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    found = torch.empty(n, dtype=torch.int32, device=dev)
    _check(lib().kerr_dense_find_time(float(a), _ptr(traj), cap, _ptr(traj_count), n,
                                      _ptr(t_target), _ptr(y), _ptr(lam), _ptr(found),
                                      _stream_ptr(stream, traj)), "kerr_dense_find_time")
    return y, lam, found


PEAK_FP32, PEAK_FP64, PEAK_FP32X2 = 0, 1, 2


def kerr_fma_chain(kind: int, rounds: int, sink, blocks_per_sm: int = 4, stream=None) -> float:
    """Launch the FMA-chain peak kernel on `stream` (the caller times it);
    returns the FLOPs the launch performs.  sink: device float32 tensor of at
    least SMs x blocks_per_sm x 256 elements."""
    flops = ctypes.c_double()
    _check(lib().kerr_fma_chain(int(kind), int(rounds), int(blocks_per_sm), _ptr(sink),
                                ctypes.byref(flops), _stream_ptr(stream, sink)), "kerr_fma_chain")
    return flops.value


# ---------------------------------------------------------------------------
# failure handling, parameter files, autotuning with a cache
# ---------------------------------------------------------------------------
class AbortFlag:
    """The context's host-writable abort flag (kerr_abort_flag): set() makes
    running and later launches stop (KERR_TIMEOUT), clear() re-arms."""

    def __init__(self, ctx: Context):
        p = ctypes.POINTER(ctypes.c_int32)()
        _check(lib().kerr_abort_flag(ctx.handle, ctypes.byref(p)), "kerr_abort_flag")
        self._p = p
        self._ctx = ctx          # the flag lives as long as the context

    def set(self, value: int = 1):
        self._p[0] = int(value)

    def clear(self):
        self._p[0] = 0

    def value(self) -> int:
        return int(self._p[0])


def kerr_abort_flag(ctx: Context) -> AbortFlag:
    return AbortFlag(ctx)


def kerr_debug_fail_alloc(n: int):
    _check(lib().kerr_debug_fail_alloc(int(n)), "kerr_debug_fail_alloc")


def kerr_params_write(path: str, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().kerr_params_write(os.fsencode(path), p.ctypes.data, p.size),
           "kerr_params_write")


def kerr_params_read(path: str) -> np.ndarray:
    out = np.empty(kerr_surrogate_num_params(), np.float32)
    _check(lib().kerr_params_read(os.fsencode(path), out.ctypes.data, out.size),
           "kerr_params_read")
    return out


def kerr_surrogate_save(s: "Surrogate", path: str):
    _check(lib().kerr_surrogate_save(s.handle, os.fsencode(path)), "kerr_surrogate_save")


def kerr_surrogate_load(path: str) -> "Surrogate":
    h = ctypes.c_void_p()
    _check(lib().kerr_surrogate_load(os.fsencode(path), ctypes.byref(h)), "kerr_surrogate_load")
    s = Surrogate.__new__(Surrogate)
    s.handle = h
    return s


def kerr_autotune_cameras(ctx: Context, cams, opts: Opts | None = None, sample: int = 1 << 18,
                          cache_path: str | None = None, stream=None) -> Tuning:
    if isinstance(cams, Camera):
        cams = [cams]
    arr = (Camera * len(cams))(*cams)
    t = Tuning()
    opts = opts or default_opts()
    _check(lib().kerr_autotune_cameras(ctx.handle, arr, len(cams), ctypes.byref(opts), int(sample),
                                       os.fsencode(cache_path) if cache_path else None,
                                       ctypes.byref(t), _stream_ptr(stream)),
           "kerr_autotune_cameras")
    return t


def kerr_autotune_particles(ctx: Context, x0, v0, t_end=None, opts: Opts | None = None,
                            sample: int = 1 << 14, cache_path: str | None = None,
                            stream=None) -> Tuning:
    n = int(x0.shape[-1])
    t = Tuning()
    opts = opts or default_opts()
    _check(lib().kerr_autotune_particles(ctx.handle, _ptr(x0), _ptr(v0), _ptr(t_end), n,
                                         ctypes.byref(opts), int(sample),
                                         os.fsencode(cache_path) if cache_path else None,
                                         ctypes.byref(t), _stream_ptr(stream, x0)),
           "kerr_autotune_particles")
    return t


def kerr_tune_key_cameras(cams, opts: Opts | None = None) -> str:
    if isinstance(cams, Camera):
        cams = [cams]
    arr = (Camera * len(cams))(*cams)
    buf = ctypes.create_string_buffer(512)
    opts = opts or default_opts()
    _check(lib().kerr_tune_key_cameras(arr, len(cams), ctypes.byref(opts), buf, len(buf)),
           "kerr_tune_key_cameras")
    return buf.value.decode()


def kerr_tune_key_particles(n: int, opts: Opts | None = None) -> str:
    buf = ctypes.create_string_buffer(512)
    opts = opts or default_opts()
    _check(lib().kerr_tune_key_particles(int(n), ctypes.byref(opts), buf, len(buf)),
           "kerr_tune_key_particles")
    return buf.value.decode()


def kerr_tune_cache_lookup(path: str, gpu: str, key: str) -> Tuning | None:
    """The stored choice for (gpu, key), or None when the cache has none."""
    t = Tuning()
    rc = lib().kerr_tune_cache_lookup(os.fsencode(path), gpu.encode(), key.encode(),
                                      ctypes.byref(t))
    if rc == 1:
        return None
    _check(rc, "kerr_tune_cache_lookup")
    return t


def kerr_tune_cache_store(path: str, gpu: str, key: str, t: Tuning):
    _check(lib().kerr_tune_cache_store(os.fsencode(path), gpu.encode(), key.encode(),
                                       ctypes.byref(t)), "kerr_tune_cache_store")
