"""Python handle on the plain FP64 CPU oracle (``kerr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline / reference leg use this module; the library's product path never
imports it.  It shares no code with the CUDA library.

Everything here is argument marshalling around the C oracle plus the build
step that compiles it (gcc, no CUDA).  Cited passages are in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kerr_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

ESCAPED, CAPTURED, ENDTIME, MAXSTEPS, TIMEOUT, NONFINITE, INVALID_IC = 1, 2, 3, 4, 5, 6, 7


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fcx-limited-range",
           "-o", tmp, SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("h0", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("r_escape", ctypes.c_double),
                ("t_end", ctypes.c_double), ("renorm_every", ctypes.c_int32),
                ("clip_maxit", ctypes.c_int32), ("noise", ctypes.c_double),
                ("noise_zone", ctypes.c_double), ("noise_seed", ctypes.c_uint64)]


class _Counts(ctypes.Structure):
    _fields_ = [("attempts", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("rhs_evals", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I32 = ctypes.POINTER(ctypes.c_int32)
        I64 = ctypes.POINTER(ctypes.c_int64)
        c = ctypes
        _lib.oracle_ks_r.restype = c.c_double
        _lib.oracle_ks_r.argtypes = [c.c_double] * 4
        for name in ("oracle_metric", "oracle_metric_derivs"):
            getattr(_lib, name).argtypes = [c.c_int, c.c_double, D, D]
        _lib.oracle_inverse_metric.argtypes = [c.c_int, c.c_double, D, D]
        _lib.oracle_inverse_metric.restype = c.c_int
        _lib.oracle_rhs.argtypes = [c.c_int, c.c_double, D, D]
        _lib.oracle_rk4_fixed.argtypes = [c.c_int, c.c_double, D, c.c_double, c.c_int64,
                                          c.c_int64, D]
        _lib.oracle_camera_ic.argtypes = [c.c_double, c.c_double, c.c_double, c.c_double,
                                          c.c_int32, c.c_int32, c.c_int64, D]
        _lib.oracle_camera_ic.restype = c.c_int
        _lib.oracle_particle_ic.argtypes = [c.c_double, D, D, D]
        _lib.oracle_particle_ic.restype = c.c_int
        _lib.oracle_constants.argtypes = [c.c_double, D, D]
        _lib.oracle_trace_one.argtypes = [c.c_double, D, c.POINTER(_Opts), D,
                                          c.POINTER(_Counts), D]
        _lib.oracle_trace_one.restype = c.c_int
        _lib.oracle_trace_batch.argtypes = [c.c_int64, D, D, D, c.POINTER(_Opts), D, I32, I64,
                                            I64, D, c.c_int]
        _lib.oracle_trace_batch.restype = c.c_int
        _lib.oracle_trace_coordtime.argtypes = [c.c_double, c.c_double, D, c.c_double,
                                                c.POINTER(_Opts), D, D, I64]
        _lib.oracle_trace_coordtime.restype = c.c_int
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(x, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


@dataclass
class Opts:
    """Integration options; the meaning of each field is in kerr_oracle.c."""
    tol: float = 1e-10
    h0: float = 1.0
    max_steps: int = 1_000_000
    r_escape: float = 0.0
    t_end: float = float("inf")
    renorm_every: int = 0
    clip_maxit: int = 40
    # conditioning test only: relative perturbation of every accepted
    # increment that starts outside noise_zone * r_h (0 = off)
    noise: float = 0.0
    noise_zone: float = 0.0
    noise_seed: int = 0

    def c(self) -> _Opts:
        return _Opts(self.tol, self.h0, self.max_steps, self.r_escape, self.t_end,
                     self.renorm_every, self.clip_maxit, self.noise, self.noise_zone,
                     self.noise_seed)


# ---------------------------------------------------------------------------
# pointwise helpers
# ---------------------------------------------------------------------------
KS, BL = 0, 1


def ks_r(a: float, x: float, y: float, z: float) -> float:
    return lib().oracle_ks_r(a, x, y, z)


def metric(a: float, x, coords: int = KS) -> np.ndarray:
    x = _f64(x, (4,))
    g = np.zeros(16)
    lib().oracle_metric(coords, a, _dp(x), _dp(g))
    return g.reshape(4, 4)


def metric_derivs(a: float, x, coords: int = KS) -> np.ndarray:
    """dg[al, m, n] = d g_mn / d x^al."""
    x = _f64(x, (4,))
    dg = np.zeros(64)
    lib().oracle_metric_derivs(coords, a, _dp(x), _dp(dg))
    return dg.reshape(4, 4, 4)


def inverse_metric(a: float, x, coords: int = KS) -> np.ndarray:
    x = _f64(x, (4,))
    gi = np.zeros(16)
    lib().oracle_inverse_metric(coords, a, _dp(x), _dp(gi))
    return gi.reshape(4, 4)


def rhs(a: float, y, coords: int = KS) -> np.ndarray:
    y = _f64(y, (8,))
    dy = np.zeros(8)
    lib().oracle_rhs(coords, a, _dp(y), _dp(dy))
    return dy


def rk4_fixed(a: float, y0, h: float, nsteps: int, stride: int = 1,
              coords: int = KS) -> np.ndarray:
    """Fixed-step classic RK4 trajectory, every `stride`-th state, shape (rows, 8)."""
    y0 = _f64(y0, (8,))
    rows = nsteps // stride + 1
    traj = np.zeros((rows, 8))
    lib().oracle_rk4_fixed(coords, a, _dp(y0), h, nsteps, stride, _dp(traj))
    return traj


def camera_ic(a: float, incl: float, r_obs: float, half_width: float, nx: int, ny: int,
              idx) -> np.ndarray:
    """Initial states (n, 8) of the camera rays with flat indices `idx`."""
    idx = np.atleast_1d(np.asarray(idx, dtype=np.int64))
    out = np.zeros((idx.size, 8))
    L = lib()
    for j, i in enumerate(idx):
        row = out[j]
        if L.oracle_camera_ic(a, incl, r_obs, half_width, nx, ny, int(i), _dp(row)) != 0:
            row[4] = np.nan
    return out


def particle_ic(a: float, x4, v3) -> tuple[np.ndarray, np.ndarray]:
    """Initial states (n, 8) from positions (n, 4) and velocities dx/dt (n, 3).

    Returns (states, ok) where ok is False for a non-time-like velocity."""
    x4 = _f64(x4).reshape(-1, 4)
    v3 = _f64(v3).reshape(-1, 3)
    out = np.zeros((x4.shape[0], 8))
    ok = np.zeros(x4.shape[0], dtype=bool)
    L = lib()
    for j in range(x4.shape[0]):
        xr, vr, row = np.ascontiguousarray(x4[j]), np.ascontiguousarray(v3[j]), out[j]
        ok[j] = L.oracle_particle_ic(a, _dp(xr), _dp(vr), _dp(row)) == 0
    return out, ok


def constants(a: float, y) -> np.ndarray:
    """(E, L_z, Q, u^2) per state; y is (8,) or (n, 8)."""
    y = _f64(y)
    flat = y.reshape(-1, 8)
    out = np.zeros((flat.shape[0], 4))
    L = lib()
    for j in range(flat.shape[0]):
        row_in = np.ascontiguousarray(flat[j])
        row = out[j]
        L.oracle_constants(a, _dp(row_in), _dp(row))
    return out.reshape(y.shape[:-1] + (4,))


# ---------------------------------------------------------------------------
# integration
# ---------------------------------------------------------------------------
@dataclass
class TraceResult:
    y: np.ndarray          # (n, 8) end states
    status: np.ndarray     # (n,) int32
    attempts: np.ndarray   # (n,) int64 attempted steps
    rhs_evals: np.ndarray  # (n,) int64 right-hand-side evaluations
    cross: np.ndarray | None = None   # (n, 5): r1, phi1, r2, phi2, g1 (NaN if missing)


def trace(a, y0, opts: Opts, nthreads: int | None = None, t_end=None,
          crossings: bool = False) -> TraceResult:
    """Integrate each row of y0 (n, 8); `a` is a scalar or one spin per row;
    `t_end` optionally gives one end time per row (overrides opts.t_end);
    `crossings` also records the first two equatorial crossings and g."""
    y0 = _f64(y0).reshape(-1, 8)
    n = y0.shape[0]
    av = _f64(np.broadcast_to(np.asarray(a, dtype=np.float64), (n,)))
    te = None if t_end is None else _f64(np.broadcast_to(np.asarray(t_end, np.float64), (n,)))
    yend = np.zeros((n, 8))
    status = np.zeros(n, dtype=np.int32)
    att = np.zeros(n, dtype=np.int64)
    ev = np.zeros(n, dtype=np.int64)
    cr = np.full((n, 5), np.nan) if crossings else None
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    co = opts.c()
    if n:
        lib().oracle_trace_batch(
            n, _dp(av), _dp(te) if te is not None else None, _dp(y0), ctypes.byref(co), _dp(yend),
            status.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            att.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            _dp(cr) if cr is not None else None, int(nthreads))
    return TraceResult(yend, status, att, ev, cr)


# FP32 rounding model of the conditioning test: each component of each
# accepted increment outside the FP64 zone perturbed by up to 8 units of FP32
# roundoff (an increment combines eleven right-hand sides of ~100 FP32
# operations each), in three independent draws.
FP32_NOISE = 2.0 ** -21
FP32_NOISE_SEEDS = (1, 2, 3)


def ill_conditioned(a, y0, opts: Opts, ref: TraceResult | None = None,
                    rel: float = 1e-5, nthreads: int | None = None, t_end=None,
                    noise_zone: float | None = 1.5) -> np.ndarray:
    """Flag rays whose endpoint is not determined to `rel` by the integration.

    A ray is ill-conditioned if its end state moves by more than `rel`
    (relative, in x^i and in k), or its status changes, when (i) the
    tolerance is tightened 100x, (ii) the initial spatial position is
    perturbed by 1e-7 relative, or (iii) every accepted step that starts
    outside noise_zone * r_h carries FP32-sized rounding in its increment
    (FP32_NOISE, three seeded draws; None skips this test).  Rays close to
    the photon ring, or spiralling into the horizon, amplify perturbations
    exponentially -- a perturbation made along the way can matter far more
    than one made at the start -- so their endpoints are not comparable
    between two correct integrators."""
    y0 = _f64(y0).reshape(-1, 8)
    if ref is None:
        ref = trace(a, y0, opts, nthreads, t_end=t_end)
    tight = Opts(**{**opts.__dict__, "tol": opts.tol / 100.0})
    runs = [trace(a, y0, tight, nthreads, t_end=t_end)]
    yp = y0.copy()
    yp[:, 1:4] *= (1.0 + 1e-7)
    runs.append(trace(a, yp, opts, nthreads, t_end=t_end))
    if noise_zone is not None:
        for seed in FP32_NOISE_SEEDS:
            noisy = Opts(**{**opts.__dict__, "noise": FP32_NOISE, "noise_zone": noise_zone,
                            "noise_seed": seed})
            runs.append(trace(a, y0, noisy, nthreads, t_end=t_end))

    def rel_err(u, v):
        ex = np.linalg.norm(u[:, 1:4] - v[:, 1:4], axis=1) / np.linalg.norm(v[:, 1:4], axis=1)
        ek = np.linalg.norm(u[:, 4:8] - v[:, 4:8], axis=1) / np.linalg.norm(v[:, 4:8], axis=1)
        return np.maximum(ex, ek)

    bad = np.zeros(len(y0), dtype=bool)
    for r in runs:
        bad |= (rel_err(r.y, ref.y) > rel) | (r.status != ref.status)
    return bad


@dataclass
class CoordTimeResult:
    w: np.ndarray        # (n, 6): x, y, z, v^x, v^y, v^z at the end
    t: np.ndarray        # (n,) coordinate time at the end
    status: np.ndarray   # (n,) int32
    attempts: np.ndarray


def trace_coordtime(a: float, t0, w0, t_end, opts: Opts) -> CoordTimeResult:
    """Coordinate-time integration (Sec. 2.2, eq. geo_t) of each row of
    w0 (n, 6) = (x, y, z, dx/dt, dy/dt, dz/dt) from t0 to t_end (scalars or
    one per row); see oracle_trace_coordtime in kerr_oracle.c."""
    w0 = _f64(w0).reshape(-1, 6)
    n = w0.shape[0]
    t0 = np.broadcast_to(np.asarray(t0, dtype=np.float64), (n,))
    te = np.broadcast_to(np.asarray(t_end, dtype=np.float64), (n,))
    w = np.zeros((n, 6))
    t = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    att = np.zeros(n, dtype=np.int64)
    o = opts.c()
    for i in range(n):
        wi = np.zeros(6)
        ti = ctypes.c_double()
        ai = ctypes.c_int64()
        st[i] = lib().oracle_trace_coordtime(a, float(t0[i]), _dp(np.ascontiguousarray(w0[i])),
                                             float(te[i]), ctypes.byref(o), _dp(wi),
                                             ctypes.byref(ti), ctypes.byref(ai))
        w[i], t[i], att[i] = wi, ti.value, ai.value
    return CoordTimeResult(w, t, st, att)
