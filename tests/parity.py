"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs, and compare end states."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_1706_07062_gb300 import kerr as K


def rel_errors(gpu_x, gpu_k, ref_y):
    """Per-geodesic relative end-point errors: e_x = |dx_{1:3}| / |x_{1:3}|,
    e_k = |dk| / |k| (4-vector Euclidean norms), and |dt| / max(1, |t|).
    gpu_x, gpu_k: (4, n) planes; ref_y: (n, 8) oracle states."""
    gx = np.asarray(gpu_x).T
    gk = np.asarray(gpu_k).T
    ex = np.linalg.norm(gx[:, 1:4] - ref_y[:, 1:4], axis=1) / np.linalg.norm(ref_y[:, 1:4], axis=1)
    ek = np.linalg.norm(gk - ref_y[:, 4:8], axis=1) / np.linalg.norm(ref_y[:, 4:8], axis=1)
    et = np.abs(gx[:, 0] - ref_y[:, 0]) / np.maximum(1.0, np.abs(ref_y[:, 0]))
    return ex, ek, et


def to_np(t):
    if hasattr(t, "detach"):
        return t.detach().cpu().numpy()
    return np.asarray(t)


def oracle_flags(a, y0, opts: O.Opts, ref: O.TraceResult, gate: float, fp32: bool, t_end=None):
    """Geodesics whose end point is not determined to `gate` for this
    comparison.  FP32 runs take different accept/reject decisions than the
    FP64 oracle, so a ray counts as ill-conditioned if its end point moves by
    more than the gate when the tolerance is tightened 100x or the start
    position is perturbed by 1e-7.  The FP64 path follows the oracle's step
    sequence, so only sensitivity to a 1e-12 perturbation matters there."""
    if fp32:
        return O.ill_conditioned(a, y0, opts, ref=ref, rel=gate, t_end=t_end)
    yp = y0.copy()
    yp[:, 1:4] *= 1.0 + 1e-12
    rp = O.trace(a, yp, opts, t_end=t_end)
    ex, ek, _ = rel_errors(rp.y[:, :4].T, rp.y[:, 4:].T, ref.y)
    return (np.maximum(ex, ek) > gate) | (rp.status != ref.status)


def compare(name, a, y0, opts, out, idx, gate, fp32, ref=None, max_bad_frac=0.0, t_end=None,
            max_ill_frac=0.10, flags=None):
    """Compare the GPU outputs `out` at indices `idx` with the oracle from the
    initial states y0 (len(idx), 8).  Returns a summary dict; asserts that
    every well-conditioned geodesic meets the gate, that status
    disagreements occur only on ill-conditioned ones, and that the oracle
    flags at most `max_ill_frac` of the geodesics as ill-conditioned (the
    exclusion must not swallow the comparison)."""
    if ref is None:
        ref = O.trace(a, y0, opts, t_end=t_end)
    if flags is None:
        flags = oracle_flags(a, y0, opts, ref, gate, fp32, t_end=t_end)
    assert flags.mean() <= max_ill_frac, (
        f"{name}: {int(flags.sum())} of {len(flags)} geodesics ill-conditioned "
        f"(cap {max_ill_frac:.3f})")
    gx = to_np(out.x)[:, idx]
    gk = to_np(out.k)[:, idx]
    st = to_np(out.status)[idx]
    ex, ek, et = rel_errors(gx, gk, ref.y)
    e = np.maximum(ex, ek)
    good = ~flags
    status_bad = (st != ref.status)
    assert not np.any(status_bad & good), (
        f"{name}: status differs on {int(np.sum(status_bad & good))} well-conditioned geodesics")
    over = good & (e > gate)
    frac = float(np.mean(over[good])) if good.any() else 0.0
    summary = dict(name=name, n=int(len(idx)), ill_conditioned=int(flags.sum()),
                   status_mismatch=int(status_bad.sum()),
                   max_err_good=float(e[good].max()) if good.any() else 0.0,
                   median_err=float(np.median(e)), over_gate=int(over.sum()))
    assert frac <= max_bad_frac, f"{name}: {summary}"
    return summary


def label_flags(a, y0, opts: O.Opts, ref: O.TraceResult, gate: float, fp32: bool = True):
    """Crossing labels not determined to `gate` by the integration: a label
    (r, phi or g of either crossing) is ill-conditioned if the oracle's own
    value moves by more than the gate (relative for r and g, absolute for
    phi), or appears/disappears, when the start position is perturbed by
    1e-6 relative or the tolerance is tightened 100x (FP32 comparison: an
    FP32 trajectory accumulates ~1e-6 relative rounding over its steps), or
    when the start position is perturbed by 1e-12 (FP64 comparison, which
    follows the oracle's step sequence).  Grazing crossings, where the ray
    meets z = 0 at a shallow angle, turn a tiny error in z into a large one in
    r.  Returns a (n, 5) boolean array."""
    yp = y0.copy()
    yp[:, 1:4] *= 1.0 + (1e-6 if fp32 else 1e-12)
    runs = [O.trace(a, yp, opts, crossings=True)]
    if fp32:
        runs.append(O.trace(a, y0, O.Opts(**{**opts.__dict__, "tol": opts.tol / 100.0}),
                            crossings=True))
    bad = np.zeros(ref.cross.shape, dtype=bool)
    rc = ref.cross
    for r in runs:
        c = r.cross
        bad |= np.isnan(c) != np.isnan(rc)
        with np.errstate(invalid="ignore", divide="ignore"):
            d = np.abs(c - rc)
            d[:, [0, 2, 4]] /= np.abs(rc[:, [0, 2, 4]])
            d[:, [1, 3]] = np.abs((c[:, [1, 3]] - rc[:, [1, 3]] + np.pi) % (2 * np.pi) - np.pi)
        bad |= np.nan_to_num(d, nan=0.0) > gate
    return bad
