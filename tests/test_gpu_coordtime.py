"""Coordinate-time integration (Sec. 2.2, eq. geo_t) on the device against the
oracle's coordinate-time integrator, and against a circular orbit's closed
form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import closed_forms as C  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1706_07062_gb300 import kerr as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def photons(a=0.9):
    """A 16 x 16 camera at r = 50 M, +-12 M (near passes, captures and escapes),
    as start events and coordinate velocities."""
    idx = np.arange(256)
    y0 = O.camera_ic(a, np.radians(60.0), 50.0, 12.0, 16, 16, idx)
    w0 = np.concatenate([y0[:, 1:4], y0[:, 5:8] / y0[:, 4:5]], axis=1)
    return y0, w0


def run(ctx, y0, w0, t_end, opts):
    x0 = torch.tensor(np.stack([y0[:, 0], w0[:, 0], w0[:, 1], w0[:, 2]]), device=DEV)
    v0 = torch.tensor(w0[:, 3:].T.copy(), device=DEV)
    te = torch.full((y0.shape[0],), float(t_end), dtype=torch.float64, device=DEV)
    out = K.kerr_trace_coordtime(ctx, x0, v0, te, opts)
    torch.cuda.synchronize()
    return out


def coordtime_err(w, ref_w):
    """Per-geodesic end-state error max_i |w_i - ref_i| / (1 + |ref_i|) over
    (x, y, z, v^x, v^y, v^z)."""
    return np.max(np.abs(w - ref_w) / (1 + np.abs(ref_w)), axis=1)


def coordtime_flags(a, y0, w0, t_end, opts, ref, gate, fp32):
    """Geodesics whose coordinate-time end state is not determined to `gate`:
    it moves by more than the gate, or the status changes, when the start
    position is perturbed (1e-12 relative for the FP64 comparison, which
    follows the oracle's step sequence; 1e-7 for FP32) or, for FP32, when the
    tolerance is tightened 100x.  Captured geodesics stop at the first step
    inside 1.01 r_h without clipping, so their end states depend on the step
    sequence and are flagged whenever it matters."""
    wp = w0.copy()
    wp[:, :3] *= 1 + (1e-7 if fp32 else 1e-12)
    runs = [O.trace_coordtime(a, y0[:, 0], wp, t_end, opts)]
    if fp32:
        runs.append(O.trace_coordtime(a, y0[:, 0], w0, t_end,
                                      O.Opts(**{**opts.__dict__, "tol": opts.tol / 100})))
    bad = np.zeros(len(w0), dtype=bool)
    for r in runs:
        bad |= (coordtime_err(r.w, ref.w) > gate) | (r.status != ref.status)
    return bad


@pytest.mark.parametrize("prec,tol,gate", [(K.FP64, 1e-10, 1e-9), (K.FP32_KAHAN, 1e-8, 1e-5)])
def test_coordtime_matches_oracle(prec, tol, gate):
    """End states against the oracle's coordinate-time integrator on every
    geodesic that reaches the end time and that the oracle finds determined
    to the gate, and the same status on every well-conditioned geodesic (at
    most 12 % are not).  Captures are compared by status only: the
    coordinate-time integrator stops at the first accepted step inside
    1.01 r_h without clipping, where rounding differences of the two
    right-hand-side forms, grown along the plunge, move the state by 1e-8 even
    in FP64 with identical step sequences.  FP32 runs at tol 1e-8: at 1e-6
    the oracle's own end states move by more than 1e-5 between tol and
    tol/100."""
    a = 0.9
    ctx = K.kerr_init(a)
    y0, w0 = photons(a)
    t_end = -100.0
    out = run(ctx, y0, w0, t_end, K.default_opts(prec=prec, tol=tol))
    oo = O.Opts(tol=tol)
    ref = O.trace_coordtime(a, y0[:, 0], w0, t_end, oo)
    flags = coordtime_flags(a, y0, w0, t_end, oo, ref, gate, prec == K.FP32_KAHAN)
    assert flags.mean() <= 0.12, flags.sum()
    good = ~flags
    st = out.status.cpu().numpy()
    x = out.x.cpu().numpy().T
    v = out.v.cpu().numpy().T
    assert set(np.unique(ref.status)) >= {O.CAPTURED, O.ENDTIME}
    assert np.array_equal(st[good], ref.status[good])
    end = good & (ref.status == O.ENDTIME)
    assert end.sum() > 200
    assert np.all(x[end, 0] == t_end)              # lands on the end time exactly
    e = coordtime_err(np.concatenate([x[:, 1:], v], axis=1), ref.w)
    assert np.all(e[end] <= gate), (np.sort(e[end])[-5:], int(flags.sum()))
    print(dict(prec=prec, ill_conditioned=int(flags.sum()), max_err_endtime=float(e[end].max()),
               median_err_endtime=float(np.median(e[end]))))
    s = K.kerr_get_stats(ctx)
    assert s.geodesics == len(y0) and sum(s.status_count) == len(y0)
    ctx.close()


def test_coordtime_circular_orbit_fp64():
    a, r = 0.5, 8.0
    Om = C.omega_circular(r, a)
    ctx = K.kerr_init(a)
    w0 = np.array([[r, a, 0.0, -a * Om, r * Om, 0.0]])
    y0 = np.zeros((1, 8))
    T = 200.0
    out = run(ctx, y0, w0, T, K.default_opts(prec=K.FP64, tol=1e-14, r_escape=-1.0))
    z = (r + 1j * a) * np.exp(1j * Om * T)
    x = out.x.cpu().numpy()[:, 0]
    assert out.status.cpu().numpy()[0] == K.ENDTIME and x[0] == T
    assert abs(x[1] + 1j * x[2] - z) < 2e-9
    ctx.close()


def test_coordtime_arguments():
    ctx = K.kerr_init(0.5)
    x0 = torch.zeros((4, 2), dtype=torch.float64)
    v0 = torch.zeros((3, 2), dtype=torch.float64)
    with pytest.raises(K.KerrError):
        K.kerr_trace_coordtime(ctx, x0, v0, None, K.default_opts(t_end=10.0))   # host memory
    xd, vd = x0.to(DEV), v0.to(DEV)
    xd[1] = 20.0
    out = K.kerr_trace_coordtime(ctx, xd, vd, None, K.default_opts(t_end=0.0))  # zero length
    torch.cuda.synchronize()
    assert (out.status.cpu().numpy() == K.ENDTIME).all() and (out.steps.cpu().numpy() == 0).all()
    ctx.close()
