"""Stored solutions and root finding on them (Sec. 2.2, the second way of
matching a target time) against the oracle's end-time event (root finding
during the integration, on actual RK4 sub-steps)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_1706_07062_gb300 import kerr as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_find_time_on_stored_solution_matches_oracle_event():
    a = 0.9
    idx = np.arange(0, 256, 3)
    y0 = O.camera_ic(a, np.radians(60.0), 50.0, 12.0, 16, 16, idx)
    ctx = K.kerr_init(a)
    x0 = torch.tensor(y0[:, :4].T.copy(), device=DEV)
    k0 = torch.tensor(y0[:, 4:].T.copy(), device=DEV)
    opts = K.default_opts(prec=K.FP64, tol=1e-10)       # escape beyond the start radius
    out, traj, cnt = K.kerr_trace_rays_dense(ctx, x0, k0, cap=4096, opts=opts)
    torch.cuda.synchronize()
    c = cnt.cpu().numpy()
    assert (c >= 2).all() and (c < 4096).all()
    # the stored end point is the trace's end point
    tr = traj.cpu().numpy()
    last = tr[np.arange(len(idx)), c - 1, 1:]
    np.testing.assert_array_equal(last, np.concatenate([out.x.cpu().numpy(), out.k.cpu().numpy()]).T)
    full = O.trace(a, y0, O.Opts(tol=1e-10))               # where each integration ends
    for t_star in (-35.0, -80.0, -120.0):
        tt = torch.full((len(idx),), t_star, dtype=torch.float64, device=DEV)
        y, lam, found = K.kerr_dense_find_time(a, traj, cnt, tt)
        torch.cuda.synchronize()
        f = found.cpu().numpy().astype(bool)
        # found exactly when the integration passes t_star before it ends
        # (t decreases along these past-directed rays)
        assert np.array_equal(f, full.y[:, 0] <= t_star)
        got = y.cpu().numpy().T
        assert np.all(np.isfinite(got[f])) and np.all(np.isnan(got[~f]))
        assert np.max(np.abs(got[f, 0] - t_star)) < 1e-11 * (1 + abs(t_star))
        # states against the oracle's end-time event where that event fires
        # (a step that also crosses the escape radius reports the escape)
        ref = O.trace(a, y0, O.Opts(tol=1e-10, t_end=t_star))
        m = f & (ref.status == O.ENDTIME)
        assert m.sum() >= 5
        e = np.abs(got[m, 1:] - ref.y[m, 1:]) / (1 + np.abs(ref.y[m, 1:]))
        assert np.median(e) < 1e-8 and e.max() < 1e-6, (np.median(e), e.max())
    ctx.close()


def test_dense_requires_fp64_and_device_buffers():
    ctx = K.kerr_init(0.5)
    x0 = torch.zeros((4, 2), dtype=torch.float64, device=DEV)
    k0 = torch.zeros((4, 2), dtype=torch.float64, device=DEV)
    with pytest.raises(K.KerrError):
        K.kerr_trace_rays_dense(ctx, x0, k0, cap=8, opts=K.default_opts())     # FP32 path
    ctx.close()
