"""Paper-mode fixed-step RK4 (Sec. 3; the timing setting of Sec. 4.2): the
device kernel against the oracle's fixed-step RK4 (Christoffel-form right-hand
side, FP64) on rays that swing past the hole and escape, in both layouts and
both precisions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_1706_07062_gb300 import kerr as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
A, INCL, R_OBS, HW, SIDE = 0.999, np.radians(60.0), 30.0, 20.0, 16
H, NSTEPS = 0.5, 160


@pytest.fixture(scope="module")
def rays():
    """Pixels of a 16 x 16 image at r = 30 M whose impact parameter exceeds
    8 M: they pass within a few M of the hole inside the 80 M window and
    leave again (no horizon crossing, where fixed steps would blow up)."""
    p = (np.arange(SIDE) + 0.5) * 2 * HW / SIDE - HW
    al, be = np.meshgrid(p, p)
    idx = np.nonzero(np.hypot(al, be).ravel() > 8.0)[0]
    y0 = O.camera_ic(A, INCL, R_OBS, HW, SIDE, SIDE, idx)
    ref = np.stack([O.rk4_fixed(A, y, H, NSTEPS, stride=NSTEPS)[-1] for y in y0])
    # the window really passes near the hole: smallest radius reached
    rmin = min(np.min(np.linalg.norm(O.rk4_fixed(A, y, H, NSTEPS, stride=8)[:, 1:4], axis=1))
               for y in y0[::9])
    assert rmin < 12.0
    return y0, ref


def rel(got, ref):
    return np.abs(got - ref) / (1.0 + np.abs(ref))


@pytest.mark.parametrize("layout", [K.LAYOUT_SOA, K.LAYOUT_AOS])
@pytest.mark.parametrize("dtype,gate_max,gate_med", [(torch.float64, 1e-11, 1e-13),
                                                     (torch.float32, 2e-3, 3e-5)])
def test_fixed_rk4_matches_oracle(rays, layout, dtype, gate_max, gate_med):
    y0, ref = rays
    st = torch.tensor(y0.T if layout == K.LAYOUT_SOA else y0, dtype=dtype, device=DEV).contiguous()
    K.kerr_rk4_fixed(A, st, NSTEPS, H, layout=layout)
    torch.cuda.synchronize()
    got = st.double().cpu().numpy()
    got = got.T if layout == K.LAYOUT_SOA else got
    e = rel(got, ref)
    assert np.isfinite(got).all()
    assert e.max() < gate_max and np.median(e) < gate_med, (e.max(), np.median(e))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_layouts_agree_bit_for_bit(rays, dtype):
    y0, _ = rays
    soa = torch.tensor(y0.T, dtype=dtype, device=DEV).contiguous()
    aos = torch.tensor(y0, dtype=dtype, device=DEV).contiguous()
    K.kerr_rk4_fixed(A, soa, 50, H, layout=K.LAYOUT_SOA)
    K.kerr_rk4_fixed(A, aos, 50, H, layout=K.LAYOUT_AOS)
    torch.cuda.synchronize()
    assert torch.equal(soa.T.contiguous(), aos)


def test_fixed_rk4_arguments():
    st = torch.zeros((8, 4), dtype=torch.float64, device=DEV)
    K.kerr_rk4_fixed(A, st, 0, H)                       # no-op
    with pytest.raises(K.KerrError):
        K.kerr_rk4_fixed(1.5, st, 1, H)                 # |a| > 1
    with pytest.raises(K.KerrError):
        K.kerr_rk4_fixed(A, st, 1, H, layout=7)
    with pytest.raises(K.KerrError):
        K.kerr_rk4_fixed(A, torch.zeros((8, 4), dtype=torch.float64), 1, H)   # host memory
