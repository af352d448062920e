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


@pytest.mark.parametrize("layout", [K.LAYOUT_SOA, K.LAYOUT_AOS])
@pytest.mark.parametrize("n", [1, 2, 7, 193])
def test_paired_fp32_matches_one_per_thread(rays, layout, n):
    """Two geodesics per thread on packed f32x2 instructions: the same IEEE
    operations per geodesic as one per thread (odd n: the last thread's second
    half repeats a geodesic and stores nothing), and within the FP32 gate of
    the oracle."""
    y0, ref = rays
    idx = np.arange(n) % len(y0)
    ys = y0[idx]
    mk = lambda: torch.tensor(ys.T if layout == K.LAYOUT_SOA else ys, dtype=torch.float32,
                              device=DEV).contiguous()
    one, two = mk(), mk()
    K.kerr_rk4_fixed(A, one, NSTEPS, H, layout=layout)
    K.kerr_rk4_fixed(A, two, NSTEPS, H, layout=layout, paired=True)
    torch.cuda.synchronize()
    g1, g2 = one.double().cpu().numpy(), two.double().cpu().numpy()
    # fused multiply-adds are explicit in both forms; allow a few ulps in case
    # a compiler contracts the scalar form differently
    assert np.allclose(g1, g2, rtol=1e-6, atol=0.0), np.abs(g1 - g2).max()
    got = g2.T if layout == K.LAYOUT_SOA else g2
    e = rel(got, ref[idx])
    assert e.max() < 2e-3 and np.median(e) < 3e-5


def test_paired_arguments():
    st = torch.zeros((8, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(K.KerrError):
        K.kerr_rk4_fixed(A, st, 1, H, paired=True)            # FP64 state
    st32 = torch.zeros((8, 4), dtype=torch.float32, device=DEV)
    with pytest.raises(K.KerrError):
        K.kerr_rk4_fixed(0.5, st32, 1, H, coords="bl", paired=True)   # KS only
    # an unknown precision code is rejected at the C boundary
    assert K.lib().kerr_rk4_fixed(A, 3, K.LAYOUT_SOA, st32.data_ptr(), 4, 1, H, None) != 0


def test_fp64_step_inside_the_zone_matches_oracle():
    """One FP64 RK4 step from states between 1.02 r_h and 1.5 r_h -- the FP64
    zone of the FP32 path, where f l l is large: the kernel's rearranged
    right-hand side (eqs. opt0/opti, the vector e of d l never formed) and its
    RK4 increments from stage sums against the oracle's Christoffel-form step
    (Sec. 3), component by component.  The geodesic equation is a quadratic
    form in k whatever the norm of k, so the momenta are drawn freely
    (past-directed k^t).  Each state's increment is compared relative to its
    largest component: a direct bound on the right-hand side's error there."""
    a, h, n = 0.99, 2e-3, 512
    rh = 1 + np.sqrt(1 - a * a)
    rng = np.random.default_rng(1706)
    r = rng.uniform(1.02 * rh, 1.5 * rh, n)
    th = np.arccos(rng.uniform(-0.95, 0.95, n))
    ph = rng.uniform(0, 2 * np.pi, n)
    # Kerr-Schild Cartesian position of (r, theta, phi): x + i y = (r + i a) sin(theta) e^(i phi)
    x = np.sin(th) * (r * np.cos(ph) - a * np.sin(ph))
    y = np.sin(th) * (r * np.sin(ph) + a * np.cos(ph))
    z = r * np.cos(th)
    assert max(abs(O.ks_r(a, *p) - ri) for p, ri in zip(zip(x, y, z), r)) < 1e-12
    y0 = np.column_stack([np.zeros(n), x, y, z, -rng.uniform(1.0, 3.0, n),
                          rng.uniform(-1.0, 1.0, (n, 3))])
    ref = np.stack([O.rk4_fixed(a, yi, h, 1)[-1] for yi in y0])
    st = torch.tensor(y0.T, dtype=torch.float64, device=DEV).contiguous()
    K.kerr_rk4_fixed(a, st, 1, h)
    torch.cuda.synchronize()
    got = st.cpu().numpy().T
    d_ref, d_got = ref - y0, got - y0
    e_inc = np.abs(d_got - d_ref).max(1) / np.abs(d_ref).max(1)
    assert e_inc.max() < 1e-12, e_inc.max()
    assert rel(got, ref).max() < 1e-14


def test_fixed_rk4_arguments():
    st = torch.zeros((8, 4), dtype=torch.float64, device=DEV)
    K.kerr_rk4_fixed(A, st, 0, H)                       # no-op
    with pytest.raises(K.KerrError):
        K.kerr_rk4_fixed(1.5, st, 1, H)                 # |a| > 1
    with pytest.raises(K.KerrError):
        K.kerr_rk4_fixed(A, st, 1, H, layout=7)
    with pytest.raises(K.KerrError):
        K.kerr_rk4_fixed(A, torch.zeros((8, 4), dtype=torch.float64), 1, H)   # host memory


# ---------------------------------------------------------------------------
# Boyer-Lindquist paper mode (Hamiltonian form) against the oracle's BL
# integration (Christoffel form of eq. 1, complex-step derivatives)
# ---------------------------------------------------------------------------
import closed_forms as Cf  # noqa: E402


def bl_states(a, n=24, seed=5):
    """Null BL states at r = 25 M heading inward at various angles: oracle
    form (x, k) and the GPU's (x, p = g k)."""
    rng = np.random.default_rng(seed)
    ys, ps = [], []
    for _ in range(n):
        r, th, ph = 25.0, rng.uniform(0.6, 2.5), rng.uniform(0, 2 * np.pi)
        g = Cf.bl_metric(r, th, a)
        kr, kth, kph = -1.0, rng.uniform(-0.02, 0.02), rng.uniform(-0.01, 0.01)
        # null condition for k^t (past-directed root not needed: k^t > 0)
        A = g[0, 0]
        B = 2 * g[0, 3] * kph
        Cc = g[1, 1] * kr ** 2 + g[2, 2] * kth ** 2 + g[3, 3] * kph ** 2
        kt = (-B - np.sqrt(B * B - 4 * A * Cc)) / (2 * A)
        k = np.array([kt, kr, kth, kph])
        y = np.array([0.0, r, th, ph, *k])
        ys.append(y)
        ps.append(np.array([0.0, r, th, ph, *(g @ k)]))
    return np.array(ys), np.array(ps)


@pytest.mark.parametrize("layout", [K.LAYOUT_SOA, K.LAYOUT_AOS])
def test_fixed_rk4_bl_matches_oracle(layout):
    a, h, nsteps = 0.9, 0.02, 1000                      # 20 M of path toward the hole
    ys, ps = bl_states(a)
    ref = np.stack([O.rk4_fixed(a, y, h, nsteps, stride=nsteps, coords=O.BL)[-1] for y in ys])
    st = torch.tensor(ps.T if layout == K.LAYOUT_SOA else ps, dtype=torch.float64,
                      device=DEV).contiguous()
    K.kerr_rk4_fixed(a, st, nsteps, h, layout=layout, coords="bl")
    torch.cuda.synchronize()
    got = st.cpu().numpy()
    got = got.T if layout == K.LAYOUT_SOA else got
    # positions: the same geodesic through different formulations of the same
    # equations; fixed-step truncation differs at O(h^4)
    e = np.abs(got[:, :4] - ref[:, :4]) / (1 + np.abs(ref[:, :4]))
    assert e.max() < 1e-8, e.max()
    # momenta: p = g k at the end point
    for j in range(len(ys)):
        g = Cf.bl_metric(ref[j, 1], ref[j, 2], a)
        np.testing.assert_allclose(got[j, 4:], g @ ref[j, 4:], rtol=1e-7, atol=1e-9)
    # p_t and p_phi are constants of the Hamiltonian form
    assert np.all(got[:, 4] == ps[:, 4]) and np.all(got[:, 7] == ps[:, 7])


def test_bl_camera_states_are_null_and_inward():
    a = 0.9
    cam = K.camera(a, np.radians(60.0), 1024.0, 20.0, 16, 16)
    st = K.kerr_bl_camera_states(cam).cpu().numpy().T       # (n, 8)
    assert np.all(st[:, 5] < 0)                                # p_r < 0: moving inward
    for y in st[::17]:
        g = Cf.bl_metric(y[1], y[2], a)
        p = y[4:]
        assert abs(p @ np.linalg.solve(g, p)) < 1e-9         # g^{ab} p_a p_b = 0
