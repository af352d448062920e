"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (Table 1), closed forms (Teo 2003, Bardeen-Press-Teukolsky),
exact identities of the geodesic equation, the Boyer-Lindquist form of the
metric (eq. 1) and brute force.  Every part of the oracle (metric, derivative,
inverse, right-hand side, RK4, step control, clipping, camera and particle set
up, constants of motion) is covered by at least one test that a plausible
mistake in it would fail.
"""
import os

import numpy as np
import pytest

import closed_forms as C
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def load_table1():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            lab, *vals = line.split()
            rows.append((lab, *map(float, vals)))
    return rows


def rand_points(rng, n, a, rmin=1.5, rmax=30.0):
    """Random KS Cartesian points outside r = rmin."""
    pts = []
    while len(pts) < n:
        r = rng.uniform(rmin, rmax)
        th = rng.uniform(0.05, np.pi - 0.05)
        ph = rng.uniform(0, 2 * np.pi)
        pts.append(np.array([rng.normal(), *C.ks_cartesian(r, th, ph, a)]))
    return pts


# ---------------------------------------------------------------------------
# metric (Sec. 2.1, eq. def:CKS / CKSr) against eq. 1 and algebraic structure
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("a", [0.0, 0.3, 0.9, 0.998])
def test_ks_radius_solves_implicit_equation(a):
    rng = np.random.default_rng(1)
    for _ in range(50):
        r, th, ph = rng.uniform(0.5, 50), rng.uniform(0, np.pi), rng.uniform(0, 6.3)
        x, y, z = C.ks_cartesian(r, th, ph, a)
        assert abs(O.ks_r(a, x, y, z) - r) <= 1e-12 * r


@pytest.mark.parametrize("a", [0.3, 0.9])
def test_ks_metric_pulls_back_to_boyer_lindquist(a):
    """J^T g_KS J = g_BL (eq. 1), J = d(t,x,y,z)_KS / d(t,r,th,ph)_BL from the
    analytic coordinate map, differentiated by complex step here."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        r, th, ph = rng.uniform(2.2, 40), rng.uniform(0.1, 3.0), rng.uniform(0, 6.3)
        Delta = r * r - 2 * r + a * a
        h = 1e-30

        def cart(rr, tt, pp):
            return np.array([(rr * np.cos(pp) - a * np.sin(pp)) * np.sin(tt),
                             (rr * np.sin(pp) + a * np.cos(pp)) * np.sin(tt),
                             rr * np.cos(tt)])
        J = np.zeros((4, 4))
        J[0, 0] = 1.0
        J[0, 1] = 2 * r / Delta
        d_r = np.imag(cart(r + 1j * h, th, ph)) / h
        d_th = np.imag(cart(r, th + 1j * h, ph)) / h
        d_ph = np.imag(cart(r, th, ph + 1j * h)) / h
        J[1:, 1] = d_r + d_ph * a / Delta
        J[1:, 2] = d_th
        J[1:, 3] = d_ph
        X = np.array([0.0, *cart(r, th, ph)])
        g = O.metric(a, X)
        np.testing.assert_allclose(J.T @ g @ J, C.bl_metric(r, th, a), rtol=0, atol=1e-11 * r * r)


@pytest.mark.parametrize("a", [0.0, 0.5, 0.99])
def test_metric_is_minkowski_plus_null_rank_one(a):
    """g - eta = f l l with l null under eta and l_0 = 1 (Sec. 2.1)."""
    rng = np.random.default_rng(3)
    eta = np.diag([-1.0, 1, 1, 1])
    for X in rand_points(rng, 30, a):
        D = O.metric(a, X) - eta
        assert D[0, 0] > 0
        l = D[0] / D[0, 0]
        np.testing.assert_allclose(D, D[0, 0] * np.outer(l, l), atol=1e-14)
        assert abs(l @ eta @ l) < 1e-13
        # f = 2 r^3/(r^4 + a^2 z^2)
        r = O.ks_r(a, *X[1:])
        assert abs(D[0, 0] - 2 * r ** 3 / (r ** 4 + a * a * X[3] ** 2)) < 1e-14


@pytest.mark.parametrize("a", [0.0, 0.7, 1.0])
def test_inverse_metric(a):
    rng = np.random.default_rng(4)
    eta = np.diag([-1.0, 1, 1, 1])
    for X in rand_points(rng, 30, a):
        g = O.metric(a, X)
        gi = O.inverse_metric(a, X)
        np.testing.assert_allclose(g @ gi, np.eye(4), atol=1e-13)
        # closed form for Kerr-Schild: g^{mn} = eta^{mn} - f l^m l^n, l^m = eta^{mn} l_n
        D = g - eta
        l = D[0] / D[0, 0]
        lu = eta @ l
        np.testing.assert_allclose(gi, eta - D[0, 0] * np.outer(lu, lu), atol=1e-13)


@pytest.mark.parametrize("a", [0.2, 0.9])
def test_metric_derivatives_match_finite_differences(a):
    rng = np.random.default_rng(5)
    for X in rand_points(rng, 10, a):
        dg = O.metric_derivs(a, X)
        for al in range(4):
            e = np.zeros(4)
            e[al] = 1e-5
            fd = (O.metric(a, X + e) - O.metric(a, X - e)) / 2e-5
            np.testing.assert_allclose(dg[al], fd, atol=1e-8)
        assert np.all(dg[0] == 0.0)  # stationary


def test_frame_dragging_sign():
    """g_{t phi} < 0 for a > 0 with d_phi = -y d_x + x d_y, as in eq. 1."""
    a = 0.8
    X = np.array([0.0, *C.ks_cartesian(5.0, 1.2, 0.3, a)])
    g = O.metric(a, X)
    xi = np.array([0.0, -X[2], X[1], 0.0])
    gtphi = g[0] @ xi
    assert gtphi < 0
    assert abs(gtphi - C.bl_metric(5.0, 1.2, a)[0, 3]) < 1e-12


# ---------------------------------------------------------------------------
# right-hand side (eq. geo): exact identities of the geodesic flow
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("a", [0.0, 0.6, 0.99])
def test_rhs_conserves_killing_quantities_pointwise(a):
    """d/dlambda of E = -p_t, L_z = p_phi and u^2 = k.p vanish identically
    along the geodesic flow; evaluate the derivative with the oracle's RHS."""
    rng = np.random.default_rng(6)
    for X in rand_points(rng, 25, a, rmin=1.2 + np.sqrt(1 - a * a)):
        k = rng.normal(size=4)
        y = np.concatenate([X, k])
        dy = O.rhs(a, y)
        acc = dy[4:]
        np.testing.assert_array_equal(dy[:4], k)
        g = O.metric(a, X)
        dg = O.metric_derivs(a, X)
        dg_k = np.einsum("amn,a->mn", dg, k)        # d/dlambda g along k
        dp = dg_k @ k + g @ acc                     # d p_m / d lambda
        scale = np.abs(dg_k @ k).max() + np.abs(g @ acc).max() + 1e-300
        assert abs(dp[0]) <= 1e-12 * scale           # E
        xi = np.array([0.0, -X[2], X[1], 0.0])
        dxi = np.array([0.0, -k[2], k[1], 0.0])     # d xi / d lambda
        p = g @ k
        dLz = dxi @ p + xi @ dp
        assert abs(dLz) <= 1e-12 * (np.abs(xi).max() * scale + np.abs(p).max() * np.abs(k).max())
        du2 = k @ dg_k @ k + 2 * k @ g @ acc
        assert abs(du2) <= 1e-12 * scale * np.abs(k).max()


def test_rhs_flat_space_limit():
    """Far from the hole the acceleration falls off as 1/r^2 (Newtonian limit)."""
    a = 0.5
    y1 = np.array([0, 1e3, 0, 0, 1.0, 0, 0.2, 0])
    y2 = np.array([0, 2e3, 0, 0, 1.0, 0, 0.2, 0])
    a1 = np.linalg.norm(O.rhs(a, y1)[5:])
    a2 = np.linalg.norm(O.rhs(a, y2)[5:])
    assert 3.5 < a1 / a2 < 4.5


# ---------------------------------------------------------------------------
# spherical photon orbits: Sec. 3.1, Table 1
# ---------------------------------------------------------------------------
def spherical_orbit_ic(r, Phi, Q, a=1.0):
    """BL state at theta = pi/2, phi = 0 with p_t = -1, p_r = 0, p_phi = Phi,
    p_theta = -sqrt(Q) ("moving upward"), mapped to Cartesian KS."""
    gi = np.linalg.inv(C.bl_metric(r, np.pi / 2, a))
    p = np.array([-1.0, 0.0, -np.sqrt(Q), Phi])
    kk = gi @ p
    Y = np.array([0.0, r, np.pi / 2, 0.0, *kk])
    y0 = C.bl_state_to_ks(Y, a)
    return y0


@pytest.mark.parametrize("row", load_table1(), ids=lambda r: r[0])
def test_table1_constants_at_start(row):
    """The printed Phi and Q agree with Teo's closed forms to the printed digits,
    and the oracle's constants of motion at the mapped start state return them."""
    lab, a, r, Phi_tab, Q_tab, mc, dphi = row
    Phi, Q = C.spherical_photon_constants(r, a)
    assert abs(Phi - Phi_tab) <= 5e-5 and abs(Q - Q_tab) <= 5e-5
    assert abs(C.spherical_photon_max_cos(Phi, Q, a) - mc) <= 5e-5
    assert abs(C.spherical_photon_dphi(r, a) - dphi) <= 5e-5
    y0 = spherical_orbit_ic(r, Phi, Q, a)
    E, Lz, Qo, u2 = O.constants(a, y0)
    assert abs(E - 1.0) < 1e-12
    assert abs(Lz - Phi) < 1e-12
    assert abs(Qo - Q) < 1e-11 * max(1, Q)
    assert abs(u2) < 1e-13


def _peak_quadratic(lam, v, i):
    """Vertex of the parabola through samples i-1, i, i+1."""
    c = np.polyfit(lam[i - 1:i + 2] - lam[i], v[i - 1:i + 2], 2)
    return c[2] - c[1] ** 2 / (4 * c[0])


@pytest.mark.parametrize("row", load_table1(), ids=lambda r: r[0])
def test_table1_max_cos_theta_and_delta_phi(row):
    """Integrate each Table 1 orbit with fixed-step RK4 (Sec. 3) and measure
    max|cos theta| by a quadratic fit to the three largest samples of the first
    peak, and Delta phi by linear interpolation of the first upward zero of
    z(phi) after one full polar oscillation; both must reproduce the table."""
    lab, a, r, Phi, Q, maxcos_tab, dphi_tab = row
    Phi_exact, Q_exact = C.spherical_photon_constants(r, a)
    y0 = spherical_orbit_ic(r, Phi_exact, Q_exact, a)
    h = 1.0 / 256
    traj = O.rk4_fixed(a, y0, h, nsteps=int(40 / h))
    lam = np.arange(traj.shape[0]) * h
    z = traj[:, 3]
    rr = np.array([O.ks_r(a, *s[1:4]) for s in traj])
    cth = z / rr
    # first local maximum of cos(theta)
    i = next(j for j in range(1, len(cth) - 1) if cth[j] >= cth[j - 1] and cth[j] > cth[j + 1])
    assert abs(_peak_quadratic(lam, cth, i) - maxcos_tab) < 6e-5
    assert abs(_peak_quadratic(lam, cth, i) - C.spherical_photon_max_cos(Phi_exact, Q_exact, a)) < 1e-7
    # Delta phi: unwrap phi, find the first down- then up-crossing of z = 0
    phi = np.unwrap(np.arctan2(traj[:, 2], traj[:, 1]))
    down = next(j for j in range(1, len(z)) if z[j - 1] > 0 >= z[j])
    up = next(j for j in range(down + 1, len(z)) if z[j - 1] < 0 <= z[j])
    w = -z[up - 1] / (z[up] - z[up - 1])
    phi_up = phi[up - 1] + w * (phi[up] - phi[up - 1])
    dphi = phi_up - phi[0]
    dd = (dphi - dphi_tab + np.pi) % (2 * np.pi) - np.pi   # Test C crosses the poles
    assert abs(dd) < 1e-3
    if lab != "C":
        assert abs(dphi - dphi_tab) < 1e-3


def test_u2_converges_at_fourth_order():
    """max|u^2| over a fixed lambda window falls as dlambda^4 (Sec. 3.1, Fig. 5)."""
    a = 1.0
    r = 1.8
    Phi, Q = C.spherical_photon_constants(r, a)
    y0 = spherical_orbit_ic(r, Phi, Q, a)
    errs = []
    for h in (1 / 16, 1 / 32, 1 / 64):
        traj = O.rk4_fixed(a, y0, h, nsteps=int(8 / h), stride=1)
        errs.append(np.abs(O.constants(a, traj)[:, 3]).max())
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 3.6) and np.all(order < 4.6), (errs, order)


# ---------------------------------------------------------------------------
# time-like orbits: Sec. 3.2
# ---------------------------------------------------------------------------
def circular_ic(r, a, kick_z=0.0, kick_r=0.0):
    """Prograde circular equatorial orbit at BL radius r: u^t (BPT 1972),
    u^phi = Omega u^t; at theta = pi/2, phi_KS = 0 the Cartesian KS position
    is (r, a, 0) and u^x = -a u^phi, u^y = r u^phi.  Optional kicks add to
    u^z / u^x and u^t is re-solved from u.u = -1 by the oracle's particle set-up."""
    ut = C.ut_circular(r, a)
    uph = C.omega_circular(r, a) * ut
    v = np.array([-a * uph + kick_r, r * uph, kick_z]) / ut
    y0, ok = O.particle_ic(a, np.array([[0.0, r, a, 0.0]]), v[None, :])
    assert ok[0]
    return y0[0]


def _crossing_times(t, s, upward=True):
    out = []
    for j in range(1, len(s)):
        if (s[j - 1] < 0 <= s[j]) if upward else (s[j - 1] > 0 >= s[j]):
            w = -s[j - 1] / (s[j] - s[j - 1])
            out.append(t[j - 1] + w * (t[j] - t[j - 1]))
    return np.array(out)


@pytest.mark.parametrize("a,r", [(0.9, 3.0), (1.0, 1.5)])
def test_circular_orbit_frequency(a, r):
    """Omega = 1/(r^{3/2} + a) from the time for phi to advance by 2 pi; the
    error falls at 4th order in the step and the orbit keeps its radius."""
    y0 = circular_ic(r, a)
    assert abs(y0[4] - C.ut_circular(r, a)) < 1e-12 * y0[4]
    errs = []
    for h in (1 / 256, 1 / 512):
        traj = O.rk4_fixed(a, y0, h, nsteps=int(2 * np.pi / C.omega_circular(r, a) / y0[4] * 1.3 / h))
        phi = np.unwrap(np.arctan2(traj[:, 2], traj[:, 1])) - np.arctan2(a, r)
        T = _crossing_times(traj[:, 0], phi - 2 * np.pi)[0]
        errs.append(abs(2 * np.pi / T / C.omega_circular(r, a) - 1))
        rr = np.array([O.ks_r(a, *s[1:4]) for s in traj])
        assert np.abs(rr - r).max() < 1e-8
    assert errs[1] < 1e-10
    assert errs[1] < errs[0] / 10 or errs[0] < 1e-12


@pytest.mark.parametrize("r", [1.3, 1.5, 2.5])
def test_vertical_epicyclic_frequency(r):
    """Sec. 3.2, Fig. 9: a = 1, vertical kick 1e-12; the interval between
    successive upward zero crossings of z(t) gives Omega_perp.  The remaining
    difference is RK4 truncation error (slow radial drift), so it must fall at
    4th order with the step."""
    a = 1.0
    y0 = circular_ic(r, a, kick_z=1e-12)
    Tp = 2 * np.pi / C.omega_vertical(r, a)
    errs = []
    for h in (1 / 512, 1 / 1024):
        traj = O.rk4_fixed(a, y0, h, nsteps=int(2.2 * Tp / y0[4] / h), stride=1)
        tz = _crossing_times(traj[:, 0], traj[:, 3])
        errs.append(abs(2 * np.pi / (tz[1] - tz[0]) / C.omega_vertical(r, a) - 1))
    assert errs[1] < 1e-8
    assert errs[1] < errs[0] / 10 or errs[1] < 1e-11


def test_radial_epicyclic_frequency():
    """Radial oscillation of a slightly eccentric orbit at r = 6, a = 0.7
    has frequency kappa (which vanishes at the ISCO)."""
    a, r = 0.7, 6.0
    y0 = circular_ic(r, a, kick_r=1e-7)
    h = 1 / 16
    Tk = 2 * np.pi / C.kappa_radial(r, a)
    traj = O.rk4_fixed(a, y0, h, nsteps=int(3.3 * Tk / y0[4] / h))
    rr = np.array([O.ks_r(a, *s[1:4]) for s in traj])
    tr = _crossing_times(traj[:, 0], rr - 0.5 * (rr.max() + rr.min()))
    T = np.diff(tr).mean()
    assert abs(2 * np.pi / T / C.kappa_radial(r, a) - 1) < 1e-4


def test_isco_separates_stable_from_plunging():
    a = 0.7
    ri = C.r_isco(a)
    assert abs(ri - 3.39313) < 1e-5
    opts = O.Opts(tol=1e-10, r_escape=-1.0, max_steps=200000,
                  t_end=40 * 2 * np.pi / C.omega_circular(ri, a))
    inside = circular_ic(0.97 * ri, a, kick_r=-1e-6)
    outside = circular_ic(1.03 * ri, a, kick_r=-1e-6)
    res = O.trace(a, np.stack([inside, outside]), opts)
    assert res.status[0] == O.CAPTURED
    assert res.status[1] == O.ENDTIME
    assert abs(O.ks_r(a, *res.y[1, 1:4]) / (1.03 * ri) - 1) < 1e-3


def test_schwarzschild_photon_sphere():
    """a = 0: the circular photon orbit sits at r = 3 (r_p = r_r = 3, Sec. 3.1)."""
    a = 0.0
    assert C.r_circular_photon(0.0) == pytest.approx((3.0, 3.0))
    gi = np.linalg.inv(C.bl_metric(3.0, np.pi / 2, 0.0))
    kk = gi @ np.array([-1.0, 0.0, 0.0, 3.0 * np.sqrt(3.0)])   # b = 3 sqrt 3
    y0 = C.bl_state_to_ks(np.array([0, 3.0, np.pi / 2, 0, *kk]), 1e-300)
    traj = O.rk4_fixed(a, y0, 1 / 256, nsteps=256 * 10)
    rr = np.array([O.ks_r(a, *s[1:4]) for s in traj])
    assert np.abs(rr - 3.0).max() < 1e-7


def test_schwarzschild_capture_threshold():
    """Bisection on the camera's alpha at beta = 0 converges to b = L/E = 3 sqrt 3."""
    a = 0.0
    opts = O.Opts(tol=1e-11)
    lo, hi = 5.0, 5.4
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        y0 = camera_ic_at(a, np.pi / 2, 1000.0, mid, 0.0)
        st = O.trace(a, y0[None, :], opts, nthreads=1).status[0]
        if st == O.CAPTURED:
            lo = mid
        else:
            hi = mid
    y0 = camera_ic_at(a, np.pi / 2, 1000.0, 0.5 * (lo + hi), 0.0)
    E, Lz, Q, u2 = O.constants(a, y0)
    assert abs(abs(Lz / E) - 3 * np.sqrt(3)) < 1e-6


def camera_ic_at(a, incl, r_obs, alpha, beta):
    """Camera ray through image point (alpha, beta): a 1x1 camera of half-width
    w whose single pixel centre is at (0, 0) shifted by the requested point."""
    # Use a 2 x 1 camera where pixel 1's centre is at alpha: w = alpha for nx=2 gives
    # centres at -alpha/2.. so instead build from a 1-pixel camera and translate.
    y0 = O.camera_ic(a, incl, r_obs, 1.0, 1, 1, [0])[0]
    si, ci = np.sin(incl), np.cos(incl)
    y0[1:4] = r_obs * np.array([si, 0, ci]) + alpha * np.array([0, 1.0, 0]) + beta * np.array([-ci, 0, si])
    # re-solve k^t for the new position with the oracle's null condition
    y0[4] = 0.0
    return _null_kt(a, y0)


def _null_kt(a, y):
    g = O.metric(a, y[:4])
    k = y[5:8]
    A = g[0, 0]
    B = 2 * g[0, 1:] @ k
    Cc = k @ g[1:, 1:] @ k
    y = y.copy()
    y[4] = min(np.roots([A, B, Cc]).real)
    return y


# ---------------------------------------------------------------------------
# Kerr shadow: capture status against the radial potential (brute force)
# ---------------------------------------------------------------------------
def test_camera_capture_matches_radial_potential():
    """Config of the 64x64, a = 0.9, i = 60 deg camera: a ray is captured iff
    R(r) has no root outside the horizon, with xi = L_z/E, eta = Q/E^2 exact
    from the initial state.  Rays within 1e-6 of the critical curve (where the
    minimum of R is ~0) are skipped."""
    a, incl = 0.9, np.radians(60)
    n = 64
    idx = np.arange(n * n)
    y0 = O.camera_ic(a, incl, 1000.0, 20.0, n, n, idx)
    res = O.trace(a, y0, O.Opts(tol=1e-10))
    consts = O.constants(a, y0)
    xi = consts[:, 1] / consts[:, 0]
    eta = consts[:, 2] / consts[:, 0] ** 2
    rh = C.r_horizon(a)
    rgrid = rh + np.geomspace(1e-6, 1000.0, 20000)
    checked = 0
    for j in idx:
        R = C.kerr_radial_potential(rgrid, xi[j], eta[j], a)
        scale = rgrid ** 4
        m = (R / scale).min()
        if abs(m) < 1e-6:
            continue
        captured = m > 0
        assert (res.status[j] == O.CAPTURED) == captured, j
        checked += 1
    assert checked > 4000
    assert set(np.unique(res.status)) <= {O.CAPTURED, O.ESCAPED}
    assert (res.status == O.CAPTURED).sum() > 100


# ---------------------------------------------------------------------------
# Boyer-Lindquist integration agrees at equal affine parameter
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("timelike", [False, True])
def test_bl_and_ks_integrations_agree(timelike):
    a = 0.6
    r0, th0 = 8.0, 1.1
    gbl = C.bl_metric(r0, th0, a)
    kr, kth, kph = -0.3, 0.02, 0.015
    # k^t from the norm condition in BL
    target = -1.0 if timelike else 0.0
    A = gbl[0, 0]
    B = 2 * gbl[0, 3] * kph
    Cc = gbl[1, 1] * kr ** 2 + gbl[2, 2] * kth ** 2 + gbl[3, 3] * kph ** 2 - target
    kt = max(np.roots([A, B, Cc]).real)
    Y0 = np.array([0.0, r0, th0, 0.3, kt, kr, kth, kph])
    h, n = 1 / 64, 64 * 12
    ybl = O.rk4_fixed(a, Y0, h, n, stride=n, coords=O.BL)[-1]
    yks = O.rk4_fixed(a, C.bl_state_to_ks(Y0, a), h, n, stride=n)[-1]
    np.testing.assert_allclose(yks, C.bl_state_to_ks(ybl, a), rtol=0, atol=2e-9)


# ---------------------------------------------------------------------------
# set-up helpers
# ---------------------------------------------------------------------------
def test_camera_initial_conditions():
    a, incl, ro, w, nx, ny = 0.99, np.radians(17), 1000.0, 25.0, 8, 6
    y = O.camera_ic(a, incl, ro, w, nx, ny, np.arange(nx * ny))
    n_hat = np.array([np.sin(incl), 0, np.cos(incl)])
    eb = np.array([-np.cos(incl), 0, np.sin(incl)])
    for idx in range(nx * ny):
        p, q = idx % nx, idx // nx
        al = -w + (p + 0.5) * 2 * w / nx
        be = -w + (q + 0.5) * 2 * w / ny
        np.testing.assert_allclose(y[idx, 1:4], ro * n_hat + al * np.array([0, 1, 0]) + be * eb,
                                   rtol=1e-15, atol=1e-12)
        np.testing.assert_allclose(y[idx, 5:8], -n_hat, atol=1e-15)
        assert y[idx, 0] == 0.0
        assert y[idx, 4] < 0                                  # past-directed
        assert abs(O.constants(a, y[idx])[3]) < 1e-14         # null
    # mirror symmetry of pixel centres
    assert y[0, 2] == -y[nx - 1, 2]


def test_particle_initial_conditions():
    a = 0.7
    rng = np.random.default_rng(7)
    x = np.zeros((20, 4))
    x[:, 1:] = rng.normal(size=(20, 3)) * 20
    v = rng.normal(size=(20, 3)) * 0.1
    y, ok = O.particle_ic(a, x, v)
    assert ok.all()
    u2 = O.constants(a, y)[:, 3]
    np.testing.assert_allclose(u2, -1.0, atol=1e-13)
    np.testing.assert_allclose(y[:, 5:8] / y[:, 4:5], v, rtol=1e-14)
    # superluminal coordinate velocity far from the hole is rejected
    _, ok = O.particle_ic(a, np.array([[0, 100.0, 0, 0]]), np.array([[1.2, 0, 0]]))
    assert not ok[0]


# ---------------------------------------------------------------------------
# adaptive controller, termination and clipping (the project's reading)
# ---------------------------------------------------------------------------
def test_endpoints_lie_on_termination_surfaces():
    a = 0.99
    idx = np.arange(0, 64 * 64, 37)
    y0 = O.camera_ic(a, np.radians(17), 1000.0, 25.0, 64, 64, idx)
    res = O.trace(a, y0, O.Opts(tol=1e-6))
    rh = C.r_horizon(a)
    r_end = np.array([O.ks_r(a, *s[1:4]) for s in res.y])
    r_start = np.array([O.ks_r(a, *s[1:4]) for s in y0])
    cap = res.status == O.CAPTURED
    esc = res.status == O.ESCAPED
    assert cap.sum() > 0 and esc.sum() > 0 and cap.sum() + esc.sum() == len(idx)
    assert np.abs(r_end[cap] / (1.01 * rh) - 1).max() <= 1.01e-12
    assert np.abs(r_end[esc] / r_start[esc] - 1).max() <= 1.01e-12
    # escaped rays leave outward
    assert np.all(np.einsum("ij,ij->i", res.y[esc, 1:4], res.y[esc, 5:8]) > 0)


def test_tolerance_controls_endpoint_error():
    """Endpoint error shrinks with tol at roughly the controller's order."""
    a = 0.9
    idx = np.array([5, 700, 1500, 2300, 3100, 3900])
    y0 = O.camera_ic(a, np.radians(60), 1000.0, 20.0, 64, 64, idx)
    ref = O.trace(a, y0, O.Opts(tol=1e-13))
    e = []
    for tol in (1e-6, 1e-8):
        r = O.trace(a, y0, O.Opts(tol=tol))
        assert (r.status == ref.status).all()
        e.append(np.abs(r.y[:, 1:] - ref.y[:, 1:]).max() / np.abs(ref.y[:, 1:]).max())
    assert e[0] < 5e-5 and e[1] < 2e-6
    assert e[1] < e[0] / 10


def test_conservation_along_adaptive_integration():
    """E, L_z, Q and u^2 stay constant along adaptive integrations; the allowed
    drift follows the mixed error scale tol (1 + |y_i|), which near the horizon
    grows with |k^t|."""
    a = 0.9
    idx = np.concatenate([np.arange(0, 4096, 97), 64 * np.arange(28, 36) + 32])
    y0 = O.camera_ic(a, np.radians(60), 1000.0, 20.0, 64, 64, idx)
    res = O.trace(a, y0, O.Opts(tol=1e-10))
    c0 = O.constants(a, y0)
    c1 = O.constants(a, res.y)
    esc = res.status == O.ESCAPED
    cap = res.status == O.CAPTURED
    assert esc.sum() > 10 and cap.sum() > 3
    d = np.abs(c1 - c0)
    assert d[esc, 0].max() < 2e-8
    assert d[esc, 1].max() < 2e-8 * np.abs(c0[:, 1]).max()
    assert d[esc, 2].max() < 2e-8 * np.abs(c0[:, 2]).max()
    assert d[esc, 3].max() < 2e-8
    kt = np.abs(res.y[:, 4])
    assert np.all(d[cap, 0] < 1e-9 * kt[cap])
    assert np.all(d[cap, 1] < 1e-9 * kt[cap] * np.abs(c0[:, 1]).max())
    assert np.all(d[cap, 3] < 1e-9 * kt[cap] ** 2)


def test_degenerate_inputs():
    a = 0.9
    rh = C.r_horizon(a)
    inside = np.array([0, 1.005 * rh, 0, 0, -1.0, 0.1, 0, 0])
    nan = np.array([0, np.nan, 0, 0, -1.0, 0.1, 0, 0])
    far = O.camera_ic(a, 1.0, 1000.0, 20.0, 4, 4, [5])[0]
    res = O.trace(a, np.stack([inside, nan, far]), O.Opts(tol=1e-8, max_steps=5))
    assert res.status.tolist() == [O.CAPTURED, O.NONFINITE, O.MAXSTEPS]
    assert res.attempts.tolist() == [0, 0, 5]
    np.testing.assert_array_equal(res.y[0], inside)
    assert O.trace(a, np.zeros((0, 8)), O.Opts()).y.shape == (0, 8)


def test_renormalisation_keeps_null_constraint():
    """Re-solving k^t after every accepted step keeps u^2 at rounding level and
    stays on the past-directed branch (k^t continuous, not the other root)."""
    a = 0.99
    y0 = O.camera_ic(a, np.radians(17), 1000.0, 25.0, 64, 64, [2080, 2100])
    plain = O.trace(a, y0, O.Opts(tol=1e-6))
    ren = O.trace(a, y0, O.Opts(tol=1e-6, renorm_every=1))
    assert (plain.status == ren.status).all()
    u_plain = np.abs(O.constants(a, plain.y)[:, 3])
    u_ren = np.abs(O.constants(a, ren.y)[:, 3])
    kt = np.abs(ren.y[:, 4])
    # the last (terminating) step is not re-normalised: one step's drift remains
    assert np.all(u_ren < 1e-9 * np.maximum(1.0, kt) ** 2)
    assert np.all(u_ren < u_plain)
    np.testing.assert_allclose(ren.y[:, 4], plain.y[:, 4], rtol=1e-3)


def test_time_surface_for_particles():
    a = 0.7
    y0 = circular_ic(10.0, a)
    res = O.trace(a, y0[None], O.Opts(tol=1e-10, r_escape=-1.0, t_end=500.0))
    assert res.status[0] == O.ENDTIME
    assert abs(res.y[0, 0] - 500.0) < 1e-9


# ---------------------------------------------------------------------------
# equatorial-crossing labels (the surrogate's targets)
# ---------------------------------------------------------------------------
def test_crossing_labels_schwarzschild_face_on():
    """a = 0, face-on camera: every orbital plane contains the z axis, so the
    first equatorial crossing is where the in-plane angle, measured from the
    z axis, reaches pi/2.  With u = 1/r and b = L/E from the start state,
    phi(u) = phi0 + int_{u0}^{u} du / sqrt(1/b^2 - u^2 + 2u^3) (inward branch)
    gives r1 by quadrature; a prograde Keplerian emitter there has
    g = sqrt(1 - 3/r1) (L_z = 0 for this camera)."""
    from scipy import integrate, optimize
    a, r_obs = 0.0, 1000.0
    pts = [(6.0, 0.0), (0.0, 9.0), (-12.0, 4.0), (15.0, -15.0)]
    y0 = np.stack([camera_ic_at(a, 0.0, r_obs, al, be) for al, be in pts])
    res = O.trace(a, y0, O.Opts(tol=1e-11), crossings=True)
    for j, (al, be) in enumerate(pts):
        E, Lz, Q, u2 = O.constants(a, y0[j])
        # total angular momentum from Carter's constant at a = 0: L^2 = Q + L_z^2
        b = np.sqrt(Q + Lz ** 2) / abs(E)
        u0 = 1.0 / O.ks_r(a, *y0[j, 1:4])
        phi0 = np.arctan2(np.hypot(y0[j, 1], y0[j, 2]), y0[j, 3])

        def ang(u):
            return phi0 + integrate.quad(lambda w: 1.0 / np.sqrt(1 / b ** 2 - w * w + 2 * w ** 3),
                                         u0, u, epsabs=1e-13, epsrel=1e-12, limit=200)[0]
        # periastron: largest root below u where 1/b^2 - u^2 + 2u^3 = 0
        up = optimize.brentq(lambda w: 1 / b ** 2 - w * w + 2 * w ** 3, u0, 1.0 / 3.0)
        assert ang(up * (1 - 1e-12)) > np.pi / 2          # crosses before periastron
        u1 = optimize.brentq(lambda w: ang(w) - np.pi / 2, u0, up * (1 - 1e-12), xtol=1e-15)
        r1 = 1.0 / u1
        assert res.status[j] == O.ESCAPED
        assert abs(res.cross[j, 0] / r1 - 1) < 1e-8, (j, res.cross[j, 0], r1)
        if r1 >= 6.0:                                   # ISCO of a = 0
            assert abs(res.cross[j, 4] - np.sqrt(1 - 3 / r1)) < 1e-8
        else:
            assert np.isnan(res.cross[j, 4])
        # azimuth: the first crossing lies on the start's side of the axis
        wrap = lambda p: (p + np.pi) % (2 * np.pi) - np.pi
        az = np.arctan2(y0[j, 2], y0[j, 1])
        assert abs(wrap(res.cross[j, 1] - az)) < 1e-9
        # second crossing: in-plane angle 3 pi / 2, on the outward branch
        # after periastron (angle there: ang(up)), or absent if the total
        # swept angle to infinity stays below 3 pi / 2
        phi_p = ang(up * (1 - 1e-12))

        def ang_out(u):
            return phi_p + integrate.quad(lambda w: 1.0 / np.sqrt(1 / b ** 2 - w * w + 2 * w ** 3),
                                          u, up * (1 - 1e-12), epsabs=1e-13, epsrel=1e-12,
                                          limit=200)[0]
        total = ang_out(1e-300)
        if total > 1.5 * np.pi:
            u2c = optimize.brentq(lambda w: ang_out(w) - 1.5 * np.pi, 1e-12, up * (1 - 1e-12),
                                  xtol=1e-15)
            assert abs(res.cross[j, 2] * u2c - 1) < 1e-7, (j, res.cross[j, 2], 1 / u2c)
            assert abs(wrap(res.cross[j, 3] - az - np.pi)) < 1e-9
        elif total < 1.5 * np.pi - 1e-3:
            assert np.isnan(res.cross[j, 2])


def test_crossing_labels_are_on_the_plane_and_ordered():
    a = 0.9
    y0 = O.camera_ic(a, np.radians(75), 1000.0, 15.0, 24, 24, np.arange(576))
    res = O.trace(a, y0, O.Opts(tol=1e-9), crossings=True)
    c = res.cross
    has1 = ~np.isnan(c[:, 0])
    has2 = ~np.isnan(c[:, 2])
    assert has1.sum() > 400 and has2.sum() > 10
    assert not np.any(has2 & ~has1)                     # second only after first
    assert np.all((c[has1, 1] > -np.pi) & (c[has1, 1] <= np.pi))
    rh = C.r_horizon(a)
    assert np.all(c[has1, 0] > rh)
    g_ok = ~np.isnan(c[:, 4])
    assert np.all(c[g_ok, 0] >= C.r_isco(a) - 1e-9) and g_ok.sum() > 100
    assert np.all(np.isnan(c[has1 & ~g_ok, 4]))


# ---------------------------------------------------------------------------
# coordinate-time form (Sec. 2.2, eq. geo_t)
# ---------------------------------------------------------------------------
def test_coordtime_matches_affine_integration():
    """The same photons integrated in coordinate time and in the affine
    parameter (with the end-time event) end at the same events: positions
    and v = k^i / k^t agree to the tolerance at t = t_end."""
    a, incl, r_obs = 0.9, np.radians(60.0), 50.0
    idx = np.array([3, 20, 27, 36, 45, 60])           # 8 x 8 image, +-12 M: near passes
    y0 = O.camera_ic(a, incl, r_obs, 12.0, 8, 8, idx)
    t_end = -70.0                                      # past-directed: t decreases
    aff = O.trace(a, y0, O.Opts(tol=1e-12, t_end=t_end, r_escape=-1.0))
    assert np.all(aff.status == O.ENDTIME)
    w0 = np.concatenate([y0[:, 1:4], y0[:, 5:8] / y0[:, 4:5]], axis=1)
    ct = O.trace_coordtime(a, y0[:, 0], w0, t_end, O.Opts(tol=1e-12, r_escape=-1.0))
    assert np.all(ct.status == O.ENDTIME) and np.all(ct.t == t_end)
    rmin = min(np.min(np.linalg.norm(O.rk4_fixed(a, y, 0.25, 400, stride=4)[:, 1:4], axis=1))
               for y in y0)
    assert rmin < 10.0                                 # the window reaches the strong field
    np.testing.assert_allclose(ct.w[:, :3], aff.y[:, 1:4], rtol=0, atol=1e-7)
    np.testing.assert_allclose(ct.w[:, 3:], aff.y[:, 5:8] / aff.y[:, 4:5], rtol=0, atol=1e-8)


def test_coordtime_circular_orbit():
    """A prograde circular equatorial orbit in coordinate time: in Cartesian
    KS coordinates x + i y = (r + i a) e^{i Omega t} with Omega = 1/(r^{3/2} + a)
    (the KS and BL azimuths differ by a function of r only)."""
    a, r = 0.5, 8.0
    Om = C.omega_circular(r, a)
    w0 = np.array([[r, a, 0.0, -a * Om, r * Om, 0.0]])
    T = 200.0                                          # ~1.4 orbits
    z = (r + 1j * a) * np.exp(1j * Om * T)
    v = 1j * Om * z
    errs = []
    for tol in (1e-10, 1e-14):
        ct = O.trace_coordtime(a, 0.0, w0, T, O.Opts(tol=tol, r_escape=-1.0))
        assert ct.status[0] == O.ENDTIME and ct.t[0] == T
        assert abs(ct.w[0, 2]) < 1e-12 and abs(ct.w[0, 5]) < 1e-12
        errs.append(abs(ct.w[0, 0] + 1j * ct.w[0, 1] - z))
    # the global error of the local-error controller shrinks like tol^(4/5)
    assert errs[1] < 2e-9 and errs[0] / errs[1] > 500
    assert abs(ct.w[0, 3] + 1j * ct.w[0, 4] - v) < 2e-10


def test_coordtime_terminations():
    """Capture, escape and the exact end time in coordinate time."""
    a = 0.7
    # radial infall from rest at r = 6 on the axis: captured
    cap = O.trace_coordtime(a, 0.0, [[0.0, 0.0, 6.0, 0.0, 0.0, 0.0]], 1e4, O.Opts(tol=1e-9))
    assert cap.status[0] == O.CAPTURED
    # outgoing photon far away: escapes beyond its start radius (r_escape = 0)
    esc = O.trace_coordtime(a, 0.0, [[30.0, 0.0, 0.0, 1.0, 0.0, 0.0]], 1e4,
                            O.Opts(tol=1e-9, r_escape=0.0))
    assert esc.status[0] == O.ESCAPED
    # zero-length interval and attempt cap
    z = O.trace_coordtime(a, 5.0, [[30.0, 0.0, 0.0, 0.5, 0.0, 0.0]], 5.0, O.Opts())
    assert z.status[0] == O.ENDTIME and z.attempts[0] == 0
    m = O.trace_coordtime(a, 0.0, [[30.0, 0.0, 0.0, 0.0, 0.1, 0.0]], 1e6,
                          O.Opts(tol=1e-9, max_steps=3, r_escape=-1.0))
    assert m.status[0] == O.MAXSTEPS and m.attempts[0] == 3


def test_redshift_label_sign_convention():
    """g1 = 1 / (u^t (1 - Omega xi)) with xi = L_z / E of the ray, for a
    prograde Keplerian emitter (a = 0: u^t = 1/sqrt(1 - 3/r), Omega = r^{-3/2}):
    photons moving with the disk's rotation (xi > 0) are blueshifted relative
    to those moving against it.  Checked at the oracle's own first crossing
    radius, with xi from the start state's constants."""
    a, incl, r_obs = 0.0, np.radians(60.0), 1000.0
    pts = [(12.0, 4.0), (-12.0, 4.0), (9.0, -6.0), (-9.0, -6.0)]
    y0 = np.stack([camera_ic_at(a, incl, r_obs, al, be) for al, be in pts])
    res = O.trace(a, y0, O.Opts(tol=1e-10), crossings=True)
    gs = []
    for j in range(len(pts)):
        E, Lz, Q, u2 = O.constants(a, y0[j])
        xi = Lz / E
        r1 = res.cross[j, 0]
        assert r1 > 6.0
        want = np.sqrt(1 - 3 / r1) / (1 - r1 ** -1.5 * xi)
        assert abs(res.cross[j, 4] - want) < 1e-7, (j, res.cross[j, 4], want)
        gs.append((xi, res.cross[j, 4]))
    # the two mirror-image pairs: the sign of xi decides blue- or redshift
    for (x1, g1), (x2, g2) in ((gs[0], gs[1]), (gs[2], gs[3])):
        assert np.sign(x1) == -np.sign(x2) and (g1 - g2) * (x1 - x2) > 0


# ---------------------------------------------------------------------------
# the conditioning test's FP32 rounding model (test infrastructure of the
# end-point comparison; the plain integration is unchanged)
# ---------------------------------------------------------------------------
def test_noise_mode_is_off_by_default_and_reproducible():
    y0 = O.camera_ic(0.9, np.radians(60.0), 1000.0, 20.0, 16, 16, np.arange(256))
    plain = O.trace(0.9, y0, O.Opts(tol=1e-6))
    zero = O.trace(0.9, y0, O.Opts(tol=1e-6, noise=0.0, noise_zone=1.5, noise_seed=5))
    assert np.array_equal(plain.y, zero.y) and np.array_equal(plain.attempts, zero.attempts)
    n1 = O.trace(0.9, y0, O.Opts(tol=1e-6, noise=2.0 ** -21, noise_zone=1.5, noise_seed=1))
    n1b = O.trace(0.9, y0, O.Opts(tol=1e-6, noise=2.0 ** -21, noise_zone=1.5, noise_seed=1))
    n2 = O.trace(0.9, y0, O.Opts(tol=1e-6, noise=2.0 ** -21, noise_zone=1.5, noise_seed=2))
    assert np.array_equal(n1.y, n1b.y)                 # one seed, one draw
    assert not np.array_equal(n1.y, n2.y)              # another seed, another draw
    assert not np.array_equal(n1.y, plain.y)


def test_noise_mode_stays_outside_its_zone_and_is_small():
    # a zone radius beyond every step's start: no step is perturbed
    y0 = O.camera_ic(0.9, np.radians(60.0), 1000.0, 20.0, 8, 8, np.arange(64))
    plain = O.trace(0.9, y0, O.Opts(tol=1e-8))
    far = O.trace(0.9, y0, O.Opts(tol=1e-8, noise=1e-3, noise_zone=1e4, noise_seed=3))
    assert np.array_equal(plain.y, far.y)
    # a wide ray (b ~ 25 M, far from the photon ring): 8-ulp kicks to every
    # increment add up, as a random walk over its steps, to a small multiple
    # of the kick -- far below the 1e-5 gate, but not nothing
    y1 = O.camera_ic(0.5, np.radians(45.0), 1000.0, 20.0, 2, 2, [0])
    p = O.trace(0.5, y1, O.Opts(tol=1e-8))
    n = O.trace(0.5, y1, O.Opts(tol=1e-8, noise=2.0 ** -21, noise_zone=0.0, noise_seed=4))
    assert p.status[0] == n.status[0] == O.ESCAPED
    dx = np.linalg.norm(n.y[0, 1:4] - p.y[0, 1:4]) / np.linalg.norm(p.y[0, 1:4])
    assert 2.0 ** -24 < dx < 2e-6
