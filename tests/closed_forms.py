"""Closed-form Kerr results used to pin the oracle (M = 1 throughout).

These are textbook / paper formulas written out independently of the oracle;
tests compare the oracle's numerical integrations against them.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate


def r_horizon(a: float) -> float:
    """Outer horizon r_h = 1 + sqrt(1 - a^2)."""
    return 1.0 + np.sqrt(1.0 - a * a)


def r_circular_photon(a: float) -> tuple[float, float]:
    """Prograde / retrograde circular photon orbit radii (Sec. 3.1):
    r = 2{1 + cos[(2/3) arccos(-/+|a|)]}."""
    rp = 2.0 * (1.0 + np.cos(2.0 / 3.0 * np.arccos(-abs(a))))
    rr = 2.0 * (1.0 + np.cos(2.0 / 3.0 * np.arccos(abs(a))))
    return rp, rr


def spherical_photon_constants(r: float, a: float) -> tuple[float, float]:
    """Teo (2003) constants of a spherical photon orbit at BL radius r with E = 1:
    Phi = -(r^3 - 3r^2 + a^2 r + a^2)/(a (r - 1)),
    Q   = -r^3 (r^3 - 6r^2 + 9r - 4a^2)/(a^2 (r - 1)^2)."""
    Phi = -(r ** 3 - 3 * r ** 2 + a * a * r + a * a) / (a * (r - 1.0))
    Q = -r ** 3 * (r ** 3 - 6 * r ** 2 + 9 * r - 4 * a * a) / (a * a * (r - 1.0) ** 2)
    return Phi, Q


def spherical_photon_max_cos(Phi: float, Q: float, a: float) -> float:
    """Largest |cos theta| reached: u = cos^2 theta is the positive root of the
    polar potential a^2 u^2 + (Q + Phi^2 - a^2) u - Q = 0."""
    b = Q + Phi * Phi - a * a
    u = (-b + np.sqrt(b * b + 4 * a * a * Q)) / (2 * a * a)
    return float(np.sqrt(u))


def spherical_photon_dphi(r: float, a: float) -> float:
    """Change of azimuth over one full polar oscillation of a spherical photon
    orbit (Teo 2003, eq. 17), by quadrature over mu = cos theta.

    With E = 1 the BL equations of motion give
      dphi/dmu = [a (r^2 + a^2 - a Phi)/Delta - a + Phi/(1 - mu^2)] / sqrt(Theta(mu)),
      Theta(mu) = Q (1 - mu^2) - mu^2 (Phi^2 - a^2 (1 - mu^2))   (times 1/(1-mu^2) factored),
    and one oscillation is four quarter-swings 0 -> mu_+.  Here Theta is written
    as a^2 (mu_+^2 - mu^2)(mu^2 + mu_-^2)."""
    Phi, Q = spherical_photon_constants(r, a)
    Delta = r * r - 2 * r + a * a
    b = Q + Phi * Phi - a * a
    up = (-b + np.sqrt(b * b + 4 * a * a * Q)) / (2 * a * a)
    um = (b + np.sqrt(b * b + 4 * a * a * Q)) / (2 * a * a)
    mup = np.sqrt(up)
    # substitute mu = mu_+ sin(s) to remove the endpoint singularity
    def integrand(s):
        mu = mup * np.sin(s)
        num = a * (r * r + a * a - a * Phi) / Delta - a + Phi / (1.0 - mu * mu)
        den = a * np.sqrt(mu * mu + um)
        return num / den
    val, _ = integrate.quad(integrand, 0.0, np.pi / 2, epsabs=1e-14, epsrel=1e-13, limit=200)
    return 4.0 * val


def omega_circular(r: float, a: float) -> float:
    """Prograde circular equatorial orbital frequency Omega = 1/(r^{3/2} + a)."""
    return 1.0 / (r ** 1.5 + a)


def ut_circular(r: float, a: float) -> float:
    """u^t of a prograde circular equatorial orbit (Bardeen, Press & Teukolsky 1972):
    u^t = (r^{3/2} + a) / (r^{3/4} sqrt(r^{3/2} - 3 r^{1/2} + 2a))."""
    return (r ** 1.5 + a) / (r ** 0.75 * np.sqrt(r ** 1.5 - 3 * r ** 0.5 + 2 * a))


def omega_vertical(r: float, a: float) -> float:
    """Vertical epicyclic frequency Omega_perp = Omega sqrt(1 - 4a r^{-3/2} + 3a^2 r^{-2})."""
    return omega_circular(r, a) * np.sqrt(1 - 4 * a * r ** -1.5 + 3 * a * a / (r * r))


def kappa_radial(r: float, a: float) -> float:
    """Radial epicyclic frequency kappa = Omega sqrt(1 - 6/r + 8a r^{-3/2} - 3a^2/r^2)."""
    k2 = 1 - 6 / r + 8 * a * r ** -1.5 - 3 * a * a / (r * r)
    return omega_circular(r, a) * np.sqrt(k2)


def r_isco(a: float) -> float:
    """Prograde ISCO radius (Bardeen, Press & Teukolsky 1972)."""
    z1 = 1 + (1 - a * a) ** (1 / 3) * ((1 + a) ** (1 / 3) + (1 - a) ** (1 / 3))
    z2 = np.sqrt(3 * a * a + z1 * z1)
    return 3 + z2 - np.sqrt((3 - z1) * (3 + z1 + 2 * z2))


def bl_metric(r: float, th: float, a: float) -> np.ndarray:
    """BL metric components, Sec. 2.1 eq. 1, as a 4x4 array in (t, r, th, ph)."""
    s2, c2 = np.sin(th) ** 2, np.cos(th) ** 2
    rho2 = r * r + a * a * c2
    Delta = r * r - 2 * r + a * a
    g = np.zeros((4, 4))
    g[0, 0] = -(1 - 2 * r / rho2)
    g[0, 3] = g[3, 0] = -2 * r * a * s2 / rho2
    g[1, 1] = rho2 / Delta
    g[2, 2] = rho2
    g[3, 3] = (r * r + a * a + 2 * r * a * a * s2 / rho2) * s2
    return g


def bl_to_ks_offsets(r: float, a: float) -> tuple[float, float]:
    """Antiderivatives T(r) = int 2r/Delta dr and P(r) = int a/Delta dr, so that
    t_KS = t_BL + T(r) and phi_KS = phi_BL + P(r) (ingoing Kerr-Schild).  Valid
    for r > r_+ and a < 1."""
    rp = 1 + np.sqrt(1 - a * a)
    rm = 1 - np.sqrt(1 - a * a)
    T = 2.0 / (rp - rm) * (rp * np.log(r - rp) - rm * np.log(r - rm))
    P = a / (rp - rm) * np.log((r - rp) / (r - rm))
    return T, P


def ks_cartesian(r: float, th: float, phk: float, a: float) -> np.ndarray:
    """Spherical KS (r, theta, phi) -> Cartesian KS:
    x + i y = (r + i a) sin(theta) e^{i phi},  z = r cos(theta)."""
    return np.array([(r * np.cos(phk) - a * np.sin(phk)) * np.sin(th),
                     (r * np.sin(phk) + a * np.cos(phk)) * np.sin(th),
                     r * np.cos(th)])


def bl_state_to_ks(Y: np.ndarray, a: float) -> np.ndarray:
    """Map a BL state (t, r, th, ph, k^t, k^r, k^th, k^ph) to a Cartesian KS
    state (t, x, y, z, k^t, k^x, k^y, k^z)."""
    t, r, th, ph, kt, kr, kth, kph = Y
    Delta = r * r - 2 * r + a * a
    T, P = bl_to_ks_offsets(r, a) if a < 1 else (0.0, 0.0)
    tk = t + T
    phk = ph + P
    ktk = kt + 2 * r / Delta * kr
    kphk = kph + a / Delta * kr
    X = ks_cartesian(r, th, phk, a)
    s, c = np.sin(th), np.cos(th)
    cp, sp = np.cos(phk), np.sin(phk)
    dX_dr = np.array([cp * s, sp * s, c])
    dX_dth = np.array([(r * cp - a * sp) * c, (r * sp + a * cp) * c, -r * s])
    dX_dph = np.array([-(r * sp + a * cp) * s, (r * cp - a * sp) * s, 0.0])
    K = dX_dr * kr + dX_dth * kth + dX_dph * kphk
    return np.array([tk, *X, ktk, *K])


def kerr_radial_potential(r, xi: float, eta: float, a: float):
    """R(r) = (r^2 + a^2 - a xi)^2 - Delta (eta + (xi - a)^2), E = 1 units."""
    Delta = r * r - 2 * r + a * a
    return (r * r + a * a - a * xi) ** 2 - Delta * (eta + (xi - a) ** 2)


def bardeen_curve(a: float, incl: float, n: int = 20000) -> np.ndarray:
    """Critical curve of a distant observer (Bardeen 1973) as (m, 2) points
    (alpha, beta): spherical photon orbits r in [r_p, r_r] with
    xi = -(r^3 - 3r^2 + a^2 r + a^2)/(a(r - 1)) (the Teo Phi above),
    eta = -r^3 (r^3 - 6r^2 + 9r - 4a^2)/(a^2 (r - 1)^2) (Teo's Q),
    alpha = -xi / sin i, beta = +-sqrt(eta + a^2 cos^2 i - xi^2 cot^2 i).
    a = 0: the circle of radius 3 sqrt 3."""
    if abs(a) < 1e-9:
        th = np.linspace(0, 2 * np.pi, n, endpoint=False)
        return 3 * np.sqrt(3) * np.stack([np.cos(th), np.sin(th)], axis=1)
    rp, rr = r_circular_photon(a)
    r = np.linspace(rp, rr, n)
    xi, eta = spherical_photon_constants(r, a)
    si, ci = np.sin(incl), np.cos(incl)
    b2 = eta + a * a * ci * ci - xi * xi * ci * ci / (si * si)
    ok = b2 >= 0
    al = -xi[ok] / si
    be = np.sqrt(b2[ok])
    return np.concatenate([np.stack([al, be], 1), np.stack([al, -be], 1)])
