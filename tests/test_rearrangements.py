"""The exact rearrangements behind the device arithmetic, written out in
numpy from the mathematics and checked against the oracle on the CPU:

- the Kerr-Schild radius from eq. CKSr in halved form,
  r^2 = D + sqrt(D^2 + a^2 z^2) with D = (x^2 + y^2 + z^2 - a^2) / 2;
- the geodesic acceleration of eqs. opt0/opti with the vector e of
  d_al l_i = (d_al r) e_i + M_{al i} never formed: e.k from the x, y parts
  of l.k and of (x, y, z~).k, and x'', y'' through the coefficients of
  (x, y) and (l_x, l_y), since e_{x,y} = (x_i - 2 r l_i) / s;
- the classic RK4 increment (Sec. 3) from stage sums: positions
  h k + (h^2/6)(A0 + A1 + A2), momenta (h/6)(A0 + 2 (A1 + A2) + A3).

The device kernels themselves are checked against the oracle on the GPU
(tests/test_gpu_fixed.py); these tests pin the algebra they rest on."""
import numpy as np
import pytest

from oracle import oracle as O


def ks_r_halved(a, x, y, z):
    D = 0.5 * (x * x + y * y + z * z - a * a)
    return np.sqrt(D + np.sqrt(D * D + a * a * z * z))


def accel_folded(a, s):
    """d k / d lambda at s = (t, x, y, z, k^t, k^x, k^y, k^z), folded form."""
    _, x, y, z, kt, kx, ky, kz = s
    a2 = a * a
    r2 = ks_r_halved(a, x, y, z) ** 2
    r = np.sqrt(r2)
    q, sg = r2 * r2 + a2 * z * z, r2 + a2
    hf = r * r2 / q                       # f / 2
    f = 2 * hf
    P, Q = r / sg, a / sg
    lx, ly, lz = P * x + Q * y, P * y - Q * x, z / r
    Lxy = lx * kx + ly * ky
    L = Lxy + lz * kz + kt
    zt = z + a2 * z / r2
    Kxy = x * kx + y * ky
    kr = hf * (Kxy + zt * kz)             # k . grad r
    c1 = f * (3 / r - 2 * f)
    g = -2 * f * a2 * z / q
    ez = -z / r2
    ek = (Kxy - 2 * r * Lxy) / sg + ez * kz
    gk = c1 * kr + g * kz
    dLk = kr * ek + P * (kx * kx + ky * ky) + kz * kz / r
    Ak = L * gk + f * dLk
    lf = c1 + g * lz
    at = hf * L * L * lf + Ak
    fL, FmA = f * L, -at
    hw = hf * (0.5 * L * L * c1 + fL * ek)
    fLkr, fLQ2 = fL * kr, 2 * fL * Q
    al, be = hw - fLkr / sg, FmA + 2 * P * fLkr
    ax = x * al + lx * be - fLQ2 * ky
    ay = y * al + ly * be + fLQ2 * kx
    az = zt * hw - fLkr * ez + 0.5 * L * L * g + lz * FmA
    return np.array([at, ax, ay, az])


def random_states(a, n, seed, r_hi=60.0):
    rng = np.random.default_rng(seed)
    rh = 1 + np.sqrt(1 - a * a)
    out = []
    for _ in range(n):
        r = rng.uniform(1.02 * rh, r_hi)
        th, ph = np.arccos(rng.uniform(-0.98, 0.98)), rng.uniform(0, 2 * np.pi)
        X = [(r * np.cos(ph) - a * np.sin(ph)) * np.sin(th),
             (r * np.sin(ph) + a * np.cos(ph)) * np.sin(th), r * np.cos(th)]
        out.append((r, np.array([0.0, *X, -rng.uniform(1, 3), *rng.uniform(-1, 1, 3)])))
    return out


@pytest.mark.parametrize("a", [0.0, 0.5, 0.99, 0.999])
def test_halved_radius_root(a):
    for r, s in random_states(a, 60, 3):
        assert abs(ks_r_halved(a, *s[1:4]) - r) <= 1e-13 * r
        assert abs(ks_r_halved(a, *s[1:4]) - O.ks_r(a, *s[1:4])) <= 1e-13 * r


@pytest.mark.parametrize("a", [0.0, 0.5, 0.99, 0.999])
def test_folded_acceleration_matches_christoffel_form(a):
    for _, s in random_states(a, 60, 7):
        ref = O.rhs(a, s)[4:]
        got = accel_folded(a, s)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), (got, ref)


def test_folded_acceleration_fails_without_the_e_terms():
    """The check above is sensitive to the folded terms: dropping the
    -f L (k.grad r) e_i contribution from x'' (al = hw, be = F - A.k) is
    caught."""
    a = 0.9
    _, s = random_states(a, 1, 11, r_hi=4.0)[0]
    ref = O.rhs(a, s)[4:]
    _, x, y, z, kt, kx, ky, kz = s
    full = accel_folded(a, s)
    r = O.ks_r(a, x, y, z)
    sg = r * r + a * a
    # the e-vector part of x'' alone: -f L (k.grad r) (x - 2 r l_x) / s
    lx = (r * x + a * y) / sg
    hf = r ** 3 / (r ** 4 + a * a * z * z)
    L = lx * kx + ((r * y - a * x) / sg) * ky + (z / r) * kz + kt
    kr = hf * (x * kx + y * ky + (z + a * a * z / (r * r)) * kz)
    e_part = -2 * hf * L * kr * (x - 2 * r * lx) / sg
    assert abs(e_part) > 1e-3 * np.abs(ref).max()
    assert abs((full[1] - e_part) - ref[1]) > 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("a", [0.0, 0.99])
def test_rk4_increment_from_stage_sums(a):
    h = 0.05
    for _, s in random_states(a, 20, 5, r_hi=20.0):
        F = lambda u: O.rhs(a, u)             # noqa: E731  (dy/dlambda, all 8)
        k = s[4:]
        A0 = F(s)[4:]
        s2 = s.copy(); s2[:4] += 0.5 * h * k; s2[4:] = k + 0.5 * h * A0
        A1 = F(s2)[4:]
        m2 = s2[4:]
        s3 = s.copy(); s3[:4] += 0.5 * h * m2; s3[4:] = k + 0.5 * h * A1
        A2 = F(s3)[4:]
        m3 = s3[4:]
        s4 = s.copy(); s4[:4] += h * m3; s4[4:] = k + h * A2
        A3 = F(s4)[4:]
        d_pos = h * k + h * h / 6 * (A0 + A1 + A2)
        d_mom = h / 6 * (A0 + 2 * (A1 + A2) + A3)
        ref = O.rk4_fixed(a, s, h, 1)[-1] - s
        scale = np.abs(ref).max()
        assert np.abs(d_pos - ref[:4]).max() <= 1e-13 * scale
        assert np.abs(d_mom - ref[4:]).max() <= 1e-13 * scale
