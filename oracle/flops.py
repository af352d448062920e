"""FLOP count of one geodesic right-hand side in the paper's optimised form.

TEST / MEASUREMENT INFRASTRUCTURE ONLY (used by the tests and by the
benchmark to turn counted right-hand-side evaluations into algorithmic FLOPs).

`rhs_opt` is a plain FP64 transcription of Sec. 2.1, eqs. opt0 and opti:

    x0'' =  k^al D_{0 al} - F
    xi'' = -k^al (D_{i al} - 1/2 D_{al i}) + F l^i,
    D_{be al} = g_{be ga, al} k^ga,  F = f (l^be k^al - 1/2 l^al k^be) D_{be al},

evaluated for g = eta + f l l by the product rule, with the two identities of
the Kerr-Schild vector used to drop terms that vanish exactly:
  * l is null (l^be l_be = 0, so l^be d_al l_be = 0), and
  * l is an affinely parametrised geodesic of the flat metric (l^i d_i l_be = 0),
which together reduce F to -1/2 f L^2 (l . grad f) with L = l_ga k^ga.
Running it on the `Flop` scalar counts every add, multiply, divide and square
root; a fused multiply-add counts as two FLOPs (one multiply plus one add).

The counts define the "algorithmic FLOPs per RHS" that the benchmark divides
by kernel time.  `rhs_opt` is checked against the oracle's Christoffel-form
right-hand side in the tests, so the counted algebra is the right one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field


@dataclass
class Tally:
    add: int = 0
    mul: int = 0
    div: int = 0
    sqrt: int = 0

    @property
    def flops(self) -> int:
        return self.add + self.mul + self.div + self.sqrt


class Flop:
    """Float wrapper that counts arithmetic into a shared Tally."""
    __slots__ = ("v", "t")

    def __init__(self, v: float, t: Tally):
        self.v = float(v)
        self.t = t

    def _w(self, o):
        return o.v if isinstance(o, Flop) else float(o)

    def __add__(self, o):
        self.t.add += 1
        return Flop(self.v + self._w(o), self.t)

    __radd__ = __add__

    def __sub__(self, o):
        self.t.add += 1
        return Flop(self.v - self._w(o), self.t)

    def __rsub__(self, o):
        self.t.add += 1
        return Flop(self._w(o) - self.v, self.t)

    def __mul__(self, o):
        self.t.mul += 1
        return Flop(self.v * self._w(o), self.t)

    __rmul__ = __mul__

    def __truediv__(self, o):
        self.t.div += 1
        return Flop(self.v / self._w(o), self.t)

    def __rtruediv__(self, o):
        self.t.div += 1
        return Flop(self._w(o) / self.v, self.t)

    def __neg__(self):
        return Flop(-self.v, self.t)   # sign flips are free


def fsqrt(x):
    if isinstance(x, Flop):
        x.t.sqrt += 1
        return Flop(math.sqrt(x.v), x.t)
    return math.sqrt(x)


def rhs_opt(a, a2, y, sqrt=fsqrt):
    """Optimised-form acceleration (x0'', x1'', x2'', x3'') at state y.

    `a2` = a^2 is a per-geodesic constant (computed once per ray, not per RHS)."""
    _, x, yy, z, kt, kx, ky, kz = y
    # --- metric pieces: r from eq. CKSr, f and l_al from eq. def:CKS
    R2 = x * x + yy * yy + z * z
    d = R2 - a2
    az2 = a2 * (z * z)
    r2 = 0.5 * d + sqrt(0.25 * (d * d) + az2)
    r = sqrt(r2)
    ir = 1.0 / r
    iq = 1.0 / (r2 * r2 + az2)        # 1/(r^4 + a^2 z^2)
    is_ = 1.0 / (r2 + a2)             # 1/(r^2 + a^2)
    hf = r * r2 * iq                  # f/2
    f = 2.0 * hf
    lx = (r * x + a * yy) * is_
    ly = (r * yy - a * x) * is_
    lz = z * ir
    L = kt + lx * kx + ly * ky + lz * kz          # l_ga k^ga
    # --- gradient of r (implicit differentiation of eq. CKSr)
    rx = hf * x
    ry = hf * yy
    rz = hf * z * (1.0 + a2 * (ir * ir))
    # --- gradient of f
    c1 = f * (3.0 * ir - 2.0 * f)
    fx = c1 * rx
    fy = c1 * ry
    fz = c1 * rz - f * 2.0 * a2 * z * iq
    # --- d_al l_i = r_al e_i + M_{al i}
    ex = is_ * (x - 2.0 * r * lx)
    ey = is_ * (yy - 2.0 * r * ly)
    ez = -lz * ir
    ek = ex * kx + ey * ky + ez * kz
    kr = rx * kx + ry * ky + rz * kz
    dLx = rx * ek + is_ * (r * kx - a * ky)      # (d_x l_ga) k^ga
    dLy = ry * ek + is_ * (a * kx + r * ky)
    dLz = rz * ek + ir * kz
    kdlx = kr * ex + is_ * (r * kx + a * ky)     # k^al d_al l_x
    kdly = kr * ey + is_ * (r * ky - a * kx)
    kdlz = kr * ez + ir * kz
    # --- D_{be al} = l_be A_al + f L d_al l_be, A_al = f_al L + f dL_al
    Ax = fx * L + f * dLx
    Ay = fy * L + f * dLy
    Az = fz * L + f * dLz
    Ak = Ax * kx + Ay * ky + Az * kz             # k^al D_{0 al}
    # --- F (null + affinely geodesic l)
    F = -0.5 * f * (L * L) * (lx * fx + ly * fy + lz * fz)
    fL = f * L
    hL = 0.5 * L
    at = Ak - F
    ax = hL * (Ax + f * dLx) - (lx * Ak + fL * kdlx) + F * lx
    ay = hL * (Ay + f * dLy) - (ly * Ak + fL * kdly) + F * ly
    az = hL * (Az + f * dLz) - (lz * Ak + fL * kdlz) + F * lz
    return at, ax, ay, az


def count_rhs() -> Tally:
    """FLOPs of one right-hand side (accelerations; x' = k costs nothing)."""
    t = Tally()
    y = [Flop(v, t) for v in (0.0, 7.0, -3.0, 5.0, -1.0, 0.3, 0.2, -0.9)]
    a = 0.7
    rhs_opt(a, a * a, y)
    return t


def count_attempt() -> Tally:
    """FLOPs of one step-doubling attempt excluding the 11 RHS evaluations:
    three classic RK4 steps (stage points for the 7 components that enter the
    RHS, the weighted sum for all 8) plus the scaled error norm over 7
    components and the compensated (Kahan) update of 8 components."""
    t = Tally()
    h = Flop(0.5, t)
    y = [Flop(1.0 + i, t) for i in range(8)]
    k = [[Flop(0.1 * (i + j), t) for i in range(8)] for j in range(4)]
    for _ in range(3):
        # stage points y + c h k_j (c h computed once per step)
        for c in (0.5, 0.5, 1.0):
            ch = h * c
            for i in range(1, 8):
                _ = y[i] + ch * k[0][i]
        h6 = h * (1.0 / 6.0)
        for i in range(8):
            _ = y[i] + h6 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i])
    # error norm: |d_i| / (tol (1 + max(|y|,|y'|))), 7 components, max is free
    for i in range(1, 8):
        d = (y[i] - y[i]) * (1.0 / 15.0)
        _ = d / (1.0 + y[i])
    # Kahan update: s = dy + c; y' = y + s; c' = s - (y' - y)
    for i in range(8):
        s_ = y[i] + y[i]
        yn = y[i] + s_
        _ = s_ - (yn - y[i])
    return t


RHS_PER_ATTEMPT = 11
