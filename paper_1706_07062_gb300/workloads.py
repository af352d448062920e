"""Seeded synthetic workloads shaped like the paper's (arXiv:1706.07062, Sec. 4:
backward null geodesics from a distant image plane; Sec. 3.2: massive
particles on bound orbits).

This module only draws inputs: camera geometries, seeded subsets and
Newtonian orbital elements converted to a start position and coordinate
velocity.  It holds none of the geodesic method's arithmetic (no metric, no
right-hand side, no normalisation), so both the CUDA path and the CPU oracle
can take its outputs as their inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DEG = math.pi / 180.0


@dataclass(frozen=True)
class CameraSpec:
    a: float
    incl: float         # radians
    r_obs: float
    half_width: float
    nx: int
    ny: int

    @property
    def n(self) -> int:
        return self.nx * self.ny

    def as_tuple(self):
        return (self.a, self.incl, self.r_obs, self.half_width, self.nx, self.ny)


# 64 x 64 image, a = 0.9, i = 60 deg, r_obs = 1000, alpha, beta in [-20, 20],
# tolerance 1e-10, FP64: the small case the oracle runs in full.
CAMERA_64 = CameraSpec(0.9, 60 * DEG, 1000.0, 20.0, 64, 64)
TOL_64 = 1e-10

# 1024 x 1024 image, a = 0.99, i = 17 deg, image plane +-25, tolerance 1e-6.
CAMERA_1024 = CameraSpec(0.99, 17 * DEG, 1000.0, 25.0, 1024, 1024)
TOL_1024 = 1e-6
SUBSET_SEED_1024 = 1706


def camera_subset(spec: CameraSpec, k: int = 4096, seed: int = SUBSET_SEED_1024) -> np.ndarray:
    """Sorted seeded subset of k ray indices (without replacement)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(spec.n, size=min(k, spec.n), replace=False))


# ---------------------------------------------------------------------------
# 64 uneven images in one launch
# ---------------------------------------------------------------------------
BATCH_SEED = 1708
BATCH_SIDES = (128, 256, 512, 1024, 2048)


def camera_batch(n_images: int = 64, seed: int = BATCH_SEED, r_obs: float = 1000.0,
                 half_width: float = 25.0, sides=BATCH_SIDES) -> list[CameraSpec]:
    """Images with sides drawn uniformly from `sides`, spin a ~ U[0, 0.998],
    inclination ~ U[5, 85] deg, observer at r_obs, image plane +-half_width."""
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sides), size=n_images)
    a = rng.uniform(0.0, 0.998, size=n_images)
    inc = rng.uniform(5.0, 85.0, size=n_images) * DEG
    return [CameraSpec(float(a[i]), float(inc[i]), r_obs, half_width, int(side[i]), int(side[i]))
            for i in range(n_images)]


# ---------------------------------------------------------------------------
# particles: bound orbits with seeded elements
# ---------------------------------------------------------------------------
PARTICLE_SPIN = 0.7
PARTICLE_SEED = 1707
PARTICLE_PERIODS = 100


@dataclass
class ParticleSet:
    a: float
    x0: np.ndarray       # (4, n) start events (t = 0)
    v0: np.ndarray       # (3, n) coordinate velocities dx/dt
    t_end: np.ndarray    # (n,) end times: PARTICLE_PERIODS Newtonian radial periods
    semi_major: np.ndarray
    ecc: np.ndarray


def kepler_state(A, e, inc, node, peri, mean_anom):
    """Newtonian (GM = 1) position and velocity from orbital elements; the
    eccentric anomaly solves E - e sin E = M by Newton iteration."""
    E = mean_anom.copy()
    for _ in range(60):
        E = E - (E - e * np.sin(E) - mean_anom) / (1.0 - e * np.cos(E))
    cE, sE = np.cos(E), np.sin(E)
    q = np.sqrt(1.0 - e * e)
    xp = A * (cE - e)
    yp = A * q * sE
    nmot = A ** -1.5
    den = 1.0 - e * cE
    vxp = -A * nmot * sE / den
    vyp = A * nmot * q * cE / den
    cO, sO = np.cos(node), np.sin(node)
    ci, si = np.cos(inc), np.sin(inc)
    cw, sw = np.cos(peri), np.sin(peri)
    # rotation R = Rz(node) Rx(inc) Rz(peri), applied to in-plane vectors
    r11 = cO * cw - sO * sw * ci
    r12 = -cO * sw - sO * cw * ci
    r21 = sO * cw + cO * sw * ci
    r22 = -sO * sw + cO * cw * ci
    r31 = sw * si
    r32 = cw * si
    pos = np.stack([r11 * xp + r12 * yp, r21 * xp + r22 * yp, r31 * xp + r32 * yp])
    vel = np.stack([r11 * vxp + r12 * vyp, r21 * vxp + r22 * vyp, r31 * vxp + r32 * vyp])
    return pos, vel


def particles(n: int = 1 << 20, seed: int = PARTICLE_SEED, a: float = PARTICLE_SPIN,
              periods: int = PARTICLE_PERIODS) -> ParticleSet:
    """Semi-major axes log-uniform in [10, 1000], eccentricity U[0, 0.9],
    isotropic orbital planes, uniform mean anomaly; integrate for `periods`
    Newtonian radial periods 2 pi A^{3/2} (or until capture)."""
    rng = np.random.default_rng(seed)
    A = np.exp(rng.uniform(np.log(10.0), np.log(1000.0), size=n))
    e = rng.uniform(0.0, 0.9, size=n)
    inc = np.arccos(rng.uniform(-1.0, 1.0, size=n))
    node = rng.uniform(0.0, 2 * np.pi, size=n)
    peri = rng.uniform(0.0, 2 * np.pi, size=n)
    M = rng.uniform(0.0, 2 * np.pi, size=n)
    pos, vel = kepler_state(A, e, inc, node, peri, M)
    x0 = np.zeros((4, n))
    x0[1:] = pos
    t_end = periods * 2 * np.pi * A ** 1.5
    return ParticleSet(a, np.ascontiguousarray(x0), np.ascontiguousarray(vel), t_end, A, e)


def particle_subset(ps: ParticleSet, k: int = 4096, seed: int = PARTICLE_SEED) -> np.ndarray:
    """Seeded subset stratified by log A: k/16 draws from each of 16 bins."""
    rng = np.random.default_rng(seed + 1)
    bins = np.linspace(np.log(10.0), np.log(1000.0), 17)
    la = np.log(ps.semi_major)
    out = []
    per = max(1, k // 16)
    for b in range(16):
        idx = np.nonzero((la >= bins[b]) & (la < bins[b + 1]))[0]
        out.append(rng.choice(idx, size=min(per, idx.size), replace=False))
    return np.sort(np.concatenate(out))


# ---------------------------------------------------------------------------
# the learned surrogate: training rays and evaluation images
# ---------------------------------------------------------------------------
SURR_TRAIN_SEED = 1710
SURR_EVAL_SEED = 1709


def surrogate_points(n: int = 10_000_000, seed: int = SURR_TRAIN_SEED,
                     half_width: float = 25.0) -> np.ndarray:
    """Training rays (n, 4): alpha, beta ~ U[-25, 25], spin a ~ U[0, 0.998],
    inclination ~ U[5, 85] deg (radians)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(-half_width, half_width, n),
                     rng.uniform(-half_width, half_width, n),
                     rng.uniform(0.0, 0.998, n),
                     rng.uniform(5.0, 85.0, n) * DEG], axis=1)


def surrogate_eval_cameras(n_images: int = 8, side: int = 2048, seed: int = SURR_EVAL_SEED,
                           r_obs: float = 1000.0, half_width: float = 25.0) -> list[CameraSpec]:
    """Evaluation images: spin and inclination drawn per image as for training."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 0.998, n_images)
    inc = rng.uniform(5.0, 85.0, n_images) * DEG
    return [CameraSpec(float(a[i]), float(inc[i]), r_obs, half_width, side, side)
            for i in range(n_images)]


def surrogate_init(seed: int = SURR_TRAIN_SEED) -> np.ndarray:
    """Seeded initial parameters of the surrogate in the C ABI's padded layout
    (uniform +-1/sqrt(fan_in) on the live weights, zero padding and biases)."""
    rng = np.random.default_rng(seed + 1000)
    ins, outs = [16, 256, 256, 256, 256], [256, 256, 256, 256, 64]
    live_in, live_out = [4, 256, 256, 256, 256], [256, 256, 256, 256, 8]
    parts = []
    for l in range(5):
        W = np.zeros((outs[l], ins[l]), dtype=np.float32)
        lim = 1.0 / np.sqrt(live_in[l])
        W[:live_out[l], :live_in[l]] = rng.uniform(-lim, lim, size=(live_out[l], live_in[l]))
        parts += [W.ravel(), np.zeros(outs[l], dtype=np.float32)]
    return np.concatenate(parts)
