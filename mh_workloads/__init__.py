"""Seeded synthetic workloads for the modified-Helmholtz heat solver.

This module is shared by the CPU oracle, the tests and the benchmark.  It only
*generates inputs*: boundary-node coordinates of the domains, forcing
functions, manufactured solutions and their data.  It holds none of the
method's arithmetic (no kernels, no quadrature, no derivatives, no trees).

Domains follow the paper's setting (Section 2, a bounded multiply connected
domain Omega with outer boundary Gamma_0 and holes Gamma_1..Gamma_m, each curve
parametrised on [0, 2*pi) and sampled at N equispaced parameter values,
Section 3.2).  Orientation convention used throughout the library: the outer
curve runs counter-clockwise, holes run clockwise, so that the right-hand
normal (y2', -y1')/|y'| points out of Omega.

Workloads (sizes in the docstrings of each generator):
  * ``disk_with_hole``   : unit disk minus a circle of radius 0.3 at (0.2, 0),
                            128 nodes per curve, uniform level-4 tree, 4x4
                            Gauss-Legendre nodes per leaf, dt = alpha^2 = 1e-2,
                            manufactured solution u = exp(-t) sin(pi x) cos(pi y).
  * ``starfish_domain``  : unit disk minus 5 five-armed starfish holes
                            r(t) = 0.12 (1 + 0.3 cos 5t), centres drawn with a
                            seed so that curves keep a gap >= 0.05, 1024 nodes
                            per curve; forcing = sum of 20 Gaussians (widths
                            0.02-0.1); adaptive tree to level 8 with 8x8 nodes
                            per leaf; dt = alpha^2 = 1e-3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


def curve_params(n: int) -> np.ndarray:
    """Equispaced parameter values t_n = 2 pi n / N, n = 0..N-1 (Section 3.2)."""
    return TWO_PI * np.arange(n, dtype=np.float64) / n


def circle_nodes(center, radius: float, n: int, clockwise: bool) -> np.ndarray:
    """Nodes of a circle, shape (n, 2)."""
    t = curve_params(n)
    s = -1.0 if clockwise else 1.0
    return np.stack([center[0] + radius * np.cos(t), center[1] + s * radius * np.sin(t)], axis=1)


def starfish_nodes(center, r0: float, eps: float, arms: int, n: int, clockwise: bool,
                   phase: float = 0.0) -> np.ndarray:
    """Nodes of r(t) = r0 (1 + eps cos(arms (t - phase))), shape (n, 2)."""
    t = curve_params(n)
    r = r0 * (1.0 + eps * np.cos(arms * (t - phase)))
    s = -1.0 if clockwise else 1.0
    return np.stack([center[0] + r * np.cos(t), center[1] + s * r * np.sin(t)], axis=1)


@dataclass
class GaussianForcing:
    """F(x) = sum_i A_i exp(-|x - c_i|^2 / (2 s_i^2)), time independent."""
    amp: np.ndarray
    width: np.ndarray
    center: np.ndarray  # (n, 2)

    def __call__(self, xy: np.ndarray) -> np.ndarray:
        xy = np.asarray(xy, dtype=np.float64)
        out = np.zeros(xy.shape[0])
        for a, s, c in zip(self.amp, self.width, self.center):
            d2 = (xy[:, 0] - c[0]) ** 2 + (xy[:, 1] - c[1]) ** 2
            out += a * np.exp(-d2 / (2.0 * s * s))
        return out


def gaussian_forcing(seed: int = 3, n: int = 20) -> GaussianForcing:
    """20 Gaussians, amplitudes U[-1,1], widths U[0.02,0.1], centres uniform in the unit disk."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(-1.0, 1.0, n)
    width = rng.uniform(0.02, 0.1, n)
    rad = np.sqrt(rng.uniform(0.0, 1.0, n))
    ang = rng.uniform(0.0, TWO_PI, n)
    center = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    return GaussianForcing(amp, width, center)


class Manufactured:
    """u = exp(-t) sin(pi x) cos(pi y);  u_t - Lap u = F = (2 pi^2 - 1) u;  f = u on Gamma."""

    @staticmethod
    def u(t: float, xy: np.ndarray) -> np.ndarray:
        xy = np.asarray(xy, dtype=np.float64)
        return math.exp(-t) * np.sin(math.pi * xy[:, 0]) * np.cos(math.pi * xy[:, 1])

    @staticmethod
    def F(t: float, xy: np.ndarray) -> np.ndarray:
        return (2.0 * math.pi ** 2 - 1.0) * Manufactured.u(t, xy)


@dataclass
class Workload:
    name: str
    curves: list                      # list of (N_k, 2) float64 arrays, curve 0 = outer
    box: tuple                        # (xmin, ymin, width) of the square D
    q: int                            # Gauss-Legendre nodes per leaf side
    min_level: int
    max_level: int
    refine_tol: float                 # absolute interpolation-error tolerance on F (inf = uniform)
    dt: float
    alpha: float                      # screening length, alpha^2 = dt for IMEX Euler
    steps: int
    p: int                            # multipole order
    forcing: object = None            # callable F(xy) (time independent) or None
    manufactured: bool = False
    ext_const: list = field(default_factory=list)  # exterior constants C_k per curve

    @property
    def n_gamma(self) -> int:
        return int(sum(c.shape[0] for c in self.curves))


def disk_with_hole(n_per_curve: int = 128, level: int = 4, q: int = 4, dt: float = 1e-2,
                   steps: int = 10, p: int = 20) -> Workload:
    """Unit disk minus the circle r = 0.3 centred at (0.2, 0): N_Gamma = 2 x 128, uniform
    level-4 tree on [-1,1]^2 with 4x4 nodes per leaf (N_D = 4096), dt = alpha^2 = 1e-2."""
    outer = circle_nodes((0.0, 0.0), 1.0, n_per_curve, clockwise=False)
    hole = circle_nodes((0.2, 0.0), 0.3, n_per_curve, clockwise=True)
    return Workload("disk_with_hole", [outer, hole], (-1.0, -1.0, 2.0), q, level, level,
                    math.inf, dt, math.sqrt(dt), steps, p, None, True, [0.0, 0.0])


def starfish_centres(seed: int = 2, n_holes: int = 5, r_max: float = 0.12 * 1.3,
                     gap: float = 0.05, outer_radius: float = 1.0):
    """Rejection-sample hole centres so that the bounding circles of the holes keep a gap
    >= `gap` from each other and from the outer circle (hence so do the curves)."""
    rng = np.random.default_rng(seed)
    centres = []
    lim = outer_radius - r_max - gap
    while len(centres) < n_holes:
        c = rng.uniform(-lim, lim, 2)
        if np.hypot(c[0], c[1]) > lim:
            continue
        if all(np.hypot(c[0] - d[0], c[1] - d[1]) >= 2 * r_max + gap for d in centres):
            centres.append(c)
    return np.array(centres)


# Absolute refinement tolerance for the starfish workload's Gaussian forcing: with 8x8 nodes
# per leaf, min level 4 and max level 8 it gives an adaptive tree of 4027 leaves
# (257,728 volume nodes, leaves on levels 4..8); the closest refinement decision is
# 4e-4 (relative) away from the tolerance, so trees built in any FP64 arithmetic agree.
STARFISH_REFINE_TOL = 3.0e-10


def starfish_domain(n_per_curve: int = 1024, n_holes: int = 5, seed: int = 2, q: int = 8,
                    min_level: int = 4, max_level: int = 8, refine_tol: float = STARFISH_REFINE_TOL,
                    dt: float = 1e-3, steps: int = 100, p: int = 20,
                    forcing_seed: int = 3) -> Workload:
    """Radius-1 disk minus 5 starfish holes r(t) = 0.12 (1 + 0.3 cos 5t) (clockwise), 1024
    nodes per curve (N_Gamma = 6144); Gaussian-sum forcing; adaptive tree (8x8 per leaf);
    dt = alpha^2 = 1e-3; f = 0 on every curve; exterior constants C_k = 0."""
    outer = circle_nodes((0.0, 0.0), 1.0, n_per_curve, clockwise=False)
    cs = starfish_centres(seed, n_holes)
    holes = [starfish_nodes(c, 0.12, 0.3, 5, n_per_curve, clockwise=True) for c in cs]
    return Workload("starfish_domain", [outer] + holes, (-1.0, -1.0, 2.0), q, min_level,
                    max_level, refine_tol, dt, math.sqrt(dt), steps, p,
                    gaussian_forcing(forcing_seed), False, [0.0] * (n_holes + 1))


class Example1:
    """The annulus problem with a known solution (the paper's Example 1): Gamma_0 the circle
    r = 0.4 (counter-clockwise), Gamma_1 the circle r = 0.1 (clockwise), forcing
    F = 400 cos(20 r) + 20 sin(20 r) / r and
        u(x, t) = exp(-lam^2 t) [Y0(0.1 lam) J0(lam r) - J0(0.1 lam) Y0(lam r)] + cos(20 r),
    lam the first root of Y0(0.1 lam) J0(0.4 lam) - J0(0.1 lam) Y0(0.4 lam) (about 10.244), so
    that u = cos(8) on Gamma_0 and cos(2) on Gamma_1.  `u_ext` continues u inside the hole
    (r < 0.1) by a polynomial in r^2 matching u, u_r and u_rr at r = 0.1 (C^2), so that data
    extended outside Omega stay smooth; outside r = 0.4 the formula itself is used."""

    R0, R1 = 0.4, 0.1

    def __init__(self):
        from scipy import optimize, special
        self._j0, self._y0, self._j1, self._y1 = special.j0, special.y0, special.j1, special.y1
        f = lambda l: special.y0(0.1 * l) * special.j0(0.4 * l) - special.j0(0.1 * l) * special.y0(0.4 * l)
        self.lam = optimize.brentq(f, 5.0, 12.0)

    def radial(self, t, r):
        lam = self.lam
        c1, c2 = self._y0(0.1 * lam), self._j0(0.1 * lam)
        e = math.exp(-lam * lam * t)
        v = e * (c1 * self._j0(lam * r) - c2 * self._y0(lam * r)) + np.cos(20 * r)
        # d/dr and d2/dr2 (J0' = -J1, J1' = J0 - J1/z; same for Y)
        z = lam * r
        d1 = e * lam * (-c1 * self._j1(z) + c2 * self._y1(z)) - 20 * np.sin(20 * r)
        d2 = e * lam * lam * (-c1 * (self._j0(z) - self._j1(z) / z) + c2 * (self._y0(z) - self._y1(z) / z)) \
            - 400 * np.cos(20 * r)
        return v, d1, d2

    def u(self, t, xy):
        xy = np.asarray(xy, dtype=np.float64)
        r = np.hypot(xy[:, 0], xy[:, 1])
        out = np.empty_like(r)
        big = r >= self.R1
        out[big] = self.radial(t, r[big])[0]
        if np.any(~big):
            # u_ext = a + b s + c s^2 with s = r^2 - R1^2, matching v, v', v'' at r = R1
            v, d1, d2 = (float(np.asarray(q).reshape(-1)[0]) for q in self.radial(t, np.array([self.R1])))
            b = d1 / (2 * self.R1)
            c = (d2 - 2 * b) / (8 * self.R1 ** 2)
            s = r[~big] ** 2 - self.R1 ** 2
            out[~big] = v + b * s + c * s * s
        return out

    def F(self, xy):
        xy = np.asarray(xy, dtype=np.float64)
        r = np.hypot(xy[:, 0], xy[:, 1])
        safe = np.where(r > 1e-12, r, 1.0)
        return 400 * np.cos(20 * r) + np.where(r > 1e-12, 20 * np.sin(20 * r) / safe, 400.0)

    def boundary_data(self):
        return [math.cos(8.0), math.cos(2.0)]

    def curves(self, n_outer, n_inner):
        return [circle_nodes((0.0, 0.0), self.R0, n_outer, clockwise=False),
                circle_nodes((0.0, 0.0), self.R1, n_inner, clockwise=True)]


# ---------------------------------------------------------------------------- learned warm start
WARM_TRAIN_SEEDS = tuple(range(100, 200))     # forcings whose trajectories train the network
WARM_VALID_SEEDS = tuple(range(200, 210))     # validation trajectories (early stopping)
WARM_TEST_SEEDS = tuple(range(300, 305))      # held-out trajectories


def warm_start_draws(n: int, width: int, steps: int, batch: int, seed: int = 7):
    """Random numbers of the learned warm start's training, drawn here and passed in:
    omega (n x width standard normal, binary32) for the range finder of the closed-form start
    and the Adam minibatches (steps x batch row indices, uniform with replacement, int32)."""
    rng = np.random.default_rng(seed)
    omega = rng.standard_normal((n, width)).astype(np.float32)
    idx = rng.integers(0, n, size=(steps, batch)).astype(np.int32)
    return omega, idx


def warm_start_toy_data(n: int, d: int, rank: int, seed: int = 11):
    """Small synthetic pairs for parity tests of the training kernels: rows of X in a random
    rank-`rank` subspace with a decaying spectrum plus a mean, Y = X M^T + c (binary32)."""
    rng = np.random.default_rng(seed)
    basis = np.linalg.qr(rng.standard_normal((d, rank)))[0]
    mu = rng.standard_normal(d)
    coef = rng.standard_normal((n, rank)) * np.geomspace(1.0, 1e-2, rank)
    X = mu + coef @ basis.T
    M = rng.standard_normal((d, d)) / math.sqrt(d)
    c = rng.standard_normal(d)
    return X.astype(np.float32), (X @ M.T + c).astype(np.float32)


# ---------------------------------------------------------------------------- batched problems
def ellipse_nodes(center, a: float, b: float, angle: float, n: int, clockwise: bool) -> np.ndarray:
    """Nodes of an ellipse with semi-axes a, b rotated by `angle`, shape (n, 2)."""
    t = curve_params(n)
    s = -1.0 if clockwise else 1.0
    x, y = a * np.cos(t), s * b * np.sin(t)
    c, sn = math.cos(angle), math.sin(angle)
    return np.stack([center[0] + c * x - sn * y, center[1] + sn * x + c * y], axis=1)


BATCH_SIZE = 64
BATCH_SEED = 4


def batch_problem(i: int, seed: int = BATCH_SEED, steps: int = 20, npc=None, refine_tol=None) -> Workload:
    """Problem i of the batched workload: the unit disk minus 1-8 holes (starfish
    r(t) = r0 (1 + 0.3 cos 5t) or rotated ellipses, each kind with probability 1/2), hole sizes
    r0 ~ U[0.05, min(0.12, 0.36 / sqrt(holes))], centres by rejection sampling keeping a gap
    >= 0.05 between the holes' bounding circles and from the outer circle; nodes per curve
    32 * U{8..64} (256-2048); alpha^2 = dt log-uniform in [1e-4, 1e-2]; Gaussian-sum forcing
    (seed 1000 + i); adaptive tree (8x8 nodes per leaf, levels 4-8) with the absolute
    refinement tolerance 10^U[-10, -5] (16k to a few 100k volume nodes); f = 0, C_k = 0.
    npc / refine_tol override the drawn values (smaller cases for tests)."""
    rng = np.random.default_rng([seed, i])
    n_holes = int(rng.integers(1, 9))
    npc_drawn = 32 * int(rng.integers(8, 65))
    refine_tol_override = refine_tol
    npc = npc_drawn if npc is None else npc
    alpha2 = 10.0 ** rng.uniform(-4.0, -2.0)
    refine_tol = 10.0 ** rng.uniform(-10.0, -5.0)
    r_hi = min(0.12, 0.36 / math.sqrt(n_holes))
    holes, placed = [], []          # placed: (centre, bounding radius)
    while len(holes) < n_holes:
        kind = rng.integers(0, 2)
        r0 = rng.uniform(0.05, r_hi)
        if kind == 0:
            extent = 1.3 * r0
        else:
            a, b = r0, r0 * rng.uniform(0.5, 1.0)
            ang = rng.uniform(0.0, math.pi)
            extent = a
        lim = 1.0 - extent - 0.05
        c = rng.uniform(-lim, lim, 2)
        if np.hypot(c[0], c[1]) > lim:
            continue
        if any(np.hypot(c[0] - d[0], c[1] - d[1]) < extent + e + 0.05 for d, e in placed):
            continue
        placed.append((c, extent))
        if kind == 0:
            holes.append(starfish_nodes(c, r0, 0.3, 5, npc, clockwise=True, phase=rng.uniform(0.0, TWO_PI)))
        else:
            holes.append(ellipse_nodes(c, a, b, ang, npc, clockwise=True))
    outer = circle_nodes((0.0, 0.0), 1.0, npc, clockwise=False)
    if refine_tol_override is not None:
        refine_tol = refine_tol_override
    return Workload(f"batch_{i}", [outer] + holes, (-1.0, -1.0, 2.0), 8, 4, 8, refine_tol, alpha2,
                    math.sqrt(alpha2), steps, 20, gaussian_forcing(1000 + i), False, [0.0] * (n_holes + 1))
