"""Boundary geometry and point classification for the oracle.

Each boundary component Gamma_k is parametrised on [0, 2 pi) and sampled at
N_k equispaced values t_n with spacing h_k = 2 pi / N_k (Section 3.2).  Normals
are obtained pseudospectrally (Section 3.2): y', y'' at the nodes come from
the trigonometric interpolant of the node coordinates (FFT).  The outward
normal of Omega is the right-hand normal n = (y2', -y1') / |y'| (outer curve
counter-clockwise, holes clockwise).  The curvature enters through the
diagonal limit of the double-layer kernel (Section 2, after
eq. dirichlet:inteqn): K(x, x) = -(y'' . n) / (2 |y'|^2).

Point classification and the distance to Gamma are not spelled out in the
paper (it needs them implicitly to restrict U = U^p + U^h to Omega, Section 2);
the reading used here:
  * nearest node n* of curve k (smallest index on ties); h* = |y'(t_n*)| h_k;
  * if |y_n* - x| < 12 h*: Newton on phi(t) = |y(t) - x|^2 / 2 from t_n*, giving the
    foot t*, the distance d = |y(t*) - x| and the side sign (x - y(t*)) . n(t*)
    (negative = Omega side);
  * otherwise the side comes from the trapezoid Laplace double layer of unit
    density, W_k(x) = (1/2 pi) sum_n (y_n - x).n_n / |y_n - x|^2 |y'_n| h_k, which
    is 1 inside the outer curve, -1 inside a hole and 0 elsewhere.
Pins: circle geometry (closed-form normals and curvature), spectral
convergence on a starfish, classification of points at known distances.
"""
import math

import numpy as np

from .quadrature import trig_eval

NEAR_NODE_FACTOR = 12.0    # Newton projection when the nearest node is within 12 h*


class Curve:
    def __init__(self, nodes: np.ndarray):
        self.nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        self.n = self.nodes.shape[0]
        if self.n % 2:
            raise ValueError("curves must have an even number of nodes")
        self.h = 2.0 * math.pi / self.n
        self.t = self.h * np.arange(self.n)
        self.d1 = trig_eval(self.nodes, self.t, 1)
        self.d2 = trig_eval(self.nodes, self.t, 2)
        self.speed = np.hypot(self.d1[:, 0], self.d1[:, 1])
        self.normal = np.stack([self.d1[:, 1], -self.d1[:, 0]], axis=1) / self.speed[:, None]
        # diagonal limit of K(y, x) = (1/alpha) K1(|y-x|/alpha) (y-x).n_y/|y-x| as y -> x
        self.kdiag = -np.einsum("ij,ij->i", self.d2, self.normal) / (2.0 * self.speed ** 2)
        # signed curvature kappa = (y1' y2'' - y2' y1'') / |y'|^3 (positive on a CCW circle)
        self.kappa = (self.d1[:, 0] * self.d2[:, 1] - self.d1[:, 1] * self.d2[:, 0]) / self.speed ** 3

    def eval(self, t, deriv: int = 0) -> np.ndarray:
        return trig_eval(self.nodes, t, deriv)

    def signed_area(self) -> float:
        # area enclosed, positive for counter-clockwise curves (spectral: 1/2 int (x y' - y x') dt)
        return 0.5 * self.h * float(np.sum(self.nodes[:, 0] * self.d1[:, 1] - self.nodes[:, 1] * self.d1[:, 0]))


def make_curves(curve_nodes) -> list:
    return [Curve(c) for c in curve_nodes]


def check_orientation(curves) -> bool:
    """Outer curve counter-clockwise (positive area), holes clockwise (negative)."""
    if curves[0].signed_area() <= 0:
        return False
    return all(c.signed_area() < 0 for c in curves[1:])


def project(curve: Curve, x: np.ndarray, t0: float, iters: int = 30):
    """Newton on phi(t) = |y(t) - x|^2 / 2 from t0; returns (t*, y*, y'*, d, side)."""
    t = float(t0)
    for _ in range(iters):
        y = curve.eval(t, 0)[0]
        y1 = curve.eval(t, 1)[0]
        y2 = curve.eval(t, 2)[0]
        r = y - x
        g = float(r @ y1)
        hss = float(y1 @ y1 + r @ y2)
        if hss <= 0:
            hss = float(y1 @ y1)
        dt = g / hss
        t -= dt
        if abs(dt) < 1e-15:
            break
    t = math.fmod(t, 2.0 * math.pi)
    if t < 0:
        t += 2.0 * math.pi
    y = curve.eval(t, 0)[0]
    y1 = curve.eval(t, 1)[0]
    nrm = np.array([y1[1], -y1[0]]) / math.hypot(y1[0], y1[1])
    d = float(math.hypot(*(x - y)))
    side = float((x - y) @ nrm)
    return t, y, y1, d, side


def winding(curve: Curve, pts: np.ndarray) -> np.ndarray:
    """W_k(x) = (1/2pi) sum_n (y_n - x).n_n / |y_n - x|^2 |y'_n| h (trapezoid)."""
    dx = curve.nodes[None, :, 0] - pts[:, None, 0]
    dy = curve.nodes[None, :, 1] - pts[:, None, 1]
    num = dx * curve.normal[None, :, 0] + dy * curve.normal[None, :, 1]
    return (num / (dx * dx + dy * dy) * (curve.speed * curve.h)[None, :]).sum(axis=1) / (2.0 * math.pi)


class PointInfo:
    """Per target: region (-1 = in Omega, k = exterior side of curve k) and, per curve,
    the projection data (None when the nearest node is >= 12 h* away)."""

    def __init__(self, n_pts, n_curves):
        self.region = np.full(n_pts, -1, dtype=np.int64)
        self.proj = [[None] * n_curves for _ in range(n_pts)]


def classify(curves, pts: np.ndarray) -> PointInfo:
    pts = np.asarray(pts, dtype=np.float64)
    info = PointInfo(pts.shape[0], len(curves))
    for k, c in enumerate(curves):
        d2 = (c.nodes[None, :, 0] - pts[:, None, 0]) ** 2 + (c.nodes[None, :, 1] - pts[:, None, 1]) ** 2
        nstar = np.argmin(d2, axis=1)
        dmin = np.sqrt(d2[np.arange(pts.shape[0]), nstar])
        hstar = c.speed[nstar] * c.h
        near = dmin < NEAR_NODE_FACTOR * hstar
        far_idx = np.nonzero(~near)[0]
        if far_idx.size:
            w = winding(c, pts[far_idx])
            outside = (w < 0.5) if k == 0 else (w < -0.5)
            for i, o in zip(far_idx, outside):
                if o and info.region[i] == -1:
                    info.region[i] = k
        for i in np.nonzero(near)[0]:
            t, y, y1, d, side = project(c, pts[i], c.t[nstar[i]])
            info.proj[i][k] = dict(t=t, y=y, d=d, hs=math.hypot(*y1) * c.h, side=side, node=int(nstar[i]))
            if side >= 0 and info.region[i] == -1:
                info.region[i] = k
    return info
