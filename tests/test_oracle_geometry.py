"""Pins of the oracle's geometry: closed-form circle normals, curvature and
diagonal kernel limit (Section 2: d/dnu K0 -> -kappa/2); spectral derivatives
of a starfish against the analytic parametrisation; classification of points
at known distances."""
import math

import numpy as np

import mh_workloads as W
from oracle import geometry as G


def test_circle_geometry():
    R = 0.7
    c = G.Curve(W.circle_nodes((0.1, -0.2), R, 64, clockwise=False))
    assert np.allclose(c.speed, R, atol=1e-13)
    assert np.allclose(c.kappa, 1 / R, atol=1e-12)
    assert np.allclose(c.kdiag, 1 / (2 * R), atol=1e-12)
    radial = (c.nodes - np.array([0.1, -0.2])) / R
    assert np.allclose(c.normal, radial, atol=1e-13)
    h = G.Curve(W.circle_nodes((0.0, 0.0), R, 64, clockwise=True))
    assert np.allclose(h.normal, -h.nodes / R, atol=1e-13)    # into the hole = out of Omega
    assert np.allclose(h.kdiag, -1 / (2 * R), atol=1e-12)


def test_starfish_spectral_derivatives():
    n = 256
    c = G.Curve(W.starfish_nodes((0.1, 0.2), 0.12, 0.3, 5, n, clockwise=True))
    t = c.t
    r = 0.12 * (1 + 0.3 * np.cos(5 * t))
    dr = -0.12 * 0.3 * 5 * np.sin(5 * t)
    dx = dr * np.cos(t) - r * np.sin(t)
    dy = -(dr * np.sin(t) + r * np.cos(t))
    assert np.allclose(c.d1[:, 0], dx, atol=1e-12) and np.allclose(c.d1[:, 1], dy, atol=1e-12)


def test_orientation_and_classification():
    wl = W.disk_with_hole()
    curves = G.make_curves(wl.curves)
    assert G.check_orientation(curves)
    assert not G.check_orientation(G.make_curves([wl.curves[1], wl.curves[0]]))
    pts = np.array([[0.0, 0.6], [0.2, 0.0], [1.2, 0.3], [0.999, 0.0], [0.2, 0.3 + 1e-3], [0.2, 0.3 - 1e-3],
                    [0.0, -0.95]])
    info = G.classify(curves, pts)
    assert list(info.region) == [-1, 1, 0, -1, -1, 1, -1]
    p = info.proj[3][0]
    assert abs(p["d"] - 1e-3) < 1e-12 and p["side"] < 0
    p = info.proj[4][1]
    assert abs(p["d"] - 1e-3) < 1e-12
