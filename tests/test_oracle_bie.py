"""Pins of the oracle's boundary integral equation (Section 2 eq. dirichlet:inteqn,
Section 3.2 eq. discrete_sys) against closed forms:
  * circle of radius R, sigma = cos(n t): A sigma = mu_n sigma with
    mu_n = z I_n(z) [K_{n-1}(z) + K_{n+1}(z)], z = R/alpha (Graf's addition theorem);
  * the Dirichlet problem with g = cos(n theta) on that circle has the interior
    solution U^h = I_n(r/alpha) / I_n(z) cos(n theta) -- checked far from Gamma and
    in both near-boundary regimes of the evaluation rule;
  * exact homogeneous solutions K0(|x - x0|/alpha), x0 outside Omega, on the
    disk-with-hole domain, with spectral convergence in N;
  * GMRES against a dense LU solve."""
import math

import numpy as np
import pytest
from scipy.special import iv, kv, k0

import mh_workloads as W
from oracle import bie, geometry as G


@pytest.mark.parametrize("n", [0, 1, 4])
def test_circle_spectrum(n):
    R, alpha = 0.7, 0.1
    c = G.make_curves([W.circle_nodes((0, 0), R, 128, False)])
    A = bie.nystrom_matrix(c, alpha)
    z = R / alpha
    mu = z * iv(n, z) * (kv(n - 1, z) + kv(n + 1, z))
    sig = np.cos(n * c[0].t)
    assert np.max(np.abs(A @ sig - mu * sig)) < 1e-10
    # the plain trapezoid rule with the diagonal limit converges to the same operator, O(h^3)
    e = [np.max(np.abs(bie.nystrom_matrix(G.make_curves([W.circle_nodes((0, 0), R, m, False)]),
                                          alpha, None) @ np.cos(n * 2 * np.pi * np.arange(m) / m)
                       - mu * np.cos(n * 2 * np.pi * np.arange(m) / m))) for m in (64, 128)]
    assert e[0] / e[1] > 7.0


def test_circle_interior_field_all_regimes():
    R, alpha, n, N = 0.5, 0.1, 3, 128
    curves = G.make_curves([W.circle_nodes((0, 0), R, N, False)])
    A = bie.nystrom_matrix(curves, alpha)
    g = np.cos(n * curves[0].t)
    sigma = np.linalg.solve(A, -2 * alpha ** 2 * g)
    hs = R * 2 * np.pi / N
    r = np.array([0.1, R - 8 * hs, R - 2 * hs, R - 0.6 * hs, R - 0.2 * hs, R - 0.03 * hs])
    th = np.array([0.3, 1.1, 2.0, 0.013, 4.0, 5.5])
    pts = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    info = G.classify(curves, pts)
    assert np.all(info.region == -1)
    U = bie.dlp_eval(curves, sigma, alpha, pts, info, A @ sigma)
    exact = iv(n, r / alpha) / iv(n, R / alpha) * np.cos(n * th)
    err = np.abs(U - exact)
    assert np.max(err[:4]) < 1e-12, err          # plain and 16x upsampled rules
    assert np.max(err[4:]) < 5e-8, err           # interpolation along the normal (d < h_s/4)


def test_exact_homogeneous_solutions_converge():
    alpha = 0.1
    errs = []
    for N in (64, 128):
        wl = W.disk_with_hole(n_per_curve=N)
        curves = G.make_curves(wl.curves)
        A = bie.nystrom_matrix(curves, alpha)
        bn = np.concatenate([c.nodes for c in curves])
        pts = np.array([[0.6, 0.1], [-0.5, -0.4], [0.2, 0.45], [0.0, 0.85]])
        info = G.classify(curves, pts)
        e = 0.0
        for x0 in ([0.2, 0.0], [1.5, 0.3]):
            f = lambda p: k0(np.hypot(p[:, 0] - x0[0], p[:, 1] - x0[1]) / alpha)
            sigma, its, hist = bie.gmres(A, -2 * alpha ** 2 * f(bn), tol=1e-13)
            assert its < 60
            assert np.allclose(sigma, np.linalg.solve(A, -2 * alpha ** 2 * f(bn)), rtol=0, atol=1e-12)
            U = bie.dlp_eval(curves, sigma, alpha, pts, info)
            e = max(e, np.max(np.abs(U - f(pts))) / np.max(np.abs(f(pts))))
        errs.append(e)
    assert errs[1] < 1e-9 and errs[0] / errs[1] > 10, errs


def test_gmres_matches_lu_and_reports_history():
    rng = np.random.default_rng(0)
    A = np.eye(40) + 0.3 * rng.standard_normal((40, 40)) / np.sqrt(40)
    b = rng.standard_normal(40)
    x, its, hist = bie.gmres(A, b, tol=1e-12)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
    assert hist[-1] <= 1e-12 and all(hist[i + 1] <= hist[i] + 1e-15 for i in range(len(hist) - 1))
    x2, its2, _ = bie.gmres(A, b, x0=x, tol=1e-10)
    assert its2 <= 1
