"""Pins of the oracle's quadrature helpers: closed-form periodic sinc against its
cosine-sum definition, exactness of the trigonometric interpolant on
trigonometric polynomials, Gauss-Legendre exactness, Lagrange cardinality."""
import numpy as np

from oracle import quadrature as Q


def test_trig_kernel_closed_form():
    for n in [8, 16, 64]:
        tau = np.linspace(-7, 7, 301) + 1e-3
        assert np.allclose(Q.trig_kernel(tau, n), Q.trig_kernel_sum(tau, n), atol=1e-13)
        assert np.allclose(Q.trig_kernel(2 * np.pi * np.arange(n) / n, n), np.eye(n)[0], atol=1e-14)


def test_trig_eval_exact_on_trig_polynomials():
    n = 32
    t = 2 * np.pi * np.arange(n) / n
    f = lambda s: 1.5 + np.cos(3 * s) - 0.25 * np.sin(7 * s) + 0.1 * np.cos(15 * s)
    df = lambda s: -3 * np.sin(3 * s) - 1.75 * np.cos(7 * s) - 1.5 * np.sin(15 * s)
    d2f = lambda s: -9 * np.cos(3 * s) + 12.25 * np.sin(7 * s) - 22.5 * np.cos(15 * s)
    s = np.linspace(0, 2 * np.pi, 97)
    assert np.allclose(Q.trig_eval(f(t), s, 0), f(s), atol=1e-13)
    assert np.allclose(Q.trig_eval(f(t), s, 1), df(s), atol=1e-12)
    assert np.allclose(Q.trig_eval(f(t), s, 2), d2f(s), atol=1e-11)
    # interpolation weights reproduce the same interpolant
    w = Q.trig_kernel(s[:, None] - t[None, :], n)
    assert np.allclose(w @ f(t), f(s), atol=1e-13)


def test_gauss_legendre_and_lagrange():
    x, w = Q.gauss_legendre(8)
    for k in range(16):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    L = Q.lagrange_matrix(x, x)
    assert np.allclose(L, np.eye(8), atol=1e-14)
    pts = np.linspace(-1, 1, 11)
    assert np.allclose(Q.lagrange_matrix(x, pts).sum(axis=0), 1.0, atol=1e-13)
