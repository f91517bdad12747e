"""Pins of the Alpert log-singular correction table (Section 3.2): the defining
Hurwitz-zeta conditions, and convergence on
int_0^{2 pi} log(4 sin^2(s/2)) cos(m s) ds = -2 pi / m   (m >= 1)."""
import numpy as np
import pytest

from oracle import alpert


@pytest.mark.parametrize("l", [2, 4, 6, 8, 10])
def test_defining_conditions(l):
    mp = pytest.importorskip("mpmath")
    a, x, w = alpert.rule(l)
    assert a == l and np.all(x > 0) and np.all(x < a) and np.all(w > 0)
    for g in range(l):
        p = sum(wi * xi ** g for xi, wi in zip(x, w))
        lg = sum(wi * xi ** g * np.log(xi) for xi, wi in zip(x, w))
        assert abs(p + float(mp.zeta(-g, a))) < 1e-12 * max(1.0, abs(p))
        assert abs(lg - float(mp.zeta(-g, a, 1))) < 1e-12 * max(1.0, abs(lg))


def test_log_integral_convergence():
    m = 3
    exact = -2 * np.pi / m
    f = lambda s: np.log(4 * np.sin(0.5 * s) ** 2) * np.cos(m * s) * np.exp(0.3 * np.cos(s) ** 2) ** 0
    errs = {}
    for l in (4, 8):
        errs[l] = [abs(alpert.periodic_quadrature(f, n, l) - exact) for n in (32, 64, 128)]
    # order-l rules: error falls at least like h^(l-1) here; plain trapezoid would stall at O(h)
    assert errs[8][-1] < 1e-12
    assert errs[4][1] / errs[4][2] > 2 ** 3
