"""The binary32 tables of g(z) = K1(z)/z compiled into the library (the double-layer pair
term of Section 3.2: (1/alpha) K1(r/alpha) (d.n)/r = g(r/alpha) (d.n)/alpha^2), read from
the generated header and checked against scipy's K1 -- a library routine independent of
the generator:

  z <= 2 : g = 1/z^2 + log2(y) sum a_k y^k - sum b_k y^k,   y = z^2/4
  z > 2  : g = e^{-z} z^{-3/2} sum m_j x^j,                  x = 4/z - 1

The tables are evaluated in binary64 with their binary32 values, so what is left is the
truncation of the series / interpolant (below 1e-8) plus the binary32 rounding of every
coefficient, at most 2^-24 of each term: the bound is 2^-24 * sum|terms| / |g| + 1e-8.
A dropped term, a wrong sign or a misplaced factor of the generator fails by orders of
magnitude."""
import os
import re

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_1007_5335_gb300", "csrc", "bessel_coefs.h")


def _table(name):
    src = open(HDR).read()
    m = re.search(r"float %s\[(\d+)\] = \{([^}]*)\}" % re.escape(name), src)
    assert m, name
    vals = np.array([float(v) for v in m.group(2).replace("\n", " ").split(",")])
    assert len(vals) == int(m.group(1))
    return vals.astype(np.float32).astype(np.float64)


def test_small_argument_series():
    a, b = _table("mh_k1oz_a_f"), _table("mh_k1oz_b_f")
    assert len(a) == 6 and len(b) == 8
    for z in np.geomspace(1e-3, 2.0, 400):
        y = 0.25 * z * z
        lg = np.log2(y)
        ta = lg * a * y ** np.arange(len(a))
        tb = b * y ** np.arange(len(b))
        g = 1.0 / (z * z) + ta.sum() - tb.sum()
        ref = special.k1(z) / z
        bound = 2.0 ** -24 * (1.0 / (z * z) + np.abs(ta).sum() + np.abs(tb).sum()) / abs(ref) + 1e-8
        assert abs(g / ref - 1.0) <= bound, (z, g, ref)


def test_large_argument_monomial_interpolant():
    m = _table("mh_k1_mono_f")
    assert len(m) == 10
    for z in np.linspace(2.0, 60.0, 400):
        x = 4.0 / z - 1.0
        tm = m * x ** np.arange(len(m))
        g = np.exp(-z) * z ** -1.5 * tm.sum()
        ref = special.k1e(z) * np.exp(-z) / z
        bound = 2.0 ** -24 * np.abs(tm).sum() / abs(tm.sum()) + 1e-8
        assert abs(g / ref - 1.0) <= bound, (z, g, ref)


def test_branches_meet_at_two():
    # both forms are evaluated on either side of the switch at z = 2 (r^2 = 4 alpha^2)
    a, b, m = _table("mh_k1oz_a_f"), _table("mh_k1oz_b_f"), _table("mh_k1_mono_f")
    z = 2.0
    y = 1.0
    small = 1.0 / (z * z) + np.log2(y) * np.polyval(a[::-1], y) - np.polyval(b[::-1], y)
    large = np.exp(-z) * z ** -1.5 * np.polyval(m[::-1], 4.0 / z - 1.0)
    assert abs(small / large - 1.0) < 1e-6
