"""Hybrid Gauss-trapezoidal correction for log-singular periodic integrands
(Alpert's rules, Section 3.2).  The table ``alpert_rules.json`` is written by
``oracle/gen_alpert_rules.py`` from the defining Hurwitz-zeta conditions.

For a 2 pi-periodic f with a log singularity at t_j, the corrected rule is
    h sum_{|k| >= a} f(t_j + k h) + h sum_{m=1}^{l} w_m [f(t_j + x_m h) + f(t_j - x_m h)],
i.e. the trapezoid rule with the 2a-1 nodes |k| < a removed (the diagonal
included) and 2l off-grid nodes added.  Pins: the defining conditions, and
convergence of int_0^{2pi} log(4 sin^2(s/2)) cos(ms) ds = -2 pi / m.
"""
import json
import os

import numpy as np

_PATH = os.path.join(os.path.dirname(__file__), "alpert_rules.json")
DEFAULT_ORDER = 8


def rule(l: int = DEFAULT_ORDER):
    """Return (a, nodes x_m, weights w_m) of the l-point log-singular correction."""
    with open(_PATH) as fh:
        tab = json.load(fh)
    r = tab[str(int(l))]
    return int(r["a"]), np.array([float(v) for v in r["nodes"]]), np.array([float(v) for v in r["weights"]])


def periodic_quadrature(f, n: int, l: int = DEFAULT_ORDER) -> float:
    """Alpert-corrected trapezoid rule for int_0^{2pi} f(s) ds, singular point s = 0."""
    a, x, w = rule(l)
    h = 2.0 * np.pi / n
    k = np.arange(a, n - a + 1)
    total = h * np.sum(f(k * h))
    total += h * np.sum(w * (f(x * h) + f(-x * h)))
    return float(total)
