"""Values the paper prints, used as fixtures (tests/golden/paper_values.json)."""
import json
import os

import numpy as np
from scipy import optimize, special

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_example1_lambda_is_first_root():
    # Example 1 (Section 4): lambda makes Y0(0.1 l) J0(|x| l) - J0(0.1 l) Y0(|x| l) vanish at |x| = 0.4
    r0, r1 = GOLD["example1_radii"]["inner"], GOLD["example1_radii"]["outer"]
    f = lambda l: special.y0(r0 * l) * special.j0(r1 * l) - special.j0(r0 * l) * special.y0(r1 * l)
    lam = optimize.brentq(f, 5.0, 12.0)
    assert abs(lam - GOLD["example1_lambda"]["value"]) < 5e-4


def test_table1_orders():
    dt = np.array(GOLD["table1_dt"]["value"])
    e1 = np.array(GOLD["table1_error_imex_euler"]["value"])
    e2 = np.array(GOLD["table1_error_gear"]["value"])
    o1 = np.log(e1[:3][:-1] / e1[1:3]) / np.log(dt[:2] / dt[1:3])
    o2 = np.log(e2[:-1] / e2[1:]) / np.log(dt[:-1] / dt[1:])
    assert np.all(np.abs(o1 - 1) < 0.1)          # IMEX Euler: first order
    assert np.all(np.abs(o2 - 2) < 0.3)          # extrapolated Gear: second order
