"""Pin of the oracle's Allen-Cahn step (Section 4, Example 3: u_t - eps Lap u = u (1 - u^2),
u = 0 on Gamma, the reaction term explicit, alpha^2 = eps dt).

Far from Gamma the boundary correction U^h decays like exp(-d / alpha), and the volume
potential of a smooth B is the free-space resolvent (1 - alpha^2 Lap)^{-1} B = B + alpha^2
Lap B + O(alpha^4 Lap^2 B).  So on the smooth start u^N = a sin(pi x / 2) cos(pi y / 2) the
step at nodes farther than 0.25 from both curves must equal B + alpha^2 Lap B, with B =
u^N + dt u^N (1 - (u^N)^2) and Lap B written out by hand, to within the leaf interpolation
error of B (q = 4, leaf width 0.125) -- far below the size of the reaction term, of its
cubic part and of the alpha^2 term, so a dropped or mis-signed reaction term, a dt missing
from it, or alpha^2 = dt instead of eps dt each fail."""
import math

import numpy as np

import mh_workloads as W
from oracle import bie, geometry as G, step as S, tree as T, volume as V

EPS, DT, AMP = 1e-4, 1.0, 0.6


def _u0(x, y):
    return AMP * np.sin(0.5 * math.pi * x) * np.cos(0.5 * math.pi * y)


def _B_and_lap(x, y):
    k = 0.5 * math.pi
    u = _u0(x, y)
    lap_u = -2.0 * k * k * u
    grad2 = (AMP * k) ** 2 * (np.cos(k * x) ** 2 * np.cos(k * y) ** 2 + np.sin(k * x) ** 2 * np.sin(k * y) ** 2)
    lap_u3 = 3.0 * u * u * lap_u + 6.0 * u * grad2      # Lap(u^3) = 3 u^2 Lap u + 6 u |grad u|^2
    B = u + DT * (u - u ** 3)
    lap_B = lap_u + DT * (lap_u - lap_u3)
    return B, lap_B, u


def test_allen_cahn_far_field_is_the_free_space_resolvent():
    wl = W.disk_with_hole()
    alpha = math.sqrt(EPS * DT)
    curves = G.make_curves(wl.curves)
    tr = T.build(wl.box, wl.q, wl.min_level, wl.max_level)
    nodes = tr.nodes()
    info = G.classify(curves, nodes)
    bn = np.concatenate([c.nodes for c in curves])
    bleaf = [tr.locate(p) for p in bn]
    M = V.uniform_operator(wl.min_level, wl.box, wl.q, alpha, order=[(b[1], b[2]) for b in tr.leaves])
    A = bie.nystrom_matrix(curves, alpha)
    pb = S.Problem(curves, tr, alpha, DT, info, bleaf, A, ext_mode="const", ext_const=[0.0, 0.0],
                   volume_op=lambda b: M @ b, use_lu=True)
    x, y = nodes[:, 0], nodes[:, 1]
    u0 = _u0(x, y)
    u1, _, _ = S.allen_cahn_step(pb, u0.copy(), np.zeros(len(bn)))
    B, lap_B, u = _B_and_lap(x, y)
    d_outer = 1.0 - np.hypot(x, y)
    d_hole = np.hypot(x - 0.2, y) - 0.3
    far = pb.inside & (d_outer > 0.25) & (d_hole > 0.25)
    assert far.sum() > 200
    expect = B + alpha ** 2 * lap_B
    err = np.max(np.abs(u1[far] - expect[far]))
    # sizes of what the pin must resolve, at those nodes
    reaction = np.max(np.abs(DT * (u - u ** 3))[far])
    cubic = np.max(np.abs(DT * u ** 3)[far])
    lap_term = np.max(np.abs(alpha ** 2 * lap_B)[far])
    assert reaction > 0.1 and cubic > 0.02 and lap_term > 5e-5
    assert err < 5e-6, (err, reaction, cubic, lap_term)
    # alpha^2 = dt would move the far field by (dt - eps dt) Lap B, far above the bar
    assert np.max(np.abs((DT - EPS * DT) * lap_B[far])) > 1e3 * err
