"""Pin of the oracle's IMEX Euler heat step (Section 2) on the manufactured
solution u = exp(-t) sin(pi x) cos(pi y) (F = (2 pi^2 - 1) u, f = u on Gamma) on
the disk-with-hole domain: the error at t = 0.05 is small and falls by ~2 when
dt halves (first order in time, Section 2: "first-order backward Euler")."""
import math

import numpy as np

import mh_workloads as W
from oracle import bie, geometry as G, step as S, tree as T, volume as V


def _run(dt, t_end):
    wl = W.disk_with_hole(dt=dt)
    curves = G.make_curves(wl.curves)
    tr = T.build(wl.box, wl.q, wl.min_level, wl.max_level)
    nodes = tr.nodes()
    info = G.classify(curves, nodes)
    bn = np.concatenate([c.nodes for c in curves])
    bleaf = [tr.locate(p) for p in bn]
    M = V.uniform_operator(wl.min_level, wl.box, wl.q, wl.alpha, order=[(b[1], b[2]) for b in tr.leaves])
    A = bie.nystrom_matrix(curves, wl.alpha)
    pb = S.Problem(curves, tr, wl.alpha, dt, info, bleaf, A, ext_mode="array", volume_op=lambda b: M @ b,
                   gmres_tol=1e-12)
    mf = W.Manufactured
    u = mf.u(0.0, nodes)
    t = 0.0
    nsteps = int(round(t_end / dt))
    its = []
    for _ in range(nsteps):
        b_ext = mf.u(t, nodes) + dt * mf.F(t, nodes)
        u, sigma, k = S.heat_step(pb, u, mf.F(t, nodes), mf.u(t + dt, bn), b_ext=b_ext)
        its.append(k)
        t += dt
    inside = pb.inside
    err = np.max(np.abs(u[inside] - mf.u(t, nodes[inside])))
    return err, its


def _scalar_scheme_error(dt, t_end):
    """sin(pi x) cos(pi y) is an eigenfunction of -Lap (eigenvalue lam = 2 pi^2), so the
    semi-discrete IMEX Euler step reduces to a(1 + lam dt) = a_prev + dt (lam - 1) e^{-t}
    for its amplitude; the fully discrete error must match this temporal error."""
    lam = 2 * math.pi ** 2
    a, t = 1.0, 0.0
    for _ in range(int(round(t_end / dt))):
        a = (a + dt * (lam - 1) * math.exp(-t)) / (1 + lam * dt)
        t += dt
    return abs(a - math.exp(-t))


def test_manufactured_first_order():
    e1, its1 = _run(1e-2, 0.04)
    e2, its2 = _run(5e-3, 0.04)
    p1, p2 = _scalar_scheme_error(1e-2, 0.04), _scalar_scheme_error(5e-3, 0.04)
    # max |sin(pi x) cos(pi y)| over the nodes in Omega is close to 1
    assert abs(e1 - p1) < 0.03 * p1 and abs(e2 - p2) < 0.05 * p2, (e1, p1, e2, p2)
    assert 1.7 < e1 / e2 < 2.3
    assert max(its1 + its2) < 40


def _run_gear(dt, t_end):
    """Extrapolated Gear (alpha^2 = 2 dt / 3) started from exact data at t = 0 and dt."""
    wl = W.disk_with_hole(dt=dt)
    alpha = math.sqrt(2 * dt / 3)
    curves = G.make_curves(wl.curves)
    tr = T.build(wl.box, wl.q, wl.min_level, wl.max_level)
    nodes = tr.nodes()
    info = G.classify(curves, nodes)
    bn = np.concatenate([c.nodes for c in curves])
    bleaf = [tr.locate(p) for p in bn]
    M = V.uniform_operator(wl.min_level, wl.box, wl.q, alpha, order=[(b[1], b[2]) for b in tr.leaves])
    A = bie.nystrom_matrix(curves, alpha)
    pb = S.Problem(curves, tr, alpha, dt, info, bleaf, A, ext_mode="array", volume_op=lambda b: M @ b, use_lu=True)
    mf = W.Manufactured
    u_prev, u = mf.u(0.0, nodes), mf.u(dt, nodes)
    t = dt
    for _ in range(int(round(t_end / dt)) - 1):
        F, Fp = mf.F(t, nodes), mf.F(t - dt, nodes)
        b_ext = (4 * mf.u(t, nodes) - mf.u(t - dt, nodes)) / 3 + dt * (4 * F - 2 * Fp) / 3
        un, _, _ = S.heat_step_gear(pb, u, u_prev, F, Fp, mf.u(t + dt, bn), b_ext=b_ext)
        u_prev, u = u, un
        t += dt
    return float(np.max(np.abs(u[pb.inside] - mf.u(t, nodes[pb.inside]))))


def _scalar_gear_error(dt, t_end):
    lam = 2 * math.pi ** 2
    a_prev, a, t = 1.0, math.exp(-dt), dt
    for _ in range(int(round(t_end / dt)) - 1):
        rhs = (4 * a - a_prev) / 3 + dt * (lam - 1) * (4 * math.exp(-t) - 2 * math.exp(-(t - dt))) / 3
        a_prev, a = a, rhs / (1 + 2 * dt * lam / 3)
        t += dt
    return abs(a - math.exp(-t))


def test_manufactured_gear_second_order():
    # steps large enough that the temporal error dominates the spatial error of this small
    # discretisation (alpha >= 2.3 boundary spacings)
    e1, e2 = _run_gear(4e-2, 0.16), _run_gear(2e-2, 0.16)
    p1, p2 = _scalar_gear_error(4e-2, 0.16), _scalar_gear_error(2e-2, 0.16)
    assert abs(e1 - p1) < 0.05 * p1 and abs(e2 - p2) < 0.1 * p2, (e1, p1, e2, p2)
    assert 3.0 < e1 / e2 < 5.0
