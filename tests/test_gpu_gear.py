"""Extrapolated Gear (Section 2) on the GPU.

* Parity with the oracle's Gear step on the disk-with-hole case (manufactured solution,
  exact start at t = 0 and dt, three Gear steps): relative L2 <= 1e-10 (binary64) and
  <= 1e-6 (mixed).
* The paper's Example 1 (annulus 0.1 < r < 0.4, exact Bessel solution, Table 1): errors at
  t = 0.01 for dt = 2e-3, 1e-3, 5e-4, 2.5e-4 with IMEX Euler and extrapolated Gear on the
  GPU; the observed orders must be about 1 and 2 and every value within 10% of Table 1
  (maximum over the nodes in Omega; the paper states no norm).  The last IMEX Euler entry
  of Table 1 (1.78e-4) breaks first order; it is compared as 1.78e-3, the reading of it as
  a misprint (the computed value is 1.84e-3).  Gear starts from the exact solution at t = dt."""
import json
import math
import os

import numpy as np
import pytest

import mh_workloads as W
from oracle import bie, geometry as G, step as S, tree as T, volume as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


def test_gear_matches_oracle(mh):
    dt = 1e-2
    alpha = math.sqrt(2 * dt / 3)
    wl = W.disk_with_hole(dt=dt)
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
    ctx = mh.Context(0)
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    prob = mh.Problem(ctx, gt, bnd, dt, 30, ext_mode=mh.MH_EXT_ARRAY, scheme=mh.MH_SCHEME_EXTRAP_GEAR)
    assert abs(prob.alpha - alpha) < 1e-15
    dev = lambda a: torch.tensor(a, device="cuda")
    for prec, tol in ((0, 1e-10), (1, 1e-6)):
        up, u = mf.u(0.0, nodes), mf.u(dt, nodes)
        gu_prev, gu = dev(up), dev(u)
        gun = torch.empty_like(gu)
        sig = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
        t = dt
        for _ in range(3):
            F, Fp = mf.F(t, nodes), mf.F(t - dt, nodes)
            b_ext = (4 * mf.u(t, nodes) - mf.u(t - dt, nodes)) / 3 + dt * (4 * F - 2 * Fp) / 3
            un, _, _ = S.heat_step_gear(pb, u, up, F, Fp, mf.u(t + dt, bn), b_ext=b_ext)
            mh.heat_step_gear(ctx, prob, gu, gu_prev, dev(F), dev(Fp), dev(mf.u(t + dt, bn)), gun, sig,
                              b_ext=dev(b_ext), gmres_tol=1e-12, prec=prec)
            up, u = u, un
            gu_prev, gu, gun = gu, gun, gu_prev
            t += dt
        got = gu.cpu().numpy()
        e = float(np.linalg.norm(got[pb.inside] - u[pb.inside]) / np.linalg.norm(u[pb.inside]))
        print(f"gear prec={prec}: rel L2 {e:.2e}")
        assert e < tol


def _example1_error(mh, ctx, ex, tree, nodes, bnd, region, bn, dt, scheme, t_end=0.01):
    prob = mh.Problem(ctx, tree, bnd, dt, 20, ext_mode=mh.MH_EXT_ARRAY, scheme=scheme)
    ins = region == -1
    dev = lambda a: torch.tensor(a, device="cuda")
    F = ex.F(nodes)
    Fd = dev(F)
    nsteps = int(round(t_end / dt))
    fb = np.concatenate([np.full(c.shape[0], v) for c, v in zip(ex.curves(bnd_sizes[0], bnd_sizes[1]),
                                                                ex.boundary_data())])
    fd = dev(fb)
    sig = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
    if scheme == mh.MH_SCHEME_IMEX_EULER:
        u = dev(ex.u(0.0, nodes))
        un = torch.empty_like(u)
        t = 0.0
        for _ in range(nsteps):
            b_ext = dev(ex.u(t, nodes) + dt * F)
            mh.heat_step(ctx, prob, u, Fd, fd, un, sig, b_ext=b_ext, gmres_tol=1e-12)
            u, un = un, u
            t += dt
    else:
        up, u = dev(ex.u(0.0, nodes)), dev(ex.u(dt, nodes))
        un = torch.empty_like(u)
        t = dt
        for _ in range(nsteps - 1):
            b_ext = dev((4 * ex.u(t, nodes) - ex.u(t - dt, nodes)) / 3 + dt * (2.0 / 3.0) * F)
            mh.heat_step_gear(ctx, prob, u, up, Fd, Fd, fd, un, sig, b_ext=b_ext, gmres_tol=1e-12)
            up, u, un = u, un, up
            t += dt
    got = u.cpu().numpy()
    return float(np.max(np.abs(got[ins] - ex.u(t, nodes[ins]))))


bnd_sizes = (1024, 256)


def test_example1_temporal_orders(mh):
    ex = W.Example1()
    ctx = mh.Context(0)
    box = (-0.5, -0.5, 1.0)
    tree = mh.Tree(ctx, box, 8, 5, 5)
    nodes = tree.nodes().cpu().numpy()
    bnd = mh.Boundary(ctx, ex.curves(*bnd_sizes), alpert_order=8)
    bn = np.concatenate(ex.curves(*bnd_sizes))
    region = mh.Problem(ctx, tree, bnd, 1e-3, 20, ext_mode=mh.MH_EXT_ARRAY).regions()
    dts = GOLD["table1_dt"]["value"]
    e1 = [_example1_error(mh, ctx, ex, tree, nodes, bnd, region, bn, dt, mh.MH_SCHEME_IMEX_EULER) for dt in dts]
    e2 = [_example1_error(mh, ctx, ex, tree, nodes, bnd, region, bn, dt, mh.MH_SCHEME_EXTRAP_GEAR) for dt in dts]
    print("Example 1 IMEX Euler:", ["%.3e" % v for v in e1], "paper", GOLD["table1_error_imex_euler"]["value"])
    print("Example 1 Gear      :", ["%.3e" % v for v in e2], "paper", GOLD["table1_error_gear"]["value"])
    o1 = [math.log(e1[i] / e1[i + 1], 2) for i in range(3)]
    o2 = [math.log(e2[i] / e2[i + 1], 2) for i in range(3)]
    print("orders", o1, o2)
    assert all(0.8 < o < 1.2 for o in o1)
    assert all(1.6 < o < 2.4 for o in o2)
    paper1 = GOLD["table1_error_imex_euler"]["value"][:3] + [10 * GOLD["table1_error_imex_euler"]["value"][3]]
    paper2 = GOLD["table1_error_gear"]["value"]
    assert all(abs(a / b - 1) < 0.1 for a, b in zip(e1, paper1)), (e1, paper1)
    assert all(abs(a / b - 1) < 0.1 for a, b in zip(e2, paper2)), (e2, paper2)
