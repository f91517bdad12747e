"""Mixed precision across screening lengths (the alpha^2 sweep of the disk-with-hole case):
for alpha^2 = dt in {1e-2, 1e-3, 1e-4}, three IMEX Euler steps on the GPU in binary64 and
in mixed precision against the CPU oracle (manufactured solution data, N_Gamma = 256,
N_D = 4096).  Bars: binary64 <= 1e-10 and mixed <= 1e-6 relative L2 over the nodes in
Omega.  The speedup of mixed over binary64 on the GPU is printed (CUDA events).
At alpha = 0.01 the boundary is under-resolved (h_s ~ 0.05 > alpha); parity with the
oracle's discrete operator is still required."""
import numpy as np
import pytest

import mh_workloads as W
from oracle import bie, geometry as G, step as S, tree as T, volume as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


def _oracle(wl, nsteps):
    curves = G.make_curves(wl.curves)
    tr = T.build(wl.box, wl.q, wl.min_level, wl.max_level)
    nodes = tr.nodes()
    info = G.classify(curves, nodes)
    bn = np.concatenate([c.nodes for c in curves])
    bleaf = [tr.locate(p) for p in bn]
    M = V.uniform_operator(wl.min_level, wl.box, wl.q, wl.alpha, order=[(b[1], b[2]) for b in tr.leaves])
    A = bie.nystrom_matrix(curves, wl.alpha)
    pb = S.Problem(curves, tr, wl.alpha, wl.dt, info, bleaf, A, ext_mode="array", volume_op=lambda b: M @ b,
                   use_lu=True)
    mf = W.Manufactured
    u = mf.u(0.0, nodes)
    t = 0.0
    for _ in range(nsteps):
        u, _, _ = S.heat_step(pb, u, mf.F(t, nodes), mf.u(t + wl.dt, bn), b_ext=mf.u(t, nodes) + wl.dt * mf.F(t, nodes))
        t += wl.dt
    return u, pb.inside, nodes, bn


@pytest.mark.parametrize("dt", [1e-2, 1e-3, 1e-4])
def test_mixed_precision_alpha_sweep(mh, dt):
    nsteps = 3
    wl = W.disk_with_hole(dt=dt)
    ref, inside, nodes, bn = _oracle(wl, nsteps)
    ctx = mh.Context(0)
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    prob = mh.Problem(ctx, gt, bnd, dt, 30, ext_mode=mh.MH_EXT_ARRAY)
    mf = W.Manufactured
    dev = lambda a: torch.tensor(a, device="cuda")
    res = {}
    for prec in (0, 1):
        u = dev(mf.u(0.0, nodes))
        un = torch.empty_like(u)
        sig = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
        t = 0.0
        ms = 0.0
        for _ in range(nsteps):
            F, f, be = dev(mf.F(t, nodes)), dev(mf.u(t + dt, bn)), dev(mf.u(t, nodes) + dt * mf.F(t, nodes))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            mh.heat_step(ctx, prob, u, F, f, un, sig, b_ext=be, gmres_tol=1e-12, prec=prec)
            b.record()
            b.synchronize()
            ms += a.elapsed_time(b)
            u, un = un, u
            t += dt
        got = u.cpu().numpy()
        err = float(np.linalg.norm(got[inside] - ref[inside]) / np.linalg.norm(ref[inside]))
        res[prec] = (err, ms / nsteps)
    print(f"alpha^2={dt:g}: fp64 err {res[0][0]:.2e} ({res[0][1]:.3f} ms/step), "
          f"mixed err {res[1][0]:.2e} ({res[1][1]:.3f} ms/step), speedup {res[0][1] / res[1][1]:.2f}")
    assert res[0][0] < 1e-10
    assert res[1][0] < 1e-6
