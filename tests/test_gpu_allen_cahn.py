"""GPU parity of allen_cahn_step (Section 4, Example 3: u_t - eps Lap u = u (1 - u^2), u = 0
on Gamma, the reaction term explicit, alpha^2 = eps dt) against the oracle's Allen-Cahn step
on the disk-with-hole geometry (uniform level-4 tree, q = 4, N_Gamma = 256, N_D = 4096),
started, as in the paper, from values drawn uniformly from [-1/2, 1/2] (seeded): u after three
steps of dt = 1 with eps = 1e-4 (alpha = 0.01, a fifth of the boundary spacing) and with the
paper's eps = 1e-5 (alpha = 0.0032) to relative L2 <= 1e-10 in FP64 (GMRES tolerance 1e-12
on both sides) and <= 1e-6 in mixed precision."""
import math

import numpy as np
import pytest

import mh_workloads as W
from oracle import bie, geometry as G, step as S, tree as T, volume as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT, STEPS = 1.0, 3


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


@pytest.fixture(scope="module", params=[1e-4, 1e-5])
def case(request):
    EPS = request.param
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
                   volume_op=lambda b: M @ b, gmres_tol=1e-12, use_lu=True)
    u0 = np.random.default_rng(3).uniform(-0.5, 0.5, len(nodes))
    u0[~pb.inside] = 0.0
    u = u0.copy()
    zero = np.zeros(len(bn))
    for _ in range(STEPS):
        u, _, _ = S.allen_cahn_step(pb, u, zero)
    return wl, pb, u0, u, EPS


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_allen_cahn_step_matches_oracle(mh, case, prec, tol):
    wl, pb, u0, ref, EPS = case
    ctx = mh.Context(0)
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    prob = mh.Problem(ctx, gt, bnd, EPS * DT, 30, ext_mode=mh.MH_EXT_CONST, ext_const=[0.0, 0.0])
    assert np.array_equal(prob.regions(), pb.info.region)
    u = torch.tensor(u0, device="cuda")
    un = torch.empty_like(u)
    sigma = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
    f0 = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
    for _ in range(STEPS):
        mh.allen_cahn_step(ctx, prob, EPS, u, f0, un, sigma, gmres_tol=1e-12, prec=prec)
        u, un = un, u
    got = u.cpu().numpy()
    inside = pb.inside
    e = float(np.linalg.norm(got[inside] - ref[inside]) / np.linalg.norm(ref[inside]))
    print(f"allen_cahn_step eps={EPS} prec={prec}: rel L2 {e:.2e}")
    assert e < tol
    # outside Omega the step leaves the constant extension
    assert np.all(got[~inside] == 0.0)
