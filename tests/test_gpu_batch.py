"""Batched stepping (one CUDA graph launch per time step) and the autotuner on the GPU.

* A batch of small problems of the batched workload (fewer nodes per curve, coarser trees)
  stepped three times (an eager step that records the graph, then two graph launches) agrees
  with the same problems stepped one by one by heat_step (host-synchronised GMRES): the two
  GMRES variants differ only in rounding and in where they stop below the tolerance.
* A one-problem batch in binary64 agrees with heat_step to 1e-10.
* A solve outside the batch that grows the Krylov workspace between batch steps makes the
  batch record its graph again (a recorded graph holds the workspace).
* The autotuner's choice is among the candidates, its error report falls with p and the
  chosen order meets the tolerance."""
import numpy as np
import pytest

import mh_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = [(0, 192, 1e-5), (3, 160, 3e-6), (7, 224, 1e-5), (11, 128, 1e-6)]


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(mh):
    return mh.Context(0)


def _make(mh, ctx, wl, p=16):
    tree = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    prob = mh.Problem(ctx, tree, bnd, wl.dt, p, ext_mode=mh.MH_EXT_CONST, ext_const=wl.ext_const)
    nodes = tree.nodes().cpu().numpy()
    F = torch.tensor(wl.forcing(nodes), device="cuda")
    return tree, bnd, prob, F


def _inside(prob):
    return torch.tensor(prob.regions() == -1, device="cuda")


@pytest.mark.parametrize("prec,tol", [(1, 1e-7)])
def test_batch_matches_single_steps(mh, ctx, prec, tol):
    wls = [W.batch_problem(i, npc=npc, refine_tol=rt) for i, npc, rt in SMALL]
    a = [_make(mh, ctx, wl) for wl in wls]      # batched
    b = [_make(mh, ctx, wl) for wl in wls]      # one by one
    for grp in (a, b):                          # two problems with the previous-increment start
        grp[0][2].set_warm_start(mh.MH_WARM_SECANT)
        grp[2][2].set_warm_start(mh.MH_WARM_SECANT)
    batch = mh.Batch(ctx, [x[2] for x in a])
    u = [torch.zeros(x[0].n_nodes, dtype=torch.float64, device="cuda") for x in a]
    s = [torch.zeros(x[1].n, dtype=torch.float64, device="cuda") for x in a]
    f = [torch.zeros(x[1].n, dtype=torch.float64, device="cuda") for x in a]
    F = [x[3] for x in a]
    for step in range(3):
        infos = batch.step(u, F, f, s, gmres_tol=1e-10, prec=prec)
        assert all(i.gmres_rel_residual <= 1e-10 for i in infos)
        if step == 0:
            assert batch.graph_kernels > 0
    for k, (tree, bnd, prob, Fk) in enumerate(b):
        uu = torch.zeros(tree.n_nodes, dtype=torch.float64, device="cuda")
        un = torch.empty_like(uu)
        ss = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
        for _ in range(3):
            mh.heat_step(ctx, prob, uu, Fk, f[k], un, ss, gmres_tol=1e-10, prec=prec)
            uu, un = un, uu
        ins = _inside(prob)
        err = (torch.linalg.norm((u[k] - uu)[ins]) / torch.linalg.norm(uu[ins])).item()
        assert err <= tol, (k, err)


def test_one_problem_batch_fp64(mh, ctx):
    wl = W.batch_problem(3, npc=160, refine_tol=3e-6)
    t1, b1, p1, F1 = _make(mh, ctx, wl)
    t2, b2, p2, F2 = _make(mh, ctx, wl)
    batch = mh.Batch(ctx, [p1])
    u1 = torch.zeros(t1.n_nodes, dtype=torch.float64, device="cuda")
    s1 = torch.zeros(b1.n, dtype=torch.float64, device="cuda")
    f = torch.zeros(b1.n, dtype=torch.float64, device="cuda")
    u2, un = torch.zeros_like(u1), torch.empty_like(u1)
    s2 = torch.zeros_like(s1)
    for _ in range(3):
        batch.step([u1], [F1], [f], [s1], gmres_tol=1e-12, prec=mh.MH_PREC_FP64)
        mh.heat_step(ctx, p2, u2, F2, f, un, s2, gmres_tol=1e-12, prec=mh.MH_PREC_FP64)
        u2, un = un, u2
    ins = _inside(p2)
    assert (torch.linalg.norm((u1 - u2)[ins]) / torch.linalg.norm(u2[ins])).item() <= 1e-10


def test_batch_after_outside_solve(mh, ctx):
    """A solve outside the batch (heat_step, whose GMRES grows the problem's Krylov workspace)
    between two batch steps: the batch records its graph again on the new workspace, and the
    steps agree with heat_step throughout (mixed precision)."""
    wl = W.batch_problem(0, npc=192, refine_tol=1e-5)
    t1, b1, p1, F1 = _make(mh, ctx, wl)
    t2, b2, p2, F2 = _make(mh, ctx, wl)
    batch = mh.Batch(ctx, [p1])
    u1 = torch.zeros(t1.n_nodes, dtype=torch.float64, device="cuda")
    s1 = torch.zeros(b1.n, dtype=torch.float64, device="cuda")
    f = torch.zeros(b1.n, dtype=torch.float64, device="cuda")
    u2, un = torch.zeros_like(u1), torch.empty_like(u1)
    s2 = torch.zeros_like(s1)
    tmp = torch.empty_like(u1)
    for step in range(4):
        if step == 2:   # an outside solve on the batch's own problem: same u and density
            mh.heat_step(ctx, p1, u1, F1, f, tmp, s1, gmres_tol=1e-10, prec=mh.MH_PREC_MIXED)
            u1.copy_(tmp)
            mh.heat_step(ctx, p2, u2, F2, f, un, s2, gmres_tol=1e-10, prec=mh.MH_PREC_MIXED)
            u2, un = un, u2
        infos = batch.step([u1], [F1], [f], [s1], gmres_tol=1e-10, prec=mh.MH_PREC_MIXED)
        assert infos[0].gmres_rel_residual <= 1e-10
        mh.heat_step(ctx, p2, u2, F2, f, un, s2, gmres_tol=1e-10, prec=mh.MH_PREC_MIXED)
        u2, un = un, u2
    ins = _inside(p2)
    assert (torch.linalg.norm((u1 - u2)[ins]) / torch.linalg.norm(u2[ins])).item() <= 1e-7


def test_autotuner(mh, ctx):
    wl = W.batch_problem(7, npc=224, refine_tol=1e-5)
    tree, bnd, prob, F = _make(mh, ctx, wl)
    f = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
    p, tile, rep = mh.mh_autotune(ctx, tree, bnd, wl.dt, F, f, p_cand=(10, 16, 24), err_tol=1e-7, steps=3)
    assert p in (10, 16, 24) and tile in (128, 256, 512)
    errs = {e.p: e.rel_err for e in rep[:3]}
    assert errs[10] >= errs[24]
    if min(errs.values()) <= 1e-7:
        assert errs[p] <= 1e-7
    assert [e.near_tile for e in rep[3:]] == [128, 256, 512] and all(e.p == p for e in rep[3:])
    assert all(e.ms_per_step > 0 for e in rep)


def test_full_size_graph_step_matches_binary64(mh, ctx):
    """The starfish workload at full size (N_Gamma = 6144, N_D = 257,728, p = 20) in the form
    the headline is timed in: one graph launch per step through the batch API, mixed precision.
    Three steps agree with three binary64 heat_step calls on the stream to the 1e-6 bar of the
    metric (relative L2 over Omega)."""
    wl = W.starfish_domain()
    t1, b1, p1, F1 = _make(mh, ctx, wl, p=wl.p)
    t2, b2, p2, F2 = _make(mh, ctx, wl, p=wl.p)
    batch = mh.Batch(ctx, [p1])
    u1 = torch.zeros(t1.n_nodes, dtype=torch.float64, device="cuda")
    s1 = torch.zeros(b1.n, dtype=torch.float64, device="cuda")
    f = torch.zeros(b1.n, dtype=torch.float64, device="cuda")
    u2, un = torch.zeros_like(u1), torch.empty_like(u1)
    s2 = torch.zeros_like(s1)
    for _ in range(3):
        info = batch.step([u1], [F1], [f], [s1], gmres_tol=1e-10, prec=mh.MH_PREC_MIXED)[0]
        assert info.gmres_rel_residual <= 1e-10
        mh.heat_step(ctx, p2, u2, F2, f, un, s2, gmres_tol=1e-10, prec=mh.MH_PREC_FP64)
        u2, un = un, u2
    ins = _inside(p2)
    err = (torch.linalg.norm((u1 - u2)[ins]) / torch.linalg.norm(u2[ins])).item()
    assert err <= 1e-6, err
