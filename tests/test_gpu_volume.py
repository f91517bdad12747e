"""GPU parity of mh_volume_potential (Section 3.1) against the oracle's direct sum of
exact leaf integrals.

* uniform level-4 tree (q = 4, alpha = 0.1, N_D = 4096), every node: relative L2
  <= 1e-10 in FP64 at p = 20 (the multipole truncation error there is ~1e-11), and
  <= 1e-6 in mixed precision;
* a small adaptive tree (levels 2..6, q = 4, U, V, W and X lists all populated),
  sampled nodes: <= 1e-10 at p = 40;
* the full-size adaptive tree of the starfish workload (4027 leaves, 257,728 nodes,
  alpha^2 = 1e-3, p = 20), 256 nodes sampled over every leaf level: <= 1e-8 (multipole truncation at p = 20 on the
  one-level-apart W/X interactions dominates; see the p = 40 case for the exact bar)."""
import math

import numpy as np
import pytest

import mh_workloads as W
from oracle import pool, tree as T, volume as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(mh):
    return mh.Context(0)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _smooth_plus_noise(nodes, seed):
    rng = np.random.default_rng(seed)
    x, y = nodes[:, 0], nodes[:, 1]
    return np.sin(3 * x) * np.cos(2 * y) + 0.3 * rng.standard_normal(nodes.shape[0])


def test_uniform_tree_all_nodes(mh, ctx):
    wl = W.disk_with_hole()
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level)
    ot = T.build(wl.box, wl.q, wl.min_level, wl.max_level)
    M = V.uniform_operator(wl.min_level, wl.box, wl.q, wl.alpha, order=[(b[1], b[2]) for b in ot.leaves])
    b = _smooth_plus_noise(ot.nodes(), 0)
    ref = M @ b
    out = torch.empty(gt.n_nodes, dtype=torch.float64, device="cuda")
    bd = torch.tensor(b, device="cuda")
    mh.mh_volume_potential(ctx, gt, wl.alpha, 20, bd, out)
    e64 = _rel(out.cpu().numpy(), ref)
    mh.mh_volume_potential(ctx, gt, wl.alpha, 20, bd, out, prec=mh.MH_PREC_MIXED)
    e32 = _rel(out.cpu().numpy(), ref)
    print(f"uniform: fp64 {e64:.2e} mixed {e32:.2e}")
    assert e64 < 1e-10
    assert e32 < 1e-6


def test_small_adaptive_tree(mh, ctx):
    wl = W.starfish_domain(n_per_curve=64)
    alpha = 0.05
    gt = mh.Tree(ctx, wl.box, 4, 2, 6, wl.forcing, 1e-6)
    ot = T.build(wl.box, 4, 2, 6, wl.forcing, 1e-6)
    U, Vl, Wl, Xl = T.lists(ot)
    assert sum(len(v) for v in Wl.values()) > 0 and sum(len(v) for v in Xl.values()) > 0
    nodes = ot.nodes()
    b = _smooth_plus_noise(nodes, 1)
    rng = np.random.default_rng(2)
    sel = rng.choice(nodes.shape[0], 120, replace=False)
    ref = V.volume_potential(ot.leaf_array(), b.reshape(len(ot.leaves), -1), 4, alpha, nodes[sel])
    out = torch.empty(gt.n_nodes, dtype=torch.float64, device="cuda")
    errs = {}
    for p in (20, 40):
        mh.mh_volume_potential(ctx, gt, alpha, p, torch.tensor(b, device="cuda"), out)
        errs[p] = _rel(out.cpu().numpy()[sel], ref)
    print("small adaptive:", errs)
    assert errs[40] < 1e-10
    assert errs[20] < 1e-6


def test_full_size_adaptive_sampled(mh, ctx):
    wl = W.starfish_domain()
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    ot = T.build(wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    nodes = ot.nodes()
    b = wl.forcing(nodes) * wl.dt + np.cos(2 * nodes[:, 0]) * np.sin(nodes[:, 1])
    out = torch.empty(gt.n_nodes, dtype=torch.float64, device="cuda")
    mh.mh_volume_potential(ctx, gt, wl.alpha, wl.p, torch.tensor(b, device="cuda"), out)
    # 256 sampled nodes spread over every leaf level (levels 4..8: about 51 per level), so
    # that targets in small and large leaves and every list type contribute
    rng = np.random.default_rng(3)
    qq = wl.q * wl.q
    lev = np.repeat(np.array([l[0] for l in ot.leaves]), qq)
    levels = sorted(set(lev.tolist()))
    assert levels == [4, 5, 6, 7, 8]
    per = [256 // len(levels) + (1 if k < 256 % len(levels) else 0) for k in range(len(levels))]
    sel = np.concatenate([rng.choice(np.nonzero(lev == l)[0], n, replace=False) for l, n in zip(levels, per)])
    assert sel.size == 256
    ref = pool.volume_potential(ot.leaf_array(), b.reshape(len(ot.leaves), -1), wl.q, wl.alpha, nodes[sel])
    got = out.cpu().numpy()[sel]
    e = _rel(got, ref)
    print(f"full-size adaptive p=20, 256 nodes: {e:.2e}; per level " +
          " ".join(f"{l}:{_rel(got[lev[sel] == l], ref[lev[sel] == l]):.1e}" for l in levels))
    assert e < 1e-8


@pytest.mark.parametrize("prec", [0, 1])
def test_overlapped_and_timed_forms_identical(mh, ctx, prec):
    """Without region timers the near tables run on the context stream while the multipole
    passes run on a second stream; with the timers every phase runs in order on one stream.
    Both write U as near, then add far, and no sum depends on timing: identical results."""
    wl = W.starfish_domain(n_per_curve=64)
    gt = mh.Tree(ctx, wl.box, 4, 2, 6, wl.forcing, 1e-6)
    rng = np.random.default_rng(7)
    b = torch.tensor(rng.standard_normal(gt.n_nodes), device="cuda")
    fast, timed = torch.empty_like(b), torch.empty_like(b)
    mh.mh_volume_potential(ctx, gt, 0.05, 20, b, fast, prec=prec)
    ctx.profile(True)
    try:
        mh.mh_volume_potential(ctx, gt, 0.05, 20, b, timed, prec=prec)
        _, launches, _, _ = ctx.profile_read("volume_contract", reset=True)
    finally:
        ctx.profile(False)
    assert launches >= 4   # near tables, P2M, M2L + P2L, output: one timed region each
    assert torch.equal(fast, timed)


def test_minimal_uniform_tree(mh, ctx):
    """The smallest tree with a far field: uniform level 2 (16 leaves, q = 4).  Multipoles exist
    only at the leaf level (no M2M / L2L chain), M2L couples the non-adjacent leaves and the near
    tables the adjacent ones.  A missing or doubled interaction shows at 1e-2; the bar leaves
    room for the truncation at p = 20."""
    box, q, alpha = (-1.0, -1.0, 2.0), 4, 0.1
    gt = mh.Tree(ctx, box, q, 2, 2)
    ot = T.build(box, q, 2, 2)
    assert gt.n_nodes == 256
    M = V.uniform_operator(2, box, q, alpha, order=[(b[1], b[2]) for b in ot.leaves])
    b = _smooth_plus_noise(ot.nodes(), 3)
    out = torch.empty(gt.n_nodes, dtype=torch.float64, device="cuda")
    for prec, tol in ((0, 1e-8), (1, 1e-6)):
        mh.mh_volume_potential(ctx, gt, alpha, 20, torch.tensor(b, device="cuda"), out, prec=prec)
        assert _rel(out.cpu().numpy(), M @ b) < tol, prec
