"""The binary32 contractions of the multipole passes on the tensor cores (Section 3.1: near-field
tables, P2M, M2L, P2L, L2P, M2P as batched matrix products; tcgen05 TF32 head/tail products).

* the uniform small case (q = 4, alpha = 0.1, N_D = 4096): the mixed-precision volume potential
  with the tensor cores agrees with the oracle's direct sum to 1e-6 and with the CUDA-core
  binary32 form to 1e-6, and the tensor-core launches ran;
* the full-size starfish tree (4027 leaves, p = 20): the same against the binary64 path;
* one full-size heat step in mixed precision: the double layer's multipole pass also runs on
  the tensor cores, and the step agrees with the CUDA-core form to 1e-6;
* no bounded device wait gave up (mh_tree_check)."""
import numpy as np
import pytest

import mh_workloads as W
from oracle import tree as T, volume as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _volume(mh, ctx, tree, alpha, p, b, prec, tc):
    out = torch.empty_like(b)
    ctx.tensor_cores(tc)
    ctx.profile(True)
    try:
        mh.mh_volume_potential(ctx, tree, alpha, p, b, out, prec=prec)
        tc_launches = ctx.profile_read("volume_contract_tc", reset=True)[1]
    finally:
        ctx.profile(False)
        ctx.tensor_cores(True)
    tree.check()
    return out, tc_launches


def test_uniform_volume_on_tensor_cores(mh):
    ctx = mh.Context(0)
    wl = W.disk_with_hole()
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level)
    ot = T.build(wl.box, wl.q, wl.min_level, wl.max_level)
    M = V.uniform_operator(wl.min_level, wl.box, wl.q, wl.alpha, order=[(b[1], b[2]) for b in ot.leaves])
    rng = np.random.default_rng(0)
    x = ot.nodes()
    bn = np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]) + 0.3 * rng.standard_normal(x.shape[0])
    ref = torch.tensor(M @ bn, device="cuda")
    b = torch.tensor(bn, device="cuda")
    tc, n_tc = _volume(mh, ctx, gt, wl.alpha, 20, b, mh.MH_PREC_MIXED, True)
    cc, n_cc = _volume(mh, ctx, gt, wl.alpha, 20, b, mh.MH_PREC_MIXED, False)
    print(f"uniform: tensor cores {_rel(tc, ref):.2e}, CUDA cores {_rel(cc, ref):.2e}, between {_rel(tc, cc):.2e}")
    assert n_tc > 0 and n_cc == 0
    assert _rel(tc, ref) < 1e-6 and _rel(tc, cc) < 1e-6


def test_full_size_volume_on_tensor_cores(mh):
    ctx = mh.Context(0)
    wl = W.starfish_domain()
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    x = gt.nodes().cpu().numpy()
    b = torch.tensor(wl.forcing(x) * wl.dt + np.cos(2 * x[:, 0]) * np.sin(x[:, 1]), device="cuda")
    f64, _ = _volume(mh, ctx, gt, wl.alpha, wl.p, b, mh.MH_PREC_FP64, True)
    tc, n_tc = _volume(mh, ctx, gt, wl.alpha, wl.p, b, mh.MH_PREC_MIXED, True)
    cc, _ = _volume(mh, ctx, gt, wl.alpha, wl.p, b, mh.MH_PREC_MIXED, False)
    print(f"full size: tensor cores vs binary64 {_rel(tc, f64):.2e}, CUDA cores vs binary64 {_rel(cc, f64):.2e}")
    assert n_tc > 0
    assert _rel(tc, f64) < 1e-6 and _rel(tc, cc) < 1e-6


def test_full_size_step_on_tensor_cores(mh):
    ctx = mh.Context(0)
    wl = W.starfish_domain()
    tree = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    prob = mh.Problem(ctx, tree, bnd, wl.dt, wl.p, ext_mode=mh.MH_EXT_CONST, ext_const=wl.ext_const)
    F = torch.tensor(wl.forcing(tree.nodes().cpu().numpy()), device="cuda")
    f = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
    out = []
    for tc in (True, False):
        u = torch.zeros(tree.n_nodes, dtype=torch.float64, device="cuda")
        un = torch.empty_like(u)
        s = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
        ctx.tensor_cores(tc)
        ctx.profile(True)
        try:
            for _ in range(2):
                mh.heat_step(ctx, prob, u, F, f, un, s, gmres_tol=1e-10, prec=mh.MH_PREC_MIXED)
                u, un = un, u
            n_dl = ctx.profile_read("dlp_fmm_contract_tc", reset=True)[1]
        finally:
            ctx.profile(False)
            ctx.tensor_cores(True)
        tree.check()
        assert (n_dl > 0) == tc
        out.append(u)
    ins = torch.tensor(prob.regions() == -1, device="cuda")
    d = _rel(out[0][ins], out[1][ins])
    print(f"full-size step: tensor cores vs CUDA cores {d:.2e}")
    assert d < 1e-6
