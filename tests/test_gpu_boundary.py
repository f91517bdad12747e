"""GPU parity of the boundary path through the C ABI against the CPU oracle:
geometry (Section 3.2), the Nystrom operator of eq. discrete_sys, GMRES (FP64 and
mixed precision with FP64 refinement), and the off-surface double layer with the
near-boundary rules.  Tolerances: geometry 1e-12 relative to the max entry; operator
products, solves and off-surface values 1e-10 relative L2 (the FP64 bar).  The operator
cannot be compared more tightly: the innermost Alpert nodes sit x_1 h |y'| ~ 5e-6 from
their target, where (y - x).n_y is formed from coordinates of size 1 with cancellation,
so both implementations carry ~1e-11 relative rounding in those entries."""
import numpy as np
import pytest

import mh_workloads as W
from oracle import bie, geometry as G

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


@pytest.mark.parametrize("geom", ["disk_with_hole", "starfish_small"])
def test_geometry_and_operator(mh, ctx, geom):
    wl = W.disk_with_hole() if geom == "disk_with_hole" else W.starfish_domain(n_per_curve=128, n_holes=3)
    curves = G.make_curves(wl.curves)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    g = bnd.geometry()
    d1 = np.concatenate([c.d1 for c in curves])
    d2 = np.concatenate([c.d2 for c in curves])
    kd = np.concatenate([c.kdiag for c in curves])
    assert np.max(np.abs(g[:, 2:4] - d1)) < 1e-12 * np.max(np.abs(d1))
    assert np.max(np.abs(g[:, 4:6] - d2)) < 1e-11 * np.max(np.abs(d2))
    assert np.max(np.abs(g[:, 7] - kd)) < 1e-11 * np.max(np.abs(kd))
    A = bie.nystrom_matrix(curves, wl.alpha)
    rng = np.random.default_rng(1)
    for _ in range(2):
        s = rng.standard_normal(bnd.n)
        out = torch.empty(bnd.n, dtype=torch.float64, device="cuda")
        mh.mh_double_layer_apply(ctx, bnd, wl.alpha, torch.tensor(s, device="cuda"), out)
        assert _rel(out.cpu().numpy(), A @ s) < 1e-10
    # plain trapezoid with the diagonal limit
    bnd0 = mh.Boundary(ctx, wl.curves, alpert_order=0)
    A0 = bie.nystrom_matrix(curves, wl.alpha, None)
    s = rng.standard_normal(bnd.n)
    out = torch.empty(bnd.n, dtype=torch.float64, device="cuda")
    mh.mh_double_layer_apply(ctx, bnd0, wl.alpha, torch.tensor(s, device="cuda"), out)
    assert _rel(out.cpu().numpy(), A0 @ s) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_gmres_matches_lu(mh, ctx, prec):
    wl = W.disk_with_hole()
    curves = G.make_curves(wl.curves)
    A = bie.nystrom_matrix(curves, wl.alpha)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    rng = np.random.default_rng(2)
    rhs = rng.standard_normal(bnd.n)
    x = np.linalg.solve(A, rhs)
    sig = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
    info = mh.mh_gmres_solve(ctx, bnd, wl.alpha, torch.tensor(rhs, device="cuda"), sig, tol=1e-12, prec=prec)
    assert info.converged and info.rel_residual <= 1e-12
    assert _rel(sig.cpu().numpy(), x) < 1e-10
    if prec == 1:
        assert info.refinements >= 1


def test_gmres_reports_non_convergence(mh, ctx):
    wl = W.disk_with_hole()
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    rhs = torch.ones(bnd.n, dtype=torch.float64, device="cuda")
    sig = torch.zeros_like(rhs)
    with pytest.raises(mh.MHError) as e:
        mh.mh_gmres_solve(ctx, bnd, wl.alpha, rhs, sig, tol=1e-14, max_iter=2)
    assert e.value.status == 5


def test_bad_orientation_is_rejected(mh, ctx):
    wl = W.disk_with_hole()
    with pytest.raises(mh.MHError) as e:
        mh.Boundary(ctx, [wl.curves[1], wl.curves[0]])
    assert e.value.status == 2


def test_off_surface_all_regimes(mh, ctx):
    wl = W.disk_with_hole()
    curves = G.make_curves(wl.curves)
    A = bie.nystrom_matrix(curves, wl.alpha)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    rng = np.random.default_rng(3)
    sigma = rng.standard_normal(bnd.n) * 0.1 + np.cos(np.concatenate([c.t for c in curves]))
    hs = 2 * np.pi / 128
    # random interior points plus points at 3 h_s, 0.5 h_s, 0.1 h_s from each curve
    r = np.sqrt(rng.uniform(0.0, 0.95, 300))
    th = rng.uniform(0, 2 * np.pi, 300)
    pts = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    near = []
    for d in (3.0, 0.5, 0.1, 0.02):
        for t0 in (0.3, 2.0, 4.4):
            near.append([(1 - d * hs) * np.cos(t0), (1 - d * hs) * np.sin(t0)])
            near.append([0.2 + (0.3 + d * 0.3 * hs) * np.cos(t0), (0.3 + d * 0.3 * hs) * np.sin(t0)])
    pts = np.concatenate([pts, np.array(near)])
    info = G.classify(curves, pts)
    pts = pts[info.region == -1]
    info = G.classify(curves, pts)
    ref = bie.dlp_eval(curves, sigma, wl.alpha, pts, info, A @ sigma)
    out = torch.empty(pts.shape[0], dtype=torch.float64, device="cuda")
    mh.mh_double_layer_apply(ctx, bnd, wl.alpha, torch.tensor(sigma, device="cuda"), out,
                             targets=torch.tensor(pts, device="cuda"))
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def test_full_size_starfish_operator_sampled_rows(mh, ctx):
    """N_Gamma = 6144 (6 curves x 1024): A sigma on 24 sampled rows against the oracle's rows."""
    wl = W.starfish_domain()
    curves = G.make_curves(wl.curves)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    rng = np.random.default_rng(4)
    s = rng.standard_normal(bnd.n)
    out = torch.empty(bnd.n, dtype=torch.float64, device="cuda")
    mh.mh_double_layer_apply(ctx, bnd, wl.alpha, torch.tensor(s, device="cuda"), out)
    rows = np.sort(rng.choice(bnd.n, 24, replace=False))
    R = bie.nystrom_matrix(curves, wl.alpha, rows=rows)
    ref = R @ s
    assert _rel(out.cpu().numpy()[rows], ref) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_gmres_zero_rhs(mh, ctx, prec):
    """A zero right-hand side has the solution 0: returned at once, no iteration."""
    wl = W.disk_with_hole()
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    sig = torch.ones(bnd.n, dtype=torch.float64, device="cuda")
    rhs = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
    info = mh.mh_gmres_solve(ctx, bnd, wl.alpha, rhs, sig, tol=1e-10, prec=prec)
    assert info.converged and info.iterations == 0 and info.rel_residual == 0.0
    assert torch.count_nonzero(sig).item() == 0


def test_empty_target_set(mh, ctx):
    """No targets: nothing is evaluated and the output buffer is left as it was, through the
    binding (an empty tensor) and through the C ABI (a valid pointer with n_targets = 0)."""
    wl = W.disk_with_hole()
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    sig = torch.ones(bnd.n, dtype=torch.float64, device="cuda")
    out = torch.full((bnd.n,), 7.0, dtype=torch.float64, device="cuda")
    buf = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    mh.mh_double_layer_apply(ctx, bnd, wl.alpha, sig, out, targets=buf[:0])
    st = mh._lib.mh_double_layer_apply(ctx.h, bnd.h, wl.alpha, mh._ptr(sig), mh._ptr(buf), 0, mh._ptr(out), 0)
    assert st == 0
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())


def test_ragged_boundary(mh, ctx):
    """N_Gamma = 126 + 128 = 254: not a multiple of 4 (the 8-byte GEMV and the binary64 residual
    of the mixed solve), one 128-node source tile straddling the two curves, and a ragged last
    128-node chunk of the 16x fine grid on the outer curve (2016 = 15 x 128 + 96).  Same bars as
    the aligned case: binary64 products, solves and off-surface values 1e-10 relative."""
    spec = [W.circle_nodes((0.0, 0.0), 1.0, 126, clockwise=False),
            W.circle_nodes((0.2, 0.0), 0.3, 128, clockwise=True)]
    alpha = 0.1
    curves = G.make_curves(spec)
    A = bie.nystrom_matrix(curves, alpha)
    bnd = mh.Boundary(ctx, spec, alpert_order=8)
    assert bnd.n == 254
    rng = np.random.default_rng(5)
    s = rng.standard_normal(bnd.n)
    out = torch.empty(bnd.n, dtype=torch.float64, device="cuda")
    mh.mh_double_layer_apply(ctx, bnd, alpha, torch.tensor(s, device="cuda"), out)
    assert _rel(out.cpu().numpy(), A @ s) < 1e-10
    mh.mh_double_layer_apply(ctx, bnd, alpha, torch.tensor(s, device="cuda"), out, prec=mh.MH_PREC_MIXED)
    assert _rel(out.cpu().numpy(), A @ s) < 1e-6
    rhs = rng.standard_normal(bnd.n)
    x = np.linalg.solve(A, rhs)
    for prec in (mh.MH_PREC_FP64, mh.MH_PREC_MIXED):
        sig = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
        info = mh.mh_gmres_solve(ctx, bnd, alpha, torch.tensor(rhs, device="cuda"), sig, tol=1e-12, prec=prec)
        assert info.converged and info.rel_residual <= 1e-12
        assert _rel(sig.cpu().numpy(), x) < 1e-10
    # off-surface (binary64): interior points and points at 3, 0.5 and 0.1 h_s from each curve
    sigma = rng.standard_normal(bnd.n) * 0.1 + np.cos(np.concatenate([c.t for c in curves]))
    r = np.sqrt(rng.uniform(0.0, 0.95, 60))
    th = rng.uniform(0, 2 * np.pi, 60)
    pts = [np.stack([r * np.cos(th), r * np.sin(th)], axis=1)]
    for d in (3.0, 0.5, 0.1):
        for t0 in (0.3, 2.0):
            h0, h1 = 2 * np.pi / 126, 0.3 * 2 * np.pi / 128
            pts.append(np.array([[(1 - d * h0) * np.cos(t0), (1 - d * h0) * np.sin(t0)],
                                 [0.2 + (0.3 + d * h1) * np.cos(t0), (0.3 + d * h1) * np.sin(t0)]]))
    pts = np.concatenate(pts)
    info = G.classify(curves, pts)
    pts = pts[info.region == -1]
    info = G.classify(curves, pts)
    ref = bie.dlp_eval(curves, sigma, alpha, pts, info, A @ sigma)
    got = torch.empty(pts.shape[0], dtype=torch.float64, device="cuda")
    mh.mh_double_layer_apply(ctx, bnd, alpha, torch.tensor(sigma, device="cuda"), got,
                             targets=torch.tensor(pts, device="cuda"))
    assert np.max(np.abs(got.cpu().numpy() - ref)) < 1e-10 * np.max(np.abs(ref))
