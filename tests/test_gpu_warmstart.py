"""Learned warm start on the GPU.

Parity (disk with a hole, 2 x 128 nodes, 16 modes per curve, width 16) against the oracle
(oracle/warmstart.py): training pairs, the binary32 loss and gradient, Adam steps, the
closed-form start, the three inference arithmetics, and the judged starts (LEARNED, SECANT).

Gain (starfish domain, 6 x 1024 nodes, 256 modes, width 256): the network trained on 2000
solver steps (100 Gaussian-sum forcings x 20 steps) cuts the GMRES iterations over 500
held-out steps (5 held-out forcings x 100 steps) against the previous-step and zero starts,
and every start gives the same solution.  On the held-out pairs the network's loss is set
beside a plain linear predictor (ridge least squares on the top principal components): the
target is linear in the network's input, so the linear predictor is the one to match."""
import math

import numpy as np
import pytest

import mh_workloads as W
from oracle import bie, geometry as G
from oracle import warmstart as ws

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K_SMALL, W_SMALL = 16, 16
N_HELD = 100     # held-out steps per held-out forcing (after the first step from u = 0)


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(mh):
    return mh.Context(0)


@pytest.fixture(scope="module")
def c1(mh, ctx):
    """Three solved IMEX Euler steps on the disk with a hole (binary64): sigma^1..3 and rhs^3."""
    wl = W.disk_with_hole()
    dev = torch.device("cuda:0")
    tree = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    prob = mh.Problem(ctx, tree, bnd, wl.dt, 20, ext_mode=mh.MH_EXT_CONST, ext_const=[0.0, 0.0])
    nodes = tree.nodes().cpu().numpy()
    bn = np.concatenate(wl.curves)
    mf = W.Manufactured
    F = torch.tensor(mf.F(0.0, nodes), device=dev)
    u = torch.zeros(tree.n_nodes, dtype=torch.float64, device=dev)
    un = torch.empty_like(u)
    sig = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
    dens = []
    for k in range(3):
        mh.heat_step(ctx, prob, u, F, torch.tensor(mf.u((k + 1) * wl.dt, bn), device=dev), un, sig)
        dens.append(sig.clone())
        u, un = un, u
    rhs = torch.empty_like(sig)
    prob.rhs(rhs)
    A = bie.nystrom_matrix(G.make_curves(wl.curves), wl.alpha)
    return dict(wl=wl, bnd=bnd, prob=prob, s1=dens[0], s2=dens[1], s3=dens[2], rhs=rhs, A=A,
                nn=[c.shape[0] for c in wl.curves])


def _rand_params(net, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(net.n_params) * scale).astype(np.float32)


def _split(net, flat):
    """Flat parameter vector -> [(W, b)] in binary64 (layout of include/mh.h)."""
    d, w = net.d, net.width
    shapes = [(w, d), (w, w), (w, w), (d, w)]
    out, o = [], 0
    for (r, c) in shapes:
        Wm = flat[o:o + r * c].reshape(r, c).astype(np.float64)
        o += r * c
        b = flat[o:o + r].astype(np.float64)
        o += r
        out.append((Wm, b))
    return out


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def test_sample_matches_oracle(mh, ctx, c1):
    net = mh.Net(ctx, c1["bnd"], K_SMALL, W_SMALL)
    x = torch.empty(net.d, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    rn = net.sample(c1["prob"], c1["s2"], c1["s3"], x, y)
    xo, yo, rno = ws.sample(c1["A"], c1["s2"].cpu().numpy(), c1["rhs"].cpu().numpy(), c1["s3"].cpu().numpy(),
                            c1["nn"], K_SMALL)
    assert abs(rn - rno) <= 1e-9 * rno
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-6 * np.max(np.abs(xo))
    assert np.max(np.abs(y.cpu().numpy() - yo)) <= 1e-6 * np.max(np.abs(yo))


def test_loss_and_gradient_match_oracle(mh, ctx, c1):
    net = mh.Net(ctx, c1["bnd"], K_SMALL, W_SMALL)
    p = _rand_params(net, 1)
    net.set_params(p)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((37, net.d)).astype(np.float32)      # 37 rows: a ragged tile
    T = rng.standard_normal((37, net.d)).astype(np.float32)
    g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), g)
    lo, go = ws.mlp_loss_grad(_split(net, p), X.astype(np.float64), T.astype(np.float64))
    go = _flat(go)
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.max(np.abs(g.cpu().numpy() - go)) <= 1e-4 * np.max(np.abs(go))


@pytest.mark.parametrize("arith", [0, 1, 2])
def test_inference_arithmetics(mh, ctx, c1, arith):
    net = mh.Net(ctx, c1["bnd"], K_SMALL, W_SMALL)
    p = _rand_params(net, 3)
    net.set_params(p)
    X = np.random.default_rng(4).standard_normal((5, net.d)).astype(np.float32)
    Y = torch.empty(5, net.d, dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(X, device="cuda"), Y, arith=arith, training_kernels=False)
    params = _split(net, p)
    if arith == mh.MH_NET_BF16:
        params = [(ws.bf16_round(Wm), b) for Wm, b in params]
    elif arith == mh.MH_NET_BF16X2:
        def pair(Wm):
            hi = ws.bf16_round(Wm)
            return hi + ws.bf16_round(Wm.astype(np.float32) - hi.astype(np.float32))
        params = [(pair(Wm), b) for Wm, b in params]
    yo, _ = ws.mlp_forward(params, X.astype(np.float64))
    assert np.max(np.abs(Y.cpu().numpy() - yo)) <= 2e-5 * np.max(np.abs(yo))
    # the training kernels agree with the binary32 inference kernels
    if arith == mh.MH_NET_FP32:
        Yt = torch.empty_like(Y)
        net.forward(torch.tensor(X, device="cuda"), Yt, training_kernels=True)
        assert torch.max(torch.abs(Yt - Y)).item() <= 2e-5 * np.max(np.abs(yo))


def test_adam_steps_match_oracle(mh, ctx, c1):
    net = mh.Net(ctx, c1["bnd"], K_SMALL, W_SMALL)
    X, Y = W.warm_start_toy_data(48, net.d, 20)
    p = _rand_params(net, 5, scale=0.1)
    net.set_params(p, 1.0, 1.0)
    _, idx = W.warm_start_draws(48, net.width, 6, 16)
    lr = 1e-3
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    first, best, step = net.train(Xd, Yd, torch.tensor(idx, device="cuda"), lr, Xd, Yd, eval_every=6)
    params = _split(net, p)
    m, v = ws.adam_init(params)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    for t in range(1, 7):
        _, g = ws.mlp_loss_grad(params, X64[idx[t - 1]], Y64[idx[t - 1]])
        params, m, v = ws.adam_step(params, g, m, v, t, lr)
    l_end, _ = ws.mlp_loss_grad(params, X64, Y64)
    l_start, _ = ws.mlp_loss_grad(_split(net, p), X64, Y64)
    assert step == 6 and best < first
    assert abs(first - l_start) <= 1e-5 * l_start and abs(best - l_end) <= 1e-4 * l_end
    pg, _, _ = net.get_params()
    assert np.max(np.abs(pg.astype(np.float64) - _flat(params))) <= 0.05 * lr


def test_closed_form_start_matches_oracle(mh, ctx, c1):
    net = mh.Net(ctx, c1["bnd"], K_SMALL, W_SMALL)
    n = 200
    X, Y = W.warm_start_toy_data(n, net.d, 40, seed=12)
    omega, _ = W.warm_start_draws(n, net.width, 0, 1, seed=13)
    eps = 1e-3
    net.fit(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), torch.tensor(omega, device="cuda"),
            eps=eps, power_iters=2, ridge=1e-12)
    pg, gx, gy = net.get_params()
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    gxo, gyo = math.sqrt(np.mean(X64 ** 2)), math.sqrt(np.mean(Y64 ** 2))
    assert abs(gx - gxo) <= 1e-12 * gxo and abs(gy - gyo) <= 1e-12 * gyo
    po = ws.fit(X64 / gxo, Y64 / gyo, omega.astype(np.float64), eps=eps, power_iters=2, ridge=1e-12)
    pgs = _split(net, pg)
    for (Wg, bg), (Wo, bo) in zip(pgs, po):
        assert np.max(np.abs(Wg - Wo)) <= 1e-5 * np.max(np.abs(Wo))
        assert np.max(np.abs(bg - bo)) <= 1e-5 * max(np.max(np.abs(bo)), 1e-30) + 1e-30
    Xn, Yn = W.warm_start_toy_data(20, net.d, 40, seed=12)
    Yh = torch.empty(20, net.d, dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(Xn / np.float32(gx), device="cuda"), Yh)
    yo, _ = ws.mlp_forward(po, Xn.astype(np.float64) / gxo)
    assert np.max(np.abs(Yh.cpu().numpy() - yo)) <= 1e-4 * np.max(np.abs(yo))


def test_judged_starts_match_oracle(mh, ctx, c1):
    net = mh.Net(ctx, c1["bnd"], K_SMALL, W_SMALL)
    p = _rand_params(net, 6, scale=0.1)
    gx, gy = 0.05, 0.01
    net.set_params(p, gx, gy)
    alpha = c1["wl"].alpha
    s1, s2, rhs = c1["s1"], c1["s2"], c1["rhs"]      # previous densities and the next right-hand side
    x0 = torch.empty_like(s2)
    r0 = torch.empty_like(s2)
    c = mh.mh_warm_start(ctx, c1["bnd"], alpha, mh.MH_WARM_LEARNED, s2, rhs, x0, r0, net=net, arith=mh.MH_NET_FP32)
    A = c1["A"]
    s2n, rhsn = s2.cpu().numpy(), rhs.cpu().numpy()
    xo, ro, co = ws.warm_start(A, _split(net, p), gx, gy, s2n, rhsn, c1["nn"], K_SMALL)
    assert abs(c - co) <= 1e-4 * abs(co)
    step = np.linalg.norm(xo - s2n)
    assert np.max(np.abs(x0.cpu().numpy() - xo)) <= 1e-4 * step
    assert np.linalg.norm(r0.cpu().numpy() - ro) <= 1e-4 * np.linalg.norm(rhsn - A @ s2n)
    assert np.linalg.norm(r0.cpu().numpy()) <= np.linalg.norm(rhsn - A @ s2n)
    # secant: binary64 throughout
    c = mh.mh_warm_start(ctx, c1["bnd"], alpha, mh.MH_WARM_SECANT, s2, rhs, x0, r0, sigma_prev2=s1)
    xo, ro, co = ws.secant_start(A, s2n, s1.cpu().numpy(), rhsn)
    assert abs(c - co) <= 1e-8 * abs(co)
    assert np.max(np.abs(x0.cpu().numpy() - xo)) <= 1e-10 * np.max(np.abs(xo))


def test_learned_start_cuts_gmres_iterations(mh, ctx):
    from paper_1007_5335_gb300 import warmstart as wsg
    wl = W.starfish_domain()
    dev = torch.device("cuda:0")
    tree = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    prob = mh.Problem(ctx, tree, bnd, wl.dt, wl.p, ext_mode=mh.MH_EXT_CONST, ext_const=wl.ext_const)
    nodes = tree.nodes().cpu().numpy()
    f0 = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
    forc = lambda seeds: [torch.tensor(W.gaussian_forcing(s)(nodes), device=dev) for s in seeds]
    net = mh.Net(ctx, bnd, 256, 256)
    X, Y, _ = wsg.collect_samples(ctx, prob, net, forc(W.WARM_TRAIN_SEEDS), 20, f0)
    Xv, Yv, _ = wsg.collect_samples(ctx, prob, net, forc(W.WARM_VALID_SEEDS), 20, f0)
    assert X.shape[0] == 2000
    omega, idx = W.warm_start_draws(X.shape[0], net.width, 200, 64)
    first, best, best_step = wsg.train(net, X, Y, Xv, Yv, torch.tensor(omega, device=dev),
                                       torch.tensor(idx, device=dev))
    tests = forc(W.WARM_TEST_SEEDS)          # 5 held-out forcings x 100 steps = 500 held-out steps
    # the network against a plain linear predictor on the held-out pairs: the target
    # sigma^{N+1} - sigma^N - r = (A^{-1} - I) r is linear in the input r, so the best
    # predictor is linear; ridge least squares on the top 256 principal components of the
    # training inputs (the network's width), in network units
    Xt, Yt, _ = wsg.collect_samples(ctx, prob, net, tests, N_HELD + 1, f0, take=range(1, N_HELD + 1))
    assert Xt.shape[0] == 5 * N_HELD
    _, gx, gy = net.get_params()
    Yh = torch.empty_like(Xt)
    net.forward(Xt / gx, Yh)
    loss_net = 0.5 * float(torch.mean((Yh.double() - Yt.double() / gy) ** 2))
    Xn, Yn = X.double().cpu().numpy() / gx, Y.double().cpu().numpy() / gy
    mu = Xn.mean(axis=0)
    Q = np.linalg.svd(Xn - mu, full_matrices=False)[2][:net.width].T
    Ha = np.hstack([(Xn - mu) @ Q, np.ones((Xn.shape[0], 1))])
    G = Ha.T @ Ha
    Wl = np.linalg.solve(G + 1e-12 * np.trace(G) / G.shape[0] * np.eye(G.shape[0]), Ha.T @ Yn)
    Ht = np.hstack([(Xt.double().cpu().numpy() / gx - mu) @ Q, np.ones((Xt.shape[0], 1))])
    loss_lin = 0.5 * float(np.mean((Ht @ Wl - Yt.double().cpu().numpy() / gy) ** 2))
    loss_zero = 0.5 * float(np.mean((Yt.double().cpu().numpy() / gy) ** 2))
    print(f"held-out loss: network {loss_net:.3e} (closed form {first:.3e} -> Adam best {best:.3e} at step "
          f"{best_step}), linear PCA-ridge {loss_lin:.3e}, zero prediction {loss_zero:.3e}")
    assert loss_net <= 1e-2 * loss_zero and loss_lin <= 1e-2 * loss_zero
    assert loss_net <= 2.0 * loss_lin          # the network does what the best linear map does
    results = {}
    finals = {}
    for name, mode, arith in (("previous", mh.MH_WARM_PREVIOUS, 0), ("zero", mh.MH_WARM_ZERO, 0),
                              ("secant", mh.MH_WARM_SECANT, 0), ("learned_bf16x2", mh.MH_WARM_LEARNED, 2),
                              ("learned_bf16", mh.MH_WARM_LEARNED, 1)):
        its, init = [], []
        fin = []
        for F in tests:
            prob.set_warm_start(mode, net, arith)
            u = torch.zeros(tree.n_nodes, dtype=torch.float64, device=dev)
            un = torch.empty_like(u)
            sig = torch.zeros(bnd.n, dtype=torch.float64, device=dev)
            for s in range(N_HELD + 1):
                info = mh.heat_step(ctx, prob, u, F, f0, un, sig, gmres_tol=1e-10, prec=mh.MH_PREC_MIXED)
                assert info.gmres_rel_residual <= 1e-10
                if s > 0:
                    its.append(info.gmres_iterations)
                    init.append(info.initial_rel_residual)
                u, un = un, u
            fin.append(u.clone())
        results[name] = (float(np.mean(its)), float(np.exp(np.mean(np.log(init)))))
        finals[name] = fin
    prob.set_warm_start(mh.MH_WARM_PREVIOUS)
    assert all(len(v) == 5 for v in finals.values())
    print("mean GMRES iterations, geometric-mean initial residual over 500 held-out steps:", results)
    for name in results:
        for a, b in zip(finals[name], finals["previous"]):
            assert (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item() <= 1e-6
    assert results["zero"][0] > results["previous"][0]
    assert results["learned_bf16x2"][0] <= results["previous"][0] - 2.0
    assert results["learned_bf16x2"][0] < results["secant"][0]
    assert results["learned_bf16x2"][1] <= 1e-3 * results["previous"][1]
