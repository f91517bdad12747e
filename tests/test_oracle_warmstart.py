"""Pins of the learned-warm-start oracle (oracle/warmstart.py) against closed forms,
finite differences and library routines."""
import numpy as np
import pytest

from oracle import warmstart as ws


def test_pure_mode_coefficients():
    n, K = 64, 10
    j = np.arange(n)
    for m, phi in ((0, 0.0), (3, 0.7), (9, -1.1)):
        v = np.cos(2 * np.pi * m * j / n + phi)
        x = ws.fourier_features(v, [n], K)
        c = x[0::2] + 1j * x[1::2]
        want = np.zeros(K, dtype=complex)
        want[m] = 1.0 if m == 0 else 0.5 * np.exp(1j * phi)
        if m == 0:
            want[0] = np.cos(phi)
        assert np.max(np.abs(c - want)) < 1e-14


def test_synthesis_inverts_band_limited():
    rng = np.random.default_rng(0)
    nodes, K = [32, 48], 12
    v = []
    for n in nodes:
        j = np.arange(n)
        vi = np.full(n, rng.normal())
        for k in range(1, K):
            a, b = rng.normal(size=2)
            vi += a * np.cos(2 * np.pi * k * j / n) + b * np.sin(2 * np.pi * k * j / n)
        v.append(vi)
    v = np.concatenate(v)
    x = ws.fourier_features(v, nodes, K)
    assert np.max(np.abs(ws.fourier_synthesis(x, nodes, K) - v)) < 1e-12
    # beyond the band the round trip is the orthogonal projection: idempotent
    w = rng.normal(size=sum(nodes))
    p1 = ws.fourier_synthesis(ws.fourier_features(w, nodes, K), nodes, K)
    p2 = ws.fourier_synthesis(ws.fourier_features(p1, nodes, K), nodes, K)
    assert np.max(np.abs(p1 - p2)) < 1e-12
    assert abs(np.dot(w - p1, p1)) < 1e-10 * np.dot(w, w)


def _rand_params(rng, sizes, scale=0.5):
    return [(rng.normal(scale=scale, size=(o, i)), rng.normal(scale=0.1, size=o)) for i, o in zip(sizes[:-1], sizes[1:])]


def test_gradient_against_finite_differences():
    rng = np.random.default_rng(1)
    params = _rand_params(rng, [5, 4, 4, 4, 3])
    X = rng.normal(size=(7, 5))
    T = rng.normal(size=(7, 3))
    _, grads = ws.mlp_loss_grad(params, X, T)
    h = 1e-6
    for li in range(len(params)):
        for which in (0, 1):
            P = params[li][which]
            G = grads[li][which]
            for idx in np.ndindex(P.shape):
                old = P[idx]
                P[idx] = old + h
                lp, _ = ws.mlp_loss_grad(params, X, T)
                P[idx] = old - h
                lm, _ = ws.mlp_loss_grad(params, X, T)
                P[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - G[idx]) <= 1e-7 * max(1e-3, abs(fd)), (li, which, idx)


def test_one_layer_is_least_squares():
    rng = np.random.default_rng(2)
    W, b = rng.normal(size=(3, 6)), rng.normal(size=3)
    X, T = rng.normal(size=(10, 6)), rng.normal(size=(10, 3))
    loss, g = ws.mlp_loss_grad([(W, b)], X, T)
    R = X @ W.T + b - T
    assert abs(loss - 0.5 * np.sum(R * R) / 30) < 1e-14
    assert np.max(np.abs(g[0][0] - R.T @ X / 30)) < 1e-14
    assert np.max(np.abs(g[0][1] - R.sum(0) / 30)) < 1e-14


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(3)
    params = _rand_params(rng, [4, 3, 2])
    X, T = rng.normal(size=(5, 4)), rng.normal(size=(5, 2))
    _, g = ws.mlp_loss_grad(params, X, T)
    m, v = ws.adam_init(params)
    lr, eps = 1e-2, 1e-8
    new, _, _ = ws.adam_step(params, g, m, v, 1, lr, eps=eps)
    for (W0, b0), (W1, b1), (gW, gb) in zip(params, new, g):
        assert np.max(np.abs((W1 - W0) + lr * gW / (np.abs(gW) + eps))) < 1e-15
        assert np.max(np.abs((b1 - b0) + lr * gb / (np.abs(gb) + eps))) < 1e-15


def test_adam_descends():
    rng = np.random.default_rng(4)
    params = _rand_params(rng, [6, 8, 8, 8, 2])
    X = rng.normal(size=(40, 6))
    T = np.tanh(X[:, :2])
    m, v = ws.adam_init(params)
    l0, _ = ws.mlp_loss_grad(params, X, T)
    for t in range(1, 301):
        _, g = ws.mlp_loss_grad(params, X, T)
        params, m, v = ws.adam_step(params, g, m, v, t, 1e-2)
    l1, _ = ws.mlp_loss_grad(params, X, T)
    assert l1 < 0.05 * l0


def _linear_data(rng, n, d, k, d_out):
    basis = np.linalg.qr(rng.normal(size=(d, k)))[0]
    mu = rng.normal(size=d)
    coef = rng.normal(size=(n, k)) * np.linspace(1.0, 0.1, k)
    X = mu + coef @ basis.T
    M = rng.normal(size=(d_out, d))
    c = rng.normal(size=d_out)
    return X, X @ M.T + c, (basis, mu, M, c)


def test_fit_reproduces_low_rank_linear_map():
    rng = np.random.default_rng(5)
    n, d, k, width, d_out = 300, 24, 6, 8, 10
    X, Y, (basis, mu, M, c) = _linear_data(rng, n, d, k, d_out)
    omega = rng.normal(size=(n, width))
    Xn = mu + (rng.normal(size=(50, k)) * np.linspace(1.0, 0.1, k)) @ basis.T
    Yn = Xn @ M.T + c
    errs = []
    for eps in (1e-2, 1e-3):
        params = ws.fit(X, Y, omega, eps=eps, power_iters=2, ridge=1e-14)
        assert params[0][0].shape == (width, d) and params[3][0].shape == (d_out, width)
        Yh, _ = ws.mlp_forward(params, Xn)
        errs.append(np.linalg.norm(Yh - Yn) / np.linalg.norm(Yn))
    # the only error left is the curvature of tanh, O(eps^2)
    assert errs[1] < 1e-5
    assert 20 < errs[0] / errs[1] < 500


def test_judge_never_increases_residual():
    rng = np.random.default_rng(6)
    nodes, K = [16, 12], 5
    n = sum(nodes)
    A = np.eye(n) + 0.3 * rng.normal(size=(n, n)) / np.sqrt(n)
    params = _rand_params(rng, [4 * K, 6, 6, 6, 4 * K], scale=0.3)
    for trial in range(5):
        sp, rhs = rng.normal(size=n), rng.normal(size=n)
        x0, r0, cst = ws.warm_start(A, params, 1.0, 0.1, sp, rhs, nodes, K)
        r_prev = rhs - A @ sp
        assert np.linalg.norm(r0) <= np.linalg.norm(r_prev) * (1 + 1e-14)
        assert np.max(np.abs(rhs - A @ x0 - r0)) < 1e-12
        # c is the minimiser: the residual is orthogonal to the search direction's image
        delta = (x0 - sp) / cst
        assert abs(np.dot(r0, A @ delta)) < 1e-10 * np.linalg.norm(r_prev) * np.linalg.norm(A @ delta)


def test_exact_correction_gives_zero_residual():
    rng = np.random.default_rng(7)
    n = 20
    A = np.eye(n) + 0.2 * rng.normal(size=(n, n)) / np.sqrt(n)
    s1 = rng.normal(size=n)
    s2 = rng.normal(size=n)
    rhs = A @ (2 * s2 - s1)          # the next density continues the previous increment exactly
    x0, r0, cst = ws.secant_start(A, s2, s1, rhs)
    assert abs(cst - 1.0) < 1e-12 and np.linalg.norm(r0) < 1e-12


def test_bf16_rounding():
    assert ws.bf16_round(1.0) == 1.0
    assert ws.bf16_round(1.0 + 2.0 ** -8) == 1.0                       # tie to even
    assert ws.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie to even (upwards)
    assert ws.bf16_round(-(1.0 + 2.0 ** -7)) == -(1.0 + 2.0 ** -7)
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(8).normal(size=1000) * 10.0 ** np.random.default_rng(9).uniform(-5, 5, 1000)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ws.bf16_round(v), ref)
