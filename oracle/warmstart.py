"""Learned warm start for the boundary solve: the plain FP64 CPU reference.

THIS MODULE IS TEST INFRASTRUCTURE (see the package docstring).

The paper solves one second-kind system A sigma^{N+1} = b^{N+1} per time step by
GMRES to a relative residual of 1e-10 (Section 3.2 and Section 4) and gives no
initial guess.  The learned warm start predicts sigma^{N+1} from the previous
density sigma^N and the next right-hand side b^{N+1}.  Both enter through the
residual of the previous-step start,
    r = b^{N+1} - A sigma^N,
whose exact correction A^{-1} r = sigma^{N+1} - sigma^N the network learns in
the form  delta = r + e,  e = -K A^{-1} r  (A = I + K, K the smoothing double-layer part):

  features  x = F(r) / (|r| g_x),   F = the first n_modes complex Fourier
            coefficients c_k = (1/n) sum_j v_j exp(-2 pi i j k / n) of every curve,
            stored curve-major as [Re c_0, Im c_0, Re c_1, Im c_1, ...];
  network   y = W4 t(W3 t(W2 t(W1 x + b1) + b2) + b3) + b4,  t = tanh (a 4-layer MLP);
  output    delta = r + |r| g_y S(y),  S the Fourier synthesis
            v_j = Re c_0 + 2 sum_{k>=1} Re(c_k exp(2 pi i j k / n));
  judge     w = A delta, c = <r, w>/<w, w> (0 when w = 0): x0 = sigma^N + c delta is the
            minimum-residual point on the line through sigma^N, so its residual
            r0 = r - c w is never larger than that of the previous-step start (c = 0).

Training samples come from solver trajectories: x = F(r)/|r|, y = F(sigma^{N+1} -
sigma^N - r)/|r|; g_x and g_y are the RMS entries of the training X and Y.

Training (the closed-form start followed by gradient steps):
  fit   1. mu = mean row of X, Xc = X - mu.
        2. Range finder for the dominant row space of Xc: Q = orth(Xc^T Omega)
           (Omega: n x width Gaussian, passed in), then ``power_iters`` times
           Q = orth(Xc^T (Xc Q)); orth = the Q factor of a QR factorisation whose R has
           a positive diagonal (unique).
        3. s_j = RMS over samples of (Xc Q)_j, floored at 1e-8 max_j s_j;
           W1 = eps diag(1/s) Q^T, b1 = -W1 mu,
           so every first-layer pre-activation has RMS eps (tanh in its near-linear range).
        4. W2 = W3 = I, b2 = b3 = 0.
        5. H = the third hidden layer on the training X; [W4 | b4]^T solves the ridge
           normal equations (Ha^T Ha + lam I) Z = Ha^T Y, Ha = [H, 1],
           lam = ridge * trace(Ha^T Ha) / (width + 1).
  Adam  loss L = (1/(2 B d)) sum (y_hat - y)^2 over a batch of B rows; Adam (Kingma &
        Ba 2015) with bias correction.

Pins (tests/test_oracle_warmstart.py): a pure cosine mode has the coefficient
e^{i phi}/2 and synthesis reproduces every band-limited vector; gradients against
central finite differences; a one-layer network against the closed-form
least-squares gradient; the first Adam step against its closed form
-lr g/(|g| + eps); the fit reproduces an exact linear low-rank map to O(eps^2);
the judge never increases the residual and is exact for a perfect correction.
"""
import numpy as np


# ----------------------------------------------------------------------------- Fourier features
def fourier_features(v, n_nodes, n_modes):
    """Truncated Fourier coefficients of every curve's values (curve-major, re/im pairs)."""
    v = np.asarray(v, dtype=np.float64)
    out = []
    off = 0
    for n in n_nodes:
        c = np.fft.fft(v[off:off + n]) / n
        seg = np.empty(2 * n_modes)
        seg[0::2] = c[:n_modes].real
        seg[1::2] = c[:n_modes].imag
        out.append(seg)
        off += n
    return np.concatenate(out)


def fourier_synthesis(x, n_nodes, n_modes):
    """Real values at the nodes from truncated coefficients (inverse of fourier_features on
    vectors whose spectrum lies in |k| < n_modes)."""
    x = np.asarray(x, dtype=np.float64)
    out = []
    for c_i, n in enumerate(n_nodes):
        seg = x[c_i * 2 * n_modes:(c_i + 1) * 2 * n_modes]
        c = seg[0::2] + 1j * seg[1::2]
        j = np.arange(n)
        v = np.full(n, c[0].real)
        for k in range(1, n_modes):
            v += 2.0 * (c[k] * np.exp(2j * np.pi * j * k / n)).real
        out.append(v)
    return np.concatenate(out)


# ----------------------------------------------------------------------------- the network
def mlp_forward(params, X):
    """params = [(W, b), ...] with W of shape (out, in); tanh after every layer but the last.
    Returns the output and the list of layer inputs (activations) for the backward pass."""
    acts = [np.asarray(X, dtype=np.float64)]
    h = acts[0]
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        h = np.tanh(z) if li + 1 < len(params) else z
        acts.append(h)
    return h, acts


def mlp_loss_grad(params, X, T):
    """L = (1/(2 B d)) sum (Y - T)^2 and its gradient with respect to every W and b."""
    Y, acts = mlp_forward(params, X)
    T = np.asarray(T, dtype=np.float64)
    B, d = T.shape
    diff = Y - T
    loss = 0.5 * np.sum(diff * diff) / (B * d)
    grads = [None] * len(params)
    dz = diff / (B * d)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        a_in = acts[li]
        grads[li] = (dz.T @ a_in, dz.sum(axis=0))
        if li > 0:
            da = dz @ W
            dz = da * (1.0 - acts[li] ** 2)        # tanh' = 1 - tanh^2
    return loss, grads


def adam_init(params):
    return [(np.zeros_like(W), np.zeros_like(b)) for W, b in params], \
           [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t = 1, 2, ...), returns new params, m, v."""
    new_p, new_m, new_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        out = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = beta1 * mm + (1.0 - beta1) * g
            vv = beta2 * vv + (1.0 - beta2) * g * g
            mhat = mm / (1.0 - beta1 ** t)
            vhat = vv / (1.0 - beta2 ** t)
            out.append((p - lr * mhat / (np.sqrt(vhat) + eps), mm, vv))
        new_p.append((out[0][0], out[1][0]))
        new_m.append((out[0][1], out[1][1]))
        new_v.append((out[0][2], out[1][2]))
    return new_p, new_m, new_v


def _orth(M):
    Q, R = np.linalg.qr(M)
    return Q * np.sign(np.diag(R))


def fit(X, Y, omega, eps, power_iters, ridge):
    """The closed-form start of training (steps 1-5 of the module docstring)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    width = omega.shape[1]
    mu = X.mean(axis=0)
    Xc = X - mu
    Q = _orth(Xc.T @ omega)
    for _ in range(power_iters):
        Q = _orth(Xc.T @ (Xc @ Q))
    Z = Xc @ Q
    s = np.sqrt(np.mean(Z * Z, axis=0))
    s = np.maximum(s, 1e-8 * s.max())        # directions without data get no gain
    W1 = eps * (Q / s).T
    b1 = -W1 @ mu
    I = np.eye(width)
    params = [(W1, b1), (I.copy(), np.zeros(width)), (I.copy(), np.zeros(width))]
    _, acts = mlp_forward(params, X)
    H = acts[-1]
    Ha = np.hstack([H, np.ones((H.shape[0], 1))])
    G = Ha.T @ Ha
    lam = ridge * np.trace(G) / G.shape[0]
    Zs = np.linalg.solve(G + lam * np.eye(G.shape[0]), Ha.T @ Y)
    params.append((Zs[:-1].T.copy(), Zs[-1].copy()))
    return params


# ----------------------------------------------------------------------------- samples and the start
def sample(A, sigma_prev, rhs, sigma_next, n_nodes, n_modes):
    """Training pair (x, y) and |r| from one solved step."""
    r = rhs - A @ sigma_prev
    rn = np.linalg.norm(r)
    if rn == 0.0:
        z = np.zeros(2 * n_modes * len(n_nodes))
        return z, z.copy(), 0.0
    x = fourier_features(r, n_nodes, n_modes) / rn
    y = fourier_features(sigma_next - sigma_prev - r, n_nodes, n_modes) / rn
    return x, y, rn


def warm_start(A, params, gx, gy, sigma_prev, rhs, n_nodes, n_modes):
    """Initial guess x0, its residual r0 and the step length c (module docstring)."""
    r = rhs - A @ sigma_prev
    rn = np.linalg.norm(r)
    if rn == 0.0:
        return sigma_prev.copy(), r, 0.0
    x = fourier_features(r, n_nodes, n_modes) / (rn * gx)
    y, _ = mlp_forward(params, x[None, :])
    delta = r + rn * gy * fourier_synthesis(y[0], n_nodes, n_modes)
    w = A @ delta
    ww = float(w @ w)
    c = float(r @ w) / ww if ww > 0 else 0.0
    return sigma_prev + c * delta, r - c * w, c


def secant_start(A, sigma_prev, sigma_prev2, rhs):
    """Non-learned comparison: minimum-residual step along the previous increment."""
    r = rhs - A @ sigma_prev
    d = sigma_prev - sigma_prev2
    w = A @ d
    ww = float(w @ w)
    c = float(r @ w) / ww if ww > 0 else 0.0
    return sigma_prev + c * d, r - c * w, c


def bf16_round(a):
    """Round binary64 values to bfloat16 (round to nearest even on the binary32 value)."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
