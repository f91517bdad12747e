"""Second-kind boundary integral equation for the homogeneous part U^h
(Section 2, eq. dirichlet:inteqn; Section 3.2, eq. discrete_sys).

Double-layer kernel (Section 3.2):
    K(y, x) = (1/alpha) K1(|y - x| / alpha) (y - x) . n_y / |y - x|,
with d/dnu_y K0(|y - x|/alpha) = -K(y, x).  Multiplying eq. dirichlet:inteqn by
-2 alpha^2 gives the operator solved here (reading of eq. discrete_sys with
the garbled sign and the missing quadrature factors restored from the
continuous equation):
    (A sigma)_j = sigma_j + (1/pi) Q_j[ K(., y_j) sigma ] = -2 alpha^2 g_j,
where Q_j is the Nystrom quadrature with weights h_m |y'_n|: the trapezoid rule
on the other curves, and on the curve of y_j the trapezoid rule outside the
Alpert window |n - j| < a plus 2l off-grid correction nodes t_j +- x_m h whose
density and geometry come from Fourier interpolation (Section 3.2).  With
``alpert=None`` the own-curve sum is the plain trapezoid rule with the
diagonal limit K(x, x) = -(y''.n)/(2|y'|^2) (Section 2, the limit -kappa/2 of
d/dnu K0).

Off-surface evaluation (Section 2, the double-layer representation of U^h):
    U^h(x) = (1/(2 pi alpha^2)) int d/dnu_y K0 sigma ds
           = -(1/(2 pi alpha^2)) sum_curves sum_n K(y_n, x) sigma_n |y'_n| h,
with the near-boundary reading (the paper is silent on targets close to Gamma):
  * d >= 10 h_s          : trapezoid rule on curve k;
  * 0.25 h_s <= d < 10 h_s: trapezoid rule on 16x upsampled curve k (density and
                            geometry by Fourier interpolation);
  * d < 0.25 h_s          : degree-4 polynomial in the distance along the normal
                            through the interior limit v_0 = -(A sigma)(t*)/(2 alpha^2)
                            (Fourier-interpolated) and the upsampled values at
                            0.25, 0.5, 0.75, 1.0 h_s inside Omega;
where d, t* and h_s = |y'(t*)| h come from ``geometry.classify``.
Pins: the closed-form circle spectrum mu_n = z I_n(z) [K_{n-1}(z) + K_{n+1}(z)]
(z = R/alpha) and the exact interior field I_n(r/alpha)/I_n(z) cos(n theta);
exact homogeneous solutions K0(|x - x0|/alpha) with x0 outside Omega.
"""
import math

import numpy as np

from . import alpert as _alpert
from .quadrature import trig_kernel
from .special import k1

UPSAMPLE = 16
NEAR_FAR = 10.0       # d < 10 h_s: upsampled rule (the plain rule is within ~1e-14 beyond)
NEAR_LINE = 0.25      # d < 0.25 h_s: interpolation along the normal


def kernel(yx, ny, alpha, x):
    """K(y, x) for sources y (..., 2) with normals ny at target x (2,)."""
    d = yx - x
    r = np.hypot(d[..., 0], d[..., 1])
    return k1(r / alpha) / alpha * (d[..., 0] * ny[..., 0] + d[..., 1] * ny[..., 1]) / r


def nystrom_matrix(curves, alpha: float, alpert_order=_alpert.DEFAULT_ORDER, rows=None) -> np.ndarray:
    """Dense N_Gamma x N_Gamma matrix of the operator A (eq. discrete_sys), or only the
    listed global row indices (array of shape (len(rows), N_Gamma))."""
    offs = np.cumsum([0] + [c.n for c in curves])
    ntot = int(offs[-1])
    wanted = None if rows is None else {int(r): i for i, r in enumerate(rows)}
    A = np.zeros((ntot if rows is None else len(rows), ntot))
    allnodes = np.concatenate([c.nodes for c in curves])
    allnorm = np.concatenate([c.normal for c in curves])
    allw = np.concatenate([c.speed * c.h for c in curves])
    if alpert_order is not None:
        a, xm, wm = _alpert.rule(alpert_order)
    for k, c in enumerate(curves):
        for jj in range(c.n):
            j = offs[k] + jj
            if wanted is not None and j not in wanted:
                continue
            x = c.nodes[jj]
            d = allnodes - x
            r = np.hypot(d[:, 0], d[:, 1])
            r[j] = 1.0
            row = k1(r / alpha) / alpha * (d[:, 0] * allnorm[:, 0] + d[:, 1] * allnorm[:, 1]) / r * allw
            if alpert_order is None:
                row[j] = c.kdiag[jj] * allw[j]
            else:
                idx = (np.arange(c.n) - jj) % c.n
                circ = np.minimum(idx, c.n - idx)
                row[offs[k]:offs[k + 1]][circ < a] = 0.0
                # 2l off-grid nodes: geometry and density by Fourier interpolation
                tt = np.concatenate([c.t[jj] + xm * c.h, c.t[jj] - xm * c.h])
                yy = c.eval(tt, 0)
                y1 = c.eval(tt, 1)
                sp = np.hypot(y1[:, 0], y1[:, 1])
                nn = np.stack([y1[:, 1], -y1[:, 0]], axis=1) / sp[:, None]
                kv = kernel(yy, nn, alpha, x)
                coef = np.concatenate([wm, wm]) * c.h * sp * kv            # (2l,)
                interp = trig_kernel(tt[:, None] - c.t[None, :], c.n)     # (2l, N)
                row[offs[k]:offs[k + 1]] += coef @ interp
            r_out = j if wanted is None else wanted[j]
            A[r_out] = row / math.pi
            A[r_out, j] += 1.0
    return A


def gmres(A: np.ndarray, b: np.ndarray, x0=None, tol: float = 1e-10, max_iter: int = 200):
    """Unrestarted GMRES with modified Gram-Schmidt and Givens rotations; stops when
    the residual norm is <= tol * ||b|| (Section 4: GMRES tolerance 1e-10).
    Returns (x, iterations, relative residual history)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    bn = np.linalg.norm(b)
    if bn == 0:
        return np.zeros(n), 0, [0.0]
    beta = np.linalg.norm(r)
    hist = [beta / bn]
    if beta <= tol * bn:
        return x, 0, hist
    m = min(max_iter, n)
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[0] = r / beta
    k_done = 0
    for k in range(m):
        w = A @ V[k]
        for i in range(k + 1):
            H[i, k] = w @ V[i]
            w = w - H[i, k] * V[i]
        H[k + 1, k] = np.linalg.norm(w)
        if H[k + 1, k] > 0:
            V[k + 1] = w / H[k + 1, k]
        for i in range(k):
            t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
            H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
            H[i, k] = t
        den = math.hypot(H[k, k], H[k + 1, k])
        cs[k] = H[k, k] / den
        sn[k] = H[k + 1, k] / den
        H[k, k] = den
        H[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        k_done = k + 1
        hist.append(abs(g[k + 1]) / bn)
        if abs(g[k + 1]) <= tol * bn:
            break
    y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
    x = x + V[:k_done].T @ y
    return x, k_done, hist


def _upsampled(c, sigma_c, factor=UPSAMPLE):
    nf = c.n * factor
    tf = 2.0 * math.pi * np.arange(nf) / nf
    yf = c.eval(tf, 0)
    y1 = c.eval(tf, 1)
    sp = np.hypot(y1[:, 0], y1[:, 1])
    nf_ = np.stack([y1[:, 1], -y1[:, 0]], axis=1) / sp[:, None]
    # density on the fine grid by Fourier interpolation (zero-padded spectrum, Nyquist split)
    from .quadrature import trig_eval
    sf = trig_eval(sigma_c, tf, 0)
    return yf, nf_, sf * sp * (2.0 * math.pi / nf)


def dlp_eval(curves, sigma, alpha: float, targets: np.ndarray, info, a_sigma=None):
    """U^h at targets (all assumed in Omega), with the near-boundary reading above.
    `info` is geometry.classify(curves, targets); `a_sigma` = A sigma at the nodes
    (needed only when some target is closer than 0.25 h_s to Gamma)."""
    offs = np.cumsum([0] + [c.n for c in curves])
    sig = [sigma[offs[k]:offs[k + 1]] for k in range(len(curves))]
    pref = -1.0 / (2.0 * math.pi * alpha * alpha)
    fine = {}

    def fine_of(k):
        if k not in fine:
            fine[k] = _upsampled(curves[k], sig[k])
        return fine[k]

    def curve_sum(k, x, use_fine):
        c = curves[k]
        if use_fine:
            yf, nf_, wf = fine_of(k)
            return float(np.sum(kernel(yf, nf_, alpha, x) * wf))
        return float(np.sum(kernel(c.nodes, c.normal, alpha, x) * sig[k] * c.speed * c.h))

    def value_at(x, prj):
        tot = 0.0
        for k in range(len(curves)):
            p = prj[k]
            tot += curve_sum(k, x, p is not None and p["d"] < NEAR_FAR * p["hs"])
        return pref * tot

    out = np.zeros(targets.shape[0])
    for i, x in enumerate(targets):
        prj = info.proj[i]
        line = [k for k in range(len(curves)) if prj[k] is not None and prj[k]["d"] < NEAR_LINE * prj[k]["hs"]]
        if not line:
            out[i] = value_at(x, prj)
            continue
        k = min(line, key=lambda kk: prj[kk]["d"])
        p = prj[k]
        c = curves[k]
        y1 = c.eval(p["t"], 1)[0]
        nrm = np.array([y1[1], -y1[0]]) / math.hypot(y1[0], y1[1])
        v0 = -float(trig_kernel(p["t"] - c.t, c.n) @ a_sigma[offs[k]:offs[k + 1]]) / (2.0 * alpha * alpha)
        dist = [0.0]
        vals = [v0]
        for m in range(1, 5):
            dm = m * NEAR_LINE * p["hs"]
            xm = p["y"] - dm * nrm
            # the auxiliary points sit at >= 0.25 h_s from Gamma_k; other curves by their own rule
            pr = [None] * len(curves)
            for kk in range(len(curves)):
                if kk == k:
                    pr[kk] = {"d": dm, "hs": p["hs"]}
                else:
                    q2 = prj[kk]
                    pr[kk] = q2
            dist.append(dm)
            vals.append(value_at(xm, pr))
        # Lagrange interpolation in the distance variable
        dd = p["d"]
        acc = 0.0
        for a_ in range(5):
            wgt = 1.0
            for b_ in range(5):
                if b_ != a_:
                    wgt *= (dd - dist[b_]) / (dist[a_] - dist[b_])
            acc += wgt * vals[a_]
        out[i] = acc
    return out
