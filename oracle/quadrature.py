"""Quadrature and interpolation building blocks of the oracle.

* Gauss-Legendre nodes/weights on [-1, 1] (numpy.polynomial.legendre.leggauss,
  a library routine) in increasing order.
* Tensor Lagrange basis on a leaf's q x q Gauss-Legendre nodes.  The paper fits
  a 10-term cubic on a 4x4 cell-centred grid (Section 3.1); this library uses
  q x q Gauss-Legendre nodes with the full tensor Lagrange interpolant instead
  (a stated deviation).  Node j of a leaf is (ix, iy) with j = iy*q + ix.
* Trigonometric interpolation of periodic data sampled at t_n = 2 pi n / N
  (N even), with the Nyquist mode split symmetrically, used for Fourier
  interpolation of the density and of the geometry (Section 3.2):
      p(t) = sum_n v_n D_N(t - t_n),
      D_N(tau) = (1/N) [1 + 2 sum_{k=1}^{N/2-1} cos(k tau) + cos(N tau / 2)]
               = sin(N tau / 2) cot(tau / 2) / N.
  ``trig_kernel_sum`` is the cosine-sum definition, ``trig_kernel`` the closed
  form; the tests check one against the other.
"""
import math

import numpy as np


def gauss_legendre(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return x.astype(np.float64), w.astype(np.float64)


def lagrange_matrix(xi: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """L[i, k] = l_i(pts[k]) for the Lagrange polynomials l_i on nodes xi."""
    xi = np.asarray(xi, dtype=np.float64)
    pts = np.asarray(pts, dtype=np.float64)
    q = xi.shape[0]
    out = np.ones((q,) + pts.shape)
    for i in range(q):
        for m in range(q):
            if m != i:
                out[i] = out[i] * (pts - xi[m]) / (xi[i] - xi[m])
    return out


def trig_kernel_sum(tau, n: int):
    tau = np.asarray(tau, dtype=np.float64)
    acc = np.ones_like(tau)
    for k in range(1, n // 2):
        acc = acc + 2.0 * np.cos(k * tau)
    acc = acc + np.cos(0.5 * n * tau)
    return acc / n


def trig_kernel(tau, n: int):
    tau = np.asarray(tau, dtype=np.float64)
    s = np.sin(0.5 * tau)
    small = np.abs(s) < 1e-300
    safe = np.where(small, 1.0, s)
    val = np.sin(0.5 * n * tau) * np.cos(0.5 * tau) / safe / n
    return np.where(small, 1.0, val)


def trig_eval(values: np.ndarray, t, deriv: int = 0) -> np.ndarray:
    """Evaluate the d-th derivative of the trigonometric interpolant of periodic samples
    `values` (shape (N,) or (N, c)) at parameters t, through the FFT coefficients."""
    v = np.asarray(values, dtype=np.float64)
    n = v.shape[0]
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    c = np.fft.fft(v, axis=0) / n
    k = np.fft.fftfreq(n, d=1.0 / n)            # 0..N/2-1, -N/2..-1
    half = n // 2
    # modes |k| < N/2 as complex exponentials; the Nyquist mode as c cos(N t / 2)
    keep = np.abs(k) < half
    kk = k[keep]
    ck = c[keep]
    ph = np.exp(1j * np.outer(t, kk)) * (1j * kk) ** deriv
    out = ph @ ck
    cn = c[half].real
    ang = half * t
    # d^d/dt^d cos(h t) = h^d cos(h t + d pi/2)
    nyq = (half ** deriv) * np.cos(ang + 0.5 * math.pi * deriv)
    out = out.real + (np.outer(nyq, cn) if v.ndim == 2 else nyq * cn)
    return out
