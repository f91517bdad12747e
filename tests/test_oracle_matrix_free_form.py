"""The matrix-free form of the discrete system (Section 3.2: the system evaluated without a
stored matrix), pinned on the CPU against the oracle's dense Nystrom rows.

The GPU's matrix-free product splits row j of A sigma into
  sigma_j + (1/pi) [T_j - W_j] + sum_p coef_j[p] sigma~(t_j + s_p x_m h),
T_j the trapezoid sum over every node but j (all curves), W_j the own-curve terms with
0 < |i - j| < a (the Alpert window), sigma~ the curve's trigonometric interpolant taken from
its spectrum at the shifted grid, and takes the length-N transforms by Bluestein's chirp
convolution when N is not a power of two.  Here each of those identities is written out in
numpy from its definition and compared with the oracle:
  * the spectrum form of the interpolant at a shifted grid equals the periodic-kernel sum the
    oracle's assembly uses (trig_kernel), to rounding;
  * Bluestein's chirp convolution at length M >= 2N - 1 equals the DFT (numpy's FFT) for
    N = 96, 160, 250 and the odd 97 (where a filter laid out as b_{N-m} instead of b_m at
    M - m would show: the two agree for even N);
  * the decomposition reproduces every row of oracle.bie.nystrom_matrix (two curves of 96 and
    64 nodes, alpha = 0.1, Alpert order 8) to 1e-13.
A dropped window term, a window of the wrong width, a Nyquist weight of 2, a wrong shift sign or
a missing 1/pi each moves the rows by far more than that bar."""
import math

import numpy as np
import pytest

from oracle import alpert, bie, geometry, quadrature

import mh_workloads as W


def _spectrum_shift(sig, delta):
    """Re sum_{m <= N/2} w_m c_m e^{i m delta} e^{2 pi i m j / N}, c = FFT(sig) / N."""
    n = sig.shape[0]
    c = np.fft.fft(sig) / n
    half = np.zeros(n, dtype=complex)
    m = np.arange(n // 2 + 1)
    w = np.where((m == 0) | (2 * m == n), 1.0, 2.0)
    half[: n // 2 + 1] = w * c[: n // 2 + 1] * np.exp(1j * m * delta)
    return np.real(np.fft.ifft(half) * n)


def _bluestein(x):
    """X_k = conj(b_k) sum_n (x_n conj(b_n)) b_{k-n}, b_n = e^{i pi n^2 / N}, as a cyclic
    convolution of length M = 2^L >= 2N - 1."""
    n = x.shape[0]
    M = 1
    while M < 2 * n - 1:
        M *= 2
    k = np.arange(n)
    b = np.exp(1j * np.pi * ((k * k) % (2 * n)) / n)
    a = np.zeros(M, dtype=complex)
    a[:n] = x * np.conj(b)
    B = np.zeros(M, dtype=complex)
    B[:n] = b
    B[M - n + 1:] = b[1:][::-1]
    conv = np.fft.ifft(np.fft.fft(a) * np.fft.fft(B))
    return np.conj(b) * conv[:n]


@pytest.mark.parametrize("n", [64, 96, 160])
def test_spectrum_shift_equals_periodic_kernel_sum(n):
    rng = np.random.default_rng(n)
    sig = rng.standard_normal(n)
    h = 2 * math.pi / n
    t = h * np.arange(n)
    _, xm, _ = alpert.rule(8)
    for s in (1.0, -1.0):
        for x in xm:
            d = s * x * h
            ref = quadrature.trig_kernel(t[:, None] + d - t[None, :], n) @ sig
            got = _spectrum_shift(sig, d)
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(sig)), (n, s, x)


@pytest.mark.parametrize("n", [96, 97, 160, 250])
def test_bluestein_equals_dft(n):
    rng = np.random.default_rng(3 * n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    got = _bluestein(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_matrix_free_decomposition_reproduces_the_nystrom_rows():
    nodes = [W.circle_nodes((0.0, 0.0), 1.0, 96, clockwise=False),
             W.ellipse_nodes((0.3, 0.1), 0.25, 0.15, 0.4, 64, clockwise=True)]
    alpha = 0.1
    curves = geometry.make_curves(nodes)
    A = bie.nystrom_matrix(curves, alpha)
    rng = np.random.default_rng(17)
    sig = rng.standard_normal(A.shape[0])
    ref = A @ sig
    a, xm, wm = alpert.rule(8)
    offs = np.cumsum([0] + [c.n for c in curves])
    allnodes = np.concatenate([c.nodes for c in curves])
    allnorm = np.concatenate([c.normal for c in curves])
    allw = np.concatenate([c.speed * c.h for c in curves])
    got = np.empty_like(ref)
    for k, c in enumerate(curves):
        sk = sig[offs[k]:offs[k + 1]]
        shifted = {(s, m): _spectrum_shift(sk, s * xm[m] * c.h) for s in (1.0, -1.0) for m in range(len(xm))}
        for jj in range(c.n):
            j = offs[k] + jj
            x = c.nodes[jj]
            with np.errstate(invalid="ignore", divide="ignore"):
                kv = bie.kernel(allnodes, allnorm, alpha, x)
            kv[j] = 0.0
            T = np.sum(kv * allw * sig)                         # every node but j
            d = np.array([dd for dd in range(1, a)] + [-dd for dd in range(1, a)])
            ii = offs[k] + (jj + d) % c.n
            Wj = np.sum(kv[ii] * allw[ii] * sig[ii])            # own-curve window
            C = 0.0
            for s in (1.0, -1.0):
                tt = c.t[jj] + s * xm * c.h
                yy = c.eval(tt, 0)
                y1 = c.eval(tt, 1)
                sp = np.hypot(y1[:, 0], y1[:, 1])
                nn = np.stack([y1[:, 1], -y1[:, 0]], axis=1) / sp[:, None]
                coef = wm * c.h * sp * bie.kernel(yy, nn, alpha, x) / math.pi
                C += sum(coef[m] * shifted[(s, m)][jj] for m in range(len(xm)))
            got[j] = sig[j] + (T - Wj) / math.pi + C
    e = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert e <= 1e-13, e
