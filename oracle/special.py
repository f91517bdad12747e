"""Modified Bessel functions for the oracle.

G(x) = K0(|x|/alpha) / (2 pi alpha^2) is the free-space Green's function of
1 - alpha^2 Lap (Section 2, the display after eq. vol_potential); the
double-layer kernel uses K1 (Section 3.2, the kernel K(y, x) after
eq. discrete_sys).  The oracle takes these from scipy.special (a library
routine, Cephes), which the tests pin against mpmath and against the
Wronskian I_n K_n' - I_n' K_n = -1/z.
"""
import math

import numpy as np
from scipy import special as _sp


def k0(z):
    return _sp.k0(z)


def k1(z):
    return _sp.k1(z)


def kn(n, z):
    return _sp.kv(n, z)


def i_n(n, z):
    return _sp.iv(n, z)


def green(r, alpha):
    """G(r) = K0(r/alpha) / (2 pi alpha^2) (Section 2)."""
    return _sp.k0(np.asarray(r) / alpha) / (2.0 * math.pi * alpha * alpha)
