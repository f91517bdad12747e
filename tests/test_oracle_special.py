"""Pins of the oracle's Bessel functions (library routines) against mpmath and
the Wronskian I_n K_n' - I_n' K_n = -1/z (DLMF 10.28.2)."""
import numpy as np
import pytest

from oracle import special


def test_k0_k1_against_mpmath():
    mp = pytest.importorskip("mpmath")
    for z in [1e-8, 1e-3, 0.1, 0.5, 1.0, 1.999, 2.0, 2.5, 5.0, 10.0, 30.0, 80.0, 300.0]:
        for f, nu in ((special.k0, 0), (special.k1, 1)):
            ref = float(mp.besselk(nu, z))
            assert abs(f(z) - ref) <= 2e-15 * abs(ref), (nu, z)


def test_wronskian():
    for n in [0, 1, 2, 5, 10]:
        z = np.array([0.05, 0.3, 1.0, 4.0, 12.0])
        i = special.i_n(n, z)
        k = special.kn(n, z)
        ip = 0.5 * (special.i_n(n - 1, z) + special.i_n(n + 1, z))
        kp = -0.5 * (special.kn(n - 1, z) + special.kn(n + 1, z))
        assert np.allclose(i * kp - ip * k, -1.0 / z, rtol=1e-12, atol=0)


def test_green_integrates_to_one():
    # int_{R^2} G dA = int_0^inf r K0(r/a)/a^2 dr = 1, and the disk integral is 1 - z K1(z)
    from scipy import integrate
    a = 0.07
    val = integrate.quad(lambda r: 2 * np.pi * r * special.green(r, a), 0, 60 * a, limit=200)[0]
    assert abs(val - 1.0) < 1e-10
    R = 0.1
    disk = integrate.quad(lambda r: 2 * np.pi * r * special.green(r, a), 0, R, limit=200)[0]
    assert abs(disk - (1 - R / a * special.k1(R / a))) < 1e-12
