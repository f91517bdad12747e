"""Pins of the oracle's volume potential (Section 3.1): exact box integrals
against brute-force 2-D quadrature (scipy dblquad), the polynomial identity
(1 - a^2 Lap)^{-1} B = B + a^2 Lap B + a^4 Lap^2 B for B of degree <= 3 per
variable far from the edge of D, int G = 1, and agreement of the dense uniform
operator with the direct sum."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import k0

from oracle import volume as V
from oracle.quadrature import gauss_legendre, lagrange_matrix


def _brute(x0, box, j, q, alpha):
    xi, _ = gauss_legendre(q)
    cx, cy, w = box
    ix, iy = j % q, j // q

    def f(y, x):
        r = math.hypot(x - x0[0], y - x0[1])
        lx = lagrange_matrix(xi, np.array([(x - cx) * 2 / w]))[ix][0]
        ly = lagrange_matrix(xi, np.array([(y - cy) * 2 / w]))[iy][0]
        return k0(r / alpha) / (2 * math.pi * alpha ** 2) * lx * ly

    xs = sorted(set([cx - w / 2, cx + w / 2] + ([x0[0]] if abs(x0[0] - cx) < w / 2 else [])))
    ys = sorted(set([cy - w / 2, cy + w / 2] + ([x0[1]] if abs(x0[1] - cy) < w / 2 else [])))
    return sum(integrate.dblquad(f, xs[i], xs[i + 1], ys[k], ys[k + 1], epsabs=1e-16, epsrel=1e-11)[0]
               for i in range(len(xs) - 1) for k in range(len(ys) - 1))


@pytest.mark.parametrize("q,alpha,x0", [(4, 0.1, (0.013, -0.04)), (4, 0.1, (0.0655, 0.01)),
                                        (8, 0.0316, (0.0, 0.01)), (8, 0.0316, (0.0159, 0.0155)),
                                        (8, 0.0316, (0.046975, 0.0))])
def test_box_integrals_brute_force(q, alpha, x0):
    box = (0.0, 0.0, 0.125 if q == 4 else 0.03125)
    a = V.box_integrals(np.array(x0), *box, q, alpha)
    for j in ((q + 1,) if q == 8 else (0, q * q - 1)):
        assert abs(a[j] - _brute(x0, box, j, q, alpha)) < 1e-15


def _uniform(nb, q, half):
    xi, _ = gauss_legendre(q)
    w = 2 * half / nb
    leaves, pts = [], []
    for iy in range(nb):
        for ix in range(nb):
            cx, cy = -half + (ix + 0.5) * w, -half + (iy + 0.5) * w
            leaves.append((cx, cy, w))
            pts.append(np.stack([np.tile(cx + 0.5 * w * xi, q), np.repeat(cy + 0.5 * w * xi, q)], axis=1))
    return np.array(leaves), np.concatenate(pts)


def test_polynomial_identity():
    alpha, q = 0.01, 4
    leaves, pts = _uniform(16, q, 0.5)
    B = lambda x, y: x ** 3 * y ** 2 + 2 * x * y ** 3 - x ** 2 + 0.5
    lapB = lambda x, y: 6 * x * y ** 2 + 2 * x ** 3 + 12 * x * y - 2
    lap2B = lambda x, y: 24 * x
    tg = np.array([[0.0123, -0.031], [0.05, 0.08], [-0.1, 0.02], [0.0, 0.0]])
    U = V.volume_potential(leaves, B(pts[:, 0], pts[:, 1]).reshape(len(leaves), -1), q, alpha, tg)
    ex = B(*tg.T) + alpha ** 2 * lapB(*tg.T) + alpha ** 4 * lap2B(*tg.T)
    assert np.max(np.abs(U - ex)) < 5e-14


def test_uniform_operator_matches_direct_sum():
    q, alpha, level = 4, 0.3, 2
    box = (-1.0, -1.0, 2.0)
    M = V.uniform_operator(level, box, q, alpha)
    leaves, pts = _uniform(4, q, 1.0)
    rng = np.random.default_rng(1)
    B = rng.standard_normal(pts.shape[0])
    sel = [0, 7, 40, 63]
    U = V.volume_potential(leaves, B.reshape(16, -1), q, alpha, pts[sel])
    assert np.allclose((M @ B)[sel], U, atol=1e-14, rtol=0)
    # constant density far from the edge of D (alpha small): U -> 1
    M2 = V.uniform_operator(3, (-0.5, -0.5, 1.0), 4, 0.01)
    ones = M2 @ np.ones(M2.shape[0])
    _, p2 = _uniform(8, 4, 0.5)
    deep = np.max(np.abs(p2), axis=1) < 0.1
    assert np.max(np.abs(ones[deep] - 1.0)) < 1e-13


def test_volume_rows_apply_the_direct_sum():
    """volume_rows lays out the integrals of volume_potential as matrix rows: on a small
    adaptive tree (leaves of three sizes, targets in near and far leaves) R @ B equals the
    direct sum, and with B = 1 on every node a row sums to int G over the covered part of D,
    which is 1 up to e^{-dist/alpha} for a target far inside D (int_{R^2} G = 1)."""
    from oracle import tree as T
    tr = T.build((-1.0, -1.0, 2.0), 4, 2, 5, lambda xy: np.exp(-40 * ((xy[:, 0] - 0.3) ** 2 + xy[:, 1] ** 2)), 1e-3)
    leaves = tr.leaf_array()
    nodes = tr.nodes()
    assert len(set(int(round(math.log2(2.0 / w))) for w in leaves[:, 2])) >= 3
    rng = np.random.default_rng(5)
    sel = rng.choice(nodes.shape[0], 6, replace=False)
    alpha = 0.05
    B = np.sin(2 * nodes[:, 0]) + np.cos(3 * nodes[:, 1])
    R = V.volume_rows(leaves, 4, alpha, nodes[sel])
    ref = V.volume_potential(leaves, B.reshape(len(leaves), -1), 4, alpha, nodes[sel])
    assert np.max(np.abs(R @ B - ref)) <= 1e-13 * np.max(np.abs(ref))
    # the mass of G beyond the nearest edge of D (distance d) is about e^{-d/alpha} / 2:
    # alpha = 0.02 and d >= 0.7 leave 3e-16
    deep = V.volume_rows(leaves, 4, 0.02, np.array([[0.3, 0.0], [-0.2, 0.1]]))
    assert np.allclose(deep.sum(axis=1), 1.0, rtol=0, atol=1e-12)


def test_pool_gives_the_serial_values():
    """The process pool cuts targets / rows into chunks and stacks the serial results."""
    from oracle import bie, geometry as G, pool, tree as T
    import mh_workloads as W
    tr = T.build((-1.0, -1.0, 2.0), 4, 3, 3)
    leaves, nodes = tr.leaf_array(), tr.nodes()
    tg = nodes[::97]
    serial = V.volume_rows(leaves, 4, 0.1, tg)
    assert np.array_equal(pool.volume_rows(leaves, 4, 0.1, tg, procs=2), serial)
    B = np.cos(nodes[:, 0])
    assert np.array_equal(pool.volume_potential(leaves, B, 4, 0.1, tg, procs=2),
                          V.volume_potential(leaves, B, 4, 0.1, tg))
    wl = W.disk_with_hole(n_per_curve=32)
    rows = np.array([0, 5, 31, 32, 60])
    got = pool.nystrom_matrix(wl.curves, 0.1, rows=rows, procs=2)
    assert np.array_equal(got, bie.nystrom_matrix(G.make_curves(wl.curves), 0.1, rows=rows))
