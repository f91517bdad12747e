"""Volume potential of the extended right-hand side (Section 3.1,
eq. volume_potential):
    U~^p(x) = int_D B~(y) G(x - y) dA_y,   G(r) = K0(r/alpha) / (2 pi alpha^2),
approximated, as in Section 3.1, by replacing B~ on each leaf D_i by its
interpolating polynomial:
    U~^p(x) ~= sum_i int_{D_i} G(x - y) P_i(y) dA,
    P_i(y)  = sum_j B~_j L^i_j(y)  (tensor Lagrange basis on q x q Gauss-Legendre nodes).
The oracle evaluates this definition directly, O(N_D M): it is the quantity
the fast multipole method approximates (Section 3.1: "direct evaluation ...
would require O(N_D^2) work").

Integrals I^i_j(x) = int_{D_i} G(x - y) L^i_j(y) dA:
  * box separated from x (dist(x, D_i) >= side of D_i): 16 x 16 tensor
    Gauss-Legendre rule on D_i;
  * x inside the box: the box is split into the four triangles (x, P, Q)
    over its edges PQ; each triangle is mapped from [0,1]^2 by
    (s, tau) -> x + s (P + tau (Q - P) - x) (Duffy), Jacobian 2 |T| s, with
    16-point Gauss-Legendre panels graded geometrically (ratio 4) toward s = 0
    (log singularity of K0) and toward the foot of the perpendicular from x
    on the edge line (near-singular when x is close to that line);
  * x outside but not separated: quadrisect the box and apply these rules to
    the pieces (the basis stays that of the leaf).
U~^p on Gamma (Section 3.1, last paragraph): the interpolating polynomial of
U~^p on the leaf that contains the boundary point, evaluated there.
Pins: int_{R^2} G = 1; for B of degree <= 3 per variable,
U~^p = B + alpha^2 Lap B + alpha^4 Lap^2 B deep inside D; brute-force 2-D
quadrature (scipy dblquad) of single box integrals.
"""
import math

import numpy as np

from .quadrature import gauss_legendre, lagrange_matrix
from .special import green

NGL = 16
_GX, _GW = gauss_legendre(NGL)


def _panels(breaks):
    """Gauss-Legendre nodes/weights on consecutive intervals given by `breaks`."""
    b = np.asarray(breaks, dtype=np.float64)
    lo, hi = b[:-1], b[1:]
    mid = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo)
    nodes = (mid[:, None] + half[:, None] * _GX[None, :]).ravel()
    wts = (half[:, None] * _GW[None, :]).ravel()
    return nodes, wts


def _s_rule():
    br = [0.0] + [4.0 ** (-k) for k in range(14, 0, -1)] + [1.0]
    return _panels(br)


_S_NODES, _S_WTS = _s_rule()


def _tau_rule(c, scale):
    """Panels on [0, 1] graded geometrically toward c with smallest half-width `scale`."""
    if scale >= 0.25:
        br = [0.0, 1.0] if not (0.0 < c < 1.0) else [0.0, c, 1.0]
        return _panels(br)
    pts = {0.0, 1.0}
    if 0.0 < c < 1.0:
        pts.add(c)
    d = scale
    while d < 1.0:
        for v in (c - d, c + d):
            if 0.0 < v < 1.0:
                pts.add(v)
        d *= 4.0
    return _panels(sorted(pts))


def _basis(pts, cx, cy, w, xi):
    """Tensor Lagrange basis at points pts (..., 2): returns (..., q*q) with j = iy*q + ix."""
    q = xi.shape[0]
    lx = lagrange_matrix(xi, (pts[..., 0] - cx) * (2.0 / w))   # (q, ...)
    ly = lagrange_matrix(xi, (pts[..., 1] - cy) * (2.0 / w))
    out = ly[:, None] * lx[None, :]                           # (q_y, q_x, ...)
    return np.moveaxis(out.reshape((q * q,) + pts.shape[:-1]), 0, -1)


def _duffy(x0, region, leaf, q, alpha):
    """int_region G(x0 - y) L_j(y) dA for x0 inside the closed square `region`
    (cx, cy, side): four Duffy triangles with apex x0 (all of non-negative area).
    The basis L_j is that of `leaf` (cx, cy, w)."""
    xi, _ = gauss_legendre(q)
    cx, cy, w = region
    hw = 0.5 * w
    corners = [np.array([cx - hw, cy - hw]), np.array([cx + hw, cy - hw]),
               np.array([cx + hw, cy + hw]), np.array([cx - hw, cy + hw])]
    total = np.zeros(q * q)
    for e in range(4):
        P = corners[e]
        Q = corners[(e + 1) % 4]
        a = P - x0
        b = Q - x0
        area2 = a[0] * b[1] - a[1] * b[0]          # 2 x area (>= 0 for x0 inside)
        if area2 <= 0.0:
            continue
        E = Q - P
        L = math.hypot(E[0], E[1])
        dist = area2 / L                           # distance from x0 to the edge line
        tau0 = -float(a @ E) / (L * L)             # foot of the perpendicular
        tn, tw = _tau_rule(min(max(tau0, 0.0), 1.0), dist / L)
        ray = a[None, :] + tn[:, None] * E[None, :]            # (nt, 2)
        rlen = np.hypot(ray[:, 0], ray[:, 1])                  # (nt,)
        pts = x0[None, None, :] + _S_NODES[None, :, None] * ray[:, None, :]
        r = _S_NODES[None, :] * rlen[:, None]
        wt = area2 * tw[:, None] * (_S_WTS * _S_NODES)[None, :]
        f = green(r, alpha) * wt
        total += np.einsum("ts,tsj->j", f, _basis(pts, *leaf, xi))
    return total


def _tensor_gl(x0, region, leaf, q, alpha):
    """16 x 16 tensor Gauss-Legendre rule on `region` with the basis of `leaf`."""
    xi, _ = gauss_legendre(q)
    cx, cy, w = region
    X = cx + 0.5 * w * _GX
    Y = cy + 0.5 * w * _GX
    r = np.sqrt((Y[:, None] - x0[1]) ** 2 + (X[None, :] - x0[0]) ** 2)     # (v, u)
    gm = green(r, alpha) * np.outer(_GW, _GW) * (0.25 * w * w)
    lx = lagrange_matrix(xi, (X - leaf[0]) * (2.0 / leaf[2]))               # (q, u)
    ly = lagrange_matrix(xi, (Y - leaf[1]) * (2.0 / leaf[2]))               # (q, v)
    return (ly @ gm @ lx.T).reshape(q * q)


def _separated(x0, region):
    cx, cy, w = region
    dx = max(abs(x0[0] - cx) - 0.5 * w, 0.0)
    dy = max(abs(x0[1] - cy) - 0.5 * w, 0.0)
    return math.hypot(dx, dy) >= w


def _inside(x0, region):
    cx, cy, w = region
    return abs(x0[0] - cx) <= 0.5 * w and abs(x0[1] - cy) <= 0.5 * w


def _integrate(x0, region, leaf, q, alpha):
    if _separated(x0, region):
        return _tensor_gl(x0, region, leaf, q, alpha)
    if _inside(x0, region):
        return _duffy(x0, region, leaf, q, alpha)
    cx, cy, w = region
    qw = 0.25 * w
    return sum(_integrate(x0, (cx + sx * qw, cy + sy * qw, 0.5 * w), leaf, q, alpha)
               for sy in (-1, 1) for sx in (-1, 1))


def box_integrals_near(x0, cx, cy, w, q, alpha):
    """I_j = int_box G(x0 - y) L_j(y) dA for a box not separated from x0: Duffy
    triangles from x0 when x0 lies in the box, otherwise quadrisection until
    every piece is separated from x0 or contains it."""
    x0 = np.asarray(x0, dtype=np.float64)
    return _integrate(x0, (cx, cy, w), (cx, cy, w), q, alpha)


def box_integrals_far(x0, boxes, q, alpha):
    """Tensor 16x16 Gauss-Legendre rule for many boxes at once.
    boxes: (M, 3) array of (cx, cy, w).  Returns (M, q*q)."""
    xi, _ = gauss_legendre(q)
    lq = lagrange_matrix(xi, _GX)                                # (q, 16)
    cx, cy, w = boxes[:, 0], boxes[:, 1], boxes[:, 2]
    X = cx[:, None] + 0.5 * w[:, None] * _GX[None, :]           # (M, 16)
    Y = cy[:, None] + 0.5 * w[:, None] * _GX[None, :]
    dx = X - x0[0]
    dy = Y - x0[1]
    r = np.sqrt(dy[:, :, None] ** 2 + dx[:, None, :] ** 2)      # (M, v, u)
    gm = green(r, alpha) * (_GW[None, :, None] * _GW[None, None, :]) * (0.25 * w * w)[:, None, None]
    out = np.einsum("iv,mvu,ju->mij", lq, gm, lq)                # (M, iy, ix)
    return out.reshape(boxes.shape[0], q * q)


def box_integrals(x0, cx, cy, w, q, alpha):
    x0 = np.asarray(x0, dtype=np.float64)
    hw = 0.5 * w
    dx = max(abs(x0[0] - cx) - hw, 0.0)
    dy = max(abs(x0[1] - cy) - hw, 0.0)
    if math.hypot(dx, dy) >= w:
        return box_integrals_far(x0, np.array([[cx, cy, w]]), q, alpha)[0]
    return box_integrals_near(x0, cx, cy, w, q, alpha)


def volume_potential(leaves, B, q, alpha, targets):
    """Direct sum  U(x) = sum_i sum_j B[i, j] I^i_j(x)  at each target.
    leaves: (M, 3) array (cx, cy, w); B: (M, q*q)."""
    leaves = np.asarray(leaves, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64).reshape(leaves.shape[0], q * q)
    out = np.zeros(targets.shape[0])
    hw = 0.5 * leaves[:, 2]
    for t, x0 in enumerate(np.asarray(targets, dtype=np.float64)):
        dx = np.maximum(np.abs(x0[0] - leaves[:, 0]) - hw, 0.0)
        dy = np.maximum(np.abs(x0[1] - leaves[:, 1]) - hw, 0.0)
        far = np.hypot(dx, dy) >= leaves[:, 2]
        fi = np.nonzero(far)[0]
        acc = 0.0
        if fi.size:
            acc += float(np.sum(box_integrals_far(x0, leaves[fi], q, alpha) * B[fi]))
        for i in np.nonzero(~far)[0]:
            acc += float(box_integrals_near(x0, *leaves[i], q, alpha) @ B[i])
        out[t] = acc
    return out


def volume_rows(leaves, q, alpha, targets):
    """The direct sum as a matrix: R[t, i q^2 + j] = I^i_j(x_t), the same integrals as
    ``volume_potential`` (same rule per leaf), so that volume_potential(B) = R @ B.ravel().
    Lets a test apply the definition to several right-hand sides at the cost of one."""
    leaves = np.asarray(leaves, dtype=np.float64)
    qq = q * q
    targets = np.asarray(targets, dtype=np.float64)
    R = np.zeros((targets.shape[0], leaves.shape[0] * qq))
    hw = 0.5 * leaves[:, 2]
    for t, x0 in enumerate(targets):
        dx = np.maximum(np.abs(x0[0] - leaves[:, 0]) - hw, 0.0)
        dy = np.maximum(np.abs(x0[1] - leaves[:, 1]) - hw, 0.0)
        far = np.hypot(dx, dy) >= leaves[:, 2]
        row = R[t].reshape(leaves.shape[0], qq)
        fi = np.nonzero(far)[0]
        if fi.size:
            row[fi] = box_integrals_far(x0, leaves[fi], q, alpha)
        for i in np.nonzero(~far)[0]:
            row[i] = box_integrals_near(x0, *leaves[i], q, alpha)
    return R


def uniform_operator(level: int, box, q: int, alpha: float, order=None) -> np.ndarray:
    """Dense N_D x N_D matrix of the direct volume sum on a uniform tree (all leaves at
    `level`, leaf-major node order; leaves in the order of `order`, a list of (ix, iy),
    default row-major (iy, ix)).
    By translation invariance each (leaf offset, target node, basis) integral is
    computed once."""
    xi, _ = gauss_legendre(q)
    nb = 2 ** level
    w = box[2] / nb
    qq = q * q
    # target node positions relative to the target leaf centre
    tx = np.tile(0.5 * w * xi, q)
    ty = np.repeat(0.5 * w * xi, q)
    tab = {}
    for di in range(-(nb - 1), nb):
        for dj in range(-(nb - 1), nb):
            T = np.zeros((qq, qq))
            for t in range(qq):
                x0 = np.array([tx[t], ty[t]])
                T[t] = box_integrals(x0, di * w, dj * w, w, q, alpha)
            tab[(di, dj)] = T
    if order is None:
        order = [(ix, iy) for iy in range(nb) for ix in range(nb)]
    n = nb * nb * qq
    M = np.zeros((n, n))
    for it, (tx_, ty_) in enumerate(order):
        for isrc, (sx, sy) in enumerate(order):
            M[it * qq:(it + 1) * qq, isrc * qq:(isrc + 1) * qq] = tab[(sx - tx_, sy - ty_)]
    return M


def interpolate(leaves, values, q, pts, leaf_of_pt):
    """Evaluate each leaf's interpolating polynomial of `values` at pts (leaf given)."""
    xi, _ = gauss_legendre(q)
    leaves = np.asarray(leaves, dtype=np.float64)
    V = np.asarray(values, dtype=np.float64).reshape(leaves.shape[0], q * q)
    out = np.zeros(pts.shape[0])
    for i, (p, lf) in enumerate(zip(np.asarray(pts, dtype=np.float64), leaf_of_pt)):
        cx, cy, w = leaves[lf]
        out[i] = float(_basis(p[None, :], cx, cy, w, xi)[0] @ V[lf])
    return out
