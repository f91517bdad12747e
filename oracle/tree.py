"""Adaptive quadtree and interaction lists (Section 3.1: level l+1 is obtained by
splitting every box of level l into four children; a box is refined when the
polynomial interpolating B~ on it is not accurate enough; the childless boxes
D_i, i = 1..M, carry the volume nodes).

Reading of the refinement rule (the paper gives "larger than some preset
tolerance"): a leaf b at level l < max_level is split if l < min_level, or if
    max_{children c} max_{nodes x of c} |F(x) - P_b F(x)| > tol,
where P_b F is the q x q tensor Lagrange interpolant of F on b's own
Gauss-Legendre nodes.  Refinement proceeds level by level.  The tree is then
2:1 balanced: a leaf is split while some leaf touching it (edge or corner) is
two or more levels finer; the result is the coarsest balanced refinement.

Box (l, ix, iy) covers [x0 + ix w_l, x0 + (ix+1) w_l) x [y0 + iy w_l, ...),
w_l = W / 2^l.  Leaves are ordered by the Morton key of their lower-left
corner at the finest level (x bit below y bit); all boxes are ordered by
level, then Morton key.  Lists (the adaptive FMM lists, all by brute-force
definitions here):
  U(b), leaf b : leaves touching b (including b);
  V(b), box b  : children of the boxes touching parent(b) (or parent(b) itself)
                 that have the level of b and do not touch b;
  W(b), leaf b : boxes c finer than b that do not touch b, whose parent touches b;
  X(b), box b  : leaves c with b in W(c).
Pins: balance and tiling properties, list symmetries (U symmetric, X dual to
W), and exact counts on uniform trees.
"""
import numpy as np

from .quadrature import gauss_legendre, lagrange_matrix


def morton(level, ix, iy, max_level):
    s = max_level - level
    x = int(ix) << s
    y = int(iy) << s
    key = 0
    for b in range(max_level + 1):
        key |= ((x >> b) & 1) << (2 * b)
        key |= ((y >> b) & 1) << (2 * b + 1)
    return key


class Tree:
    def __init__(self, box, q, max_level, internal, leaves):
        self.box = tuple(float(v) for v in box)
        self.q = q
        self.max_level = max_level
        self.internal = set(internal)
        key = lambda b: morton(b[0], b[1], b[2], max_level)
        self.leaves = sorted(leaves, key=key)
        self.boxes = sorted(list(self.internal) + list(self.leaves), key=lambda b: (b[0], key(b)))
        self.box_id = {b: i for i, b in enumerate(self.boxes)}
        self.leaf_id = {b: i for i, b in enumerate(self.leaves)}

    def geom(self, b):
        l, ix, iy = b
        w = self.box[2] / (1 << l)
        return (self.box[0] + (ix + 0.5) * w, self.box[1] + (iy + 0.5) * w, w)

    def leaf_array(self):
        return np.array([self.geom(b) for b in self.leaves])

    def nodes(self):
        """Volume nodes, leaf-major, node j = iy*q + ix within a leaf: (N_D, 2)."""
        xi, _ = gauss_legendre(self.q)
        out = []
        for b in self.leaves:
            cx, cy, w = self.geom(b)
            out.append(np.stack([np.tile(cx + 0.5 * w * xi, self.q), np.repeat(cy + 0.5 * w * xi, self.q)], axis=1))
        return np.concatenate(out)

    def locate(self, p):
        """Index of the leaf containing p (half-open boxes, top/right edges of D closed)."""
        x0, y0, W = self.box
        for l in range(self.max_level + 1):
            n = 1 << l
            ix = min(max(int(np.floor((p[0] - x0) / W * n)), 0), n - 1)
            iy = min(max(int(np.floor((p[1] - y0) / W * n)), 0), n - 1)
            if (l, ix, iy) in self.leaf_id:
                return self.leaf_id[(l, ix, iy)]
        raise ValueError("point outside the tree")


def _node_grid(cx, cy, w, xi):
    q = xi.shape[0]
    return np.stack([np.tile(cx + 0.5 * w * xi, q), np.repeat(cy + 0.5 * w * xi, q)], axis=1)


def refine_error(F, cx, cy, w, xi):
    """max over the 4 children's nodes of |F - P_b F| (refinement predicate)."""
    q = xi.shape[0]
    own = F(_node_grid(cx, cy, w, xi)).reshape(q, q)          # [iy, ix]
    err = 0.0
    for sy in (-1, 1):
        for sx in (-1, 1):
            ch = _node_grid(cx + 0.25 * sx * w, cy + 0.25 * sy * w, 0.5 * w, xi)
            lx = lagrange_matrix(xi, (ch[:, 0] - cx) * (2.0 / w))   # (q, n)
            ly = lagrange_matrix(xi, (ch[:, 1] - cy) * (2.0 / w))
            interp = np.einsum("an,ab,bn->n", ly, own, lx)
            err = max(err, float(np.max(np.abs(F(ch) - interp))))
    return err


def _touch(a, b):
    """Closed boxes a, b (level, ix, iy) share at least a point."""
    la, xa, ya = a
    lb, xb, yb = b
    L = max(la, lb)
    sa, sb = 1 << (L - la), 1 << (L - lb)
    ax0, ay0 = xa * sa, ya * sa
    bx0, by0 = xb * sb, yb * sb
    return ax0 <= bx0 + sb and bx0 <= ax0 + sa and ay0 <= by0 + sb and by0 <= ay0 + sa


def build(box, q, min_level, max_level, F=None, tol=np.inf, return_margin=False):
    """Adaptive refinement (level by level) followed by 2:1 balancing."""
    xi, _ = gauss_legendre(q)
    internal = set()
    leaves = []
    level_boxes = [(0, 0, 0)]
    margin = np.inf
    for l in range(max_level + 1):
        nxt = []
        for b in level_boxes:
            split = False
            if l < max_level:
                if l < min_level:
                    split = True
                elif np.isfinite(tol):
                    cx = box[0] + (b[1] + 0.5) * box[2] / (1 << l)
                    cy = box[1] + (b[2] + 0.5) * box[2] / (1 << l)
                    e = refine_error(F, cx, cy, box[2] / (1 << l), xi)
                    margin = min(margin, abs(e - tol) / tol)
                    split = e > tol
            if split:
                internal.add(b)
                nxt += [(l + 1, 2 * b[1] + dx, 2 * b[2] + dy) for dy in (0, 1) for dx in (0, 1)]
            else:
                leaves.append(b)
        level_boxes = nxt
    # 2:1 balance
    leafset = set(leaves)
    changed = True
    while changed:
        changed = False
        for b in sorted(leafset):
            l, ix, iy = b
            n = 1 << l
            need = False
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == 0 and dy == 0:
                        continue
                    nx, ny = ix + dx, iy + dy
                    if not (0 <= nx < n and 0 <= ny < n) or (l, nx, ny) not in internal:
                        continue
                    cxs = [0, 1] if dx == 0 else ([0] if dx == 1 else [1])
                    cys = [0, 1] if dy == 0 else ([0] if dy == 1 else [1])
                    if any((l + 1, 2 * nx + a, 2 * ny + c) in internal for a in cxs for c in cys):
                        need = True
            if need:
                leafset.remove(b)
                internal.add(b)
                for dy in (0, 1):
                    for dx in (0, 1):
                        leafset.add((l + 1, 2 * ix + dx, 2 * iy + dy))
                changed = True
    t = Tree(box, q, max_level, internal, leafset)
    return (t, margin) if return_margin else t


def lists(tree: Tree):
    """U, V, W, X lists as dicts box -> sorted list of box ids (brute force)."""
    boxes = tree.boxes
    leaves = set(tree.leaves)
    bid = tree.box_id
    by_level = {}
    for b in boxes:
        by_level.setdefault(b[0], []).append(b)
    U, V, W, X = {}, {}, {}, {}
    for b in tree.leaves:
        U[b] = sorted(bid[c] for c in tree.leaves if _touch(b, c))
        W[b] = sorted(bid[c] for c in boxes
                      if c[0] > b[0] and not _touch(b, c) and _touch(b, (c[0] - 1, c[1] // 2, c[2] // 2)))
    for b in boxes:
        l = b[0]
        if l < 2:
            V[b] = []
            continue
        par = (l - 1, b[1] // 2, b[2] // 2)
        V[b] = sorted(bid[c] for c in by_level[l]
                      if not _touch(b, c) and _touch(par, (l - 1, c[1] // 2, c[2] // 2)))
    for b in boxes:
        X[b] = []
    for c in tree.leaves:
        for i in W[c]:
            X[boxes[i]].append(bid[c])
    for b in boxes:
        X[b] = sorted(X[b])
    return U, V, W, X
