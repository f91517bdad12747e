"""Pins of the oracle's quadtree (Section 3.1) and FMM lists: uniform trees have
the textbook list sizes; adaptive trees are 2:1 balanced, tile D exactly and
satisfy U symmetry and W/X duality."""
import numpy as np

import mh_workloads as W
from oracle import tree as T


def test_uniform_tree_lists():
    tr = T.build((-1, -1, 2), 4, 3, 3)
    assert len(tr.leaves) == 64 and all(b[0] == 3 for b in tr.leaves)
    U, V, Wl, X = T.lists(tr)
    inner = [b for b in tr.leaves if 1 <= b[1] <= 6 and 1 <= b[2] <= 6]
    assert all(len(U[b]) == 9 for b in inner)
    deep = [b for b in tr.leaves if 2 <= b[1] <= 5 and 2 <= b[2] <= 5]
    assert all(len(V[b]) == 27 for b in deep)
    assert all(len(Wl[b]) == 0 for b in tr.leaves) and all(len(X[b]) == 0 for b in tr.boxes)
    # Morton order of leaves: the first four are the children of the first level-2 box
    assert tr.leaves[:4] == [(3, 0, 0), (3, 1, 0), (3, 0, 1), (3, 1, 1)]


def test_adaptive_tree_balanced_and_tiling():
    wl = W.starfish_domain(n_per_curve=64)
    tr = T.build(wl.box, 4, 2, 6, wl.forcing, 1e-6)
    levels = np.array([b[0] for b in tr.leaves])
    assert levels.min() >= 2 and levels.max() == 6
    area = sum((2.0 / (1 << b[0])) ** 2 for b in tr.leaves)
    assert abs(area - 4.0) < 1e-12
    leaves = tr.leaves
    for i, a in enumerate(leaves):
        for b in leaves[i + 1:]:
            if T._touch(a, b):
                assert abs(a[0] - b[0]) <= 1
    U, V, Wl, X = T.lists(tr)
    ids = tr.box_id
    for b in leaves:
        for c in U[b]:
            assert ids[b] in U[tr.boxes[c]]
        for c in Wl[b]:
            assert tr.boxes[c][0] == b[0] + 1
            assert ids[b] in X[tr.boxes[c]]
    for b in tr.boxes:
        for c in X[b]:
            assert tr.boxes[c][0] == b[0] - 1
    # every leaf node is located in its own leaf
    nodes = tr.nodes()
    for k in range(0, nodes.shape[0], 97):
        assert tr.locate(nodes[k]) == k // 16
