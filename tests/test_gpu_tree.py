"""GPU parity of the device quadtree (Section 3.1) against the oracle's tree:
leaves, boxes and the U, V, W, X interaction lists must agree exactly (integer
work: bit-exact), node coordinates to rounding.  Cases: the uniform level-4 tree,
a small adaptive tree, and the full-size adaptive tree of the starfish workload
(4027 leaves, levels 4..8), whose lists are compared on sampled boxes against the
brute-force list definitions."""
import numpy as np
import pytest

import mh_workloads as W
from oracle import tree as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(mh):
    return mh.Context(0)


def _lists_dict(gt, which):
    offs, items = gt.list(which)
    return offs, items


def _compare(gt, ot, full_lists=True, sample=None):
    assert [tuple(b) for b in gt.leaves()] == list(ot.leaves)
    assert [tuple(b) for b in gt.boxes()] == list(ot.boxes)
    nodes = gt.nodes().cpu().numpy()
    assert np.max(np.abs(nodes - ot.nodes())) < 1e-15
    if full_lists:
        U, V, Wl, X = T.lists(ot)
        ref = {"U": U, "V": V, "W": Wl, "X": X}
        for which in "UVWX":
            offs, items = gt.list(which)
            for i, b in enumerate(ot.boxes):
                got = list(items[offs[i]:offs[i + 1]])
                exp = ref[which].get(b, [])
                assert got == exp, (which, b, got, exp)
    else:
        boxes = ot.boxes
        bid = ot.box_id
        for which in "UVWX":
            offs, items = gt.list(which)
            for i in sample:
                b = boxes[i]
                got = list(items[offs[i]:offs[i + 1]])
                leaf = b in ot.leaf_id
                if which == "U":
                    exp = sorted(bid[c] for c in ot.leaves if T._touch(b, c)) if leaf else []
                elif which == "W":
                    exp = sorted(bid[c] for c in boxes if c[0] > b[0] and not T._touch(b, c)
                                 and T._touch(b, (c[0] - 1, c[1] // 2, c[2] // 2))) if leaf else []
                elif which == "V":
                    exp = [] if b[0] < 2 else sorted(
                        bid[c] for c in boxes if c[0] == b[0] and not T._touch(b, c)
                        and T._touch((b[0] - 1, b[1] // 2, b[2] // 2), (c[0] - 1, c[1] // 2, c[2] // 2)))
                else:
                    exp = sorted(bid[c] for c in ot.leaves if c[0] == b[0] - 1 and not T._touch(b, c)
                                 and T._touch((b[0] - 1, b[1] // 2, b[2] // 2), c))
                assert got == exp, (which, b, got, exp)


def test_uniform_tree(mh, ctx):
    wl = W.disk_with_hole()
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level)
    ot = T.build(wl.box, wl.q, wl.min_level, wl.max_level)
    assert gt.n_leaves == 256 and gt.n_nodes == 4096
    _compare(gt, ot)


def test_small_adaptive_tree(mh, ctx):
    wl = W.starfish_domain(n_per_curve=64)
    gt = mh.Tree(ctx, wl.box, 4, 2, 6, wl.forcing, 1e-6)
    ot = T.build(wl.box, 4, 2, 6, wl.forcing, 1e-6)
    _compare(gt, ot)


def test_full_size_adaptive_tree(mh, ctx):
    wl = W.starfish_domain()
    gt = mh.Tree(ctx, wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    ot = T.build(wl.box, wl.q, wl.min_level, wl.max_level, wl.forcing, wl.refine_tol)
    assert gt.n_leaves == 4027 and gt.n_nodes == 257728
    rng = np.random.default_rng(5)
    _compare(gt, ot, full_lists=False, sample=rng.choice(len(ot.boxes), 40, replace=False))
