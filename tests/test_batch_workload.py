"""The batched workload's geometry (mh_workloads.batch_problem): holes inside the unit disk
with the stated gap, orientations, and the stated size and alpha ranges."""
import math

import numpy as np

import mh_workloads as W


def _signed_area(c):
    x, y = c[:, 0], c[:, 1]
    return 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)


def test_batch_geometry_and_ranges():
    n_gamma, alphas, holes = [], [], []
    for i in range(W.BATCH_SIZE):
        w = W.batch_problem(i)
        curves = w.curves
        npc = curves[0].shape[0]
        assert 256 <= npc <= 2048 and npc % 32 == 0
        assert all(c.shape[0] == npc for c in curves)
        assert 1 <= len(curves) - 1 <= 8
        assert _signed_area(curves[0]) > 0 and all(_signed_area(c) < 0 for c in curves[1:])
        for k, c in enumerate(curves[1:]):
            assert np.max(np.hypot(c[:, 0], c[:, 1])) <= 1.0 - 0.05 + 1e-12
            st = max(1, npc // 256)          # every st-th node: spacing <= 2 pi * 0.16 / 256
            for c2 in curves[k + 2:]:
                a, b = c[::st], c2[::st]
                d = np.min(np.hypot(a[:, None, 0] - b[None, :, 0], a[:, None, 1] - b[None, :, 1]))
                assert d >= 0.05 - 1e-12
        assert 1e-4 <= w.alpha ** 2 <= 1e-2 and abs(w.dt - w.alpha ** 2) < 1e-15
        assert 1e-10 <= w.refine_tol <= 1e-5
        n_gamma.append(w.n_gamma)
        alphas.append(w.alpha ** 2)
        holes.append(len(curves) - 1)
    # the draws cover their ranges
    assert min(holes) == 1 and max(holes) == 8
    assert min(alphas) < 2e-4 and max(alphas) > 5e-3
    assert min(n_gamma) < 2000 and max(n_gamma) > 12000
    # deterministic
    a, b = W.batch_problem(5), W.batch_problem(5)
    assert all(np.array_equal(x, y) for x, y in zip(a.curves, b.curves))
