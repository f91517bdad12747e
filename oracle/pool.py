"""Process pool for the oracle's independent loops (test infrastructure, like the rest of
this package).

The volume direct sum is independent per target and the Nystrom matrix per row, so the
pool only cuts the target (row) set into contiguous chunks, runs the serial oracle function
on each chunk in a worker and stacks the results in order: every value is the one the
serial call computes.  Workers are started with the 'spawn' method, never 'fork' (a child
forked from a process that has initialised CUDA can hang), and get the caller's sys.path.
"""
import multiprocessing as mp
import os

import numpy as np


def cores() -> int:
    """Host cores this process may run on."""
    if hasattr(os, "sched_getaffinity"):
        return len(os.sched_getaffinity(0))
    return os.cpu_count() or 1


def _chunks(n, procs):
    k = max(1, min(procs, n))
    return [c for c in np.array_split(np.arange(n), k) if c.size]


def _run(fn, args_list, procs):
    if len(args_list) == 1:
        return [fn(args_list[0])]
    with mp.get_context("spawn").Pool(len(args_list)) as pool:
        return pool.map(fn, args_list)


def _vol_rows(a):
    from . import volume
    leaves, q, alpha, targets = a
    return volume.volume_rows(leaves, q, alpha, targets)


def _vol_pot(a):
    from . import volume
    leaves, B, q, alpha, targets = a
    return volume.volume_potential(leaves, B, q, alpha, targets)


_CURVES = {}   # per worker: curves already built from the same node arrays


def _curves(curve_nodes):
    from . import geometry
    key = tuple((len(c), np.asarray(c).tobytes().__hash__()) for c in curve_nodes)
    if key not in _CURVES:
        _CURVES.clear()
        _CURVES[key] = geometry.make_curves(curve_nodes)
    return _CURVES[key]


def _nys_rows(a):
    from . import bie
    curve_nodes, alpha, order, rows = a
    return bie.nystrom_matrix(_curves(curve_nodes), alpha, order, rows=rows)


def volume_rows(leaves, q, alpha, targets, procs=None):
    """oracle.volume.volume_rows over `procs` worker processes (default: all cores)."""
    targets = np.asarray(targets, dtype=np.float64)
    parts = _run(_vol_rows, [(leaves, q, alpha, targets[c]) for c in _chunks(len(targets), procs or cores())],
                 procs)
    return np.vstack(parts)


def volume_potential(leaves, B, q, alpha, targets, procs=None):
    """oracle.volume.volume_potential over `procs` worker processes (default: all cores)."""
    targets = np.asarray(targets, dtype=np.float64)
    parts = _run(_vol_pot, [(leaves, B, q, alpha, targets[c]) for c in _chunks(len(targets), procs or cores())],
                 procs)
    return np.concatenate(parts)


def nystrom_matrix(curve_nodes, alpha, alpert_order=8, rows=None, procs=None):
    """oracle.bie.nystrom_matrix (all rows, or the listed ones) over worker processes; the
    curves are given by their node arrays and rebuilt in every worker."""
    n = int(sum(len(c) for c in curve_nodes))
    rows = np.arange(n) if rows is None else np.asarray(rows)
    parts = _run(_nys_rows, [(curve_nodes, alpha, alpert_order, rows[c])
                             for c in _chunks(len(rows), procs or cores())], procs)
    return np.vstack(parts)


def _dlp(a):
    from . import bie, geometry
    curve_nodes, sigma, alpha, targets = a
    curves = _curves(curve_nodes)
    return bie.dlp_eval(curves, sigma, alpha, targets, geometry.classify(curves, targets), None)


def _ready(_):
    from . import bie, geometry, volume  # noqa: F401  (import the oracle once per worker)
    return 0


class Workers:
    """A spawn pool kept for several calls (each worker imports the oracle once), for timing
    the oracle on all cores: every method cuts its targets / rows into one chunk per worker
    and returns the serial function's values in order."""

    def __init__(self, procs=None):
        self.n = procs or cores()
        self.pool = mp.get_context("spawn").Pool(self.n)
        self.pool.map(_ready, range(self.n))

    def _map(self, fn, args):
        return self.pool.map(fn, args)

    def volume_potential(self, leaves, B, q, alpha, targets):
        targets = np.asarray(targets, dtype=np.float64)
        return np.concatenate(self._map(_vol_pot, [(leaves, B, q, alpha, targets[c])
                                                   for c in _chunks(len(targets), self.n)]))

    def nystrom_rows(self, curve_nodes, alpha, rows, alpert_order=8):
        rows = np.asarray(rows)
        return np.vstack(self._map(_nys_rows, [(curve_nodes, alpha, alpert_order, rows[c])
                                               for c in _chunks(len(rows), self.n)]))

    def dlp_eval(self, curve_nodes, sigma, alpha, targets):
        """U^h at targets inside Omega (classification in the workers; no normal-line targets)."""
        targets = np.asarray(targets, dtype=np.float64)
        return np.concatenate(self._map(_dlp, [(curve_nodes, sigma, alpha, targets[c])
                                               for c in _chunks(len(targets), self.n)]))

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
