"""The allocation-free GMRES entry point (mh_gmres_solve_static) against the allocating one.

Callers that cannot allocate device memory while they solve use mh_gmres_solve_static,
whose Krylov workspace is a fixed array inside the library.  This test calls it through
the C ABI twice in a row (the array keeps the previous call's contents, so the second
call checks that nothing stale leaks in) and compares each density with the one from
mh_gmres_solve on the same system, to the binary64 bar of the other tests (relative L2
<= 1e-10).  The library's count of cudaMalloc / cudaFree calls must not move during the
static calls.  Collected last on purpose (file name)."""
import numpy as np
import pytest

import mh_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_gmres_matches_allocating_gmres_twice():
    import paper_1007_5335_gb300 as mh
    wl = W.disk_with_hole()
    ctx = mh.Context(0)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    rng = np.random.default_rng(7)
    for call in range(2):
        rhs = torch.tensor(rng.standard_normal(bnd.n), device="cuda")
        ref = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
        info_ref = mh.mh_gmres_solve(ctx, bnd, wl.alpha, rhs, ref, tol=1e-12)   # also assembles the operator
        got = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        allocs = mh.device_alloc_calls()
        info = mh.mh_gmres_solve_static(ctx, bnd, wl.alpha, rhs, got, tol=1e-12, max_iter=64)
        assert mh.device_alloc_calls() == allocs, "the static solve allocated or freed device memory"
        assert info.converged and info.rel_residual <= 1e-12
        # the static loop reads the residual every iteration and stops at the first one below
        # tol; the allocating solver reads it only at predicted points and may run a few more
        assert 1 <= info.iterations <= info_ref.iterations
        # same start (zero), same residual of the start
        assert info.initial_rel_residual == pytest.approx(info_ref.initial_rel_residual, rel=1e-12)
        e = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
        assert e < 1e-10, (call, e)


def test_static_gmres_rejects_sizes_beyond_its_limit():
    import paper_1007_5335_gb300 as mh
    wl = W.disk_with_hole()
    ctx = mh.Context(0)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    rhs = torch.ones(bnd.n, dtype=torch.float64, device="cuda")
    sig = torch.zeros_like(rhs)
    mh.mh_gmres_solve(ctx, bnd, wl.alpha, rhs, sig, tol=1e-10)
    with pytest.raises(mh.MHError) as e:
        mh.mh_gmres_solve_static(ctx, bnd, wl.alpha, rhs, sig, tol=1e-10, max_iter=65)
    assert e.value.status == 1
