"""Full-size boundary solve against the oracle (Section 3.2: the Nystrom system of
eq. discrete_sys solved by GMRES; Section 4: tolerance 1e-10).

Starfish workload boundary: N_Gamma = 6 x 1024, alpha^2 = 1e-3.  The oracle assembles the
dense 6144 x 6144 Nystrom matrix (Alpert order 8) and solves it by LU; the GPU solves the
same right-hand side by mh_gmres_solve in binary64 and in mixed precision (binary32
Arnoldi inside binary64 refinement), both to relative residual 1e-12.  Both densities agree
with the LU solution to relative L2 1e-10, and the GPU's operator applied to that solution
reproduces the oracle's matrix-vector product over all 6144 rows to 1e-10.  The right-hand
side is -2 alpha^2 g with g = K0(|y - x0| / alpha) (x0 the centre of the first hole: an
exact homogeneous solution's boundary data) plus a smooth function spread over every curve.
Placed late in the run order (file name): it holds the 302 MB matrix on the host."""
import numpy as np
import pytest
from scipy.special import k0

import mh_workloads as W
from oracle import pool

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def system():
    wl = W.starfish_domain()
    y = np.concatenate(wl.curves)
    x0 = wl.curves[1].mean(axis=0)
    g = k0(np.hypot(y[:, 0] - x0[0], y[:, 1] - x0[1]) / wl.alpha) + np.cos(3 * y[:, 0]) * np.sin(2 * y[:, 1])
    rhs = -2.0 * wl.alpha ** 2 * g
    A = pool.nystrom_matrix(wl.curves, wl.alpha)
    return wl, A, rhs, np.linalg.solve(A, rhs)


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_gmres_matches_dense_solve(mh, system, prec):
    wl, A, rhs, sigma_ref = system
    ctx = mh.Context(0)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    assert bnd.n == 6144
    sig = torch.zeros(bnd.n, dtype=torch.float64, device="cuda")
    info = mh.mh_gmres_solve(ctx, bnd, wl.alpha, torch.tensor(rhs, device="cuda"), sig, tol=1e-12, max_iter=100,
                             prec=prec)
    assert info.converged and info.rel_residual <= 1e-12
    got = sig.cpu().numpy()
    e = float(np.linalg.norm(got - sigma_ref) / np.linalg.norm(sigma_ref))
    print(f"full-size GMRES prec={prec}: {info.iterations} iterations, rel L2 vs LU {e:.2e}")
    assert e <= 1e-10
    if prec == 0:
        out = torch.empty_like(sig)
        mh.mh_double_layer_apply(ctx, bnd, wl.alpha, torch.tensor(sigma_ref, device="cuda"), out)
        ref = A @ sigma_ref
        eo = float(np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref))
        print(f"full-size operator: rel L2 {eo:.2e}")
        assert eo <= 1e-10
