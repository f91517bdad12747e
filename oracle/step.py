"""One IMEX (backward) Euler step of the heat equation (Section 2):
    u^{N+1} - alpha^2 Lap u^{N+1} = B = u^N + dt F^N  in Omega,  alpha^2 = dt,
    u^{N+1} = f(t_{N+1}) on Gamma,
solved as U = U^p + U^h (Section 2):
  1. B~ = u^N + dt F^N at volume nodes in Omega; outside Omega the extension
     (Section 3.1): the constant C_k of the curve whose exterior holds the node
     plus dt F^N ("const"), or caller-supplied values ("array");
  2. U~^p = volume potential of B~ at the volume nodes (oracle.volume);
  3. U^p on Gamma by leaf interpolation (Section 3.1);
  4. g = f - U^p on Gamma; solve A sigma = -2 alpha^2 g (oracle.bie);
  5. U^h at volume nodes in Omega (oracle.bie.dlp_eval);
  6. u^{N+1} = U~^p + U^h in Omega; outside Omega u^{N+1} = C_k ("const") or
     U~^p ("array").
The volume operator is passed in as a callable so that uniform trees can use
the dense cached operator and adaptive trees the direct sum.

The Allen-Cahn equation of Section 4, Example 3, u_t - eps Lap u = u (1 - u^2), with the
reaction term explicit is ``allen_cahn_step``: alpha^2 = eps dt and
    B = u^N + dt u^N (1 - (u^N)^2),
outside Omega C_k + dt C_k (1 - C_k^2) (u = C_k there); the rest of the step is the same.
Pin: far from Gamma (d >> alpha) the step is the free-space resolvent of B,
u^{N+1} = B + alpha^2 Lap B + O(alpha^4), on a smooth u^N.

The extrapolated Gear step (Section 2, the display after eq. mod_helm_forced) is
``heat_step_gear``: alpha^2 = 2 dt / 3 and
    B = 4/3 u^N - 1/3 u^{N-1} + 4/3 dt F^N - 2/3 dt F^{N-1},
with the constant extension C_k + dt (4/3 F^N - 2/3 F^{N-1}) outside Omega; the rest of
the step is the same.  Pin: on the eigenfunction sin(pi x) cos(pi y) the fully discrete
error equals the error of the scheme's own scalar recurrence (second order in dt).
"""
import numpy as np

from . import bie


class Problem:
    def __init__(self, curves, tree, alpha, dt, info, bnd_leaf, A, ext_mode="const",
                 ext_const=None, volume_op=None, gmres_tol=1e-10, use_lu=False):
        self.curves = curves
        self.tree = tree
        self.alpha = alpha
        self.dt = dt
        self.info = info                       # geometry.classify(curves, tree.nodes())
        self.bnd_leaf = bnd_leaf               # leaf index of every boundary node
        self.A = A                             # dense Nystrom matrix
        self.ext_mode = ext_mode
        self.ext_const = ext_const
        self.volume_op = volume_op             # callable B~ (N_D,) -> U~^p (N_D,)
        self.gmres_tol = gmres_tol
        self.use_lu = use_lu
        self.nodes = tree.nodes()
        self.bnodes = np.concatenate([c.nodes for c in curves])
        self.inside = info.region == -1


def heat_step(pb: Problem, u, F, f_next, b_ext=None, sigma0=None):
    """IMEX Euler: returns (u_next, sigma, gmres_iterations)."""
    region = pb.info.region
    B = u + pb.dt * F
    out = ~pb.inside
    if pb.ext_mode == "const":
        B[out] = np.asarray(pb.ext_const)[region[out]] + pb.dt * F[out]
    else:
        B[out] = b_ext[out]
    return _solve(pb, B, f_next, sigma0)


def heat_step_gear(pb: Problem, u, u_prev, F, F_prev, f_next, b_ext=None, sigma0=None):
    """Extrapolated Gear (pb.alpha^2 must be 2 dt / 3): returns (u_next, sigma, iterations)."""
    region = pb.info.region
    forcing = pb.dt * (4.0 * F - 2.0 * F_prev) / 3.0
    B = (4.0 * u - u_prev) / 3.0 + forcing
    out = ~pb.inside
    if pb.ext_mode == "const":
        B[out] = np.asarray(pb.ext_const)[region[out]] + forcing[out]
    else:
        B[out] = b_ext[out]
    return _solve(pb, B, f_next, sigma0)


def allen_cahn_step(pb: Problem, u, f_next, b_ext=None, sigma0=None):
    """IMEX Euler for u_t - eps Lap u = u (1 - u^2) (pb.alpha^2 must be eps pb.dt): returns
    (u_next, sigma, iterations)."""
    region = pb.info.region
    B = u + pb.dt * u * (1.0 - u * u)
    out = ~pb.inside
    if pb.ext_mode == "const":
        c = np.asarray(pb.ext_const, dtype=float)[region[out]]
        B[out] = c + pb.dt * c * (1.0 - c * c)
    else:
        B[out] = b_ext[out]
    return _solve(pb, B, f_next, sigma0)


def _solve(pb: Problem, B, f_next, sigma0):
    region = pb.info.region
    out = ~pb.inside
    Up = pb.volume_op(B)
    from . import volume
    Ug = volume.interpolate(pb.tree.leaf_array(), Up, pb.tree.q, pb.bnodes, pb.bnd_leaf)
    g = f_next - Ug
    rhs = -2.0 * pb.alpha ** 2 * g
    if pb.use_lu:
        sigma = np.linalg.solve(pb.A, rhs)
        its = 0
    else:
        sigma, its, _ = bie.gmres(pb.A, rhs, sigma0, pb.gmres_tol)
    u_next = Up.copy()
    idx = np.nonzero(pb.inside)[0]
    sub_info = _subset(pb.info, idx)
    u_next[idx] += bie.dlp_eval(pb.curves, sigma, pb.alpha, pb.nodes[idx], sub_info, pb.A @ sigma)
    if pb.ext_mode == "const":
        u_next[out] = np.asarray(pb.ext_const)[region[out]]
    return u_next, sigma, its


def _subset(info, idx):
    class _S:
        pass
    s = _S()
    s.region = info.region[idx]
    s.proj = [info.proj[i] for i in idx]
    return s
