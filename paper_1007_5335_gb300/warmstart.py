"""Learned warm start: trajectory sampling and training loops over the C-ABI (no arithmetic
of the method here; every step runs in libmh).

collect_samples  runs heat_step from u = 0 under given forcings with the previous-step start
                 and records mh_net_sample pairs (x, y) of the chosen steps
train            mh_net_fit (closed-form start) followed by mh_net_train (Adam, early stopping)
"""
from . import (MH_PREC_MIXED, MH_WARM_PREVIOUS, heat_step)


def collect_samples(ctx, prob, net, forcings, n_steps: int, f_next, take=None, prec: int = MH_PREC_MIXED,
                    tol: float = 1e-10):
    """forcings: list of device arrays (F at the tree nodes); take: step indices to record
    (default all).  Returns X, Y (rows x d binary32 device tensors) and the GMRES iteration
    counts of every step."""
    import torch
    steps = list(range(n_steps)) if take is None else sorted(set(take))
    rows = len(forcings) * len(steps)
    dev = f_next.device
    X = torch.empty(rows, net.d, dtype=torch.float32, device=dev)
    Y = torch.empty_like(X)
    prob.set_warm_start(MH_WARM_PREVIOUS)
    n = prob.tree.n_nodes
    its = []
    i = 0
    for F in forcings:
        u = torch.zeros(n, dtype=torch.float64, device=dev)
        un = torch.empty_like(u)
        sigma = torch.zeros(prob.bnd.n, dtype=torch.float64, device=dev)
        sp = torch.empty_like(sigma)
        for s in range(n_steps):
            sp.copy_(sigma)
            info = heat_step(ctx, prob, u, F, f_next, un, sigma, gmres_tol=tol, prec=prec)
            its.append(info.gmres_iterations)
            if s in steps:
                net.sample(prob, sp, sigma, X[i], Y[i])
                i += 1
            u, un = un, u
    return X, Y, its


def train(net, X, Y, Xv, Yv, omega, batch_idx, lr: float = 1e-6, eps: float = 1e-3, power_iters: int = 2,
          ridge: float = 1e-12, eval_every: int = 50):
    """Closed-form start on (X, Y), then Adam over batch_idx keeping the best parameters on
    (Xv, Yv).  Returns (first validation loss, best validation loss, best step)."""
    net.fit(X, Y, omega, eps=eps, power_iters=power_iters, ridge=ridge)
    if batch_idx is None or batch_idx.shape[0] == 0:
        return None
    return net.train(X, Y, batch_idx, lr, Xv, Yv, eval_every=eval_every)
