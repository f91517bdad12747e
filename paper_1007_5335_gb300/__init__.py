"""Python binding of libmh (include/mh.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module passes device
pointers of torch tensors (torch is used for device memory and streams), sizes
and host arrays through ctypes, and raises MHError on a non-zero status.
There is no fallback: if libmh.so is missing the import fails.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmh.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with `python -m paper_1007_5335_gb300.build`")

_lib = ctypes.CDLL(_LIB_PATH)

MH_PREC_FP64 = 0
MH_PREC_MIXED = 1
MH_EXT_CONST = 0
MH_EXT_ARRAY = 1
MH_SCHEME_IMEX_EULER = 0
MH_SCHEME_EXTRAP_GEAR = 1
MH_NET_FP32 = 0
MH_NET_BF16 = 1
MH_NET_BF16X2 = 2
MH_WARM_PREVIOUS = 0
MH_WARM_ZERO = 1
MH_WARM_SECANT = 2
MH_WARM_LEARNED = 3
STATUS = {0: "MH_OK", 1: "MH_ERR_INVALID_ARG", 2: "MH_ERR_GEOMETRY", 3: "MH_ERR_CUDA", 4: "MH_ERR_OOM",
          5: "MH_ERR_NOT_CONVERGED", 6: "MH_ERR_TIMEOUT", 7: "MH_ERR_NUMERIC", 8: "MH_ERR_CALLBACK"}
LISTS = {"U": 0, "V": 1, "W": 2, "X": 3}

_p = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_d = ctypes.c_double


class GmresInfo(ctypes.Structure):
    _fields_ = [("iterations", _i), ("refinements", _i), ("rel_residual", _d), ("converged", _i),
                ("initial_rel_residual", _d)]


class StepInfo(ctypes.Structure):
    _fields_ = [("gmres_iterations", _i), ("gmres_rel_residual", _d), ("initial_rel_residual", _d), ("warm_c", _d)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("p", _i), ("near_tile", _i), ("rel_err", _d), ("ms_per_step", _d)]


FIELD_FN = ctypes.CFUNCTYPE(_i, ctypes.POINTER(_d), _i64, ctypes.POINTER(_d), _p)

_SIGS = {
    "mh_create": [_i, _p, ctypes.POINTER(_p)],
    "mh_destroy": [_p],
    "mh_kernel_launches": [_p],
    "mh_device_alloc_calls": [],
    "mh_set_tensor_cores": [_p, _i],
    "mh_tree_check": [_p, _p],
    "mh_boundary_create": [_p, _i, _p, _p, _i, ctypes.POINTER(_p)],
    "mh_boundary_destroy": [_p],
    "mh_boundary_size": [_p, ctypes.POINTER(_i64)],
    "mh_boundary_geometry": [_p, _p, _p],
    "mh_tree_build": [_p, _p, _i, _i, _i, FIELD_FN, _p, _d, ctypes.POINTER(_p)],
    "mh_tree_destroy": [_p],
    "mh_tree_size": [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "mh_tree_leaves": [_p, _p, _p],
    "mh_tree_boxes": [_p, _p, _p],
    "mh_tree_nodes": [_p, _p, _p],
    "mh_tree_list": [_p, _p, _i, _p, _p],
    "mh_volume_potential": [_p, _p, _d, _i, _p, _p, _i],
    "mh_double_layer_apply": [_p, _p, _d, _p, _p, _i64, _p, _i],
    "mh_gmres_solve": [_p, _p, _d, _p, _p, _d, _i, _i, ctypes.POINTER(GmresInfo)],
    "mh_problem_create": [_p, _p, _p, _d, _i, _i, _i, _p, ctypes.POINTER(_p)],
    "mh_problem_destroy": [_p],
    "mh_problem_matrix_free": [_p, _p, _i],
    "mh_problem_regions": [_p, _p, _p],
    "mh_problem_rhs": [_p, _p, _p],
    "heat_step": [_p, _p, _p, _p, _p, _p, _p, _p, _d, _i, ctypes.POINTER(StepInfo)],
    "allen_cahn_step": [_p, _p, _d, _p, _p, _p, _p, _p, _d, _i, ctypes.POINTER(StepInfo)],
    "heat_step_gear": [_p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _d, _i, ctypes.POINTER(StepInfo)],
    "mh_gmres_solve_static": [_p, _p, _d, _p, _p, _d, _i, ctypes.POINTER(GmresInfo)],
    "mh_net_create": [_p, _p, _i, _i, ctypes.POINTER(_p)],
    "mh_net_destroy": [_p],
    "mh_net_dims": [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "mh_net_get_params": [_p, _p, _p, ctypes.POINTER(_d), ctypes.POINTER(_d)],
    "mh_net_set_params": [_p, _p, _p, _d, _d],
    "mh_net_sample": [_p, _p, _p, _p, _p, _p, _p, ctypes.POINTER(_d)],
    "mh_net_fit": [_p, _p, _p, _p, _i64, _p, _d, _i, _d],
    "mh_net_loss_grad": [_p, _p, _p, _p, _i64, ctypes.POINTER(_d), _p],
    "mh_net_forward": [_p, _p, _p, _i64, _p, _i, _i],
    "mh_net_train": [_p, _p, _p, _p, _i64, _p, _i, _i, _d, _p, _p, _i64, _i, ctypes.POINTER(_d),
                     ctypes.POINTER(_d), ctypes.POINTER(_i)],
    "mh_warm_start": [_p, _p, _d, _p, _i, _i, _p, _p, _p, _p, _p, _i, ctypes.POINTER(_d)],
    "mh_problem_set_warm_start": [_p, _p, _i, _p, _i],
    "mh_batch_create": [_p, _i, _p, ctypes.POINTER(_p)],
    "mh_batch_destroy": [_p],
    "mh_batch_step": [_p, _p, _p, _p, _p, _p, _d, _i, _p],
    "mh_batch_graph_kernels": [_p],
    "mh_problem_set_near_tile": [_p, _p, _i],
    "mh_autotune": [_p, _p, _p, _d, _i, _p, _p, _p, _i, _p, _d, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i),
                    _p],
    "mh_profile_enable": [_p, _i],
    "mh_profile_read": [_p, ctypes.c_char_p, ctypes.POINTER(_d), ctypes.POINTER(_i64), ctypes.POINTER(_d),
                        ctypes.POINTER(_d), _i],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int64 if _name in ("mh_kernel_launches", "mh_batch_graph_kernels",
                                            "mh_device_alloc_calls") else _i
_lib.mh_last_error.argtypes = [_p]
_lib.mh_last_error.restype = ctypes.c_char_p


class MHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    """Device pointer of a contiguous CUDA float64 tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or t.dtype.itemsize != 8 or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor of 8-byte elements")
    return ctypes.c_void_p(t.data_ptr())


def _need(t, n, name):
    """Reject a buffer shorter than the n entries the library will read or write through it."""
    if t is not None and t.numel() < n:
        raise ValueError(f"{name}: {t.numel()} entries, the call needs {n}")


def _ptr4(t):
    """Device pointer of a contiguous CUDA float32 / int32 tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or t.dtype.itemsize != 4 or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor of 4-byte elements")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """mh_create / mh_destroy.  All work is issued on torch's current stream."""

    def __init__(self, device: int = 0):
        import torch
        self.device = device
        stream = torch.cuda.current_stream(device).cuda_stream
        h = _p()
        st = _lib.mh_create(device, _p(stream), ctypes.byref(h))
        if st:
            raise MHError(st, "mh_create failed")
        self.h = h

    def check(self, st):
        if st:
            raise MHError(st, _lib.mh_last_error(self.h).decode())

    @property
    def launches(self) -> int:
        return int(_lib.mh_kernel_launches(self.h))

    def tensor_cores(self, on: bool = True):
        """mh_set_tensor_cores: binary32 contractions on the tensor cores (default) or CUDA cores."""
        self.check(_lib.mh_set_tensor_cores(self.h, 1 if on else 0))

    def profile(self, on: bool = True):
        """mh_profile_enable: time the instrumented kernel regions with CUDA events."""
        self.check(_lib.mh_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, region: str, reset: bool = False):
        """mh_profile_read -> (total_ms, launches, flops, bytes) of a named region."""
        ms, n, f, b = _d(), _i64(), _d(), _d()
        self.check(_lib.mh_profile_read(self.h, region.encode(), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(f),
                                        ctypes.byref(b), 1 if reset else 0))
        return ms.value, n.value, f.value, b.value

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mh_destroy(self.h)
            self.h = None


class Boundary:
    """mh_boundary_create: curves = list of (N_k, 2) arrays (outer CCW first, holes CW)."""

    def __init__(self, ctx: Context, curves, alpert_order: int = 8):
        self.ctx = ctx
        nn = np.array([c.shape[0] for c in curves], dtype=np.int32)
        xy = np.ascontiguousarray(np.concatenate(curves), dtype=np.float64)
        h = _p()
        ctx.check(_lib.mh_boundary_create(ctx.h, len(curves), nn.ctypes.data_as(_p), xy.ctypes.data_as(_p),
                                          alpert_order, ctypes.byref(h)))
        self.h = h
        self.n = int(xy.shape[0])
        self.n_curves = len(curves)

    def geometry(self) -> np.ndarray:
        out = np.zeros((self.n, 8))
        self.ctx.check(_lib.mh_boundary_geometry(self.ctx.h, self.h, out.ctypes.data_as(_p)))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mh_boundary_destroy(self.h)
            self.h = None


class Tree:
    """mh_tree_build.  refine_fn(xy: (n,2) ndarray) -> (n,) ndarray evaluates F on the host."""

    def __init__(self, ctx: Context, box, q: int, min_level: int, max_level: int, refine_fn=None,
                 refine_tol: float = float("inf")):
        self.ctx = ctx
        self._err = None

        def cb(xy_p, n, out_p, user):
            try:
                xy = np.ctypeslib.as_array(xy_p, shape=(n, 2))
                out = np.ctypeslib.as_array(out_p, shape=(n,))
                out[:] = refine_fn(xy)
                return 0
            except Exception as e:  # reported through the status
                self._err = e
                return 1

        self._cb = FIELD_FN(cb) if refine_fn is not None else FIELD_FN()
        box = np.ascontiguousarray(box, dtype=np.float64)
        h = _p()
        ctx.check(_lib.mh_tree_build(ctx.h, box.ctypes.data_as(_p), q, min_level, max_level, self._cb, None,
                                     float(refine_tol), ctypes.byref(h)))
        self.h = h
        nl, nb, nn = _i64(), _i64(), _i64()
        _lib.mh_tree_size(h, ctypes.byref(nl), ctypes.byref(nb), ctypes.byref(nn))
        self.n_leaves, self.n_boxes, self.n_nodes = nl.value, nb.value, nn.value
        self.q = q

    def leaves(self) -> np.ndarray:
        out = np.zeros((self.n_leaves, 3), dtype=np.int32)
        self.ctx.check(_lib.mh_tree_leaves(self.ctx.h, self.h, out.ctypes.data_as(_p)))
        return out

    def boxes(self) -> np.ndarray:
        out = np.zeros((self.n_boxes, 3), dtype=np.int32)
        self.ctx.check(_lib.mh_tree_boxes(self.ctx.h, self.h, out.ctypes.data_as(_p)))
        return out

    def nodes(self):
        import torch
        out = torch.empty((self.n_nodes, 2), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        self.ctx.check(_lib.mh_tree_nodes(self.ctx.h, self.h, _ptr(out)))
        return out

    def check(self):
        """mh_tree_check: raise MHError if a bounded device wait of this tree's work gave up."""
        self.ctx.check(_lib.mh_tree_check(self.ctx.h, self.h))

    def list(self, which: str):
        offs = np.zeros(self.n_boxes + 1, dtype=np.int32)
        self.ctx.check(_lib.mh_tree_list(self.ctx.h, self.h, LISTS[which], offs.ctypes.data_as(_p), None))
        items = np.zeros(max(int(offs[-1]), 1), dtype=np.int32)
        self.ctx.check(_lib.mh_tree_list(self.ctx.h, self.h, LISTS[which], offs.ctypes.data_as(_p),
                                         items.ctypes.data_as(_p)))
        return offs, items[:offs[-1]]

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mh_tree_destroy(self.h)
            self.h = None


def mh_volume_potential(ctx: Context, tree: Tree, alpha: float, p: int, b, out, prec: int = MH_PREC_FP64):
    _need(b, tree.n_nodes, "b")
    _need(out, tree.n_nodes, "out")
    ctx.check(_lib.mh_volume_potential(ctx.h, tree.h, float(alpha), int(p), _ptr(b), _ptr(out), int(prec)))
    return out


def mh_double_layer_apply(ctx: Context, bnd: Boundary, alpha: float, sigma, out, targets=None,
                          prec: int = MH_PREC_FP64):
    n_t = 0 if targets is None else int(targets.shape[0])
    _need(sigma, bnd.n, "sigma")
    if targets is None:
        _need(out, bnd.n, "out")
    elif n_t == 0:
        return out   # no targets (an empty tensor's pointer may be null, which selects the on-surface operator)
    else:
        _need(targets, 2 * n_t, "targets")
        _need(out, n_t, "out")
    ctx.check(_lib.mh_double_layer_apply(ctx.h, bnd.h, float(alpha), _ptr(sigma), _ptr(targets), n_t, _ptr(out),
                                         int(prec)))
    return out


def mh_gmres_solve(ctx: Context, bnd: Boundary, alpha: float, rhs, sigma, tol: float = 1e-10,
                   max_iter: int = 100, prec: int = MH_PREC_FP64) -> GmresInfo:
    _need(rhs, bnd.n, "rhs")
    _need(sigma, bnd.n, "sigma")
    info = GmresInfo()
    ctx.check(_lib.mh_gmres_solve(ctx.h, bnd.h, float(alpha), _ptr(rhs), _ptr(sigma), float(tol), int(max_iter),
                                  int(prec), ctypes.byref(info)))
    return info


def mh_gmres_solve_static(ctx: Context, bnd: Boundary, alpha: float, rhs, sigma, tol: float = 1e-10,
                          max_iter: int = 64) -> GmresInfo:
    """Allocation-free binary64 GMRES (fixed workspace inside the library; see include/mh.h)."""
    _need(rhs, bnd.n, "rhs")
    _need(sigma, bnd.n, "sigma")
    info = GmresInfo()
    ctx.check(_lib.mh_gmres_solve_static(ctx.h, bnd.h, float(alpha), _ptr(rhs), _ptr(sigma), float(tol),
                                         int(max_iter), ctypes.byref(info)))
    return info


class Problem:
    """mh_problem_create: tree + boundary + dt + scheme (alpha^2 = dt or 2 dt / 3) + multipole order p."""

    def __init__(self, ctx: Context, tree: Tree, bnd: Boundary, dt: float, p: int, ext_mode: int = MH_EXT_CONST,
                 ext_const=None, scheme: int = MH_SCHEME_IMEX_EULER):
        self.ctx, self.tree, self.bnd = ctx, tree, bnd
        ec = np.ascontiguousarray(ext_const if ext_const is not None else np.zeros(bnd.n_curves), dtype=np.float64)
        h = _p()
        ctx.check(_lib.mh_problem_create(ctx.h, tree.h, bnd.h, float(dt), int(scheme), int(p), int(ext_mode),
                                         ec.ctypes.data_as(_p), ctypes.byref(h)))
        self.h = h
        self.dt = dt
        self.scheme = scheme
        self.alpha = float(np.sqrt(dt if scheme == MH_SCHEME_IMEX_EULER else 2.0 * dt / 3.0))

    def regions(self) -> np.ndarray:
        out = np.zeros(self.tree.n_nodes, dtype=np.int32)
        self.ctx.check(_lib.mh_problem_regions(self.ctx.h, self.h, out.ctypes.data_as(_p)))
        return out

    def set_warm_start(self, mode: int, net=None, arith: int = MH_NET_BF16X2):
        """mh_problem_set_warm_start: GMRES start of the following steps."""
        self.ctx.check(_lib.mh_problem_set_warm_start(self.ctx.h, self.h, int(mode), net.h if net is not None else None,
                                                      int(arith)))
        self._net = net          # keep the network alive while the problem uses it

    def matrix_free(self, enable: bool = True):
        """mh_problem_matrix_free: the boundary operator by the on-surface multipole pass and
        chirp-transform Alpert correction (binary64) instead of the dense matrix."""
        self.ctx.check(_lib.mh_problem_matrix_free(self.ctx.h, self.h, 1 if enable else 0))

    def set_near_tile(self, threads: int):
        """mh_problem_set_near_tile: threads per block of the near-field double-layer kernel."""
        self.ctx.check(_lib.mh_problem_set_near_tile(self.ctx.h, self.h, int(threads)))

    def rhs(self, out):
        """Right-hand side of the boundary equation of the last step, into the device buffer out."""
        self.ctx.check(_lib.mh_problem_rhs(self.ctx.h, self.h, _ptr(out)))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mh_problem_destroy(self.h)
            self.h = None


def _step_sizes(prob, node_bufs, bnd_bufs):
    for t in node_bufs:
        _need(t, prob.tree.n_nodes, "volume-node buffer")
    for t in bnd_bufs:
        _need(t, prob.bnd.n, "boundary buffer")


def heat_step(ctx: Context, prob: Problem, u, F, f_next, u_next, sigma, b_ext=None, gmres_tol: float = 1e-10,
              prec: int = MH_PREC_FP64) -> StepInfo:
    _step_sizes(prob, (u, F, u_next, b_ext), (f_next, sigma))
    info = StepInfo()
    ctx.check(_lib.heat_step(ctx.h, prob.h, _ptr(u), _ptr(F), _ptr(f_next), _ptr(b_ext), _ptr(u_next), _ptr(sigma),
                             float(gmres_tol), int(prec), ctypes.byref(info)))
    return info


def heat_step_gear(ctx: Context, prob: Problem, u, u_prev, F, F_prev, f_next, u_next, sigma, b_ext=None,
                   gmres_tol: float = 1e-10, prec: int = MH_PREC_FP64) -> StepInfo:
    _step_sizes(prob, (u, u_prev, F, F_prev, u_next, b_ext), (f_next, sigma))
    info = StepInfo()
    ctx.check(_lib.heat_step_gear(ctx.h, prob.h, _ptr(u), _ptr(u_prev), _ptr(F), _ptr(F_prev), _ptr(f_next),
                                  _ptr(b_ext), _ptr(u_next), _ptr(sigma), float(gmres_tol), int(prec),
                                  ctypes.byref(info)))
    return info


def allen_cahn_step(ctx: Context, prob: Problem, eps: float, u, f_next, u_next, sigma, b_ext=None,
                    gmres_tol: float = 1e-10, prec: int = MH_PREC_FP64) -> StepInfo:
    """One IMEX Euler step of u_t - eps Lap u = u (1 - u^2); prob created with dt = eps * dt."""
    _step_sizes(prob, (u, u_next, b_ext), (f_next, sigma))
    info = StepInfo()
    ctx.check(_lib.allen_cahn_step(ctx.h, prob.h, float(eps), _ptr(u), _ptr(f_next), _ptr(b_ext), _ptr(u_next),
                                   _ptr(sigma), float(gmres_tol), int(prec), ctypes.byref(info)))
    return info


class Net:
    """mh_net_create: the learned warm start's network for the boundary bnd (see include/mh.h)."""

    def __init__(self, ctx: Context, bnd: Boundary, n_modes: int = 256, width: int = 256):
        self.ctx, self.bnd = ctx, bnd
        h = _p()
        ctx.check(_lib.mh_net_create(ctx.h, bnd.h, int(n_modes), int(width), ctypes.byref(h)))
        self.h = h
        d, w, n = _i64(), _i64(), _i64()
        _lib.mh_net_dims(h, ctypes.byref(d), ctypes.byref(w), ctypes.byref(n))
        self.d, self.width, self.n_params = d.value, w.value, n.value
        self.n_modes = n_modes

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        gx, gy = _d(), _d()
        self.ctx.check(_lib.mh_net_get_params(self.ctx.h, self.h, out.ctypes.data_as(_p), ctypes.byref(gx),
                                              ctypes.byref(gy)))
        return out, gx.value, gy.value

    def set_params(self, params, gx: float = 1.0, gy: float = 1.0):
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        self.ctx.check(_lib.mh_net_set_params(self.ctx.h, self.h, a.ctypes.data_as(_p), float(gx), float(gy)))

    def sample(self, prob: "Problem", sigma_prev, sigma_next, x_out, y_out) -> float:
        rn = _d()
        self.ctx.check(_lib.mh_net_sample(self.ctx.h, prob.h, self.h, _ptr(sigma_prev), _ptr(sigma_next),
                                          _ptr4(x_out), _ptr4(y_out), ctypes.byref(rn)))
        return rn.value

    def fit(self, X, Y, omega, eps: float = 1e-3, power_iters: int = 2, ridge: float = 1e-12):
        self.ctx.check(_lib.mh_net_fit(self.ctx.h, self.h, _ptr4(X), _ptr4(Y), int(X.shape[0]), _ptr4(omega),
                                       float(eps), int(power_iters), float(ridge)))

    def loss_grad(self, X, T, grad_out=None) -> float:
        loss = _d()
        self.ctx.check(_lib.mh_net_loss_grad(self.ctx.h, self.h, _ptr4(X), _ptr4(T), int(X.shape[0]),
                                             ctypes.byref(loss), _ptr4(grad_out)))
        return loss.value

    def forward(self, X, Y_out, arith: int = MH_NET_FP32, training_kernels: bool = True):
        self.ctx.check(_lib.mh_net_forward(self.ctx.h, self.h, _ptr4(X), int(X.shape[0]), _ptr4(Y_out), int(arith),
                                           1 if training_kernels else 0))
        return Y_out

    def train(self, X, Y, batch_idx, lr: float, Xv, Yv, eval_every: int = 100):
        """Adam over the minibatches batch_idx (steps x batch int32); returns (first, best, best_step)."""
        first, best, step = _d(), _d(), _i()
        steps, batch = int(batch_idx.shape[0]), int(batch_idx.shape[1])
        self.ctx.check(_lib.mh_net_train(self.ctx.h, self.h, _ptr4(X), _ptr4(Y), int(X.shape[0]), _ptr4(batch_idx),
                                         steps, batch, float(lr), _ptr4(Xv), _ptr4(Yv), int(Xv.shape[0]),
                                         int(eval_every), ctypes.byref(first), ctypes.byref(best),
                                         ctypes.byref(step)))
        return first.value, best.value, step.value

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mh_net_destroy(self.h)
            self.h = None


def mh_warm_start(ctx: Context, bnd: Boundary, alpha: float, mode: int, sigma, rhs, x0_out, r0_out, net=None,
                  arith: int = MH_NET_BF16X2, sigma_prev2=None, prec: int = MH_PREC_FP64) -> float:
    c = _d()
    ctx.check(_lib.mh_warm_start(ctx.h, bnd.h, float(alpha), net.h if net is not None else None, int(mode), int(arith),
                                 _ptr(sigma), _ptr(sigma_prev2), _ptr(rhs), _ptr(x0_out), _ptr(r0_out), int(prec),
                                 ctypes.byref(c)))
    return c.value


def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


class Batch:
    """mh_batch_create: independent problems stepped together, one CUDA graph launch per step."""

    def __init__(self, ctx: Context, problems):
        self.ctx, self.problems = ctx, list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        h = _p()
        ctx.check(_lib.mh_batch_create(ctx.h, len(self.problems), ctypes.cast(arr, _p), ctypes.byref(h)))
        self.h = h

    def step(self, u, F, f_next, sigma, gmres_tol: float = 1e-10, prec: int = MH_PREC_MIXED):
        """One in-place IMEX Euler step of every problem; lists of device tensors."""
        for group in (u, F, f_next, sigma):
            for t in group:
                _ptr(t)
        n = len(self.problems)
        infos = (StepInfo * n)()
        self.ctx.check(_lib.mh_batch_step(self.ctx.h, self.h, ctypes.cast(_ptr_array(u), _p),
                                          ctypes.cast(_ptr_array(F), _p), ctypes.cast(_ptr_array(f_next), _p),
                                          ctypes.cast(_ptr_array(sigma), _p), float(gmres_tol), int(prec),
                                          ctypes.cast(infos, _p)))
        return list(infos)

    @property
    def graph_kernels(self) -> int:
        return int(_lib.mh_batch_graph_kernels(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mh_batch_destroy(self.h)
            self.h = None


def mh_autotune(ctx: Context, tree: Tree, bnd: Boundary, dt: float, F, f, p_cand=(10, 16, 24), err_tol: float = 1e-7,
                steps: int = 4, prec: int = MH_PREC_MIXED, ext_const=None):
    """Multipole order and near-field tile for one geometry and alpha (see include/mh.h).
    Returns (p, tile, report list of TuneEntry)."""
    pc = (ctypes.c_int * len(p_cand))(*p_cand)
    ec = np.ascontiguousarray(ext_const if ext_const is not None else np.zeros(bnd.n_curves), dtype=np.float64)
    rep = (TuneEntry * (len(p_cand) + 3))()
    p_out, t_out = _i(), _i()
    ctx.check(_lib.mh_autotune(ctx.h, tree.h, bnd.h, float(dt), MH_EXT_CONST, ec.ctypes.data_as(_p), _ptr(F), _ptr(f),
                               len(p_cand), ctypes.cast(pc, _p), float(err_tol), int(steps), int(prec),
                               ctypes.byref(p_out), ctypes.byref(t_out), ctypes.cast(rep, _p)))
    return p_out.value, t_out.value, list(rep)


def device_alloc_calls() -> int:
    """cudaMalloc plus cudaFree calls the library has made so far (all contexts)."""
    return int(_lib.mh_device_alloc_calls())


def library_path() -> str:
    return _LIB_PATH
