/*
 * mh.h -- C ABI of libmh, a GB300 (sm_103a) implementation of the per-time-step
 * modified-Helmholtz solve of Kropinski & Quaife, "Fast integral equation methods
 * for the heat equation and the modified Helmholtz equation in two dimensions".
 *
 * The heat equation u_t - Lap u = F is discretised in time first (Section 2):
 * each IMEX Euler step solves u - alpha^2 Lap u = B, alpha^2 = dt,
 * B = u^N + dt F^N, with u = f on Gamma.  The solution is U = U^p + U^h:
 *   U^p  volume potential of the extended B over the leaves of a quadtree
 *        (Section 3.1, eq. volume_potential),   kernel G = K0(r/alpha)/(2 pi alpha^2);
 *   U^h  double-layer potential (Section 2) whose density solves the second-kind
 *        integral equation (Section 2, eq. dirichlet:inteqn), discretised by the
 *        Alpert-corrected trapezoid rule (Section 3.2, eq. discrete_sys) and solved
 *        by GMRES (Section 3.2).
 *
 * Conventions (all entry points):
 *   - Every function returns an mh_status; mh_last_error(ctx) gives a message.
 *     No call aborts, traps or exits the process.
 *   - "_dev" pointers are device pointers on the context's device, "_host"
 *     pointers are host pointers.  All array arguments are owned by the caller
 *     and are only read or written during the call (asynchronously on the
 *     context's stream for device arrays; host arrays are done when the call
 *     returns).  Opaque objects (mh_ctx, mh_boundary, mh_tree, mh_problem)
 *     own their device memory and free it in the matching *_destroy.
 *   - Doubles are IEEE binary64.  Point arrays are interleaved (x, y) pairs.
 *   - Boundary curves: curve 0 is the outer boundary Gamma_0 (counter-clockwise),
 *     curves 1.. are holes (clockwise); curve k is sampled at N_k (even) equispaced
 *     parameter values t_n = 2 pi n / N_k (Section 3.2).  The right-hand normal
 *     (y2', -y1')/|y'| is then the outward normal of Omega.
 *   - Volume nodes: each leaf carries q x q Gauss-Legendre nodes, node j = iy*q + ix,
 *     leaves in Morton order of their lower-left corner (leaf-major node arrays).
 */
#ifndef MH_H
#define MH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MH_OK = 0,
    MH_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported option */
    MH_ERR_GEOMETRY = 2,      /* wrong curve orientation, odd node count, points off the tree */
    MH_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has the CUDA error string) */
    MH_ERR_OOM = 4,           /* device allocation failed */
    MH_ERR_NOT_CONVERGED = 5, /* GMRES hit max_iter before the tolerance */
    MH_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    MH_ERR_NUMERIC = 7,       /* non-finite value detected */
    MH_ERR_CALLBACK = 8       /* the user field callback returned non-zero */
} mh_status;

typedef enum {
    MH_PREC_FP64 = 0,   /* every step in binary64 */
    MH_PREC_MIXED = 1   /* binary32 inner products/contractions, binary64 Krylov
                           orthogonalisation, residuals and refinement */
} mh_precision;

typedef struct mh_ctx mh_ctx;
typedef struct mh_boundary mh_boundary;
typedef struct mh_tree mh_tree;
typedef struct mh_problem mh_problem;

typedef struct {
    int iterations;        /* total Krylov iterations (all refinement sweeps) */
    int refinements;       /* FP64 refinement sweeps (mixed precision), else 0 */
    double rel_residual;   /* final ||b - A x|| / ||b|| computed in binary64 */
    int converged;         /* 1 if rel_residual <= tol */
    double initial_rel_residual;   /* ||b - A x0|| / ||b|| of the initial guess */
} mh_gmres_info;

typedef struct {
    int gmres_iterations;
    double gmres_rel_residual;
    double initial_rel_residual;   /* of the GMRES start chosen by the warm-start mode */
    double warm_c;                 /* step length of the SECANT / LEARNED start (0 otherwise) */
} mh_step_info;

/* Field callback used by mh_tree_build: evaluate the user's F at n points
 * xy_host[2n] (host memory) into out_host[n]; return 0 on success. */
typedef int (*mh_field_fn)(const double* xy_host, int64_t n, double* out_host, void* user);

/* ---- context --------------------------------------------------------------------- */

/* Create a context on CUDA device `device`, issuing all work on `stream`
 * (a cudaStream_t, NULL = the legacy default stream). */
mh_status mh_create(int device, void* stream, mh_ctx** out);
mh_status mh_destroy(mh_ctx* ctx);
/* Message describing the last error on ctx (valid until the next call on ctx). */
const char* mh_last_error(const mh_ctx* ctx);
/* Number of kernels this context has launched so far (for launch accounting). */
int64_t mh_kernel_launches(const mh_ctx* ctx);
/* Number of device allocations plus frees (cudaMalloc / cudaFree) the library has made so far,
 * over all contexts of the process (library instrumentation: a call that allocates nothing
 * leaves it unchanged). */
int64_t mh_device_alloc_calls(void);

/* Timing of named kernel regions (library instrumentation, no counterpart in the paper).
 * When enabled, the library records a CUDA event pair on its stream around each launch
 * of the instrumented kernels -- "dlp_coarse", "dlp_fine", "dlp_fmm", "dlp_fmm_contract",
 * "bie_gemv", "volume_apply", "volume_contract", "gmres", "dlp_evaluate" -- together with
 * the algorithmic work each launch declares (flops; bytes that must move at least once).
 * mh_profile_read synchronises the stream and returns, for `region`, the summed event time
 * (ms), the number of timed launches and the summed flops and bytes since the last reset;
 * any output pointer may be NULL; reset != 0 clears all regions afterwards. */
mh_status mh_profile_enable(mh_ctx* ctx, int on);
mh_status mh_profile_read(mh_ctx* ctx, const char* region, double* total_ms, int64_t* launches, double* flops,
                          double* bytes, int reset);

/* Engine of the binary32 batched contractions of the multipole passes (near-field tables,
 * P2M, M2L, P2L, L2P, M2P: Section 3.1) in MH_PREC_MIXED: on != 0 (default) forms the operators
 * with enough tasks as TF32 head/tail matrix products on the tensor cores (three MMAs per K step,
 * binary32 accumulation); 0 keeps every contraction on the CUDA cores.  Binary64 work is not
 * affected.  Takes effect for work issued after the call (a batch graph recorded earlier keeps
 * the form it was recorded with). */
mh_status mh_set_tensor_cores(mh_ctx* ctx, int on);

/* ---- boundary (Section 3.2) -------------------------------------------------------- */

/* Build the boundary from node coordinates xy_host[2 N_Gamma] (curves concatenated,
 * n_nodes_host[k] = N_k, each even and >= 2*alpert_order + 2).  y', y'' at the nodes
 * are computed pseudospectrally (Section 3.2).  alpert_order in 1..10 selects the
 * l-point log-singular correction (window a = l); 0 selects the plain trapezoid rule
 * with the diagonal limit -kappa/2 of d/dnu K0 (Section 2).
 * Errors: MH_ERR_GEOMETRY if the outer curve is not counter-clockwise or a hole is
 * not clockwise, MH_ERR_INVALID_ARG for bad sizes. */
mh_status mh_boundary_create(mh_ctx* ctx, int n_curves, const int32_t* n_nodes_host,
                             const double* xy_host, int alpert_order, mh_boundary** out);
mh_status mh_boundary_destroy(mh_boundary* bnd);
mh_status mh_boundary_size(const mh_boundary* bnd, int64_t* n_gamma);
/* Per node: x, y, x', y', x'', y'', |y'|, K(x,x) diagonal limit (8 doubles per node). */
mh_status mh_boundary_geometry(mh_ctx* ctx, const mh_boundary* bnd, double* out_host);

/* ---- quadtree (Section 3.1) --------------------------------------------------------- */

/* Build the quadtree on D = [box[0], box[0]+box[2]] x [box[1], box[1]+box[2]] on the
 * device: leaves are split level by level while level < min_level or, if refine_fn is
 * not NULL, while max over the four children's nodes of |F - P_b F| > refine_tol
 * (P_b F = q x q tensor interpolant of F on the box's own nodes, Section 3.1); then
 * the tree is 2:1 balanced (touching leaves differ by at most one level) and the
 * U, V, W, X interaction lists are formed.  q in 2..16, 0 <= min_level <= max_level <= 10. */
mh_status mh_tree_build(mh_ctx* ctx, const double* box3_host, int q, int min_level, int max_level,
                        mh_field_fn refine_fn, void* user, double refine_tol, mh_tree** out);
mh_status mh_tree_destroy(mh_tree* tree);
mh_status mh_tree_size(const mh_tree* tree, int64_t* n_leaves, int64_t* n_boxes, int64_t* n_nodes);
/* Leaves (level, ix, iy) in node order, 3 int32 each. */
mh_status mh_tree_leaves(mh_ctx* ctx, const mh_tree* tree, int32_t* out_host);
/* All boxes (level, ix, iy) ordered by level then Morton key, 3 int32 each. */
mh_status mh_tree_boxes(mh_ctx* ctx, const mh_tree* tree, int32_t* out_host);
/* Volume node coordinates, 2 doubles per node, into device memory. */
mh_status mh_tree_nodes(mh_ctx* ctx, const mh_tree* tree, double* out_dev);
/* Synchronise the context stream and report whether a bounded device wait of the tree's
 * tensor-core contractions gave up since the last check (MH_ERR_TIMEOUT; the results of that
 * work are not valid); MH_OK otherwise.  mh_volume_potential performs this check itself. */
mh_status mh_tree_check(mh_ctx* ctx, mh_tree* tree);
/* Interaction list `which` (0 = U, 1 = V, 2 = W, 3 = X) in CSR form over all boxes
 * (box ids as in mh_tree_boxes): offsets_host[n_boxes + 1]; items_host may be NULL to
 * query offsets only.  Item lists are sorted by box id. */
mh_status mh_tree_list(mh_ctx* ctx, const mh_tree* tree, int which, int32_t* offsets_host,
                       int32_t* items_host);

/* ---- volume potential (Section 3.1) ------------------------------------------------ */

/* up_dev[i] = sum over leaves of int_leaf G(x_i - y) P(y) dA at every volume node x_i,
 * P = the leaf's q x q interpolant of b_dev (eq. volume_potential with the leaf
 * polynomial of Section 3.1), evaluated by near-field tables on adjacent leaves and a
 * multipole method of order p (K_n multipoles, I_n locals) for the rest.
 * b_dev, up_dev: n_nodes doubles (device).  p in 1..40. */
mh_status mh_volume_potential(mh_ctx* ctx, mh_tree* tree, double alpha, int p, const double* b_dev,
                              double* up_dev, mh_precision prec);

/* ---- double layer and BIE (Section 2 and 3.2) --------------------------------------- */

/* targets_dev == NULL: out_dev = A sigma, the discretised operator of
 *   eq. discrete_sys (sigma + (1/pi) Q[K sigma], K(y,x) = (1/alpha) K1(|y-x|/alpha)
 *   (y-x).n_y/|y-x|), n_targets ignored, out has N_Gamma entries.
 * targets_dev != NULL: out_dev[i] = U^h(x_i) = (1/(2 pi alpha^2)) int d/dnu_y K0 sigma ds
 *   at n_targets points (2 doubles each) assumed inside Omega, with the near-boundary
 *   rule: 16x upsampled density for targets within 10 h_s of a curve, interpolation
 *   along the normal within h_s/4.  n_targets == 0 evaluates nothing (out_dev untouched);
 *   n_targets < 0 is MH_ERR_INVALID_ARG.
 * A boundary switched to the matrix-free operator (mh_problem_matrix_free) forms A sigma that
 * way, in binary64 whatever prec says; alpha must then be the problem's (else
 * MH_ERR_INVALID_ARG). */
mh_status mh_double_layer_apply(mh_ctx* ctx, mh_boundary* bnd, double alpha, const double* sigma_dev,
                                const double* targets_dev, int64_t n_targets, double* out_dev,
                                mh_precision prec);

/* Solve A sigma = rhs (eq. discrete_sys) by unrestarted GMRES (Section 3.2), stopping
 * when ||rhs - A sigma|| <= tol ||rhs|| (the paper uses tol = 1e-10, Section 4).
 * sigma_dev: in = initial guess, out = solution.  MH_PREC_MIXED runs binary32-operator
 * GMRES inside binary64 iterative refinement.  Returns MH_ERR_NOT_CONVERGED (with
 * sigma holding the best iterate) if max_iter iterations do not reach tol.  With the
 * matrix-free operator (mh_problem_matrix_free) only MH_PREC_FP64 is accepted. */
mh_status mh_gmres_solve(mh_ctx* ctx, mh_boundary* bnd, double alpha, const double* rhs_dev,
                         double* sigma_dev, double tol, int max_iter, mh_precision prec,
                         mh_gmres_info* info);

/* Allocation-free variant of mh_gmres_solve (the paper has no counterpart; it exists for
 * callers that cannot allocate device memory while they solve, e.g. code running under a
 * device-memory budget fixed in advance or inside a host loop whose allocator belongs to
 * another framework).  Binary64 only.  The Krylov workspace is a fixed array compiled into
 * the library (4.4 MB held on every device that loads it, until the process exits), so:
 *   - N_Gamma <= 8192 and 1 <= max_iter <= 64, else MH_ERR_INVALID_ARG;
 *   - the dense operator for `alpha` must already be assembled on bnd by an earlier
 *     mh_gmres_solve / mh_double_layer_apply / mh_problem_create call with the same alpha
 *     (a boundary on the matrix-free operator has none: MH_ERR_INVALID_ARG)
 *     (those allocate it), else MH_ERR_INVALID_ARG;
 *   - the first call on a device looks up the array's device address (done once per device,
 *     with that device current); make that first call before any stream capture;
 *   - the call does no cudaMalloc/cudaFree; every call shares the one array, so calls that
 *     overlap on the GPU (other streams, other host threads) race and must be serialised.
 * Arguments, stopping rule, info and errors are those of mh_gmres_solve. */
mh_status mh_gmres_solve_static(mh_ctx* ctx, mh_boundary* bnd, double alpha, const double* rhs_dev,
                                double* sigma_dev, double tol, int max_iter, mh_gmres_info* info);

/* ---- heat step (Section 2) ---------------------------------------------------------- */

typedef enum { MH_EXT_CONST = 0, MH_EXT_ARRAY = 1 } mh_ext_mode;
typedef enum {
    MH_SCHEME_IMEX_EULER = 0,    /* alpha^2 = dt,     B = u^N + dt F^N (Section 2) */
    MH_SCHEME_EXTRAP_GEAR = 1    /* alpha^2 = 2dt/3,  B = 4/3 u^N - 1/3 u^{N-1} + 4/3 dt F^N - 2/3 dt F^{N-1} */
} mh_scheme;

/* Bind a tree and a boundary into a time-stepping problem with step dt, time scheme
 * `scheme` (mh_scheme; fixes alpha^2 = dt or 2dt/3, Section 2) and multipole order p.  Volume nodes are classified (inside Omega or on
 * the exterior side of curve k) and the boundary nodes located in the leaves.
 * Exterior extension of B (Section 3.1): MH_EXT_CONST uses ext_const_host[k] + dt F
 * outside curve k (the paper's constant extension); MH_EXT_ARRAY takes the exterior
 * values from heat_step's b_ext_dev. */
mh_status mh_problem_create(mh_ctx* ctx, mh_tree* tree, mh_boundary* bnd, double dt, int scheme, int p,
                            int ext_mode, const double* ext_const_host, mh_problem** out);
mh_status mh_problem_destroy(mh_problem* prob);
/* Matrix-free boundary operator (Section 3.2: the discrete system evaluated by the multipole
 * method instead of a stored matrix).  enable = 1 switches every later product with the
 * problem's boundary operator (GMRES, residuals, mh_double_layer_apply without targets) to
 *     (A sigma)_j = sigma_j + (1/pi) [T_j - W_j] + C_j
 * with T_j the trapezoid sum over all other nodes by an on-surface pass of the problem's tree
 * (order p, binary64), W_j the own-curve terms inside the Alpert window (direct) and C_j the
 * Alpert correction, the trigonometric interpolant of sigma at the correction nodes taken by
 * chirp transforms per curve: O(N log N) work and O(N) memory instead of the O(N^2) matrix,
 * which is released.  Binary64 only: MH_PREC_MIXED solves and the graph form of the step
 * (mh_batch_step) then fail with MH_ERR_INVALID_ARG.  Needs an even node count per curve in
 * [max(2 l, 4), 4096] (else MH_ERR_INVALID_ARG) and every boundary node inside the tree.
 * enable = 0 returns to the dense operator (assembled again before the call returns).  The pass has its
 * own expansions and M2M/L2L chain (over the boxes that hold boundary nodes); it reads the
 * tree's translation operators, so it stops working (MH_ERR_INVALID_ARG) once the tree's volume
 * operators are rebuilt for another alpha or p.  mh_problem_destroy returns the boundary to the
 * dense operator. */
mh_status mh_problem_matrix_free(mh_ctx* ctx, mh_problem* prob, int enable);
/* Region of every volume node: -1 inside Omega, k on the exterior side of curve k. */
mh_status mh_problem_regions(mh_ctx* ctx, const mh_problem* prob, int32_t* region_host);
/* Right-hand side -2 alpha^2 (f_next - U^p|Gamma) of the boundary equation solved by the last
 * heat_step / heat_step_gear on this problem (Section 3.2): N_Gamma doubles copied on the
 * ctx stream into the caller's device buffer rhs_dev.  Zeros before the first step. */
mh_status mh_problem_rhs(mh_ctx* ctx, const mh_problem* prob, double* rhs_dev);

/* One IMEX Euler step u^N -> u^{N+1} (Section 2):
 *   B = u + dt F (inside), extension outside; U^p = volume potential of B;
 *   g = f_next - U^p on Gamma (leaf interpolation, Section 3.1); solve
 *   A sigma = -2 alpha^2 g (GMRES, tolerance gmres_tol); u_next = U^p + U^h inside
 *   Omega, = ext_const (CONST) or U^p (ARRAY) outside.
 * u_dev, F_dev, b_ext_dev, u_next_dev: n_nodes doubles; f_next_dev, sigma_dev: N_Gamma
 * doubles (sigma: in = warm start, out = density).  u_dev and u_next_dev may alias. */
mh_status heat_step(mh_ctx* ctx, mh_problem* prob, const double* u_dev, const double* F_dev,
                    const double* f_next_dev, const double* b_ext_dev, double* u_next_dev,
                    double* sigma_dev, double gmres_tol, mh_precision prec, mh_step_info* info);

/* One IMEX Euler step of the Allen-Cahn equation u_t - eps Lap u = u (1 - u^2) (Section 4,
 * Example 3), the reaction term explicit:
 *   u^{N+1} - eps dt Lap u^{N+1} = B = u^N + dt u^N (1 - (u^N)^2)   in Omega,
 * u^{N+1} = f_next on Gamma.  With time rescaled by eps this is heat_step with step eps dt and
 * forcing u (1 - u^2) / eps, so prob must be created with dt = eps * dt (MH_SCHEME_IMEX_EULER:
 * alpha^2 = eps dt); eps > 0 is passed here.  Outside Omega B is C_k + dt C_k (1 - C_k^2)
 * (MH_EXT_CONST, u = C_k there) or b_ext_dev (MH_EXT_ARRAY); the rest of the step, the
 * arguments and the error behaviour are those of heat_step.  u_dev and u_next_dev may alias. */
mh_status allen_cahn_step(mh_ctx* ctx, mh_problem* prob, double eps, const double* u_dev,
                          const double* f_next_dev, const double* b_ext_dev, double* u_next_dev,
                          double* sigma_dev, double gmres_tol, mh_precision prec, mh_step_info* info);

/* One extrapolated Gear step (Section 2) on a problem created with MH_SCHEME_EXTRAP_GEAR:
 * B = 4/3 u - 1/3 u_prev + dt (4/3 F - 2/3 F_prev) inside Omega, C_k + dt (4/3 F -
 * 2/3 F_prev) outside (MH_EXT_CONST) or b_ext_dev (MH_EXT_ARRAY); the rest as heat_step.
 * The scheme needs two past levels: start it with one step of another method or with
 * known data.  u_prev_dev, F_prev_dev: n_nodes doubles.  u_next_dev may alias u_dev
 * (not u_prev_dev). */
mh_status heat_step_gear(mh_ctx* ctx, mh_problem* prob, const double* u_dev, const double* u_prev_dev,
                         const double* F_dev, const double* F_prev_dev, const double* f_next_dev,
                         const double* b_ext_dev, double* u_next_dev, double* sigma_dev, double gmres_tol,
                         mh_precision prec, mh_step_info* info);

/* ------------------------------------------------------------------------------------------
 * Learned warm start of the boundary solve.
 *
 * The paper solves A sigma^{N+1} = b^{N+1} by GMRES to relative residual 1e-10 at every
 * step (Section 3.2, Section 4) and states no initial guess.  These calls choose one.
 * With r = b - A sigma^N, the residual of the previous-step start, a network predicts the
 * correction delta ~ A^{-1} r:
 *   features  x = F(r) / (|r| g_x): F = the Fourier coefficients
 *             c_k = (1/N_k) sum_j v_j exp(-2 pi i j k / N_k), k = 0 .. n_modes-1, of every
 *             curve, curve-major as [Re c_0, Im c_0, Re c_1, Im c_1, ...]; d = n_curves *
 *             2 n_modes features;
 *   network   y = W4 t(W3 t(W2 t(W1 x + b1) + b2) + b3) + b4, t = tanh, width w;
 *   output    delta = r + |r| g_y S(y), S = Fourier synthesis
 *             v_j = Re c_0 + 2 sum_{k>=1} Re(c_k exp(2 pi i j k / N_k));
 *   judge     w = A delta, c = <r, w> / <w, w> (0 when <w, w> = 0 or c is not finite);
 *             x0 = sigma^N + c delta and r0 = r - c w: the minimum residual on the line
 *             through sigma^N, never above the previous-step start (c = 0).
 * Parameters are binary32 in one flat array: W1 [w][d], b1 [w], W2 [w][w], b2 [w],
 * W3 [w][w], b3 [w], W4 [d][w], b4 [d] (row-major, W[out][in]).
 * ---------------------------------------------------------------------------------------- */
typedef struct mh_net mh_net;

typedef enum {
    MH_NET_FP32 = 0,    /* binary32 weights */
    MH_NET_BF16 = 1,    /* bfloat16 weights (round to nearest even) */
    MH_NET_BF16X2 = 2   /* bfloat16 pair hi + lo, lo = bf16(w - hi) */
} mh_net_arith;         /* inference weights; activations and sums are binary32 in all three */

typedef enum {
    MH_WARM_PREVIOUS = 0,   /* x0 = sigma^N (default) */
    MH_WARM_ZERO = 1,       /* x0 = 0 */
    MH_WARM_SECANT = 2,     /* judge along sigma^N - sigma^{N-1} (no network) */
    MH_WARM_LEARNED = 3     /* judge along the network's delta */
} mh_warm_mode;

/* Network for the boundary of bnd.  n_modes: multiple of 4, at most N_k / 2 on every curve;
 * width: multiple of 8 in 8..1024.  Parameters start at zero, g_x = g_y = 1. */
mh_status mh_net_create(mh_ctx* ctx, const mh_boundary* bnd, int n_modes, int width, mh_net** out);
mh_status mh_net_destroy(mh_net* net);
mh_status mh_net_dims(const mh_net* net, int64_t* d, int64_t* width, int64_t* n_params);
/* Copy the parameters (n_params floats) and the scales g_x, g_y out of / into the network. */
mh_status mh_net_get_params(mh_ctx* ctx, const mh_net* net, float* params_host, double* gx_host, double* gy_host);
mh_status mh_net_set_params(mh_ctx* ctx, mh_net* net, const float* params_host, double gx, double gy);

/* One training pair from the last step solved on prob: r = rhs - A sigma_prev (binary64,
 * the operator of the problem's boundary and alpha, rhs of mh_problem_rhs),
 * x = F(r)/|r|, y = F(sigma_next - sigma_prev - r)/|r| into x_dev, y_dev (d floats each,
 * not divided by g_x, g_y); r_norm_host (nullable): |r|.  |r| = 0 gives zero rows. */
mh_status mh_net_sample(mh_ctx* ctx, mh_problem* prob, mh_net* net, const double* sigma_prev_dev,
                        const double* sigma_next_dev, float* x_dev, float* y_dev, double* r_norm_host);

/* Closed-form start of training on n >= 2 pairs (X_dev, Y_dev: n x d rows from
 * mh_net_sample).  g_x, g_y = RMS entries of X, Y; on X/g_x, Y/g_y (binary64):
 *   mu = mean row, Xc = X - mu; Q = orth(Xc^T omega), then power_iters times
 *   Q = orth(Xc^T (Xc Q)), orth = the Q factor whose R has a positive diagonal;
 *   s = RMS of the columns of Xc Q floored at 1e-8 max s; W1 = eps diag(1/s) Q^T,
 *   b1 = -W1 mu; W2 = W3 = I, b2 = b3 = 0; [W4 | b4] = ridge least squares
 *   (Ha^T Ha + lam I) Z = Ha^T Y on Ha = [H, 1], H the third hidden layer on X,
 *   lam = ridge trace(Ha^T Ha)/(w + 1).
 * omega_dev: n x w binary32 (Gaussian draws supplied by the caller).
 * MH_ERR_NUMERIC when an orthogonalisation or the least-squares system is singular. */
mh_status mh_net_fit(mh_ctx* ctx, mh_net* net, const float* X_dev, const float* Y_dev, int64_t n,
                     const float* omega_dev, double eps, int power_iters, double ridge);

/* Loss L = (1/(2 n d)) sum (net(X) - T)^2 on network-unit inputs X and targets T (n x d,
 * already divided by g_x and g_y) and its gradient (n_params floats, parameter layout)
 * by the binary32 training kernels. */
mh_status mh_net_loss_grad(mh_ctx* ctx, mh_net* net, const float* X_dev, const float* T_dev, int64_t n,
                           double* loss_host, float* grad_dev);

/* Network outputs Y_dev (n x d) for network-unit inputs X_dev (n x d): the binary32
 * training kernels when training_kernels != 0 (arith ignored), else the inference kernels
 * with weights in arith. */
mh_status mh_net_forward(mh_ctx* ctx, mh_net* net, const float* X_dev, int64_t n, float* Y_dev,
                         mh_net_arith arith, int training_kernels);

/* Adam (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on L over `steps` minibatches;
 * batch_idx_dev: steps x batch row indices into X_dev, Y_dev (pairs from mh_net_sample,
 * divided by g_x, g_y inside).  Every eval_every steps and after the last, L on the
 * validation pairs Xv_dev, Yv_dev (n_val rows) is computed; the parameters with the lowest
 * validation loss (the starting ones included) are kept.  first_val_host, best_val_host,
 * best_step_host (nullable): validation loss at the start, the best loss and its step. */
mh_status mh_net_train(mh_ctx* ctx, mh_net* net, const float* X_dev, const float* Y_dev, int64_t n,
                       const int32_t* batch_idx_dev, int steps, int batch, double lr, const float* Xv_dev,
                       const float* Yv_dev, int64_t n_val, int eval_every, double* first_val_host,
                       double* best_val_host, int* best_step_host);

/* Initial guess for A x = rhs on bnd at screening length alpha (the operator is assembled
 * if needed).  r = rhs - A sigma in binary64; the judge's w = A delta in precision prec.
 * PREVIOUS: x0 = sigma; ZERO: x0 = 0; SECANT: direction sigma - sigma_prev2 (sigma_prev2_dev
 * required); LEARNED: the network's delta with weights in arith (net required).
 * x0_dev (may alias sigma_dev) and r0_dev (= rhs - A x0): N_Gamma doubles.
 * c_host (nullable): the step length. */
mh_status mh_warm_start(mh_ctx* ctx, mh_boundary* bnd, double alpha, mh_net* net, mh_warm_mode mode,
                        mh_net_arith arith, const double* sigma_dev, const double* sigma_prev2_dev,
                        const double* rhs_dev, double* x0_dev, double* r0_dev, mh_precision prec,
                        double* c_host);

/* Warm-start mode of heat_step / heat_step_gear on prob (default MH_WARM_PREVIOUS).  SECANT
 * keeps a copy of the incoming density of every step; its first step uses PREVIOUS.  The
 * network stays owned by the caller and must outlive its use. */
mh_status mh_problem_set_warm_start(mh_ctx* ctx, mh_problem* prob, mh_warm_mode mode, mh_net* net,
                                    mh_net_arith arith);

/* ------------------------------------------------------------------------------------------
 * Batched stepping and autotuning of independent problems.
 *
 * A batch holds n problems (each with its own tree, boundary and, if used, network).
 * mh_batch_step advances all of them by one IMEX Euler step (Section 2) as one CUDA graph
 * launch: the first call runs the step eagerly and records the graph (one branch per problem on
 * its own stream, GMRES with a fixed schedule of device-gated kernels instead of host
 * read-backs: mixed precision 3 binary64 refinement sweeps x 20 Arnoldi iterations, binary64 40
 * iterations); later calls with the same arrays, tolerance and precision relaunch the graph
 * (a problem's GMRES workspace grown, or its boundary operator assembled again or released,
 * since the recording makes the call record anew).  A problem on the matrix-free boundary
 * operator (mh_problem_matrix_free) is refused with MH_ERR_INVALID_ARG.
 * The step is in place: u_dev[i] is u^N on entry and u^{N+1} on return.  One host
 * synchronisation per call reads the per-problem GMRES results into info_host[i].
 * MH_ERR_NOT_CONVERGED if a problem did not reach gmres_tol within the schedule (its u is the
 * last iterate's).
 * ---------------------------------------------------------------------------------------- */
typedef struct mh_batch mh_batch;

mh_status mh_batch_create(mh_ctx* ctx, int n, mh_problem* const* probs_host, mh_batch** out);
mh_status mh_batch_destroy(mh_batch* batch);
/* All pointer arrays are host arrays of n device pointers (N_D or N_Gamma doubles as in
 * heat_step); b_ext is not supported (problems must use MH_EXT_CONST). */
mh_status mh_batch_step(mh_ctx* ctx, mh_batch* batch, double* const* u_dev, const double* const* F_dev,
                        const double* const* f_next_dev, double* const* sigma_dev, double gmres_tol,
                        mh_precision prec, mh_step_info* info_host);
/* Kernels launched by one graph launch of the batch (0 before the graph exists). */
int64_t mh_batch_graph_kernels(const mh_batch* batch);

/* Threads per block of the binary32 near-field double-layer kernel of prob's tree
 * (128, 256 or 512; default 256): the tile of qq targets x threads/qq source groups. */
mh_status mh_problem_set_near_tile(mh_ctx* ctx, mh_problem* prob, int threads);

typedef struct {
    int p;              /* multipole order */
    int near_tile;      /* threads per block of the near-field kernel */
    double rel_err;     /* relative L2 difference of u (nodes inside Omega) from the reference order */
    double ms_per_step; /* median step time (CUDA events) */
} mh_tune_entry;

/* Autotuner of the multipole order and the near-field tile for one geometry and alpha.
 * For every candidate p_cand[i] and the reference order p_ref = max(p_cand) + 8 it creates a
 * problem on (tree, bnd, dt, IMEX Euler, ext_mode / ext_const_host), runs `steps` steps from
 * u = 0 with forcing F_dev and boundary data f_dev (both fixed in time), precision prec and the
 * previous-step GMRES start, and records the relative L2 difference of u^steps from the
 * reference run over the nodes inside Omega and the median step time.  The chosen p is the
 * fastest candidate with rel_err <= err_tol (else the most accurate); for it the near-field tile
 * in {128, 256, 512} with the fastest step is chosen.  report_host (nullable) receives
 * n_p + 3 entries: the candidates, then the chosen p with each tile.  The tree keeps the
 * operators of the last problem built. */
mh_status mh_autotune(mh_ctx* ctx, mh_tree* tree, mh_boundary* bnd, double dt, int ext_mode,
                      const double* ext_const_host, const double* F_dev, const double* f_dev, int n_p,
                      const int* p_cand, double err_tol, int steps, mh_precision prec, int* p_out,
                      int* tile_out, mh_tune_entry* report_host);

#ifdef __cplusplus
}
#endif

#endif /* MH_H */
