// Internal declarations shared by the libmh translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/mh.h"

#define MH_PI 3.14159265358979323846

// Named timing region: CUDA events recorded on the context stream around each launch.
struct prof_region {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double total_ms = 0.0;
    int64_t launches = 0;
    double flops = 0.0, bytes = 0.0;   // algorithmic work of the timed launches
};

struct mh_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;
    bool profiling = false;
    bool capturing = false;   // inside a batch step: no cooperative launches
    bool tensor_cores = true; // binary32 contractions on the tensor cores (mh_set_tensor_cores)
    int64_t loop_nodes = 0;   // graph WHILE nodes recorded (their body kernels: loop_kernels each)
    std::map<std::string, prof_region> prof;
    ~mh_ctx();
};

// RAII scope: records a start/stop event pair on ctx->stream under `name` when
// profiling is enabled (mh_profile_enable), nothing otherwise.
struct prof_scope {
    mh_ctx* ctx;
    std::string name;
    double flops, bytes;
    cudaEvent_t a = nullptr, b = nullptr;
    prof_scope(mh_ctx* c, const char* n, double flops_ = 0.0, double bytes_ = 0.0);
    ~prof_scope();
};

// Records a message on ctx and returns the status.
mh_status mh_fail(mh_ctx* ctx, mh_status st, const char* fmt, ...);

#define MH_CUDA(ctx, call)                                                                      \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return mh_fail((ctx), e_ == cudaErrorMemoryAllocation ? MH_ERR_OOM : MH_ERR_CUDA,  \
                           "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,    \
                           __LINE__);                                                           \
    } while (0)

#define MH_LAUNCHED(ctx)                                                                        \
    do {                                                                                        \
        (ctx)->launches++;                                                                      \
        cudaError_t e_ = cudaGetLastError();                                                    \
        if (e_ != cudaSuccess)                                                                  \
            return mh_fail((ctx), MH_ERR_CUDA, "kernel launch failed: %s (%s:%d)",              \
                           cudaGetErrorString(e_), __FILE__, __LINE__);                         \
    } while (0)

#define MH_TRY(expr)                                                                            \
    do {                                                                                        \
        mh_status s_ = (expr);                                                                  \
        if (s_ != MH_OK) return s_;                                                             \
    } while (0)

// Number of device allocations and frees made by the library (every one goes through dbuf),
// read by mh_device_alloc_calls.
extern std::atomic<int64_t> g_mh_alloc_calls;

// Device buffer with RAII free.
template <class T>
struct dbuf {
    T* p = nullptr;
    size_t n = 0;
    dbuf() = default;
    dbuf(const dbuf&) = delete;
    dbuf& operator=(const dbuf&) = delete;
    ~dbuf() { release(); }
    void release() {
        if (p) {
            g_mh_alloc_calls.fetch_add(1, std::memory_order_relaxed);
            cudaFree(p);
        }
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t count) {
        release();
        n = count;
        if (count == 0) return cudaSuccess;
        g_mh_alloc_calls.fetch_add(1, std::memory_order_relaxed);
        return cudaMalloc((void**)&p, count * sizeof(T));
    }
};

#define MH_ALLOC(ctx, buf, count) MH_CUDA(ctx, (buf).alloc(count))

// A second stream with fork / join events, for work that does not depend on what the context
// stream runs meanwhile: the multipole passes (latency chains, on a stream of the device's
// highest priority, so that their blocks start before queued near-field blocks) beside the
// near fields; the sums at the normal-line auxiliary points beside the double layer's
// multipole pass.  Created at set-up, outside any stream capture.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    SideStream() = default;
    SideStream(const SideStream&) = delete;
    SideStream& operator=(const SideStream&) = delete;
    ~SideStream() {
        if (join) cudaEventDestroy(join);
        if (fork) cudaEventDestroy(fork);
        if (s) cudaStreamDestroy(s);
    }
    mh_status create(mh_ctx* ctx, bool high_priority = true) {
        int least = 0, greatest = 0;
        MH_CUDA(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        MH_CUDA(ctx, cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, high_priority ? greatest : least));
        MH_CUDA(ctx, cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        MH_CUDA(ctx, cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        return MH_OK;
    }
    // the side stream waits for everything issued so far on `main`
    mh_status begin(mh_ctx* ctx, cudaStream_t main) {
        MH_CUDA(ctx, cudaEventRecord(fork, main));
        MH_CUDA(ctx, cudaStreamWaitEvent(s, fork, 0));
        return MH_OK;
    }
    mh_status end(mh_ctx* ctx) {
        MH_CUDA(ctx, cudaEventRecord(join, s));
        return MH_OK;
    }
};

// Tensor-core batched contraction (contract_tc.cu): one launch over chunks of up to 128 tasks of
// one operator each; products to temp[task][R] or, with task_dst, straight to the destinations.
struct tc_launch {
    const uint16_t* img = nullptr;       // operator images (three bfloat16 parts) in the tensor-core layout
    const int64_t* img_off = nullptr;    // per operator: offset of its image (bfloat16 elements)
    const int32_t* kpad = nullptr;       // per operator: columns rounded up to 16
    const int32_t* op_C = nullptr;       // per operator: columns
    const int32_t* chunk_op = nullptr;
    const int32_t* chunk_t0 = nullptr;   // n_chunks + 1 entries
    int64_t n_chunks = 0;
    const uint16_t* spl = nullptr;       // pre-split sources: three bfloat16 planes
    int64_t plane = 0;                   // elements per plane
    const int64_t* tc_src = nullptr;     // per task: offset of its source row in a plane
    int R = 0, npad = 0, kmax = 0;
    float* temp = nullptr;
    const int64_t* task_dst = nullptr;
    int accumulate = 0;
    void* dst = nullptr;
    bool dst_double = false;
    int* err = nullptr;                  // set when a bounded wait gave up
};
int tc_pad_rows(int R);
int tc_pad_cols(int C);
void tc_operator_image(const double* op, int R, int C, int npad, int kpad, uint16_t* out);
mh_status tc_prepare(mh_ctx* ctx);
mh_status tc_contract_launch(mh_ctx* ctx, const tc_launch& a);
// Split count binary32 vectors of length len at src into the three bfloat16 planes at dst
// (rows padded with zeros to S entries).
mh_status tc_split_launch(mh_ctx* ctx, const float* src, int len, int64_t count, int S, uint16_t* planes, int64_t plane,
                          int64_t dst);

// Device-resident state of the sync-free GMRES (gmres_run_graph): every kernel of its fixed
// schedule reads the flags at entry and returns at once when its work is not needed.
constexpr int GMRES_LOOP_KERNELS = 5;   // kernels in the body of a graph Arnoldi loop

struct gmres_dev {
    double bnorm, rn, target, rel, init_rel;
    int done;        // converged on a binary64 residual computed in this solve
    int skip;        // done, or the Arnoldi process of the current sweep has ended
    int k;           // Arnoldi iterations of the current sweep
    int total;       // all Arnoldi iterations
    int sweeps;      // sweeps started (refinement passes in mixed precision)
    int converged;
    int arrive;      // blocks of the running Arnoldi normalisation that have finished (reset by the last)
};

// GMRES workspace (kept by the boundary so that repeated solves allocate nothing).
struct gmres_ws {
    dbuf<double> V, H, cs, sn, g, y, h1, h2, small, w, r, dx;
    dbuf<double> P1, P2, Pn;             // per-slice partial dot products / squared norms
    dbuf<float> v32;                     // binary32 copy of the newest Krylov vector
    cudaStream_t body_stream = nullptr;  // captures the body of a graph loop (batch graphs)
    int m = 0;
    int64_t n = 0;
    int64_t gen = 0;                     // bumped whenever the buffers are reallocated (recorded graphs hold them)
    gmres_ws() = default;
    gmres_ws(const gmres_ws&) = delete;
    gmres_ws& operator=(const gmres_ws&) = delete;
    ~gmres_ws() {
        if (body_stream) cudaStreamDestroy(body_stream);
    }
};

// Assembled boundary operator for one alpha (eq. discrete_sys), row-major N x N.
struct bie_operator {
    double alpha = -1.0;
    int64_t gen = 0;     // bumped whenever a form below is allocated or released (recorded graphs hold them)
    dbuf<double> A64;
    dbuf<float> A32;
    dbuf<float> A32lo;   // A64 - A32 rounded to binary32: A32 + A32lo carries A64 to ~2^-48
    // (A64 - A32) 2^24 rounded to binary16 (bit patterns), used instead of A32lo when N is a
    // multiple of 8: A32 + 2^-24 A16lo carries A64 to 2^-35 |A| + 2^-49
    dbuf<uint16_t> A16lo;
};

struct mh_boundary {
    int n_curves = 0;
    int64_t n = 0;                       // N_Gamma
    int alpert_order = 0;                // l (window a = l), 0 = plain trapezoid
    std::vector<int32_t> n_nodes, offset; // per curve (host)
    dbuf<int32_t> d_nn, d_off;           // per curve (device)
    dbuf<int32_t> d_curve_of;            // curve index of every node
    dbuf<double> xy;                     // [n][2]
    dbuf<double> geo;                    // [n][8]: x y x' y' x'' y'' |y'| kdiag
    dbuf<double> coef;                   // per curve Fourier coefficients: [off*2 ...] see boundary.cu
    dbuf<double2> tw, half;              // per node (cos, sin)(2 pi r / N) and (cos, sin)(pi r / N)
    // fine (16x) grid per curve: positions, normals, speed*h_fine
    int64_t n_fine = 0;
    std::vector<int64_t> fine_off;
    dbuf<int64_t> d_fine_off;
    dbuf<double> fine_geo;               // [n_fine][5]: x y nx ny |y'| h_f
    bie_operator op;
    gmres_ws ws;
    // binary32 source data for the mixed-precision double layer: offsets from tile
    // centres (tiles of MH_TILE nodes, fine chunks of MH_TILE fine nodes per curve)
    int64_t n_tiles = 0, n_fchunks = 0;
    std::vector<int64_t> fchunk_off;     // per curve first chunk
    dbuf<int64_t> d_fchunk_off;
    dbuf<float4> src32, fine32;          // (dx, dy, nx, ny)
    dbuf<double2> tile_c, fchunk_c;
    dbuf<float> tile_r;                  // per source tile: largest distance of a node from its centre
    dbuf<float2> tw32;                   // binary32 copy of the twiddles e^{2 pi i r / N_k}
    dbuf<float> xhi32, xlo32;            // float-float split of the input of a residual product
    dbuf<float4> fchunk_cf;              // fine chunk centres as float-float (x_hi, x_lo, y_hi, y_lo)
    dbuf<float> fchunk_r;                // fine chunk radii
    dbuf<float> w32, wf32, x32;          // per call: weights, fine weights, GEMV input
    dbuf<double> sc64, wf64;             // per call: density Fourier coefficients, fine weights
    // matrix-free operator: the trapezoid sum by the on-surface multipole pass of a tree that
    // holds every node, the Alpert correction by binary64 chirp transforms per curve
    bool mfree = false;
    mh_tree* mf_tree = nullptr;          // not owned (the problem's tree)
    double mf_alpha = -1.0;
    dbuf<double> mf_cp;                  // [n][2 l] Alpert node weights (kernel x rule weight x h / pi)
    dbuf<double> mf_win;                 // [n][2 (a - 1)] own-curve window weights (kernel x |y'| h / pi)
    dbuf<double2> mf_chirp, mf_bh, mf_tw;   // per curve: e^{i pi n^2/N}, transformed chirp filter, twiddles
    dbuf<int64_t> mf_moff;               // per curve: offset of its M_k-entry blocks (twiddles at moff/2)
    dbuf<int32_t> mf_M;                  // per curve: transform length M_k (power of two >= 2 N_k - 1)
    int mf_mmax = 0;
    dbuf<double2> mf_spec;               // per call: spectra c_m, m <= N_k/2
    dbuf<double> mf_S;                   // per call: [2 l][n] interpolated density at the Alpert nodes
    dbuf<double> mf_w, mf_u;             // per call: dipole strengths, multipole-pass output
    SideStream mf_side;                  // the Alpert transforms run there beside the multipole pass
    dbuf<double> warm_dir, warm_w, warm_scal;   // warm-start direction, its image, scalars
    dbuf<float2> fcp32;                  // fine-grid coefficients by sub-offset (binary32)
    dbuf<double2> fcp64;                 // (binary64)
};

#define MH_TILE 128

// Classified target set for off-surface evaluation.
struct dlp_targets {
    int64_t n = 0;          // user targets
    int64_t n_ext = 0;      // user targets + auxiliary points of the normal-line rule
    dbuf<double> xy;        // [n_ext][2]
    dbuf<uint32_t> fine;    // [n_ext] bit k: use the upsampled rule on curve k
    dbuf<int32_t> region;   // [n] -1 inside Omega, k exterior side of curve k
    // normal-line rule: per line target
    int64_t n_line = 0;
    dbuf<int32_t> line_tgt;     // target index
    dbuf<int32_t> line_curve;   // curve
    dbuf<double> line_data;     // [n_line][4]: t*, d, h_s, unused
    dbuf<double> line_w;        // trigonometric interpolation weights at t*, N_k per line target
    dbuf<int64_t> line_woff;    // [n_line + 1] offsets into line_w
    // fine pairs (ext target, curve)
    int64_t n_pairs = 0, n_pairs_main = 0;   // pairs of user targets come first
    double fine_nodes_main = 0, fine_nodes_aux = 0, curve_nodes_main = 0;   // work counts
    dbuf<int32_t> pair_tgt, pair_curve;
    // binary32 upsampled rule at the auxiliary points: groups of FINE_TG pairs on one curve
    // (grp_pair, -1 padded), each group's fine chunks in fine_slices slices, one block per
    // (group, slice); partial sums per (group, slice, pair) in grp_part
    int64_t n_groups = 0;
    int fine_slices = 1;
    dbuf<int32_t> grp_curve, grp_pair;
    dbuf<double> grp_part;
    dbuf<unsigned> grp_cnt;
    // evaluation workspaces (allocated once by dlp_classify)
    dbuf<double> ext, sc, wf, asig, part;
};

struct mh_tree {
    double box[3];
    int q = 0, min_level = 0, max_level = 0;
    int64_t n_leaves = 0, n_boxes = 0, n_nodes = 0;
    std::vector<int32_t> lvl_start;      // box id range per level (host), size max_level+2
    dbuf<int32_t> boxes;                 // [n_boxes][3] level ix iy, level then Morton order
    dbuf<int32_t> leaf_box;              // [n_leaves] box id of each leaf (node order)
    dbuf<int32_t> box_leaf;              // [n_boxes] leaf index or -1
    dbuf<int32_t> box_parent;            // [n_boxes]
    dbuf<int32_t> box_child;             // [n_boxes][4] or -1
    dbuf<int32_t> status;                // dense per-level status map (Morton indexed), box id or -1
    std::vector<int64_t> status_off;     // per level offset into status
    dbuf<double> nodes;                  // [n_nodes][2]
    dbuf<int32_t> list_off[4], list_item[4];   // U V W X in CSR over boxes
    std::vector<int64_t> list_len;       // total items per list
    void* vol = nullptr;                 // volume operator data (volume.cu)
};

struct mh_problem {
    mh_tree* tree = nullptr;
    mh_boundary* bnd = nullptr;
    double dt = 0, alpha = 0;
    int scheme = 0;
    int p = 0;
    int ext_mode = 0;
    std::vector<double> ext_const;
    dbuf<double> d_ext_const;
    dlp_targets tg;                      // volume nodes inside Omega (classification of all nodes)
    dbuf<int32_t> region;                // [n_nodes]
    dbuf<int32_t> inside_idx;            // indices of nodes inside Omega
    int64_t n_inside = 0;
    dbuf<int32_t> bnd_leaf;              // leaf of every boundary node
    dbuf<double> B, Up, Ug, rhs, Uh;     // work arrays
    SideStream aux;                      // the normal-line auxiliary sums beside the double layer's pass
    // GMRES start (mh_problem_set_warm_start)
    int warm_mode = 0;
    int warm_arith = 0;
    struct mh_net* net = nullptr;
    bool have_prev = false;              // sig_prev holds the density entering the previous step
    dbuf<double> sig_prev, r0, c_dev;
    double* c_host = nullptr;            // pinned
    // batched stepping (mh_batch_step): sync-free GMRES with its state in gstat (device)
    bool graph_mode = false;
    gmres_dev* gstat = nullptr;
    // residual recycling: the density, right-hand side and binary64 residual the last step
    // ended with; b - A sigma for an unchanged sigma is b - rc_b + rc_r (no operator product)
    bool rc_valid = false;
    dbuf<double> rc_sigma, rc_b, rc_r, r_start;
    dbuf<int> rc_same;
    ~mh_problem() {
        if (c_host) cudaFreeHost(c_host);
    }
};

// ---- net.cu ----
// Initial guess for A x = rhs (see mh_warm_start in mh.h); c_dev receives the step length.
// save (nullable) receives the incoming sigma before x0 is written.
// r_ready: r0 already holds rhs - A sigma (binary64).
mh_status warm_start_run(mh_ctx* ctx, mh_boundary* bnd, double alpha, struct mh_net* net, int mode, int arith,
                         const double* sigma, const double* sigma_prev2, const double* rhs, double* x0, double* r0,
                         mh_precision prec, double* c_dev, double* save, bool r_ready = false);
bool net_matches(const struct mh_net* net, const mh_boundary* b);
// Workspace of the SECANT / LEARNED starts (allocated once per boundary).
mh_status warm_start_prepare(mh_ctx* ctx, mh_boundary* b);

// ---- boundary.cu ----
mh_status bie_assemble(mh_ctx* ctx, mh_boundary* b, double alpha);
mh_status bie_apply(mh_ctx* ctx, mh_boundary* b, const double* x, double* y, mh_precision prec);
// Matrix-free operator: set-up after volume_bie_setup on tree t (releases the dense forms; every
// later operator product of b goes through it), and one product y = A x (binary64).
mh_status bie_mfree_setup(mh_ctx* ctx, mh_boundary* b, mh_tree* t, double alpha);
mh_status bie_apply_mfree(mh_ctx* ctx, mh_boundary* b, const double* x, double* y);
// y = A x in binary64, skipped when *gate != 0 (gate nullable).
mh_status bie_apply64_gated(mh_ctx* ctx, mh_boundary* b, const double* x, double* y, const int* gate,
                            mh_precision prec);
// y = A x accurate to binary64 for residuals: float-float in mixed precision, binary64 otherwise
mh_status bie_apply_resid(mh_ctx* ctx, mh_boundary* b, const double* x, double* y, mh_precision prec);
// Where the last solve left the binary64 residual rhs - A x of its result.
const double* gmres_final_residual(mh_boundary* b, mh_precision prec, bool graph);
// Everything a sync-free solve in precision prec needs (binary32 operator copy).
mh_status bie_prepare(mh_ctx* ctx, mh_boundary* b, mh_precision prec);
mh_status dlp_classify(mh_ctx* ctx, mh_boundary* b, const double* xy_dev, int64_t n, dlp_targets* tg);
mh_status dlp_evaluate(mh_ctx* ctx, mh_boundary* b, double alpha, dlp_targets* tg,
                       const double* sigma, double* out, mh_precision prec);
// U^h when the trapezoid sum at the user targets (main_vals, n values) comes from the
// multipole method: adds the near-boundary corrections and the normal-line rule.
// fine_in_fmm: main_vals already use the 16x upsampled rule on every curve (the fine
// nodes went through the multipole method), so only the auxiliary points of the
// normal-line rule need near-boundary work.  Requires dlp_fine_weights for this sigma.
// part (fine_in_fmm only): 0 = everything; 1 = the sums at the auxiliary points (they need
// sigma and its fine weights only, so they may run beside the pass that produces main_vals);
// 2 = the rest, after part 1 (main_vals, the normal-line rule, out).
mh_status dlp_evaluate_fmm_tail(mh_ctx* ctx, mh_boundary* b, double alpha, dlp_targets* tg, const double* sigma,
                                const double* main_vals, double* out, mh_precision prec, bool fine_in_fmm,
                                const double* asig_given = nullptr, int part = 0);
// Density on the 16x fine grid times |y'| h_f (binary64 in b->wf64; binary32 also in b->wf32
// when prec is mixed).
mh_status dlp_fine_weights(mh_ctx* ctx, mh_boundary* b, const double* sigma, mh_precision prec);
// r0 (nullable): the binary64 residual rhs - A x of the initial guess, computed by the caller.
mh_status gmres_run(mh_ctx* ctx, mh_boundary* b, const double* rhs, double* x, double tol, int max_iter,
                    mh_precision prec, mh_gmres_info* info, const double* r0 = nullptr);
// The same solve without host synchronisation, for capture in a CUDA graph: a fixed schedule of
// sweeps x m_max Arnoldi iterations whose kernels return at once when the device flags in gs
// say their work is not needed.  gs (device) holds the result; gmres_graph_ensure sizes the
// workspace beforehand (no allocation happens in gmres_run_graph).
mh_status gmres_graph_ensure(mh_ctx* ctx, mh_boundary* b, int m_max);
mh_status gmres_run_graph(mh_ctx* ctx, mh_boundary* b, const double* rhs, double* x, double tol, mh_precision prec,
                          const double* r0, gmres_dev* gs);
void gmres_graph_schedule(mh_precision prec, int* sweeps, int* m_max);
mh_status gmres_info_from_dev(const gmres_dev& g, double tol, mh_gmres_info* info);

// ---- tree.cu ----
void mh_gauss_legendre(int n, double* x, double* w);
const double* tree_gl_nodes(const mh_tree* t);

// ---- volume.cu ----
mh_status volume_apply(mh_ctx* ctx, mh_tree* t, double alpha, int p, const double* b, double* up,
                       mh_precision prec);
void volume_free(mh_tree* t);
// Threads per block of the binary32 near-field double-layer kernel (128, 256 or 512).
mh_status volume_set_near_tile(mh_ctx* ctx, mh_tree* t, int threads);
int volume_near_tile(const mh_tree* t);
// double layer through the multipole method (dipoles sorted by leaf)
mh_status volume_dipole_setup(mh_ctx* ctx, mh_tree* t, double alpha, int p, const double* dxy, const double* dnrm,
                              const int32_t* dleaf, int64_t nd, bool near_blocks);
mh_status volume_dipole_apply(mh_ctx* ctx, mh_tree* t, const double* w_sorted, mh_precision prec, const double** u);
// On-surface double layer through the multipole method (binary64): set-up for the boundary
// nodes (host arrays in node order: positions, unit normals, leaf of every node), then
// u_i = -(1/(2 pi alpha^2)) sum_{d != i} w_d (1/alpha) K1(r/alpha) (y_d - x_i).nu_d / r at every
// node for device strengths w (node order).
mh_status volume_bie_setup(mh_ctx* ctx, mh_tree* t, double alpha, int p, const double* xy, const double* nrm,
                           const int32_t* leaf, int64_t nd);
bool volume_bie_ready(const mh_tree* t);
mh_status volume_bie_apply(mh_ctx* ctx, mh_tree* t, const double* w, double* u);
mh_status tree_locate(mh_ctx* ctx, const mh_tree* t, const double* xy_dev, int64_t n, int32_t* leaf_out);
mh_status tree_interpolate(mh_ctx* ctx, const mh_tree* t, const double* vals, const double* xy_dev,
                           const int32_t* leaf, int64_t n, double* out);

inline int mh_grid(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 2147483647LL) g = 2147483647LL;
    return (int)g;
}
