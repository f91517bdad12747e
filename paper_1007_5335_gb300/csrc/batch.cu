// Batched stepping of independent problems as one CUDA graph per time step, and the
// autotuner of the multipole order and the near-field tile.
//
// A time step of one problem is sync-free in graph mode (GMRES on a fixed schedule of
// device-gated kernels, gmres_run_graph), so the steps of all problems of a batch can be
// captured into one graph: one branch per problem, each on its own forked stream, joined at
// the end.  The graph is recorded after an eager step that also makes every lazy allocation
// (nothing is allocated while capturing) and is relaunched as long as the arrays, the
// tolerance and the precision stay the same.
#include <algorithm>
#include <cmath>
#include <memory>
#include <set>
#include <vector>

#include "mh_internal.cuh"

struct mh_batch {
    int n = 0;
    std::vector<mh_problem*> probs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;          // capture origin (the context stream may be the legacy stream)
    dbuf<gmres_dev> stat;
    std::vector<gmres_dev> stat_h;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_kernels = 0;           // kernel nodes, a loop body counted once
    int64_t loop_nodes = 0;              // GMRES WHILE nodes (bodies of GMRES_LOOP_KERNELS kernels)
    std::vector<const void*> key;
    std::vector<int64_t> key_gen;        // GMRES workspace generation of every problem's boundary
    std::vector<int64_t> key_opgen;      // operator generation of every boundary when recorded
    double key_tol = -1.0;
    int key_prec = -1;
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        graph_kernels = 0;
    }
    ~mh_batch() {
        drop_graph();
        for (auto s : streams) cudaStreamDestroy(s);
        if (cap) cudaStreamDestroy(cap);
        for (auto e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (auto* p : probs) {
            p->graph_mode = false;
            p->gstat = nullptr;
        }
    }
};

namespace {

// Restores the problems' eager mode when a batch step returns.
struct GraphModeScope {
    std::vector<mh_problem*>& probs;
    explicit GraphModeScope(std::vector<mh_problem*>& p) : probs(p) {
        for (auto* q : probs) q->graph_mode = true;
    }
    ~GraphModeScope() {
        for (auto* q : probs) q->graph_mode = false;
    }
};

// sum over nodes inside Omega of (a - b)^2 and b^2 (binary64, per-block partials)
__global__ void k_diff_inside(const double* __restrict__ a, const double* __restrict__ b,
                              const int32_t* __restrict__ region, int64_t n, double* part) {
    __shared__ double s1[256], s2[256];
    double d = 0.0, r = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (region[i] < 0) {
            const double e = a[i] - b[i];
            d = fma(e, e, d);
            r = fma(b[i], b[i], r);
        }
    s1[threadIdx.x] = d;
    s2[threadIdx.x] = r;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

}  // namespace

extern "C" mh_status mh_batch_create(mh_ctx* ctx, int n, mh_problem* const* probs_host, mh_batch** out) {
    if (!ctx || !probs_host || !out || n < 1) return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    std::set<const void*> trees, bnds, nets;
    for (int i = 0; i < n; ++i) {
        const mh_problem* p = probs_host[i];
        if (!p) return mh_fail(ctx, MH_ERR_INVALID_ARG, "problem %d is null", i);
        if (p->scheme != MH_SCHEME_IMEX_EULER)
            return mh_fail(ctx, MH_ERR_INVALID_ARG, "problem %d: batches step IMEX Euler problems", i);
        if (p->ext_mode != MH_EXT_CONST)
            return mh_fail(ctx, MH_ERR_INVALID_ARG, "problem %d: batches need MH_EXT_CONST", i);
        // the branches of the graph run concurrently: no shared workspaces
        if (!trees.insert(p->tree).second || !bnds.insert(p->bnd).second)
            return mh_fail(ctx, MH_ERR_INVALID_ARG, "problem %d shares its tree or boundary with another", i);
        if (p->net && !nets.insert(p->net).second)
            return mh_fail(ctx, MH_ERR_INVALID_ARG, "problem %d shares its network with another", i);
        if (p->gstat) return mh_fail(ctx, MH_ERR_INVALID_ARG, "problem %d already belongs to a batch", i);
    }
    std::unique_ptr<mh_batch> b(new mh_batch());
    b->n = n;
    b->probs.assign(probs_host, probs_host + n);
    MH_ALLOC(ctx, b->stat, n);
    b->stat_h.resize(n);
    b->streams.resize(n, nullptr);
    b->join.resize(n, nullptr);
    for (int i = 0; i < n; ++i) {
        MH_CUDA(ctx, cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking));
        MH_CUDA(ctx, cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming));
    }
    MH_CUDA(ctx, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    MH_CUDA(ctx, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    for (int i = 0; i < n; ++i) b->probs[i]->gstat = b->stat.p + i;
    *out = b.release();
    return MH_OK;
}

extern "C" mh_status mh_batch_destroy(mh_batch* batch) {
    delete batch;
    return MH_OK;
}

extern "C" int64_t mh_batch_graph_kernels(const mh_batch* batch) { return batch ? batch->graph_kernels : 0; }

extern "C" mh_status mh_batch_step(mh_ctx* ctx, mh_batch* B, double* const* u_dev, const double* const* F_dev,
                                   const double* const* f_next_dev, double* const* sigma_dev, double gmres_tol,
                                   mh_precision prec, mh_step_info* info_host) {
    if (!ctx || !B || !u_dev || !F_dev || !f_next_dev || !sigma_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (!(gmres_tol > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "gmres_tol must be positive");
    if (prec != MH_PREC_FP64 && prec != MH_PREC_MIXED) return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad precision");
    const int n = B->n;
    std::vector<const void*> key;
    for (int i = 0; i < n; ++i) {
        if (!u_dev[i] || !F_dev[i] || !f_next_dev[i] || !sigma_dev[i])
            return mh_fail(ctx, MH_ERR_INVALID_ARG, "null array for problem %d", i);
        if (B->probs[i]->bnd->mfree)
            return mh_fail(ctx, MH_ERR_INVALID_ARG,
                           "problem %d uses the matrix-free boundary operator: the graph form needs the dense one", i);
        key.insert(key.end(), {u_dev[i], F_dev[i], f_next_dev[i], sigma_dev[i]});
    }
    GraphModeScope scope(B->probs);
    struct CaptureFlag {
        mh_ctx* c;
        ~CaptureFlag() { c->capturing = false; }
    } cflag{ctx};
    ctx->capturing = true;   // the eager step takes the same kernels as the recorded graph
    // a recorded graph holds the GMRES workspaces: a solve outside the batch that grew one
    // (reallocated it) forces a new recording
    int S, m;
    gmres_graph_schedule(prec, &S, &m);
    std::vector<int64_t> gen(n), opgen(n);
    for (int i = 0; i < n; ++i) {
        MH_TRY(gmres_graph_ensure(ctx, B->probs[i]->bnd, m));
        gen[i] = B->probs[i]->bnd->ws.gen;
        opgen[i] = B->probs[i]->bnd->op.gen;
    }
    // ... and the operator's forms: one reassembled (another alpha) or released since the
    // recording also forces a new one
    const bool record = !B->exec || key != B->key || gen != B->key_gen || opgen != B->key_opgen ||
                        gmres_tol != B->key_tol || (int)prec != B->key_prec;
    if (record) {
        for (auto* p : B->probs) MH_TRY(bie_prepare(ctx, p->bnd, prec));
        // the eager step of this call (makes every lazy allocation)
        for (int i = 0; i < n; ++i)
            MH_TRY(heat_step(ctx, B->probs[i], u_dev[i], F_dev[i], f_next_dev[i], nullptr, u_dev[i], sigma_dev[i],
                             gmres_tol, prec, nullptr));
        // record the graph of the following steps
        B->drop_graph();
        const int64_t l0 = ctx->launches, ln0 = ctx->loop_nodes;
        const bool prof = ctx->profiling;
        ctx->profiling = false;
        cudaStream_t main = ctx->stream;
        cudaStream_t cap = B->cap;
        MH_CUDA(ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        mh_status st = MH_OK;
        cudaError_t ce = cudaEventRecord(B->fork, cap);
        for (int i = 0; i < n && st == MH_OK && ce == cudaSuccess; ++i) {
            ce = cudaStreamWaitEvent(B->streams[i], B->fork, 0);
            if (ce != cudaSuccess) break;
            ctx->stream = B->streams[i];
            st = heat_step(ctx, B->probs[i], u_dev[i], F_dev[i], f_next_dev[i], nullptr, u_dev[i], sigma_dev[i],
                           gmres_tol, prec, nullptr);
            ctx->stream = main;
            if (st == MH_OK) ce = cudaEventRecord(B->join[i], B->streams[i]);
        }
        ctx->stream = main;
        for (int i = 0; i < n && st == MH_OK && ce == cudaSuccess; ++i) ce = cudaStreamWaitEvent(cap, B->join[i], 0);
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cap, &g);
        ctx->profiling = prof;
        B->graph_kernels = ctx->launches - l0;
        B->loop_nodes = ctx->loop_nodes - ln0;
        ctx->launches = l0;
        if (st != MH_OK || ce != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            B->graph_kernels = 0;
            if (st != MH_OK) return st;
            return mh_fail(ctx, MH_ERR_CUDA, "recording the batch graph failed: %s",
                           cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        }
        B->graph = g;
        MH_CUDA(ctx, cudaGraphInstantiate(&B->exec, B->graph, cudaGraphInstantiateFlagUseNodePriority));
        B->key = key;
        B->key_gen = gen;
        // the operator forms the graph holds: taken after the eager step, which makes them
        B->key_opgen.assign(n, 0);
        for (int i = 0; i < n; ++i) B->key_opgen[i] = B->probs[i]->bnd->op.gen;
        B->key_tol = gmres_tol;
        B->key_prec = (int)prec;
    }
    const bool launched = !record;
    if (launched) MH_CUDA(ctx, cudaGraphLaunch(B->exec, ctx->stream));
    MH_CUDA(ctx, cudaMemcpyAsync(B->stat_h.data(), B->stat.p, n * sizeof(gmres_dev), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (launched) {   // kernels run: the recorded nodes, each loop body once per Arnoldi iteration
        int64_t its = 0;
        for (int i = 0; i < n; ++i) its += B->stat_h[i].total;
        ctx->launches += B->graph_kernels + (B->loop_nodes ? GMRES_LOOP_KERNELS * (its - B->loop_nodes) : 0);
    }
    int bad = -1;
    for (int i = 0; i < n; ++i) {
        mh_gmres_info gi{};
        gmres_info_from_dev(B->stat_h[i], gmres_tol, &gi);
        if (info_host) {
            info_host[i].gmres_iterations = gi.iterations;
            info_host[i].gmres_rel_residual = gi.rel_residual;
            info_host[i].initial_rel_residual = gi.initial_rel_residual;
            const mh_problem* p = B->probs[i];
            info_host[i].warm_c = (p->warm_mode == MH_WARM_SECANT || p->warm_mode == MH_WARM_LEARNED) && p->c_host
                                      ? *p->c_host : 0.0;
        }
        if (!gi.converged && bad < 0) bad = i;
    }
    if (bad >= 0)
        return mh_fail(ctx, MH_ERR_NOT_CONVERGED, "problem %d: GMRES stopped at relative residual %.3e", bad,
                       B->stat_h[bad].rel);
    return MH_OK;
}

extern "C" mh_status mh_problem_set_near_tile(mh_ctx* ctx, mh_problem* prob, int threads) {
    if (!ctx || !prob) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    return volume_set_near_tile(ctx, prob->tree, threads);
}

extern "C" mh_status mh_autotune(mh_ctx* ctx, mh_tree* tree, mh_boundary* bnd, double dt, int ext_mode,
                                 const double* ext_const_host, const double* F_dev, const double* f_dev, int n_p,
                                 const int* p_cand, double err_tol, int steps, mh_precision prec, int* p_out,
                                 int* tile_out, mh_tune_entry* report_host) {
    if (!ctx || !tree || !bnd || !F_dev || !f_dev || !p_cand || !p_out || !tile_out)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (n_p < 1 || n_p > 16 || steps < 2 || !(err_tol > 0) || ext_mode != MH_EXT_CONST)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad autotuner arguments (n_p 1..16, steps >= 2, MH_EXT_CONST)");
    int pmax = 0;
    for (int i = 0; i < n_p; ++i) {
        if (p_cand[i] < 4 || p_cand[i] > 40) return mh_fail(ctx, MH_ERR_INVALID_ARG, "candidate p out of 4..40");
        pmax = std::max(pmax, p_cand[i]);
    }
    const int p_ref = std::min(40, pmax + 8);
    cudaStream_t st = ctx->stream;
    const int64_t nn = tree->n_nodes, nb = bnd->n;
    dbuf<double> u, sigma, uref, part;
    dbuf<int32_t> region;
    MH_ALLOC(ctx, u, nn);
    MH_ALLOC(ctx, uref, nn);
    MH_ALLOC(ctx, sigma, nb);
    MH_ALLOC(ctx, region, nn);
    MH_ALLOC(ctx, part, 2 * 304);
    cudaEvent_t e0, e1;
    MH_CUDA(ctx, cudaEventCreate(&e0));
    MH_CUDA(ctx, cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evg{e0, e1};
    auto make = [&](int p, mh_problem** P) -> mh_status {
        MH_TRY(mh_problem_create(ctx, tree, bnd, dt, MH_SCHEME_IMEX_EULER, p, ext_mode, ext_const_host, P));
        MH_CUDA(ctx, cudaMemcpyAsync(region.p, (*P)->region.p, nn * 4, cudaMemcpyDeviceToDevice, st));
        return MH_OK;
    };
    auto run = [&](mh_problem* P, double* u_out, double* ms) -> mh_status {
        MH_CUDA(ctx, cudaMemsetAsync(u_out, 0, nn * 8, st));
        MH_CUDA(ctx, cudaMemsetAsync(sigma.p, 0, nb * 8, st));
        std::vector<float> t;
        for (int s = 0; s < steps; ++s) {
            MH_CUDA(ctx, cudaEventRecord(e0, st));
            mh_step_info info{};
            MH_TRY(heat_step(ctx, P, u_out, F_dev, f_dev, nullptr, u_out, sigma.p, 1e-10, prec, &info));
            MH_CUDA(ctx, cudaEventRecord(e1, st));
            MH_CUDA(ctx, cudaEventSynchronize(e1));
            float e = 0.f;
            MH_CUDA(ctx, cudaEventElapsedTime(&e, e0, e1));
            if (s > 0) t.push_back(e);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return MH_OK;
    };
    using PG = std::unique_ptr<mh_problem, mh_status (*)(mh_problem*)>;
    auto rel_err = [&](double* out) -> mh_status {
        k_diff_inside<<<304, 256, 0, st>>>(u.p, uref.p, region.p, nn, part.p);
        MH_LAUNCHED(ctx);
        double h[2 * 304];
        MH_CUDA(ctx, cudaMemcpyAsync(h, part.p, sizeof(h), cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
        double d = 0.0, r = 0.0;
        for (int i = 0; i < 304; ++i) {
            d += h[2 * i];
            r += h[2 * i + 1];
        }
        *out = r > 0.0 ? std::sqrt(d / r) : std::sqrt(d);
        return MH_OK;
    };
    double ms_ref = 0.0;
    {
        mh_problem* P = nullptr;
        MH_TRY(make(p_ref, &P));
        PG g(P, mh_problem_destroy);
        MH_TRY(run(P, uref.p, &ms_ref));
    }
    std::vector<mh_tune_entry> rep;
    int best = -1;
    for (int i = 0; i < n_p; ++i) {
        mh_tune_entry e{p_cand[i], 256, 0.0, 0.0};
        mh_problem* P = nullptr;
        MH_TRY(make(p_cand[i], &P));
        PG g(P, mh_problem_destroy);
        MH_TRY(run(P, u.p, &e.ms_per_step));
        MH_TRY(rel_err(&e.rel_err));
        rep.push_back(e);
    }
    for (int i = 0; i < n_p; ++i) {
        const bool ok = rep[i].rel_err <= err_tol;
        if (ok && (best < 0 || rep[best].rel_err > err_tol || rep[i].ms_per_step < rep[best].ms_per_step)) best = i;
    }
    if (best < 0)   // none meets the tolerance: the most accurate
        for (int i = 0; i < n_p; ++i)
            if (best < 0 || rep[i].rel_err < rep[best].rel_err) best = i;
    const int p_best = rep[best].p;
    int tile_best = 256;
    double t_best = 1e300;
    {
        mh_problem* P = nullptr;
        MH_TRY(make(p_best, &P));
        PG g(P, mh_problem_destroy);
        for (int tile : {128, 256, 512}) {
            mh_tune_entry e{p_best, tile, 0.0, 0.0};
            MH_TRY(volume_set_near_tile(ctx, tree, tile));
            MH_TRY(run(P, u.p, &e.ms_per_step));
            MH_TRY(rel_err(&e.rel_err));
            rep.push_back(e);
            if (e.ms_per_step < t_best) {
                t_best = e.ms_per_step;
                tile_best = tile;
            }
        }
    }
    *p_out = p_best;
    *tile_out = tile_best;
    if (report_host) std::copy(rep.begin(), rep.end(), report_host);
    return MH_OK;
}
