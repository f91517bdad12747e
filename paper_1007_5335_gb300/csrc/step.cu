// IMEX (backward) Euler heat step (Section 2): u^{N+1} - alpha^2 Lap u^{N+1} = u^N + dt F^N,
// alpha^2 = dt, solved as U = U^p + U^h.  The per-step work is
//   form B~ (extension outside Omega, Section 3.1) -> volume potential -> leaf
//   interpolation onto Gamma (Section 3.1) -> rhs = -2 alpha^2 (f - U^p) -> GMRES ->
//   double layer at the nodes in Omega -> combine,
// all on the context's stream.  Classification of the volume nodes, the leaf of every
// boundary node, the boundary operator and the multipole operators are built once by
// mh_problem_create.
#include <algorithm>
#include <cmath>
#include <memory>

#include "mh_internal.cuh"

namespace {

__global__ void k_form_B(const double* __restrict__ u, const double* __restrict__ F,
                         const int32_t* __restrict__ region, const double* __restrict__ ext_const,
                         const double* __restrict__ b_ext, int ext_mode, double dt, int64_t n, double* B) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = region[i];
    double v;
    if (r < 0)
        v = u[i] + dt * F[i];
    else
        v = ext_mode == MH_EXT_CONST ? ext_const[r] + dt * F[i] : b_ext[i];
    B[i] = v;
}

// Allen-Cahn right-hand side (Section 4, Example 3): B = u + dt u (1 - u^2) inside Omega; outside
// the constant extension C_k + dt C_k (1 - C_k^2) (u = C_k there) or caller-supplied values.
__global__ void k_form_B_allen_cahn(const double* __restrict__ u, const int32_t* __restrict__ region,
                                    const double* __restrict__ ext_const, const double* __restrict__ b_ext,
                                    int ext_mode, double dt, int64_t n, double* B) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = region[i];
    double v;
    if (r < 0) {
        const double a = u[i];
        v = a + dt * a * (1.0 - a * a);
    } else if (ext_mode == MH_EXT_CONST) {
        const double c = ext_const[r];
        v = c + dt * c * (1.0 - c * c);
    } else {
        v = b_ext[i];
    }
    B[i] = v;
}

__global__ void k_form_B_gear(const double* __restrict__ u, const double* __restrict__ up, const double* __restrict__ F,
                              const double* __restrict__ Fp, const int32_t* __restrict__ region,
                              const double* __restrict__ ext_const, const double* __restrict__ b_ext, int ext_mode,
                              double dt, int64_t n, double* B) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = region[i];
    const double forcing = dt * (4.0 * F[i] - 2.0 * Fp[i]) / 3.0;
    double v;
    if (r < 0)
        v = (4.0 * u[i] - up[i]) / 3.0 + forcing;
    else
        v = ext_mode == MH_EXT_CONST ? ext_const[r] + forcing : b_ext[i];
    B[i] = v;
}

// same[0] stays set (nonzero) only if a == b element by element.
__global__ void k_rc_compare(const double* __restrict__ a, const double* __restrict__ b, int64_t n, int* same) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (a[i] != b[i]) *same = 0;
}

// r = rhs - rhs_prev + r_prev when the density is the one the previous step ended with
// (rhs_prev - A sigma = r_prev), else r = rhs - Ax (Ax computed for that case).
__global__ void k_rc_resid(const double* __restrict__ rhs, const double* __restrict__ ax,
                           const double* __restrict__ rhs_prev, const double* __restrict__ r_prev,
                           const int* __restrict__ same, int64_t n, double* r) {
    const bool s = *same != 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = s ? (rhs[i] - rhs_prev[i]) + r_prev[i] : rhs[i] - ax[i];
}

__global__ void k_rhs(const double* __restrict__ f, const double* __restrict__ ug, double c, int64_t n, double* rhs) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) rhs[i] = c * (f[i] - ug[i]);
}

__global__ void k_combine(const double* __restrict__ up, const double* __restrict__ uh,
                          const int32_t* __restrict__ region, const int32_t* __restrict__ slot,
                          const double* __restrict__ ext_const, int ext_mode, int64_t n, double* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = region[i];
    if (r < 0)
        out[i] = up[i] + uh[slot[i]];
    else
        out[i] = ext_mode == MH_EXT_CONST ? ext_const[r] : up[i];
}

__global__ void k_gather_xy(const double* __restrict__ xy, const int32_t* __restrict__ idx, int64_t n, double* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[2 * i] = xy[2 * idx[i]];
    out[2 * i + 1] = xy[2 * idx[i] + 1];
}

}  // namespace

__global__ void k_dip_weights(const double* __restrict__ wf, const int32_t* __restrict__ perm, int64_t n,
                              double* w) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < n) w[j] = wf[perm[j]];
}

__global__ void k_gather(const double* __restrict__ src, const int32_t* __restrict__ idx, int64_t n, double* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = src[idx[i]];
}

struct ProblemImpl : mh_problem {
    dbuf<int32_t> slot;       // position of an inside node in the inside list, else -1
    dbuf<int32_t> perm;       // boundary nodes sorted by leaf: sorted position -> node
    dbuf<double> w_sorted;    // dipole strengths in that order
};

extern "C" mh_status mh_problem_create(mh_ctx* ctx, mh_tree* tree, mh_boundary* bnd, double dt, int scheme, int p,
                                       int ext_mode, const double* ext_const_host, mh_problem** out) {
    if (!ctx || !tree || !bnd || !out) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (!(dt > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "dt must be positive");
    if (scheme != MH_SCHEME_IMEX_EULER && scheme != MH_SCHEME_EXTRAP_GEAR)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "unknown scheme %d", scheme);
    if (p < 1 || p > 40) return mh_fail(ctx, MH_ERR_INVALID_ARG, "p must be in 1..40");
    if (ext_mode != MH_EXT_CONST && ext_mode != MH_EXT_ARRAY) return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad ext_mode");
    if (ext_mode == MH_EXT_CONST && !ext_const_host)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "MH_EXT_CONST needs ext_const_host");
    cudaStream_t st = ctx->stream;
    std::unique_ptr<ProblemImpl> P(new ProblemImpl());
    P->tree = tree;
    P->bnd = bnd;
    P->dt = dt;
    P->scheme = scheme;
    P->alpha = std::sqrt(scheme == MH_SCHEME_EXTRAP_GEAR ? 2.0 * dt / 3.0 : dt);
    P->p = p;
    P->ext_mode = ext_mode;
    const int nc = bnd->n_curves;
    P->ext_const.assign(nc, 0.0);
    if (ext_const_host) P->ext_const.assign(ext_const_host, ext_const_host + nc);
    MH_ALLOC(ctx, P->d_ext_const, nc);
    MH_CUDA(ctx, cudaMemcpyAsync(P->d_ext_const.p, P->ext_const.data(), nc * 8, cudaMemcpyHostToDevice, st));
    const int64_t n = tree->n_nodes;
    // classify every node, then re-classify the inside ones as the evaluation target set
    {
        dlp_targets all;
        MH_TRY(dlp_classify(ctx, bnd, tree->nodes.p, n, &all));
        MH_ALLOC(ctx, P->region, n);
        MH_CUDA(ctx, cudaMemcpyAsync(P->region.p, all.region.p, n * 4, cudaMemcpyDeviceToDevice, st));
        std::vector<int32_t> reg(n), slot(n, -1), idx;
        MH_CUDA(ctx, cudaMemcpyAsync(reg.data(), all.region.p, n * 4, cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
        for (int64_t i = 0; i < n; ++i)
            if (reg[i] < 0) {
                slot[i] = (int32_t)idx.size();
                idx.push_back((int32_t)i);
            }
        P->n_inside = (int64_t)idx.size();
        MH_ALLOC(ctx, P->inside_idx, std::max<int64_t>(P->n_inside, 1));
        MH_ALLOC(ctx, P->slot, n);
        MH_CUDA(ctx, cudaMemcpyAsync(P->slot.p, slot.data(), n * 4, cudaMemcpyHostToDevice, st));
        dbuf<double> xin;
        MH_ALLOC(ctx, xin, std::max<int64_t>(2 * P->n_inside, 2));
        if (P->n_inside) {
            MH_CUDA(ctx, cudaMemcpyAsync(P->inside_idx.p, idx.data(), P->n_inside * 4, cudaMemcpyHostToDevice, st));
            k_gather_xy<<<mh_grid(P->n_inside, 256), 256, 0, st>>>(tree->nodes.p, P->inside_idx.p, P->n_inside, xin.p);
            MH_LAUNCHED(ctx);
        }
        MH_TRY(dlp_classify(ctx, bnd, xin.p, P->n_inside, &P->tg));
        if (P->tg.n_ext > P->tg.n) MH_TRY(P->aux.create(ctx, false));
    }
    // leaf of every boundary node
    MH_ALLOC(ctx, P->bnd_leaf, bnd->n);
    MH_TRY(tree_locate(ctx, tree, bnd->xy.p, bnd->n, P->bnd_leaf.p));
    {
        std::vector<int32_t> bl(bnd->n);
        MH_CUDA(ctx, cudaMemcpyAsync(bl.data(), P->bnd_leaf.p, bnd->n * 4, cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
        for (int64_t i = 0; i < bnd->n; ++i)
            if (bl[i] < 0) return mh_fail(ctx, MH_ERR_GEOMETRY, "boundary node %lld lies outside the tree", (long long)i);
    }
    // Dipole sources of the double layer for the multipole pass: the 16x fine nodes of every
    // curve (the upsampled rule, applied at every volume node; for nodes at least 10 h_s from
    // a curve it agrees with the trapezoid rule to ~1e-14 for smooth densities), sorted by leaf.
    {
        const int64_t nf = bnd->n_fine;
        std::vector<double> fg(6 * nf), fxy(2 * nf);
        MH_CUDA(ctx, cudaMemcpyAsync(fg.data(), bnd->fine_geo.p, 6 * nf * 8, cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
        for (int64_t f = 0; f < nf; ++f) {
            fxy[2 * f] = fg[6 * f];
            fxy[2 * f + 1] = fg[6 * f + 1];
        }
        dbuf<double> dfxy;
        dbuf<int32_t> dfleaf;
        MH_ALLOC(ctx, dfxy, 2 * nf);
        MH_ALLOC(ctx, dfleaf, nf);
        MH_CUDA(ctx, cudaMemcpyAsync(dfxy.p, fxy.data(), 2 * nf * 8, cudaMemcpyHostToDevice, st));
        MH_TRY(tree_locate(ctx, tree, dfxy.p, nf, dfleaf.p));
        std::vector<int32_t> fl(nf);
        MH_CUDA(ctx, cudaMemcpyAsync(fl.data(), dfleaf.p, nf * 4, cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
        std::vector<int32_t> perm(nf);
        for (int64_t i = 0; i < nf; ++i) {
            if (fl[i] < 0) return mh_fail(ctx, MH_ERR_GEOMETRY, "fine boundary point %lld lies outside the tree",
                                          (long long)i);
            perm[i] = (int32_t)i;
        }
        std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t c) { return fl[a] < fl[c]; });
        std::vector<double> dxy(2 * nf), dnrm(2 * nf);
        std::vector<int32_t> dleaf(nf);
        for (int64_t j = 0; j < nf; ++j) {
            const double* g = &fg[6 * (int64_t)perm[j]];
            dxy[2 * j] = g[0];
            dxy[2 * j + 1] = g[1];
            dnrm[2 * j] = g[2];
            dnrm[2 * j + 1] = g[3];
            dleaf[j] = fl[perm[j]];
        }
        MH_TRY(volume_dipole_setup(ctx, tree, P->alpha, p, dxy.data(), dnrm.data(), dleaf.data(), nf, false));
        MH_ALLOC(ctx, P->perm, nf);
        MH_ALLOC(ctx, P->w_sorted, nf);
        MH_CUDA(ctx, cudaMemcpyAsync(P->perm.p, perm.data(), nf * 4, cudaMemcpyHostToDevice, st));
    }
    MH_ALLOC(ctx, P->B, n);
    MH_ALLOC(ctx, P->Up, n);
    MH_ALLOC(ctx, P->Ug, bnd->n);
    MH_ALLOC(ctx, P->rhs, bnd->n);
    MH_CUDA(ctx, cudaMemsetAsync(P->rhs.p, 0, bnd->n * 8, st));
    MH_ALLOC(ctx, P->rc_sigma, bnd->n);
    MH_ALLOC(ctx, P->rc_b, bnd->n);
    MH_ALLOC(ctx, P->rc_r, bnd->n);
    MH_ALLOC(ctx, P->r_start, bnd->n);
    MH_ALLOC(ctx, P->rc_same, 1);
    MH_CUDA(ctx, cudaMemsetAsync(P->rc_b.p, 0, bnd->n * 8, st));
    MH_CUDA(ctx, cudaMemsetAsync(P->rc_r.p, 0, bnd->n * 8, st));
    MH_ALLOC(ctx, P->Uh, std::max<int64_t>(P->n_inside, 1));
    // operators: boundary (alpha) and volume (alpha, p) -- built once here
    MH_TRY(bie_assemble(ctx, bnd, P->alpha));
    MH_CUDA(ctx, cudaMemsetAsync(P->B.p, 0, n * 8, st));
    MH_TRY(volume_apply(ctx, tree, P->alpha, p, P->B.p, P->Up.p, MH_PREC_FP64));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    *out = P.release();
    return MH_OK;
}

extern "C" mh_status mh_problem_destroy(mh_problem* p) {
    ProblemImpl* P = static_cast<ProblemImpl*>(p);
    // a boundary whose matrix-free operator runs on this problem's tree goes back to the dense
    // operator (assembled again at its next use): the tree may be destroyed after the problem
    if (P && P->bnd && P->bnd->mf_tree == P->tree) {
        P->bnd->mfree = false;
        P->bnd->mf_tree = nullptr;
    }
    delete P;
    return MH_OK;
}

extern "C" mh_status mh_problem_matrix_free(mh_ctx* ctx, mh_problem* prob, int enable) {
    if (!ctx || !prob) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    ProblemImpl* P = static_cast<ProblemImpl*>(prob);
    mh_boundary* b = P->bnd;
    if (!enable) {
        if (!b->mfree) return MH_OK;
        b->mfree = false;   // back to the dense operator, assembled again now
        return bie_assemble(ctx, b, P->alpha);
    }
    if (b->mfree && b->mf_tree == P->tree && b->mf_alpha == P->alpha && volume_bie_ready(P->tree)) return MH_OK;
    cudaStream_t st = ctx->stream;
    const int64_t n = b->n;
    std::vector<double> geo(8 * n), xy(2 * n), nrm(2 * n);
    std::vector<int32_t> leaf(n);
    MH_CUDA(ctx, cudaMemcpyAsync(geo.data(), b->geo.p, 8 * n * 8, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaMemcpyAsync(leaf.data(), P->bnd_leaf.p, n * 4, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    for (int64_t i = 0; i < n; ++i) {
        const double* g = &geo[8 * i];
        xy[2 * i] = g[0];
        xy[2 * i + 1] = g[1];
        nrm[2 * i] = g[3] / g[6];    // unit normal (y', -x') / |y'|, as in the operator
        nrm[2 * i + 1] = -g[2] / g[6];
    }
    MH_TRY(volume_bie_setup(ctx, P->tree, P->alpha, P->p, xy.data(), nrm.data(), leaf.data(), n));
    return bie_mfree_setup(ctx, b, P->tree, P->alpha);
}

extern "C" mh_status mh_problem_regions(mh_ctx* ctx, const mh_problem* p, int32_t* region_host) {
    if (!ctx || !p || !region_host) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_CUDA(ctx, cudaMemcpyAsync(region_host, p->region.p, p->tree->n_nodes * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return MH_OK;
}

extern "C" mh_status mh_problem_set_warm_start(mh_ctx* ctx, mh_problem* p, mh_warm_mode mode, mh_net* net,
                                               mh_net_arith arith) {
    if (!ctx || !p) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (mode < MH_WARM_PREVIOUS || mode > MH_WARM_LEARNED) return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad mode");
    if (arith < MH_NET_FP32 || arith > MH_NET_BF16X2) return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad arith");
    if (mode == MH_WARM_LEARNED && !net_matches(net, p->bnd))
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "MH_WARM_LEARNED needs a network built for this boundary");
    const int64_t ng = p->bnd->n;
    if (!p->r0.p) {
        MH_ALLOC(ctx, p->r0, ng);
        MH_ALLOC(ctx, p->c_dev, 1);
        MH_CUDA(ctx, cudaMallocHost((void**)&p->c_host, 8));
        *p->c_host = 0.0;
    }
    if (mode == MH_WARM_SECANT && !p->sig_prev.p) MH_ALLOC(ctx, p->sig_prev, ng);
    if (mode == MH_WARM_SECANT || mode == MH_WARM_LEARNED) MH_TRY(warm_start_prepare(ctx, p->bnd));
    p->warm_mode = mode;
    p->net = mode == MH_WARM_LEARNED ? net : nullptr;
    p->warm_arith = arith;
    p->have_prev = false;
    return MH_OK;
}

extern "C" mh_status mh_problem_rhs(mh_ctx* ctx, const mh_problem* p, double* rhs_dev) {
    if (!ctx || !p || !rhs_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_CUDA(ctx, cudaMemcpyAsync(rhs_dev, p->rhs.p, p->bnd->n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return MH_OK;
}

// r = rhs - A sigma in binary64 for the GMRES start; the operator product is skipped (on the
// device) when sigma is bit for bit the density the previous step ended with.
static mh_status start_residual(mh_ctx* ctx, ProblemImpl* P, const double* sigma, double* r, mh_precision prec) {
    cudaStream_t st = ctx->stream;
    mh_boundary* b = P->bnd;
    const int64_t n = b->n;
    MH_TRY(bie_assemble(ctx, b, P->alpha));
    const int grid = mh_grid(n, 256) < 152 * 4 ? mh_grid(n, 256) : 152 * 4;
    if (P->rc_valid) {
        MH_CUDA(ctx, cudaMemsetAsync(P->rc_same.p, 1, sizeof(int), st));
        k_rc_compare<<<grid, 256, 0, st>>>(sigma, P->rc_sigma.p, n, P->rc_same.p);
        MH_LAUNCHED(ctx);
        MH_TRY(bie_apply64_gated(ctx, b, sigma, r, P->rc_same.p, prec));
        k_rc_resid<<<grid, 256, 0, st>>>(P->rhs.p, r, P->rc_b.p, P->rc_r.p, P->rc_same.p, n, r);
        MH_LAUNCHED(ctx);
    } else {
        MH_TRY(bie_apply64_gated(ctx, b, sigma, r, nullptr, prec));
        MH_CUDA(ctx, cudaMemsetAsync(P->rc_same.p, 0, sizeof(int), st));
        k_rc_resid<<<grid, 256, 0, st>>>(P->rhs.p, r, P->rc_b.p, P->rc_r.p, P->rc_same.p, n, r);
        MH_LAUNCHED(ctx);
    }
    return MH_OK;
}

__global__ void k_rhs_minus_r(const double* __restrict__ rhs, const double* __restrict__ r, int64_t n,
                              double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = rhs[i] - r[i];
}

// Everything after the right-hand side B (P->B) has been formed.
static mh_status step_solve(mh_ctx* ctx, ProblemImpl* P, const double* f_next_dev, double* u_next_dev,
                            double* sigma_dev, double gmres_tol, mh_precision prec, mh_step_info* info) {
    cudaStream_t st = ctx->stream;
    mh_tree* t = P->tree;
    mh_boundary* b = P->bnd;
    const int64_t n = t->n_nodes, ng = b->n;
    MH_TRY(volume_apply(ctx, t, P->alpha, P->p, P->B.p, P->Up.p, prec));
    MH_TRY(tree_interpolate(ctx, t, P->Up.p, b->xy.p, P->bnd_leaf.p, ng, P->Ug.p));
    k_rhs<<<mh_grid(ng, 256), 256, 0, st>>>(f_next_dev, P->Ug.p, -2.0 * P->alpha * P->alpha, ng, P->rhs.p);
    MH_LAUNCHED(ctx);
    mh_gmres_info gi{};
    // GMRES start (mh_problem_set_warm_start); r0 = its binary64 residual when computed here
    const double* r0 = nullptr;
    bool have_c = false;
    const int mode = P->warm_mode;
    if (mode == MH_WARM_ZERO) {
        MH_CUDA(ctx, cudaMemsetAsync(sigma_dev, 0, ng * 8, st));
    } else if (mode == MH_WARM_SECANT || mode == MH_WARM_LEARNED) {
        MH_TRY(start_residual(ctx, P, sigma_dev, P->r0.p, prec));
        if (mode == MH_WARM_SECANT && !P->have_prev) {
            MH_CUDA(ctx, cudaMemcpyAsync(P->sig_prev.p, sigma_dev, ng * 8, cudaMemcpyDeviceToDevice, st));
            P->have_prev = true;
        } else {
            double* keep = mode == MH_WARM_SECANT ? P->sig_prev.p : nullptr;
            MH_TRY(warm_start_run(ctx, b, P->alpha, P->net, mode, P->warm_arith, sigma_dev, keep, P->rhs.p,
                                  sigma_dev, P->r0.p, prec, P->c_dev.p, keep, true));
            MH_CUDA(ctx, cudaMemcpyAsync(P->c_host, P->c_dev.p, 8, cudaMemcpyDeviceToHost, st));
            have_c = true;
        }
        r0 = P->r0.p;
    } else {   // previous-step start
        MH_TRY(start_residual(ctx, P, sigma_dev, P->r_start.p, prec));
        r0 = P->r_start.p;
    }
    if (P->graph_mode) {
        // sync-free solve: the result stays in P->gstat until the caller reads it back
        MH_TRY(gmres_run_graph(ctx, b, P->rhs.p, sigma_dev, gmres_tol, prec, r0, P->gstat));
    }
    mh_status s = P->graph_mode ? MH_OK : gmres_run(ctx, b, P->rhs.p, sigma_dev, gmres_tol, 100, prec, &gi, r0);
    // keep what the next step needs to skip its first binary64 operator product
    if (s == MH_OK) {
        MH_CUDA(ctx, cudaMemcpyAsync(P->rc_sigma.p, sigma_dev, ng * 8, cudaMemcpyDeviceToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(P->rc_b.p, P->rhs.p, ng * 8, cudaMemcpyDeviceToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(P->rc_r.p, gmres_final_residual(b, prec, P->graph_mode), ng * 8,
                                     cudaMemcpyDeviceToDevice, st));
        P->rc_valid = true;
    } else {
        P->rc_valid = false;
    }
    if (info && !P->graph_mode) {
        info->gmres_iterations = gi.iterations;
        info->gmres_rel_residual = gi.rel_residual;
        info->initial_rel_residual = gi.initial_rel_residual;
        info->warm_c = have_c ? *P->c_host : 0.0;   // gmres_run synchronised the stream
    }
    if (s != MH_OK) return s;
    // U^h: trapezoid sum by the multipole method at every node, then the near-boundary rules
    MH_TRY(dlp_fine_weights(ctx, b, sigma_dev, prec));
    // the sums at the auxiliary points of the normal-line rule need only sigma and the fine
    // weights: without region timers they run on a second stream beside the multipole pass
    const bool aux_fork = !ctx->profiling && P->aux.s && P->tg.n_ext > P->tg.n;
    if (aux_fork) {
        MH_TRY(P->aux.begin(ctx, st));
        ctx->stream = P->aux.s;
        const mh_status sa = dlp_evaluate_fmm_tail(ctx, b, P->alpha, &P->tg, sigma_dev, nullptr, nullptr, prec, true,
                                                   nullptr, 1);
        ctx->stream = st;
        MH_TRY(sa);
        MH_TRY(P->aux.end(ctx));
    }
    k_dip_weights<<<mh_grid(b->n_fine, 256), 256, 0, st>>>(b->wf64.p, P->perm.p, b->n_fine, P->w_sorted.p);
    MH_LAUNCHED(ctx);
    const double* du = nullptr;
    MH_TRY(volume_dipole_apply(ctx, t, P->w_sorted.p, prec, &du));
    if (P->n_inside) {
        k_gather<<<mh_grid(P->n_inside, 256), 256, 0, st>>>(du, P->inside_idx.p, P->n_inside, P->Uh.p);
        MH_LAUNCHED(ctx);
    }
    // A sigma for the normal-line rule from the solver's final residual r = rhs - A sigma
    // (binary64, or float-float on the binary32 operator and its low part): rhs - r, no operator product
    if (P->tg.n_line) {
        k_rhs_minus_r<<<mh_grid(ng, 256), 256, 0, st>>>(P->rhs.p, P->rc_r.p, ng, P->tg.asig.p);
        MH_LAUNCHED(ctx);
    }
    if (aux_fork) MH_CUDA(ctx, cudaStreamWaitEvent(st, P->aux.join, 0));
    MH_TRY(dlp_evaluate_fmm_tail(ctx, b, P->alpha, &P->tg, sigma_dev, P->Uh.p, P->Uh.p, prec, true,
                                 P->tg.n_line ? P->tg.asig.p : nullptr, aux_fork ? 2 : 0));
    k_combine<<<mh_grid(n, 256), 256, 0, st>>>(P->Up.p, P->Uh.p, P->region.p, P->slot.p, P->d_ext_const.p,
                                               P->ext_mode, n, u_next_dev);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

extern "C" mh_status heat_step(mh_ctx* ctx, mh_problem* prob, const double* u_dev, const double* F_dev,
                               const double* f_next_dev, const double* b_ext_dev, double* u_next_dev,
                               double* sigma_dev, double gmres_tol, mh_precision prec, mh_step_info* info) {
    if (!ctx || !prob || !u_dev || !F_dev || !f_next_dev || !u_next_dev || !sigma_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    ProblemImpl* P = static_cast<ProblemImpl*>(prob);
    if (P->scheme != MH_SCHEME_IMEX_EULER)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "heat_step needs a problem created with MH_SCHEME_IMEX_EULER");
    if (P->ext_mode == MH_EXT_ARRAY && !b_ext_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "MH_EXT_ARRAY needs b_ext_dev");
    if (!(gmres_tol > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "gmres_tol must be positive");
    const int64_t n = P->tree->n_nodes;
    k_form_B<<<mh_grid(n, 256), 256, 0, ctx->stream>>>(u_dev, F_dev, P->region.p, P->d_ext_const.p, b_ext_dev,
                                                       P->ext_mode, P->dt, n, P->B.p);
    MH_LAUNCHED(ctx);
    return step_solve(ctx, P, f_next_dev, u_next_dev, sigma_dev, gmres_tol, prec, info);
}

extern "C" mh_status heat_step_gear(mh_ctx* ctx, mh_problem* prob, const double* u_dev, const double* u_prev_dev,
                                    const double* F_dev, const double* F_prev_dev, const double* f_next_dev,
                                    const double* b_ext_dev, double* u_next_dev, double* sigma_dev, double gmres_tol,
                                    mh_precision prec, mh_step_info* info) {
    if (!ctx || !prob || !u_dev || !u_prev_dev || !F_dev || !F_prev_dev || !f_next_dev || !u_next_dev || !sigma_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    ProblemImpl* P = static_cast<ProblemImpl*>(prob);
    if (P->scheme != MH_SCHEME_EXTRAP_GEAR)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "heat_step_gear needs a problem created with MH_SCHEME_EXTRAP_GEAR");
    if (P->ext_mode == MH_EXT_ARRAY && !b_ext_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "MH_EXT_ARRAY needs b_ext_dev");
    if (!(gmres_tol > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "gmres_tol must be positive");
    const int64_t n = P->tree->n_nodes;
    k_form_B_gear<<<mh_grid(n, 256), 256, 0, ctx->stream>>>(u_dev, u_prev_dev, F_dev, F_prev_dev, P->region.p,
                                                            P->d_ext_const.p, b_ext_dev, P->ext_mode, P->dt, n,
                                                            P->B.p);
    MH_LAUNCHED(ctx);
    return step_solve(ctx, P, f_next_dev, u_next_dev, sigma_dev, gmres_tol, prec, info);
}

extern "C" mh_status allen_cahn_step(mh_ctx* ctx, mh_problem* prob, double eps, const double* u_dev,
                                     const double* f_next_dev, const double* b_ext_dev, double* u_next_dev,
                                     double* sigma_dev, double gmres_tol, mh_precision prec, mh_step_info* info) {
    if (!ctx || !prob || !u_dev || !f_next_dev || !u_next_dev || !sigma_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    ProblemImpl* P = static_cast<ProblemImpl*>(prob);
    if (P->scheme != MH_SCHEME_IMEX_EULER)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "allen_cahn_step needs a problem created with MH_SCHEME_IMEX_EULER");
    if (!(eps > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "eps must be positive");
    if (P->ext_mode == MH_EXT_ARRAY && !b_ext_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "MH_EXT_ARRAY needs b_ext_dev");
    if (!(gmres_tol > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "gmres_tol must be positive");
    const int64_t n = P->tree->n_nodes;
    // the problem's dt is eps * dt (alpha^2 = eps dt): the time step itself is dt / eps
    k_form_B_allen_cahn<<<mh_grid(n, 256), 256, 0, ctx->stream>>>(u_dev, P->region.p, P->d_ext_const.p, b_ext_dev,
                                                                  P->ext_mode, P->dt / eps, n, P->B.p);
    MH_LAUNCHED(ctx);
    return step_solve(ctx, P, f_next_dev, u_next_dev, sigma_dev, gmres_tol, prec, info);
}
