// Volume potential (Section 3.1, eq. volume_potential): U(x) = sum over leaves of
// int_leaf G(x - y) P(y) dA with G = K0(r/alpha)/(2 pi alpha^2) and P the leaf's q x q
// interpolant of B.  Evaluated by an adaptive multipole method on the device quadtree:
//
//   near  (U list): precomputed per-(level, configuration) q^2 x q^2 tables of the exact
//                   integrals of G times the source leaf's Lagrange basis (device kernel,
//                   graded tensor Gauss-Legendre rule);
//   P2M / M2M       K_n multipoles   M_n = int P(y) I_n(k rho) e^{-i n phi} dA / (2 pi alpha^2)
//   M2L (V list)    K_n -> I_n locals through Graf's addition theorem,
//   P2L (X list), M2P (W list), L2L, L2P,
// with k = 1/alpha, n = -p..p.  Expansions are scaled by I_n(k s_l) (s_l = box radius of
// level l) so that every coefficient and operator entry is O(1), and stored in a real
// form of length 2p+1 ([a_0, a_1, b_1, ..., a_p, b_p], M_{-n} = conj(M_n) for a real B).
//
// Every pass is a batch of small dense contractions "y_dst += T_op x_src" with the
// operator T_op chosen by (level, relative configuration).  Tasks are sorted by operator;
// a block stages one operator and up to 64 source vectors in shared memory and writes
// its products to a task-indexed buffer, and a segmented reduction sums the products of
// each destination in a fixed order (deterministic, no atomics).  The near tables form their
// own phase, which needs only the node values: it runs beside the multipole passes on a
// second stream and writes U first; the output phase then adds the far field.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <memory>
#include <tuple>

#include "bessel.cuh"
#include <cooperative_groups.h>

#include "mh_internal.cuh"

namespace {

constexpr int CHUNK = 64;   // tasks per block in the contraction kernel (32 where 64 does not fit)
constexpr int NGLN = 16;    // Gauss-Legendre points per panel in the near-table rule
constexpr int NGLQ = 32;    // Gauss-Legendre points per axis for the smooth P2M/P2L integrals

// ---------------- host Bessel functions (operator construction) ----------------

double h_k0(double z) {
    if (z <= 2.0) {
        const double y = 0.25 * z * z;
        double si = mh_ser_i0_h[MH_BESSEL_NSER - 1], sh = mh_ser_k0h_h[MH_BESSEL_NSER - 1];
        for (int k = MH_BESSEL_NSER - 2; k >= 0; --k) {
            si = si * y + mh_ser_i0_h[k];
            sh = sh * y + mh_ser_k0h_h[k];
        }
        return sh - (std::log(0.5 * z) + MH_EULER_GAMMA) * si;
    }
    double x = 4.0 / z - 1.0, b1 = 0, b2 = 0;
    for (int k = MH_CHEB_K0_N64 - 1; k >= 1; --k) {
        double t = 2 * x * b1 - b2 + mh_cheb_k0_h[k];
        b2 = b1;
        b1 = t;
    }
    return std::exp(-z) / std::sqrt(z) * (x * b1 - b2 + mh_cheb_k0_h[0]);
}

double h_k1(double z) {
    if (z <= 2.0) {
        const double y = 0.25 * z * z;
        double si = mh_ser_i1_h[MH_BESSEL_NSER - 1], sp = mh_ser_k1p_h[MH_BESSEL_NSER - 1];
        for (int k = MH_BESSEL_NSER - 2; k >= 0; --k) {
            si = si * y + mh_ser_i1_h[k];
            sp = sp * y + mh_ser_k1p_h[k];
        }
        return 1.0 / z + std::log(0.5 * z) * (0.5 * z) * si - 0.25 * z * sp;
    }
    double x = 4.0 / z - 1.0, b1 = 0, b2 = 0;
    for (int k = MH_CHEB_K1_N64 - 1; k >= 1; --k) {
        double t = 2 * x * b1 - b2 + mh_cheb_k1_h[k];
        b2 = b1;
        b1 = t;
    }
    return std::exp(-z) / std::sqrt(z) * (x * b1 - b2 + mh_cheb_k1_h[0]);
}

// K_0..K_nmax(z) by the (stable) forward recurrence K_{n+1} = K_{n-1} + (2n/z) K_n.
void h_kn_all(double z, int nmax, double* K) {
    K[0] = h_k0(z);
    if (nmax >= 1) K[1] = h_k1(z);
    for (int n = 1; n < nmax; ++n) K[n + 1] = K[n - 1] + (2.0 * n / z) * K[n];
}

// I_n(z) = sum_k (z/2)^{n+2k} / (k! (n+k)!)  (all terms positive).
double h_in(int n, double z) {
    if (n < 0) n = -n;
    if (z == 0.0) return n == 0 ? 1.0 : 0.0;
    const double h = 0.5 * z;
    double t = 1.0;
    for (int i = 1; i <= n; ++i) t *= h / i;
    double s = t, y = h * h;
    for (int k = 1; k < 2000; ++k) {
        t *= y / ((double)k * (n + k));
        s += t;
        if (t < 1e-17 * s) break;
    }
    return s;
}

// Complex operator T(m, n), m = 0..p, n = -p..p, on conjugate-symmetric vectors -> real
// (2p+1) x (2p+1) matrix acting on [a_0, a_1, b_1, ..., a_p, b_p].
template <class F>
void real_form(int p, F T, double* out /* row-major (2p+1)^2 */) {
    const int P = 2 * p + 1;
    std::fill(out, out + P * P, 0.0);
    for (int m = 0; m <= p; ++m)
        for (int n = 0; n <= p; ++n) {
            const std::complex<double> t = T(m, n);
            const std::complex<double> tc = n > 0 ? T(m, -n) : std::complex<double>(0.0, 0.0);
            const int ra = m == 0 ? 0 : 2 * m - 1, rb = 2 * m;
            const int ca = n == 0 ? 0 : 2 * n - 1, cb = 2 * n;
            // y_m += t x_n + tc conj(x_n),  x_n = a + i b
            out[ra * P + ca] += (t + tc).real();
            if (m > 0) out[rb * P + ca] += (t + tc).imag();
            if (n > 0) {
                out[ra * P + cb] += (tc - t).imag();
                if (m > 0) out[rb * P + cb] += (t - tc).real();
            }
        }
}

// ---------------- device kernels ----------------

struct NearCfg {
    double sx, sy, sw;   // source box centre relative to the target box centre, source width
    double tw;           // target box width
};

// Panels on [lo, hi] graded geometrically (ratio 4) toward c from the panel size delta;
// when c lies inside, both sides are graded toward it.
__device__ int grade_side(double a, double b, bool toward_a, double delta, double* pa, double* pb, int n) {
    const double L = b - a;
    double prev = 0.0, d = delta;
    while (d < L && n < 60) {
        if (toward_a) {
            pa[n] = a + prev;
            pb[n] = a + d;
        } else {
            pa[n] = b - d;
            pb[n] = b - prev;
        }
        ++n;
        prev = d;
        d *= 4.0;
    }
    if (toward_a) {
        pa[n] = a + prev;
        pb[n] = b;
    } else {
        pa[n] = a;
        pb[n] = b - prev;
    }
    return n + 1;
}

__device__ int make_panels(double lo, double hi, double c, double delta, double* pa, double* pb) {
    if (c > lo && c < hi) {
        int n = grade_side(lo, c, false, delta, pa, pb, 0);
        return grade_side(c, hi, true, delta, pa, pb, n);
    }
    return grade_side(lo, hi, c <= lo, delta, pa, pb, 0);
}

// One block per (configuration, target node i): row i of the q^2 x q^2 near table,
//   T[i][j] = int_source G(x_i - y) L_j(y) dA,
// by a tensor Gauss-Legendre rule on panels graded toward the target point.
__global__ void k_near_tables(const NearCfg* __restrict__ cfg, int q, const double* __restrict__ xi,
                              const double* __restrict__ gx, const double* __restrict__ gw, double inv_alpha,
                              double pref, double* out) {
    __shared__ double pxa[64], pxb[64], pya[64], pyb[64];
    __shared__ int npx, npy;
    __shared__ double sG[NGLN][NGLN + 1], sLx[16][NGLN], sLy[16][NGLN], sT[NGLN][17];
    const int qq = q * q;
    const int c = blockIdx.x / qq, i = blockIdx.x % qq;
    const NearCfg C = cfg[c];
    const double tx = 0.5 * C.tw * xi[i % q], ty = 0.5 * C.tw * xi[i / q];
    const double x0 = C.sx - 0.5 * C.sw, x1 = C.sx + 0.5 * C.sw, y0 = C.sy - 0.5 * C.sw, y1 = C.sy + 0.5 * C.sw;
    if (threadIdx.x == 0) {
        const double dx = fmax(fmax(x0 - tx, tx - x1), 0.0), dy = fmax(fmax(y0 - ty, ty - y1), 0.0);
        const double d = sqrt(dx * dx + dy * dy);
        const double delta = d > 0.0 ? 0.5 * d : C.sw * 3.7252902984619141e-09;   // 4^-14
        npx = make_panels(x0, x1, tx, delta, pxa, pxb);
        npy = make_panels(y0, y1, ty, delta, pya, pyb);
    }
    __syncthreads();
    const int t = threadIdx.x;
    double acc = 0.0;
    for (int ix = 0; ix < npx; ++ix)
        for (int iy = 0; iy < npy; ++iy) {
            const double hx = 0.5 * (pxb[ix] - pxa[ix]), mx = 0.5 * (pxb[ix] + pxa[ix]);
            const double hy = 0.5 * (pyb[iy] - pya[iy]), my = 0.5 * (pyb[iy] + pya[iy]);
            {
                const int u = t % NGLN, v = t / NGLN;
                const double X = mx + hx * gx[u], Y = my + hy * gx[v];
                const double r = sqrt((X - tx) * (X - tx) + (Y - ty) * (Y - ty));
                sG[v][u] = pref * mh_k0(r * inv_alpha) * hx * hy * gw[u] * gw[v];
            }
            if (t < q * NGLN) {
                const int a = t / NGLN, u = t % NGLN;
                const double sx = (mx + hx * gx[u] - C.sx) * (2.0 / C.sw);
                const double sy = (my + hy * gx[u] - C.sy) * (2.0 / C.sw);
                double lx = 1.0, ly = 1.0;
                for (int m = 0; m < q; ++m)
                    if (m != a) {
                        lx *= (sx - xi[m]) / (xi[a] - xi[m]);
                        ly *= (sy - xi[m]) / (xi[a] - xi[m]);
                    }
                sLx[a][u] = lx;
                sLy[a][u] = ly;
            }
            __syncthreads();
            if (t < NGLN * q) {
                const int v = t / q, a = t % q;
                double s = 0.0;
                for (int u = 0; u < NGLN; ++u) s += sG[v][u] * sLx[a][u];
                sT[v][a] = s;
            }
            __syncthreads();
            if (t < qq) {
                const int b = t / q, a = t % q;
                double s = 0.0;
                for (int v = 0; v < NGLN; ++v) s += sLy[b][v] * sT[v][a];
                acc += s;
            }
            __syncthreads();
        }
    if (t < qq) out[((int64_t)c * qq + i) * qq + t] = acc;
}

// Copies src[0..n) to shared memory at row-major position (e / cols, e % cols), leading
// dimension ld, with U independent loads in flight per thread (a load-then-store loop would
// wait on every global load in turn).  The position advances incrementally (one division per
// thread, not two per element).
template <typename TD, typename TS, int U = 8>
__device__ __forceinline__ void stage_rows(TD* dst, const TS* __restrict__ src, int n, int cols, int ld) {
    const int stride = blockDim.x;
    const int dc = stride % cols, dov = (stride / cols) * ld + dc;   // per stride: column, shared offset
    int c = (int)threadIdx.x % cols, o = ((int)threadIdx.x / cols) * ld + c;
    for (int e0 = threadIdx.x; e0 < n; e0 += U * stride) {
        TS v[U];
        int oo[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * stride;
            v[u] = e < n ? src[e] : TS(0);
            oo[u] = o;
            c += dc;
            o += dov;
            if (c >= cols) {
                c -= cols;
                o += ld - cols;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (e0 + u * stride < n) dst[oo[u]] = (TD)v[u];
    }
}

// Batched contraction: each block applies one operator (R x C, row-major) to up to CHUNK
// source vectors gathered from the pool `src` (the operators' precision: node values and
// expansions are kept in that precision, so the gather converts nothing) and writes the
// products to temp[task][R].  With task_dst given (phases where every destination has exactly
// one task and sources and destinations do not overlap) the product goes straight to
// dst[task_dst + r] (added when accumulate is set); dst is the expansion pool (TD = TOP) or the
// binary64 potentials (TD = double).
template <typename TOP, typename TD>
__global__ void k_apply(const TOP* __restrict__ ops, const int64_t* __restrict__ op_off,
                        const int32_t* __restrict__ op_C, const int32_t* __restrict__ chunk_op,
                        const int32_t* __restrict__ chunk_t0, const int64_t* __restrict__ task_src,
                        const TOP* src, int R, TOP* __restrict__ temp, const int64_t* __restrict__ task_dst,
                        int accumulate, TD* dst) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TOP* sA = reinterpret_cast<TOP*>(smem_raw);
    const int ch = blockIdx.x;
    const int op = chunk_op[ch];
    const int t0 = chunk_t0[ch];
    const int nt = chunk_t0[ch + 1] - t0;   // chunks never straddle two operators
    const int C = op_C[op];
    const int lda = C + 1;
    TOP* sX = sA + R * lda;
    const TOP* A = ops + op_off[op];
    if (nt == 1) {
        // a single source vector (operators owned by one leaf: dipole P2M / P2L): a GEMV that
        // reads every operator row once, coalesced, straight from global memory
        const int64_t s0 = task_src[t0];
        for (int e = threadIdx.x; e < C; e += blockDim.x) sA[e] = src[s0 + e];
        __syncthreads();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r = warp; r < R; r += nw) {
            const TOP* a = A + (int64_t)r * C;
            TOP acc = 0;
            for (int c = lane; c < C; c += 32) acc += a[c] * sA[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                if (task_dst) {
                    TD* y = dst + task_dst[t0] + r;
                    *y = accumulate ? *y + (TD)acc : (TD)acc;
                } else {
                    temp[(int64_t)t0 * R + r] = acc;
                }
            }
        }
        return;
    }
    stage_rows<TOP, TOP>(sA, A, R * C, C, lda);
    {   // gather the sources: element e is (task e / C, column e % C), advanced incrementally
        const int stride = blockDim.x, ne = nt * C;
        const int dc = stride % C, dt = stride / C;
        int c = (int)threadIdx.x % C, tt = (int)threadIdx.x / C;
        for (int e0 = threadIdx.x; e0 < ne; e0 += 4 * stride) {
            TOP v[4];
            int oo[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = e0 + u * stride < ne;
                v[u] = in ? src[task_src[t0 + tt] + c] : TOP(0);
                oo[u] = tt * lda + c;
                c += dc;
                tt += dt;
                if (c >= C) {
                    c -= C;
                    ++tt;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e0 + u * stride < ne) sX[oo[u]] = v[u];
        }
    }
    __syncthreads();
    // register tiles of 4 rows x 4 tasks: rows rg + RG i, tasks tg + TG j (strided so that the
    // operator and source loads of a warp fall in distinct banks); 8 shared loads per 16 FMAs
    const int RG = (R + 3) / 4, TG = (nt + 3) / 4;
    for (int tile = threadIdx.x; tile < RG * TG; tile += blockDim.x) {
        const int rg = tile % RG, tg = tile / RG;
        TOP acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0;
        const TOP* a0 = sA + (rg + 0 * RG < R ? rg + 0 * RG : 0) * lda;
        const TOP* a1 = sA + (rg + 1 * RG < R ? rg + 1 * RG : 0) * lda;
        const TOP* a2 = sA + (rg + 2 * RG < R ? rg + 2 * RG : 0) * lda;
        const TOP* a3 = sA + (rg + 3 * RG < R ? rg + 3 * RG : 0) * lda;
        const TOP* x0 = sX + (tg + 0 * TG < nt ? tg + 0 * TG : 0) * lda;
        const TOP* x1 = sX + (tg + 1 * TG < nt ? tg + 1 * TG : 0) * lda;
        const TOP* x2 = sX + (tg + 2 * TG < nt ? tg + 2 * TG : 0) * lda;
        const TOP* x3 = sX + (tg + 3 * TG < nt ? tg + 3 * TG : 0) * lda;
        for (int cc = 0; cc < C; ++cc) {
            const TOP av[4] = {a0[cc], a1[cc], a2[cc], a3[cc]};
            const TOP xv[4] = {x0[cc], x1[cc], x2[cc], x3[cc]};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * xv[j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = rg + i * RG;
            if (r >= R) break;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int tt = tg + j * TG;
                if (tt >= nt) break;
                if (task_dst) {
                    TD* y = dst + task_dst[t0 + tt] + r;
                    *y = accumulate ? *y + (TD)acc[i][j] : (TD)acc[i][j];
                } else {
                    temp[(int64_t)(t0 + tt) * R + r] = acc[i][j];
                }
            }
        }
    }
}

// ---- M2M / L2L chains without grid-wide barriers ----
// The level chains are latency chains (a few small matvecs per tree level).  Both kernels
// follow the data dependences instead of the levels:
//  * upward (M2M): one block per internal box whose children are all leaves.  A block forms
//    its box's multipole, then counts its arrival at the box's parent; the last child to
//    arrive carries on with the parent (arrival counters reset by that block), so the
//    critical path is the depth of the tree, not a barrier per level.
//    M[parent] = sum over the children c = 0..3 of T_c M[child_c]: thread (c, r) forms row r
//    of T_c M[child_c] (products in column order), the four are added in the order c = 0..3.
//  * downward (L2L): one block per internal box with leaf children.  The block recomputes,
//    in shared memory, the local expansions of the box's ancestors from the top internal
//    level down (L[child] = L_m2l[child] + T'_c L[parent], the same operations in the same
//    order as a level-by-level sweep), then adds T'_c L[box] to each leaf child.  Only leaf
//    expansions are written: they are the only ones read afterwards.
// Operators are stored transposed per (level, child position): ops[((l * 4 + c) * P + col) * P
// + row], so the threads of a warp read consecutive words.
template <typename T>
__device__ __forceinline__ T chain_fma(T a, T b, T c);
template <>
__device__ __forceinline__ float chain_fma<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double chain_fma<double>(double a, double b, double c) { return fma(a, b, c); }

// Row r of an operator times x: A points at row r of the transposed operator (A[cc * P] is
// entry (r, cc)), x is in shared memory; products added in column order.
template <typename TOP>
__device__ __forceinline__ TOP chain_dot(const TOP* __restrict__ A, int P, const TOP* x) {
    TOP acc = 0;
    for (int cc = 0; cc < P; ++cc) acc = chain_fma<TOP>(A[(int64_t)cc * P], x[cc], acc);
    return acc;
}

template <typename TOP>
__global__ void k_chain_up(const TOP* __restrict__ ops, int P, const int32_t* __restrict__ ready,
                           const int32_t* __restrict__ box, const int4* __restrict__ child,
                           const int32_t* __restrict__ lvl, const int32_t* __restrict__ next,
                           const int32_t* __restrict__ need, unsigned* cnt, int64_t base, TOP* vec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TOP* x = reinterpret_cast<TOP*>(smem_raw);   // 4 x P child expansions
    TOP* part = x + 4 * P;                        // 4 x P products
    __shared__ int go;
    const int c = threadIdx.x / P, r = threadIdx.x - c * P;
    const bool act = c < 4;
    int t = ready[blockIdx.x];
    for (;;) {
        const int4 ch4 = child[t];
        const int chc = c == 0 ? ch4.x : c == 1 ? ch4.y : c == 2 ? ch4.z : ch4.w;
        // children may have been written by other blocks of this launch: read through L2
        if (act) x[c * P + r] = chc >= 0 ? __ldcg(vec + base + (int64_t)chc * P + r) : TOP(0);
        __syncthreads();
        TOP acc = 0;
        if (act && chc >= 0) acc = chain_dot<TOP>(ops + (int64_t)(lvl[t] * 4 + c) * P * P + r, P, x + c * P);
        if (act) part[c * P + r] = acc;
        __syncthreads();
        if (threadIdx.x < P) {
            TOP s = part[r] + part[P + r];
            s += part[2 * P + r];
            s += part[3 * P + r];
            vec[base + (int64_t)box[t] * P + r] = s;
            __threadfence();
        }
        const int q = next[t];
        if (q < 0) return;
        __syncthreads();
        if (threadIdx.x == 0) go = atomicAdd(cnt + q, 1u) == (unsigned)(need[q] - 1);
        __syncthreads();
        if (!go) return;
        if (threadIdx.x == 0) cnt[q] = 0u;
        __threadfence();
        t = q;
    }
}

template <typename TOP>
__global__ void k_chain_down(const TOP* __restrict__ ops, int P, const int32_t* __restrict__ poff,
                             const int32_t* __restrict__ pbox, const int32_t* __restrict__ pop,
                             const int4* __restrict__ leaf, const int32_t* __restrict__ lop, int64_t base,
                             TOP* vec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TOP* x = reinterpret_cast<TOP*>(smem_raw);   // the running ancestor expansion
    const int c = threadIdx.x / P, r = threadIdx.x - c * P;
    const int k0 = poff[blockIdx.x], k1 = poff[blockIdx.x + 1];
    const int64_t PP = (int64_t)P * P;
    if (threadIdx.x < P) x[r] = vec[base + (int64_t)pbox[k0] * P + r];
    for (int k = k0 + 1; k < k1; ++k) {
        __syncthreads();
        TOP acc = 0;
        if (threadIdx.x < P) acc = chain_dot<TOP>(ops + (int64_t)pop[k] * PP + r, P, x);
        __syncthreads();
        if (threadIdx.x < P) x[r] = vec[base + (int64_t)pbox[k] * P + r] + acc;
    }
    __syncthreads();
    if (c < 4) {
        const int4 l4 = leaf[blockIdx.x];
        const int lc = c == 0 ? l4.x : c == 1 ? l4.y : c == 2 ? l4.z : l4.w;
        if (lc >= 0) vec[base + (int64_t)lc * P + r] += chain_dot<TOP>(ops + (lop[blockIdx.x] + c) * PP + r, P, x);
    }
}

inline int chain_threads(int P) { return (4 * P + 31) / 32 * 32; }

// Per destination (one warp each): dst[r] = (acc ? dst[r] : 0) + the sum of its tasks' products,
// in task order.  Binary64 products are summed in binary64; binary32 products in float-float
// (TwoSum: the sum of the products with binary64-like accuracy and no binary64 instruction per
// product), converted once per output.
template <typename TT, typename TD>
__global__ void k_reduce(const TT* __restrict__ temp, int R, const int64_t* __restrict__ dst_off,
                         const int32_t* __restrict__ dst_ptr, const int32_t* __restrict__ dst_task, int64_t n_dst,
                         int accumulate, TD* dst) {
    const int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (d >= n_dst) return;
    const int j0 = dst_ptr[d], j1 = dst_ptr[d + 1];
    TD* y = dst + dst_off[d];
    for (int r = lane; r < R; r += 32) {
        if (sizeof(TT) == 8) {
            double s = accumulate ? (double)y[r] : 0.0;
            for (int j = j0; j < j1; ++j) s += (double)temp[(int64_t)dst_task[j] * R + r];
            y[r] = (TD)s;
        } else {
            float hi = 0.f, lo = 0.f;
            for (int j = j0; j < j1; ++j) {
                const float v = (float)temp[(int64_t)dst_task[j] * R + r];
                const float t = hi + v;
                const float bb = t - hi;
                lo += (hi - (t - bb)) + (v - bb);
                hi = t;
            }
            if (sizeof(TD) == 8)
                y[r] = (TD)((accumulate ? (double)y[r] : 0.0) + ((double)hi + (double)lo));
            else
                y[r] = (TD)(accumulate ? (float)y[r] + (hi + lo) : hi + lo);
        }
    }
}

// ---------------- host structures ----------------

struct Task {
    int op;
    int64_t src, dst;
};

struct Phase {
    int R = 0;
    bool accumulate = false;
    bool direct = false;           // one task per destination: products written in place
    bool dst_out = false;          // destinations are the binary64 potentials (else expansions)
    dbuf<int64_t> task_dst;        // destination offset of every (sorted) task when direct
    double flops = 0, bytes = 0;   // per run: 2 R C per task; operators, sources, products, outputs
    int64_t n_tasks = 0, n_dst = 0, n_chunks = 0;
    int smem = 0;
    dbuf<int32_t> chunk_op, chunk_t0, dst_ptr, dst_task;
    dbuf<int64_t> task_src, dst_off;
    // binary32 form on the tensor cores: the tasks of operators with at least TC_MIN_TASKS tasks
    // in chunks of up to 128 (k_contract_tc), the others in the CUDA-core chunks ("rest");
    // both write the same products, the reduction is shared
    int64_t n_tc = 0, n_rest = 0, first_rest = 0;   // rest = CUDA-core chunks first_rest.. of chunk_op
    int tc_npad = 0, tc_kmax = 0;
    double tc_flops = 0, tc_bytes = 0;   // algorithmic work of the tensor-core launch (binary32 data)
    std::vector<int> tc_ops;
    std::vector<int64_t> tc_src_host;      // binary32 source offsets of the tensor-core tasks
    dbuf<int64_t> tc_src;                  // their rows in the split planes
    dbuf<int32_t> tc_chunk_op, tc_chunk_t0;
};

constexpr int TC_MIN_TASKS = 1;    // operators with fewer tasks stay on the CUDA cores
constexpr int TC_POOL_PAD = 16;    // slack floats after the binary32 pool (aligned-window gathers)
constexpr int TC_TASKS = 128;      // tasks per tensor-core chunk (rows of the MMA)

// Operator images of the tensor-core path for one operator pool.
// The pool's source vectors are also kept pre-split into three bfloat16 planes (rows padded to
// a multiple of 16 entries), refreshed by tc_split after each range is final, so that the
// tensor-core gather copies bytes instead of splitting every source once per task.
struct TcImages {
    dbuf<uint16_t> img;                // three bfloat16 parts per operator
    dbuf<int64_t> off;                 // per operator (-1: no image)
    dbuf<int32_t> kpad;                // per operator
    dbuf<int> err;                     // set by a tensor-core launch whose bounded wait gave up
    bool ready = false;
    struct Range {                     // count vectors of length len at src in the binary32 pool,
        int64_t src;                   // rows of S entries at dst in every plane
        int len;
        int64_t count;
        int S;
        int64_t dst;
    };
    std::vector<Range> ranges;
    int64_t plane = 0;                 // entries per plane
    dbuf<uint16_t> planes;             // 3 * plane
    // plane offset of the row of the vector starting at binary32 offset o (-1: none)
    int64_t map(int64_t o, int* S) const {
        for (const Range& r : ranges)
            if (o >= r.src && o < r.src + r.count * r.len && (o - r.src) % r.len == 0) {
                *S = r.S;
                return r.dst + (o - r.src) / r.len * r.S;
            }
        return -1;
    }
};

// Refresh the split planes of range k from the binary32 pool (after its values are final).
mh_status tc_split(mh_ctx* ctx, const TcImages& T, int k, const float* pool32) {
    if (!T.ready || !ctx->tensor_cores || k >= (int)T.ranges.size()) return MH_OK;
    const TcImages::Range& r = T.ranges[k];
    return tc_split_launch(ctx, pool32 + r.src, r.len, r.count, r.S, T.planes.p, T.plane, r.dst);
}

struct OpPool {
    std::vector<double> data;
    std::vector<int64_t> off;
    std::vector<int32_t> R, C;
    int add(int r, int c, const double* v) {
        off.push_back((int64_t)data.size());
        R.push_back(r);
        C.push_back(c);
        data.insert(data.end(), v, v + (size_t)r * c);
        return (int)off.size() - 1;
    }
};

// M2M / L2L of every level 2 <= l < L in parent-centric form (shared by the volume and the
// double-layer passes: same tree, same operators at the same pool offsets).
// Device description of the M2M / L2L chains (k_chain_up / k_chain_down).
struct DfChain {
    int64_t n_int = 0;                   // internal boxes of levels >= 2 (upward tasks)
    int64_t n_ready = 0;                 // of which all children are leaves
    int64_t n_down = 0;                  // internal boxes with leaf children (downward blocks)
    double flops = 0, bytes = 0;         // one sweep (either direction), algorithmic
    dbuf<int32_t> up_box, up_lvl, up_next, up_need, up_ready;
    dbuf<int4> up_child;
    dbuf<unsigned> up_cnt;
    dbuf<int32_t> dn_off, dn_box, dn_op, dn_lop;
    dbuf<int4> dn_leaf;
    dbuf<float> m2m32, l2l32;            // transposed operators, [level][position][col][row]
    dbuf<double> m2m64, l2l64;
};

struct DipData;
struct BieData;

struct VolData {
    double alpha = -1;
    int p = -1;
    // host copies kept for the dipole (double-layer) multipole pass
    OpPool pool_host;
    std::map<std::tuple<int, int, int, int>, int> m2l_key, m2p_key;
    std::vector<int> op_p2m, op_l2p;
    std::vector<std::array<int, 4>> op_m2m, op_l2l;
    std::unique_ptr<DipData> dip;
    std::unique_ptr<BieData> bie;        // on-surface double layer (matrix-free BIE operator)
    int P = 0, qq = 0;
    int64_t B_off = 0, U_off = 0, M_off = 0, L_off = 0, vec_len = 0;
    dbuf<double> ops64, vec, temp;
    dbuf<float> ops32, vec32;            // vec32: binary32 mirror of vec (node values, expansions)
    dbuf<int64_t> d_op_off;
    dbuf<int32_t> d_op_C;
    std::vector<int> op_C;
    std::unique_ptr<Phase> p2m, m2l, out;
    std::unique_ptr<Phase> near;                      // U list: near tables on the node values
    dbuf<double> temp_near;                           // its products (it may run beside the others)
    bool near_cover = true;                           // every leaf has a U-list task
    SideStream side;
    std::unique_ptr<DfChain> chain;                   // M2M / L2L chains
    int64_t temp_len = 0;
    int64_t n_near_tables = 0;
    TcImages tc;                                      // tensor-core images (mixed precision)
};

// ranges: the split ranges of the pool (tensor-core sources); an operator takes the tensor-core
// form only if every one of its tasks reads a whole vector of a range whose length is its C.
mh_status build_phase(mh_ctx* ctx, std::vector<Task>& tasks, int R, bool accumulate, const std::vector<int>& op_C,
                      Phase* ph, int64_t* temp_need, const std::vector<TcImages::Range>* ranges = nullptr) {
    ph->R = R;
    ph->accumulate = accumulate;
    ph->n_tasks = (int64_t)tasks.size();
    // operators of the tensor-core form: >= TC_MIN_TASKS tasks and at most 64 x 64
    std::map<int, int64_t> per_op;
    for (const Task& t : tasks) per_op[t.op] += 1;
    std::map<int, bool> on_tc;
    for (auto& kv : per_op)
        on_tc[kv.first] = ranges && R <= 64 && kv.second >= TC_MIN_TASKS && op_C[kv.first] <= 64;
    if (ranges)
        for (const Task& t : tasks) {
            if (!on_tc[t.op]) continue;
            bool found = false;
            for (const TcImages::Range& r : *ranges)
                found = found || (r.len == op_C[t.op] && t.src >= r.src && t.src < r.src + r.count * r.len &&
                                  (t.src - r.src) % r.len == 0);
            if (!found) on_tc[t.op] = false;
        }
    // sort by (CUDA-core form, operator), stable: keeps the generation order inside an operator
    // and puts the tensor-core operators' tasks first, so that both forms cover contiguous
    // ranges of the sorted tasks (the binary64 form runs over all of them)
    std::vector<int64_t> order(tasks.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int64_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const bool ra = !on_tc[tasks[a].op], rb = !on_tc[tasks[b].op];
        return ra != rb ? rb : tasks[a].op < tasks[b].op;
    });
    std::vector<int64_t> src(tasks.size());
    std::vector<int32_t> cop, ct0;
    int maxC = 1;
    for (const Task& t : tasks) maxC = std::max(maxC, op_C[t.op]);
    // tasks per block: CHUNK (more threads busy in the 4 x 4 tiling, the operator staged for
    // more vectors) unless the staged operator and sources would not fit
    const int chunk = (size_t)(R + CHUNK) * (maxC + 1) * sizeof(double) <= 160 * 1024 ? CHUNK : 32;
    for (size_t s = 0; s < order.size(); ++s) {
        const Task& t = tasks[order[s]];
        src[s] = t.src;
        if (s == 0 || tasks[order[s - 1]].op != t.op || (int64_t)(s - ct0.back()) >= chunk) {
            cop.push_back(t.op);
            ct0.push_back((int32_t)s);
        }
        ph->flops += 2.0 * R * op_C[t.op];
        ph->bytes += 8.0 * op_C[t.op] + 16.0 * R;   // source vector, product write + read
    }
    for (size_t c = 0; c < cop.size(); ++c) ph->bytes += 8.0 * R * op_C[cop[c]];   // operator per chunk
    ph->n_chunks = (int64_t)cop.size();
    ct0.push_back((int32_t)order.size());   // end of the last chunk
    // tensor-core chunks over the leading tasks: ceil(n / 128) nearly equal chunks per
    // operator; the CUDA-core chunks after them are the tail of the chunk list above
    std::vector<int32_t> tcop, tct0;
    int64_t n_tc_tasks = 0;
    {
        size_t s = 0;
        while (s < order.size() && on_tc[tasks[order[s]].op]) {
            const int op = tasks[order[s]].op;
            size_t e = s;
            while (e < order.size() && tasks[order[e]].op == op) ++e;
            const int64_t n = (int64_t)(e - s);
            const int64_t nc = (n + TC_TASKS - 1) / TC_TASKS;
            for (int64_t c = 0; c < nc; ++c) {
                tcop.push_back(op);
                tct0.push_back((int32_t)(s + n * c / nc));
            }
            // 2 R C flop per task; bytes: the operator once per chunk (at binary32 size), every
            // task's binary32 source vector and product
            ph->tc_flops += 2.0 * R * op_C[op] * n;
            ph->tc_bytes += 4.0 * R * op_C[op] * nc + 4.0 * (op_C[op] + R) * n;
            ph->tc_kmax = std::max(ph->tc_kmax, tc_pad_cols(op_C[op]));
            ph->tc_ops.push_back(op);
            s = e;
        }
        n_tc_tasks = (int64_t)s;
    }
    tct0.push_back((int32_t)n_tc_tasks);
    ph->tc_src_host.assign(src.begin(), src.begin() + n_tc_tasks);
    ph->n_tc = (int64_t)tcop.size();
    ph->tc_npad = tc_pad_rows(R);
    ph->first_rest = 0;
    while (ph->first_rest < ph->n_chunks && ct0[ph->first_rest] < n_tc_tasks) ++ph->first_rest;
    ph->n_rest = ph->n_chunks - ph->first_rest;
    // destinations: tasks grouped by destination in generation order
    std::vector<int64_t> rank(tasks.size());
    for (size_t s = 0; s < order.size(); ++s) rank[order[s]] = (int64_t)s;
    std::map<int64_t, std::vector<int32_t>> bydst;
    for (size_t i = 0; i < tasks.size(); ++i) bydst[tasks[i].dst].push_back((int32_t)rank[i]);
    std::vector<int64_t> doff;
    std::vector<int32_t> dptr{0}, dtask;
    for (auto& kv : bydst) {
        doff.push_back(kv.first);
        dtask.insert(dtask.end(), kv.second.begin(), kv.second.end());
        dptr.push_back((int32_t)dtask.size());
    }
    ph->n_dst = (int64_t)doff.size();
    // direct mode: a single task per destination and source / destination ranges apart
    if (ph->n_dst == ph->n_tasks && ph->n_tasks > 0) {
        int64_t smin = INT64_MAX, smax = 0, dmin = INT64_MAX, dmax = 0;
        for (const Task& t : tasks) {
            smin = std::min(smin, t.src);
            smax = std::max(smax, t.src + op_C[t.op]);
            dmin = std::min(dmin, t.dst);
            dmax = std::max(dmax, t.dst + R);
        }
        ph->direct = smax <= dmin || dmax <= smin;
    }
    ph->smem = (int)((R + chunk) * (maxC + 1) * sizeof(double));
    if (ph->smem > 160 * 1024)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "contraction operator too large for shared memory (%d x %d)", R, maxC);
    cudaStream_t st = ctx->stream;
    auto up32 = [&](dbuf<int32_t>& b, const std::vector<int32_t>& v) -> mh_status {
        MH_ALLOC(ctx, b, std::max<size_t>(v.size(), 1));
        if (!v.empty()) MH_CUDA(ctx, cudaMemcpyAsync(b.p, v.data(), v.size() * 4, cudaMemcpyHostToDevice, st));
        return MH_OK;
    };
    auto up64 = [&](dbuf<int64_t>& b, const std::vector<int64_t>& v) -> mh_status {
        MH_ALLOC(ctx, b, std::max<size_t>(v.size(), 1));
        if (!v.empty()) MH_CUDA(ctx, cudaMemcpyAsync(b.p, v.data(), v.size() * 8, cudaMemcpyHostToDevice, st));
        return MH_OK;
    };
    MH_TRY(up32(ph->chunk_op, cop));
    MH_TRY(up32(ph->chunk_t0, ct0));
    MH_TRY(up32(ph->tc_chunk_op, tcop));
    MH_TRY(up32(ph->tc_chunk_t0, tct0));
    MH_TRY(up32(ph->dst_ptr, dptr));
    MH_TRY(up32(ph->dst_task, dtask));
    MH_TRY(up64(ph->task_src, src));
    MH_TRY(up64(ph->dst_off, doff));
    if (ph->direct) {
        std::vector<int64_t> tdst(tasks.size());
        for (size_t q = 0; q < order.size(); ++q) tdst[q] = tasks[order[q]].dst;
        MH_TRY(up64(ph->task_dst, tdst));
    }
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    *temp_need = std::max<int64_t>(*temp_need, ph->n_tasks * R);
    return MH_OK;
}

// Tensor-core images (three-part bfloat16 split of the binary64 operator) of every operator that one of
// `phases` runs on the tensor cores.  ops64: the pool's operators (binary64, row-major at off).
mh_status build_tc_images(mh_ctx* ctx, const double* ops64, const std::vector<int64_t>& off,
                          const std::vector<int32_t>& R, const std::vector<int32_t>& C,
                          std::initializer_list<Phase*> phases, const std::vector<TcImages::Range>& ranges,
                          TcImages* T) {
    std::vector<int64_t> ioff(off.size(), -1);
    std::vector<int32_t> kp(off.size(), 0);
    size_t total = 0;
    for (const Phase* ph : phases)
        for (int op : ph->tc_ops) {
            if (ioff[op] >= 0) continue;
            if (tc_pad_rows(R[op]) != ph->tc_npad)
                return mh_fail(ctx, MH_ERR_INVALID_ARG, "tensor-core operator rows differ from its phase");
            bool len_ok = false;   // the operator's columns are the length of one split range
            for (const TcImages::Range& r : ranges) len_ok = len_ok || r.len == C[op];
            if (!len_ok)
                return mh_fail(ctx, MH_ERR_INVALID_ARG, "tensor-core operator columns match no source vector length");
            ioff[op] = (int64_t)total;
            kp[op] = tc_pad_cols(C[op]);
            total += 3 * (size_t)tc_pad_rows(R[op]) * kp[op];
        }
    T->ready = total > 0;
    if (!T->ready) return MH_OK;
    // split planes: every range's rows, padded to a multiple of 16 entries
    T->ranges = ranges;
    T->plane = 0;
    for (TcImages::Range& r : T->ranges) {
        r.S = (r.len + 15) / 16 * 16;
        r.dst = T->plane;
        T->plane += r.count * r.S;
    }
    MH_ALLOC(ctx, T->planes, std::max<int64_t>(3 * T->plane, 8));
    MH_CUDA(ctx, cudaMemsetAsync(T->planes.p, 0, std::max<int64_t>(3 * T->plane, 8) * 2, ctx->stream));
    for (Phase* ph : phases) {
        std::vector<int64_t> rows(ph->tc_src_host.size());
        for (size_t i = 0; i < rows.size(); ++i) {
            int S = 0;
            rows[i] = T->map(ph->tc_src_host[i], &S);
            if (rows[i] < 0)
                return mh_fail(ctx, MH_ERR_INVALID_ARG, "tensor-core source %lld is not a vector of the split ranges",
                               (long long)ph->tc_src_host[i]);
        }
        MH_ALLOC(ctx, ph->tc_src, std::max<size_t>(rows.size(), 1));
        if (!rows.empty())
            MH_CUDA(ctx, cudaMemcpyAsync(ph->tc_src.p, rows.data(), rows.size() * 8, cudaMemcpyHostToDevice,
                                         ctx->stream));
    }
    std::vector<uint16_t> img(total);
    for (size_t op = 0; op < off.size(); ++op)
        if (ioff[op] >= 0)
            tc_operator_image(ops64 + off[op], R[op], C[op], tc_pad_rows(R[op]), kp[op], img.data() + ioff[op]);
    cudaStream_t st = ctx->stream;
    MH_ALLOC(ctx, T->img, total);
    MH_ALLOC(ctx, T->off, off.size());
    MH_ALLOC(ctx, T->kpad, off.size());
    MH_ALLOC(ctx, T->err, 1);
    MH_CUDA(ctx, cudaMemcpyAsync(T->img.p, img.data(), total * 2, cudaMemcpyHostToDevice, st));
    MH_CUDA(ctx, cudaMemcpyAsync(T->off.p, ioff.data(), ioff.size() * 8, cudaMemcpyHostToDevice, st));
    MH_CUDA(ctx, cudaMemcpyAsync(T->kpad.p, kp.data(), kp.size() * 4, cudaMemcpyHostToDevice, st));
    MH_CUDA(ctx, cudaMemsetAsync(T->err.p, 0, sizeof(int), st));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    MH_TRY(tc_prepare(ctx));
    return MH_OK;
}

// Expansion pool of the operators' precision: binary64 uses the main pool itself, binary32 its
// float mirror (same layout).
template <typename TOP>
inline TOP* typed_pool(dbuf<double>& v64, dbuf<float>& v32);
template <>
inline double* typed_pool<double>(dbuf<double>& v64, dbuf<float>&) { return v64.p; }
template <>
inline float* typed_pool<float>(dbuf<double>&, dbuf<float>& v32) { return v32.p; }

template <typename TOP>
mh_status run_phase_on(mh_ctx* ctx, const TOP* ops, const int64_t* op_off, const int32_t* op_C, TOP* pool,
                       double* out, double* temp, const Phase* ph, const char* region,
                       const TcImages* tc = nullptr) {
    if (ph->n_tasks == 0) return MH_OK;
    const int smem = (int)(ph->smem / sizeof(double) * sizeof(TOP));
    // binary32 with images: the leading operators on the tensor cores, the rest on the CUDA cores
    const bool on_tc = sizeof(TOP) == 4 && tc && tc->ready && ctx->tensor_cores && ph->n_tc > 0;
    prof_scope ps(ctx, region, ph->flops, ph->bytes + 8.0 * ph->R * ph->n_dst * (ph->accumulate ? 2 : 1));
    TOP* tmp = reinterpret_cast<TOP*>(temp);   // sized in binary64 words: room for either type
    const int acc = ph->accumulate ? 1 : 0;
    const int64_t* tdst = ph->direct ? ph->task_dst.p : nullptr;
    const unsigned rg = (unsigned)mh_grid(ph->n_dst * 32, 256);
    const int64_t c0 = on_tc ? ph->first_rest : 0;          // first CUDA-core chunk
    const unsigned ncc = (unsigned)(ph->n_chunks - c0);     // CUDA-core chunks
    if (on_tc) {
        tc_launch a;
        a.img = tc->img.p;
        a.img_off = tc->off.p;
        a.kpad = tc->kpad.p;
        a.op_C = op_C;
        a.chunk_op = ph->tc_chunk_op.p;
        a.chunk_t0 = ph->tc_chunk_t0.p;
        a.n_chunks = ph->n_tc;
        a.spl = tc->planes.p;
        a.plane = tc->plane;
        a.tc_src = ph->tc_src.p;
        a.R = ph->R;
        a.npad = ph->tc_npad;
        a.kmax = ph->tc_kmax;
        a.temp = reinterpret_cast<float*>(temp);
        a.task_dst = tdst;
        a.accumulate = acc;
        a.dst = ph->dst_out ? static_cast<void*>(out) : static_cast<void*>(pool);
        a.dst_double = ph->dst_out;
        a.err = tc->err.p;
        // the tensor-core launch alone is also timed in "<region>_tc"
        prof_scope pt(ctx, std::strcmp(region, "volume_contract") == 0 ? "volume_contract_tc" : "dlp_fmm_contract_tc",
                      ph->tc_flops, ph->tc_bytes);
        MH_TRY(tc_contract_launch(ctx, a));
    }
    if (ph->dst_out) {
        if (ncc) {
            k_apply<TOP, double><<<ncc, 256, smem, ctx->stream>>>(ops, op_off, op_C, ph->chunk_op.p + c0,
                                                                  ph->chunk_t0.p + c0, ph->task_src.p, pool, ph->R,
                                                                  tmp, tdst, acc, out);
            MH_LAUNCHED(ctx);
        }
        if (!ph->direct) {
            k_reduce<TOP, double><<<rg, 256, 0, ctx->stream>>>(tmp, ph->R, ph->dst_off.p, ph->dst_ptr.p,
                                                               ph->dst_task.p, ph->n_dst, acc, out);
            MH_LAUNCHED(ctx);
        }
    } else {
        if (ncc) {
            k_apply<TOP, TOP><<<ncc, 256, smem, ctx->stream>>>(ops, op_off, op_C, ph->chunk_op.p + c0,
                                                               ph->chunk_t0.p + c0, ph->task_src.p, pool, ph->R, tmp,
                                                               tdst, acc, pool);
            MH_LAUNCHED(ctx);
        }
        if (!ph->direct) {
            k_reduce<TOP, TOP><<<rg, 256, 0, ctx->stream>>>(tmp, ph->R, ph->dst_off.p, ph->dst_ptr.p,
                                                            ph->dst_task.p, ph->n_dst, acc, pool);
            MH_LAUNCHED(ctx);
        }
    }
    return MH_OK;
}

template <typename TOP>
mh_status run_chain(mh_ctx* ctx, const DfChain* ch, int P, int64_t m_base, int64_t l_base, TOP* vec,
                    bool upward, const char* region) {
    // the level chains are timed in their own region: "<pass>_chain"
    if (!ch || ch->n_int == 0) return MH_OK;
    prof_scope ps(ctx, region, ch->flops, ch->bytes);
    const bool f32 = sizeof(TOP) == 4;
    const TOP* ops = reinterpret_cast<const TOP*>(upward ? (f32 ? (const void*)ch->m2m32.p : (const void*)ch->m2m64.p)
                                                         : (f32 ? (const void*)ch->l2l32.p : (const void*)ch->l2l64.p));
    const int nt = chain_threads(P);
    if (upward) {
        k_chain_up<TOP><<<(unsigned)ch->n_ready, nt, 8 * P * sizeof(TOP), ctx->stream>>>(
            ops, P, ch->up_ready.p, ch->up_box.p, ch->up_child.p, ch->up_lvl.p, ch->up_next.p, ch->up_need.p,
            ch->up_cnt.p, m_base, vec);
    } else {
        if (ch->n_down == 0) return MH_OK;
        k_chain_down<TOP><<<(unsigned)ch->n_down, nt, P * sizeof(TOP), ctx->stream>>>(
            ops, P, ch->dn_off.p, ch->dn_box.p, ch->dn_op.p, ch->dn_leaf.p, ch->dn_lop.p, l_base, vec);
    }
    MH_LAUNCHED(ctx);
    return MH_OK;
}

template <typename TOP>
mh_status run_phase(mh_ctx* ctx, VolData* V, const TOP* ops, const Phase* ph) {
    return run_phase_on<TOP>(ctx, ops, V->d_op_off.p, V->d_op_C.p, typed_pool<TOP>(V->vec, V->vec32), V->vec.p,
                             V->temp.p, ph, "volume_contract", &V->tc);
}

struct HostTree {
    std::vector<int32_t> boxes, box_leaf, leaf_box;
    std::vector<int32_t> off[4], item[4];
};

mh_status fetch_tree(mh_ctx* ctx, const mh_tree* t, HostTree* h) {
    cudaStream_t st = ctx->stream;
    h->boxes.resize(3 * t->n_boxes);
    h->box_leaf.resize(t->n_boxes);
    h->leaf_box.resize(t->n_leaves);
    MH_CUDA(ctx, cudaMemcpyAsync(h->boxes.data(), t->boxes.p, 3 * t->n_boxes * 4, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaMemcpyAsync(h->box_leaf.data(), t->box_leaf.p, t->n_boxes * 4, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaMemcpyAsync(h->leaf_box.data(), t->leaf_box.p, t->n_leaves * 4, cudaMemcpyDeviceToHost, st));
    for (int w = 0; w < 4; ++w) {
        h->off[w].resize(t->n_boxes + 1);
        h->item[w].resize(std::max<int64_t>(t->list_len[w], 1));
        MH_CUDA(ctx, cudaMemcpyAsync(h->off[w].data(), t->list_off[w].p, (t->n_boxes + 1) * 4, cudaMemcpyDeviceToHost,
                                     st));
        if (t->list_len[w])
            MH_CUDA(ctx, cudaMemcpyAsync(h->item[w].data(), t->list_item[w].p, t->list_len[w] * 4,
                                         cudaMemcpyDeviceToHost, st));
    }
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    return MH_OK;
}

// Build every operator and pass of the multipole method for (tree, alpha, p).
// M2M / L2L chains (k_chain_up / k_chain_down) of tree t: the internal boxes of levels
// 2 <= l < L with their children.  With `active`, only active boxes take part (an inactive
// child counts as absent).
mh_status build_chain(mh_ctx* ctx, const mh_tree* t, const HostTree& h, int P, const OpPool& pool,
                      const std::vector<std::array<int, 4>>& op_m2m, const std::vector<std::array<int, 4>>& op_l2l,
                      const std::vector<char>* active, std::unique_ptr<DfChain>* out) {
    const int64_t nb = t->n_boxes;
    const int L = t->max_level;
    auto lev = [&](int b) { return h.boxes[3 * b]; };
    {
        std::vector<int32_t> child(4 * nb);
        MH_CUDA(ctx, cudaMemcpyAsync(child.data(), t->box_child.p, 4 * nb * 4, cudaMemcpyDeviceToHost, ctx->stream));
        MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        std::unique_ptr<DfChain> ch(new DfChain());
        std::vector<int32_t> idx(nb, -1), parent(nb, -1), quad(nb, -1);
        if (active)   // children outside the active set are left out (zero expansions, no use)
            for (int64_t b = 0; b < nb; ++b)
                for (int c = 0; c < 4; ++c)
                    if (child[4 * b + c] >= 0 && !(*active)[child[4 * b + c]]) child[4 * b + c] = -1;
        for (int64_t b = 0; b < nb; ++b)
            for (int c = 0; c < 4; ++c)
                if (child[4 * b + c] >= 0) {
                    parent[child[4 * b + c]] = (int32_t)b;
                    quad[child[4 * b + c]] = c;
                }
        std::vector<int32_t> ubox, ulvl, unext, uneed, uready;
        std::vector<int4> uchild;
        std::vector<int64_t> npar(L + 1, 0), nchild(L + 1, 0);
        for (int64_t b = 0; b < nb; ++b) {
            const int l = lev((int)b);
            if (h.box_leaf[b] >= 0 || l < 2 || l >= L || (active && !(*active)[b])) continue;
            int cnt = 0;
            for (int c = 0; c < 4; ++c) cnt += child[4 * b + c] >= 0;
            if (!cnt) continue;
            idx[b] = (int32_t)ubox.size();
            ubox.push_back((int32_t)b);
            ulvl.push_back(l);
            uchild.push_back(make_int4(child[4 * b], child[4 * b + 1], child[4 * b + 2], child[4 * b + 3]));
            npar[l] += 1;
            nchild[l] += cnt;
        }
        for (int l = 2; l < L; ++l)
            if (npar[l]) {
                ch->flops += 2.0 * P * P * nchild[l];
                ch->bytes += 8.0 * (4.0 * P * P + 2.0 * P * (nchild[l] + npar[l]));
            }
        const int64_t ni = (int64_t)ubox.size();
        ch->n_int = ni;
        unext.assign(ni, -1);
        uneed.assign(ni, 0);
        // downward blocks: internal boxes with leaf children, each with its internal ancestors
        std::vector<int32_t> doff{0}, dbox, dop, dlop;
        std::vector<int4> dleaf;
        for (int64_t i = 0; i < ni; ++i) {
            const int b = ubox[i];
            if (parent[b] >= 0 && idx[parent[b]] >= 0) unext[i] = idx[parent[b]];
            int leaves[4] = {-1, -1, -1, -1};
            bool any_leaf = false;
            for (int c = 0; c < 4; ++c) {
                const int cb = child[4 * b + c];
                if (cb < 0) continue;
                if (idx[cb] >= 0)
                    uneed[i] += 1;
                else if (h.box_leaf[cb] >= 0) {
                    leaves[c] = cb;
                    any_leaf = true;
                }
            }
            if (uneed[i] == 0) uready.push_back((int32_t)i);
            if (!any_leaf) continue;
            std::vector<int32_t> path{b};
            while (parent[path.back()] >= 0 && idx[parent[path.back()]] >= 0) path.push_back(parent[path.back()]);
            for (size_t k = path.size(); k-- > 0;) {
                const int e = path[k];
                dbox.push_back(e);
                dop.push_back(k + 1 == path.size() ? -1 : lev(parent[e]) * 4 + quad[e]);
            }
            doff.push_back((int32_t)dbox.size());
            dleaf.push_back(make_int4(leaves[0], leaves[1], leaves[2], leaves[3]));
            dlop.push_back(ulvl[i] * 4);
        }
        ch->n_ready = (int64_t)uready.size();
        ch->n_down = (int64_t)dleaf.size();
        // operators, transposed per (level, child position)
        const size_t PP = (size_t)P * P;
        std::vector<double> tm((size_t)L * 4 * PP, 0.0), tl((size_t)L * 4 * PP, 0.0);
        for (int l = 2; l < L; ++l) {
            if (!npar[l]) continue;
            for (int c = 0; c < 4; ++c) {
                const double* om = pool.data.data() + pool.off[op_m2m[l][c]];
                const double* ol = pool.data.data() + pool.off[op_l2l[l][c]];
                for (int r = 0; r < P; ++r)
                    for (int cc = 0; cc < P; ++cc) {
                        tm[(l * 4 + c) * PP + (size_t)cc * P + r] = om[(size_t)r * P + cc];
                        tl[(l * 4 + c) * PP + (size_t)cc * P + r] = ol[(size_t)r * P + cc];
                    }
            }
        }
        std::vector<float> tm32(tm.begin(), tm.end()), tl32(tl.begin(), tl.end());
        cudaStream_t cs = ctx->stream;
        auto up_i = [&](dbuf<int32_t>& d, const std::vector<int32_t>& v) -> mh_status {
            MH_ALLOC(ctx, d, std::max<size_t>(v.size(), 1));
            if (!v.empty()) MH_CUDA(ctx, cudaMemcpyAsync(d.p, v.data(), v.size() * 4, cudaMemcpyHostToDevice, cs));
            return MH_OK;
        };
        auto up_4 = [&](dbuf<int4>& d, const std::vector<int4>& v) -> mh_status {
            MH_ALLOC(ctx, d, std::max<size_t>(v.size(), 1));
            if (!v.empty()) MH_CUDA(ctx, cudaMemcpyAsync(d.p, v.data(), v.size() * 16, cudaMemcpyHostToDevice, cs));
            return MH_OK;
        };
        MH_TRY(up_i(ch->up_box, ubox));
        MH_TRY(up_i(ch->up_lvl, ulvl));
        MH_TRY(up_i(ch->up_next, unext));
        MH_TRY(up_i(ch->up_need, uneed));
        MH_TRY(up_i(ch->up_ready, uready));
        MH_TRY(up_4(ch->up_child, uchild));
        MH_TRY(up_i(ch->dn_off, doff));
        MH_TRY(up_i(ch->dn_box, dbox));
        MH_TRY(up_i(ch->dn_op, dop));
        MH_TRY(up_i(ch->dn_lop, dlop));
        MH_TRY(up_4(ch->dn_leaf, dleaf));
        MH_ALLOC(ctx, ch->up_cnt, std::max<int64_t>(ni, 1));
        MH_CUDA(ctx, cudaMemsetAsync(ch->up_cnt.p, 0, std::max<int64_t>(ni, 1) * sizeof(unsigned), cs));
        MH_ALLOC(ctx, ch->m2m32, tm32.size());
        MH_ALLOC(ctx, ch->l2l32, tl32.size());
        MH_ALLOC(ctx, ch->m2m64, tm.size());
        MH_ALLOC(ctx, ch->l2l64, tl.size());
        MH_CUDA(ctx, cudaMemcpyAsync(ch->m2m32.p, tm32.data(), tm32.size() * 4, cudaMemcpyHostToDevice, cs));
        MH_CUDA(ctx, cudaMemcpyAsync(ch->l2l32.p, tl32.data(), tl32.size() * 4, cudaMemcpyHostToDevice, cs));
        MH_CUDA(ctx, cudaMemcpyAsync(ch->m2m64.p, tm.data(), tm.size() * 8, cudaMemcpyHostToDevice, cs));
        MH_CUDA(ctx, cudaMemcpyAsync(ch->l2l64.p, tl.data(), tl.size() * 8, cudaMemcpyHostToDevice, cs));
        MH_CUDA(ctx, cudaStreamSynchronize(cs));
        *out = std::move(ch);
    }
    return MH_OK;
}

mh_status volume_setup(mh_ctx* ctx, mh_tree* t, double alpha, int p, VolData* V) {
    const int q = t->q, qq = q * q, P = 2 * p + 1, L = t->max_level;
    const double k = 1.0 / alpha, pref = 1.0 / (2.0 * MH_PI * alpha * alpha);
    const double W = t->box[2];
    V->alpha = alpha;
    V->p = p;
    V->P = P;
    V->qq = qq;
    HostTree h;
    MH_TRY(fetch_tree(ctx, t, &h));
    const int64_t nb = t->n_boxes, nl = t->n_leaves;
    V->B_off = 0;
    V->U_off = nl * qq;
    V->M_off = 2 * nl * qq;
    V->L_off = V->M_off + nb * P;
    V->vec_len = V->L_off + nb * P;
    auto lev = [&](int b) { return h.boxes[3 * b]; };
    auto bx = [&](int b) { return h.boxes[3 * b + 1]; };
    auto by = [&](int b) { return h.boxes[3 * b + 2]; };
    auto width = [&](int l) { return W / (double)(1 << l); };
    // level scales: s_l = box radius, I_n(k s_l) for n = 0..p
    std::vector<std::vector<double>> Is(L + 1, std::vector<double>(p + 1));
    for (int l = 0; l <= L; ++l)
        for (int n = 0; n <= p; ++n) {
            Is[l][n] = h_in(n, k * width(l) * 0.70710678118654752);
            if (!(Is[l][n] > 1e-300) || !std::isfinite(Is[l][n]))
                return mh_fail(ctx, MH_ERR_NUMERIC, "expansion scale I_%d(%g) out of range at level %d", n,
                               k * width(l) * 0.707, l);
        }
    std::vector<double> glx(NGLQ), glw(NGLQ), qx(q), qw(q), g16x(NGLN), g16w(NGLN);
    mh_gauss_legendre(NGLQ, glx.data(), glw.data());
    mh_gauss_legendre(q, qx.data(), qw.data());
    mh_gauss_legendre(NGLN, g16x.data(), g16w.data());
    // Lagrange basis of the leaf nodes at the 32-point rule: LG[a * NGLQ + u] = l_a(glx[u])
    std::vector<double> LG((size_t)q * NGLQ);
    for (int a = 0; a < q; ++a)
        for (int u = 0; u < NGLQ; ++u) {
            double v = 1.0;
            for (int m = 0; m < q; ++m)
                if (m != a) v *= (glx[u] - qx[m]) / (qx[a] - qx[m]);
            LG[a * NGLQ + u] = v;
        }
    auto lag = [&](int a, int u) { return LG[a * NGLQ + u]; };
    OpPool pool;
    std::vector<double> buf;
    // ---- P2M and L2P per level ----
    std::vector<int> op_p2m(L + 1, -1), op_l2p(L + 1, -1);
    for (int l = 2; l <= L; ++l) {
        const double w = width(l);
        buf.assign((size_t)P * qq, 0.0);
        for (int v = 0; v < NGLQ; ++v)
            for (int u = 0; u < NGLQ; ++u) {
                const double X = 0.5 * w * glx[u], Y = 0.5 * w * glx[v];
                const double wt = 0.25 * w * w * glw[u] * glw[v] * pref;
                const double rho = std::hypot(X, Y), ph = std::atan2(Y, X);
                for (int n = 0; n <= p; ++n) {
                    const double f = h_in(n, k * rho) / Is[l][n] * wt;
                    const double cr = f * std::cos(n * ph), ci = -f * std::sin(n * ph);
                    for (int j = 0; j < qq; ++j) {
                        const double lj = lag(j % q, u) * lag(j / q, v);
                        if (n == 0)
                            buf[j] += cr * lj;
                        else {
                            buf[(2 * n - 1) * qq + j] += cr * lj;
                            buf[(2 * n) * qq + j] += ci * lj;
                        }
                    }
                }
            }
        op_p2m[l] = pool.add(P, qq, buf.data());
        buf.assign((size_t)qq * P, 0.0);
        for (int i = 0; i < qq; ++i) {
            const double X = 0.5 * w * qx[i % q], Y = 0.5 * w * qx[i / q];
            const double r = std::hypot(X, Y), th = std::atan2(Y, X);
            for (int n = 0; n <= p; ++n) {
                const double b = h_in(n, k * r) / Is[l][n];
                if (n == 0)
                    buf[i * P] = b;
                else {
                    buf[i * P + 2 * n - 1] = 2 * b * std::cos(n * th);
                    buf[i * P + 2 * n] = -2 * b * std::sin(n * th);
                }
            }
        }
        op_l2p[l] = pool.add(qq, P, buf.data());
    }
    // ---- M2M and L2L (child c at level l+1, parent at l) ----
    std::vector<std::array<int, 4>> op_m2m(L + 1), op_l2l(L + 1);
    for (int l = 2; l < L; ++l)
        for (int c = 0; c < 4; ++c) {
            const double h2 = 0.25 * width(l);
            const std::complex<double> d((c & 1) ? h2 : -h2, (c & 2) ? h2 : -h2);
            const double dr = std::abs(d), da = std::arg(d);
            std::vector<double> Id(2 * p + 1);
            for (int j = 0; j <= 2 * p; ++j) Id[j] = h_in(j, k * dr);
            buf.assign((size_t)P * P, 0.0);
            real_form(p,
                      [&](int m, int n) {
                          const int j = m - n;
                          return Is[l + 1][std::abs(n)] * Id[std::abs(j)] * std::polar(1.0, -j * da) / Is[l][m];
                      },
                      buf.data());
            op_m2m[l][c] = pool.add(P, P, buf.data());
            real_form(p,
                      [&](int m, int n) {
                          const int j = n - m;
                          return Is[l + 1][m] * Id[std::abs(j)] * std::polar(1.0, j * da) / Is[l][std::abs(n)];
                      },
                      buf.data());
            op_l2l[l][c] = pool.add(P, P, buf.data());
        }
    // ---- configuration-keyed operators discovered from the lists ----
    std::map<std::tuple<int, int, int, int>, int> near_key, m2l_key, m2p_key, p2l_key;
    std::vector<NearCfg> near_cfg;
    std::vector<int> near_level;
    std::vector<Task> t_out, t_m2l, t_p2m, t_near;
    // relative centre offset (source minus target) from integer coordinates
    auto rel = [&](int tb, int sb) {
        const int lt = lev(tb), ls = lev(sb), f = std::max(lt, ls);
        const double wf = width(f);
        const double dx = ((2.0 * bx(sb) + 1) * (1 << (f - ls)) - (2.0 * bx(tb) + 1) * (1 << (f - lt))) * 0.5 * wf;
        const double dy = ((2.0 * by(sb) + 1) * (1 << (f - ls)) - (2.0 * by(tb) + 1) * (1 << (f - lt))) * 0.5 * wf;
        return std::complex<double>(dx, dy);
    };
    std::vector<double> Kb(2 * p + 2);
    for (int64_t b = 0; b < nb; ++b) {
        const int l = lev((int)b);
        const int leaf = h.box_leaf[b];
        // U list -> near tables
        if (leaf >= 0) {
            for (int j = h.off[0][b]; j < h.off[0][b + 1]; ++j) {
                const int c = h.item[0][j];
                const int lc = lev(c), f = std::max(l, lc);
                const int ox = bx(c) * (1 << (f - lc)) - bx((int)b) * (1 << (f - l));
                const int oy = by(c) * (1 << (f - lc)) - by((int)b) * (1 << (f - l));
                auto key = std::make_tuple(l, lc - l, ox, oy);
                auto it = near_key.find(key);
                int id;
                if (it == near_key.end()) {
                    id = (int)near_cfg.size();
                    near_key[key] = id;
                    const std::complex<double> r = rel((int)b, c);
                    near_cfg.push_back(NearCfg{r.real(), r.imag(), width(lc), width(l)});
                    near_level.push_back(l);
                } else {
                    id = it->second;
                }
                t_near.push_back(Task{-1 - id, V->B_off + (int64_t)h.box_leaf[c] * qq, V->U_off + (int64_t)leaf * qq});
            }
            if (l >= 2) t_out.push_back(Task{op_l2p[l], V->L_off + b * P, V->U_off + (int64_t)leaf * qq});
            // W list -> M2P
            for (int j = h.off[2][b]; j < h.off[2][b + 1]; ++j) {
                const int c = h.item[2][j];
                auto key = std::make_tuple(l, bx(c) - 2 * bx((int)b), by(c) - 2 * by((int)b), 0);
                auto it = m2p_key.find(key);
                int id;
                if (it == m2p_key.end()) {
                    const std::complex<double> r = rel((int)b, c);   // source centre - target centre
                    const double w = width(l);
                    buf.assign((size_t)qq * P, 0.0);
                    for (int i = 0; i < qq; ++i) {
                        const std::complex<double> z =
                            std::complex<double>(0.5 * w * qx[i % q], 0.5 * w * qx[i / q]) - r;
                        const double rr = std::abs(z), th = std::arg(z);
                        h_kn_all(k * rr, p, Kb.data());
                        for (int n = 0; n <= p; ++n) {
                            const double v = Is[l + 1][n] * Kb[n];
                            if (n == 0)
                                buf[i * P] = v;
                            else {
                                buf[i * P + 2 * n - 1] = 2 * v * std::cos(n * th);
                                buf[i * P + 2 * n] = -2 * v * std::sin(n * th);
                            }
                        }
                    }
                    id = pool.add(qq, P, buf.data());
                    m2p_key[key] = id;
                } else {
                    id = it->second;
                }
                t_out.push_back(Task{id, V->M_off + (int64_t)c * P, V->U_off + (int64_t)leaf * qq});
            }
            if (l >= 2) t_p2m.push_back(Task{op_p2m[l], V->B_off + (int64_t)leaf * qq, V->M_off + b * P});
        }
        if (l < 2) continue;
        // V list -> M2L
        for (int j = h.off[1][b]; j < h.off[1][b + 1]; ++j) {
            const int s = h.item[1][j];
            auto key = std::make_tuple(l, bx(s) - bx((int)b), by(s) - by((int)b), 0);
            auto it = m2l_key.find(key);
            int id;
            if (it == m2l_key.end()) {
                const std::complex<double> D = -rel((int)b, s);   // target centre - source centre
                const double R = std::abs(D), Ph = std::arg(D);
                h_kn_all(k * R, 2 * p, Kb.data());
                buf.assign((size_t)P * P, 0.0);
                real_form(p,
                          [&](int m, int n) {
                              const int jj = n - m;
                              const double sg = (m & 1) ? -1.0 : 1.0;
                              return Is[l][m] * sg * Kb[std::abs(jj)] * std::polar(1.0, jj * Ph) * Is[l][std::abs(n)];
                          },
                          buf.data());
                id = pool.add(P, P, buf.data());
                m2l_key[key] = id;
            } else {
                id = it->second;
            }
            t_m2l.push_back(Task{id, V->M_off + (int64_t)s * P, V->L_off + b * P});
        }
        // X list -> P2L
        for (int j = h.off[3][b]; j < h.off[3][b + 1]; ++j) {
            const int c = h.item[3][j];
            auto key = std::make_tuple(l, 2 * bx(c) - bx((int)b), 2 * by(c) - by((int)b), 0);
            auto it = p2l_key.find(key);
            int id;
            if (it == p2l_key.end()) {
                const std::complex<double> r = rel((int)b, c);   // source centre - target centre
                const double wc = width(l - 1);
                buf.assign((size_t)P * qq, 0.0);
                for (int v = 0; v < NGLQ; ++v)
                    for (int u = 0; u < NGLQ; ++u) {
                        const std::complex<double> uu =
                            r + std::complex<double>(0.5 * wc * glx[u], 0.5 * wc * glx[v]);
                        const double wt = 0.25 * wc * wc * glw[u] * glw[v] * pref;
                        const double ru = std::abs(uu), au = std::arg(uu);
                        h_kn_all(k * ru, p, Kb.data());
                        for (int m = 0; m <= p; ++m) {
                            const double f = Is[l][m] * Kb[m] * wt;
                            const double cr = f * std::cos(m * au), ci = -f * std::sin(m * au);
                            for (int jj = 0; jj < qq; ++jj) {
                                const double lj = lag(jj % q, u) * lag(jj / q, v);
                                if (m == 0)
                                    buf[jj] += cr * lj;
                                else {
                                    buf[(2 * m - 1) * qq + jj] += cr * lj;
                                    buf[(2 * m) * qq + jj] += ci * lj;
                                }
                            }
                        }
                    }
                id = pool.add(P, qq, buf.data());
                p2l_key[key] = id;
            } else {
                id = it->second;
            }
            t_m2l.push_back(Task{id, V->B_off + (int64_t)h.box_leaf[c] * qq, V->L_off + b * P});
        }
    }
    // M2M / L2L chains: the internal boxes of levels 2 <= l < L with their four children
    MH_TRY(build_chain(ctx, t, h, P, pool, op_m2m, op_l2l, nullptr, &V->chain));
    // near tables on the device, appended to the pool
    const int nnear = (int)near_cfg.size();
    V->n_near_tables = nnear;
    V->m2l_key = m2l_key;
    V->m2p_key = m2p_key;
    V->op_p2m = op_p2m;
    V->op_l2p = op_l2p;
    V->op_m2m = op_m2m;
    V->op_l2l = op_l2l;
    V->pool_host = pool;   // before the near tables are appended (their data lives on the device only)
    const int64_t near_base = (int64_t)pool.data.size();
    const int first_near_op = (int)pool.off.size();
    for (int i = 0; i < nnear; ++i) {
        pool.off.push_back(near_base + (int64_t)i * qq * qq);
        pool.R.push_back(qq);
        pool.C.push_back(qq);
    }
    for (auto& tk : t_near) tk.op = first_near_op + (-1 - tk.op);
    const int64_t total = near_base + (int64_t)nnear * qq * qq;
    MH_ALLOC(ctx, V->ops64, total);
    cudaStream_t st = ctx->stream;
    if (near_base) MH_CUDA(ctx, cudaMemcpyAsync(V->ops64.p, pool.data.data(), near_base * 8, cudaMemcpyHostToDevice, st));
    if (nnear) {
        dbuf<NearCfg> dcfg;
        dbuf<double> dxi, dgx, dgw;
        MH_ALLOC(ctx, dcfg, nnear);
        MH_ALLOC(ctx, dxi, q);
        MH_ALLOC(ctx, dgx, NGLN);
        MH_ALLOC(ctx, dgw, NGLN);
        MH_CUDA(ctx, cudaMemcpyAsync(dcfg.p, near_cfg.data(), nnear * sizeof(NearCfg), cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(dxi.p, qx.data(), q * 8, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(dgx.p, g16x.data(), NGLN * 8, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(dgw.p, g16w.data(), NGLN * 8, cudaMemcpyHostToDevice, st));
        k_near_tables<<<(unsigned)(nnear * qq), 256, 0, st>>>(dcfg.p, q, dxi.p, dgx.p, dgw.p, k, pref,
                                                              V->ops64.p + near_base);
        MH_LAUNCHED(ctx);
        MH_CUDA(ctx, cudaStreamSynchronize(st));
    }
    MH_ALLOC(ctx, V->ops32, total);
    // every operator in binary64 on the host (the near tables were formed on the device): source
    // of the binary32 copy and of the tensor-core images
    std::vector<double> all(total);
    MH_CUDA(ctx, cudaMemcpyAsync(all.data(), V->ops64.p, total * 8, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    {
        // binary32 copy of every operator (mixed precision)
        std::vector<float> f(all.begin(), all.end());
        MH_CUDA(ctx, cudaMemcpyAsync(V->ops32.p, f.data(), total * 4, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
    }
    V->op_C.assign(pool.C.begin(), pool.C.end());
    MH_ALLOC(ctx, V->d_op_off, pool.off.size());
    MH_ALLOC(ctx, V->d_op_C, pool.C.size());
    MH_CUDA(ctx, cudaMemcpyAsync(V->d_op_off.p, pool.off.data(), pool.off.size() * 8, cudaMemcpyHostToDevice, st));
    MH_CUDA(ctx, cudaMemcpyAsync(V->d_op_C.p, pool.C.data(), pool.C.size() * 4, cudaMemcpyHostToDevice, st));
    // phases; split ranges of the tensor-core sources: node values (B), multipoles (M), locals (L)
    const std::vector<TcImages::Range> rg = {{V->B_off, qq, nl, 0, 0}, {V->M_off, P, nb, 0, 0},
                                             {V->L_off, P, nb, 0, 0}};
    int64_t need = 1;
    V->p2m.reset(new Phase());
    MH_TRY(build_phase(ctx, t_p2m, P, false, V->op_C, V->p2m.get(), &need, &rg));
    V->m2l.reset(new Phase());
    MH_TRY(build_phase(ctx, t_m2l, P, false, V->op_C, V->m2l.get(), &need, &rg));
    // U^h = near (U list, written first) + far (L2P, M2P: added once the passes are done)
    {
        std::vector<char> has(t->n_leaves, 0);
        for (const Task& tk : t_near) has[(tk.dst - V->U_off) / qq] = 1;
        V->near_cover = std::find(has.begin(), has.end(), 0) == has.end();
    }
    int64_t need_near = 1;
    V->near.reset(new Phase());
    MH_TRY(build_phase(ctx, t_near, qq, false, V->op_C, V->near.get(), &need_near, &rg));
    V->near->dst_out = true;
    V->out.reset(new Phase());
    MH_TRY(build_phase(ctx, t_out, qq, true, V->op_C, V->out.get(), &need, &rg));
    V->out->dst_out = true;
    {
        std::vector<int64_t> off(pool.off.begin(), pool.off.end());
        std::vector<int32_t> rr(pool.R.begin(), pool.R.end()), cc(pool.C.begin(), pool.C.end());
        MH_TRY(build_tc_images(ctx, all.data(), off, rr, cc, {V->p2m.get(), V->m2l.get(), V->near.get(), V->out.get()},
                               rg, &V->tc));
    }
    MH_ALLOC(ctx, V->vec, V->vec_len);
    // binary32 mirror with TC_POOL_PAD floats of slack at the end: the tensor-core gather
    // reads sources in aligned 16-byte windows that may reach past a vector's last entry
    MH_ALLOC(ctx, V->vec32, V->vec_len + TC_POOL_PAD);
    MH_ALLOC(ctx, V->temp, need);
    MH_ALLOC(ctx, V->temp_near, need_near);
    MH_TRY(V->side.create(ctx));
    V->temp_len = need;
    MH_CUDA(ctx, cudaMemsetAsync(V->vec.p, 0, V->vec_len * 8, st));
    MH_CUDA(ctx, cudaMemsetAsync(V->vec32.p, 0, (V->vec_len + TC_POOL_PAD) * 4, st));
    // shared-memory opt-in for the contraction kernel
    int maxs = 0;
    for (auto* ph : {V->p2m.get(), V->m2l.get(), V->out.get(), V->near.get()}) maxs = std::max(maxs, ph->smem);
    MH_CUDA(ctx, cudaFuncSetAttribute(k_apply<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      160 * 1024));
    MH_CUDA(ctx, cudaFuncSetAttribute(k_apply<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    MH_CUDA(ctx, cudaFuncSetAttribute(k_apply<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      160 * 1024));
    if (chain_threads(P) > 1024)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "multipole order too large for the chain kernels");
    return MH_OK;
}

}  // namespace

// ---------------- double layer through the multipole method ----------------
//
// Dipole sources at the boundary nodes y_d (unit normal nu_d = e^{i psi}, strength w_d =
// sigma_d |y'_d| h) give U^h(x) = (1/(2 pi alpha^2)) sum_d w_d d/dnu K0(k |x - y_d|)
// (Section 2).  With G_n(v) = I_n(k|v|) e^{-i n arg v} and H_n(u) = K_n(k|u|) e^{-i n arg u}:
//   d/dnu G_n = (k/2) [e^{-i psi} G_{n-1} + e^{i psi} G_{n+1}]    (dipole multipole, P2M)
//   d/dnu H_n = -(k/2) [e^{-i psi} H_{n-1} + e^{i psi} H_{n+1}]   (dipole local, P2L)
// and the near field is the trapezoid kernel value itself.  The translation operators
// (M2M, M2L, L2L, L2P, M2P) are those of the volume pass.
namespace {

// Near field of the double layer on the fly.  The dipoles of a target leaf's U list form
// one flat run (their offsets from the TARGET leaf centre precomputed in binary64, then
// rounded); the run is cut into chunks of at most NEAR_CHUNK dipoles, one block per chunk,
// largest chunks first, so that no leaf with a long U list holds one SM while the others
// idle.  Thread t handles node t % q^2 for the share t / q^2 of every staged tile (q^2 <= 64).
// A leaf in one chunk writes its nodes directly; otherwise every chunk stores its partial
// sums and the last chunk of the leaf to finish (counted per leaf, reset by that chunk)
// adds them in chunk order: the result does not depend on the block schedule.
//   out[node] += -(1/(2 pi alpha^2)) sum_d w_d (1/alpha) K1(r/alpha) (y_d - x).nu_d / r
constexpr int NEAR_T = 256;
constexpr int NEAR_CHUNK = 512;

struct NearChunk {
    int32_t leaf, k0, k1;   // target leaf, flat dipole range [k0, k1)
    int32_t slot;           // partial-sum slot, -1 for a leaf in one chunk
};

// Finish a chunk: block-sum the per-share partials of node i, then write or hand over.
template <int NT>
__device__ __forceinline__ void near_finish(double acc, bool act, int qq, int i, int groups, const NearChunk& ch,
                                            const int2* __restrict__ leaf_red, double pref, double* part,
                                            unsigned* cnt, double* out) {
    __shared__ double red[NT];
    __shared__ int last;
    red[threadIdx.x] = act ? acc : 0.0;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x < qq)
        for (int gg = 0; gg < groups; ++gg) tot += red[gg * qq + threadIdx.x];
    const int64_t node = (int64_t)ch.leaf * qq + i;
    if (ch.slot < 0) {
        if (threadIdx.x < qq) out[node] -= pref * tot;
        return;
    }
    if (threadIdx.x < qq) part[(int64_t)ch.slot * qq + i] = tot;
    __threadfence();
    __syncthreads();
    const int2 lr = leaf_red[ch.leaf];   // {first slot, chunks}
    if (threadIdx.x == 0) last = atomicAdd(cnt + ch.leaf, 1u) == (unsigned)(lr.y - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < qq) {
        double s = 0.0;
        for (int c = 0; c < lr.y; ++c) s += __ldcg(part + (int64_t)(lr.x + c) * qq + i);
        out[node] -= pref * s;
    }
    if (threadIdx.x == 0) cnt[ch.leaf] = 0u;
}

__global__ void __launch_bounds__(NEAR_T) k_dip_near64(
    const double* __restrict__ nodes, const NearChunk* __restrict__ chunks, const int2* __restrict__ leaf_red,
    const int32_t* __restrict__ flat_idx, const double2* __restrict__ dxy, const double2* __restrict__ dnrm,
    const double* __restrict__ w, int qq, double inv_alpha, double pref, double* part, unsigned* cnt,
    double* out) {
    __shared__ double2 sp[NEAR_T], sn[NEAR_T];
    __shared__ double sw[NEAR_T];
    const NearChunk ch = chunks[blockIdx.x];
    const int groups = NEAR_T / qq;   // >= 4 for q <= 8
    const int i = threadIdx.x % qq, g = threadIdx.x / qq;
    const bool act = g < groups;
    const int64_t node = (int64_t)ch.leaf * qq + i;
    const double px = nodes[2 * node], py = nodes[2 * node + 1];
    double acc = 0.0;
    for (int k0 = ch.k0; k0 < ch.k1; k0 += NEAR_T) {
        const int m = min(NEAR_T, ch.k1 - k0);
        __syncthreads();
        if (threadIdx.x < m) {
            const int d = flat_idx[k0 + threadIdx.x];
            sp[threadIdx.x] = dxy[d];
            sn[threadIdx.x] = dnrm[d];
            sw[threadIdx.x] = w[d];
        }
        __syncthreads();
        if (act)
            for (int e = g; e < m; e += groups) {
                const double dx = sp[e].x - px, dy = sp[e].y - py;
                const double r = sqrt(dx * dx + dy * dy);
                // pairs beyond 45 alpha are below the binary64 rounding of the sum (e^{-45})
                if (r > 0.0 && r * inv_alpha <= 45.0)
                    acc += mh_k1(r * inv_alpha) * inv_alpha * (dx * sn[e].x + dy * sn[e].y) / r * sw[e];
            }
    }
    near_finish<NEAR_T>(acc, act, qq, i, groups, ch, leaf_red, pref, part, cnt, out);
}

// Binary32: the staged dipole carries its weight in the normal, (x, y, w nx, w ny), and the
// pair term is g(z) (d . w n) (mh_dl32_pair); pref already holds the factor 1/alpha^2.
// NT threads per block (the tile: qq targets x NT / qq source shares, NT dipoles staged per
// round); NT in {128, 256, 512} is picked per problem by timing.
template <int NT>
__global__ void __launch_bounds__(NT) k_dip_near32(
    const double* __restrict__ nodes, const NearChunk* __restrict__ chunks, const int2* __restrict__ leaf_red,
    const double2* __restrict__ leaf_c, const int32_t* __restrict__ flat_idx, const float4* __restrict__ flat32,
    const float* __restrict__ w, int qq, mh_dl32 c32, double pref, double* part, unsigned* cnt, double* out) {
    __shared__ float4 s4[NT];
    const NearChunk ch = chunks[blockIdx.x];
    const int groups = NT / qq;
    const int i = threadIdx.x % qq, g = threadIdx.x / qq;
    const bool act = g < groups;
    const int64_t node = (int64_t)ch.leaf * qq + i;
    const double2 c = leaf_c[ch.leaf];
    const float tx = (float)(nodes[2 * node] - c.x), ty = (float)(nodes[2 * node + 1] - c.y);
    float ah = 0.f, al = 0.f;   // float-float sum of the tile sums (no binary64 per tile)
    for (int k0 = ch.k0; k0 < ch.k1; k0 += NT) {
        const int m = min(NT, ch.k1 - k0);
        __syncthreads();
        if (threadIdx.x < m) {
            const float4 v = flat32[k0 + threadIdx.x];
            const float wd = w[flat_idx[k0 + threadIdx.x]];
            s4[threadIdx.x] = make_float4(v.x, v.y, v.z * wd, v.w * wd);
        }
        __syncthreads();
        if (act) {
            // two staged dipoles per iteration (the warp's threads share g: a uniform branch);
            // the dipoles of neighbour leaves are near by construction: no per-pair tests
            float pt = 0.f, pu = 0.f;
            int e = g;
            for (; e + groups < m; e += 2 * groups) {
                const float4 v = s4[e], u = s4[e + groups];
                pt += mh_dl32_pair_nt(v.x - tx, v.y - ty, v.z, v.w, c32);
                pu += mh_dl32_pair_nt(u.x - tx, u.y - ty, u.z, u.w, c32);
            }
            if (e < m) {
                const float4 v = s4[e];
                pt += mh_dl32_pair_nt(v.x - tx, v.y - ty, v.z, v.w, c32);
            }
            pt += pu;
            const float t = ah + pt, bb = t - ah;
            al += (ah - (t - bb)) + (pt - bb);
            ah = t;
        }
    }
    near_finish<NT>((double)ah + (double)al, act, qq, i, groups, ch, leaf_red, pref, part, cnt, out);
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

struct DipData {
    int64_t nd = 0;
    int64_t W_off = 0, DM_off = 0, DL_off = 0, DU_off = 0, vec_len = 0;
    // near field evaluated on the fly: per target leaf the dipoles of its U list, flattened
    bool near_blocks = true;
    int qq = 0;
    dbuf<NearChunk> chunks;                // largest first
    int64_t n_chunks = 0;
    dbuf<int2> leaf_red;                   // per leaf: first partial slot, chunk count
    dbuf<double> part;                     // partial sums of leaves in several chunks (slot x qq)
    dbuf<unsigned> red_cnt;                // per leaf: chunks finished in the running launch
    dbuf<int32_t> flat_idx;                // dipole of every flat entry
    dbuf<float4> flat32;                   // its offset from the target leaf centre + normal (binary32)
    dbuf<double2> leaf_c, dxy, dnrm;       // leaf centres; dipole positions and normals (sorted)
    double pref = 0, inv_alpha = 0;
    double near_pairs = 0;
    int near_t = 256;                      // threads per block of the binary32 near-field kernel
    dbuf<double> vec, temp, ops64;
    dbuf<float> ops32, vec32;              // vec32: binary32 mirror of vec (weights, expansions)
    dbuf<int64_t> d_op_off;
    dbuf<int32_t> d_op_C;
    std::unique_ptr<Phase> p2m, m2l, out;
    std::unique_ptr<DfChain> chain_up;     // M2M over the boxes that hold dipoles
    SideStream side;                       // the near field runs there beside the passes
    TcImages tc;                           // tensor-core images (mixed precision)
};
}  // namespace

static mh_status volume_ensure(mh_ctx* ctx, mh_tree* t, double alpha, int p) {
    VolData* V = static_cast<VolData*>(t->vol);
    if (V && V->alpha == alpha && V->p == p) return MH_OK;
    delete V;
    V = new VolData();
    t->vol = V;
    mh_status s = volume_setup(ctx, t, alpha, p, V);
    if (s != MH_OK) {
        delete V;
        t->vol = nullptr;
    }
    return s;
}

namespace {

// ---- dipole pass set-up helpers (shared by the volume-node and the boundary-node outputs) ----

// Box geometry of the host tree and the expansion scales I_n(k s_l) (s_l = box radius of level l).
struct DipGeo {
    const HostTree* h = nullptr;
    double x0 = 0, y0 = 0, W = 0;
    std::vector<std::vector<double>> Is;
    int lev(int b) const { return h->boxes[3 * b]; }
    double width(int l) const { return W / (double)(1 << l); }
    std::complex<double> centre(int b) const {
        const double w = width(lev(b));
        return std::complex<double>(x0 + (h->boxes[3 * b + 1] + 0.5) * w, y0 + (h->boxes[3 * b + 2] + 0.5) * w);
    }
};

DipGeo dip_geo(const mh_tree* t, const HostTree& h, int p, double k) {
    DipGeo G;
    G.h = &h;
    G.x0 = t->box[0];
    G.y0 = t->box[1];
    G.W = t->box[2];
    G.Is.assign(t->max_level + 1, std::vector<double>(p + 2));
    for (int l = 0; l <= t->max_level; ++l)
        for (int n = 0; n <= p + 1; ++n) G.Is[l][n] = h_in(n, k * G.width(l) * 0.70710678118654752);
    return G;
}

// Entry n of an expansion in the real form [a_0, a_1, b_1, ...] as column col of a matrix with
// cols columns.
void dip_set_row(double* m, int cols, int col, int n, std::complex<double> v) {
    if (n == 0)
        m[col] = v.real();
    else {
        m[(2 * n - 1) * cols + col] = v.real();
        m[(2 * n) * cols + col] = v.imag();
    }
}

// T[|m|] e^{-i m arg v} for a table T of I_n or K_n values at k|v|.
std::complex<double> dip_g(int m, std::complex<double> v, const std::vector<double>& T) {
    return T[std::abs(m)] * std::polar(1.0, -m * std::arg(v));
}

// Operators wider than DIP_CMAX columns are split into column blocks reducing into one destination.
constexpr int DIP_CMAX = 128;
void dip_add_split(OpPool& pool, int R, int nc, const std::vector<double>& m, int64_t src, int64_t dst,
                   std::vector<Task>& tl) {
    std::vector<double> sub;
    for (int c0 = 0; c0 < nc; c0 += DIP_CMAX) {
        const int cw = std::min(DIP_CMAX, nc - c0);
        sub.assign((size_t)R * cw, 0.0);
        for (int r = 0; r < R; ++r)
            for (int c = 0; c < cw; ++c) sub[(size_t)r * cw + c] = m[(size_t)r * nc + c0 + c];
        tl.push_back(Task{pool.add(R, cw, sub.data()), src + c0, dst});
    }
}

// Boxes whose subtree holds a dipole: every leaf with segn > 0 and its ancestors.
std::vector<char> dipole_active_boxes(const HostTree& h, const std::vector<int64_t>& segn) {
    const int64_t nb = (int64_t)h.box_leaf.size();
    std::vector<char> active(nb, 0);
    std::map<std::tuple<int, int, int>, int> id;
    for (int64_t b = 0; b < nb; ++b) id[std::make_tuple(h.boxes[3 * b], h.boxes[3 * b + 1], h.boxes[3 * b + 2])] = (int)b;
    for (int64_t b = 0; b < nb; ++b) {
        const int lf = h.box_leaf[b];
        if (lf < 0 || segn[lf] == 0) continue;
        int l = h.boxes[3 * b], x = h.boxes[3 * b + 1], y = h.boxes[3 * b + 2];
        for (;;) {
            auto it = id.find(std::make_tuple(l, x, y));
            if (it == id.end() || active[it->second]) break;
            active[it->second] = 1;
            if (l == 0) break;
            --l;
            x >>= 1;
            y >>= 1;
        }
    }
    return active;
}

// The source side of a dipole pass: per box of level >= 2, the P2M of a leaf's dipoles (weights
// at W_off + their sorted position, multipoles at DM_off), the M2L over the V list and the dipole
// P2L over the X list (locals at DL_off).  Dipoles are sorted by leaf: leaf i owns the run
// [seg0[i], seg0[i] + segn[i]).  `active` marks the boxes whose subtree holds a dipole: M2L
// tasks are made only from active sources (the other multipoles are zero, so leaving them out
// changes no sum), and with `dst_active_only` (the targets are the dipoles themselves) M2L and
// P2L tasks only into active boxes (the other locals are never evaluated).
void dipole_source_tasks(const DipGeo& G, const VolData* V, OpPool& pool, int p, double k, double pref,
                         const double* dxy, const double* dnrm, const std::vector<int64_t>& seg0,
                         const std::vector<int64_t>& segn, int64_t W_off, int64_t DM_off, int64_t DL_off,
                         std::vector<Task>& t_p2m, std::vector<Task>& t_m2l,
                         const std::vector<char>* active = nullptr, bool dst_active_only = false) {
    const HostTree& h = *G.h;
    const int P = 2 * p + 1;
    const int64_t nb = (int64_t)h.box_leaf.size();
    std::vector<double> buf, Kb(p + 3), Ib(p + 3);
    for (int64_t b = 0; b < nb; ++b) {
        const int l = G.lev((int)b);
        if (l < 2) continue;
        const int leaf = h.box_leaf[b];
        // dipole P2M of this leaf
        if (leaf >= 0 && segn[leaf] > 0) {
            const int nc = (int)segn[leaf];
            buf.assign((size_t)P * nc, 0.0);
            const std::complex<double> c = G.centre((int)b);
            for (int j = 0; j < nc; ++j) {
                const int64_t d = seg0[leaf] + j;
                const std::complex<double> v = std::complex<double>(dxy[2 * d], dxy[2 * d + 1]) - c;
                const double psi = std::atan2(dnrm[2 * d + 1], dnrm[2 * d]);
                for (int n = 0; n <= p + 1; ++n) Ib[n] = h_in(n, k * std::abs(v));
                for (int n = 0; n <= p; ++n) {
                    const std::complex<double> Dn = 0.5 * k * (std::polar(1.0, -psi) * dip_g(n - 1, v, Ib) +
                                                               std::polar(1.0, psi) * dip_g(n + 1, v, Ib));
                    dip_set_row(buf.data(), nc, j, n, pref * Dn / G.Is[l][n]);
                }
            }
            dip_add_split(pool, P, nc, buf, W_off + seg0[leaf], DM_off + b * P, t_p2m);
        }
        if (active && dst_active_only && !(*active)[b]) continue;
        for (int j = h.off[1][b]; j < h.off[1][b + 1]; ++j) {
            const int s2 = h.item[1][j];
            if (active && !(*active)[s2]) continue;
            auto key = std::make_tuple(l, h.boxes[3 * s2 + 1] - h.boxes[3 * b + 1], h.boxes[3 * s2 + 2] - h.boxes[3 * b + 2], 0);
            t_m2l.push_back(Task{V->m2l_key.at(key), DM_off + (int64_t)s2 * P, DL_off + b * P});
        }
        // X list: dipole P2L
        for (int j = h.off[3][b]; j < h.off[3][b + 1]; ++j) {
            const int c = h.item[3][j];
            const int lc = h.box_leaf[c];
            if (segn[lc] == 0) continue;
            const int nc = (int)segn[lc];
            buf.assign((size_t)P * nc, 0.0);
            const std::complex<double> ct = G.centre((int)b);
            for (int jj = 0; jj < nc; ++jj) {
                const int64_t d = seg0[lc] + jj;
                const std::complex<double> u = std::complex<double>(dxy[2 * d], dxy[2 * d + 1]) - ct;
                const double psi = std::atan2(dnrm[2 * d + 1], dnrm[2 * d]);
                h_kn_all(k * std::abs(u), p + 1, Kb.data());
                for (int m = 0; m <= p; ++m) {
                    const std::complex<double> Dm = -0.5 * k * (std::polar(1.0, -psi) * dip_g(m - 1, u, Kb) +
                                                                std::polar(1.0, psi) * dip_g(m + 1, u, Kb));
                    dip_set_row(buf.data(), nc, jj, m, G.Is[l][m] * pref * Dm);
                }
            }
            dip_add_split(pool, P, nc, buf, W_off + seg0[lc], DL_off + b * P, t_m2l);
        }
    }
}

}  // namespace

mh_status volume_dipole_setup(mh_ctx* ctx, mh_tree* t, double alpha, int p, const double* dxy, const double* dnrm,
                              const int32_t* dleaf, int64_t nd, bool near_blocks) {
    if (!near_blocks && t->q * t->q > 64) near_blocks = true;   // the on-the-fly kernel handles q <= 8
    MH_TRY(volume_ensure(ctx, t, alpha, p));
    VolData* V = static_cast<VolData*>(t->vol);
    const int q = t->q, qq = q * q, P = 2 * p + 1;
    const double k = 1.0 / alpha, pref = 1.0 / (2.0 * MH_PI * alpha * alpha);
    HostTree h;
    MH_TRY(fetch_tree(ctx, t, &h));
    const int64_t nb = t->n_boxes, nl = t->n_leaves;
    const DipGeo G = dip_geo(t, h, p, k);
    std::vector<double> qx(q), qw(q);
    mh_gauss_legendre(q, qx.data(), qw.data());
    // dipole segments per leaf (sources are sorted by leaf)
    std::vector<int64_t> seg0(nl, -1), segn(nl, 0);
    for (int64_t d = 0; d < nd; ++d) {
        const int lf = dleaf[d];
        if (seg0[lf] < 0) seg0[lf] = d;
        segn[lf]++;
    }
    std::unique_ptr<DipData> D(new DipData());
    D->nd = nd;
    D->near_blocks = near_blocks;
    D->qq = qq;
    D->pref = pref;
    D->inv_alpha = k;
    std::vector<int32_t> nleaf;
    D->W_off = 0;
    D->DM_off = nd;
    D->DL_off = D->DM_off + nb * P;
    D->DU_off = D->DL_off + nb * P;
    D->vec_len = D->DU_off + nl * qq;
    OpPool pool = V->pool_host;
    std::vector<Task> t_p2m, t_m2l, t_out;
    // multipoles are non-zero only in boxes that hold dipoles: M2L from those alone, and the
    // upward chain over those alone (the downward chain serves every leaf: targets everywhere)
    const std::vector<char> active = dipole_active_boxes(h, segn);
    dipole_source_tasks(G, V, pool, p, k, pref, dxy, dnrm, seg0, segn, D->W_off, D->DM_off, D->DL_off, t_p2m, t_m2l,
                        &active, false);
    MH_TRY(build_chain(ctx, t, h, P, V->pool_host, V->op_m2m, V->op_l2l, &active, &D->chain_up));
    std::vector<double> buf;
    for (int64_t b = 0; b < nb; ++b) {
        const int l = G.lev((int)b);
        const int leaf = h.box_leaf[b];
        if (leaf < 0) continue;
        if (l >= 2) t_out.push_back(Task{V->op_l2p[l], D->DL_off + b * P, D->DU_off + (int64_t)leaf * qq});
        // W list: M2P with the volume operators
        for (int j = h.off[2][b]; j < h.off[2][b + 1]; ++j) {
            const int c = h.item[2][j];
            auto key = std::make_tuple(l, h.boxes[3 * c + 1] - 2 * h.boxes[3 * b + 1],
                                       h.boxes[3 * c + 2] - 2 * h.boxes[3 * b + 2], 0);
            t_out.push_back(Task{V->m2p_key.at(key), D->DM_off + (int64_t)c * P, D->DU_off + (int64_t)leaf * qq});
        }
        // U list: direct dipole sums from neighbour leaves, as dense (q^2 x n_c) blocks or
        // (near_blocks == false) evaluated on the fly by k_dip_near
        const std::complex<double> cb = G.centre((int)b);
        const double wb = G.width(l);
        for (int j = h.off[0][b]; j < h.off[0][b + 1]; ++j) {
            const int c = h.item[0][j];
            const int lc = h.box_leaf[c];
            if (segn[lc] == 0) continue;
            if (!near_blocks) {
                nleaf.push_back(lc);
                D->near_pairs += (double)qq * segn[lc];
                continue;
            }
            const int nc = (int)segn[lc];
            buf.assign((size_t)qq * nc, 0.0);
            for (int i = 0; i < qq; ++i) {
                const double xx = cb.real() + 0.5 * wb * qx[i % q], xy = cb.imag() + 0.5 * wb * qx[i / q];
                for (int jj = 0; jj < nc; ++jj) {
                    const int64_t d = seg0[lc] + jj;
                    const double dx = dxy[2 * d] - xx, dy = dxy[2 * d + 1] - xy;
                    const double r = std::hypot(dx, dy);
                    if (r > 0)
                        buf[(size_t)i * nc + jj] =
                            -pref * h_k1(r * k) * k * (dx * dnrm[2 * d] + dy * dnrm[2 * d + 1]) / r;
                }
            }
            dip_add_split(pool, qq, nc, buf, D->W_off + seg0[lc], D->DU_off + (int64_t)leaf * qq, t_out);
        }
    }
    if (!near_blocks) {
        // CSR over target leaves (in leaf order) of the source leaves holding dipoles
        std::vector<std::vector<int32_t>> per(nl);
        {
            size_t pos = 0;
            for (int64_t b = 0; b < nb; ++b) {
                const int leaf = h.box_leaf[b];
                if (leaf < 0) continue;
                for (int j = h.off[0][b]; j < h.off[0][b + 1]; ++j) {
                    const int lc = h.box_leaf[h.item[0][j]];
                    if (segn[lc] == 0) continue;
                    per[leaf].push_back(nleaf[pos++]);
                }
            }
        }
        std::vector<double2> lc(nl), pxy(nd), pn(nd);
        for (int64_t i = 0; i < nl; ++i) {
            const std::complex<double> c = G.centre(h.leaf_box[i]);
            lc[i] = make_double2(c.real(), c.imag());
        }
        for (int64_t d = 0; d < nd; ++d) {
            pxy[d] = make_double2(dxy[2 * d], dxy[2 * d + 1]);
            pn[d] = make_double2(dnrm[2 * d], dnrm[2 * d + 1]);
        }
        // flat runs: target leaf i owns entries [kof[i], kof[i + 1])
        std::vector<int64_t> kof(nl + 1, 0);
        for (int64_t i = 0; i < nl; ++i) {
            int64_t n_i = 0;
            for (int32_t lc_i : per[i]) n_i += segn[lc_i];
            kof[i + 1] = kof[i] + n_i;
        }
        const int64_t K = kof[nl];
        if (K >= INT32_MAX) return mh_fail(ctx, MH_ERR_INVALID_ARG, "near-field lists exceed 2^31 entries");
        std::vector<int32_t> fidx((size_t)K);
        std::vector<float4> f32((size_t)K);
        for (int64_t i = 0; i < nl; ++i) {
            int64_t k = kof[i];
            for (int32_t lc_i : per[i])
                for (int64_t d = seg0[lc_i]; d < seg0[lc_i] + segn[lc_i]; ++d, ++k) {
                    fidx[k] = (int32_t)d;
                    f32[k] = make_float4((float)(dxy[2 * d] - lc[i].x), (float)(dxy[2 * d + 1] - lc[i].y),
                                         (float)dnrm[2 * d], (float)dnrm[2 * d + 1]);
                }
        }
        // chunks of at most NEAR_CHUNK entries, equal within a leaf, largest first
        std::vector<NearChunk> ch;
        std::vector<int2> lred(nl, make_int2(0, 1));
        int32_t slots = 0;
        for (int64_t i = 0; i < nl; ++i) {
            const int64_t n_i = kof[i + 1] - kof[i];
            if (n_i == 0) continue;
            const int64_t nc = (n_i + NEAR_CHUNK - 1) / NEAR_CHUNK;
            lred[i] = make_int2(nc > 1 ? slots : 0, (int)nc);
            for (int64_t c = 0; c < nc; ++c)
                ch.push_back(NearChunk{(int32_t)i, (int32_t)(kof[i] + n_i * c / nc),
                                       (int32_t)(kof[i] + n_i * (c + 1) / nc), nc > 1 ? slots + (int32_t)c : -1});
            if (nc > 1) slots += (int32_t)nc;
        }
        std::stable_sort(ch.begin(), ch.end(),
                         [](const NearChunk& x, const NearChunk& y) { return x.k1 - x.k0 > y.k1 - y.k0; });
        D->n_chunks = (int64_t)ch.size();
        cudaStream_t st = ctx->stream;
        MH_ALLOC(ctx, D->chunks, std::max<size_t>(ch.size(), 1));
        MH_ALLOC(ctx, D->leaf_red, nl);
        MH_ALLOC(ctx, D->part, std::max<int64_t>((int64_t)slots * qq, 1));
        MH_ALLOC(ctx, D->red_cnt, nl);
        MH_ALLOC(ctx, D->flat_idx, std::max<int64_t>(K, 1));
        MH_ALLOC(ctx, D->flat32, std::max<int64_t>(K, 1));
        MH_ALLOC(ctx, D->leaf_c, nl);
        MH_ALLOC(ctx, D->dxy, std::max<int64_t>(nd, 1));
        MH_ALLOC(ctx, D->dnrm, std::max<int64_t>(nd, 1));
        if (!ch.empty())
            MH_CUDA(ctx, cudaMemcpyAsync(D->chunks.p, ch.data(), ch.size() * sizeof(NearChunk), cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(D->leaf_red.p, lred.data(), nl * sizeof(int2), cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemsetAsync(D->red_cnt.p, 0, nl * sizeof(unsigned), st));
        if (K) {
            MH_CUDA(ctx, cudaMemcpyAsync(D->flat_idx.p, fidx.data(), K * 4, cudaMemcpyHostToDevice, st));
            MH_CUDA(ctx, cudaMemcpyAsync(D->flat32.p, f32.data(), K * 16, cudaMemcpyHostToDevice, st));
        }
        MH_CUDA(ctx, cudaMemcpyAsync(D->leaf_c.p, lc.data(), nl * 16, cudaMemcpyHostToDevice, st));
        if (nd) {
            MH_CUDA(ctx, cudaMemcpyAsync(D->dxy.p, pxy.data(), nd * 16, cudaMemcpyHostToDevice, st));
            MH_CUDA(ctx, cudaMemcpyAsync(D->dnrm.p, pn.data(), nd * 16, cudaMemcpyHostToDevice, st));
        }
        MH_CUDA(ctx, cudaStreamSynchronize(st));
    }
    // upload the operator pool (volume translation operators + dipole blocks)
    cudaStream_t st = ctx->stream;
    const int64_t total = (int64_t)pool.data.size();
    MH_ALLOC(ctx, D->ops64, total);
    MH_ALLOC(ctx, D->ops32, total);
    MH_CUDA(ctx, cudaMemcpyAsync(D->ops64.p, pool.data.data(), total * 8, cudaMemcpyHostToDevice, st));
    {
        std::vector<float> f(pool.data.begin(), pool.data.end());
        MH_CUDA(ctx, cudaMemcpyAsync(D->ops32.p, f.data(), total * 4, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
    }
    MH_ALLOC(ctx, D->d_op_off, pool.off.size());
    MH_ALLOC(ctx, D->d_op_C, pool.C.size());
    MH_CUDA(ctx, cudaMemcpyAsync(D->d_op_off.p, pool.off.data(), pool.off.size() * 8, cudaMemcpyHostToDevice, st));
    MH_CUDA(ctx, cudaMemcpyAsync(D->d_op_C.p, pool.C.data(), pool.C.size() * 4, cudaMemcpyHostToDevice, st));
    std::vector<int> opC(pool.C.begin(), pool.C.end());
    // split ranges of the tensor-core sources: dipole multipoles (DM), locals (DL); the dipole
    // P2M / P2L operators (one task each, on the weights) stay on the CUDA cores
    const std::vector<TcImages::Range> rg = {{D->DM_off, P, nb, 0, 0}, {D->DL_off, P, nb, 0, 0}};
    int64_t need = 1;
    D->p2m.reset(new Phase());
    MH_TRY(build_phase(ctx, t_p2m, P, false, opC, D->p2m.get(), &need, &rg));
    D->m2l.reset(new Phase());
    MH_TRY(build_phase(ctx, t_m2l, P, false, opC, D->m2l.get(), &need, &rg));
    D->out.reset(new Phase());
    MH_TRY(build_phase(ctx, t_out, qq, !near_blocks, opC, D->out.get(), &need, &rg));
    D->out->dst_out = true;
    {
        std::vector<int64_t> off(pool.off.begin(), pool.off.end());
        std::vector<int32_t> rr(pool.R.begin(), pool.R.end()), cc(pool.C.begin(), pool.C.end());
        MH_TRY(build_tc_images(ctx, pool.data.data(), off, rr, cc, {D->p2m.get(), D->m2l.get(), D->out.get()}, rg,
                               &D->tc));
    }
    MH_ALLOC(ctx, D->vec, D->vec_len);
    // binary32 mirror with TC_POOL_PAD floats of slack at the end: the tensor-core gather
    // reads sources in aligned 16-byte windows that may reach past a vector's last entry
    MH_ALLOC(ctx, D->vec32, D->vec_len + TC_POOL_PAD);
    MH_ALLOC(ctx, D->temp, need);
    MH_CUDA(ctx, cudaMemsetAsync(D->vec.p, 0, D->vec_len * 8, st));
    MH_CUDA(ctx, cudaMemsetAsync(D->vec32.p, 0, (D->vec_len + TC_POOL_PAD) * 4, st));
    MH_TRY(D->side.create(ctx));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    V->dip = std::move(D);
    return MH_OK;
}

template <typename TOP>
static mh_status dipole_passes(mh_ctx* ctx, VolData* V, DipData* D, const TOP* ops) {
    TOP* pool = typed_pool<TOP>(D->vec, D->vec32);
    auto run = [&](const Phase* ph) {
        return run_phase_on<TOP>(ctx, ops, D->d_op_off.p, D->d_op_C.p, pool, D->vec.p, D->temp.p, ph,
                                 "dlp_fmm_contract", &D->tc);
    };
    MH_TRY(run(D->p2m.get()));
    MH_TRY(run_chain<TOP>(ctx, D->chain_up.get(), V->P, D->DM_off, D->DL_off, pool, true, "dlp_fmm_chain"));
    if (sizeof(TOP) == 4) MH_TRY(tc_split(ctx, D->tc, 0, D->vec32.p));   // multipoles final
    // boxes whose V and X lists hold no dipoles get no M2L / P2L task: their locals are zeroed
    // here, since the downward chain adds into the leaves' locals
    MH_CUDA(ctx, cudaMemsetAsync(pool + D->DL_off, 0, (D->DU_off - D->DL_off) * sizeof(TOP), ctx->stream));
    MH_TRY(run(D->m2l.get()));
    MH_TRY(run_chain<TOP>(ctx, V->chain.get(), V->P, D->DM_off, D->DL_off, pool, false, "dlp_fmm_chain"));
    if (sizeof(TOP) == 4) MH_TRY(tc_split(ctx, D->tc, 1, D->vec32.p));   // locals final
    return MH_OK;
}

template <typename TOP>
static mh_status dipole_out(mh_ctx* ctx, DipData* D, const TOP* ops) {
    return run_phase_on<TOP>(ctx, ops, D->d_op_off.p, D->d_op_C.p, typed_pool<TOP>(D->vec, D->vec32), D->vec.p,
                             D->temp.p, D->out.get(), "dlp_fmm_contract", &D->tc);
}

// w_sorted: dipole strengths in the leaf-sorted order given to volume_dipole_setup.
// Returns a device pointer to U^h at every volume node (leaf-major), valid until the next call.
mh_status volume_dipole_apply(mh_ctx* ctx, mh_tree* t, const double* w_sorted, mh_precision prec, const double** u) {
    VolData* V = static_cast<VolData*>(t->vol);
    if (!V || !V->dip) return mh_fail(ctx, MH_ERR_INVALID_ARG, "dipole multipole pass not set up");
    DipData* D = V->dip.get();
    prof_scope ps(ctx, "dlp_fmm");
    cudaStream_t st = ctx->stream;
    const bool mixed = prec == MH_PREC_MIXED;
    if (!D->near_blocks) MH_CUDA(ctx, cudaMemsetAsync(D->vec.p + D->DU_off, 0, t->n_leaves * D->qq * 8, st));
    if (mixed) {
        // weights in binary32 once: the contractions and the near-field kernel read them
        k_d2f<<<mh_grid(D->nd, 256), 256, 0, st>>>(w_sorted, D->vec32.p + D->W_off, D->nd);
        MH_LAUNCHED(ctx);
    } else {
        MH_CUDA(ctx, cudaMemcpyAsync(D->vec.p + D->W_off, w_sorted, D->nd * 8, cudaMemcpyDeviceToDevice, st));
    }
    // The near field reads the weights and adds into U^h only; the passes read the weights and
    // touch only the expansions until their output phase adds the far field to U^h.  Without
    // region timers the passes run on the side stream while the near field runs on the context
    // stream, joined before the output phase; with the timers everything runs in order on the
    // context stream.  Both forms add near, then far.
    const bool near = !D->near_blocks && D->n_chunks;
    const bool fork = near && !ctx->profiling && D->side.s;
    if (fork) {
        MH_TRY(D->side.begin(ctx, st));
        ctx->stream = D->side.s;
        const mh_status s = mixed ? dipole_passes<float>(ctx, V, D, D->ops32.p)
                                  : dipole_passes<double>(ctx, V, D, D->ops64.p);
        ctx->stream = st;
        MH_TRY(s);
        MH_TRY(D->side.end(ctx));
    }
    if (near) {
        prof_scope ps2(ctx, "dlp_near", 68.0 * D->near_pairs, 24.0 * (double)D->nd);
        const unsigned nb = (unsigned)D->n_chunks;
        double* out = D->vec.p + D->DU_off;
        if (mixed) {
            const float* w32 = D->vec32.p + D->W_off;
            const mh_dl32 c32 = mh_dl32_make(1.0 / D->inv_alpha, 30.0);
            const double pref32 = D->pref * D->inv_alpha * D->inv_alpha;
#define MH_NEAR32(NTV)                                                                                         \
    k_dip_near32<NTV><<<nb, NTV, 0, st>>>(t->nodes.p, D->chunks.p, D->leaf_red.p, D->leaf_c.p, D->flat_idx.p,  \
                                          D->flat32.p, w32, D->qq, c32, pref32, D->part.p, D->red_cnt.p, out)
            if (D->near_t == 128)
                MH_NEAR32(128);
            else if (D->near_t == 512)
                MH_NEAR32(512);
            else
                MH_NEAR32(256);
#undef MH_NEAR32
        } else {
            k_dip_near64<<<nb, NEAR_T, 0, st>>>(t->nodes.p, D->chunks.p, D->leaf_red.p, D->flat_idx.p, D->dxy.p,
                                                D->dnrm.p, D->vec.p + D->W_off, D->qq, D->inv_alpha, D->pref,
                                                D->part.p, D->red_cnt.p, out);
        }
        MH_LAUNCHED(ctx);
    }
    if (fork)
        MH_CUDA(ctx, cudaStreamWaitEvent(st, D->side.join, 0));
    else
        MH_TRY(mixed ? dipole_passes<float>(ctx, V, D, D->ops32.p) : dipole_passes<double>(ctx, V, D, D->ops64.p));
    MH_TRY(mixed ? dipole_out<float>(ctx, D, D->ops32.p) : dipole_out<double>(ctx, D, D->ops64.p));
    *u = D->vec.p + D->DU_off;
    return MH_OK;
}

// ---------------- on-surface double layer through the multipole method ----------------
//
// The trapezoid part of the discrete system (Section 3.2) without the dense operator: the
// boundary nodes are both the dipoles (strength w_d = sigma_d |y'_d| h) and the targets, and
//   u(x_i) = -(1/(2 pi alpha^2)) sum_{d != i} w_d (1/alpha) K1(r/alpha) (y_d - x_i).nu_d / r
// is formed by the dipole passes of the volume tree (P2M, M2M, M2L + P2L, L2L) followed by an
// output phase for point targets: per leaf, targets in groups of at most BIE_RT, each group with
// its L2P at the targets, M2P from its W list and direct dipole blocks from its U list (the
// leaf itself included, the target's own node left out).  All in binary64.
namespace {

constexpr int BIE_RT = 16;   // targets per output group (rows of every output operator)

struct BieData {
    int64_t nd = 0, n_groups = 0;
    int64_t W_off = 0, DM_off = 0, DL_off = 0, T_off = 0, vec_len = 0;
    double flops = 0, near_pairs = 0;
    dbuf<double> vec, temp, ops64;
    dbuf<int64_t> d_op_off;
    dbuf<int32_t> d_op_C;
    dbuf<int32_t> perm;   // sorted position -> node
    dbuf<int32_t> slot;   // node -> output slot (from T_off)
    std::unique_ptr<Phase> p2m, m2l, out;
    std::unique_ptr<DfChain> chain;   // M2M / L2L over the active boxes (own arrival counters)
};

// Angular part of an expansion row in the real form: v0 at n = 0, then 2 v_n cos(n th) and
// -2 v_n sin(n th).
void bie_row(double* row, int p, const double* v, double th) {
    row[0] = v[0];
    for (int n = 1; n <= p; ++n) {
        row[2 * n - 1] = 2 * v[n] * std::cos(n * th);
        row[2 * n] = -2 * v[n] * std::sin(n * th);
    }
}

__global__ void k_bie_gather_w(const double* __restrict__ w, const int32_t* __restrict__ perm, int64_t n,
                               double* __restrict__ ws) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) ws[i] = w[perm[i]];
}

__global__ void k_bie_scatter_u(const double* __restrict__ t, const int32_t* __restrict__ slot, int64_t n,
                                double* __restrict__ u) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) u[i] = t[slot[i]];
}

}  // namespace

mh_status volume_bie_setup(mh_ctx* ctx, mh_tree* t, double alpha, int p, const double* xy, const double* nrm,
                           const int32_t* leaf, int64_t nd) {
    MH_TRY(volume_ensure(ctx, t, alpha, p));
    VolData* V = static_cast<VolData*>(t->vol);
    const int P = 2 * p + 1;
    const double k = 1.0 / alpha, pref = 1.0 / (2.0 * MH_PI * alpha * alpha);
    HostTree h;
    MH_TRY(fetch_tree(ctx, t, &h));
    const int64_t nb = t->n_boxes, nl = t->n_leaves;
    const DipGeo G = dip_geo(t, h, p, k);
    // nodes sorted by leaf (stable: node order within a leaf)
    std::vector<int32_t> perm(nd);
    for (int64_t i = 0; i < nd; ++i) {
        if (leaf[i] < 0 || leaf[i] >= nl) return mh_fail(ctx, MH_ERR_GEOMETRY, "boundary node %lld has no leaf", (long long)i);
        perm[i] = (int32_t)i;
    }
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t c) { return leaf[a] < leaf[c]; });
    std::vector<double> sxy(2 * nd), snrm(2 * nd);
    std::vector<int64_t> seg0(nl, -1), segn(nl, 0);
    for (int64_t j = 0; j < nd; ++j) {
        const int32_t i = perm[j];
        sxy[2 * j] = xy[2 * i];
        sxy[2 * j + 1] = xy[2 * i + 1];
        snrm[2 * j] = nrm[2 * i];
        snrm[2 * j + 1] = nrm[2 * i + 1];
        if (seg0[leaf[i]] < 0) seg0[leaf[i]] = j;
        segn[leaf[i]]++;
    }
    std::unique_ptr<BieData> B(new BieData());
    B->nd = nd;
    for (int64_t i = 0; i < nl; ++i) B->n_groups += (segn[i] + BIE_RT - 1) / BIE_RT;
    B->W_off = 0;
    B->DM_off = nd;
    B->DL_off = B->DM_off + nb * P;
    B->T_off = B->DL_off + nb * P;
    B->vec_len = B->T_off + B->n_groups * BIE_RT;
    OpPool pool = V->pool_host;
    std::vector<Task> t_p2m, t_m2l, t_out;
    const std::vector<char> active = dipole_active_boxes(h, segn);
    dipole_source_tasks(G, V, pool, p, k, pref, sxy.data(), snrm.data(), seg0, segn, B->W_off, B->DM_off, B->DL_off,
                        t_p2m, t_m2l, &active, true);
    MH_TRY(build_chain(ctx, t, h, P, V->pool_host, V->op_m2m, V->op_l2l, &active, &B->chain));
    std::vector<int32_t> slot(nd);
    std::vector<double> buf, v(p + 2), Kb(p + 3);
    int64_t gi = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int lf = h.box_leaf[b];
        if (lf < 0 || segn[lf] == 0) continue;
        const int l = G.lev((int)b);
        const std::complex<double> cb = G.centre((int)b);
        for (int64_t g0 = 0; g0 < segn[lf]; g0 += BIE_RT, ++gi) {
            const int cnt = (int)std::min<int64_t>(BIE_RT, segn[lf] - g0);
            const int64_t dst = B->T_off + gi * BIE_RT;
            auto tgt = [&](int i) {
                const int64_t j = seg0[lf] + g0 + i;
                return std::complex<double>(sxy[2 * j], sxy[2 * j + 1]);
            };
            for (int i = 0; i < cnt; ++i) slot[perm[seg0[lf] + g0 + i]] = (int32_t)(gi * BIE_RT + i);
            // L2P at the targets
            if (l >= 2) {
                buf.assign((size_t)BIE_RT * P, 0.0);
                for (int i = 0; i < cnt; ++i) {
                    const std::complex<double> z = tgt(i) - cb;
                    for (int n = 0; n <= p; ++n) v[n] = h_in(n, k * std::abs(z)) / G.Is[l][n];
                    bie_row(&buf[(size_t)i * P], p, v.data(), std::arg(z));
                }
                t_out.push_back(Task{pool.add(BIE_RT, P, buf.data()), B->DL_off + b * P, dst});
                B->flops += 2.0 * BIE_RT * P;
            }
            // W list: M2P at the targets
            for (int j = h.off[2][b]; j < h.off[2][b + 1]; ++j) {
                const int c = h.item[2][j];
                const std::complex<double> cc = G.centre(c);
                const int lc = G.lev(c);
                buf.assign((size_t)BIE_RT * P, 0.0);
                for (int i = 0; i < cnt; ++i) {
                    const std::complex<double> z = tgt(i) - cc;
                    h_kn_all(k * std::abs(z), p, Kb.data());
                    for (int n = 0; n <= p; ++n) v[n] = G.Is[lc][n] * Kb[n];
                    bie_row(&buf[(size_t)i * P], p, v.data(), std::arg(z));
                }
                t_out.push_back(Task{pool.add(BIE_RT, P, buf.data()), B->DM_off + (int64_t)c * P, dst});
                B->flops += 2.0 * BIE_RT * P;
            }
            // U list: direct dipole blocks (the leaf itself included; r = 0 is the target's own node)
            for (int j = h.off[0][b]; j < h.off[0][b + 1]; ++j) {
                const int lc = h.box_leaf[h.item[0][j]];
                if (segn[lc] == 0) continue;
                const int nc = (int)segn[lc];
                buf.assign((size_t)BIE_RT * nc, 0.0);
                for (int i = 0; i < cnt; ++i) {
                    const std::complex<double> x = tgt(i);
                    for (int jj = 0; jj < nc; ++jj) {
                        const int64_t d = seg0[lc] + jj;
                        const double dx = sxy[2 * d] - x.real(), dy = sxy[2 * d + 1] - x.imag();
                        const double r = std::hypot(dx, dy);
                        if (r > 0)
                            buf[(size_t)i * nc + jj] =
                                -pref * h_k1(r * k) * k * (dx * snrm[2 * d] + dy * snrm[2 * d + 1]) / r;
                    }
                }
                dip_add_split(pool, BIE_RT, nc, buf, B->W_off + seg0[lc], dst, t_out);
                B->near_pairs += (double)cnt * nc;
                B->flops += 2.0 * BIE_RT * nc;
            }
        }
    }
    cudaStream_t st = ctx->stream;
    const int64_t total = (int64_t)pool.data.size();
    MH_ALLOC(ctx, B->ops64, total);
    MH_CUDA(ctx, cudaMemcpyAsync(B->ops64.p, pool.data.data(), total * 8, cudaMemcpyHostToDevice, st));
    MH_ALLOC(ctx, B->d_op_off, pool.off.size());
    MH_ALLOC(ctx, B->d_op_C, pool.C.size());
    MH_CUDA(ctx, cudaMemcpyAsync(B->d_op_off.p, pool.off.data(), pool.off.size() * 8, cudaMemcpyHostToDevice, st));
    MH_CUDA(ctx, cudaMemcpyAsync(B->d_op_C.p, pool.C.data(), pool.C.size() * 4, cudaMemcpyHostToDevice, st));
    std::vector<int> opC(pool.C.begin(), pool.C.end());
    int64_t need = 1;
    B->p2m.reset(new Phase());
    MH_TRY(build_phase(ctx, t_p2m, P, false, opC, B->p2m.get(), &need));
    B->m2l.reset(new Phase());
    MH_TRY(build_phase(ctx, t_m2l, P, false, opC, B->m2l.get(), &need));
    B->out.reset(new Phase());
    MH_TRY(build_phase(ctx, t_out, BIE_RT, false, opC, B->out.get(), &need));
    B->out->dst_out = true;
    B->flops += B->p2m->flops + B->m2l->flops;
    MH_ALLOC(ctx, B->vec, B->vec_len);
    MH_ALLOC(ctx, B->temp, need);
    MH_CUDA(ctx, cudaMemsetAsync(B->vec.p, 0, B->vec_len * 8, st));
    MH_ALLOC(ctx, B->perm, std::max<int64_t>(nd, 1));
    MH_ALLOC(ctx, B->slot, std::max<int64_t>(nd, 1));
    if (nd) {
        MH_CUDA(ctx, cudaMemcpyAsync(B->perm.p, perm.data(), nd * 4, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(B->slot.p, slot.data(), nd * 4, cudaMemcpyHostToDevice, st));
    }
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    V->bie = std::move(B);
    return MH_OK;
}

bool volume_bie_ready(const mh_tree* t) {
    const VolData* V = static_cast<const VolData*>(t->vol);
    return V && V->bie;
}

// w: dipole strengths in node order (device); u: the trapezoid double layer at every node, in
// node order (device), as defined above.  Runs on the context stream, with its own M2M / L2L
// chain over the boxes that hold boundary nodes.
mh_status volume_bie_apply(mh_ctx* ctx, mh_tree* t, const double* w, double* u) {
    VolData* V = static_cast<VolData*>(t->vol);
    if (!V || !V->bie) return mh_fail(ctx, MH_ERR_INVALID_ARG, "on-surface multipole pass not set up");
    BieData* B = V->bie.get();
    if (B->nd == 0) return MH_OK;
    prof_scope ps(ctx, "bie_fmm", B->flops, 0.0);
    cudaStream_t st = ctx->stream;
    const unsigned g = (unsigned)mh_grid(B->nd, 256);
    k_bie_gather_w<<<g, 256, 0, st>>>(w, B->perm.p, B->nd, B->vec.p + B->W_off);
    MH_LAUNCHED(ctx);
    auto run = [&](const Phase* ph) {
        return run_phase_on<double>(ctx, B->ops64.p, B->d_op_off.p, B->d_op_C.p, B->vec.p, B->vec.p, B->temp.p, ph,
                                    "bie_fmm_contract");
    };
    MH_TRY(run(B->p2m.get()));
    MH_TRY(run_chain<double>(ctx, B->chain.get(), V->P, B->DM_off, B->DL_off, B->vec.p, true, "bie_fmm_chain"));
    MH_CUDA(ctx, cudaMemsetAsync(B->vec.p + B->DL_off, 0, (B->T_off - B->DL_off) * 8, st));
    MH_TRY(run(B->m2l.get()));
    MH_TRY(run_chain<double>(ctx, B->chain.get(), V->P, B->DM_off, B->DL_off, B->vec.p, false, "bie_fmm_chain"));
    MH_TRY(run(B->out.get()));
    k_bie_scatter_u<<<g, 256, 0, st>>>(B->vec.p + B->T_off, B->slot.p, B->nd, u);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

mh_status volume_set_near_tile(mh_ctx* ctx, mh_tree* t, int threads) {
    VolData* V = static_cast<VolData*>(t->vol);
    if (!V || !V->dip) return mh_fail(ctx, MH_ERR_INVALID_ARG, "double-layer multipole pass not set up");
    if (threads != 128 && threads != 256 && threads != 512)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "near-field tile must be 128, 256 or 512 threads");
    if (threads < V->dip->qq) return mh_fail(ctx, MH_ERR_INVALID_ARG, "near-field tile smaller than a leaf");
    V->dip->near_t = threads;
    return MH_OK;
}

int volume_near_tile(const mh_tree* t) {
    const VolData* V = static_cast<const VolData*>(t->vol);
    return V && V->dip ? V->dip->near_t : 0;
}

void volume_free(mh_tree* t) {
    delete static_cast<VolData*>(t->vol);
    t->vol = nullptr;
}

// The near tables read only the node values and write U^h; the passes touch only the
// expansions until the output phase adds L2P and M2P to U^h.  Without region timers the passes
// run on the side stream while the near phase runs on the context stream, joined before the
// output phase; with the timers everything runs in order on the context stream.  Both forms
// write U^h as near, then add far.
template <typename TOP>
static mh_status volume_passes(mh_ctx* ctx, VolData* V, const TOP* ops) {
    TOP* pool = typed_pool<TOP>(V->vec, V->vec32);
    MH_TRY(run_phase(ctx, V, ops, V->p2m.get()));
    MH_TRY(run_chain<TOP>(ctx, V->chain.get(), V->P, V->M_off, V->L_off, pool, true, "volume_chain"));
    if (sizeof(TOP) == 4) MH_TRY(tc_split(ctx, V->tc, 1, V->vec32.p));   // multipoles final
    MH_TRY(run_phase(ctx, V, ops, V->m2l.get()));
    MH_TRY(run_chain<TOP>(ctx, V->chain.get(), V->P, V->M_off, V->L_off, pool, false, "volume_chain"));
    if (sizeof(TOP) == 4) MH_TRY(tc_split(ctx, V->tc, 2, V->vec32.p));   // locals final
    return MH_OK;
}

template <typename TOP>
static mh_status volume_run(mh_ctx* ctx, mh_tree* t, VolData* V, const TOP* ops) {
    TOP* pool = typed_pool<TOP>(V->vec, V->vec32);
    cudaStream_t main = ctx->stream;
    if (!V->near_cover)
        MH_CUDA(ctx, cudaMemsetAsync(V->vec.p + V->U_off, 0, t->n_leaves * V->qq * 8, main));
    const bool near = V->near->n_tasks > 0;
    const bool fork = near && !ctx->profiling && V->side.s;
    if (fork) {
        MH_TRY(V->side.begin(ctx, main));
        ctx->stream = V->side.s;
        const mh_status s = volume_passes<TOP>(ctx, V, ops);
        ctx->stream = main;
        MH_TRY(s);
        MH_TRY(V->side.end(ctx));
    }
    if (near)
        MH_TRY(run_phase_on<TOP>(ctx, ops, V->d_op_off.p, V->d_op_C.p, pool, V->vec.p, V->temp_near.p,
                                 V->near.get(), "volume_contract", &V->tc));
    if (fork)
        MH_CUDA(ctx, cudaStreamWaitEvent(main, V->side.join, 0));
    else
        MH_TRY(volume_passes<TOP>(ctx, V, ops));
    MH_TRY(run_phase(ctx, V, ops, V->out.get()));
    return MH_OK;
}

mh_status volume_apply(mh_ctx* ctx, mh_tree* t, double alpha, int p, const double* b, double* up,
                       mh_precision prec) {
    VolData* V = static_cast<VolData*>(t->vol);
    if (!V || V->alpha != alpha || V->p != p) {
        delete V;
        V = new VolData();
        t->vol = V;
        mh_status s = volume_setup(ctx, t, alpha, p, V);
        if (s != MH_OK) {
            delete V;
            t->vol = nullptr;
            return s;
        }
    }
    const int64_t nn = t->n_nodes;
    prof_scope ps(ctx, "volume_apply");
    if (prec == MH_PREC_MIXED) {
        // node values in binary32 once: every contraction then gathers binary32
        k_d2f<<<mh_grid(nn, 256), 256, 0, ctx->stream>>>(b, V->vec32.p + V->B_off, nn);
        MH_LAUNCHED(ctx);
        MH_TRY(tc_split(ctx, V->tc, 0, V->vec32.p));   // node values final
        MH_TRY(volume_run<float>(ctx, t, V, V->ops32.p));
    } else {
        MH_CUDA(ctx, cudaMemcpyAsync(V->vec.p + V->B_off, b, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        MH_TRY(volume_run<double>(ctx, t, V, V->ops64.p));
    }
    MH_CUDA(ctx, cudaMemcpyAsync(up, V->vec.p + V->U_off, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return MH_OK;
}

extern "C" mh_status mh_tree_check(mh_ctx* ctx, mh_tree* t) {
    if (!ctx || !t) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    VolData* V = static_cast<VolData*>(t->vol);
    if (!V) return MH_OK;
    int code = 0;
    for (TcImages* T : {&V->tc, V->dip ? &V->dip->tc : static_cast<TcImages*>(nullptr)}) {
        if (!T || !T->err.p) continue;
        int e = 0;
        MH_CUDA(ctx, cudaMemcpy(&e, T->err.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            code = e;
            MH_CUDA(ctx, cudaMemset(T->err.p, 0, sizeof(int)));
        }
    }
    if (code)
        return mh_fail(ctx, MH_ERR_TIMEOUT, "a tensor-core contraction gave up waiting for its %s",
                       code == 1 ? "operator copy" : "matrix products");
    return MH_OK;
}

extern "C" mh_status mh_volume_potential(mh_ctx* ctx, mh_tree* t, double alpha, int p, const double* b_dev,
                                         double* up_dev, mh_precision prec) {
    if (!ctx || !t || !b_dev || !up_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (!(alpha > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "alpha must be positive");
    if (p < 1 || p > 40) return mh_fail(ctx, MH_ERR_INVALID_ARG, "p must be in 1..40");
    MH_TRY(volume_apply(ctx, t, alpha, p, b_dev, up_dev, prec));
    return mh_tree_check(ctx, t);
}
