// Learned warm start of the boundary solve (the paper states no GMRES initial guess;
// Section 3.2 and Section 4 give only the tolerance).  With r = b - A sigma^N the
// residual of the previous-step start, a tanh MLP on the truncated Fourier coefficients
// of r predicts the correction delta ~ A^{-1} r = r + (smooth part), and a minimum-
// residual step along delta picks the start (formulas in include/mh.h).
//
// Kernels:
//   k_features      truncated DFT of every curve (warp per coefficient, float-float sums)
//   k_synth         Fourier synthesis plus r at every node (float-float sums)
//   k_gemv_layer    one network layer for one input vector, weights binary32 / bfloat16 /
//                   bfloat16 pair, binary32 accumulation: HBM/L2-bound matrix-vector work,
//                   so the tensor pipe is not used
//   k_gemm<T, EPI>  tiled matrix product (64 x 64 tiles, 4 x 4 outputs per thread) with
//                   bias / tanh / tanh-derivative epilogues: binary32 training passes and
//                   the binary64 closed-form start
//   k_chol, k_trinv_lower   one-block Cholesky and triangular inverse (CholeskyQR2 and
//                   the ridge normal equations, sizes <= 1025)
//   k_adam          Adam update (Kingma & Ba) with bias correction
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "mh_internal.cuh"

struct mh_net {
    int n_curves = 0, K = 0, w = 0, max_nodes = 0;
    int64_t d = 0, n_bnd = 0, n_params = 0;
    int64_t oW[4] = {0, 0, 0, 0}, ob[4] = {0, 0, 0, 0};
    int lin[4] = {0, 0, 0, 0}, lout[4] = {0, 0, 0, 0};
    std::vector<int32_t> nn, off;
    dbuf<int32_t> d_nn, d_off;
    dbuf<double> tw;                 // [n_bnd][2] cos, sin of 2 pi m / N_k (per curve, m < N_k)
    dbuf<float2> tw32;               // the same, rounded to binary32
    dbuf<float> v32;                 // binary32 copy of the vector being transformed
    double gx = 1.0, gy = 1.0;
    dbuf<float> P;                   // parameters (layout in mh.h)
    dbuf<uint16_t> Bhi, Blo;         // bfloat16 copies of P (only the weight blocks are read)
    bool bf_ready = false;
    // one-vector inference scratch
    dbuf<float> xin, hA, hB, yout;
    dbuf<double> rbuf, ebuf, scal;   // scal: |r|, 1/(|r| g), <r,w>, <w,w>
    // training scratch
    dbuf<float> G, Mo, Vo, best, xb, yb, yh, act[3], dzd, dzw1, dzw2;
    dbuf<double> lpart;
    int64_t cap_rows = 0;
};

namespace {

constexpr int GEMM_T = 64;   // tile edge
constexpr int GEMM_K = 16;   // k slab

enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_TANH = 2, EPI_TANH_BACK = 3 };

// C[i][j] = epi(sum_k A(i,k) B(k,j)); A(i,k) = A[i sam + k sak], B(k,j) = B[k sbk + j sbn].
// EPI_BIAS: + bias[j]; EPI_BIAS_TANH: tanh(. + bias[j]); EPI_TANH_BACK: . * (1 - aux[i][j]^2).
template <typename T, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const T* __restrict__ A, int64_t sam, int64_t sak,
                                              const T* __restrict__ B, int64_t sbk, int64_t sbn, T* __restrict__ C,
                                              int64_t ldc, const T* __restrict__ bias, const T* __restrict__ aux) {
    __shared__ T As[GEMM_K][GEMM_T + 1];
    __shared__ T Bs[GEMM_K][GEMM_T + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * GEMM_T, j0 = blockIdx.x * GEMM_T;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
    for (int k0 = 0; k0 < K; k0 += GEMM_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            int ii, kk;
            if (sak == 1) {
                kk = e & 15;
                ii = e >> 4;
            } else {
                ii = e & 63;
                kk = e >> 6;
            }
            int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < K) ? A[(int64_t)gi * sam + (int64_t)gk * sak] : T(0);
            int jj;
            if (sbn == 1) {
                jj = e & 63;
                kk = e >> 6;
            } else {
                kk = e & 15;
                jj = e >> 4;
            }
            const int gj = j0 + jj;
            gk = k0 + kk;
            Bs[kk][jj] = (gj < N && gk < K) ? B[(int64_t)gk * sbk + (int64_t)gj * sbn] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GEMM_K; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
            if (i >= M || j >= N) continue;
            T v = acc[r][c];
            if (EPI == EPI_BIAS || EPI == EPI_BIAS_TANH) v += bias[j];
            if (EPI == EPI_BIAS_TANH) v = tanh(v);
            if (EPI == EPI_TANH_BACK) {
                const T a = aux[(int64_t)i * ldc + j];
                v *= T(1) - a * a;
            }
            C[(int64_t)i * ldc + j] = v;
        }
}

template <typename T, int EPI>
void gemm(cudaStream_t st, int M, int N, int K, const T* A, int64_t sam, int64_t sak, const T* B, int64_t sbk,
          int64_t sbn, T* C, int64_t ldc, const T* bias = nullptr, const T* aux = nullptr) {
    dim3 grid((unsigned)((N + GEMM_T - 1) / GEMM_T), (unsigned)((M + GEMM_T - 1) / GEMM_T));
    k_gemm<T, EPI><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, aux);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide binary64 sum (blockDim.x multiple of 32, <= 1024); the result is valid in thread 0.
__device__ double block_sum_d(double v) {
    __shared__ double sh[32];
    v = warp_sum_d(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    if (warp == 0) v = warp_sum_d(v);
    return v;
}

__global__ void k_twiddle(const int32_t* __restrict__ nn, const int32_t* __restrict__ off, double* tw) {
    const int c = blockIdx.y;
    const int n = nn[c];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s, co;
    sincospi(2.0 * (double)j / (double)n, &s, &co);
    tw[2 * (off[c] + j)] = co;
    tw[2 * (off[c] + j) + 1] = s;
}

// Float-float accumulation (TwoSum; the product's rounding error from fma folded into the low
// part): sums of products of binary32 numbers to ~binary64 accuracy on the binary32 pipe (the
// binary64 pipe runs at 1/64 of its rate here).
__device__ __forceinline__ void ff_mac(float& hi, float& lo, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float t = hi + p;
    const float bb = t - hi;
    lo += ((hi - (t - bb)) + (p - bb)) + e;
    hi = t;
}

__device__ __forceinline__ void ff_warp_sum(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        const float t = hi + oh, bb = t - hi;
        lo += ((hi - (t - bb)) + (oh - bb)) + ol;
        hi = t;
    }
}

__global__ void k_to_f32(const double* __restrict__ v, int64_t n, float* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)v[i];
}

__global__ void k_tw_f32(const double* __restrict__ tw, int64_t n, float2* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)tw[2 * i], (float)tw[2 * i + 1]);
}

// x[c][2k], x[c][2k+1] = scale * (1/N_c) sum_j v_j (cos, -sin)(2 pi j k / N_c); one warp each,
// binary32 inputs and twiddles, float-float sums.
__global__ void k_features(const float* __restrict__ v, const float2* __restrict__ tw, const int32_t* __restrict__ nn,
                           const int32_t* __restrict__ off, int n_curves, int K, const double* __restrict__ scale,
                           float* __restrict__ x) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (gw >= n_curves * K) return;
    const int c = gw / K, k = gw - c * K;
    const int n = nn[c], o = off[c];
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    // twiddle index m = j k mod n, advanced by 32 k mod n per lane step
    const int step = (int)((32LL * k) % n);
    int m = (int)(((int64_t)lane * k) % n);
    for (int j = lane; j < n; j += 32) {
        const float vj = v[o + j];
        const float2 t = tw[o + m];
        ff_mac(rh, rl, vj, t.x);
        ff_mac(ih, il, -vj, t.y);
        m += step;
        if (m >= n) m -= n;
    }
    ff_warp_sum(rh, rl);
    ff_warp_sum(ih, il);
    if (lane == 0) {
        const double s = scale[0] / n;
        x[(int64_t)c * 2 * K + 2 * k] = (float)(((double)rh + (double)rl) * s);
        x[(int64_t)c * 2 * K + 2 * k + 1] = (float)(((double)ih + (double)il) * s);
    }
}

// out_j = r_j + scal[0] * gy * (Re c_0 + 2 sum_{k>=1} Re(c_k e^{2 pi i j k / N})).  Eight threads
// per node split the modes (k = 1 + g + 8 i); grid (chunks of 32 nodes, curves); binary32
// twiddles, float-float sums.
__global__ void k_synth(const float* __restrict__ y, const float2* __restrict__ tw, const int32_t* __restrict__ nn,
                        const int32_t* __restrict__ off, int K, const double* __restrict__ r,
                        const double* __restrict__ scal, double gy, double* __restrict__ out) {
    extern __shared__ float ys[];
    const int c = blockIdx.y;
    for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) ys[t] = y[(int64_t)c * 2 * K + t];
    __syncthreads();
    const int n = nn[c], o = off[c];
    const int j = blockIdx.x * (blockDim.x >> 3) + (threadIdx.x >> 3), g = threadIdx.x & 7;
    const int jj = j < n ? j : 0;
    float vh = 0.f, vl = 0.f;
    int m = (int)(((int64_t)jj * (1 + g)) % n);
    const int step = (int)((8LL * jj) % n);
    for (int k = 1 + g; k < K; k += 8) {
        const float2 t = tw[o + m];
        ff_mac(vh, vl, ys[2 * k], t.x);
        ff_mac(vh, vl, -ys[2 * k + 1], t.y);
        m += step;
        if (m >= n) m -= n;
    }
#pragma unroll
    for (int msk = 1; msk < 8; msk <<= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, vh, msk), ol = __shfl_xor_sync(0xffffffffu, vl, msk);
        const float t = vh + oh, bb = t - vh;
        vl += ((vh - (t - bb)) + (oh - bb)) + ol;
        vh = t;
    }
    if (g == 0 && j < n)
        out[o + j] = r[o + j] + scal[0] * gy * ((double)ys[0] + 2.0 * ((double)vh + (double)vl));
}

__device__ __forceinline__ void bf16x8(uint4 h, float* f) {
    f[0] = __uint_as_float(h.x << 16);
    f[1] = __uint_as_float(h.x & 0xffff0000u);
    f[2] = __uint_as_float(h.y << 16);
    f[3] = __uint_as_float(h.y & 0xffff0000u);
    f[4] = __uint_as_float(h.z << 16);
    f[5] = __uint_as_float(h.z & 0xffff0000u);
    f[6] = __uint_as_float(h.w << 16);
    f[7] = __uint_as_float(h.w & 0xffff0000u);
}

// y[row] = act(sum_k W[row][k] x[k] + b[row]) for one input vector; SPLIT warps per row
// share the row (k-slices interleaved by 32 lanes x SPLIT), x in shared memory.  in is a
// multiple of 8 (16-byte rows for the bfloat16 loads).
template <int ARITH, int SPLIT>
__global__ void __launch_bounds__(256) k_gemv_layer(const float* __restrict__ W32, const uint16_t* __restrict__ Whi,
                                                    const uint16_t* __restrict__ Wlo, const float* __restrict__ bias,
                                                    const float* __restrict__ x, int in, int out, int act,
                                                    float* __restrict__ y) {
    extern __shared__ float xs[];
    __shared__ float part[8];
    for (int k = threadIdx.x; k < in; k += blockDim.x) xs[k] = x[k];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (8 / SPLIT) + warp / SPLIT, sl = warp % SPLIT;
    float acc = 0.f;
    const float4* xv = reinterpret_cast<const float4*>(xs);
    if (row < out) {
        if (ARITH == MH_NET_FP32) {
            const float4* wr = reinterpret_cast<const float4*>(W32 + (int64_t)row * in);
            for (int k4 = lane + 32 * sl; k4 < in / 4; k4 += 32 * SPLIT) {
                const float4 a = __ldg(wr + k4), b = xv[k4];
                acc = fmaf(a.x, b.x, acc);
                acc = fmaf(a.y, b.y, acc);
                acc = fmaf(a.z, b.z, acc);
                acc = fmaf(a.w, b.w, acc);
            }
        } else {
            const uint4* hr = reinterpret_cast<const uint4*>(Whi + (int64_t)row * in);
            const uint4* lr = reinterpret_cast<const uint4*>(Wlo + (int64_t)row * in);
            for (int k8 = lane + 32 * sl; k8 < in / 8; k8 += 32 * SPLIT) {
                float wv[8];
                bf16x8(__ldg(hr + k8), wv);
                if (ARITH == MH_NET_BF16X2) {
                    float lv[8];
                    bf16x8(__ldg(lr + k8), lv);
#pragma unroll
                    for (int e = 0; e < 8; ++e) wv[e] += lv[e];
                }
                const float4 b0 = xv[2 * k8], b1 = xv[2 * k8 + 1];
                acc = fmaf(wv[0], b0.x, acc);
                acc = fmaf(wv[1], b0.y, acc);
                acc = fmaf(wv[2], b0.z, acc);
                acc = fmaf(wv[3], b0.w, acc);
                acc = fmaf(wv[4], b1.x, acc);
                acc = fmaf(wv[5], b1.y, acc);
                acc = fmaf(wv[6], b1.z, acc);
                acc = fmaf(wv[7], b1.w, acc);
            }
        }
    }
    acc = warp_sum_f(acc);
    if (SPLIT > 1) {
        if (lane == 0) part[warp] = acc;
        __syncthreads();
        if (sl != 0) return;
        for (int q = 1; q < SPLIT; ++q) acc += part[warp + q];
    }
    if (lane == 0 && row < out) {
        const float z = acc + bias[row];
        y[row] = act ? tanhf(z) : z;
    }
}

// bfloat16 (round to nearest even) of w, and of the remainder w - hi.
__device__ __forceinline__ uint16_t bf16_rne(float f) {
    uint32_t u = __float_as_uint(f);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

__global__ void k_to_bf16(const float* __restrict__ p, int64_t n, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float f = p[i];
        const uint16_t h = bf16_rne(f);
        hi[i] = h;
        lo[i] = bf16_rne(f - __uint_as_float((uint32_t)h << 16));
    }
}

// Single block: out = sqrt(sum v^2) and its scale 1/(out g) (0 when out = 0).
__global__ void k_norm_scale(const double* __restrict__ v, int64_t n, double g, double* scal) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(v[i], v[i], s);
    s = block_sum_d(s);
    if (threadIdx.x == 0) {
        const double nr = sqrt(s);
        scal[0] = nr;
        scal[1] = nr > 0.0 ? 1.0 / (nr * g) : 0.0;
    }
}

// Single block: scal[2] = <r, w>, scal[3] = <w, w>.
__global__ void k_dot2(const double* __restrict__ r, const double* __restrict__ w, int64_t n, double* scal) {
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        a = fma(r[i], w[i], a);
        b = fma(w[i], w[i], b);
    }
    a = block_sum_d(a);
    __syncthreads();
    b = block_sum_d(b);
    if (threadIdx.x == 0) {
        scal[2] = a;
        scal[3] = b;
    }
}

// x0 = sigma + c dir, r0 = r - c w with c = <r,w>/<w,w> (0 if not finite / w = 0);
// save (nullable) receives the incoming sigma first.
__global__ void k_line(const double* sigma, const double* __restrict__ dir, const double* r, const double* __restrict__ w,
                       const double* __restrict__ scal, int64_t n, double* x0, double* r0, double* save,
                       double* c_out) {
    const double ww = scal[3];
    double c = ww > 0.0 ? scal[2] / ww : 0.0;
    if (!isfinite(c)) c = 0.0;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0 && c_out) c_out[0] = c;
    if (i >= n) return;
    const double s = sigma[i];
    if (save) save[i] = s;
    x0[i] = fma(c, dir[i], s);
    r0[i] = fma(-c, w[i], r[i]);
}

__global__ void k_axmy(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i];
}

// out = a - b - c
__global__ void k_sub3(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                       int64_t n, double* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i] - c[i];
}

// out = rhs - out  (out holds A x on entry)
__global__ void k_resid(const double* __restrict__ rhs, double* out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = rhs[i] - out[i];
}

__global__ void k_gather_rows(const float* __restrict__ X, const int32_t* __restrict__ idx, int64_t rows, int64_t d,
                              float scale, float* __restrict__ out) {
    const int64_t total = rows * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / d, c = e - r * d;
        const int64_t src = idx ? (int64_t)idx[r] : r;
        out[e] = X[src * d + c] * scale;
    }
}

// dz = (yh - t) * inv; per-block partial sums of (yh - t)^2 (binary64) into part.
__global__ void k_loss_dz(const float* __restrict__ yh, const float* __restrict__ t, int64_t n, float inv,
                          float* __restrict__ dz, double* __restrict__ part) {
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float df = yh[e] - t[e];
        if (dz) dz[e] = df * inv;
        s = fma((double)df, (double)df, s);
    }
    s = block_sum_d(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double scale, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum_d(s);
    if (threadIdx.x == 0) out[0] = s * scale;
}

__global__ void k_colsum(const float* __restrict__ z, int64_t rows, int64_t cols, float* __restrict__ out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= cols) return;
    double s = 0.0;
    for (int64_t i = 0; i < rows; ++i) s += z[i * cols + j];
    out[j] = (float)s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// ---- closed-form start (binary64) ----
__global__ void k_f2d(const float* __restrict__ x, int64_t n, double scale, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)x[i] * scale;
}

__global__ void k_sumsq_f(const float* __restrict__ x, int64_t n, double* __restrict__ part) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma((double)x[i], (double)x[i], s);
    s = block_sum_d(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// column means of X (rows x cols) and X -= mean (in place)
__global__ void k_center(double* X, int64_t rows, int64_t cols, double* __restrict__ mu) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= cols) return;
    double s = 0.0;
    for (int64_t i = 0; i < rows; ++i) s += X[i * cols + j];
    s /= (double)rows;
    mu[j] = s;
    for (int64_t i = 0; i < rows; ++i) X[i * cols + j] -= s;
}

__global__ void k_colrms_floor(const double* __restrict__ Z, int64_t rows, int cols, double* __restrict__ s) {
    __shared__ double smax;
    double mx = 0.0;
    for (int j = threadIdx.x; j < cols; j += blockDim.x) {
        double a = 0.0;
        for (int64_t i = 0; i < rows; ++i) a = fma(Z[i * cols + j], Z[i * cols + j], a);
        a = sqrt(a / (double)rows);
        s[j] = a;
        mx = fmax(mx, a);
    }
    // block max
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, wm[i]);
        smax = m;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cols; j += blockDim.x) s[j] = fmax(s[j], 1e-8 * smax);
}

// W1[j][i] = eps Q[i][j] / s[j]  (Q: d x w), b1[j] = -sum_i W1[j][i] mu[i]; warp per j.
__global__ void k_first_layer(const double* __restrict__ Q, const double* __restrict__ s, const double* __restrict__ mu,
                              int64_t d, int w, double eps, float* __restrict__ W1, float* __restrict__ b1) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= w) return;
    const double g = eps / s[j];
    double acc = 0.0;
    for (int64_t i = lane; i < d; i += 32) {
        const double wi = g * Q[i * w + j];
        W1[(int64_t)j * d + i] = (float)wi;
        acc = fma(wi, mu[i], acc);
    }
    acc = warp_sum_d(acc);
    if (lane == 0) b1[j] = (float)(-acc);
}

// Ha[r] = [tanh(tanh(tanh(eps T[r][c] / s[c]))), 1]: the third hidden layer (layers 2 and 3
// start as the identity with zero bias) with a trailing column of ones.
__global__ void k_hidden_ones(const double* __restrict__ T, const double* __restrict__ s, double eps, int64_t rows, int w,
                              double* __restrict__ Ha) {
    const int64_t total = rows * (w + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / (w + 1);
        const int c = (int)(e - r * (w + 1));
        Ha[e] = c == w ? 1.0 : tanh(tanh(tanh(eps * T[r * w + c] / s[c])));
    }
}

// A += ridge * trace(A)/m * I  (single block)
__global__ void k_ridge(double* A, int m, double ridge) {
    double t = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) t += A[(int64_t)i * m + i];
    t = block_sum_d(t);
    __shared__ double lam;
    if (threadIdx.x == 0) lam = ridge * t / m;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) A[(int64_t)i * m + i] += lam;
}

// In-place Cholesky A = L L^T of an m x m SPD matrix (lower triangle), one block.  bad[0] = 1
// if a pivot is not positive (the factor is then meaningless).
__global__ void k_chol(double* A, int m, int* bad) {
    __shared__ double piv;
    for (int k = 0; k < m; ++k) {
        if (threadIdx.x == 0) {
            double a = A[(int64_t)k * m + k];
            if (!(a > 0.0)) {
                bad[0] = 1;
                a = 1.0;
            }
            piv = sqrt(a);
            A[(int64_t)k * m + k] = piv;
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[(int64_t)i * m + k] /= piv;
        __syncthreads();
        const int len = m - k - 1;
        for (int64_t e = threadIdx.x; e < (int64_t)len * len; e += blockDim.x) {
            const int i = k + 1 + (int)(e / len), j = k + 1 + (int)(e % len);
            if (j <= i) A[(int64_t)i * m + j] -= A[(int64_t)i * m + k] * A[(int64_t)j * m + k];
        }
        __syncthreads();
    }
}

// X = L^{-1} (lower triangular, zeros above the diagonal), a thread per column, one block.
__global__ void k_trinv_lower(const double* __restrict__ L, int m, double* X) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        for (int i = 0; i < j; ++i) X[(int64_t)i * m + j] = 0.0;
        for (int i = j; i < m; ++i) {
            double s = i == j ? 1.0 : 0.0;
            for (int k = j; k < i; ++k) s -= L[(int64_t)i * m + k] * X[(int64_t)k * m + j];
            X[(int64_t)i * m + j] = s / L[(int64_t)i * m + i];
        }
    }
}

// Readout: W4[i][j] = Z[j][i] (j < w), b4[i] = Z[w][i]; Z is (w+1) x d.
__global__ void k_readout(const double* __restrict__ Z, int64_t d, int w, float* __restrict__ W4, float* __restrict__ b4) {
    const int64_t total = d * (w + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / (w + 1);
        const int j = (int)(e - i * (w + 1));
        const double v = Z[(int64_t)j * d + i];
        if (j < w)
            W4[i * w + j] = (float)v;
        else
            b4[i] = (float)v;
    }
}

__global__ void k_identity_layers(float* W2, float* b2, float* W3, float* b3, int w) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w * w; e += gridDim.x * blockDim.x) {
        const float v = (e / w == e % w) ? 1.f : 0.f;
        W2[e] = v;
        W3[e] = v;
        if (e < w) {
            b2[e] = 0.f;
            b3[e] = 0.f;
        }
    }
}

int ew_grid(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 8); }

mh_status check_net(mh_ctx* ctx, const mh_net* net) {
    if (!net) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null network");
    return MH_OK;
}

mh_status ensure_rows(mh_ctx* ctx, mh_net* net, int64_t rows) {
    if (rows <= net->cap_rows) return MH_OK;
    MH_ALLOC(ctx, net->xb, rows * net->d);
    MH_ALLOC(ctx, net->yb, rows * net->d);
    MH_ALLOC(ctx, net->yh, rows * net->d);
    MH_ALLOC(ctx, net->dzd, rows * net->d);
    for (int i = 0; i < 3; ++i) MH_ALLOC(ctx, net->act[i], rows * net->w);
    MH_ALLOC(ctx, net->dzw1, rows * net->w);
    MH_ALLOC(ctx, net->dzw2, rows * net->w);
    net->cap_rows = rows;
    return MH_OK;
}

// Training-kernel forward of `rows` inputs in net->xb; output in net->yh.
mh_status train_forward(mh_ctx* ctx, mh_net* net, int64_t rows) {
    cudaStream_t st = ctx->stream;
    const float* P = net->P.p;
    const int w = net->w;
    const int64_t d = net->d;
    const float* in = net->xb.p;
    int64_t ld_in = d;
    for (int l = 0; l < 3; ++l) {
        gemm<float, EPI_BIAS_TANH>(st, (int)rows, w, net->lin[l], in, ld_in, 1, P + net->oW[l], 1, net->lin[l],
                                   net->act[l].p, w, P + net->ob[l]);
        MH_LAUNCHED(ctx);
        in = net->act[l].p;
        ld_in = w;
    }
    gemm<float, EPI_BIAS>(st, (int)rows, (int)d, w, in, w, 1, P + net->oW[3], 1, w, net->yh.p, d, P + net->ob[3]);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

// Loss of net->yh against net->yb over rows x d; dz (nullable) receives dL/dyh.  Result on device in out.
mh_status train_loss(mh_ctx* ctx, mh_net* net, int64_t rows, float* dz, double* out) {
    const int64_t n = rows * net->d;
    const int nb = ew_grid(n);
    if ((int64_t)net->lpart.n < nb) MH_ALLOC(ctx, net->lpart, 152 * 8);
    k_loss_dz<<<nb, 256, 0, ctx->stream>>>(net->yh.p, net->yb.p, n, (float)(1.0 / (double)n), dz, net->lpart.p);
    MH_LAUNCHED(ctx);
    k_sum_parts<<<1, 1024, 0, ctx->stream>>>(net->lpart.p, nb, 0.5 / (double)n, out);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

// Backward pass from dz = dL/dyh (net->dzd) into the gradient buffer g.
mh_status train_backward(mh_ctx* ctx, mh_net* net, int64_t rows, float* g) {
    cudaStream_t st = ctx->stream;
    const float* P = net->P.p;
    const int w = net->w;
    const int64_t d = net->d;
    const int R = (int)rows;
    // layer 4
    gemm<float, EPI_NONE>(st, (int)d, w, R, net->dzd.p, 1, d, net->act[2].p, w, 1, g + net->oW[3], w);
    MH_LAUNCHED(ctx);
    k_colsum<<<mh_grid(d, 256), 256, 0, st>>>(net->dzd.p, rows, d, g + net->ob[3]);
    MH_LAUNCHED(ctx);
    gemm<float, EPI_TANH_BACK>(st, R, w, (int)d, net->dzd.p, d, 1, P + net->oW[3], w, 1, net->dzw1.p, w, nullptr,
                               net->act[2].p);
    MH_LAUNCHED(ctx);
    float* dz = net->dzw1.p;
    float* dn = net->dzw2.p;
    for (int l = 2; l >= 0; --l) {
        const float* a_in = l > 0 ? net->act[l - 1].p : net->xb.p;
        const int64_t ld_in = l > 0 ? w : d;
        gemm<float, EPI_NONE>(st, w, net->lin[l], R, dz, 1, w, a_in, ld_in, 1, g + net->oW[l], net->lin[l]);
        MH_LAUNCHED(ctx);
        k_colsum<<<mh_grid(w, 256), 256, 0, st>>>(dz, rows, w, g + net->ob[l]);
        MH_LAUNCHED(ctx);
        if (l > 0) {
            gemm<float, EPI_TANH_BACK>(st, R, w, w, dz, w, 1, P + net->oW[l], w, 1, dn, w, nullptr,
                                       net->act[l - 1].p);
            MH_LAUNCHED(ctx);
            std::swap(dz, dn);
        }
    }
    return MH_OK;
}

mh_status ensure_bf16(mh_ctx* ctx, mh_net* net) {
    if (net->bf_ready) return MH_OK;
    if (!net->Bhi.p) {
        MH_ALLOC(ctx, net->Bhi, net->n_params);
        MH_ALLOC(ctx, net->Blo, net->n_params);
    }
    k_to_bf16<<<ew_grid(net->n_params), 256, 0, ctx->stream>>>(net->P.p, net->n_params, net->Bhi.p, net->Blo.p);
    MH_LAUNCHED(ctx);
    net->bf_ready = true;
    return MH_OK;
}

template <int ARITH>
void launch_gemv(cudaStream_t st, const mh_net* net, int l, const float* in, float* out) {
    const int rows = net->lout[l], cols = net->lin[l];
    const size_t smem = (size_t)cols * sizeof(float);
    const int act = l < 3;
    const float* W32 = net->P.p + net->oW[l];
    const uint16_t* hi = net->Bhi.p ? net->Bhi.p + net->oW[l] : nullptr;
    const uint16_t* lo = net->Blo.p ? net->Blo.p + net->oW[l] : nullptr;
    const float* b = net->P.p + net->ob[l];
    if (cols >= 1024)   // long rows: four warps per row
        k_gemv_layer<ARITH, 4><<<(rows + 1) / 2, 256, smem, st>>>(W32, hi, lo, b, in, cols, rows, act, out);
    else
        k_gemv_layer<ARITH, 1><<<(rows + 7) / 8, 256, smem, st>>>(W32, hi, lo, b, in, cols, rows, act, out);
}

// Inference of one feature vector x (d floats) into y (d floats).
mh_status infer_one(mh_ctx* ctx, mh_net* net, int arith, const float* x, float* y) {
    if (arith != MH_NET_FP32) MH_TRY(ensure_bf16(ctx, net));
    cudaStream_t st = ctx->stream;
    const float* in = x;
    float* bufs[2] = {net->hA.p, net->hB.p};
    for (int l = 0; l < 4; ++l) {
        float* out = l == 3 ? y : bufs[l & 1];
        if (arith == MH_NET_FP32)
            launch_gemv<MH_NET_FP32>(st, net, l, in, out);
        else if (arith == MH_NET_BF16)
            launch_gemv<MH_NET_BF16>(st, net, l, in, out);
        else
            launch_gemv<MH_NET_BF16X2>(st, net, l, in, out);
        MH_LAUNCHED(ctx);
        in = out;
    }
    return MH_OK;
}

mh_status features(mh_ctx* ctx, mh_net* net, const double* v, const double* scale, float* x) {
    const int warps = net->n_curves * net->K;
    k_to_f32<<<mh_grid(net->n_bnd, 256), 256, 0, ctx->stream>>>(v, net->n_bnd, net->v32.p);
    MH_LAUNCHED(ctx);
    k_features<<<(warps + 7) / 8, 256, 0, ctx->stream>>>(net->v32.p, net->tw32.p, net->d_nn.p, net->d_off.p,
                                                         net->n_curves, net->K, scale, x);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

bool same_boundary(const mh_net* net, const mh_boundary* b) {
    if (net->n_curves != b->n_curves || net->n_bnd != b->n) return false;
    for (int c = 0; c < b->n_curves; ++c)
        if (net->nn[c] != b->n_nodes[c]) return false;
    return true;
}

}  // namespace

// ------------------------------------------------------------------------------------------ API
extern "C" mh_status mh_net_create(mh_ctx* ctx, const mh_boundary* bnd, int n_modes, int width, mh_net** out) {
    if (!ctx || !bnd || !out) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n_modes < 4 || n_modes % 4) return mh_fail(ctx, MH_ERR_INVALID_ARG, "n_modes must be a positive multiple of 4");
    if (width < 8 || width > 1024 || width % 8)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "width must be a multiple of 8 in 8..1024");
    for (int c = 0; c < bnd->n_curves; ++c)
        if (2 * n_modes > bnd->n_nodes[c])
            return mh_fail(ctx, MH_ERR_INVALID_ARG, "n_modes %d exceeds half the %d nodes of curve %d", n_modes,
                           bnd->n_nodes[c], c);
    const int64_t d = (int64_t)bnd->n_curves * 2 * n_modes;
    if (d > 49152) return mh_fail(ctx, MH_ERR_INVALID_ARG, "too many features (%lld > 49152)", (long long)d);
    std::unique_ptr<mh_net> net(new mh_net());
    net->n_curves = bnd->n_curves;
    net->K = n_modes;
    net->w = width;
    net->d = d;
    net->n_bnd = bnd->n;
    net->nn = bnd->n_nodes;
    net->off = bnd->offset;
    net->max_nodes = *std::max_element(bnd->n_nodes.begin(), bnd->n_nodes.end());
    const int w = width;
    int64_t o = 0;
    const int lin[4] = {(int)d, w, w, w}, lout[4] = {w, w, w, (int)d};
    for (int l = 0; l < 4; ++l) {
        net->lin[l] = lin[l];
        net->lout[l] = lout[l];
        net->oW[l] = o;
        o += (int64_t)lin[l] * lout[l];
        net->ob[l] = o;
        o += lout[l];
    }
    net->n_params = o;
    cudaStream_t st = ctx->stream;
    MH_ALLOC(ctx, net->d_nn, bnd->n_curves);
    MH_ALLOC(ctx, net->d_off, bnd->n_curves);
    MH_CUDA(ctx, cudaMemcpyAsync(net->d_nn.p, bnd->n_nodes.data(), bnd->n_curves * 4, cudaMemcpyHostToDevice, st));
    MH_CUDA(ctx, cudaMemcpyAsync(net->d_off.p, bnd->offset.data(), bnd->n_curves * 4, cudaMemcpyHostToDevice, st));
    MH_ALLOC(ctx, net->tw, 2 * bnd->n);
    k_twiddle<<<dim3((unsigned)mh_grid(net->max_nodes, 256), (unsigned)bnd->n_curves), 256, 0, st>>>(
        net->d_nn.p, net->d_off.p, net->tw.p);
    MH_LAUNCHED(ctx);
    MH_ALLOC(ctx, net->tw32, bnd->n);
    MH_ALLOC(ctx, net->v32, bnd->n);
    k_tw_f32<<<mh_grid(bnd->n, 256), 256, 0, st>>>(net->tw.p, bnd->n, net->tw32.p);
    MH_LAUNCHED(ctx);
    MH_ALLOC(ctx, net->P, net->n_params);
    MH_CUDA(ctx, cudaMemsetAsync(net->P.p, 0, net->n_params * 4, st));
    MH_ALLOC(ctx, net->xin, d);
    MH_ALLOC(ctx, net->yout, d);
    MH_ALLOC(ctx, net->hA, w);
    MH_ALLOC(ctx, net->hB, w);
    MH_ALLOC(ctx, net->rbuf, bnd->n);
    MH_ALLOC(ctx, net->ebuf, bnd->n);
    MH_ALLOC(ctx, net->scal, 8);
    const int smem = (int)(std::max<int64_t>(d, w) * 4);
    if (smem > 48 * 1024) {
#define MH_GEMV_ATTR(A, S)                                                                         \
    MH_CUDA(ctx, cudaFuncSetAttribute(k_gemv_layer<A, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))
        MH_GEMV_ATTR(MH_NET_FP32, 1);
        MH_GEMV_ATTR(MH_NET_FP32, 4);
        MH_GEMV_ATTR(MH_NET_BF16, 1);
        MH_GEMV_ATTR(MH_NET_BF16, 4);
        MH_GEMV_ATTR(MH_NET_BF16X2, 1);
        MH_GEMV_ATTR(MH_NET_BF16X2, 4);
#undef MH_GEMV_ATTR
    }
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    *out = net.release();
    return MH_OK;
}

extern "C" mh_status mh_net_destroy(mh_net* net) {
    delete net;
    return MH_OK;
}

extern "C" mh_status mh_net_dims(const mh_net* net, int64_t* d, int64_t* width, int64_t* n_params) {
    if (!net) return MH_ERR_INVALID_ARG;
    if (d) *d = net->d;
    if (width) *width = net->w;
    if (n_params) *n_params = net->n_params;
    return MH_OK;
}

extern "C" mh_status mh_net_get_params(mh_ctx* ctx, const mh_net* net, float* params_host, double* gx_host,
                                       double* gy_host) {
    if (!ctx) return MH_ERR_INVALID_ARG;
    MH_TRY(check_net(ctx, net));
    if (params_host) {
        MH_CUDA(ctx, cudaMemcpyAsync(params_host, net->P.p, net->n_params * 4, cudaMemcpyDeviceToHost, ctx->stream));
        MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (gx_host) *gx_host = net->gx;
    if (gy_host) *gy_host = net->gy;
    return MH_OK;
}

extern "C" mh_status mh_net_set_params(mh_ctx* ctx, mh_net* net, const float* params_host, double gx, double gy) {
    if (!ctx) return MH_ERR_INVALID_ARG;
    MH_TRY(check_net(ctx, net));
    if (!(gx > 0) || !(gy > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "scales must be positive");
    if (params_host) {
        MH_CUDA(ctx, cudaMemcpyAsync(net->P.p, params_host, net->n_params * 4, cudaMemcpyHostToDevice, ctx->stream));
        MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    net->gx = gx;
    net->gy = gy;
    net->bf_ready = false;
    return MH_OK;
}

extern "C" mh_status mh_net_sample(mh_ctx* ctx, mh_problem* prob, mh_net* net, const double* sigma_prev_dev,
                                   const double* sigma_next_dev, float* x_dev, float* y_dev, double* r_norm_host) {
    if (!ctx || !prob || !sigma_prev_dev || !sigma_next_dev || !x_dev || !y_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_TRY(check_net(ctx, net));
    mh_boundary* b = prob->bnd;
    if (!same_boundary(net, b)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "network built for another boundary");
    cudaStream_t st = ctx->stream;
    const int64_t n = b->n;
    MH_TRY(bie_assemble(ctx, b, prob->alpha));
    MH_TRY(bie_apply(ctx, b, sigma_prev_dev, net->rbuf.p, MH_PREC_FP64));
    k_resid<<<mh_grid(n, 256), 256, 0, st>>>(prob->rhs.p, net->rbuf.p, n);
    MH_LAUNCHED(ctx);
    k_norm_scale<<<1, 1024, 0, st>>>(net->rbuf.p, n, 1.0, net->scal.p);
    MH_LAUNCHED(ctx);
    MH_TRY(features(ctx, net, net->rbuf.p, net->scal.p + 1, x_dev));
    k_sub3<<<mh_grid(n, 256), 256, 0, st>>>(sigma_next_dev, sigma_prev_dev, net->rbuf.p, n, net->ebuf.p);
    MH_LAUNCHED(ctx);
    MH_TRY(features(ctx, net, net->ebuf.p, net->scal.p + 1, y_dev));
    if (r_norm_host) {
        MH_CUDA(ctx, cudaMemcpyAsync(r_norm_host, net->scal.p, 8, cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
    }
    return MH_OK;
}

extern "C" mh_status mh_net_fit(mh_ctx* ctx, mh_net* net, const float* X_dev, const float* Y_dev, int64_t n,
                                const float* omega_dev, double eps, int power_iters, double ridge) {
    if (!ctx || !X_dev || !Y_dev || !omega_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_TRY(check_net(ctx, net));
    if (n < 2) return mh_fail(ctx, MH_ERR_INVALID_ARG, "need at least 2 training pairs");
    if (!(eps > 0) || power_iters < 0 || power_iters > 20 || !(ridge >= 0))
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad eps / power_iters / ridge");
    cudaStream_t st = ctx->stream;
    const int64_t d = net->d;
    const int w = net->w, m = w + 1;
    // g_x, g_y: RMS entries
    dbuf<double> part, sums;
    MH_ALLOC(ctx, part, 152 * 8);
    MH_ALLOC(ctx, sums, 2);
    const int nb = ew_grid(n * d);
    k_sumsq_f<<<nb, 256, 0, st>>>(X_dev, n * d, part.p);
    MH_LAUNCHED(ctx);
    k_sum_parts<<<1, 1024, 0, st>>>(part.p, nb, 1.0 / (double)(n * d), sums.p);
    MH_LAUNCHED(ctx);
    k_sumsq_f<<<nb, 256, 0, st>>>(Y_dev, n * d, part.p);
    MH_LAUNCHED(ctx);
    k_sum_parts<<<1, 1024, 0, st>>>(part.p, nb, 1.0 / (double)(n * d), sums.p + 1);
    MH_LAUNCHED(ctx);
    double ms[2];
    MH_CUDA(ctx, cudaMemcpyAsync(ms, sums.p, 16, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    if (!(ms[0] > 0) || !(ms[1] > 0) || !std::isfinite(ms[0]) || !std::isfinite(ms[1]))
        return mh_fail(ctx, MH_ERR_NUMERIC, "training features or targets are all zero or not finite");
    const double gx = std::sqrt(ms[0]), gy = std::sqrt(ms[1]);
    dbuf<double> Xs, Ys, mu, Om, Q, Q2, T, Gm, Li, s, Ha, Rh, Z1;
    dbuf<int> bad;
    MH_ALLOC(ctx, Xs, n * d);
    MH_ALLOC(ctx, Ys, n * d);
    MH_ALLOC(ctx, mu, d);
    MH_ALLOC(ctx, Om, n * w);
    MH_ALLOC(ctx, Q, d * w);
    MH_ALLOC(ctx, Q2, d * w);
    MH_ALLOC(ctx, T, n * w);
    MH_ALLOC(ctx, Gm, (int64_t)m * m);
    MH_ALLOC(ctx, Li, (int64_t)m * m);
    MH_ALLOC(ctx, s, w);
    MH_ALLOC(ctx, bad, 1);
    MH_CUDA(ctx, cudaMemsetAsync(bad.p, 0, 4, st));
    k_f2d<<<ew_grid(n * d), 256, 0, st>>>(X_dev, n * d, 1.0 / gx, Xs.p);
    MH_LAUNCHED(ctx);
    k_f2d<<<ew_grid(n * d), 256, 0, st>>>(Y_dev, n * d, 1.0 / gy, Ys.p);
    MH_LAUNCHED(ctx);
    k_f2d<<<ew_grid(n * w), 256, 0, st>>>(omega_dev, n * w, 1.0, Om.p);
    MH_LAUNCHED(ctx);
    k_center<<<mh_grid(d, 128), 128, 0, st>>>(Xs.p, n, d, mu.p);
    MH_LAUNCHED(ctx);
    const int N = (int)n, D = (int)d;
    // CholeskyQR2 of a rows x w matrix M in place (tmp: same size): M <- M L^{-T}, twice
    // (M^T M = L L^T); the result is the Q factor whose R has a positive diagonal.
    dbuf<double> T2;
    MH_ALLOC(ctx, T2, n * w);
    auto orth = [&](double*& M, double*& tmp, int rows) -> mh_status {
        for (int pass = 0; pass < 2; ++pass) {
            gemm<double, EPI_NONE>(st, w, w, rows, M, 1, w, M, w, 1, Gm.p, w);
            MH_LAUNCHED(ctx);
            k_chol<<<1, 1024, 0, st>>>(Gm.p, w, bad.p);
            MH_LAUNCHED(ctx);
            k_trinv_lower<<<1, 256, 0, st>>>(Gm.p, w, Li.p);
            MH_LAUNCHED(ctx);
            gemm<double, EPI_NONE>(st, rows, w, w, M, w, 1, Li.p, 1, w, tmp, w);
            MH_LAUNCHED(ctx);
            std::swap(M, tmp);
        }
        return MH_OK;
    };
    // range finder: Q = orth(Xc^T Omega), then power iterations Q = orth(Xc^T (Xc Q)).  The
    // product Xc Q is orthonormalised too: orth(Xc^T Xc Q R^{-1}) = orth(Xc^T Xc Q) for any
    // upper-triangular R with positive diagonal, and each factorisation then sees the
    // condition number of one product only.
    gemm<double, EPI_NONE>(st, D, w, N, Xs.p, 1, d, Om.p, w, 1, Q.p, w);
    MH_LAUNCHED(ctx);
    MH_TRY(orth(Q.p, Q2.p, D));
    for (int it = 0; it < power_iters; ++it) {
        gemm<double, EPI_NONE>(st, N, w, D, Xs.p, d, 1, Q.p, w, 1, T.p, w);
        MH_LAUNCHED(ctx);
        MH_TRY(orth(T.p, T2.p, N));
        gemm<double, EPI_NONE>(st, D, w, N, Xs.p, 1, d, T.p, w, 1, Q.p, w);
        MH_LAUNCHED(ctx);
        MH_TRY(orth(Q.p, Q2.p, D));
    }
    // first layer: W1 = eps diag(1/s) Q^T, b1 = -W1 mu
    gemm<double, EPI_NONE>(st, N, w, D, Xs.p, d, 1, Q.p, w, 1, T.p, w);
    MH_LAUNCHED(ctx);
    k_colrms_floor<<<1, 256, 0, st>>>(T.p, n, w, s.p);
    MH_LAUNCHED(ctx);
    float* P = net->P.p;
    k_first_layer<<<(w + 7) / 8, 256, 0, st>>>(Q.p, s.p, mu.p, d, w, eps, P + net->oW[0], P + net->ob[0]);
    MH_LAUNCHED(ctx);
    k_identity_layers<<<mh_grid((int64_t)w * w, 256), 256, 0, st>>>(P + net->oW[1], P + net->ob[1], P + net->oW[2],
                                                                    P + net->ob[2], w);
    MH_LAUNCHED(ctx);
    // third hidden layer on the training inputs: the first pre-activation is
    // W1 x + b1 = W1 (x - mu) = (eps / s_j) (Xc Q)_j, and layers 2, 3 are tanh of the identity
    Q2.release();
    T2.release();
    MH_ALLOC(ctx, Ha, n * m);
    k_hidden_ones<<<ew_grid(n * m), 256, 0, st>>>(T.p, s.p, eps, n, w, Ha.p);
    MH_LAUNCHED(ctx);
    // ridge normal equations (Ha^T Ha + lam I) Z = Ha^T Y by Cholesky: Z = L^{-T} L^{-1} Ha^T Y
    MH_ALLOC(ctx, Gm, (int64_t)m * m);
    MH_ALLOC(ctx, Li, (int64_t)m * m);
    MH_ALLOC(ctx, Rh, (int64_t)m * d);
    MH_ALLOC(ctx, Z1, (int64_t)m * d);
    gemm<double, EPI_NONE>(st, m, m, N, Ha.p, 1, m, Ha.p, m, 1, Gm.p, m);
    MH_LAUNCHED(ctx);
    gemm<double, EPI_NONE>(st, m, D, N, Ha.p, 1, m, Ys.p, d, 1, Rh.p, d);
    MH_LAUNCHED(ctx);
    k_ridge<<<1, 1024, 0, st>>>(Gm.p, m, ridge);
    MH_LAUNCHED(ctx);
    k_chol<<<1, 1024, 0, st>>>(Gm.p, m, bad.p);
    MH_LAUNCHED(ctx);
    k_trinv_lower<<<1, 256, 0, st>>>(Gm.p, m, Li.p);
    MH_LAUNCHED(ctx);
    gemm<double, EPI_NONE>(st, m, D, m, Li.p, m, 1, Rh.p, d, 1, Z1.p, d);
    MH_LAUNCHED(ctx);
    gemm<double, EPI_NONE>(st, m, D, m, Li.p, 1, m, Z1.p, d, 1, Rh.p, d);
    MH_LAUNCHED(ctx);
    k_readout<<<ew_grid(d * m), 256, 0, st>>>(Rh.p, d, w, P + net->oW[3], P + net->ob[3]);
    MH_LAUNCHED(ctx);
    int hb = 0;
    MH_CUDA(ctx, cudaMemcpyAsync(&hb, bad.p, 4, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    if (hb) return mh_fail(ctx, MH_ERR_NUMERIC, "singular Gram matrix in the closed-form start (rank-deficient data)");
    net->gx = gx;
    net->gy = gy;
    net->bf_ready = false;
    return MH_OK;
}

extern "C" mh_status mh_net_loss_grad(mh_ctx* ctx, mh_net* net, const float* X_dev, const float* T_dev, int64_t n,
                                      double* loss_host, float* grad_dev) {
    if (!ctx || !X_dev || !T_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_TRY(check_net(ctx, net));
    if (n < 1) return mh_fail(ctx, MH_ERR_INVALID_ARG, "n must be positive");
    cudaStream_t st = ctx->stream;
    MH_TRY(ensure_rows(ctx, net, n));
    MH_CUDA(ctx, cudaMemcpyAsync(net->xb.p, X_dev, n * net->d * 4, cudaMemcpyDeviceToDevice, st));
    MH_CUDA(ctx, cudaMemcpyAsync(net->yb.p, T_dev, n * net->d * 4, cudaMemcpyDeviceToDevice, st));
    MH_TRY(train_forward(ctx, net, n));
    MH_TRY(train_loss(ctx, net, n, net->dzd.p, net->scal.p + 4));
    if (grad_dev) MH_TRY(train_backward(ctx, net, n, grad_dev));
    if (loss_host) {
        MH_CUDA(ctx, cudaMemcpyAsync(loss_host, net->scal.p + 4, 8, cudaMemcpyDeviceToHost, st));
    }
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    return MH_OK;
}

extern "C" mh_status mh_net_forward(mh_ctx* ctx, mh_net* net, const float* X_dev, int64_t n, float* Y_dev,
                                    mh_net_arith arith, int training_kernels) {
    if (!ctx || !X_dev || !Y_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_TRY(check_net(ctx, net));
    if (n < 1) return mh_fail(ctx, MH_ERR_INVALID_ARG, "n must be positive");
    if (arith < MH_NET_FP32 || arith > MH_NET_BF16X2) return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad arith");
    cudaStream_t st = ctx->stream;
    const int64_t d = net->d;
    if (training_kernels) {
        MH_TRY(ensure_rows(ctx, net, n));
        MH_CUDA(ctx, cudaMemcpyAsync(net->xb.p, X_dev, n * d * 4, cudaMemcpyDeviceToDevice, st));
        MH_TRY(train_forward(ctx, net, n));
        MH_CUDA(ctx, cudaMemcpyAsync(Y_dev, net->yh.p, n * d * 4, cudaMemcpyDeviceToDevice, st));
    } else {
        for (int64_t r = 0; r < n; ++r) MH_TRY(infer_one(ctx, net, arith, X_dev + r * d, Y_dev + r * d));
    }
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    return MH_OK;
}

extern "C" mh_status mh_net_train(mh_ctx* ctx, mh_net* net, const float* X_dev, const float* Y_dev, int64_t n,
                                  const int32_t* batch_idx_dev, int steps, int batch, double lr, const float* Xv_dev,
                                  const float* Yv_dev, int64_t n_val, int eval_every, double* first_val_host,
                                  double* best_val_host, int* best_step_host) {
    if (!ctx || !X_dev || !Y_dev || !batch_idx_dev || !Xv_dev || !Yv_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_TRY(check_net(ctx, net));
    if (n < 1 || steps < 0 || batch < 1 || n_val < 1 || eval_every < 1 || !(lr > 0))
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad training sizes or learning rate");
    cudaStream_t st = ctx->stream;
    const int64_t d = net->d, np = net->n_params;
    MH_TRY(ensure_rows(ctx, net, std::max<int64_t>(batch, n_val)));
    if (!net->G.p) {
        MH_ALLOC(ctx, net->G, np);
        MH_ALLOC(ctx, net->Mo, np);
        MH_ALLOC(ctx, net->Vo, np);
        MH_ALLOC(ctx, net->best, np);
    }
    MH_CUDA(ctx, cudaMemsetAsync(net->Mo.p, 0, np * 4, st));
    MH_CUDA(ctx, cudaMemsetAsync(net->Vo.p, 0, np * 4, st));
    const float sx = (float)(1.0 / net->gx), sy = (float)(1.0 / net->gy);
    auto val_loss = [&](double* out) -> mh_status {
        k_gather_rows<<<ew_grid(n_val * d), 256, 0, st>>>(Xv_dev, nullptr, n_val, d, sx, net->xb.p);
        MH_LAUNCHED(ctx);
        k_gather_rows<<<ew_grid(n_val * d), 256, 0, st>>>(Yv_dev, nullptr, n_val, d, sy, net->yb.p);
        MH_LAUNCHED(ctx);
        MH_TRY(train_forward(ctx, net, n_val));
        MH_TRY(train_loss(ctx, net, n_val, nullptr, net->scal.p + 5));
        MH_CUDA(ctx, cudaMemcpyAsync(out, net->scal.p + 5, 8, cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
        return MH_OK;
    };
    double first = 0.0;
    MH_TRY(val_loss(&first));
    if (!std::isfinite(first)) return mh_fail(ctx, MH_ERR_NUMERIC, "validation loss is not finite");
    double best = first;
    int best_step = 0;
    MH_CUDA(ctx, cudaMemcpyAsync(net->best.p, net->P.p, np * 4, cudaMemcpyDeviceToDevice, st));
    const float b1 = 0.9f, b2 = 0.999f;
    for (int t = 1; t <= steps; ++t) {
        const int32_t* idx = batch_idx_dev + (int64_t)(t - 1) * batch;
        k_gather_rows<<<ew_grid((int64_t)batch * d), 256, 0, st>>>(X_dev, idx, batch, d, sx, net->xb.p);
        MH_LAUNCHED(ctx);
        k_gather_rows<<<ew_grid((int64_t)batch * d), 256, 0, st>>>(Y_dev, idx, batch, d, sy, net->yb.p);
        MH_LAUNCHED(ctx);
        MH_TRY(train_forward(ctx, net, batch));
        MH_TRY(train_loss(ctx, net, batch, net->dzd.p, net->scal.p + 4));
        MH_TRY(train_backward(ctx, net, batch, net->G.p));
        const float bc1 = (float)(1.0 - std::pow(0.9, t)), bc2 = (float)(1.0 - std::pow(0.999, t));
        k_adam<<<ew_grid(np), 256, 0, st>>>(net->P.p, net->G.p, net->Mo.p, net->Vo.p, np, (float)lr, b1, b2, 1e-8f,
                                            bc1, bc2);
        MH_LAUNCHED(ctx);
        if (t % eval_every == 0 || t == steps) {
            double v = 0.0;
            MH_TRY(val_loss(&v));
            if (std::isfinite(v) && v < best) {
                best = v;
                best_step = t;
                MH_CUDA(ctx, cudaMemcpyAsync(net->best.p, net->P.p, np * 4, cudaMemcpyDeviceToDevice, st));
            }
        }
    }
    MH_CUDA(ctx, cudaMemcpyAsync(net->P.p, net->best.p, np * 4, cudaMemcpyDeviceToDevice, st));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    net->bf_ready = false;
    if (first_val_host) *first_val_host = first;
    if (best_val_host) *best_val_host = best;
    if (best_step_host) *best_step_host = best_step;
    return MH_OK;
}

mh_status warm_start_prepare(mh_ctx* ctx, mh_boundary* b) {
    if (b->warm_dir.p) return MH_OK;
    MH_ALLOC(ctx, b->warm_dir, b->n);
    MH_ALLOC(ctx, b->warm_w, b->n);
    MH_ALLOC(ctx, b->warm_scal, 8);
    return MH_OK;
}

// Shared by mh_warm_start and the time step.  r0 first holds r = rhs - A sigma (binary64).
mh_status warm_start_run(mh_ctx* ctx, mh_boundary* b, double alpha, mh_net* net, int mode, int arith,
                         const double* sigma, const double* sigma_prev2, const double* rhs, double* x0, double* r0,
                         mh_precision prec, double* c_dev, double* save, bool r_ready) {
    cudaStream_t st = ctx->stream;
    const int64_t n = b->n;
    MH_TRY(bie_assemble(ctx, b, alpha));
    if (mode == MH_WARM_ZERO) {
        MH_CUDA(ctx, cudaMemsetAsync(x0, 0, n * 8, st));
        MH_CUDA(ctx, cudaMemcpyAsync(r0, rhs, n * 8, cudaMemcpyDeviceToDevice, st));
        if (c_dev) MH_CUDA(ctx, cudaMemsetAsync(c_dev, 0, 8, st));
        return MH_OK;
    }
    prof_scope ps(ctx, "warm_start");
    if (!r_ready) {
        MH_TRY(bie_apply_resid(ctx, b, sigma, r0, prec));
        k_resid<<<mh_grid(n, 256), 256, 0, st>>>(rhs, r0, n);
        MH_LAUNCHED(ctx);
    }
    if (mode == MH_WARM_PREVIOUS) {
        if (x0 != sigma) MH_CUDA(ctx, cudaMemcpyAsync(x0, sigma, n * 8, cudaMemcpyDeviceToDevice, st));
        if (c_dev) MH_CUDA(ctx, cudaMemsetAsync(c_dev, 0, 8, st));
        return MH_OK;
    }
    MH_TRY(warm_start_prepare(ctx, b));
    double* scal = b->warm_scal.p;
    if (mode == MH_WARM_SECANT) {
        k_axmy<<<mh_grid(n, 256), 256, 0, st>>>(sigma, sigma_prev2, n, b->warm_dir.p);
        MH_LAUNCHED(ctx);
    } else {
        prof_scope pn(ctx, "warm_net");
        k_norm_scale<<<1, 1024, 0, st>>>(r0, n, net->gx, scal);
        MH_LAUNCHED(ctx);
        MH_TRY(features(ctx, net, r0, scal + 1, net->xin.p));
        MH_TRY(infer_one(ctx, net, arith, net->xin.p, net->yout.p));
        k_synth<<<dim3((unsigned)mh_grid(net->max_nodes, 32), (unsigned)net->n_curves), 256, 2 * net->K * 4, st>>>(
            net->yout.p, net->tw32.p, net->d_nn.p, net->d_off.p, net->K, r0, scal, net->gy, b->warm_dir.p);
        MH_LAUNCHED(ctx);
    }
    // binary64 image of the direction: r0 = r - c w is handed to GMRES as the residual of x0, and
    // a binary32 operator would leave an error of ~1e-7 |A| |c delta| in it (above the tolerance)
    (void)prec;
    MH_TRY(bie_apply_resid(ctx, b, b->warm_dir.p, b->warm_w.p, prec));
    k_dot2<<<1, 1024, 0, st>>>(r0, b->warm_w.p, n, scal);
    MH_LAUNCHED(ctx);
    k_line<<<mh_grid(n, 256), 256, 0, st>>>(sigma, b->warm_dir.p, r0, b->warm_w.p, scal, n, x0, r0, save, c_dev);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

extern "C" mh_status mh_warm_start(mh_ctx* ctx, mh_boundary* bnd, double alpha, mh_net* net, mh_warm_mode mode,
                                   mh_net_arith arith, const double* sigma_dev, const double* sigma_prev2_dev,
                                   const double* rhs_dev, double* x0_dev, double* r0_dev, mh_precision prec,
                                   double* c_host) {
    if (!ctx || !bnd || !sigma_dev || !rhs_dev || !x0_dev || !r0_dev)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (mode < MH_WARM_PREVIOUS || mode > MH_WARM_LEARNED) return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad mode");
    if (arith < MH_NET_FP32 || arith > MH_NET_BF16X2) return mh_fail(ctx, MH_ERR_INVALID_ARG, "bad arith");
    if (!(alpha > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "alpha must be positive");
    if (mode == MH_WARM_SECANT && !sigma_prev2_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "SECANT needs sigma_prev2");
    if (mode == MH_WARM_LEARNED) {
        MH_TRY(check_net(ctx, net));
        if (!same_boundary(net, bnd)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "network built for another boundary");
    }
    dbuf<double> c;
    MH_ALLOC(ctx, c, 1);
    MH_TRY(warm_start_run(ctx, bnd, alpha, net, mode, arith, sigma_dev, sigma_prev2_dev, rhs_dev, x0_dev, r0_dev, prec,
                          c.p, nullptr));
    double ch = 0.0;
    MH_CUDA(ctx, cudaMemcpyAsync(&ch, c.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (c_host) *c_host = ch;
    return MH_OK;
}

bool net_matches(const mh_net* net, const mh_boundary* b) { return net && same_boundary(net, b); }
