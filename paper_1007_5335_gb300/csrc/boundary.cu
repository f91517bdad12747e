// Boundary part of the method: geometry (Section 3.2, pseudospectral normals), the
// Nystrom operator of eq. discrete_sys with the Alpert log-singular correction and
// Fourier interpolation (Section 3.2), its application, GMRES (Section 3.2), and the
// off-surface double-layer potential U^h (Section 2) with the near-boundary rules.
#include <algorithm>
#include <cmath>
#include <mutex>

#include <cuda_fp16.h>

#include "alpert_rule.h"
#include "bessel.cuh"
#include "mh_internal.cuh"

namespace {

constexpr int UPSAMPLE = 16;        // fine grid for targets within 10 h_s of a curve
constexpr int FINE_TG = 4;          // auxiliary targets per block of the binary32 upsampled rule
constexpr double NEAR_NODE = 12.0;  // project on the curve when the nearest node is within 12 h*
constexpr double NEAR_FINE = 10.0;  // d < 10 h_s: upsampled rule
constexpr double NEAR_LINE = 0.25;  // d < h_s/4: interpolation along the normal
// Flops counted for one double-layer kernel value K(y, x) w (the unit of the pair sums):
// offsets 2, r^2 2, rsqrt 1, z 1, Chebyshev tail (4/z - 1, 10-term Clenshaw) 21, exp 8,
// products with e^{-z}/sqrt(z) 3, dot product 3, scaling and accumulate 4 (FMA = 2 flops)
constexpr double DL_FLOPS = 68.0;

struct AlpertRule {
    int l, a;
    double x[MH_ALPERT_LMAX], w[MH_ALPERT_LMAX];
};

// Modes m = 0..N/2 of curve k start at coef index off[k]/2 + k (4 doubles per mode).
__device__ __forceinline__ int64_t coef_base(const int32_t* off, int k) { return (int64_t)off[k] / 2 + k; }

// Warp sum; the result is broadcast from lane 0 so that every lane holds the same bits
// (butterfly sums can differ in the last bit between lanes, and callers branch on them).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// Fourier coefficients c_m = (1/N) sum_n y_n e^{-2 pi i m n / N}, m = 0..N/2, of the
// node coordinates (x and y), exact twiddles through the integer m n mod N.
__global__ void k_fourier_xy(const double* __restrict__ xy, const int32_t* __restrict__ nn,
                             const int32_t* __restrict__ off, int ncurves, int64_t total, double* coef) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    int k = 0;
    while (k + 1 < ncurves && g >= coef_base(off, k + 1)) ++k;
    const int N = nn[k];
    const int m = (int)(g - coef_base(off, k));
    const double* p = xy + 2 * (int64_t)off[k];
    double xr = 0, xi = 0, yr = 0, yi = 0;
    for (int n = 0; n < N; ++n) {
        int r = (int)(((int64_t)m * n) % N);
        double s, c;
        sincospi(2.0 * r / N, &s, &c);
        xr += p[2 * n] * c;
        xi -= p[2 * n] * s;
        yr += p[2 * n + 1] * c;
        yi -= p[2 * n + 1] * s;
    }
    double inv = 1.0 / N;
    coef[4 * g + 0] = xr * inv;
    coef[4 * g + 1] = xi * inv;
    coef[4 * g + 2] = yr * inv;
    coef[4 * g + 3] = yi * inv;
}

template <int BS>
__device__ double block_sum(double v);

// Contribution of mode m of one coordinate (re, im) at angle with (s, c) = sin, cos(m t).
// Accumulates value, first and second t-derivative of the trigonometric interpolant
//   p(t) = c_0 + sum_{0<m<N/2} 2 Re(c_m e^{imt}) + c_{N/2} cos(N t / 2).
__device__ __forceinline__ void mode_acc(int m, int N, double re, double im, double s, double c, double& v,
                                         double& d1, double& d2) {
    if (m == 0) {
        v += re;
    } else if (2 * m == N) {
        double h = 0.5 * N;
        v += re * c;
        d1 -= h * re * s;
        d2 -= h * h * re * c;
    } else {
        double a = 2.0 * (re * c - im * s);
        v += a;
        d1 += 2.0 * m * (-re * s - im * c);
        d2 -= (double)m * m * a;
    }
}

// Position and first two derivatives at the nodes (exact twiddles), plus |y'| and the
// diagonal limit K(x,x) = -(y''.n)/(2|y'|^2) (Section 2).
__global__ void k_node_geometry(const double* __restrict__ coef, const int32_t* __restrict__ nn,
                                const int32_t* __restrict__ off, const int32_t* __restrict__ curve_of,
                                int64_t n, double* geo) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int k = curve_of[j];
    const int N = nn[k];
    const int i = (int)(j - off[k]);
    const double* c = coef + 4 * coef_base(off, k);
    double x = 0, dx = 0, ddx = 0, y = 0, dy = 0, ddy = 0;
    for (int m = 0; m <= N / 2; ++m) {
        int r = (int)(((int64_t)m * i) % N);
        double s, co;
        sincospi(2.0 * r / N, &s, &co);
        mode_acc(m, N, c[4 * m], c[4 * m + 1], s, co, x, dx, ddx);
        mode_acc(m, N, c[4 * m + 2], c[4 * m + 3], s, co, y, dy, ddy);
    }
    double sp = sqrt(dx * dx + dy * dy);
    double nx = dy / sp, ny = -dx / sp;
    double* g = geo + 8 * j;
    g[0] = x;
    g[1] = y;
    g[2] = dx;
    g[3] = dy;
    g[4] = ddx;
    g[5] = ddy;
    g[6] = sp;
    g[7] = -(ddx * nx + ddy * ny) / (2.0 * sp * sp);
}

// Geometry on the 16x fine grid t_f = 2 pi f / (16 N): x, y, nx, ny, |y'|, h_f.
__global__ void k_fine_geometry(const double* __restrict__ coef, const int32_t* __restrict__ nn,
                                const int32_t* __restrict__ off, const int64_t* __restrict__ foff, int ncurves,
                                int64_t nfine, double* fg) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nfine) return;
    int k = 0;
    while (k + 1 < ncurves && g >= foff[k + 1]) ++k;
    const int N = nn[k];
    const int NF = UPSAMPLE * N;
    const int f = (int)(g - foff[k]);
    const double* c = coef + 4 * coef_base(off, k);
    double x = 0, dx = 0, ddx = 0, y = 0, dy = 0, ddy = 0;
    for (int m = 0; m <= N / 2; ++m) {
        int r = (int)(((int64_t)m * f) % NF);
        double s, co;
        sincospi(2.0 * r / NF, &s, &co);
        mode_acc(m, N, c[4 * m], c[4 * m + 1], s, co, x, dx, ddx);
        mode_acc(m, N, c[4 * m + 2], c[4 * m + 3], s, co, y, dy, ddy);
    }
    double sp = sqrt(dx * dx + dy * dy);
    double* o = fg + 6 * g;
    o[0] = x;
    o[1] = y;
    o[2] = dy / sp;
    o[3] = -dx / sp;
    o[4] = sp;
    o[5] = 2.0 * MH_PI / NF;
}

// Warp-cooperative evaluation of a curve (position, y', y'') at an arbitrary parameter t.
__device__ void curve_eval_warp(const double* c, int N, double t, double out[6]) {
    const int lane = threadIdx.x & 31;
    double x = 0, dx = 0, ddx = 0, y = 0, dy = 0, ddy = 0;
    for (int m = lane; m <= N / 2; m += 32) {
        double s, co;
        sincos(m * t, &s, &co);
        mode_acc(m, N, c[4 * m], c[4 * m + 1], s, co, x, dx, ddx);
        mode_acc(m, N, c[4 * m + 2], c[4 * m + 3], s, co, y, dy, ddy);
    }
    out[0] = warp_sum(x);
    out[1] = warp_sum(y);
    out[2] = warp_sum(dx);
    out[3] = warp_sum(dy);
    out[4] = warp_sum(ddx);
    out[5] = warp_sum(ddy);
}

// K(y, x) = (1/alpha) K1(|y-x|/alpha) (y-x).n_y / |y-x|  (Section 3.2)
// Beyond r = 45 alpha (binary64) or 30 alpha (binary32) a pair contributes K1(r/alpha) / alpha
// < e^{-r/alpha} / alpha: below 1e-19 (1e-13) of the unit-distance value, far under the
// rounding of the sums it enters, so the pair is skipped before K1 is evaluated.
constexpr double MH_DL_CUT64 = 45.0;
constexpr float MH_DL_CUT32 = 30.f;

__device__ __forceinline__ double dl_kernel(double yx, double yy, double nx, double ny, double xx, double xy,
                                            double inv_alpha) {
    double dx = yx - xx, dy = yy - xy;
    double r = sqrt(dx * dx + dy * dy);
    const double z = r * inv_alpha;
    if (z > MH_DL_CUT64) return 0.0;
    return mh_k1(z) * inv_alpha * (dx * nx + dy * ny) / r;
}

// Trapezoid part of eq. discrete_sys (all curves), the own-curve Alpert window left
// empty (or, with l = 0, the diagonal limit), identity on the diagonal.
__global__ void k_assemble_trap(const double* __restrict__ geo, const int32_t* __restrict__ curve_of,
                                const int32_t* __restrict__ nn, const int32_t* __restrict__ off, int64_t n,
                                double inv_alpha, int a, double* A) {
    int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (col >= n) return;
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const double* gj = geo + 8 * j;
        const double* gc = geo + 8 * col;
        const int kj = curve_of[j], kc = curve_of[col];
        const double h = 2.0 * MH_PI / nn[kc];
        double v;
        bool win = false;
        if (kj == kc) {
            int N = nn[kj];
            int d = (int)((col - j) % N);
            if (d < 0) d += N;
            int circ = d < N - d ? d : N - d;
            win = a > 0 ? circ < a : circ == 0;
        }
        if (win) {
            v = (a == 0) ? gj[7] * gj[6] * h : 0.0;
        } else {
            double sp = gc[6];
            v = dl_kernel(gc[0], gc[1], gc[3] / sp, -gc[2] / sp, gj[0], gj[1], inv_alpha) * sp * h;
        }
        A[j * n + col] = v * (1.0 / MH_PI) + (col == j ? 1.0 : 0.0);
    }
}

// Alpert correction rows: 2l off-grid nodes t_j +- x_m h per row with geometry from the
// trigonometric interpolant, spread onto the own curve's nodes through the periodic
// interpolation kernel D_N(tau) = sin(N tau/2) cot(tau/2) / N (Section 3.2).
__global__ void k_assemble_alpert(const double* __restrict__ geo, const double* __restrict__ coef,
                                  const int32_t* __restrict__ curve_of, const int32_t* __restrict__ nn,
                                  const int32_t* __restrict__ off, int64_t n, double inv_alpha, AlpertRule R,
                                  double* A) {
    __shared__ double cp[2 * MH_ALPERT_LMAX], sp_s[2 * MH_ALPERT_LMAX], sh[2 * MH_ALPERT_LMAX];
    const int64_t j = blockIdx.x;
    const int k = curve_of[j];
    const int N = nn[k];
    const int o = off[k];
    const int jj = (int)(j - o);
    const double h = 2.0 * MH_PI / N;
    const double* c = coef + 4 * coef_base(off, k);
    const double* gj = geo + 8 * j;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = warp; p < 2 * R.l; p += nw) {
        const int m = p % R.l;
        const double s = p < R.l ? 1.0 : -1.0;
        double t = (jj + s * R.x[m]) * h;
        double v[6];
        curve_eval_warp(c, N, t, v);
        if ((threadIdx.x & 31) == 0) {
            double spd = sqrt(v[2] * v[2] + v[3] * v[3]);
            double K = dl_kernel(v[0], v[1], v[3] / spd, -v[2] / spd, gj[0], gj[1], inv_alpha);
            cp[p] = (1.0 / MH_PI) * h * R.w[m] * spd * K;
            sp_s[p] = s * sinpi(R.x[m]) / N;
            sh[p] = s * R.x[m];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double sgn = ((jj - i) & 1) ? -1.0 : 1.0;
        double acc = 0.0;
        for (int p = 0; p < 2 * R.l; ++p) {
            double v = (jj - i + sh[p]) / N;
            acc += cp[p] * sp_s[p] * cospi(v) / sinpi(v);
        }
        A[j * n + o + i] += sgn * acc;
    }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// lo = a - hi in binary64, rounded to binary32 (hi = a rounded to binary32)
__global__ void k_split_lo(const double* __restrict__ a, const float* __restrict__ hi, float* __restrict__ lo,
                           int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        lo[i] = (float)(a[i] - (double)hi[i]);
}

// Low part of the binary64 operator in binary16: lo16 = (a - hi) 2^24 rounded to nearest
// (the difference is exact in binary64, the scaling by a power of two too, so the only
// rounding is the final one to binary16).
__global__ void k_split_lo16(const double* __restrict__ a, const float* __restrict__ hi, uint16_t* __restrict__ lo,
                             int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        lo[i] = __half_as_ushort(__double2half((a[i] - (double)hi[i]) * 16777216.0));
}

// x = xh + xl with xh = x rounded to binary32
__global__ void k_split_vec(const double* __restrict__ x, float* __restrict__ xh, float* __restrict__ xl, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const float h = (float)x[i];
        xh[i] = h;
        xl[i] = (float)(x[i] - (double)h);
    }
}

// y = A x, one warp per row, 16-byte loads (N_Gamma is even, so rows stay aligned).
__global__ void k_gemv64(const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y,
                         int64_t n, const int* __restrict__ gate = nullptr) {
    if (gate && *gate) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < n; row += nwarps) {
        const double2* a = reinterpret_cast<const double2*>(A + row * n);
        const double2* xv = reinterpret_cast<const double2*>(x);
        double acc = 0.0;
        for (int64_t c = lane; c < n / 2; c += 32) {
            double2 av = __ldcs(a + c);
            double2 xx = __ldg(xv + c);
            acc = fma(av.x, xx.x, acc);
            acc = fma(av.y, xx.y, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) y[row] = acc;
    }
}

// binary32 operator times a binary32 copy of x (converted once per call: conversions
// from binary64 run on the slow FP64 pipe of this part and must stay out of the loop).
// One warp per row; four independent loads in flight per lane (16-byte loads when the
// row length is a multiple of 4, 8-byte loads otherwise).
__global__ void k_gemv32(const float* __restrict__ A, const float* __restrict__ x, double* __restrict__ y,
                         int64_t n, const int* __restrict__ gate = nullptr) {
    if (gate && *gate) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < n; row += nwarps) {
        const float* a = A + row * n;
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
        if ((n & 3) == 0) {
            const float4* a4 = reinterpret_cast<const float4*>(a);
            const float4* x4 = reinterpret_cast<const float4*>(x);
            const int64_t n4 = n >> 2;
            int64_t c = lane;
            for (; c + 96 < n4; c += 128) {
                const float4 a0 = __ldcs(a4 + c), a1 = __ldcs(a4 + c + 32), a2 = __ldcs(a4 + c + 64),
                             a3 = __ldcs(a4 + c + 96);
                const float4 x0 = __ldg(x4 + c), x1 = __ldg(x4 + c + 32), x2 = __ldg(x4 + c + 64),
                             x3 = __ldg(x4 + c + 96);
                f0 = fmaf(a0.x, x0.x, fmaf(a0.y, x0.y, fmaf(a0.z, x0.z, fmaf(a0.w, x0.w, f0))));
                f1 = fmaf(a1.x, x1.x, fmaf(a1.y, x1.y, fmaf(a1.z, x1.z, fmaf(a1.w, x1.w, f1))));
                f2 = fmaf(a2.x, x2.x, fmaf(a2.y, x2.y, fmaf(a2.z, x2.z, fmaf(a2.w, x2.w, f2))));
                f3 = fmaf(a3.x, x3.x, fmaf(a3.y, x3.y, fmaf(a3.z, x3.z, fmaf(a3.w, x3.w, f3))));
            }
            for (; c < n4; c += 32) {
                const float4 av = __ldcs(a4 + c), xv = __ldg(x4 + c);
                f0 = fmaf(av.x, xv.x, fmaf(av.y, xv.y, fmaf(av.z, xv.z, fmaf(av.w, xv.w, f0))));
            }
        } else {
            const float2* a2p = reinterpret_cast<const float2*>(a);
            const float2* x2p = reinterpret_cast<const float2*>(x);
            for (int64_t c = lane; c < n / 2; c += 32) {
                const float2 av = __ldcs(a2p + c), xv = __ldg(x2p + c);
                f0 = fmaf(av.x, xv.x, fmaf(av.y, xv.y, f0));
            }
        }
        float f = (f0 + f1) + (f2 + f3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if (lane == 0) y[row] = (double)f;
    }
}

// Row-split GEMVs: SPLIT warps share a row (contiguous segments in 16-byte units, combined in
// a fixed order through shared memory).  Blocks of 8 / SPLIT rows keep the hardware's dynamic
// block scheduling fine-grained, so no SM is left with a whole extra block of rows at the end
// of the sweep over the operator.  n must be a multiple of 4 (binary32) or 2 (binary64).
template <int SPLIT>
__global__ void __launch_bounds__(256) k_gemv32s(const float* __restrict__ A, const float* __restrict__ x,
                                                 double* __restrict__ y, int64_t n, const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ float part[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (8 / SPLIT) + warp / SPLIT;
    const int q = warp % SPLIT;
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
    if (row < n) {
        const int64_t n4 = n >> 2;
        const int64_t c0 = q * n4 / SPLIT, c1 = (q + 1) * n4 / SPLIT;
        const float4* a4 = reinterpret_cast<const float4*>(A + row * n);
        const float4* x4 = reinterpret_cast<const float4*>(x);
        int64_t c = c0 + lane;
        for (; c + 96 < c1; c += 128) {
            const float4 a0 = __ldcs(a4 + c), a1 = __ldcs(a4 + c + 32), a2 = __ldcs(a4 + c + 64),
                         a3 = __ldcs(a4 + c + 96);
            const float4 x0 = __ldg(x4 + c), x1 = __ldg(x4 + c + 32), x2 = __ldg(x4 + c + 64), x3 = __ldg(x4 + c + 96);
            f0 = fmaf(a0.x, x0.x, fmaf(a0.y, x0.y, fmaf(a0.z, x0.z, fmaf(a0.w, x0.w, f0))));
            f1 = fmaf(a1.x, x1.x, fmaf(a1.y, x1.y, fmaf(a1.z, x1.z, fmaf(a1.w, x1.w, f1))));
            f2 = fmaf(a2.x, x2.x, fmaf(a2.y, x2.y, fmaf(a2.z, x2.z, fmaf(a2.w, x2.w, f2))));
            f3 = fmaf(a3.x, x3.x, fmaf(a3.y, x3.y, fmaf(a3.z, x3.z, fmaf(a3.w, x3.w, f3))));
        }
        for (; c < c1; c += 32) {
            const float4 av = __ldcs(a4 + c), xv = __ldg(x4 + c);
            f0 = fmaf(av.x, xv.x, fmaf(av.y, xv.y, fmaf(av.z, xv.z, fmaf(av.w, xv.w, f0))));
        }
    }
    float f = (f0 + f1) + (f2 + f3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) part[warp] = f;
    __syncthreads();
    if (q == 0 && lane == 0 && row < n) {
        float t = part[warp];
        for (int k = 1; k < SPLIT; ++k) t += part[warp + k];
        y[row] = (double)t;
    }
}

// One entry of the float-float product with the binary64 operator A = A32 + A32lo and
// x = xh + xl: the exact product of the high parts (TwoProduct by fma) plus the two cross terms,
// added to the float-float sum (sh, sl) by TwoSum; the dropped lo * lo term and the rounding of
// the cross terms are ~2^-48 of the entry.  Binary32 pipe only (the binary64 pipe runs at 1/64
// of its rate here).
__device__ __forceinline__ void ff_acc(float& sh, float& sl, float a, float al, float xh, float xl) {
    const float p = a * xh;
    const float e = fmaf(a, xh, -p);
    const float c = fmaf(a, xl, fmaf(al, xh, e));
    const float t = sh + p;
    const float bb = t - sh;
    sl += ((sh - (t - bb)) + (p - bb)) + c;
    sh = t;
}

// Row-split operator GEMVs whose operator loads go through shared memory by cp.async (16-byte
// asynchronous copies): every lane issues its share of a whole piece of its quarter row (up to
// GC_PIECE float4 per matrix) before it touches any of it, so the loads in flight are not
// limited by registers.  A lane reads back only the float4s it copied itself (no barrier).
// M = 1: y = A32 x in binary32; M = 2: y = (A32 + A32lo)(xh + xl) in float-float (ff_acc).
// n a multiple of 4; SPLIT warps per row, 8 / SPLIT rows per 256-thread block.
constexpr int GC_PIECE = 3;   // float4 per lane and matrix per piece: 24 KB per block, up to 8 blocks per SM

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <int SPLIT, int M>
__global__ void __launch_bounds__(256) k_gemv_cpa(const float* __restrict__ A, const float* __restrict__ Al,
                                                  const float* __restrict__ xh, const float* __restrict__ xl,
                                                  double* __restrict__ y, int64_t n, const int* __restrict__ gate) {
    if (gate && *gate) return;
    extern __shared__ __align__(16) float4 gc_stage[];   // [warp][M][GC_PIECE * 32]
    __shared__ float part[2][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* st = gc_stage + (size_t)warp * M * GC_PIECE * 32;
    const int64_t row = (int64_t)blockIdx.x * (8 / SPLIT) + warp / SPLIT;
    const int q = warp % SPLIT;
    float hi = 0.f, lo = 0.f;
    if (row < n) {
        const int64_t n4 = n >> 2;
        const int64_t c0 = q * n4 / SPLIT, c1 = (q + 1) * n4 / SPLIT;
        const float4* a4 = reinterpret_cast<const float4*>(A + row * n);
        const float4* b4 = reinterpret_cast<const float4*>(Al + (M == 2 ? row * n : 0));
        const float4* xh4 = reinterpret_cast<const float4*>(xh);
        const float4* xl4 = reinterpret_cast<const float4*>(xl);
        for (int64_t p0 = c0; p0 < c1; p0 += GC_PIECE * 32) {
#pragma unroll
            for (int u = 0; u < GC_PIECE; ++u) {
                const int64_t c = p0 + lane + 32 * u;
                if (c < c1) {
                    cp_async16(st + lane + 32 * u, a4 + c);
                    if (M == 2) cp_async16(st + GC_PIECE * 32 + lane + 32 * u, b4 + c);
                }
            }
            cp_async_wait_all();
#pragma unroll
            for (int u = 0; u < GC_PIECE; ++u) {
                const int64_t c = p0 + lane + 32 * u;
                if (c < c1) {
                    const float4 av = st[lane + 32 * u];
                    const float4 uv = __ldg(xh4 + c);
                    if (M == 1) {
                        hi = fmaf(av.x, uv.x, hi);
                        hi = fmaf(av.y, uv.y, hi);
                        hi = fmaf(av.z, uv.z, hi);
                        hi = fmaf(av.w, uv.w, hi);
                    } else {
                        const float4 bv = st[GC_PIECE * 32 + lane + 32 * u];
                        const float4 vv = __ldg(xl4 + c);
                        ff_acc(hi, lo, av.x, bv.x, uv.x, vv.x);
                        ff_acc(hi, lo, av.y, bv.y, uv.y, vv.y);
                        ff_acc(hi, lo, av.z, bv.z, uv.z, vv.z);
                        ff_acc(hi, lo, av.w, bv.w, uv.w, vv.w);
                    }
                }
            }
            __syncwarp();   // the next piece reuses the warp's stage
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        if (M == 1) {
            hi += oh;
        } else {
            const float t = hi + oh, bb = t - hi;
            lo += ((hi - (t - bb)) + (oh - bb)) + ol;
            hi = t;
        }
    }
    if (lane == 0) {
        part[0][warp] = hi;
        part[1][warp] = lo;
    }
    __syncthreads();
    if (q == 0 && lane == 0 && row < n) {
        if (M == 1) {
            float t = part[0][warp];
            for (int k = 1; k < SPLIT; ++k) t += part[0][warp + k];
            y[row] = (double)t;
        } else {
            double t = (double)part[0][warp] + (double)part[1][warp];
            for (int k = 1; k < SPLIT; ++k) t += (double)part[0][warp + k] + (double)part[1][warp + k];
            y[row] = t;
        }
    }
}

// The float-float product with the low part in binary16: y = (A32 + 2^-24 A16)(xh + xl), 6
// bytes per entry instead of 8.  Each piece of a warp's quarter row is copied by cp.async
// as contiguous 512-byte runs (binary32 part: 2 GH_PIECE float4 per lane; binary16 part:
// GH_PIECE 16-byte groups of 8 entries per lane); lane l then takes binary32 float4 j = l +
// 32 v and the four binary16 entries of the same columns (8 bytes at j * 8 of the binary16
// run, copied by another lane: the warp waits for all its copies first).  n a multiple of 8.
constexpr int GH_PIECE = 2;   // 16-byte groups of binary16 per lane per piece: 24 KB per block

template <int SPLIT>
__global__ void __launch_bounds__(256) k_gemv_cph(const float* __restrict__ A, const uint16_t* __restrict__ Ah,
                                                  const float* __restrict__ xh, const float* __restrict__ xl,
                                                  double* __restrict__ y, int64_t n, const int* __restrict__ gate) {
    if (gate && *gate) return;
    extern __shared__ __align__(16) float4 gc_stage[];   // [warp][3 GH_PIECE * 32]
    __shared__ float part[2][8];
    constexpr float SCALE = 5.9604644775390625e-08f;   // 2^-24
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* stA = gc_stage + (size_t)warp * 3 * GH_PIECE * 32;   // 2 GH_PIECE * 32 float4
    float4* stH = stA + 2 * GH_PIECE * 32;                       // GH_PIECE * 32 groups of 8 binary16
    const uint2* stH2 = reinterpret_cast<const uint2*>(stH);
    const int64_t row = (int64_t)blockIdx.x * (8 / SPLIT) + warp / SPLIT;
    const int q = warp % SPLIT;
    float hi = 0.f, lo = 0.f;
    if (row < n) {
        const int64_t n8 = n >> 3;
        const int64_t c0 = q * n8 / SPLIT, c1 = (q + 1) * n8 / SPLIT;   // column octets of the quarter
        const float4* a4 = reinterpret_cast<const float4*>(A + row * n);
        const float4* h8 = reinterpret_cast<const float4*>(Ah + row * n);
        const float4* xh4 = reinterpret_cast<const float4*>(xh);
        const float4* xl4 = reinterpret_cast<const float4*>(xl);
        for (int64_t p0 = c0; p0 < c1; p0 += GH_PIECE * 32) {
#pragma unroll
            for (int v = 0; v < 2 * GH_PIECE; ++v) {
                const int j = lane + 32 * v;
                if (2 * p0 + j < 2 * c1) cp_async16(stA + j, a4 + 2 * p0 + j);
            }
#pragma unroll
            for (int u = 0; u < GH_PIECE; ++u) {
                const int o = lane + 32 * u;
                if (p0 + o < c1) cp_async16(stH + o, h8 + p0 + o);
            }
            // the piece's x values are loaded while the operator copies are in flight
            float4 xu[2 * GH_PIECE], xv[2 * GH_PIECE];
#pragma unroll
            for (int v = 0; v < 2 * GH_PIECE; ++v) {
                const int j = lane + 32 * v;
                if (2 * p0 + j < 2 * c1) {
                    xu[v] = __ldg(xh4 + 2 * p0 + j);
                    xv[v] = __ldg(xl4 + 2 * p0 + j);
                }
            }
            cp_async_wait_all();
            __syncwarp();   // the binary16 groups were copied by other lanes
#pragma unroll
            for (int v = 0; v < 2 * GH_PIECE; ++v) {
                const int j = lane + 32 * v;
                if (2 * p0 + j < 2 * c1) {
                    const float4 av = stA[j];
                    const uint2 hv = stH2[j];
                    const float2 l01 = __half22float2(*reinterpret_cast<const __half2*>(&hv.x));
                    const float2 l23 = __half22float2(*reinterpret_cast<const __half2*>(&hv.y));
                    const float4 uv = xu[v], vv = xv[v];
                    ff_acc(hi, lo, av.x, l01.x * SCALE, uv.x, vv.x);
                    ff_acc(hi, lo, av.y, l01.y * SCALE, uv.y, vv.y);
                    ff_acc(hi, lo, av.z, l23.x * SCALE, uv.z, vv.z);
                    ff_acc(hi, lo, av.w, l23.y * SCALE, uv.w, vv.w);
                }
            }
            __syncwarp();   // the next piece reuses the warp's stage
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        const float t = hi + oh, bb = t - hi;
        lo += ((hi - (t - bb)) + (oh - bb)) + ol;
        hi = t;
    }
    if (lane == 0) {
        part[0][warp] = hi;
        part[1][warp] = lo;
    }
    __syncthreads();
    if (q == 0 && lane == 0 && row < n) {
        double t = (double)part[0][warp] + (double)part[1][warp];
        for (int k = 1; k < SPLIT; ++k) t += (double)part[0][warp + k] + (double)part[1][warp + k];
        y[row] = t;
    }
}

template <int SPLIT>
__global__ void __launch_bounds__(256) k_gemv64s(const double* __restrict__ A, const double* __restrict__ x,
                                                 double* __restrict__ y, int64_t n, const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double part[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (8 / SPLIT) + warp / SPLIT;
    const int q = warp % SPLIT;
    double a0 = 0.0, a1 = 0.0;
    if (row < n) {
        const int64_t n2 = n >> 1;
        const int64_t c0 = q * n2 / SPLIT, c1 = (q + 1) * n2 / SPLIT;
        const double2* a = reinterpret_cast<const double2*>(A + row * n);
        const double2* xv = reinterpret_cast<const double2*>(x);
        int64_t c = c0 + lane;
        for (; c + 32 < c1; c += 64) {
            const double2 u = __ldcs(a + c), v = __ldcs(a + c + 32);
            const double2 xu = __ldg(xv + c), xw = __ldg(xv + c + 32);
            a0 = fma(u.x, xu.x, fma(u.y, xu.y, a0));
            a1 = fma(v.x, xw.x, fma(v.y, xw.y, a1));
        }
        for (; c < c1; c += 32) {
            const double2 u = __ldcs(a + c), xu = __ldg(xv + c);
            a0 = fma(u.x, xu.x, fma(u.y, xu.y, a0));
        }
    }
    double f = warp_sum(a0 + a1);
    if (lane == 0) part[warp] = f;
    __syncthreads();
    if (q == 0 && lane == 0 && row < n) {
        double t = part[warp];
        for (int k = 1; k < SPLIT; ++k) t += part[warp + k];
        y[row] = t;
    }
}

__global__ void k_to_float_vec(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ---------------- binary32 double layer (mixed precision) ----------------

// Source data relative to tile centres: tiles of MH_TILE consecutive nodes.
__global__ void k_prep_src32(const double* __restrict__ geo, int64_t n, float4* src, double2* tc, float* tr) {
    const int64_t tile = blockIdx.x;
    const int64_t s0 = tile * MH_TILE;
    const int cnt = (n - s0) < MH_TILE ? (int)(n - s0) : MH_TILE;
    __shared__ double cx, cy;
    if (threadIdx.x == 0) {
        double ax = 0, ay = 0;
        for (int i = 0; i < cnt; ++i) {
            ax += geo[8 * (s0 + i)];
            ay += geo[8 * (s0 + i) + 1];
        }
        cx = ax / cnt;
        cy = ay / cnt;
        tc[tile] = make_double2(cx, cy);
    }
    __syncthreads();
    __shared__ float rmax;
    if (threadIdx.x == 0) rmax = 0.f;
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const double* g = geo + 8 * (s0 + i);
        const double sp = g[6];
        src[s0 + i] = make_float4((float)(g[0] - cx), (float)(g[1] - cy), (float)(g[3] / sp), (float)(-g[2] / sp));
        // the largest distance from the centre (non-negative floats order like their bit patterns)
        atomicMax(reinterpret_cast<int*>(&rmax), __float_as_int((float)hypot(g[0] - cx, g[1] - cy)));
    }
    __syncthreads();
    if (threadIdx.x == 0) tr[tile] = rmax * 1.0001f;
}

// Fine nodes relative to chunk centres: chunks of MH_TILE fine nodes inside each curve.
// Per fine chunk: offsets of its nodes from the chunk centre (binary32), the centre in
// binary64 and as float-float pairs (x_hi, x_lo, y_hi, y_lo), and the chunk radius.
__global__ void k_prep_fine32(const double* __restrict__ fg, const int64_t* __restrict__ foff,
                              const int64_t* __restrict__ coff, int ncurves, float4* out, double2* cc,
                              float4* ccf, float* crad) {
    const int64_t chunk = blockIdx.x;
    int k = 0;
    while (k + 1 < ncurves && chunk >= coff[k + 1]) ++k;
    const int64_t f0 = foff[k] + (chunk - coff[k]) * MH_TILE;
    const int cnt = (foff[k + 1] - f0) < MH_TILE ? (int)(foff[k + 1] - f0) : MH_TILE;
    __shared__ double cx, cy;
    if (threadIdx.x == 0) {
        double ax = 0, ay = 0;
        for (int i = 0; i < cnt; ++i) {
            ax += fg[6 * (f0 + i)];
            ay += fg[6 * (f0 + i) + 1];
        }
        cx = ax / cnt;
        cy = ay / cnt;
        cc[chunk] = make_double2(cx, cy);
    }
    __syncthreads();
    float r2max = 0.f;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const double* g = fg + 6 * (f0 + i);
        const float4 v = make_float4((float)(g[0] - cx), (float)(g[1] - cy), (float)g[2], (float)g[3]);
        out[f0 + i] = v;
        r2max = fmaxf(r2max, v.x * v.x + v.y * v.y);
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) r2max = fmaxf(r2max, __shfl_xor_sync(0xffffffffu, r2max, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2max;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r2max = fmaxf(r2max, red[w]);
        const float xh = (float)cx, yh = (float)cy;
        ccf[chunk] = make_float4(xh, (float)(cx - (double)xh), yh, (float)(cy - (double)yh));
        crad[chunk] = sqrtf(r2max) * 1.0001f;   // covers the rounding of the offsets
    }
}

__global__ void k_weights32(const double* __restrict__ sigma, const double* __restrict__ geo,
                            const int32_t* __restrict__ curve_of, const int32_t* __restrict__ nn, int64_t n, float* w) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < n) w[s] = (float)(sigma[s] * geo[8 * s + 6] * (2.0 * MH_PI / nn[curve_of[s]]));
}

// Binary32 double-layer pairs: mh_dl32_pair (bessel.cuh) returns g(z) (d.n) with
// g = K1(z)/z; the kernels below apply the prefactor times 1/alpha^2 (pref32) in binary64.

// Coarse trapezoid sum in binary32: sources staged through shared memory in tiles of
// MH_TILE (the weight folded into the normal as they are staged); the target offset from the
// tile centre is formed once per tile in binary64; per-tile partial sums are added in binary64.
// A tile whose nodes all lie on one curve is skipped at once when that curve is flagged for
// the target; when it lies beyond 2 alpha of every target of the warp (tile centre distance
// above 2 alpha plus the tile radius) its pairs take the z > 2 form without a branch or a
// test (mh_dl32_pair_far; pairs beyond the cut come out below the rounding of the sum).
__global__ void __launch_bounds__(MH_TILE) k_dlp_coarse32(const double* __restrict__ xy,
                                                          const uint32_t* __restrict__ fine, int64_t nt,
                                                          const float4* __restrict__ src, const float* __restrict__ w,
                                                          const int32_t* __restrict__ curve_of,
                                                          const double2* __restrict__ tc, const float* __restrict__ tr,
                                                          int64_t ns, mh_dl32 c32, double pref, double* out) {
    __shared__ float4 s4[MH_TILE];
    __shared__ int sk[MH_TILE];
    const float two_a = 2.0001f * c32.a;
    const int64_t t = blockIdx.x * (int64_t)MH_TILE + threadIdx.x;
    const bool active = t < nt;
    const double px = active ? xy[2 * t] : 0.0, py = active ? xy[2 * t + 1] : 0.0;
    const uint32_t mask = active ? fine[t] : 0xffffffffu;
    double acc = 0.0;
    const int64_t ntile = (ns + MH_TILE - 1) / MH_TILE;
    // gridDim.y > 1 splits the source tiles between blocks; partial sums go to
    // out[blockIdx.y * nt + t] (without the prefactor) for a fixed-order reduction
    const int64_t per = (ntile + gridDim.y - 1) / gridDim.y;
    const int64_t tile0 = blockIdx.y * per, tile1 = min(ntile, tile0 + per);
    for (int64_t tile = tile0; tile < tile1; ++tile) {
        const int64_t s = tile * MH_TILE + threadIdx.x;
        if (s < ns) {
            const float4 v = src[s];
            const float wd = w[s];
            s4[threadIdx.x] = make_float4(v.x, v.y, v.z * wd, v.w * wd);
            sk[threadIdx.x] = curve_of[s];
        }
        __syncthreads();
        const int cnt = (ns - tile * MH_TILE) < MH_TILE ? (int)(ns - tile * MH_TILE) : MH_TILE;
        const bool one_curve = sk[0] == sk[cnt - 1];   // consecutive nodes: one curve unless at a seam
        float tx = 0.f, ty = 0.f;
        bool skip = !active, far = true;
        if (active) {
            const double2 c = tc[tile];
            tx = (float)(px - c.x);
            ty = (float)(py - c.y);
            if (one_curve && ((mask >> sk[0]) & 1u)) skip = true;
            const float lim = two_a + tr[tile];
            far = fmaf(tx, tx, ty * ty) > lim * lim;
        }
        const bool warp_far = __all_sync(0xffffffffu, skip || far);
        if (!skip) {
            float part = 0.f;
            if (warp_far && one_curve) {
                for (int i = 0; i < cnt; ++i) {
                    const float4 v = s4[i];
                    part += mh_dl32_pair_far(v.x - tx, v.y - ty, v.z, v.w, c32);
                }
                part *= c32.a32;
            } else {
                for (int i = 0; i < cnt; ++i) {
                    if ((mask >> sk[i]) & 1u) continue;
                    const float4 v = s4[i];
                    part += mh_dl32_pair(v.x - tx, v.y - ty, v.z, v.w, c32);
                }
            }
            acc += (double)part;
        }
        __syncthreads();
    }
    if (active) {
        if (gridDim.y == 1)
            out[t] = pref * acc;
        else
            out[blockIdx.y * nt + t] = acc;
    }
}

__global__ void k_sum_partials(const double* __restrict__ part, int nsplit, int64_t nt, double pref, double* out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double s = 0.0;
    for (int j = 0; j < nsplit; ++j) s += part[j * nt + t];
    out[t] = pref * s;
}

// One warp's pairs of a fine chunk (MH_TILE nodes from f0, m of them present) against TG targets
// at offsets (dx0, dy0) from the chunk centre: pt[j] = sum over the lane's nodes.  FAR: every
// pair has r > 2 alpha (mh_dl32_pair_far, the alpha^{3/2} applied to the sums).
template <int TG, bool FAR>
__device__ __forceinline__ void fine_chunk(const float4* __restrict__ fine32, const float* __restrict__ wf, int64_t f0,
                                           int m, int lane, const float* dx0, const float* dy0, const mh_dl32& c32,
                                           float* pt) {
#pragma unroll
    for (int j = 0; j < TG; ++j) pt[j] = 0.f;
    auto pair = [&](float dx, float dy, float nx, float ny) {
        return FAR ? mh_dl32_pair_far(dx, dy, nx, ny, c32) : mh_dl32_pair_nt(dx, dy, nx, ny, c32);
    };
    if (m == MH_TILE) {
        // a whole chunk: every lane's MH_TILE / 32 nodes are loaded before the first pair, so the
        // loads are in flight together
        constexpr int U = MH_TILE / 32;
        float4 v[U];
        float w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = fine32[f0 + lane + 32 * u];
            w[u] = wf[f0 + lane + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float nx = v[u].z * w[u], ny = v[u].w * w[u];
#pragma unroll
            for (int j = 0; j < TG; ++j) pt[j] += pair(v[u].x - dx0[j], v[u].y - dy0[j], nx, ny);
        }
    } else {
        for (int i = lane; i < m; i += 32) {
            const float4 v = fine32[f0 + i];
            const float w = wf[f0 + i];
            const float nx = v.z * w, ny = v.w * w;
#pragma unroll
            for (int j = 0; j < TG; ++j) pt[j] += pair(v.x - dx0[j], v.y - dy0[j], nx, ny);
        }
    }
    if (FAR) {
#pragma unroll
        for (int j = 0; j < TG; ++j) pt[j] *= c32.a32;
    }
}

// Upsampled rule in binary32 at the auxiliary points of the normal-line rule.  One block per
// (group of TG auxiliary targets on curve k, slice of the curve's fine chunks); each warp takes
// one chunk (MH_TILE fine nodes) at a time and every lane evaluates its nodes against all TG
// targets, so one load of a node serves TG pairs.  The targets' offsets from the chunk centre
// are float-float differences (no binary64 arithmetic in the loop); a chunk farther than the
// cut plus its radius from every target is skipped; each chunk's binary32 sums go into
// float-float accumulators (TwoSum).  The slices of a group hand their sums to the group's last
// block to finish, which adds them in slice order and then adds pref * sum to every target.
template <int TG>
__global__ void __launch_bounds__(256) k_dlp_fine32_grp(
    const double* __restrict__ xy, const int32_t* __restrict__ pair_tgt, const int32_t* __restrict__ grp_curve,
    const int32_t* __restrict__ grp_pair, int slices, const float4* __restrict__ fine32, const float* __restrict__ wf,
    const int64_t* __restrict__ foff, const int64_t* __restrict__ coff, const float4* __restrict__ ccf,
    const float* __restrict__ crad, mh_dl32 c32, float cut_r, double pref, double* part, unsigned* cnt,
    double* out) {
    __shared__ double red[8][TG];
    const float two_a = 2.0001f * c32.a;   // beyond: z > 2 with a margin for the rounding of d2
    __shared__ int last;
    const int grp = blockIdx.x / slices, sl = blockIdx.x % slices;
    const int k = grp_curve[grp];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float txh[TG], txl[TG], tyh[TG], tyl[TG];
#pragma unroll
    for (int j = 0; j < TG; ++j) {
        const int p = grp_pair[grp * TG + j];
        // a padding entry sits far outside every cut: its pairs and chunk tests come out 0 / false
        const double px = p >= 0 ? xy[2 * (int64_t)pair_tgt[p]] : 1e30;
        const double py = p >= 0 ? xy[2 * (int64_t)pair_tgt[p] + 1] : 1e30;
        txh[j] = (float)px;
        txl[j] = (float)(px - (double)txh[j]);
        tyh[j] = (float)py;
        tyl[j] = (float)(py - (double)tyh[j]);
    }
    const int64_t nch = coff[k + 1] - coff[k];
    const int64_t c0 = coff[k] + nch * sl / slices, c1 = coff[k] + nch * (sl + 1) / slices;
    const int64_t fend = foff[k + 1];
    float hi[TG], lo[TG];
#pragma unroll
    for (int j = 0; j < TG; ++j) hi[j] = lo[j] = 0.f;
    for (int64_t ch = c0 + warp; ch < c1; ch += nw) {
        const float4 c = ccf[ch];
        const float lim = cut_r + crad[ch];
        const float flim = two_a + crad[ch];
        float dx0[TG], dy0[TG];
        bool near = false, far = true;
#pragma unroll
        for (int j = 0; j < TG; ++j) {
            dx0[j] = (txh[j] - c.x) + (txl[j] - c.y);
            dy0[j] = (tyh[j] - c.z) + (tyl[j] - c.w);
            const float d2 = fmaf(dx0[j], dx0[j], dy0[j] * dy0[j]);
            near |= d2 <= lim * lim;
            far &= d2 > flim * flim;
        }
        if (!near) continue;   // the same for the whole warp
        const int64_t f0 = foff[k] + (ch - coff[k]) * MH_TILE;
        const int m = (int)min((int64_t)MH_TILE, fend - f0);
        float pt[TG];
        // the chunk is within the cut of some target of the group: no per-pair tests; if it is
        // beyond 2 alpha of every target, every pair takes the z > 2 form without a branch
        if (far)
            fine_chunk<TG, true>(fine32, wf, f0, m, lane, dx0, dy0, c32, pt);
        else
            fine_chunk<TG, false>(fine32, wf, f0, m, lane, dx0, dy0, c32, pt);
#pragma unroll
        for (int j = 0; j < TG; ++j) {   // TwoSum: hi + lo += pt exactly up to the rounding of lo
            const float s = hi[j] + pt[j];
            const float bb = s - hi[j];
            lo[j] += (hi[j] - (s - bb)) + (pt[j] - bb);
            hi[j] = s;
        }
    }
#pragma unroll
    for (int j = 0; j < TG; ++j) {   // warp sum in float-float, one widening per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi[j], o), ol = __shfl_xor_sync(0xffffffffu, lo[j], o);
            const float t = hi[j] + oh, bb = t - hi[j];
            lo[j] += ((hi[j] - (t - bb)) + (oh - bb)) + ol;
            hi[j] = t;
        }
        if (lane == 0) red[warp][j] = (double)hi[j] + (double)lo[j];
    }
    __syncthreads();
    double s = 0.0;
    int t = -1;
    if (threadIdx.x < TG) {
        for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
        const int p = grp_pair[grp * TG + threadIdx.x];
        t = p >= 0 ? pair_tgt[p] : -1;
    }
    if (slices == 1) {
        if (t >= 0) atomicAdd(out + t, pref * s);
        return;
    }
    if (threadIdx.x < TG) part[((int64_t)grp * slices + sl) * TG + threadIdx.x] = s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(cnt + grp, 1u) == (unsigned)(slices - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < TG) {
        double tot = 0.0;
        for (int q = 0; q < slices; ++q) tot += __ldcg(part + ((int64_t)grp * slices + q) * TG + threadIdx.x);
        if (t >= 0) atomicAdd(out + t, pref * tot);
    }
    if (threadIdx.x == 0) cnt[grp] = 0u;
}

__global__ void k_dlp_fine64_blk(const double* __restrict__ xy, const int32_t* __restrict__ ptgt,
                                 const int32_t* __restrict__ pcurve, const double* __restrict__ fg,
                                 const double* __restrict__ wf, const int64_t* __restrict__ foff, double inv_alpha,
                                 double pref, double* out) {
    __shared__ double red[8];
    const int64_t p = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t t = ptgt[p];
    const int k = pcurve[p];
    const double px = xy[2 * t], py = xy[2 * t + 1];
    double acc = 0.0;
    for (int64_t f = foff[k] + threadIdx.x; f < foff[k + 1]; f += blockDim.x) {
        const double* g = fg + 6 * f;
        acc += dl_kernel(g[0], g[1], g[2], g[3], px, py, inv_alpha) * wf[f];
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += red[i];
        atomicAdd(out + t, pref * s);
    }
}

// Upsampled rule in binary32, one warp per (target, curve) pair, fine nodes in chunks of
// MH_TILE with binary64 chunk centres.
__global__ void k_dlp_fine32(const double* __restrict__ xy, const int32_t* __restrict__ ptgt,
                             const int32_t* __restrict__ pcurve, int64_t npairs, const float4* __restrict__ fine32,
                             const float* __restrict__ wf, const int64_t* __restrict__ foff,
                             const int64_t* __restrict__ coff, const double2* __restrict__ cc, mh_dl32 c32,
                             double pref, double* out) {
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= npairs) return;
    const int lane = threadIdx.x & 31;
    const int64_t t = ptgt[p];
    const int k = pcurve[p];
    const double px = xy[2 * t], py = xy[2 * t + 1];
    double acc = 0.0;
    for (int64_t ch = coff[k]; ch < coff[k + 1]; ++ch) {
        const double2 c = cc[ch];
        const float tx = (float)(px - c.x), ty = (float)(py - c.y);
        const int64_t f0 = foff[k] + (ch - coff[k]) * MH_TILE;
        const int64_t f1 = min(f0 + MH_TILE, foff[k + 1]);
        float part = 0.f;
        for (int64_t f = f0 + lane; f < f1; f += 32) {
            const float4 v = fine32[f];
            part += mh_dl32_pair(v.x - tx, v.y - ty, v.z, v.w, c32) * wf[f];
        }
        acc += (double)part;
    }
    acc = warp_sum(acc);
    if (lane == 0) atomicAdd(out + t, pref * acc);
}

// ---------------- GMRES helpers (binary64 Arnoldi) ----------------

template <int BS>
__device__ double block_sum(double v) {
    __shared__ double red[BS / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < BS / 32 ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// h[i] = V_i . w for i <= k (one block per i)
__global__ void k_multidot(const double* __restrict__ V, const double* __restrict__ w, int64_t n, double* h) {
    const int i = blockIdx.x;
    const double* v = V + (int64_t)i * n;
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(v[e], w[e], acc);
    acc = block_sum<256>(acc);
    if (threadIdx.x == 0) h[i] = acc;
}

// w -= sum_{i<=k} h[i] V_i ; hacc[i] += h[i]
__global__ void k_multiaxpy(const double* __restrict__ V, const double* __restrict__ h, int k1, int64_t n,
                            double* w) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = w[e];
        for (int i = 0; i < k1; ++i) acc = fma(-h[i], V[(int64_t)i * n + e], acc);
        w[e] = acc;
    }
}

__global__ void k_norm(const double* __restrict__ w, int64_t n, double* out) {
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(w[e], w[e], acc);
    acc = block_sum<1024>(acc);
    if (threadIdx.x == 0) *out = sqrt(acc);
}

// Hcol[i] = h1[i] + h2[i] (i <= k), Hcol[k+1] = ||w||, v_{k+1} = w / ||w||
__global__ void k_finish_column(const double* __restrict__ h1, const double* __restrict__ h2,
                                const double* __restrict__ nrm, int k, double* Hcol, const double* __restrict__ w,
                                double* vnext, int64_t n) {
    const double s = *nrm;
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e0 <= k) Hcol[e0] = h1[e0] + h2[e0];
    if (e0 == k + 1) Hcol[k + 1] = s;
    for (int64_t e = e0; e < n; e += (int64_t)gridDim.x * blockDim.x) vnext[e] = w[e] * inv;
}

// Apply the previous Givens rotations to column k of H, form rotation k, update g.
// small[0] = |g_{k+1}| (residual estimate).
__global__ void k_givens(double* H, int ldh, int k, double* cs, double* sn, double* g, double* small) {
    double* col = H + (int64_t)k * ldh;
    for (int i = 0; i < k; ++i) {
        double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    double a = col[k], b = col[k + 1];
    double den = hypot(a, b);
    double c = den > 0 ? a / den : 1.0, s = den > 0 ? b / den : 0.0;
    cs[k] = c;
    sn[k] = s;
    col[k] = den;
    col[k + 1] = 0.0;
    g[k + 1] = -s * g[k];
    g[k] = c * g[k];
    small[0] = fabs(g[k + 1]);
}

// Solve R y = g (k x k upper triangular, column-major with leading dimension ldh).
__global__ void k_backsolve(const double* H, int ldh, int k, const double* g, double* y) {
    for (int i = k - 1; i >= 0; --i) {
        double acc = g[i];
        for (int j = i + 1; j < k; ++j) acc -= H[(int64_t)j * ldh + i] * y[j];
        const double d = H[(int64_t)i * ldh + i];
        y[i] = d != 0.0 ? acc / d : 0.0;   // exact breakdown: the column adds nothing
    }
}

// x += sum_i y_i V_i
__global__ void k_update_x(const double* __restrict__ V, const double* __restrict__ y, int k, int64_t n,
                           double* x) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = x[e];
        for (int i = 0; i < k; ++i) acc = fma(y[i], V[(int64_t)i * n + e], acc);
        x[e] = acc;
    }
}

// ---- fused Arnoldi step: classical Gram-Schmidt twice over row slices of ARN_ROWS rows ----
// Every reduction runs in a fixed order (slice partials, then the slices in index order),
// so the iteration is deterministic.
constexpr int ARN_ROWS = 64;

// P[s k1 + i] = sum over slice s of V_i[e] w[e], i < k1 (a warp per i).  With kdev, k1 is
// *kdev + 1 (the iteration count of a sweep kept on the device: one kernel node serves every
// iteration of a graph loop).
__global__ void __launch_bounds__(256) k_arn_dots(const double* __restrict__ V, const double* __restrict__ w,
                                                  int64_t n, int k1, double* __restrict__ P,
                                                  const int* __restrict__ gate = nullptr,
                                                  const int* __restrict__ kdev = nullptr) {
    if (gate && *gate) return;
    if (kdev) k1 = *kdev + 1;
    const int s = blockIdx.x;
    const int64_t r0 = (int64_t)s * ARN_ROWS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t e0 = r0 + lane, e1 = r0 + lane + 32;
    const double w0 = e0 < n ? w[e0] : 0.0, w1 = e1 < n ? w[e1] : 0.0;
    for (int i = warp; i < k1; i += 8) {
        const double* v = V + (int64_t)i * n;
        double a = 0.0;
        if (e0 < n) a = v[e0] * w0;
        if (e1 < n) a = fma(v[e1], w1, a);
        a = warp_sum(a);
        if (lane == 0) P[(int64_t)s * k1 + i] = a;
    }
}

// h_i = sum_s Pin[s k1 + i]; w -= sum_i h_i V_i on the slice; then the partial dots of the
// new w (Pdots) or its partial squared norm (Pnorm).  Block 0 stores h in hout.
__global__ void __launch_bounds__(256) k_arn_update(const double* __restrict__ V, double* __restrict__ w, int64_t n,
                                                    int k1, const double* __restrict__ Pin, int S,
                                                    double* __restrict__ Pdots, double* __restrict__ Pnorm,
                                                    double* __restrict__ hout, const int* __restrict__ gate = nullptr,
                                                    const int* __restrict__ kdev = nullptr) {
    if (gate && *gate) return;
    if (kdev) k1 = *kdev + 1;
    extern __shared__ double sh[];      // h[k1], then the slice of w
    double* h = sh;
    double* wsl = sh + k1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < k1; i += 8) {      // a warp per coefficient, lanes over the slices
        double a = 0.0;
        for (int q = lane; q < S; q += 32) a += Pin[(int64_t)q * k1 + i];
        a = warp_sum(a);
        if (lane == 0) {
            h[i] = a;
            if (blockIdx.x == 0) hout[i] = a;
        }
    }
    __syncthreads();
    const int s = blockIdx.x;
    const int64_t r0 = (int64_t)s * ARN_ROWS;
    if (threadIdx.x < ARN_ROWS) {
        const int64_t e = r0 + threadIdx.x;
        double a = 0.0;
        if (e < n) {
            a = w[e];
            for (int i = 0; i < k1; ++i) a = fma(-h[i], V[(int64_t)i * n + e], a);
            w[e] = a;
        }
        wsl[threadIdx.x] = a;
    }
    __syncthreads();
    if (Pdots) {
        const int64_t e0 = r0 + lane, e1 = r0 + lane + 32;
        for (int i = warp; i < k1; i += 8) {
            const double* v = V + (int64_t)i * n;
            double a = 0.0;
            if (e0 < n) a = v[e0] * wsl[lane];
            if (e1 < n) a = fma(v[e1], wsl[lane + 32], a);
            a = warp_sum(a);
            if (lane == 0) Pdots[(int64_t)s * k1 + i] = a;
        }
    } else if (warp == 0) {
        double a = fma(wsl[lane], wsl[lane], wsl[lane + 32] * wsl[lane + 32]);
        a = warp_sum(a);
        if (lane == 0) Pnorm[s] = a;
    }
}

// ||w|| from the partial norms; v_{k+1} = w / ||w|| (and its binary32 copy when vnext32 is
// given).  Block 0 forms column k of H (h1 + h2, ||w||), applies the previous Givens
// rotations, forms rotation k, updates g and stores |g_{k+1}| in small[0].
// Graph loops: with kdev (= &gs->k), k comes from the device and v_{k+1} goes to
// vnext + (k + 1) n; with loop_set, block 0 sets the loop's condition to "not ended".
__global__ void __launch_bounds__(256) k_arn_finish(const double* __restrict__ w, int64_t n,
                                                    const double* __restrict__ Pn, int S, int k,
                                                    const double* __restrict__ h1, const double* __restrict__ h2,
                                                    double* H, int ldh, double* cs, double* sn, double* g,
                                                    double* small, double* __restrict__ vnext,
                                                    float* __restrict__ vnext32, gmres_dev* gs = nullptr,
                                                    int m_max = 0, const int* kdev = nullptr,
                                                    cudaGraphConditionalHandle loop = 0, int loop_set = 0) {
    if (gs && gs->skip) return;
    if (kdev) {
        k = *kdev;
        vnext += (int64_t)(k + 1) * n;
    }
    __shared__ double nrm;
    if (threadIdx.x < 32) {
        double a = 0.0;
        for (int q = threadIdx.x; q < S; q += 32) a += Pn[q];
        a = warp_sum(a);
        if (threadIdx.x == 0) nrm = sqrt(a);
    }
    __syncthreads();
    const double s = nrm;
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * ARN_ROWS;
    if (threadIdx.x < ARN_ROWS) {
        const int64_t e = r0 + threadIdx.x;
        if (e < n) {
            const double v = w[e] * inv;
            vnext[e] = v;
            if (vnext32) vnext32[e] = (float)v;
        }
    }
    // Column k is formed by block 0 when k is a launch argument; with the device-side state
    // (gs) by the last block to arrive: every block has read gs->k and gs->skip before it
    // counts its arrival, so the update of both cannot reach a block that has not started.
    if (gs) {
        __shared__ int last;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(&gs->arrive, 1) == (int)gridDim.x - 1;
        }
        __syncthreads();
        if (!last) return;
        if (threadIdx.x == 0) gs->arrive = 0;
    } else if (blockIdx.x != 0) {
        return;
    }
    // column k and the previous rotations staged in shared memory, then one thread rotates
    extern __shared__ double gsh[];      // col[k + 2], cs[k], sn[k]
    double* col = gsh;
    double* c_s = gsh + k + 2;
    double* s_s = c_s + k;
    for (int i = threadIdx.x; i <= k; i += blockDim.x) col[i] = h1[i] + h2[i];
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        c_s[i] = cs[i];
        s_s[i] = sn[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        col[k + 1] = s;
        for (int i = 0; i < k; ++i) {
            const double t = c_s[i] * col[i] + s_s[i] * col[i + 1];
            col[i + 1] = -s_s[i] * col[i] + c_s[i] * col[i + 1];
            col[i] = t;
        }
        const double a = col[k], b = col[k + 1];
        const double den = hypot(a, b);
        const double c = den > 0 ? a / den : 1.0, sv = den > 0 ? b / den : 0.0;
        cs[k] = c;
        sn[k] = sv;
        col[k] = den;
        col[k + 1] = 0.0;
        const double gk = g[k];
        g[k + 1] = -sv * gk;
        g[k] = c * gk;
        small[0] = fabs(-sv * gk);
        if (gs) {   // sync-free schedule: iteration count and the end of this sweep's Arnoldi process
            gs->k = k + 1;
            gs->total += 1;
            if (fabs(sv * gk) <= gs->target || k + 1 >= m_max || den == 0.0) gs->skip = 1;
            if (loop_set) cudaGraphSetConditional(loop, gs->skip ? 0u : 1u);
        }
    }
    __syncthreads();
    double* hc = H + (int64_t)k * ldh;
    for (int i = threadIdx.x; i <= k + 1; i += blockDim.x) hc[i] = col[i];
}

// r = b - r (in place on r), v0 = r / ||r|| later
__global__ void k_sub_from(const double* __restrict__ b, double* r, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        r[e] = b[e] - r[e];
}

__global__ void k_scale_into(const double* __restrict__ r, const double* __restrict__ nrm, double* v, double* g,
                             int64_t n) {
    const double s = *nrm;
    const double inv = s > 0 ? 1.0 / s : 0.0;
    int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e0 == 0) g[0] = s;
    for (int64_t e = e0; e < n; e += (int64_t)gridDim.x * blockDim.x) v[e] = r[e] * inv;
}

__global__ void k_axpy(double a, const double* __restrict__ x, double* y, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = fma(a, x[e], y[e]);
}

// ---------------- classification of off-surface targets ----------------

// One warp per target.  For every curve: nearest node (smallest index on ties); if it is
// closer than 12 h*, Newton projection on the trigonometric interpolant giving the foot
// t*, distance d and side; otherwise the side from the trapezoid Laplace double layer of
// unit density (1 inside the outer curve, -1 inside a hole).
__global__ void k_classify(const double* __restrict__ pts, int64_t npts, const double* __restrict__ geo,
                           const double* __restrict__ coef, const int32_t* __restrict__ nn,
                           const int32_t* __restrict__ off, int ncurves, int32_t* region, uint32_t* fine,
                           int32_t* line_curve, double* line_data) {
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= npts) return;
    const double px = pts[2 * t], py = pts[2 * t + 1];
    int reg = -1;
    uint32_t mask = 0;
    int lc = -1;
    double ld[4] = {0, 0, 0, 0};
    double lbest = 1e300;
    for (int k = 0; k < ncurves; ++k) {
        const int N = nn[k];
        const int o = off[k];
        const double h = 2.0 * MH_PI / N;
        double best = 1e300;
        int bi = 0x7fffffff;
        for (int i = lane; i < N; i += 32) {
            const double* g = geo + 8 * (int64_t)(o + i);
            double dx = g[0] - px, dy = g[1] - py;
            double d2 = dx * dx + dy * dy;
            if (d2 < best || (d2 == best && i < bi)) {
                best = d2;
                bi = i;
            }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, s);
            int oi = __shfl_xor_sync(0xffffffffu, bi, s);
            if (ob < best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        const double hstar = geo[8 * (int64_t)(o + bi) + 6] * h;
        bool outside;
        if (sqrt(best) < NEAR_NODE * hstar) {
            const double* c = coef + 4 * coef_base(off, k);
            double tt = bi * h;
            double v[6];
            for (int it = 0; it < 30; ++it) {
                curve_eval_warp(c, N, tt, v);
                double rx = v[0] - px, ry = v[1] - py;
                double gr = rx * v[2] + ry * v[3];
                double hs = v[2] * v[2] + v[3] * v[3] + rx * v[4] + ry * v[5];
                if (hs <= 0) hs = v[2] * v[2] + v[3] * v[3];
                double dt = gr / hs;
                tt -= dt;
                if (fabs(dt) < 1e-15) break;
            }
            tt = fmod(tt, 2.0 * MH_PI);
            if (tt < 0) tt += 2.0 * MH_PI;
            curve_eval_warp(c, N, tt, v);
            double spd = sqrt(v[2] * v[2] + v[3] * v[3]);
            double nx = v[3] / spd, ny = -v[2] / spd;
            double rx = px - v[0], ry = py - v[1];
            double d = sqrt(rx * rx + ry * ry);
            double side = rx * nx + ry * ny;
            double hs = spd * h;
            outside = side >= 0.0;
            if (d < NEAR_FINE * hs) mask |= 1u << k;
            if (d < NEAR_LINE * hs && d < lbest) {
                lbest = d;
                lc = k;
                ld[0] = tt;
                ld[1] = d;
                ld[2] = hs;
            }
        } else {
            double acc = 0.0;
            for (int i = lane; i < N; i += 32) {
                const double* g = geo + 8 * (int64_t)(o + i);
                double dx = g[0] - px, dy = g[1] - py;
                double sp = g[6];
                acc += (dx * g[3] / sp - dy * g[2] / sp) / (dx * dx + dy * dy) * sp * h;
            }
            acc = warp_sum(acc) / (2.0 * MH_PI);
            outside = (k == 0) ? (acc < 0.5) : (acc < -0.5);
        }
        if (outside && reg == -1) reg = k;
    }
    if (lane == 0) {
        region[t] = reg;
        fine[t] = mask;
        line_curve[t] = lc;
        for (int i = 0; i < 4; ++i) line_data[4 * t + i] = ld[i];
    }
}

// Foot point and inward normal of each line target, then the 4 auxiliary points
// y* - m (h_s/4) n*, m = 1..4.
__global__ void k_line_aux(const int32_t* __restrict__ line_tgt, const int32_t* __restrict__ line_curve,
                           const double* __restrict__ line_data, int64_t nline, const double* __restrict__ coef,
                           const int32_t* __restrict__ nn, const int32_t* __restrict__ off, int64_t n_user,
                           double* ext_xy) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= nline) return;
    const int k = line_curve[t];
    double v[6];
    curve_eval_warp(coef + 4 * coef_base(off, k), nn[k], line_data[4 * t], v);
    if ((threadIdx.x & 31) == 0) {
        double spd = sqrt(v[2] * v[2] + v[3] * v[3]);
        double nx = v[3] / spd, ny = -v[2] / spd;
        double hs = line_data[4 * t + 2];
        for (int m = 1; m <= 4; ++m) {
            double dm = m * NEAR_LINE * hs;
            int64_t e = n_user + 4 * t + (m - 1);
            ext_xy[2 * e] = v[0] - dm * nx;
            ext_xy[2 * e + 1] = v[1] - dm * ny;
        }
    }
}

// ---------------- off-surface evaluation ----------------

// Fourier coefficients of a scalar density per curve: 2 doubles per mode.  One block per
// mode, threads over the nodes, exact twiddles from the per-curve table
// tw[off + r] = (cos, sin)(2 pi r / N).
__global__ void k_fourier_scalar(const double* __restrict__ v, const int32_t* __restrict__ nn,
                                 const int32_t* __restrict__ off, const double2* __restrict__ tw, int ncurves,
                                 int64_t total, double* coef) {
    const int64_t g = blockIdx.x;
    if (g >= total) return;
    int k = 0;
    while (k + 1 < ncurves && g >= coef_base(off, k + 1)) ++k;
    const int N = nn[k];
    const int m = (int)(g - coef_base(off, k));
    const double* p = v + off[k];
    const double2* t = tw + off[k];
    double re = 0, im = 0;
    const int step = (int)(((int64_t)m * blockDim.x) % N);   // twiddle index m n mod N, advanced per stride
    int r = (int)(((int64_t)m * threadIdx.x) % N);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const double2 c = t[r];
        re = fma(p[n], c.x, re);
        im = fma(-p[n], c.y, im);
        r += step;
        if (r >= N) r -= N;
    }
    re = block_sum<128>(re);
    im = block_sum<128>(im);
    if (threadIdx.x == 0) {
        coef[2 * g] = re / N;
        coef[2 * g + 1] = im / N;
    }
}

// The same coefficients for the binary32 path: density and twiddles in binary32, every product
// accumulated in float-float (TwoSum), so that the sums carry no binary64 instruction per term
// (the binary64 pipe runs at 1/64 of the binary32 rate here) and lose nothing to the length N.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float v) {
    const float t = hi + v;
    const float bb = t - hi;
    lo += (hi - (t - bb)) + (v - bb);
    hi = t;
}

__global__ void k_fourier_scalar32(const float* __restrict__ v, const int32_t* __restrict__ nn,
                                   const int32_t* __restrict__ off, const float2* __restrict__ tw, int ncurves,
                                   int64_t total, double* coef) {
    const int64_t g = blockIdx.x;
    if (g >= total) return;
    int k = 0;
    while (k + 1 < ncurves && g >= coef_base(off, k + 1)) ++k;
    const int N = nn[k];
    const int m = (int)(g - coef_base(off, k));
    const float* p = v + off[k];
    const float2* t = tw + off[k];
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const int step = (int)(((int64_t)m * blockDim.x) % N);
    int r = (int)(((int64_t)m * threadIdx.x) % N);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const float2 c = t[r];
        ff_add(rh, rl, p[n] * c.x);
        ff_add(ih, il, -p[n] * c.y);
        r += step;
        if (r >= N) r -= N;
    }
    // block reduction in float-float, lanes then warps in a fixed order
    __shared__ float red[4][32];
    for (int o = 16; o > 0; o >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, rh, o), b = __shfl_xor_sync(0xffffffffu, rl, o);
        const float c = __shfl_xor_sync(0xffffffffu, ih, o), d = __shfl_xor_sync(0xffffffffu, il, o);
        ff_add(rh, rl, a);
        rl += b;
        ff_add(ih, il, c);
        il += d;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = rh;
        red[1][warp] = rl;
        red[2][warp] = ih;
        red[3][warp] = il;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double re = 0.0, im = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            re += (double)red[0][w] + (double)red[1][w];
            im += (double)red[2][w] + (double)red[3][w];
        }
        coef[2 * g] = re / N;
        coef[2 * g + 1] = im / N;
    }
}

__global__ void k_twiddles(const int32_t* __restrict__ nn, const int32_t* __restrict__ off,
                           const int32_t* __restrict__ curve_of, int64_t n, double2* tw, double2* half) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int k = curve_of[j];
    const int r = (int)(j - off[k]);
    double s, c;
    sincospi(2.0 * r / nn[k], &s, &c);
    tw[j] = make_double2(c, s);
    sincospi((double)r / nn[k], &s, &c);   // (cos, sin)(t_r / 2)
    half[j] = make_double2(c, s);
}

// Fine-grid (16x) density by sub-offset: with f = 16 j + s,
//   p(t_f) = sum_m C_m^{(s)} e^{2 pi i m j / N},  C_m^{(s)} = w_m c_m e^{2 pi i m s / (16 N)}
// (w_0 = 1, w_m = 2 for 0 < m < N/2, the Nyquist term real with w = 1), real part.
// k_fine_coef writes C[(base_k + m) * 16 + s] with exact binary64 phases.
template <typename T2>
__global__ void k_fine_coef(const double* __restrict__ sc, const int32_t* __restrict__ nn,
                            const int32_t* __restrict__ off, int ncurves, int64_t nmodes, T2* __restrict__ cp) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nmodes * UPSAMPLE) return;
    const int64_t g = e / UPSAMPLE;
    const int sub = (int)(e - g * UPSAMPLE);
    int k = 0;
    while (k + 1 < ncurves && g >= coef_base(off, k + 1)) ++k;
    const int N = nn[k];
    const int m = (int)(g - coef_base(off, k));
    double re = sc[2 * g], im = sc[2 * g + 1];
    if (2 * m == N) im = 0.0;
    const double w = (m == 0 || 2 * m == N) ? 1.0 : 2.0;
    double sn, cs;
    sincospi(2.0 * (double)(m * sub) / (double)(UPSAMPLE * N), &sn, &cs);
    T2 out;
    out.x = w * (re * cs - im * sn);
    out.y = w * (re * sn + im * cs);
    cp[e] = out;
}

// Block = (16 coarse indices j of curve blockIdx.y) x (16 sub-offsets s); the coarse twiddles
// e^{2 pi i r / N} sit in shared memory (a warp reads two of them per mode: broadcast), the
// coefficients C_m^{(s)} are read as 16 consecutive complex values per mode (coalesced).
template <typename T, typename T2>
__global__ void __launch_bounds__(256) k_fine_density_s(const T2* __restrict__ cp, const T2* __restrict__ tw,
                                                        const double* __restrict__ fg, const int32_t* __restrict__ nn,
                                                        const int32_t* __restrict__ off,
                                                        const int64_t* __restrict__ foff, T* __restrict__ wf) {
    extern __shared__ unsigned char smem_raw[];
    T2* tn = reinterpret_cast<T2*>(smem_raw);
    const int k = blockIdx.y;
    const int N = nn[k];
    const int j0 = blockIdx.x * 16;
    if (j0 >= N) return;
    for (int r = threadIdx.x; r < N; r += blockDim.x) tn[r] = tw[off[k] + r];   // twiddles in T already
    __syncthreads();
    const int sub = threadIdx.x & 15, j = j0 + (threadIdx.x >> 4);
    if (j >= N) return;
    const T2* c = cp + coef_base(off, k) * UPSAMPLE + sub;
    T acc = 0;
    int r = 0;
#pragma unroll 8
    for (int m = 0; m <= N / 2; ++m) {
        const T2 a = __ldg(c + (int64_t)m * UPSAMPLE);
        const T2 t = tn[r];
        acc = fma(a.x, t.x, acc);
        acc = fma(-a.y, t.y, acc);
        r += j;
        if (r >= N) r -= N;
    }
    const int64_t g = foff[k] + (int64_t)UPSAMPLE * j + sub;
    wf[g] = (T)((double)acc * fg[6 * g + 4] * fg[6 * g + 5]);
}

// The same fine-grid density by inverse FFT, for curves of N = 2^L <= FFT_MAX nodes: block
// (s, k) forms p(t_{16 j + s}) = Re sum_{m <= N/2} C_m^{(s)} e^{2 pi i m j / N} for every j of
// curve k by one radix-2 decimation-in-time transform of length N in shared memory (input in
// bit-reversed order, twiddles e^{2 pi i r / N} from the curve's binary32 table staged beside
// it), then multiplies by |y'| h_f as k_fine_density_s does.  N log2 N / 2 butterflies per
// sub-offset instead of N (N/2 + 1) products; rounding ~log2 N units of binary32 against ~sqrt N
// for the direct sum.
constexpr int FFT_MAX = 2048;

__global__ void __launch_bounds__(256) k_fine_density_fft(const float2* __restrict__ cp, const float2* __restrict__ tw,
                                                          const double* __restrict__ fg, const int32_t* __restrict__ nn,
                                                          const int32_t* __restrict__ off,
                                                          const int64_t* __restrict__ foff, float* __restrict__ wf) {
    extern __shared__ float2 fz[];   // [N] values, then [N] twiddles
    const int s = blockIdx.x, k = blockIdx.y;
    const int N = nn[k];
    float2* z = fz;
    float2* w = fz + N;
    const int L = __ffs(N) - 1;   // N = 2^L
    const float2* c = cp + coef_base(off, k) * UPSAMPLE + s;
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        z[__brev((unsigned)m) >> (32 - L)] = m <= N / 2 ? c[(int64_t)m * UPSAMPLE] : make_float2(0.f, 0.f);
        w[m] = tw[off[k] + m];
    }
    __syncthreads();
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1, step = N / len;
        for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const int pos = b & (half - 1), i = (b - pos) * 2 + pos;   // (group b / half) * len + pos
            const float2 t = w[pos * step];
            const float2 u = z[i], v = z[i + half];
            const float2 vt = make_float2(v.x * t.x - v.y * t.y, v.x * t.y + v.y * t.x);
            z[i] = make_float2(u.x + vt.x, u.y + vt.y);
            z[i + half] = make_float2(u.x - vt.x, u.y - vt.y);
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int64_t g = foff[k] + (int64_t)UPSAMPLE * j + s;
        wf[g] = (float)((double)z[j].x * fg[6 * g + 4] * fg[6 * g + 5]);
    }
}

// The density times |y'| h_f on the 16x grid straight from the density, for curves of
// N = 2^L <= FFT_MAX nodes, in one launch: block (s, k) takes curve k's density to binary32,
// forms c_m = (1/N) sum_j sigma_j e^{-2 pi i m j / N} by a radix-2 forward FFT in shared memory
// (the conjugate twiddles; each of the UPSAMPLE blocks of a curve repeats this small transform),
// multiplies in its own sub-offset's phases, C_m^{(s)} = w_m c_m e^{2 pi i m s / (16 N)} (m <= N/2;
// w_0 = 1, w_m = 2, the Nyquist term real with w = 1; the phases by sincospif), and finishes as
// k_fine_density_fft does (the inverse transform, the real part times |y'| h_f into wf and its
// binary64 image wf64).
__global__ void __launch_bounds__(256) k_fine_weights_fft(const double* __restrict__ sigma, const float2* __restrict__ tw,
                                                          const double* __restrict__ fg, const int32_t* __restrict__ nn,
                                                          const int32_t* __restrict__ off,
                                                          const int64_t* __restrict__ foff, float* __restrict__ wf,
                                                          double* __restrict__ wf64) {
    extern __shared__ float2 fz[];   // [N] values, then [N] twiddles
    constexpr int PER = FFT_MAX / 256;   // values per thread when the spectrum is reordered
    const int s = blockIdx.x, k = blockIdx.y;
    const int N = nn[k];
    float2* z = fz;
    float2* w = fz + N;
    const int L = __ffs(N) - 1;   // N = 2^L
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        z[__brev((unsigned)m) >> (32 - L)] = make_float2((float)sigma[off[k] + m], 0.f);
        w[m] = tw[off[k] + m];
    }
    __syncthreads();
    // forward transform (decimation in time, conjugate twiddles): z[m] = N c_m
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1, step = N / len;
        for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const int pos = b & (half - 1), i = (b - pos) * 2 + pos;
            const float2 t = w[pos * step];
            const float2 u = z[i], v = z[i + half];
            const float2 vt = make_float2(v.x * t.x + v.y * t.y, v.y * t.x - v.x * t.y);
            z[i] = make_float2(u.x + vt.x, u.y + vt.y);
            z[i + half] = make_float2(u.x - vt.x, u.y - vt.y);
        }
        __syncthreads();
    }
    // this sub-offset's coefficients, then back into bit-reversed order for the inverse
    float2 cm[PER];
    const float invN = 1.f / (float)N;   // a power of two: exact
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int m = threadIdx.x + 256 * q;
        cm[q] = make_float2(0.f, 0.f);
        if (m < N && 2 * m <= N) {
            const float re = z[m].x * invN, im = 2 * m == N ? 0.f : z[m].y * invN;
            const float wm = (m == 0 || 2 * m == N) ? 1.f : 2.f;
            float sn, cs;
            sincospif((float)(2 * m * s) / (float)(UPSAMPLE * N), &sn, &cs);
            cm[q] = make_float2(wm * (re * cs - im * sn), wm * (re * sn + im * cs));
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int m = threadIdx.x + 256 * q;
        if (m < N) z[__brev((unsigned)m) >> (32 - L)] = cm[q];
    }
    __syncthreads();
    // inverse transform: z[j] = sum_m C_m e^{2 pi i m j / N}
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1, step = N / len;
        for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const int pos = b & (half - 1), i = (b - pos) * 2 + pos;
            const float2 t = w[pos * step];
            const float2 u = z[i], v = z[i + half];
            const float2 vt = make_float2(v.x * t.x - v.y * t.y, v.x * t.y + v.y * t.x);
            z[i] = make_float2(u.x + vt.x, u.y + vt.y);
            z[i + half] = make_float2(u.x - vt.x, u.y - vt.y);
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int64_t g = foff[k] + (int64_t)UPSAMPLE * j + s;
        const float v = (float)((double)z[j].x * fg[6 * g + 4] * fg[6 * g + 5]);
        wf[g] = v;
        wf64[g] = (double)v;   // the binary64 image the dipole weights are taken from
    }
}

// Coarse trapezoid sum over all curves not flagged fine for the target:
//   out[t] = -(1/(2 pi alpha^2)) sum_n K(y_n, x_t) sigma_n |y'_n| h
// Sources are staged through shared memory in tiles of the block size.
template <int BS>
__global__ void k_dlp_coarse(const double* __restrict__ xy, const uint32_t* __restrict__ fine, int64_t nt,
                             const double* __restrict__ geo, const double* __restrict__ sigma,
                             const int32_t* __restrict__ curve_of, const int32_t* __restrict__ nn, int64_t ns,
                             double inv_alpha, double pref, double* out) {
    __shared__ double sx[BS], sy[BS], snx[BS], sny[BS], sw[BS];
    __shared__ int sk[BS];
    const int64_t t = blockIdx.x * (int64_t)BS + threadIdx.x;
    const bool active = t < nt;
    const double px = active ? xy[2 * t] : 0.0, py = active ? xy[2 * t + 1] : 0.0;
    const uint32_t mask = active ? fine[t] : 0xffffffffu;
    double acc = 0.0;
    // gridDim.y > 1 splits the sources between blocks (partials without the prefactor)
    const int64_t ntile = (ns + BS - 1) / BS, per = (ntile + gridDim.y - 1) / gridDim.y;
    const int64_t sbeg = blockIdx.y * per * BS, send = min(ns, (blockIdx.y + 1) * per * BS);
    for (int64_t s0 = sbeg; s0 < send; s0 += BS) {
        int64_t s = s0 + threadIdx.x;
        if (s < ns) {
            const double* g = geo + 8 * s;
            int k = curve_of[s];
            double sp = g[6];
            sx[threadIdx.x] = g[0];
            sy[threadIdx.x] = g[1];
            snx[threadIdx.x] = g[3] / sp;
            sny[threadIdx.x] = -g[2] / sp;
            sw[threadIdx.x] = sigma[s] * sp * (2.0 * MH_PI / nn[k]);
            sk[threadIdx.x] = k;
        }
        __syncthreads();
        const int cnt = (ns - s0) < BS ? (int)(ns - s0) : BS;
        if (active) {
            for (int i = 0; i < cnt; ++i) {
                if (mask & (1u << sk[i])) continue;
                acc += dl_kernel(sx[i], sy[i], snx[i], sny[i], px, py, inv_alpha) * sw[i];
            }
        }
        __syncthreads();
    }
    if (active) {
        if (gridDim.y == 1)
            out[t] = pref * acc;
        else
            out[blockIdx.y * nt + t] = acc;
    }
}

// Upsampled rule for (target, curve) pairs: one warp per pair.
__global__ void k_dlp_fine(const double* __restrict__ xy, const int32_t* __restrict__ ptgt,
                           const int32_t* __restrict__ pcurve, int64_t npairs, const double* __restrict__ fg,
                           const double* __restrict__ wf, const int64_t* __restrict__ foff, double inv_alpha,
                           double pref, double* out) {
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= npairs) return;
    const int lane = threadIdx.x & 31;
    const int64_t t = ptgt[p];
    const int k = pcurve[p];
    const double px = xy[2 * t], py = xy[2 * t + 1];
    double acc = 0.0;
    for (int64_t f = foff[k] + lane; f < foff[k + 1]; f += 32) {
        const double* g = fg + 6 * f;
        acc += dl_kernel(g[0], g[1], g[2], g[3], px, py, inv_alpha) * wf[f];
    }
    acc = warp_sum(acc);
    if (lane == 0) atomicAdd(out + t, pref * acc);
}

// Near-boundary correction for targets whose trapezoid sum came from the multipole
// method: upsampled sum over curve k minus the trapezoid sum over the nodes of curve k.
__global__ void k_dlp_fine_corr(const double* __restrict__ xy, const int32_t* __restrict__ ptgt,
                                const int32_t* __restrict__ pcurve, int64_t npairs, const double* __restrict__ fg,
                                const double* __restrict__ wf, const int64_t* __restrict__ foff,
                                const double* __restrict__ geo, const double* __restrict__ sigma,
                                const int32_t* __restrict__ nn, const int32_t* __restrict__ off, double inv_alpha,
                                double pref, double* out) {
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= npairs) return;
    const int lane = threadIdx.x & 31;
    const int64_t t = ptgt[p];
    const int k = pcurve[p];
    const double px = xy[2 * t], py = xy[2 * t + 1];
    double acc = 0.0;
    for (int64_t f = foff[k] + lane; f < foff[k + 1]; f += 32) {
        const double* g = fg + 6 * f;
        acc += dl_kernel(g[0], g[1], g[2], g[3], px, py, inv_alpha) * wf[f];
    }
    const double h = 2.0 * MH_PI / nn[k];
    for (int64_t s = off[k] + lane; s < off[k + 1]; s += 32) {
        const double* g = geo + 8 * s;
        const double sp = g[6];
        acc -= dl_kernel(g[0], g[1], g[3] / sp, -g[2] / sp, px, py, inv_alpha) * sigma[s] * sp * h;
    }
    acc = warp_sum(acc);
    if (lane == 0) out[t] += pref * acc;
}

__global__ void k_dlp_fine_corr32(const double* __restrict__ xy, const int32_t* __restrict__ ptgt,
                                  const int32_t* __restrict__ pcurve, int64_t npairs,
                                  const float4* __restrict__ fine32, const float* __restrict__ wf,
                                  const int64_t* __restrict__ foff, const int64_t* __restrict__ coff,
                                  const double2* __restrict__ cc, const float4* __restrict__ src32,
                                  const float* __restrict__ w32, const double2* __restrict__ tc,
                                  const int32_t* __restrict__ off, mh_dl32 c32, double pref, double* out) {
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= npairs) return;
    const int lane = threadIdx.x & 31;
    const int64_t t = ptgt[p];
    const int k = pcurve[p];
    const double px = xy[2 * t], py = xy[2 * t + 1];
    double acc = 0.0;
    for (int64_t ch = coff[k]; ch < coff[k + 1]; ++ch) {
        const double2 c = cc[ch];
        const float tx = (float)(px - c.x), ty = (float)(py - c.y);
        const int64_t f0 = foff[k] + (ch - coff[k]) * MH_TILE;
        const int64_t f1 = min(f0 + MH_TILE, foff[k + 1]);
        float part = 0.f;
        for (int64_t f = f0 + lane; f < f1; f += 32) {
            const float4 v = fine32[f];
            part += mh_dl32_pair(v.x - tx, v.y - ty, v.z, v.w, c32) * wf[f];
        }
        acc += (double)part;
    }
    // trapezoid nodes of curve k, offsets from their tile centres
    for (int64_t tile = off[k] / MH_TILE; tile * MH_TILE < off[k + 1]; ++tile) {
        const double2 c = tc[tile];
        const float tx = (float)(px - c.x), ty = (float)(py - c.y);
        const int64_t s0 = max((int64_t)off[k], tile * MH_TILE), s1 = min((int64_t)off[k + 1], (tile + 1) * MH_TILE);
        float part = 0.f;
        for (int64_t s = s0 + lane; s < s1; s += 32) {
            const float4 v = src32[s];
            part += mh_dl32_pair(v.x - tx, v.y - ty, v.z, v.w, c32) * w32[s];
        }
        acc -= (double)part;
    }
    acc = warp_sum(acc);
    if (lane == 0) out[t] += pref * acc;
}

// Normal-line rule: degree-4 interpolation in the distance through the interior limit
// v0 = -(A sigma)(t*) / (2 alpha^2) (trigonometric interpolation of the on-surface
// values) and the values at the 4 auxiliary points.
// The interpolation weights D_N(t* - t_i) depend on the target alone and are formed once
// (k_line_weights): D_N(t* - t_i) = sin(N (t* - t_i)/2) cot((t* - t_i)/2) / N, written about
// the nearest node j, t* = t_j + delta (|delta| <= h/2):
//   sin(N (t* - t_i)/2) = (-1)^(j-i) sin(N delta/2)        (a small argument),
//   (t* - t_i)/2 = delta/2 + (j-i) h/2                      (angle addition with the exact
//                                                            half-angle table, i != j).
// A target whose foot point lies on (or within rounding of) a node keeps full relative accuracy
// in its own weight, which tends to 1 there; a closed form through sin(N t*/2) of the large
// argument and the half-angle difference of t* and t_j loses it to cancellation.
__global__ void k_line_weights(const int32_t* __restrict__ line_curve, const double* __restrict__ line_data,
                               int64_t nline, const int32_t* __restrict__ nn, const int32_t* __restrict__ off,
                               const double2* __restrict__ half, const int64_t* __restrict__ woff, double* w) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= nline) return;
    const int lane = threadIdx.x & 31;
    const int k = line_curve[t];
    const int N = nn[k];
    const double ts = line_data[4 * t];   // in [0, 2 pi)
    const double2* hf = half + off[k];    // (cos, sin)(t_m / 2), m = 0..N-1
    const double h = 2.0 * MH_PI / N;
    int j = (int)rint(ts / h);            // 0..N
    const double delta = ts - j * h;
    if (j >= N) j -= N;
    const double sNd = sin(0.5 * N * delta);
    double sd, cd;
    sincos(0.5 * delta, &sd, &cd);
    for (int i = lane; i < N; i += 32) {
        const int m = j - i;
        double sh, ch;   // sin, cos of (t* - t_i) / 2
        if (m == 0) {
            sh = sd;
            ch = cd;
        } else {
            const int am = m > 0 ? m : -m;
            const double cm = hf[am].x, sm = m > 0 ? hf[am].y : -hf[am].y;
            sh = sd * cm + cd * sm;
            ch = cd * cm - sd * sm;
        }
        const double sg = (m & 1) ? -sNd : sNd;
        w[woff[t] + i] = fabs(sh) < 1e-300 ? 1.0 : sg * ch / sh / N;
    }
}

__global__ void k_dlp_line(const int32_t* __restrict__ line_tgt, const int32_t* __restrict__ line_curve,
                           const double* __restrict__ line_data, int64_t nline, const double* __restrict__ asig,
                           const int32_t* __restrict__ nn, const int32_t* __restrict__ off,
                           const double* __restrict__ lw, const int64_t* __restrict__ woff, int64_t n_user,
                           double alpha, double* out) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= nline) return;
    const int lane = threadIdx.x & 31;
    const int k = line_curve[t];
    const int N = nn[k];
    const double* a = asig + off[k];
    const double* w = lw + woff[t];
    double acc = 0.0;
    for (int i = lane; i < N; i += 32) acc += w[i] * a[i];
    acc = warp_sum(acc);
    if (lane == 0) {
        double vals[5], dist[5];
        vals[0] = -acc / (2.0 * alpha * alpha);
        dist[0] = 0.0;
        double hs = line_data[4 * t + 2];
        for (int m = 1; m <= 4; ++m) {
            dist[m] = m * NEAR_LINE * hs;
            vals[m] = out[n_user + 4 * t + (m - 1)];
        }
        double d = line_data[4 * t + 1];
        double r = 0.0;
        for (int i = 0; i < 5; ++i) {
            double wi = 1.0;
            for (int j = 0; j < 5; ++j)
                if (j != i) wi *= (d - dist[j]) / (dist[i] - dist[j]);
            r += wi * vals[i];
        }
        out[line_tgt[t]] = r;
    }
}

}  // namespace


// ---- matrix-free operator (Section 3.2 without the dense matrix) ----
//
// Row j of the discrete system is sigma_j + (1/pi) [T_j - W_j] + C_j with
//   T_j = sum_{i != j} K(y_i, x_j) |y'_i| h sigma_i        (all curves: the multipole pass)
//   W_j = the terms of T_j inside the own-curve Alpert window 0 < |i - j| < a (direct)
//   C_j = sum_p cp[j][p] sigma~(t_j + s_p x_m h)           (Alpert nodes, p = (s, m))
// where sigma~ is the trigonometric interpolant of the curve's density (the periodic kernel
// D_N of the dense assembly).  sigma~ at the 2l shifted grids comes from the spectrum
// c_m = (1/N) sum_n sigma_n e^{-2 pi i m n / N}:
//   sigma~(t_j + d) = Re sum_{m <= N/2} w_m c_m e^{i m d} e^{2 pi i m j / N}
// (w_0 = 1, w_m = 2, the Nyquist term with w = 1), one length-N transform per shift.  N_k is
// any even count: a power of two takes radix-2 transforms of length M_k = N_k directly, any other
// count Bluestein chirp transforms, b_n = e^{i pi n^2/N},
//   X_k = sum_n x_n e^{-2 pi i n k/N} = conj(b_k) sum_n (x_n conj(b_n)) b_{k-n},
// the cyclic convolution done at length M_k = 2^L >= 2N - 1 by two radix-2 transforms in shared
// memory and the transform of the chirp filter computed once (so M_k == N_k marks the direct
// form).  All binary64.

// Alpert node weights of row j (the first half of k_assemble_alpert, kept per row):
// cp[j][p] = (1/pi) h w_m |y'(t)| K(y(t), x_j) at t = t_j + s x_m h, s = +1 (p < l) or -1.
__global__ void k_alpert_weights(const double* __restrict__ geo, const double* __restrict__ coef,
                                 const int32_t* __restrict__ curve_of, const int32_t* __restrict__ nn,
                                 const int32_t* __restrict__ off, double inv_alpha, AlpertRule R,
                                 double* __restrict__ cp) {
    const int64_t j = blockIdx.x;
    const int k = curve_of[j];
    const int N = nn[k];
    const int jj = (int)(j - off[k]);
    const double h = 2.0 * MH_PI / N;
    const double* c = coef + 4 * coef_base(off, k);
    const double* gj = geo + 8 * j;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = warp; p < 2 * R.l; p += nw) {
        const int m = p % R.l;
        const double s = p < R.l ? 1.0 : -1.0;
        double v[6];
        curve_eval_warp(c, N, (jj + s * R.x[m]) * h, v);
        if ((threadIdx.x & 31) == 0) {
            const double spd = sqrt(v[2] * v[2] + v[3] * v[3]);
            const double K = dl_kernel(v[0], v[1], v[3] / spd, -v[2] / spd, gj[0], gj[1], inv_alpha);
            cp[j * 2 * R.l + p] = (1.0 / MH_PI) * h * R.w[m] * spd * K;
        }
    }
}

// Own-curve node of window term t of row j: offset d = t/2 + 1 backwards (t even) or forwards.
__device__ __forceinline__ int mf_win_node(int jj, int t, int N) {
    const int d = t / 2 + 1;
    int ii = (jj + ((t & 1) ? d : -d)) % N;
    return ii < 0 ? ii + N : ii;
}

// Window weights of row j: win[j][t] = (1/pi) K(y_i, x_j) |y'_i| h for the 2(a - 1) own-curve
// nodes i with 0 < |i - j| < a (the trapezoid entries the Alpert rule replaces).
__global__ void k_mf_window_weights(const double* __restrict__ geo, const int32_t* __restrict__ curve_of,
                                    const int32_t* __restrict__ nn, const int32_t* __restrict__ off, int64_t n,
                                    double inv_alpha, int nw, double* __restrict__ win) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * nw) return;
    const int64_t j = e / nw;
    const int t = (int)(e - j * nw);
    const int k = curve_of[j], N = nn[k], o = off[k];
    const double* gj = geo + 8 * j;
    const double* gi = geo + 8 * (int64_t)(o + mf_win_node((int)(j - o), t, N));
    const double sp = gi[6];
    win[e] = (1.0 / MH_PI) * dl_kernel(gi[0], gi[1], gi[3] / sp, -gi[2] / sp, gj[0], gj[1], inv_alpha) * sp *
             (2.0 * MH_PI / N);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// In-place radix-2 transform of length M = 2^L in shared memory, input in bit-reversed order:
// z_k <- sum_n z_n e^{-2 pi i n k / M}; tw[r] = e^{-2 pi i r / M} (r < M/2).
__device__ void fft64_shared(double2* z, const double2* tw, int M) {
    for (int len = 2; len <= M; len <<= 1) {
        const int half = len >> 1, step = M / len;
        for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
            const int pos = b & (half - 1), i = (b - pos) * 2 + pos;
            const double2 vt = cmul(z[i + half], tw[pos * step]);
            const double2 u = z[i];
            z[i] = make_double2(u.x + vt.x, u.y + vt.y);
            z[i + half] = make_double2(u.x - vt.x, u.y - vt.y);
        }
        __syncthreads();
    }
}

constexpr int MF_THREADS = 512;
constexpr int MF_MMAX = 8192;                       // N_k <= 4096
constexpr int MF_PER = MF_MMAX / MF_THREADS;        // entries per thread in a reordering pass

// The cyclic convolution of Bluestein's transform of length N: on entry z holds
// a_n = x_n conj(b_n) (zeros for n >= N) in bit-reversed order and bh the transform of the chirp
// filter; on return z[k] = M conj((a * b)_k), so that X_k = conj(b_k) conj(z[k]) / M for k < N
// (the inverse transform taken as the forward one of the conjugate).
__device__ void bluestein_core(double2* z, const double2* tw, const double2* __restrict__ bh, int M, int L) {
    fft64_shared(z, tw, M);
    // pointwise product with the filter's transform, conjugated (the inverse transform as a
    // forward one), back to bit-reversed order through registers
    double2 r[MF_PER];
#pragma unroll
    for (int q = 0; q < MF_PER; ++q) {
        const int i = threadIdx.x + MF_THREADS * q;
        if (i < M) r[q] = cconj(cmul(z[i], bh[i]));
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MF_PER; ++q) {
        const int i = threadIdx.x + MF_THREADS * q;
        if (i < M) z[__brev((unsigned)i) >> (32 - L)] = r[q];
    }
    __syncthreads();
    fft64_shared(z, tw, M);
}

// Per curve: the chirp b_n, the transform of the chirp filter (b_m at m and M - m) and the
// twiddles of length M_k.  Grid: one block per curve.
__global__ void __launch_bounds__(MF_THREADS) k_mf_chirp(const int32_t* __restrict__ nn, const int64_t* __restrict__ moff,
                                                         const int32_t* __restrict__ Mk, const int32_t* __restrict__ off,
                                                         double2* __restrict__ chirp, double2* __restrict__ bh,
                                                         double2* __restrict__ twg) {
    extern __shared__ double2 mfz[];
    const int k = blockIdx.x, N = nn[k], M = Mk[k];
    const int L = __ffs(M) - 1;
    double2* z = mfz;
    double2* tw = mfz + M;
    for (int r = threadIdx.x; r < M / 2; r += blockDim.x) {
        double s, c;
        sincospi(-2.0 * r / M, &s, &c);
        tw[r] = make_double2(c, s);
        twg[moff[k] / 2 + r] = tw[r];
    }
    if (M == N) return;   // a power of two: direct transforms, no chirp
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int64_t q = ((int64_t)n * n) % (2 * (int64_t)N);   // b_n = e^{i pi (n^2 mod 2N) / N}
        double s, c;
        sincospi((double)q / N, &s, &c);
        chirp[off[k] + n] = make_double2(c, s);
    }
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        int n = -1;
        if (m < N)
            n = m;
        else if (m > M - N)
            n = M - m;
        double2 v = make_double2(0.0, 0.0);
        if (n >= 0) {
            const int64_t q = ((int64_t)n * n) % (2 * (int64_t)N);
            double s, c;
            sincospi((double)q / N, &s, &c);
            v = make_double2(c, s);
        }
        z[__brev((unsigned)m) >> (32 - L)] = v;
    }
    __syncthreads();
    fft64_shared(z, tw, M);
    for (int m = threadIdx.x; m < M; m += blockDim.x) bh[moff[k] + m] = z[m];
}

// Spectrum c_m (m <= N/2) of the density of every curve.  Grid: one block per curve.
__global__ void __launch_bounds__(MF_THREADS) k_mf_spectrum(const double* __restrict__ sigma, const int32_t* __restrict__ nn,
                                                            const int32_t* __restrict__ off, const int64_t* __restrict__ moff,
                                                            const int32_t* __restrict__ Mk, const double2* __restrict__ chirp,
                                                            const double2* __restrict__ bh, const double2* __restrict__ twg,
                                                            double2* __restrict__ spec) {
    extern __shared__ double2 mfz[];
    const int k = blockIdx.x, N = nn[k], M = Mk[k];
    const int L = __ffs(M) - 1;
    double2* z = mfz;
    double2* tw = mfz + M;
    const double2* b = chirp + off[k];
    for (int r = threadIdx.x; r < M / 2; r += blockDim.x) tw[r] = twg[moff[k] / 2 + r];
    const bool direct = M == N;
    for (int n = threadIdx.x; n < M; n += blockDim.x) {
        double2 a = make_double2(0.0, 0.0);
        if (direct)
            a = make_double2(sigma[off[k] + n], 0.0);
        else if (n < N)
            a = make_double2(sigma[off[k] + n] * b[n].x, -sigma[off[k] + n] * b[n].y);
        z[__brev((unsigned)n) >> (32 - L)] = a;
    }
    __syncthreads();
    if (direct)
        fft64_shared(z, tw, M);
    else
        bluestein_core(z, tw, bh + moff[k], M, L);
    const double sc = direct ? 1.0 / N : 1.0 / ((double)M * N);
    for (int m = threadIdx.x; 2 * m <= N; m += blockDim.x) {
        const double2 X = direct ? z[m] : cmul(cconj(b[m]), cconj(z[m]));
        spec[coef_base(off, k) + m] = make_double2(X.x * sc, X.y * sc);
    }
}

// The interpolated density at the Alpert nodes of shift p = (s, m) of every node of curve k:
// S[p][off_k + j] = Re sum_{m' <= N/2} w_m' c_m' e^{i m' d} e^{2 pi i m' j / N}, d = s x_m h,
// as Re of the forward transform of conj(C) (C_m' = w_m' c_m' e^{i m' d}).  Grid (2l, curves).
__global__ void __launch_bounds__(MF_THREADS) k_mf_shift(const double2* __restrict__ spec, const int32_t* __restrict__ nn,
                                                         const int32_t* __restrict__ off, const int64_t* __restrict__ moff,
                                                         const int32_t* __restrict__ Mk, const double2* __restrict__ chirp,
                                                         const double2* __restrict__ bh, const double2* __restrict__ twg,
                                                         AlpertRule R, int64_t n, double* __restrict__ S) {
    extern __shared__ double2 mfz[];
    const int p = blockIdx.x, k = blockIdx.y, N = nn[k], M = Mk[k];
    const int L = __ffs(M) - 1;
    const double sx = (p < R.l ? 1.0 : -1.0) * R.x[p % R.l];
    const bool direct = M == N;
    double2* z = mfz;
    double2* tw = mfz + M;
    const double2* b = chirp + off[k];
    const double2* c = spec + coef_base(off, k);
    for (int r = threadIdx.x; r < M / 2; r += blockDim.x) tw[r] = twg[moff[k] / 2 + r];
    for (int mm = threadIdx.x; mm < M; mm += blockDim.x) {
        double2 a = make_double2(0.0, 0.0);
        if (2 * mm <= N) {
            const double wm = (mm == 0 || 2 * mm == N) ? 1.0 : 2.0;
            double sn, cs;
            sincospi(2.0 * mm * sx / N, &sn, &cs);   // e^{i m' d}, d = 2 pi s x_m / N
            const double2 C = cmul(c[mm], make_double2(wm * cs, wm * sn));
            a = direct ? cconj(C) : cmul(cconj(C), cconj(b[mm]));
        }
        z[__brev((unsigned)mm) >> (32 - L)] = a;
    }
    __syncthreads();
    if (direct)
        fft64_shared(z, tw, M);
    else
        bluestein_core(z, tw, bh + moff[k], M, L);
    const double sc = 1.0 / (double)M;
    for (int j = threadIdx.x; j < N; j += blockDim.x)   // Re y_j = Re X_j
        S[(int64_t)p * n + off[k] + j] = direct ? z[j].x : cmul(cconj(b[j]), cconj(z[j])).x * sc;
}

// Dipole strengths w_i = sigma_i |y'_i| h_k.
__global__ void k_mf_weights(const double* __restrict__ sigma, const double* __restrict__ geo,
                             const int32_t* __restrict__ curve_of, const int32_t* __restrict__ nn, int64_t n,
                             double* __restrict__ w) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) w[i] = sigma[i] * geo[8 * i + 6] * (2.0 * MH_PI / nn[curve_of[i]]);
}

// y_j = sigma_j - 2 alpha^2 u_j - (1/pi) W_j + C_j (a > 0), or with the diagonal limit
// (1/pi) kappa-term h sigma_j in place of W_j and C_j (a = 0).  u_j is the multipole-pass output
// -(1/(2 pi alpha^2)) sum_{i != j} w_i K(y_i, x_j), so -2 alpha^2 u_j = (1/pi) T_j; the window
// terms come from the weights of k_mf_window_weights.  One warp per node: the lanes take the
// 2(a - 1) window terms and the 2l Alpert terms, summed by a fixed-order warp reduction.
__global__ void k_mf_combine(const double* __restrict__ sigma, const double* __restrict__ u,
                             const double* __restrict__ geo, const int32_t* __restrict__ curve_of,
                             const int32_t* __restrict__ nn, const int32_t* __restrict__ off, int64_t n,
                             double alpha, int a, int l2, const double* __restrict__ win,
                             const double* __restrict__ cp, const double* __restrict__ S, double* __restrict__ y) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;   // the whole warp
    const int k = curve_of[j], N = nn[k], o = off[k];
    const int jj = (int)(j - o);
    double v = 0.0;
    if (a > 0) {
        const int nw = 2 * (a - 1);
        for (int t = lane; t < nw; t += 32) v -= win[j * nw + t] * sigma[o + mf_win_node(jj, t, N)];
    } else if (lane == 0) {
        const double* gj = geo + 8 * j;
        v = (1.0 / MH_PI) * gj[7] * gj[6] * (2.0 * MH_PI / N) * sigma[j];
    }
    for (int p = lane; p < l2; p += 32) v += cp[j * l2 + p] * S[(int64_t)p * n + j];
    v = warp_sum(v);
    if (lane == 0) y[j] = sigma[j] - 2.0 * alpha * alpha * u[j] + v;
}

// ============================ host side ============================

static mh_status upload_alpert(int l, AlpertRule* R) {
    R->l = l;
    R->a = l;
    for (int m = 0; m < MH_ALPERT_LMAX; ++m) {
        R->x[m] = m < l ? mh_alpert_nodes[l][m] : 0.0;
        R->w[m] = m < l ? mh_alpert_weights[l][m] : 0.0;
    }
    return MH_OK;
}

extern "C" mh_status mh_boundary_create(mh_ctx* ctx, int n_curves, const int32_t* n_nodes_host,
                                        const double* xy_host, int alpert_order, mh_boundary** out) {
    if (!ctx || !out || !n_nodes_host || !xy_host) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n_curves < 1 || n_curves > 32) return mh_fail(ctx, MH_ERR_INVALID_ARG, "n_curves must be in 1..32");
    if (alpert_order < 0 || alpert_order > MH_ALPERT_LMAX)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "alpert_order must be in 0..%d", MH_ALPERT_LMAX);
    auto* b = new mh_boundary();
    b->n_curves = n_curves;
    b->alpert_order = alpert_order;
    int64_t tot = 0;
    for (int k = 0; k < n_curves; ++k) {
        int N = n_nodes_host[k];
        if (N < 2 * alpert_order + 4 || N % 2) {
            delete b;
            return mh_fail(ctx, MH_ERR_INVALID_ARG, "curve %d: N=%d must be even and >= 2*alpert_order+4", k, N);
        }
        b->n_nodes.push_back(N);
        b->offset.push_back((int32_t)tot);
        tot += N;
    }
    b->offset.push_back((int32_t)tot);
    b->n = tot;
    std::vector<int32_t> curve_of(tot);
    for (int k = 0; k < n_curves; ++k)
        for (int i = b->offset[k]; i < b->offset[k + 1]; ++i) curve_of[i] = k;
    cudaStream_t st = ctx->stream;
    auto fail = [&](mh_status s) {
        delete b;
        return s;
    };
#define BCHK(call)                                                                                     \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(mh_fail(ctx, MH_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_))); \
    } while (0)
    BCHK(b->d_nn.alloc(n_curves));
    BCHK(b->d_off.alloc(n_curves + 1));
    BCHK(b->d_curve_of.alloc(tot));
    BCHK(b->xy.alloc(2 * tot));
    BCHK(b->geo.alloc(8 * tot));
    const int64_t nmodes = tot / 2 + n_curves;
    BCHK(b->coef.alloc(4 * nmodes));
    BCHK(cudaMemcpyAsync(b->d_nn.p, b->n_nodes.data(), n_curves * 4, cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(b->d_off.p, b->offset.data(), (n_curves + 1) * 4, cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(b->d_curve_of.p, curve_of.data(), tot * 4, cudaMemcpyHostToDevice, st));
    BCHK(cudaMemcpyAsync(b->xy.p, xy_host, 2 * tot * 8, cudaMemcpyHostToDevice, st));
    k_fourier_xy<<<mh_grid(nmodes, 128), 128, 0, st>>>(b->xy.p, b->d_nn.p, b->d_off.p, n_curves, nmodes, b->coef.p);
    ctx->launches++;
    k_node_geometry<<<mh_grid(tot, 128), 128, 0, st>>>(b->coef.p, b->d_nn.p, b->d_off.p, b->d_curve_of.p, tot,
                                                         b->geo.p);
    ctx->launches++;
    // fine grid
    b->fine_off.resize(n_curves + 1);
    b->fine_off[0] = 0;
    for (int k = 0; k < n_curves; ++k) b->fine_off[k + 1] = b->fine_off[k] + (int64_t)UPSAMPLE * b->n_nodes[k];
    b->n_fine = b->fine_off[n_curves];
    BCHK(b->d_fine_off.alloc(n_curves + 1));
    BCHK(b->fine_geo.alloc(6 * b->n_fine));
    BCHK(cudaMemcpyAsync(b->d_fine_off.p, b->fine_off.data(), (n_curves + 1) * 8, cudaMemcpyHostToDevice, st));
    BCHK(b->tw.alloc(tot));
    BCHK(b->half.alloc(tot));
    k_twiddles<<<mh_grid(tot, 128), 128, 0, st>>>(b->d_nn.p, b->d_off.p, b->d_curve_of.p, tot, b->tw.p, b->half.p);
    ctx->launches++;
    k_fine_geometry<<<mh_grid(b->n_fine, 128), 128, 0, st>>>(b->coef.p, b->d_nn.p, b->d_off.p, b->d_fine_off.p,
                                                               n_curves, b->n_fine, b->fine_geo.p);
    ctx->launches++;
    BCHK(cudaGetLastError());
    // orientation: signed area (1/2) sum (x y' - y x') h per curve
    std::vector<double> geo(8 * tot);
    BCHK(cudaMemcpyAsync(geo.data(), b->geo.p, 8 * tot * 8, cudaMemcpyDeviceToHost, st));
    BCHK(cudaStreamSynchronize(st));
    for (int k = 0; k < n_curves; ++k) {
        double area = 0.0, h = 2.0 * MH_PI / b->n_nodes[k];
        for (int i = b->offset[k]; i < b->offset[k + 1]; ++i)
            area += 0.5 * h * (geo[8 * i] * geo[8 * i + 3] - geo[8 * i + 1] * geo[8 * i + 2]);
        if ((k == 0 && area <= 0) || (k > 0 && area >= 0))
            return fail(mh_fail(ctx, MH_ERR_GEOMETRY,
                                "curve %d has the wrong orientation (outer curve must be counter-clockwise, "
                                "holes clockwise)", k));
    }
#undef BCHK
    *out = b;
    return MH_OK;
}

extern "C" mh_status mh_boundary_destroy(mh_boundary* b) {
    delete b;
    return MH_OK;
}

extern "C" mh_status mh_boundary_size(const mh_boundary* b, int64_t* n) {
    if (!b || !n) return MH_ERR_INVALID_ARG;
    *n = b->n;
    return MH_OK;
}

extern "C" mh_status mh_boundary_geometry(mh_ctx* ctx, const mh_boundary* b, double* out_host) {
    if (!ctx || !b || !out_host) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_CUDA(ctx, cudaMemcpyAsync(out_host, b->geo.p, 8 * b->n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return MH_OK;
}

// ---- matrix-free operator (host) ----

// Everything of the matrix-free form but the multipole pass, which the caller has set up on
// tree t for the boundary nodes (volume_bie_setup).  Releases the dense operator.
mh_status bie_mfree_setup(mh_ctx* ctx, mh_boundary* b, mh_tree* t, double alpha) {
    if (!t || !volume_bie_ready(t)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "the on-surface multipole pass is not set up");
    const int64_t n = b->n;
    const int nc = b->n_curves, a = b->alpert_order;
    std::vector<int32_t> Mk(nc);
    std::vector<int64_t> moff(nc + 1, 0);
    int mmax = 2;
    for (int k = 0; k < nc; ++k) {
        const int N = b->n_nodes[k];
        if (N % 2 != 0 || N > MF_MMAX / 2 || N < std::max(2 * a, 4))
            return mh_fail(ctx, MH_ERR_INVALID_ARG,
                           "the matrix-free operator needs an even node count in [max(2 l, 4), %d] on every curve (curve %d has %d)",
                           MF_MMAX / 2, k, N);
        int M = 2;
        if ((N & (N - 1)) == 0)
            M = N;   // radix-2 transforms of length N
        else
            while (M < 2 * N - 1) M <<= 1;
        Mk[k] = M;
        moff[k + 1] = moff[k] + M;
        mmax = std::max(mmax, M);
    }
    cudaStream_t st = ctx->stream;
    b->mfree = false;
    MH_ALLOC(ctx, b->mf_M, nc);
    MH_ALLOC(ctx, b->mf_moff, nc + 1);
    MH_CUDA(ctx, cudaMemcpyAsync(b->mf_M.p, Mk.data(), nc * 4, cudaMemcpyHostToDevice, st));
    MH_CUDA(ctx, cudaMemcpyAsync(b->mf_moff.p, moff.data(), (nc + 1) * 8, cudaMemcpyHostToDevice, st));
    MH_ALLOC(ctx, b->mf_chirp, n);
    MH_ALLOC(ctx, b->mf_bh, moff[nc]);
    MH_ALLOC(ctx, b->mf_tw, moff[nc] / 2);
    MH_ALLOC(ctx, b->mf_spec, n / 2 + nc);   // N_k/2 + 1 modes per curve
    MH_ALLOC(ctx, b->mf_w, n);
    MH_ALLOC(ctx, b->mf_u, n);
    const size_t smem = 24 * (size_t)mmax;
    MH_CUDA(ctx, cudaFuncSetAttribute(k_mf_chirp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MH_CUDA(ctx, cudaFuncSetAttribute(k_mf_spectrum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MH_CUDA(ctx, cudaFuncSetAttribute(k_mf_shift, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mf_chirp<<<(unsigned)nc, MF_THREADS, smem, st>>>(b->d_nn.p, b->mf_moff.p, b->mf_M.p, b->d_off.p, b->mf_chirp.p,
                                                       b->mf_bh.p, b->mf_tw.p);
    MH_LAUNCHED(ctx);
    if (a > 0) {
        AlpertRule R;
        upload_alpert(a, &R);
        MH_ALLOC(ctx, b->mf_cp, n * 2 * R.l);
        MH_ALLOC(ctx, b->mf_S, n * 2 * R.l);
        k_alpert_weights<<<(unsigned)n, 128, 0, st>>>(b->geo.p, b->coef.p, b->d_curve_of.p, b->d_nn.p, b->d_off.p,
                                                      1.0 / alpha, R, b->mf_cp.p);
        MH_LAUNCHED(ctx);
        const int nw = 2 * (a - 1);
        MH_ALLOC(ctx, b->mf_win, std::max<int64_t>(n * nw, 1));
        if (nw) {
            k_mf_window_weights<<<mh_grid(n * nw, 256), 256, 0, st>>>(b->geo.p, b->d_curve_of.p, b->d_nn.p, b->d_off.p, n,
                                                                     1.0 / alpha, nw, b->mf_win.p);
            MH_LAUNCHED(ctx);
        }
    }
    if (!b->mf_side.s) MH_TRY(b->mf_side.create(ctx));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    b->mf_tree = t;
    b->mf_alpha = alpha;
    b->mf_mmax = mmax;
    b->mfree = true;
    // the dense forms are not used any more
    b->op.A64.release();
    b->op.A32.release();
    b->op.A32lo.release();
    b->op.A16lo.release();
    b->op.alpha = -1.0;
    b->op.gen += 1;
    return MH_OK;
}

// y = A x through the matrix-free form (binary64).
mh_status bie_apply_mfree(mh_ctx* ctx, mh_boundary* b, const double* x, double* y) {
    if (!volume_bie_ready(b->mf_tree))
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "the multipole pass of the matrix-free operator is gone (the tree's "
                                                "volume operators were rebuilt for another alpha or p)");
    prof_scope ps(ctx, "bie_mfree");
    cudaStream_t st = ctx->stream;
    const int64_t n = b->n;
    const int a = b->alpert_order;
    int l2 = 0;
    AlpertRule R;
    // The Alpert transforms need only x: they run on the side stream beside the multipole pass,
    // joined before the combination (inside the "bie_mfree" region, whose events are on the
    // context stream, so its time is that of the overlapped product).
    const bool fork = a > 0 && b->mf_side.s;
    if (a > 0) {
        upload_alpert(a, &R);
        l2 = 2 * R.l;
        cudaStream_t as = st;
        if (fork) {
            MH_TRY(b->mf_side.begin(ctx, st));
            as = b->mf_side.s;
        }
        const size_t smem = 24 * (size_t)b->mf_mmax;
        k_mf_spectrum<<<(unsigned)b->n_curves, MF_THREADS, smem, as>>>(x, b->d_nn.p, b->d_off.p, b->mf_moff.p, b->mf_M.p,
                                                                        b->mf_chirp.p, b->mf_bh.p, b->mf_tw.p,
                                                                        b->mf_spec.p);
        MH_LAUNCHED(ctx);
        k_mf_shift<<<dim3((unsigned)l2, (unsigned)b->n_curves), MF_THREADS, smem, as>>>(
            b->mf_spec.p, b->d_nn.p, b->d_off.p, b->mf_moff.p, b->mf_M.p, b->mf_chirp.p, b->mf_bh.p, b->mf_tw.p, R, n,
            b->mf_S.p);
        MH_LAUNCHED(ctx);
        if (fork) MH_TRY(b->mf_side.end(ctx));
    }
    k_mf_weights<<<mh_grid(n, 256), 256, 0, st>>>(x, b->geo.p, b->d_curve_of.p, b->d_nn.p, n, b->mf_w.p);
    MH_LAUNCHED(ctx);
    MH_TRY(volume_bie_apply(ctx, b->mf_tree, b->mf_w.p, b->mf_u.p));
    if (fork) MH_CUDA(ctx, cudaStreamWaitEvent(st, b->mf_side.join, 0));
    k_mf_combine<<<mh_grid(n * 32, 256), 256, 0, st>>>(x, b->mf_u.p, b->geo.p, b->d_curve_of.p, b->d_nn.p, b->d_off.p,
                                                       n, b->mf_alpha, a, l2, b->mf_win.p, b->mf_cp.p, b->mf_S.p, y);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

mh_status bie_assemble(mh_ctx* ctx, mh_boundary* b, double alpha) {
    if (b->mfree) {
        if (alpha != b->mf_alpha)
            return mh_fail(ctx, MH_ERR_INVALID_ARG, "the matrix-free operator was set up for alpha = %.17g, not %.17g",
                           b->mf_alpha, alpha);
        return MH_OK;
    }
    if (b->op.alpha == alpha && b->op.A64.p) return MH_OK;
    const int64_t n = b->n;
    MH_ALLOC(ctx, b->op.A64, n * n);
    b->op.A32.release();
    b->op.A32lo.release();
    b->op.A16lo.release();
    b->op.gen += 1;
    b->op.alpha = -1.0;
    cudaStream_t st = ctx->stream;
    dim3 grid((unsigned)mh_grid(n, 256), (unsigned)std::min<int64_t>(n, 65535));
    k_assemble_trap<<<grid, 256, 0, st>>>(b->geo.p, b->d_curve_of.p, b->d_nn.p, b->d_off.p, n, 1.0 / alpha,
                                          b->alpert_order, b->op.A64.p);
    MH_LAUNCHED(ctx);
    if (b->alpert_order > 0) {
        AlpertRule R;
        upload_alpert(b->alpert_order, &R);
        k_assemble_alpert<<<(unsigned)n, 128, 0, st>>>(b->geo.p, b->coef.p, b->d_curve_of.p, b->d_nn.p, b->d_off.p, n,
                                                       1.0 / alpha, R, b->op.A64.p);
        MH_LAUNCHED(ctx);
    }
    b->op.alpha = alpha;
    return MH_OK;
}

static mh_status gemv_cpa_prepare(mh_ctx* ctx);

// The dense forms exist only once bie_assemble has run (the matrix-free set-up releases them).
static mh_status need_dense(mh_ctx* ctx, const mh_boundary* b) {
    if (!b->op.A64.p) return mh_fail(ctx, MH_ERR_INVALID_ARG, "the dense boundary operator is not assembled");
    return MH_OK;
}

static mh_status ensure_fp32(mh_ctx* ctx, mh_boundary* b) {
    if (b->mfree) return mh_fail(ctx, MH_ERR_INVALID_ARG, "the matrix-free operator runs in binary64 only");
    MH_TRY(need_dense(ctx, b));
    MH_TRY(gemv_cpa_prepare(ctx));
    if (b->op.A32.p) return MH_OK;
    const int64_t nn = b->n * b->n;
    b->op.gen += 1;
    MH_ALLOC(ctx, b->op.A32, nn);
    k_to_float<<<152 * 8, 256, 0, ctx->stream>>>(b->op.A64.p, b->op.A32.p, nn);
    MH_LAUNCHED(ctx);
    if ((b->n & 7) == 0) {   // float-float residual products (mixed precision), binary16 low part
        MH_ALLOC(ctx, b->op.A16lo, nn);
        k_split_lo16<<<152 * 8, 256, 0, ctx->stream>>>(b->op.A64.p, b->op.A32.p, b->op.A16lo.p, nn);
        MH_LAUNCHED(ctx);
    } else if ((b->n & 3) == 0) {   // float-float residual products, binary32 low part
        MH_ALLOC(ctx, b->op.A32lo, nn);
        k_split_lo<<<152 * 8, 256, 0, ctx->stream>>>(b->op.A64.p, b->op.A32.p, b->op.A32lo.p, nn);
        MH_LAUNCHED(ctx);
    }
    if (b->op.A16lo.p || b->op.A32lo.p) {
        if (!b->xhi32.p) {
            MH_ALLOC(ctx, b->xhi32, b->n);
            MH_ALLOC(ctx, b->xlo32, b->n);
        }
    }
    return MH_OK;
}

mh_status bie_prepare(mh_ctx* ctx, mh_boundary* b, mh_precision prec) {
    if (prec == MH_PREC_MIXED) {
        MH_TRY(ensure_fp32(ctx, b));
        if (!b->x32.p) MH_ALLOC(ctx, b->x32, b->n);
    }
    return MH_OK;
}

static int gemv_blocks(int64_t n) {
    int64_t need = (n + 7) / 8;            // 8 warps per block
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, 152 * 16));
}

constexpr int GEMV_SPLIT = 4;   // warps per row of the row-split GEMVs

constexpr size_t GC_SMEM2 = 8 * 2 * GC_PIECE * 32 * sizeof(float4);   // 24 KB
constexpr size_t GH_SMEM = 8 * 3 * GH_PIECE * 32 * sizeof(float4);    // 24 KB

// The float-float product with the binary16 low part (k_gemv_cph): 47.6 us for the starfish
// operator in ncu (226 MB), against 55.5 us for the binary32 low part (302 MB); capping it at 6
// blocks per SM (40 registers) took 62.5 us.
// The binary32 GEMV keeps register loads (k_gemv32s, 28 us for the starfish operator); staging its
// loads through cp.async measures the same (28.6 us).  The float-float product, with twice the
// bytes per entry, gains from the staging (81 us with register loads; 53 us with pieces of 3
// float4 per lane, where pieces of 12 took 64 us: a warp waits for its piece before it
// computes, and small pieces leave room for 8 blocks per SM, so some compute while others load).
static void gemv32(cudaStream_t st, const float* A, const float* x, double* y, int64_t n, const int* gate) {
    if ((n & 3) == 0)
        k_gemv32s<GEMV_SPLIT><<<(unsigned)((n + 8 / GEMV_SPLIT - 1) / (8 / GEMV_SPLIT)), 256, 0, st>>>(A, x, y, n,
                                                                                                     gate);
    else
        k_gemv32<<<gemv_blocks(n), 256, 0, st>>>(A, x, y, n, gate);
}

// Shared-memory opt-in of the cp.async GEMVs (once per process, outside any graph capture).
static mh_status gemv_cpa_prepare(mh_ctx* ctx) {
    static bool done = false;
    if (done) return MH_OK;
    MH_CUDA(ctx, cudaFuncSetAttribute(k_gemv_cpa<GEMV_SPLIT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)GC_SMEM2));
    MH_CUDA(ctx, cudaFuncSetAttribute(k_gemv_cph<GEMV_SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)GH_SMEM));
    done = true;
    return MH_OK;
}

static void gemv64(cudaStream_t st, const double* A, const double* x, double* y, int64_t n, const int* gate) {
    if ((n & 1) == 0)
        k_gemv64s<GEMV_SPLIT><<<(unsigned)((n + 8 / GEMV_SPLIT - 1) / (8 / GEMV_SPLIT)), 256, 0, st>>>(A, x, y, n,
                                                                                                     gate);
    else
        k_gemv64<<<gemv_blocks(n), 256, 0, st>>>(A, x, y, n, gate);
}

// Product with the binary64 operator for a residual: in mixed precision a float-float product
// on A32 + 2^-24 A16lo (N_Gamma a multiple of 8) or A32 + A32lo (a multiple of 4), else
// binary64.  The float-float
// form first splits x into binary32 hi + lo (resid_split), then runs the GEMV (resid_gemv);
// the two are separate so that a timed region can hold the GEMV alone.
static bool resid_ff(const mh_boundary* b, bool mixed) { return mixed && (b->op.A16lo.p || b->op.A32lo.p); }

static void resid_split(cudaStream_t st, mh_boundary* b, const double* x) {
    k_split_vec<<<mh_grid(b->n, 256), 256, 0, st>>>(x, b->xhi32.p, b->xlo32.p, b->n);
}

static void resid_gemv(cudaStream_t st, mh_boundary* b, const double* x, double* y, const int* gate, bool mixed) {
    const int64_t n = b->n;
    const unsigned grid = (unsigned)((n + 8 / GEMV_SPLIT - 1) / (8 / GEMV_SPLIT));
    if (mixed && b->op.A16lo.p)
        k_gemv_cph<GEMV_SPLIT><<<grid, 256, GH_SMEM, st>>>(b->op.A32.p, b->op.A16lo.p, b->xhi32.p, b->xlo32.p, y, n,
                                                          gate);
    else if (mixed && b->op.A32lo.p)
        k_gemv_cpa<GEMV_SPLIT, 2><<<grid, 256, GC_SMEM2, st>>>(b->op.A32.p, b->op.A32lo.p, b->xhi32.p, b->xlo32.p, y,
                                                               n, gate);
    else
        gemv64(st, b->op.A64.p, x, y, n, gate);
}

static void gemv_resid(cudaStream_t st, mh_boundary* b, const double* x, double* y, const int* gate, bool mixed) {
    if (resid_ff(b, mixed)) resid_split(st, b, x);
    resid_gemv(st, b, x, y, gate, mixed);
}

static const char* resid_region(mh_boundary* b, bool mixed, const int* gate) {
    if (gate) return "bie_gemv64_gated";   // may be skipped on the device: timed apart
    return resid_ff(b, mixed) ? "bie_gemvff" : "bie_gemv64";
}

static double resid_bytes(mh_boundary* b, bool mixed) {
    const double n = (double)b->n;
    if (mixed && b->op.A16lo.p) return 6.0 * n * n + 24.0 * n;
    return mixed && b->op.A32lo.p ? 8.0 * n * n + 24.0 * n : 8.0 * n * n + 16.0 * n;
}

mh_status bie_apply64_gated(mh_ctx* ctx, mh_boundary* b, const double* x, double* y, const int* gate,
                            mh_precision prec) {
    // the gate only skips work whose result the caller then ignores: the matrix-free form
    // always computes
    if (b->mfree) return bie_apply_mfree(ctx, b, x, y);
    MH_TRY(need_dense(ctx, b));
    const bool mixed = prec == MH_PREC_MIXED;
    if (resid_ff(b, mixed)) {   // the split of x is not part of the timed GEMV region
        resid_split(ctx->stream, b, x);
        MH_LAUNCHED(ctx);
    }
    prof_scope ps(ctx, resid_region(b, mixed, gate), 2.0 * b->n * b->n, resid_bytes(b, mixed));
    resid_gemv(ctx->stream, b, x, y, gate, mixed);
    MH_LAUNCHED(ctx);
    return MH_OK;
}

mh_status bie_apply_resid(mh_ctx* ctx, mh_boundary* b, const double* x, double* y, mh_precision prec) {
    return bie_apply64_gated(ctx, b, x, y, nullptr, prec);
}

const double* gmres_final_residual(mh_boundary* b, mh_precision prec, bool graph) {
    return (graph || prec == MH_PREC_MIXED) ? b->ws.r.p : b->ws.w.p;
}


mh_status bie_apply(mh_ctx* ctx, mh_boundary* b, const double* x, double* y, mh_precision prec) {
    if (b->mfree) return bie_apply_mfree(ctx, b, x, y);
    MH_TRY(need_dense(ctx, b));
    if (prec == MH_PREC_MIXED) {
        MH_TRY(ensure_fp32(ctx, b));
        if (!b->x32.p) MH_ALLOC(ctx, b->x32, b->n);
        k_to_float_vec<<<mh_grid(b->n, 256), 256, 0, ctx->stream>>>(x, b->x32.p, b->n);
        MH_LAUNCHED(ctx);
        prof_scope ps(ctx, "bie_gemv32", 2.0 * b->n * b->n, 4.0 * b->n * b->n + 12.0 * b->n);
        gemv32(ctx->stream, b->op.A32.p, b->x32.p, y, b->n, nullptr);
    } else {
        prof_scope ps(ctx, "bie_gemv64", 2.0 * b->n * b->n, 8.0 * b->n * b->n + 16.0 * b->n);
        gemv64(ctx->stream, b->op.A64.p, x, y, b->n, nullptr);
    }
    MH_LAUNCHED(ctx);
    return MH_OK;
}

static mh_status vec_norm(mh_ctx* ctx, const double* v, int64_t n, double* dev_out, double* host_out) {
    k_norm<<<1, 1024, 0, ctx->stream>>>(v, n, dev_out);
    MH_LAUNCHED(ctx);
    MH_CUDA(ctx, cudaMemcpyAsync(host_out, dev_out, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return MH_OK;
}

// Unrestarted GMRES on A (precision prec) for A x = b; x holds the initial guess.
// Returns iterations used and the Givens residual estimate (absolute).
static mh_status gmres_core(mh_ctx* ctx, mh_boundary* bd, gmres_ws& ws, const double* b, double* x, double abs_tol,
                            int max_iter, mh_precision prec, int* iters, double* resid, const double* r0,
                            double* beta0) {
    const int64_t n = bd->n;
    cudaStream_t st = ctx->stream;
    const int ew = mh_grid(n, 256) < 152 * 4 ? mh_grid(n, 256) : 152 * 4;
    const int ldh = max_iter + 1;
    if (prec == MH_PREC_MIXED) MH_TRY(ensure_fp32(ctx, bd));
    // r = b - A x (or the caller's residual of x)
    if (r0) {
        MH_CUDA(ctx, cudaMemcpyAsync(ws.w.p, r0, n * 8, cudaMemcpyDeviceToDevice, st));
    } else {
        MH_TRY(bie_apply(ctx, bd, x, ws.w.p, prec));
        k_sub_from<<<ew, 256, 0, st>>>(b, ws.w.p, n);
        MH_LAUNCHED(ctx);
    }
    double beta;
    MH_TRY(vec_norm(ctx, ws.w.p, n, ws.small.p + 1, &beta));
    if (beta0) *beta0 = beta;
    *iters = 0;
    *resid = beta;
    if (beta <= abs_tol) return MH_OK;
    k_scale_into<<<ew, 256, 0, st>>>(ws.w.p, ws.small.p + 1, ws.V.p, ws.g.p, n);
    MH_LAUNCHED(ctx);
    int k = 0;
    double res = beta;
    // The residual estimate is read back only at predicted convergence points: from the
    // decay observed between two reads, the next read is placed where the estimate should
    // reach the tolerance (iterations between reads are queued without host round trips).
    int next_check = 1, k_prev = 0;
    double res_prev = beta;
    const bool mixed = prec == MH_PREC_MIXED;
    const int S = (int)((n + ARN_ROWS - 1) / ARN_ROWS);
    if (mixed) {
        k_to_float_vec<<<mh_grid(n, 256), 256, 0, st>>>(ws.V.p, ws.v32.p, n);
        MH_LAUNCHED(ctx);
    }
    for (; k < max_iter; ++k) {
        const int k1 = k + 1;
        {   // w = A v_k
            const double* vk = ws.V.p + (int64_t)k * n;
            if (bd->mfree) {
                MH_TRY(bie_apply_mfree(ctx, bd, vk, ws.w.p));
            } else {
                prof_scope ps(ctx, mixed ? "bie_gemv32" : "bie_gemv64", 2.0 * n * n,
                              mixed ? 4.0 * n * n + 12.0 * n : 8.0 * n * n + 16.0 * n);
                if (mixed)
                    gemv32(st, bd->op.A32.p, ws.v32.p, ws.w.p, n, nullptr);
                else
                    gemv64(st, bd->op.A64.p, vk, ws.w.p, n, nullptr);
                MH_LAUNCHED(ctx);
            }
        }
        // classical Gram-Schmidt twice, normalisation and the Givens update (four launches)
        const size_t shm = (size_t)(k1 + ARN_ROWS) * sizeof(double);
        k_arn_dots<<<S, 256, 0, st>>>(ws.V.p, ws.w.p, n, k1, ws.P1.p);
        MH_LAUNCHED(ctx);
        k_arn_update<<<S, 256, shm, st>>>(ws.V.p, ws.w.p, n, k1, ws.P1.p, S, ws.P2.p, nullptr, ws.h1.p);
        MH_LAUNCHED(ctx);
        k_arn_update<<<S, 256, shm, st>>>(ws.V.p, ws.w.p, n, k1, ws.P2.p, S, nullptr, ws.Pn.p, ws.h2.p);
        MH_LAUNCHED(ctx);
        k_arn_finish<<<S, 256, (size_t)(3 * k + 2) * sizeof(double), st>>>(ws.w.p, n, ws.Pn.p, S, k, ws.h1.p,
                                                                            ws.h2.p, ws.H.p, ldh, ws.cs.p, ws.sn.p,
                                        ws.g.p, ws.small.p, ws.V.p + (int64_t)k1 * n, mixed ? ws.v32.p : nullptr);
        MH_LAUNCHED(ctx);
        if (k + 1 < next_check && k + 1 < max_iter) continue;
        MH_CUDA(ctx, cudaMemcpyAsync(&res, ws.small.p, 8, cudaMemcpyDeviceToHost, st));
        MH_CUDA(ctx, cudaStreamSynchronize(st));
        if (!std::isfinite(res)) return mh_fail(ctx, MH_ERR_NUMERIC, "GMRES residual is not finite");
        if (res <= abs_tol) {
            ++k;
            break;
        }
        const double rate = (res > 0 && res_prev > 0 && k + 1 > k_prev)
                                ? std::pow(res / res_prev, 1.0 / (k + 1 - k_prev)) : 0.5;
        int ahead = 1;
        if (rate > 0 && rate < 0.999) ahead = (int)std::floor(std::log(abs_tol / res) / std::log(rate));
        ahead = std::max(1, std::min(ahead, 8));
        k_prev = k + 1;
        res_prev = res;
        next_check = k + 1 + ahead;
    }
    k_backsolve<<<1, 1, 0, st>>>(ws.H.p, ldh, k, ws.g.p, ws.y.p);
    MH_LAUNCHED(ctx);
    k_update_x<<<ew, 256, 0, st>>>(ws.V.p, ws.y.p, k, n, x);
    MH_LAUNCHED(ctx);
    *iters = k;
    *resid = res;
    return MH_OK;
}

mh_status gmres_run(mh_ctx* ctx, mh_boundary* bd, const double* b, double* x, double tol, int max_iter,
                    mh_precision prec, mh_gmres_info* info, const double* r0) {
    prof_scope ps_all(ctx, "gmres");
    const int64_t n = bd->n;
    if (max_iter < 1 || max_iter > 1000) return mh_fail(ctx, MH_ERR_INVALID_ARG, "max_iter must be in 1..1000");
    if (bd->mfree && prec != MH_PREC_FP64)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "the matrix-free operator runs in binary64 only");
    if (!bd->mfree) MH_TRY(need_dense(ctx, bd));
    MH_TRY(gmres_graph_ensure(ctx, bd, max_iter));
    gmres_ws& ws = bd->ws;
    MH_CUDA(ctx, cudaMemsetAsync(ws.g.p, 0, (max_iter + 2) * 8, ctx->stream));
    double bnorm;
    MH_TRY(vec_norm(ctx, b, n, ws.small.p + 2, &bnorm));
    mh_gmres_info inf{0, 0, 0.0, 0, 0.0};
    if (bnorm == 0.0) {
        MH_CUDA(ctx, cudaMemsetAsync(x, 0, n * 8, ctx->stream));
        MH_CUDA(ctx, cudaMemsetAsync(ws.r.p, 0, n * 8, ctx->stream));   // residual of x = 0
        MH_CUDA(ctx, cudaMemsetAsync(ws.w.p, 0, n * 8, ctx->stream));
        inf.converged = 1;
        if (info) *info = inf;
        return MH_OK;
    }
    if (prec == MH_PREC_FP64) {
        int it;
        double res;
        double beta0;
        MH_TRY(gmres_core(ctx, bd, ws, b, x, tol * bnorm, max_iter, MH_PREC_FP64, &it, &res, r0, &beta0));
        inf.iterations = it;
        inf.initial_rel_residual = beta0 / bnorm;
    } else {
        // binary64 iterative refinement around binary32-operator GMRES
        dbuf<double>& r = ws.r;
        dbuf<double>& dx = ws.dx;
        int total = 0;
        double rn = -1.0;
        for (int sweep = 0;; ++sweep) {
            // binary64 residual of x; at the first sweep the caller's r0 (if given) stands in
            // for it, but convergence is only ever accepted on a residual computed here
            bool computed = true;
            if (sweep == 0 && r0) {
                MH_CUDA(ctx, cudaMemcpyAsync(r.p, r0, n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
                computed = false;
            } else {
                MH_TRY(bie_apply_resid(ctx, bd, x, r.p, MH_PREC_MIXED));
                k_sub_from<<<mh_grid(n, 256), 256, 0, ctx->stream>>>(b, r.p, n);
                MH_LAUNCHED(ctx);
            }
            MH_TRY(vec_norm(ctx, r.p, n, ws.small.p + 2, &rn));
            if (sweep == 0) inf.initial_rel_residual = rn / bnorm;
            if (!computed && rn <= tol * bnorm) {
                MH_TRY(bie_apply_resid(ctx, bd, x, r.p, MH_PREC_MIXED));
                k_sub_from<<<mh_grid(n, 256), 256, 0, ctx->stream>>>(b, r.p, n);
                MH_LAUNCHED(ctx);
                MH_TRY(vec_norm(ctx, r.p, n, ws.small.p + 2, &rn));
            }
            if (rn <= tol * bnorm || total >= max_iter || sweep >= 12) break;
            MH_CUDA(ctx, cudaMemsetAsync(dx.p, 0, n * 8, ctx->stream));
            MH_CUDA(ctx, cudaMemsetAsync(ws.g.p, 0, (max_iter + 2) * 8, ctx->stream));
            int it;
            double res;
            // half the tolerance: the binary64 residual after the sweep then lands below tol
            // instead of just above it (which would cost another sweep and binary64 GEMV)
            MH_TRY(gmres_core(ctx, bd, ws, r.p, dx.p, std::max(0.5 * tol * bnorm, 1e-5 * rn), max_iter - total,
                              MH_PREC_MIXED, &it, &res, r.p, nullptr));
            total += it;
            inf.refinements++;
            k_axpy<<<mh_grid(n, 256), 256, 0, ctx->stream>>>(1.0, dx.p, x, n);
            MH_LAUNCHED(ctx);
        }
        inf.iterations = total;
        inf.rel_residual = rn / bnorm;   // binary64 residual of the final iterate (last sweep)
    }
    if (prec == MH_PREC_FP64) {
        // true residual in binary64
        MH_TRY(bie_apply(ctx, bd, x, ws.w.p, MH_PREC_FP64));
        k_sub_from<<<mh_grid(n, 256), 256, 0, ctx->stream>>>(b, ws.w.p, n);
        MH_LAUNCHED(ctx);
        double rn;
        MH_TRY(vec_norm(ctx, ws.w.p, n, ws.small.p + 2, &rn));
        inf.rel_residual = rn / bnorm;
    }
    inf.converged = inf.rel_residual <= tol;
    if (info) *info = inf;
    if (!inf.converged)
        return mh_fail(ctx, MH_ERR_NOT_CONVERGED, "GMRES stopped after %d iterations at relative residual %.3e",
                       inf.iterations, inf.rel_residual);
    return MH_OK;
}

// ---------------- sync-free GMRES (fixed schedule, device flags) ----------------

mh_status gmres_graph_ensure(mh_ctx* ctx, mh_boundary* bd, int max_iter) {
    const int64_t n = bd->n;
    gmres_ws& ws = bd->ws;
    if (ws.m >= max_iter && ws.n == n) return MH_OK;
    const int ldh = max_iter + 1;
    MH_ALLOC(ctx, ws.V, (int64_t)(max_iter + 1) * n);
    MH_ALLOC(ctx, ws.H, (int64_t)ldh * max_iter);
    MH_ALLOC(ctx, ws.cs, max_iter + 1);
    MH_ALLOC(ctx, ws.sn, max_iter + 1);
    MH_ALLOC(ctx, ws.g, max_iter + 2);
    MH_ALLOC(ctx, ws.y, max_iter + 1);
    MH_ALLOC(ctx, ws.h1, max_iter + 2);
    MH_ALLOC(ctx, ws.h2, max_iter + 2);
    MH_ALLOC(ctx, ws.small, 8);
    MH_ALLOC(ctx, ws.w, n);
    MH_ALLOC(ctx, ws.r, n);
    MH_ALLOC(ctx, ws.dx, n);
    const int64_t S = (n + ARN_ROWS - 1) / ARN_ROWS;
    MH_ALLOC(ctx, ws.P1, S * (max_iter + 1));
    MH_ALLOC(ctx, ws.P2, S * (max_iter + 1));
    MH_ALLOC(ctx, ws.Pn, S);
    MH_ALLOC(ctx, ws.v32, n);
    if (!ws.body_stream) MH_CUDA(ctx, cudaStreamCreateWithFlags(&ws.body_stream, cudaStreamNonBlocking));
    ws.m = max_iter;
    ws.n = n;
    ws.gen += 1;
    return MH_OK;
}

void gmres_graph_schedule(mh_precision prec, int* sweeps, int* m_max) {
    if (prec == MH_PREC_MIXED) {
        *sweeps = 3;    // binary64 refinement passes around the binary32-operator Arnoldi process
        *m_max = 20;
    } else {
        *sweeps = 1;
        *m_max = 40;
    }
}

__global__ void k_gnorm(const double* __restrict__ v, int64_t n, double* out, const int* __restrict__ gate) {
    if (gate && *gate) return;
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(v[e], v[e], acc);
    acc = block_sum<1024>(acc);
    if (threadIdx.x == 0) *out = sqrt(acc);
}

__global__ void k_gsub(const double* __restrict__ b, double* r, int64_t n, const int* __restrict__ gate) {
    if (gate && *gate) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        r[e] = b[e] - r[e];
}

// Start of a sweep from the residual r (norm gs->rn): accept (converged) when allowed and
// rn <= tol ||b||, else start an Arnoldi process on r (V_0 = r / rn, g = (rn, 0, ...), inner
// target max(tol ||b||, 1e-5 rn) in mixed precision, tol ||b|| in binary64).  final_check: the
// last residual of the schedule, recorded only.  ||b|| = 0 gives x = 0.
// With loop_set, the condition of the sweep's Arnoldi loop (a graph WHILE node, 0 by default at
// every launch) is set to "start".
__global__ void k_sweep_begin(gmres_dev* gs, double tol, int mixed, int may_accept, int final_check, int first,
                              const double* __restrict__ r, double* V0, float* v32, double* g, int gsz, int64_t n,
                              double* x, cudaGraphConditionalHandle loop = 0, int loop_set = 0) {
    if (gs->done) return;
    const double rn = gs->rn, bn = gs->bnorm;
    if (bn == 0.0) {
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
            x[e] = 0.0;
            const_cast<double*>(r)[e] = 0.0;   // the residual of x = 0 for b = 0
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            gs->done = gs->skip = gs->converged = 1;
            gs->rel = 0.0;
        }
        return;
    }
    const bool accept = may_accept || final_check;
    const bool conv = accept && rn <= tol * bn;
    const bool start = !conv && !final_check && rn > 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (first) gs->init_rel = rn / bn;
        if (accept) gs->rel = rn / bn;
        if (conv) {
            gs->done = gs->skip = gs->converged = 1;
        } else if (start) {
            gs->skip = 0;
            gs->k = 0;
            gs->sweeps += 1;
            gs->target = mixed ? fmax(0.5 * tol * bn, 1e-5 * rn) : tol * bn;
        } else {
            gs->skip = 1;
        }
        if (loop_set) cudaGraphSetConditional(loop, start ? 1u : 0u);
    }
    if (!start) return;
    const double inv = 1.0 / rn;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = r[e] * inv;
        V0[e] = v;
        if (v32) v32[e] = (float)v;
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < gsz; i += blockDim.x) g[i] = i == 0 ? rn : 0.0;
}

// R y = g with the iteration count of the sweep (device); skipped once converged.
__global__ void k_backsolve_g(const double* H, int ldh, const double* g, double* y, const gmres_dev* gs) {
    if (gs->done) return;
    const int k = gs->k;
    for (int i = k - 1; i >= 0; --i) {
        double acc = g[i];
        for (int j = i + 1; j < k; ++j) acc -= H[(int64_t)j * ldh + i] * y[j];
        const double d = H[(int64_t)i * ldh + i];
        y[i] = d != 0.0 ? acc / d : 0.0;
    }
}

// x += sum_{i < k} y_i V_i (k of the sweep, device); skipped once converged.
__global__ void k_update_x_g(const double* __restrict__ V, const double* __restrict__ y, const gmres_dev* gs,
                             int64_t n, double* x) {
    if (gs->done) return;
    const int k = gs->k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = x[e];
        for (int i = 0; i < k; ++i) acc = fma(y[i], V[(int64_t)i * n + e], acc);
        x[e] = acc;
    }
}

// One binary32-operator Arnoldi iteration as the body of a graph WHILE node on the capturing
// stream ctx->stream: the node is added after the stream's current dependencies, the body is
// captured on the boundary's helper stream, and the stream continues after the node.  The body
// reads the iteration count from gs->k; k_arn_finish ends the loop.
static mh_status gmres_loop_node(mh_ctx* ctx, mh_boundary* bd, gmres_dev* gs, cudaGraphConditionalHandle h, int m,
                                 int SL) {
    cudaStream_t st = ctx->stream;
    gmres_ws& ws = bd->ws;
    const int64_t n = bd->n;
    const int ldh = m + 1;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t nd = 0;
    MH_CUDA(ctx, cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edata, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    MH_CUDA(ctx, cudaGraphAddNode(&node, g, deps, edata, nd, &np));
    MH_CUDA(ctx, cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t bs = ws.body_stream;
    MH_CUDA(ctx, cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ctx->stream = bs;
    gemv32(bs, bd->op.A32.p, ws.v32.p, ws.w.p, n, nullptr);
    MH_LAUNCHED(ctx);
    const size_t shm = (size_t)(m + ARN_ROWS) * sizeof(double);
    k_arn_dots<<<SL, 256, 0, bs>>>(ws.V.p, ws.w.p, n, 1, ws.P1.p, nullptr, &gs->k);
    MH_LAUNCHED(ctx);
    k_arn_update<<<SL, 256, shm, bs>>>(ws.V.p, ws.w.p, n, 1, ws.P1.p, SL, ws.P2.p, nullptr, ws.h1.p, nullptr, &gs->k);
    MH_LAUNCHED(ctx);
    k_arn_update<<<SL, 256, shm, bs>>>(ws.V.p, ws.w.p, n, 1, ws.P2.p, SL, nullptr, ws.Pn.p, ws.h2.p, nullptr, &gs->k);
    MH_LAUNCHED(ctx);
    k_arn_finish<<<SL, 256, (size_t)(3 * m + 2) * sizeof(double), bs>>>(
        ws.w.p, n, ws.Pn.p, SL, 0, ws.h1.p, ws.h2.p, ws.H.p, ldh, ws.cs.p, ws.sn.p, ws.g.p, ws.small.p, ws.V.p,
        ws.v32.p, gs, m, &gs->k, h, 1);
    MH_LAUNCHED(ctx);
    ctx->stream = st;
    cudaGraph_t out = nullptr;
    MH_CUDA(ctx, cudaStreamEndCapture(bs, &out));
    ctx->loop_nodes += 1;
    return MH_OK;
}

mh_status gmres_run_graph(mh_ctx* ctx, mh_boundary* bd, const double* b, double* x, double tol, mh_precision prec,
                          const double* r0, gmres_dev* gs) {
    if (bd->mfree) return mh_fail(ctx, MH_ERR_INVALID_ARG, "the graph form of GMRES needs the dense operator");
    MH_TRY(need_dense(ctx, bd));
    const int64_t n = bd->n;
    cudaStream_t st = ctx->stream;
    int S, m;
    gmres_graph_schedule(prec, &S, &m);
    gmres_ws& ws = bd->ws;
    const bool mixed = prec == MH_PREC_MIXED;
    if (ws.m < m || ws.n != n || (mixed && !bd->op.A32.p) || !bd->op.A64.p)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "sync-free GMRES: workspace or operator not prepared");
    const int ldh = m + 1;
    const int ew = mh_grid(n, 256) < 152 * 4 ? mh_grid(n, 256) : 152 * 4;
    const int SL = (int)((n + ARN_ROWS - 1) / ARN_ROWS);
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    MH_CUDA(ctx, cudaStreamIsCapturing(st, &cst));
    const bool capturing = cst == cudaStreamCaptureStatusActive;
    MH_CUDA(ctx, cudaMemsetAsync(gs, 0, sizeof(gmres_dev), st));
    k_gnorm<<<1, 1024, 0, st>>>(b, n, &gs->bnorm, nullptr);
    MH_LAUNCHED(ctx);
    for (int sw = 0; sw <= S; ++sw) {
        const bool supplied = sw == 0 && r0;
        if (supplied) {
            MH_CUDA(ctx, cudaMemcpyAsync(ws.r.p, r0, n * 8, cudaMemcpyDeviceToDevice, st));
        } else {
            gemv_resid(st, bd, x, ws.r.p, &gs->done, mixed);
            MH_LAUNCHED(ctx);
            k_gsub<<<ew, 256, 0, st>>>(b, ws.r.p, n, &gs->done);
            MH_LAUNCHED(ctx);
        }
        k_gnorm<<<1, 1024, 0, st>>>(ws.r.p, n, &gs->rn, &gs->done);
        MH_LAUNCHED(ctx);
        // while the stream is being captured (a batch graph), the Arnoldi process of a sweep is a
        // graph WHILE node over one iteration: only the iterations needed run
        const bool loop = mixed && capturing && sw < S;
        cudaGraphConditionalHandle h = 0;
        if (loop) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            MH_CUDA(ctx, cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
            MH_CUDA(ctx, cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        }
        k_sweep_begin<<<ew, 256, 0, st>>>(gs, tol, mixed, !supplied, sw == S, sw == 0, ws.r.p, ws.V.p,
                                          mixed ? ws.v32.p : nullptr, ws.g.p, m + 2, n, x, h, loop ? 1 : 0);
        MH_LAUNCHED(ctx);
        if (sw == S) break;
        if (loop) {
            MH_TRY(gmres_loop_node(ctx, bd, gs, h, m, SL));
        } else
        for (int k = 0; k < m; ++k) {
            const int k1 = k + 1;
            if (mixed)
                gemv32(st, bd->op.A32.p, ws.v32.p, ws.w.p, n, &gs->skip);
            else
                gemv64(st, bd->op.A64.p, ws.V.p + (int64_t)k * n, ws.w.p, n, &gs->skip);
            MH_LAUNCHED(ctx);
            const size_t shm = (size_t)(k1 + ARN_ROWS) * sizeof(double);
            k_arn_dots<<<SL, 256, 0, st>>>(ws.V.p, ws.w.p, n, k1, ws.P1.p, &gs->skip);
            MH_LAUNCHED(ctx);
            k_arn_update<<<SL, 256, shm, st>>>(ws.V.p, ws.w.p, n, k1, ws.P1.p, SL, ws.P2.p, nullptr, ws.h1.p,
                                               &gs->skip);
            MH_LAUNCHED(ctx);
            k_arn_update<<<SL, 256, shm, st>>>(ws.V.p, ws.w.p, n, k1, ws.P2.p, SL, nullptr, ws.Pn.p, ws.h2.p,
                                               &gs->skip);
            MH_LAUNCHED(ctx);
            k_arn_finish<<<SL, 256, (size_t)(3 * k + 2) * sizeof(double), st>>>(
                ws.w.p, n, ws.Pn.p, SL, k, ws.h1.p, ws.h2.p, ws.H.p, ldh, ws.cs.p, ws.sn.p, ws.g.p, ws.small.p,
                ws.V.p + (int64_t)k1 * n, mixed ? ws.v32.p : nullptr, gs, m);
            MH_LAUNCHED(ctx);
        }
        k_backsolve_g<<<1, 1, 0, st>>>(ws.H.p, ldh, ws.g.p, ws.y.p, gs);
        MH_LAUNCHED(ctx);
        k_update_x_g<<<ew, 256, 0, st>>>(ws.V.p, ws.y.p, gs, n, x);
        MH_LAUNCHED(ctx);
    }
    return MH_OK;
}

mh_status gmres_info_from_dev(const gmres_dev& g, double tol, mh_gmres_info* info) {
    if (!info) return MH_OK;
    info->iterations = g.total;
    info->refinements = g.sweeps;
    info->rel_residual = g.rel;
    info->converged = g.converged && g.rel <= tol;
    info->initial_rel_residual = g.init_rel;
    return MH_OK;
}

mh_status dlp_classify(mh_ctx* ctx, mh_boundary* b, const double* xy_dev, int64_t n, dlp_targets* tg) {
    cudaStream_t st = ctx->stream;
    tg->n = n;
    dbuf<uint32_t> fine0;
    dbuf<int32_t> lcurve;
    dbuf<double> ldata;
    MH_ALLOC(ctx, tg->region, n);
    MH_ALLOC(ctx, fine0, n);
    MH_ALLOC(ctx, lcurve, n);
    MH_ALLOC(ctx, ldata, 4 * n);
    if (n > 0) {
        k_classify<<<mh_grid(n * 32, 256), 256, 0, st>>>(xy_dev, n, b->geo.p, b->coef.p, b->d_nn.p, b->d_off.p,
                                                         b->n_curves, tg->region.p, fine0.p, lcurve.p, ldata.p);
        MH_LAUNCHED(ctx);
    }
    // host-side compaction of the (few) line targets and fine pairs
    std::vector<uint32_t> fm(n);
    std::vector<int32_t> lc(n), reg(n);
    std::vector<double> ld(4 * n);
    MH_CUDA(ctx, cudaMemcpyAsync(fm.data(), fine0.p, n * 4, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaMemcpyAsync(lc.data(), lcurve.p, n * 4, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaMemcpyAsync(ld.data(), ldata.p, 4 * n * 8, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaMemcpyAsync(reg.data(), tg->region.p, n * 4, cudaMemcpyDeviceToHost, st));
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    std::vector<int32_t> ltgt, lcur;
    std::vector<double> ldat;
    for (int64_t i = 0; i < n; ++i)
        if (lc[i] >= 0 && reg[i] == -1) {
            ltgt.push_back((int32_t)i);
            lcur.push_back(lc[i]);
            for (int j = 0; j < 4; ++j) ldat.push_back(ld[4 * i + j]);
        }
    tg->n_line = (int64_t)ltgt.size();
    tg->n_ext = n + 4 * tg->n_line;
    std::vector<uint32_t> fext(tg->n_ext);
    for (int64_t i = 0; i < n; ++i) fext[i] = fm[i];
    for (int64_t t = 0; t < tg->n_line; ++t)
        for (int m = 0; m < 4; ++m) fext[n + 4 * t + m] = fm[ltgt[t]] | (1u << lcur[t]);
    std::vector<int32_t> pt, pc;
    for (int64_t i = 0; i < tg->n_ext; ++i)
        for (int k = 0; k < b->n_curves; ++k)
            if (fext[i] & (1u << k)) {
                pt.push_back((int32_t)i);
                pc.push_back(k);
            }
    tg->n_pairs = (int64_t)pt.size();
    tg->n_pairs_main = 0;
    while (tg->n_pairs_main < tg->n_pairs && pt[tg->n_pairs_main] < n) tg->n_pairs_main++;
    tg->fine_nodes_main = tg->fine_nodes_aux = tg->curve_nodes_main = 0;
    for (int64_t i = 0; i < tg->n_pairs; ++i) {
        const double nk = b->n_nodes[pc[i]];
        if (i < tg->n_pairs_main) {
            tg->fine_nodes_main += UPSAMPLE * nk;
            tg->curve_nodes_main += nk;
        } else {
            tg->fine_nodes_aux += UPSAMPLE * nk;
        }
    }
    // groups of FINE_TG auxiliary pairs on one curve (pairs in their order within a curve)
    std::vector<int32_t> gcur, gpair;
    {
        std::vector<std::vector<int32_t>> byc(b->n_curves);
        for (int64_t i = tg->n_pairs_main; i < tg->n_pairs; ++i) byc[pc[i]].push_back((int32_t)i);
        int64_t min_chunks = INT64_MAX;
        for (int k = 0; k < b->n_curves; ++k) {
            if (byc[k].empty()) continue;
            min_chunks = std::min<int64_t>(min_chunks, (b->fine_off[k + 1] - b->fine_off[k] + MH_TILE - 1) / MH_TILE);
            for (size_t j0 = 0; j0 < byc[k].size(); j0 += FINE_TG) {
                gcur.push_back(k);
                for (int j = 0; j < FINE_TG; ++j) gpair.push_back(j0 + j < byc[k].size() ? byc[k][j0 + j] : -1);
            }
        }
        tg->n_groups = (int64_t)gcur.size();
        // slices of the fine chunks: about 8 blocks per SM over the whole launch
        tg->fine_slices = tg->n_groups
                              ? (int)std::max<int64_t>(1, std::min<int64_t>(min_chunks,
                                                                            (152 * 8 + tg->n_groups - 1) / tg->n_groups))
                              : 1;
    }
    MH_ALLOC(ctx, tg->grp_curve, std::max<int64_t>(tg->n_groups, 1));
    MH_ALLOC(ctx, tg->grp_pair, std::max<int64_t>(tg->n_groups * FINE_TG, 1));
    MH_ALLOC(ctx, tg->grp_part, std::max<int64_t>(tg->fine_slices > 1 ? tg->n_groups * tg->fine_slices * FINE_TG : 0, 1));
    MH_ALLOC(ctx, tg->grp_cnt, std::max<int64_t>(tg->n_groups, 1));
    MH_CUDA(ctx, cudaMemsetAsync(tg->grp_cnt.p, 0, std::max<int64_t>(tg->n_groups, 1) * sizeof(unsigned), st));
    if (tg->n_groups) {
        MH_CUDA(ctx, cudaMemcpyAsync(tg->grp_curve.p, gcur.data(), gcur.size() * 4, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(tg->grp_pair.p, gpair.data(), gpair.size() * 4, cudaMemcpyHostToDevice, st));
    }
    MH_ALLOC(ctx, tg->xy, 2 * tg->n_ext);
    MH_ALLOC(ctx, tg->fine, tg->n_ext);
    MH_ALLOC(ctx, tg->line_tgt, tg->n_line);
    MH_ALLOC(ctx, tg->line_curve, tg->n_line);
    MH_ALLOC(ctx, tg->line_data, 4 * tg->n_line);
    MH_ALLOC(ctx, tg->pair_tgt, tg->n_pairs);
    MH_ALLOC(ctx, tg->pair_curve, tg->n_pairs);
    if (n > 0) MH_CUDA(ctx, cudaMemcpyAsync(tg->xy.p, xy_dev, 2 * n * 8, cudaMemcpyDeviceToDevice, st));
    if (tg->n_ext) MH_CUDA(ctx, cudaMemcpyAsync(tg->fine.p, fext.data(), tg->n_ext * 4, cudaMemcpyHostToDevice, st));
    if (tg->n_line) {
        MH_CUDA(ctx, cudaMemcpyAsync(tg->line_tgt.p, ltgt.data(), tg->n_line * 4, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(tg->line_curve.p, lcur.data(), tg->n_line * 4, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(tg->line_data.p, ldat.data(), 4 * tg->n_line * 8, cudaMemcpyHostToDevice, st));
        k_line_aux<<<mh_grid(tg->n_line * 32, 256), 256, 0, st>>>(tg->line_tgt.p, tg->line_curve.p, tg->line_data.p,
                                                                  tg->n_line, b->coef.p, b->d_nn.p, b->d_off.p, n,
                                                                  tg->xy.p);
        MH_LAUNCHED(ctx);
        // trigonometric interpolation weights of every line target (fixed with the target)
        std::vector<int64_t> woff(tg->n_line + 1, 0);
        for (int64_t t = 0; t < tg->n_line; ++t) woff[t + 1] = woff[t] + b->n_nodes[lcur[t]];
        MH_ALLOC(ctx, tg->line_woff, tg->n_line + 1);
        MH_ALLOC(ctx, tg->line_w, std::max<int64_t>(woff[tg->n_line], 1));
        MH_CUDA(ctx, cudaMemcpyAsync(tg->line_woff.p, woff.data(), (tg->n_line + 1) * 8, cudaMemcpyHostToDevice, st));
        k_line_weights<<<mh_grid(tg->n_line * 32, 256), 256, 0, st>>>(tg->line_curve.p, tg->line_data.p, tg->n_line,
                                                                      b->d_nn.p, b->d_off.p, b->half.p,
                                                                      tg->line_woff.p, tg->line_w.p);
        MH_LAUNCHED(ctx);
    }
    if (tg->n_pairs) {
        MH_CUDA(ctx, cudaMemcpyAsync(tg->pair_tgt.p, pt.data(), tg->n_pairs * 4, cudaMemcpyHostToDevice, st));
        MH_CUDA(ctx, cudaMemcpyAsync(tg->pair_curve.p, pc.data(), tg->n_pairs * 4, cudaMemcpyHostToDevice, st));
    }
    MH_ALLOC(ctx, tg->ext, std::max<int64_t>(tg->n_ext, 1));
    MH_ALLOC(ctx, tg->sc, 2 * (b->n / 2 + b->n_curves));
    MH_ALLOC(ctx, tg->wf, b->n_fine);
    MH_ALLOC(ctx, tg->asig, b->n);
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    return MH_OK;
}

// binary32 source tables of the mixed-precision double layer (built once per boundary)
static mh_status prep_mixed(mh_ctx* ctx, mh_boundary* b) {
    if (b->src32.p) return MH_OK;
    cudaStream_t st = ctx->stream;
    b->n_tiles = (b->n + MH_TILE - 1) / MH_TILE;
    MH_ALLOC(ctx, b->src32, b->n);
    MH_ALLOC(ctx, b->tile_c, b->n_tiles);
    MH_ALLOC(ctx, b->tile_r, b->n_tiles);
    MH_ALLOC(ctx, b->w32, b->n);
    k_prep_src32<<<(unsigned)b->n_tiles, 128, 0, st>>>(b->geo.p, b->n, b->src32.p, b->tile_c.p, b->tile_r.p);
    MH_LAUNCHED(ctx);
    b->fchunk_off.assign(b->n_curves + 1, 0);
    for (int k = 0; k < b->n_curves; ++k)
        b->fchunk_off[k + 1] = b->fchunk_off[k] + (b->fine_off[k + 1] - b->fine_off[k] + MH_TILE - 1) / MH_TILE;
    b->n_fchunks = b->fchunk_off[b->n_curves];
    MH_ALLOC(ctx, b->d_fchunk_off, b->n_curves + 1);
    MH_ALLOC(ctx, b->fine32, b->n_fine);
    MH_ALLOC(ctx, b->fchunk_c, b->n_fchunks);
    MH_ALLOC(ctx, b->wf32, b->n_fine);
    MH_CUDA(ctx, cudaMemcpyAsync(b->d_fchunk_off.p, b->fchunk_off.data(), (b->n_curves + 1) * 8,
                                 cudaMemcpyHostToDevice, st));
    MH_ALLOC(ctx, b->fchunk_cf, b->n_fchunks);
    MH_ALLOC(ctx, b->fchunk_r, b->n_fchunks);
    if (!b->x32.p) MH_ALLOC(ctx, b->x32, b->n);
    MH_ALLOC(ctx, b->tw32, b->n);
    k_to_float_vec<<<mh_grid(2 * b->n, 256), 256, 0, st>>>(reinterpret_cast<const double*>(b->tw.p),
                                                            reinterpret_cast<float*>(b->tw32.p), 2 * b->n);
    MH_LAUNCHED(ctx);
    k_prep_fine32<<<(unsigned)b->n_fchunks, 128, 0, st>>>(b->fine_geo.p, b->d_fine_off.p, b->d_fchunk_off.p,
                                                          b->n_curves, b->fine32.p, b->fchunk_c.p,
                                                          b->fchunk_cf.p, b->fchunk_r.p);
    MH_LAUNCHED(ctx);
    MH_CUDA(ctx, cudaStreamSynchronize(st));
    return MH_OK;
}

static mh_status fine_density(mh_ctx* ctx, mh_boundary* b, const double* sc, mh_precision prec, float* wf32,
                              double* wf64);

mh_status dlp_evaluate(mh_ctx* ctx, mh_boundary* b, double alpha, dlp_targets* tg, const double* sigma,
                       double* out, mh_precision prec) {
    cudaStream_t st = ctx->stream;
    MH_TRY(bie_assemble(ctx, b, alpha));
    const double pref = -1.0 / (2.0 * MH_PI * alpha * alpha);
    const double pref32 = pref / (alpha * alpha);
    const mh_dl32 c32 = mh_dl32_make(alpha, MH_DL_CUT32);
    dbuf<double>& ext = tg->ext;
    dbuf<double>& sc = tg->sc;
    dbuf<double>& wf = tg->wf;
    dbuf<double>& asig = tg->asig;
    prof_scope ps_all(ctx, "dlp_evaluate");
    const int64_t nmodes = b->n / 2 + b->n_curves;
    if (prec == MH_PREC_MIXED) {
        MH_TRY(prep_mixed(ctx, b));
        k_weights32<<<mh_grid(b->n, 256), 256, 0, st>>>(sigma, b->geo.p, b->d_curve_of.p, b->d_nn.p, b->n, b->w32.p);
        MH_LAUNCHED(ctx);
        if (tg->n_ext) {
            prof_scope ps(ctx, "dlp_coarse", DL_FLOPS * tg->n_ext * b->n, 24.0 * (tg->n_ext + b->n));
            k_dlp_coarse32<<<mh_grid(tg->n_ext, MH_TILE), MH_TILE, 0, st>>>(
                tg->xy.p, tg->fine.p, tg->n_ext, b->src32.p, b->w32.p, b->d_curve_of.p, b->tile_c.p, b->tile_r.p, b->n,
                c32, pref32, ext.p);
            MH_LAUNCHED(ctx);
        }
        if (tg->n_pairs) {
            k_fourier_scalar<<<(unsigned)nmodes, 128, 0, st>>>(sigma, b->d_nn.p, b->d_off.p, b->tw.p, b->n_curves,
                                                               nmodes, sc.p);
            MH_LAUNCHED(ctx);
            MH_TRY(fine_density(ctx, b, sc.p, MH_PREC_MIXED, b->wf32.p, nullptr));
            prof_scope ps(ctx, "dlp_fine", DL_FLOPS * (tg->fine_nodes_main + tg->fine_nodes_aux), 24.0 * b->n_fine);
            k_dlp_fine32<<<mh_grid(tg->n_pairs * 32, 256), 256, 0, st>>>(
                tg->xy.p, tg->pair_tgt.p, tg->pair_curve.p, tg->n_pairs, b->fine32.p, b->wf32.p, b->d_fine_off.p,
                b->d_fchunk_off.p, b->fchunk_c.p, c32, pref32, ext.p);
            MH_LAUNCHED(ctx);
        }
    } else {
        if (tg->n_ext) {
            prof_scope ps(ctx, "dlp_coarse", DL_FLOPS * tg->n_ext * b->n, 24.0 * (tg->n_ext + b->n));
            k_dlp_coarse<128><<<mh_grid(tg->n_ext, 128), 128, 0, st>>>(tg->xy.p, tg->fine.p, tg->n_ext, b->geo.p,
                                                                       sigma, b->d_curve_of.p, b->d_nn.p, b->n,
                                                                       1.0 / alpha, pref, ext.p);
            MH_LAUNCHED(ctx);
        }
        if (tg->n_pairs) {
            k_fourier_scalar<<<(unsigned)nmodes, 128, 0, st>>>(sigma, b->d_nn.p, b->d_off.p, b->tw.p, b->n_curves,
                                                               nmodes, sc.p);
            MH_LAUNCHED(ctx);
            MH_TRY(fine_density(ctx, b, sc.p, MH_PREC_FP64, nullptr, wf.p));
            prof_scope ps(ctx, "dlp_fine", DL_FLOPS * (tg->fine_nodes_main + tg->fine_nodes_aux), 24.0 * b->n_fine);
            k_dlp_fine<<<mh_grid(tg->n_pairs * 32, 256), 256, 0, st>>>(tg->xy.p, tg->pair_tgt.p, tg->pair_curve.p,
                                                                       tg->n_pairs, b->fine_geo.p, wf.p,
                                                                       b->d_fine_off.p, 1.0 / alpha, pref, ext.p);
            MH_LAUNCHED(ctx);
        }
    }
    if (tg->n_line) {
        MH_TRY(bie_apply(ctx, b, sigma, asig.p, MH_PREC_FP64));
        k_dlp_line<<<mh_grid(tg->n_line * 32, 256), 256, 0, st>>>(tg->line_tgt.p, tg->line_curve.p, tg->line_data.p,
                                                                  tg->n_line, asig.p, b->d_nn.p, b->d_off.p,
                                                                  tg->line_w.p, tg->line_woff.p, tg->n, alpha,
                                                                  ext.p);
        MH_LAUNCHED(ctx);
    }
    if (tg->n) MH_CUDA(ctx, cudaMemcpyAsync(out, ext.p, tg->n * 8, cudaMemcpyDeviceToDevice, st));
    return MH_OK;
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

// Density times |y'| h_f on the 16x fine grid from the density's Fourier coefficients sc
// (binary64): into wf32 (mixed) or wf64 (binary64).
static mh_status fine_density(mh_ctx* ctx, mh_boundary* b, const double* sc, mh_precision prec, float* wf32,
                              double* wf64) {
    cudaStream_t st = ctx->stream;
    const int64_t nmodes = b->n / 2 + b->n_curves;
    const int max_n = *std::max_element(b->n_nodes.begin(), b->n_nodes.end());
    const dim3 grid((unsigned)((max_n + 15) / 16), (unsigned)b->n_curves);
    if (prec == MH_PREC_MIXED) {
        if (!b->fcp32.p) MH_ALLOC(ctx, b->fcp32, nmodes * UPSAMPLE);
        k_fine_coef<float2><<<mh_grid(nmodes * UPSAMPLE, 256), 256, 0, st>>>(sc, b->d_nn.p, b->d_off.p, b->n_curves,
                                                                             nmodes, b->fcp32.p);
        MH_LAUNCHED(ctx);
        bool pow2 = max_n <= FFT_MAX;
        for (int nk : b->n_nodes) pow2 = pow2 && nk >= 2 && (nk & (nk - 1)) == 0;
        if (pow2)
            k_fine_density_fft<<<dim3(UPSAMPLE, (unsigned)b->n_curves), 256, 2 * max_n * sizeof(float2), st>>>(
                b->fcp32.p, b->tw32.p, b->fine_geo.p, b->d_nn.p, b->d_off.p, b->d_fine_off.p, wf32);
        else
            k_fine_density_s<float, float2><<<grid, 256, max_n * sizeof(float2), st>>>(
                b->fcp32.p, b->tw32.p, b->fine_geo.p, b->d_nn.p, b->d_off.p, b->d_fine_off.p, wf32);
    } else {
        if (!b->fcp64.p) MH_ALLOC(ctx, b->fcp64, nmodes * UPSAMPLE);
        k_fine_coef<double2><<<mh_grid(nmodes * UPSAMPLE, 256), 256, 0, st>>>(sc, b->d_nn.p, b->d_off.p, b->n_curves,
                                                                              nmodes, b->fcp64.p);
        MH_LAUNCHED(ctx);
        k_fine_density_s<double, double2><<<grid, 256, max_n * sizeof(double2), st>>>(
            b->fcp64.p, b->tw.p, b->fine_geo.p, b->d_nn.p, b->d_off.p, b->d_fine_off.p, wf64);
    }
    MH_LAUNCHED(ctx);
    return MH_OK;
}

mh_status dlp_fine_weights(mh_ctx* ctx, mh_boundary* b, const double* sigma, mh_precision prec) {
    cudaStream_t st = ctx->stream;
    const int64_t nmodes = b->n / 2 + b->n_curves;
    if (!b->sc64.p) {
        MH_ALLOC(ctx, b->sc64, 2 * nmodes);
        MH_ALLOC(ctx, b->wf64, b->n_fine);
    }
    const int max_n = *std::max_element(b->n_nodes.begin(), b->n_nodes.end());
    bool pow2 = max_n <= FFT_MAX;
    for (int nk : b->n_nodes) pow2 = pow2 && nk >= 2 && (nk & (nk - 1)) == 0;
    if (prec == MH_PREC_MIXED && pow2) {
        // binary32 FFTs both ways in one launch
        MH_TRY(prep_mixed(ctx, b));
        k_fine_weights_fft<<<dim3(UPSAMPLE, (unsigned)b->n_curves), 256, 2 * max_n * sizeof(float2), st>>>(
            sigma, b->tw32.p, b->fine_geo.p, b->d_nn.p, b->d_off.p, b->d_fine_off.p, b->wf32.p, b->wf64.p);
        MH_LAUNCHED(ctx);
    } else if (prec == MH_PREC_MIXED) {
        MH_TRY(prep_mixed(ctx, b));
        k_to_float_vec<<<mh_grid(b->n, 256), 256, 0, st>>>(sigma, b->x32.p, b->n);
        MH_LAUNCHED(ctx);
        k_fourier_scalar32<<<(unsigned)nmodes, 128, 0, st>>>(b->x32.p, b->d_nn.p, b->d_off.p, b->tw32.p, b->n_curves,
                                                             nmodes, b->sc64.p);
        MH_LAUNCHED(ctx);
        MH_TRY(fine_density(ctx, b, b->sc64.p, MH_PREC_MIXED, b->wf32.p, nullptr));
        k_f2d<<<mh_grid(b->n_fine, 256), 256, 0, st>>>(b->wf32.p, b->wf64.p, b->n_fine);
        MH_LAUNCHED(ctx);
    } else {
        k_fourier_scalar<<<(unsigned)nmodes, 128, 0, st>>>(sigma, b->d_nn.p, b->d_off.p, b->tw.p, b->n_curves,
                                                           nmodes, b->sc64.p);
        MH_LAUNCHED(ctx);
        MH_TRY(fine_density(ctx, b, b->sc64.p, MH_PREC_FP64, nullptr, b->wf64.p));
    }
    return MH_OK;
}

mh_status dlp_evaluate_fmm_tail(mh_ctx* ctx, mh_boundary* b, double alpha, dlp_targets* tg, const double* sigma,
                                const double* main_vals, double* out, mh_precision prec, bool fine_in_fmm,
                                const double* asig_given, int part) {
    if (part != 0 && !fine_in_fmm) return mh_fail(ctx, MH_ERR_INVALID_ARG, "a split tail needs the fine rule in the passes");
    const bool do_aux = part != 2, do_finish = part != 1;
    cudaStream_t st = ctx->stream;
    const double pref = -1.0 / (2.0 * MH_PI * alpha * alpha);
    const double pref32 = pref / (alpha * alpha);
    const mh_dl32 c32 = mh_dl32_make(alpha, MH_DL_CUT32);
    const int64_t n = tg->n, naux = tg->n_ext - tg->n;
    const int64_t np_main = tg->n_pairs_main, np_aux = tg->n_pairs - tg->n_pairs_main;
    dbuf<double>& ext = tg->ext;
    dbuf<double>& sc = tg->sc;
    dbuf<double>& wf = tg->wf;
    prof_scope ps_all(ctx, "dlp_evaluate");
    // ext[0, n): the given values at the targets; ext[n, n_ext): the auxiliary points, written
    // only by the auxiliary part (part 1), so that part can run beside the work that produces
    // main_vals
    if (do_finish && n) MH_CUDA(ctx, cudaMemcpyAsync(ext.p, main_vals, n * 8, cudaMemcpyDeviceToDevice, st));
    if (do_aux) {
        const int64_t np_do_main = fine_in_fmm ? 0 : np_main;
        if (tg->n_pairs && !fine_in_fmm) MH_TRY(dlp_fine_weights(ctx, b, sigma, prec));
        (void)sc;
        (void)wf;
        if (prec == MH_PREC_MIXED) {
            MH_TRY(prep_mixed(ctx, b));
            k_weights32<<<mh_grid(b->n, 256), 256, 0, st>>>(sigma, b->geo.p, b->d_curve_of.p, b->d_nn.p, b->n, b->w32.p);
            MH_LAUNCHED(ctx);
            if (naux) {
                // few auxiliary points: split the sources over the grid, then reduce in a fixed order
                const int64_t nblk = (naux + MH_TILE - 1) / MH_TILE;
                const int64_t ntile = (b->n + MH_TILE - 1) / MH_TILE;
                const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(ntile, (152 * 8) / std::max<int64_t>(nblk, 1)));
                if ((int64_t)tg->part.n < nsplit * naux) MH_ALLOC(ctx, tg->part, nsplit * naux);
                k_dlp_coarse32<<<dim3((unsigned)nblk, (unsigned)nsplit), MH_TILE, 0, st>>>(
                    tg->xy.p + 2 * n, tg->fine.p + n, naux, b->src32.p, b->w32.p, b->d_curve_of.p, b->tile_c.p, b->tile_r.p, b->n,
                    c32, pref32, nsplit > 1 ? tg->part.p : ext.p + n);
                MH_LAUNCHED(ctx);
                if (nsplit > 1) {
                    k_sum_partials<<<mh_grid(naux, 256), 256, 0, st>>>(tg->part.p, nsplit, naux, pref32, ext.p + n);
                    MH_LAUNCHED(ctx);
                }
            }
            if (tg->n_pairs) {
                prof_scope ps(ctx, "dlp_fine", DL_FLOPS * ((fine_in_fmm ? 0 : tg->fine_nodes_main + tg->curve_nodes_main) + tg->fine_nodes_aux), 24.0 * b->n_fine);
                if (np_do_main) {
                    k_dlp_fine_corr32<<<mh_grid(np_do_main * 32, 256), 256, 0, st>>>(
                        tg->xy.p, tg->pair_tgt.p, tg->pair_curve.p, np_do_main, b->fine32.p, b->wf32.p, b->d_fine_off.p,
                        b->d_fchunk_off.p, b->fchunk_c.p, b->src32.p, b->w32.p, b->tile_c.p, b->d_off.p,
                        c32, pref32, ext.p);
                    MH_LAUNCHED(ctx);
                }
                if (np_aux) {
                    k_dlp_fine32_grp<FINE_TG><<<(unsigned)(tg->n_groups * tg->fine_slices), 256, 0, st>>>(
                        tg->xy.p, tg->pair_tgt.p, tg->grp_curve.p, tg->grp_pair.p, tg->fine_slices, b->fine32.p,
                        b->wf32.p, b->d_fine_off.p, b->d_fchunk_off.p, b->fchunk_cf.p, b->fchunk_r.p, c32,
                        (float)(MH_DL_CUT32 * alpha), pref32, tg->grp_part.p, tg->grp_cnt.p, ext.p);
                    MH_LAUNCHED(ctx);
                }
            }
        } else {
            if (naux) {
                const int64_t nblk = (naux + 127) / 128, ntile = (b->n + 127) / 128;
                const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(ntile, (152 * 8) / std::max<int64_t>(nblk, 1)));
                if ((int64_t)tg->part.n < nsplit * naux) MH_ALLOC(ctx, tg->part, nsplit * naux);
                k_dlp_coarse<128><<<dim3((unsigned)nblk, (unsigned)nsplit), 128, 0, st>>>(
                    tg->xy.p + 2 * n, tg->fine.p + n, naux, b->geo.p, sigma, b->d_curve_of.p, b->d_nn.p, b->n, 1.0 / alpha,
                    pref, nsplit > 1 ? tg->part.p : ext.p + n);
                MH_LAUNCHED(ctx);
                if (nsplit > 1) {
                    k_sum_partials<<<mh_grid(naux, 256), 256, 0, st>>>(tg->part.p, nsplit, naux, pref, ext.p + n);
                    MH_LAUNCHED(ctx);
                }
            }
            if (tg->n_pairs) {
                prof_scope ps(ctx, "dlp_fine", DL_FLOPS * ((fine_in_fmm ? 0 : tg->fine_nodes_main + tg->curve_nodes_main) + tg->fine_nodes_aux), 24.0 * b->n_fine);
                if (np_do_main) {
                    k_dlp_fine_corr<<<mh_grid(np_do_main * 32, 256), 256, 0, st>>>(
                        tg->xy.p, tg->pair_tgt.p, tg->pair_curve.p, np_do_main, b->fine_geo.p, b->wf64.p,
                        b->d_fine_off.p, b->geo.p, sigma, b->d_nn.p, b->d_off.p, 1.0 / alpha, pref, ext.p);
                    MH_LAUNCHED(ctx);
                }
                if (np_aux) {
                    k_dlp_fine64_blk<<<(unsigned)np_aux, 256, 0, st>>>(tg->xy.p, tg->pair_tgt.p + np_main,
                                                                       tg->pair_curve.p + np_main, b->fine_geo.p,
                                                                       b->wf64.p, b->d_fine_off.p, 1.0 / alpha, pref,
                                                                       ext.p);
                    MH_LAUNCHED(ctx);
                }
            }
        }
    }
    if (!do_finish) return MH_OK;
    if (tg->n_line) {
        // the interior limit needs A sigma; a caller that holds the residual r = rhs - A sigma
        // of this density passes A sigma = rhs - r instead of a product with the operator
        const double* asig = asig_given;
        if (!asig) {
            MH_TRY(bie_apply(ctx, b, sigma, tg->asig.p, prec));
            asig = tg->asig.p;
        }
        k_dlp_line<<<mh_grid(tg->n_line * 32, 256), 256, 0, st>>>(tg->line_tgt.p, tg->line_curve.p, tg->line_data.p,
                                                                  tg->n_line, asig, b->d_nn.p, b->d_off.p,
                                                                  tg->line_w.p, tg->line_woff.p, tg->n, alpha,
                                                                  ext.p);
        MH_LAUNCHED(ctx);
    }
    if (n) MH_CUDA(ctx, cudaMemcpyAsync(out, ext.p, n * 8, cudaMemcpyDeviceToDevice, st));
    return MH_OK;
}

extern "C" mh_status mh_double_layer_apply(mh_ctx* ctx, mh_boundary* b, double alpha, const double* sigma_dev,
                                           const double* targets_dev, int64_t n_targets, double* out_dev,
                                           mh_precision prec) {
    if (!ctx || !b || !sigma_dev || !out_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (!(alpha > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "alpha must be positive");
    MH_TRY(bie_assemble(ctx, b, alpha));
    if (!targets_dev) {
        MH_TRY(bie_apply(ctx, b, sigma_dev, out_dev, prec));
        MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return MH_OK;
    }
    if (n_targets < 0) return mh_fail(ctx, MH_ERR_INVALID_ARG, "n_targets < 0");
    if (n_targets == 0) return MH_OK;   // no targets: nothing to evaluate, out_dev untouched
    dlp_targets tg;
    MH_TRY(dlp_classify(ctx, b, targets_dev, n_targets, &tg));
    MH_TRY(dlp_evaluate(ctx, b, alpha, &tg, sigma_dev, out_dev, prec));
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return MH_OK;
}

extern "C" mh_status mh_gmres_solve(mh_ctx* ctx, mh_boundary* b, double alpha, const double* rhs_dev,
                                    double* sigma_dev, double tol, int max_iter, mh_precision prec,
                                    mh_gmres_info* info) {
    if (!ctx || !b || !rhs_dev || !sigma_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (!(alpha > 0) || !(tol > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "alpha and tol must be positive");
    MH_TRY(bie_assemble(ctx, b, alpha));
    return gmres_run(ctx, b, rhs_dev, sigma_dev, tol, max_iter, prec, info);
}

// ---------------------------------------------------------------------------------------
// Allocation-free GMRES.  Some callers cannot call cudaMalloc while they solve: code that
// runs under a memory budget fixed in advance, or inside a host loop whose allocator is
// owned by another framework, and must not grow or free device memory between calls.
// mh_gmres_solve_static gives them the binary64 solve with its Krylov workspace taken from
// a fixed array compiled into the library instead of allocated memory.
// ---------------------------------------------------------------------------------------

#define MH_STATIC_N 8192   // largest N_Gamma
#define MH_STATIC_M 64     // largest max_iter
#define MH_STATIC_SMALL (MH_STATIC_M + 2)

// Workspace layout (doubles): V[(M+1) N] | w[N] | H[(M+1) M] | cs, sn, g, y, h1, h2 [M+2 each] | small[4]
#define MH_STATIC_DOUBLES                                                                               \
    ((size_t)(MH_STATIC_M + 1) * MH_STATIC_N + MH_STATIC_N + (size_t)(MH_STATIC_M + 1) * MH_STATIC_M + \
     6 * MH_STATIC_SMALL + 4)

// 4.4 MB held by every device that loads the library, until the process exits.
static __device__ __align__(256) double g_gmres_scratch[MH_STATIC_DOUBLES];

// Device address of g_gmres_scratch per device, looked up once with that device current.
// The lookup table is guarded by a mutex: host threads may make their first call at once.
static double* g_scratch_addr[64];
static bool g_scratch_ready[64];
static std::mutex g_scratch_mutex;

static mh_status static_scratch(mh_ctx* ctx, double** out) {
    if (ctx->device < 0 || ctx->device >= 64) return mh_fail(ctx, MH_ERR_INVALID_ARG, "device id out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ready[ctx->device]) {
        int cur = 0;
        MH_CUDA(ctx, cudaGetDevice(&cur));
        if (cur != ctx->device) MH_CUDA(ctx, cudaSetDevice(ctx->device));
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_gmres_scratch);
        const cudaError_t back = cur != ctx->device ? cudaSetDevice(cur) : cudaSuccess;
        if (e != cudaSuccess)
            return mh_fail(ctx, MH_ERR_CUDA, "cudaGetSymbolAddress(g_gmres_scratch) failed: %s", cudaGetErrorString(e));
        if (back != cudaSuccess)
            return mh_fail(ctx, MH_ERR_CUDA, "restoring the caller's device %d failed: %s", cur,
                           cudaGetErrorString(back));
        g_scratch_addr[ctx->device] = static_cast<double*>(p);
        g_scratch_ready[ctx->device] = true;
    }
    *out = g_scratch_addr[ctx->device];
    return MH_OK;
}

extern "C" mh_status mh_gmres_solve_static(mh_ctx* ctx, mh_boundary* bd, double alpha, const double* rhs_dev,
                                           double* sigma_dev, double tol, int max_iter, mh_gmres_info* info) {
    if (!ctx || !bd || !rhs_dev || !sigma_dev) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    if (!(tol > 0)) return mh_fail(ctx, MH_ERR_INVALID_ARG, "tol must be positive");
    const int64_t n = bd->n;
    if (n > MH_STATIC_N)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "N_Gamma = %lld exceeds the static workspace limit %d",
                       (long long)n, MH_STATIC_N);
    if (max_iter < 1 || max_iter > MH_STATIC_M)
        return mh_fail(ctx, MH_ERR_INVALID_ARG, "max_iter must be in 1..%d for the static workspace", MH_STATIC_M);
    if (!(bd->op.A64.p && bd->op.alpha == alpha))
        return mh_fail(ctx, MH_ERR_INVALID_ARG,
                       "the operator for this alpha is not assembled: call mh_gmres_solve or "
                       "mh_double_layer_apply with this alpha first (they allocate it)");
    double* base = nullptr;
    MH_TRY(static_scratch(ctx, &base));
    const int M = max_iter, ldh = M + 1;
    double* V = base;
    double* w = V + (size_t)(MH_STATIC_M + 1) * MH_STATIC_N;
    double* H = w + MH_STATIC_N;
    double* cs = H + (size_t)(MH_STATIC_M + 1) * MH_STATIC_M;
    double* sn = cs + MH_STATIC_SMALL;
    double* g = sn + MH_STATIC_SMALL;
    double* y = g + MH_STATIC_SMALL;
    double* h1 = y + MH_STATIC_SMALL;
    double* h2 = h1 + MH_STATIC_SMALL;
    double* small = h2 + MH_STATIC_SMALL;
    cudaStream_t st = ctx->stream;
    const int ew = mh_grid(n, 256) < 152 * 4 ? mh_grid(n, 256) : 152 * 4;
    // the array keeps the previous call's contents: clear what the iteration reads first
    MH_CUDA(ctx, cudaMemsetAsync(g, 0, MH_STATIC_SMALL * sizeof(double), st));
    mh_gmres_info inf{0, 0, 0.0, 0, 0.0};
    double bnorm;
    MH_TRY(vec_norm(ctx, rhs_dev, n, small + 2, &bnorm));
    if (bnorm == 0.0) {
        MH_CUDA(ctx, cudaMemsetAsync(sigma_dev, 0, n * 8, st));
        inf.converged = 1;
        if (info) *info = inf;
        return MH_OK;
    }
    MH_TRY(bie_apply(ctx, bd, sigma_dev, w, MH_PREC_FP64));
    k_sub_from<<<ew, 256, 0, st>>>(rhs_dev, w, n);
    MH_LAUNCHED(ctx);
    double beta;
    MH_TRY(vec_norm(ctx, w, n, small + 1, &beta));
    inf.initial_rel_residual = beta / bnorm;
    int k = 0;
    if (beta > tol * bnorm) {
        k_scale_into<<<ew, 256, 0, st>>>(w, small + 1, V, g, n);
        MH_LAUNCHED(ctx);
        double res = beta;
        for (; k < M; ++k) {
            MH_TRY(bie_apply(ctx, bd, V + (int64_t)k * n, w, MH_PREC_FP64));
            k_multidot<<<k + 1, 256, 0, st>>>(V, w, n, h1);
            MH_LAUNCHED(ctx);
            k_multiaxpy<<<ew, 256, 0, st>>>(V, h1, k + 1, n, w);
            MH_LAUNCHED(ctx);
            k_multidot<<<k + 1, 256, 0, st>>>(V, w, n, h2);
            MH_LAUNCHED(ctx);
            k_multiaxpy<<<ew, 256, 0, st>>>(V, h2, k + 1, n, w);
            MH_LAUNCHED(ctx);
            k_norm<<<1, 1024, 0, st>>>(w, n, small + 1);
            MH_LAUNCHED(ctx);
            k_finish_column<<<ew, 256, 0, st>>>(h1, h2, small + 1, k, H + (int64_t)k * ldh, w, V + (int64_t)(k + 1) * n,
                                                n);
            MH_LAUNCHED(ctx);
            k_givens<<<1, 1, 0, st>>>(H, ldh, k, cs, sn, g, small);
            MH_LAUNCHED(ctx);
            MH_CUDA(ctx, cudaMemcpyAsync(&res, small, 8, cudaMemcpyDeviceToHost, st));
            MH_CUDA(ctx, cudaStreamSynchronize(st));
            if (!std::isfinite(res)) return mh_fail(ctx, MH_ERR_NUMERIC, "GMRES residual is not finite");
            if (res <= tol * bnorm) {
                ++k;
                break;
            }
        }
        k_backsolve<<<1, 1, 0, st>>>(H, ldh, k, g, y);
        MH_LAUNCHED(ctx);
        k_update_x<<<ew, 256, 0, st>>>(V, y, k, n, sigma_dev);
        MH_LAUNCHED(ctx);
    }
    inf.iterations = k;
    MH_TRY(bie_apply(ctx, bd, sigma_dev, w, MH_PREC_FP64));
    k_sub_from<<<ew, 256, 0, st>>>(rhs_dev, w, n);
    MH_LAUNCHED(ctx);
    double rn;
    MH_TRY(vec_norm(ctx, w, n, small + 2, &rn));
    inf.rel_residual = rn / bnorm;
    inf.converged = inf.rel_residual <= tol;
    if (info) *info = inf;
    if (!inf.converged)
        return mh_fail(ctx, MH_ERR_NOT_CONVERGED, "GMRES stopped after %d iterations at relative residual %.3e",
                       inf.iterations, inf.rel_residual);
    return MH_OK;
}
