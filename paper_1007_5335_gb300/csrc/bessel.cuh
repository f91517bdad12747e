// Modified Bessel functions K0 and K1 on the device, binary64 and binary32.
//
// G(r) = K0(r/alpha) / (2 pi alpha^2) is the Green's function of 1 - alpha^2 Lap
// (Section 2) and (1/alpha) K1(r/alpha) enters the double-layer kernel (Section 3.2).
//   z <= 2 : power series (Abramowitz & Stegun 9.6.10, 9.6.11, 9.6.13)
//              K0(z) = -(ln(z/2) + gamma) I0(z) + sum_{k>=1} H_k (z^2/4)^k / (k!)^2
//              K1(z) = 1/z + ln(z/2) I1(z) - (z/4) sum_k (psi(k+1)+psi(k+2)) (z^2/4)^k / (k!(k+1)!)
//   z > 2  : K_nu(z) = e^{-z} / sqrt(z) * C_nu(4/z - 1), C_nu a Chebyshev interpolant
//            (own fit, see gen_constants.py) evaluated by Clenshaw's recurrence.
// The library calls log, exp and rsqrt; it does not re-implement them.
#pragma once

#include <cmath>

#include "bessel_coefs.h"

__device__ __forceinline__ double mh_clenshaw(const double* c, int n, double x) {
    double b1 = 0.0, b2 = 0.0;
    const double x2 = 2.0 * x;
    for (int k = n - 1; k >= 1; --k) {
        double t = fma(x2, b1, c[k] - b2);
        b2 = b1;
        b1 = t;
    }
    return fma(x, b1, c[0] - b2);
}

__device__ __forceinline__ float mh_clenshaw_f(const float* c, int n, float x) {
    float b1 = 0.f, b2 = 0.f;
    const float x2 = 2.f * x;
    for (int k = n - 1; k >= 1; --k) {
        float t = fmaf(x2, b1, c[k] - b2);
        b2 = b1;
        b1 = t;
    }
    return fmaf(x, b1, c[0] - b2);
}

// ---- binary64 ----
__device__ __forceinline__ double mh_k0(double z) {
    if (z <= 2.0) {
        const double y = 0.25 * z * z;
        double s_i = mh_ser_i0[MH_BESSEL_NSER - 1], s_h = mh_ser_k0h[MH_BESSEL_NSER - 1];
        for (int k = MH_BESSEL_NSER - 2; k >= 0; --k) {
            s_i = fma(s_i, y, mh_ser_i0[k]);
            s_h = fma(s_h, y, mh_ser_k0h[k]);
        }
        return s_h - (log(0.5 * z) + MH_EULER_GAMMA) * s_i;
    }
    return exp(-z) * rsqrt(z) * mh_clenshaw(mh_cheb_k0, MH_CHEB_K0_N64, 4.0 / z - 1.0);
}

__device__ __forceinline__ double mh_k1(double z) {
    if (z <= 2.0) {
        const double y = 0.25 * z * z;
        double s_i = mh_ser_i1[MH_BESSEL_NSER - 1], s_p = mh_ser_k1p[MH_BESSEL_NSER - 1];
        for (int k = MH_BESSEL_NSER - 2; k >= 0; --k) {
            s_i = fma(s_i, y, mh_ser_i1[k]);
            s_p = fma(s_p, y, mh_ser_k1p[k]);
        }
        return 1.0 / z + log(0.5 * z) * (0.5 * z) * s_i - 0.25 * z * s_p;
    }
    return exp(-z) * rsqrt(z) * mh_clenshaw(mh_cheb_k1, MH_CHEB_K1_N64, 4.0 / z - 1.0);
}

// ---- binary32 ----
__device__ __forceinline__ float mh_k0f(float z) {
    if (z <= 2.f) {
        const float y = 0.25f * z * z;
        float s_i = mh_ser_i0_f[MH_BESSEL_NSER_F - 1], s_h = mh_ser_k0h_f[MH_BESSEL_NSER_F - 1];
#pragma unroll
        for (int k = MH_BESSEL_NSER_F - 2; k >= 0; --k) {
            s_i = fmaf(s_i, y, mh_ser_i0_f[k]);
            s_h = fmaf(s_h, y, mh_ser_k0h_f[k]);
        }
        return s_h - (__logf(0.5f * z) + (float)MH_EULER_GAMMA) * s_i;
    }
    return __expf(-z) * rsqrtf(z) * mh_clenshaw_f(mh_cheb_k0_f, MH_CHEB_K0_N32, 4.f / z - 1.f);
}

// K1 with 1/z supplied by the caller (the pair kernels have it from their rsqrt: 1/z = alpha/r),
// so that neither branch divides.
__device__ __forceinline__ float mh_k1f_r(float z, float zinv) {
    if (z <= 2.f) {
        const float y = 0.25f * z * z;
        float s_i = mh_ser_i1_f[MH_BESSEL_NSER_F - 1], s_p = mh_ser_k1p_f[MH_BESSEL_NSER_F - 1];
#pragma unroll
        for (int k = MH_BESSEL_NSER_F - 2; k >= 0; --k) {
            s_i = fmaf(s_i, y, mh_ser_i1_f[k]);
            s_p = fmaf(s_p, y, mh_ser_k1p_f[k]);
        }
        return zinv + __logf(0.5f * z) * (0.5f * z) * s_i - 0.25f * z * s_p;
    }
    return __expf(-z) * rsqrtf(z) * mh_clenshaw_f(mh_cheb_k1_f, MH_CHEB_K1_N32, fmaf(4.f, zinv, -1.f));
}

__device__ __forceinline__ float mh_k1f(float z) { return mh_k1f_r(z, __frcp_rn(z)); }

// ---- the binary32 double-layer pair term ----
// (1/alpha) K1(r/alpha) (d.n)/r = g(z) (d.n) / alpha^2 with g(z) = K1(z)/z, z = r/alpha
// (Section 3.2).  Written as g, the pair needs neither r nor a division: z <= 2 is decided on
// r^2, the series runs in y = z^2/4 = r^2/(4 alpha^2) and 1/z = alpha/r comes from the
// pair's rsqrt.  Callers fold 1/alpha^2 into their binary64 prefactor.
//   z <= 2 : g = 1/z^2 + log2(y) A(y) - B(y)       (the K1 series of A&S 9.6.11 over z)
//   z > 2  : g = e^{-z} z^{-3/2} M(4/z - 1)         (M: the K1 interpolant, monomial basis)
struct mh_dl32 {
    float ia;        // 1/alpha
    float a;         // alpha
    float y_r2;      // 1/(4 alpha^2)
    float r2_small;  // (2 alpha)^2
    float r2_cut;    // (cut alpha)^2: farther pairs are below the binary32 rounding of a sum
    float a4;        // 4 alpha
    float ml2e_ia;   // -log2(e) / alpha
    float a32;       // alpha^{3/2}
};

inline mh_dl32 mh_dl32_make(double alpha, double cut) {
    mh_dl32 c;
    c.ia = (float)(1.0 / alpha);
    c.a = (float)alpha;
    c.y_r2 = (float)(0.25 / (alpha * alpha));
    c.r2_small = (float)(4.0 * alpha * alpha);
    c.r2_cut = (float)(cut * cut * alpha * alpha);
    c.a4 = (float)(4.0 * alpha);
    c.ml2e_ia = (float)(-1.4426950408889634 / alpha);
    c.a32 = (float)(alpha * std::sqrt(alpha));
    return c;
}

// The hardware's approximate special-function instructions (PTX rsqrt / lg2 / ex2 .approx)
// with subnormal inputs and results flushed to zero: the pair kernels' arguments are normal
// (r^2 is floored at 1e-30, y = r^2/(4 alpha^2) > 0) and a flushed e^{-z} is a pair far below
// the rounding of any sum, so the flush changes no result and saves the subnormal handling.
// e^{-z} is 2^{-z log2(e)}.
__device__ __forceinline__ float mh_rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mh_lg2_ftz(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mh_ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mh_sqrt_ftz(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
#define MH_LOG2E_F 1.4426950408889634f   // log2(e)

// g(z) for z <= 2 from y = z^2/4 and 1/z
__device__ __forceinline__ float mh_k1oz_small_f(float y, float zinv) {
    float a = mh_k1oz_a_f[MH_K1OZ_NA_F - 1], b = mh_k1oz_b_f[MH_K1OZ_NB_F - 1];
#pragma unroll
    for (int k = MH_K1OZ_NB_F - 2; k >= 0; --k) {
        b = fmaf(b, y, mh_k1oz_b_f[k]);
        if (k < MH_K1OZ_NA_F - 1) a = fmaf(a, y, mh_k1oz_a_f[k]);
    }
    return fmaf(zinv, zinv, fmaf(mh_lg2_ftz(y), a, -b));
}

// g(z) for z > 2 from z and 1/z
__device__ __forceinline__ float mh_k1oz_large_f(float z, float zinv) {
    const float x = fmaf(4.f, zinv, -1.f);
    float m = mh_k1_mono_f[MH_K1_MONO_N32 - 1];
#pragma unroll
    for (int k = MH_K1_MONO_N32 - 2; k >= 0; --k) m = fmaf(m, x, mh_k1_mono_f[k]);
    return mh_ex2_ftz(-MH_LOG2E_F * z) * mh_rsqrt_ftz(z) * zinv * m;
}

// g(r/alpha) (dx nx + dy ny) for the offset (dx, dy) of a source from a target, without the
// tests of mh_dl32_pair: coincident points give 0 through the zero offset (r^2 is floored at
// 1e-30, so g stays finite), and pairs far beyond the cut come out below the binary32 rounding
// of any sum (e^{-z} underflows).  For loops whose pairs are near by construction.
__device__ __forceinline__ float mh_dl32_pair_nt(float dx, float dy, float nx, float ny, const mh_dl32& c) {
    const float r2 = fmaxf(fmaf(dx, dx, dy * dy), 1e-30f);
    const float rinv = mh_rsqrt_ftz(r2);
    const float zinv = c.a * rinv;
    const float g = r2 <= c.r2_small ? mh_k1oz_small_f(r2 * c.y_r2, zinv)
                                     : mh_k1oz_large_f(r2 * rinv * c.ia, zinv);
    return g * fmaf(dx, nx, dy * ny);
}

// g(r/alpha) (dx nx + dy ny) for the offset (dx, dy) of a source from a target; 0 for
// coincident points and beyond the cut.
__device__ __forceinline__ float mh_dl32_pair(float dx, float dy, float nx, float ny, const mh_dl32& c) {
    const float r2 = fmaf(dx, dx, dy * dy);
    if (!(r2 >= 1e-30f && r2 <= c.r2_cut)) return 0.f;   // r < 1e-15: coincident in binary32 offsets
    const float rinv = mh_rsqrt_ftz(r2);
    const float zinv = c.a * rinv;
    const float g = r2 <= c.r2_small ? mh_k1oz_small_f(r2 * c.y_r2, zinv)
                                     : mh_k1oz_large_f(r2 * rinv * c.ia, zinv);
    return g * fmaf(dx, nx, dy * ny);
}

// g(r/alpha) (dx nx + dy ny) / alpha^{3/2} for a pair known to have r > 2 alpha (no branch):
// with z = r/alpha, e^{-z} z^{-3/2} = alpha^{3/2} e^{-r/alpha} r^{-3/2}, so the pair needs no
// z and no 1/z: x = 4 alpha / r - 1, e^{-z} = 2^{-log2(e) r / alpha}, r^{-3/2} = r^{-1}
// sqrt(1/r).  Callers multiply their sums by alpha^{3/2} (c.a32).
__device__ __forceinline__ float mh_dl32_pair_far(float dx, float dy, float nx, float ny, const mh_dl32& c) {
    const float r2 = fmaf(dx, dx, dy * dy);
    const float rinv = mh_rsqrt_ftz(r2);
    const float x = fmaf(c.a4, rinv, -1.f);
    float m = mh_k1_mono_f[MH_K1_MONO_N32 - 1];
#pragma unroll
    for (int k = MH_K1_MONO_N32 - 2; k >= 0; --k) m = fmaf(m, x, mh_k1_mono_f[k]);
    const float e = mh_ex2_ftz(r2 * rinv * c.ml2e_ia);
    return e * mh_sqrt_ftz(rinv) * rinv * m * fmaf(dx, nx, dy * ny);
}
