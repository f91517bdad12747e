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
