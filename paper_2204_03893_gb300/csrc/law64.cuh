// law64.cuh -- the conductivity law k(u), k'(u) in FP64 for the FP64
// element kernels, specialised at compile time on the law so that no FP64
// operation is spent on unused parameters (FP64 throughput on GB300 is about
// 2 fused multiply-adds per clock and SM, so these counts set the FP64
// path's speed).
//
// Law codes: 0..7 = polynomial with 1..8 coefficients, LAW_SIN = sine law,
// LAW_PWLIN = piecewise-linear law (the FEM_K_* laws of fem.h).
#pragma once
#include <cstdint>

#include "fem_device.cuh"

namespace fem {

constexpr int LAW_SIN = 8;
constexpr int LAW_PWLIN = 9;
constexpr int LAW_COUNT = 10;

// law code of a law in device form (the host validated it)
__host__ __device__ inline int law_code(const CoeffDev& k) {
    return k.kind == 0 ? (k.n >= 1 && k.n <= 8 ? k.n - 1 : 7) : k.kind == 1 ? LAW_SIN : LAW_PWLIN;
}

// ------------------------------------------------------------------ sine law
// sin x and cos x by table lookup and short Taylor polynomials (the
// table-driven method of Tang, and of Gal and Bachelis' accurate tables).
// x is split as k (pi/512) + h with k = rint(x 512/pi) and |h| <= pi/1024 (a
// little more after rounding).  k comes from one fused multiply-add with
// 1.5 2^52, which leaves rint(x 512/pi) in the low bits of the sum (read
// with an integer move; one subtraction gives it as a double), and the
// range test is an integer test of x's exponent, so the reduction takes 4
// FP64 operations.  The subtraction is done in two pieces (Cody and Waite):
// pi/512 = SC_HI + SC_LO with SC_HI holding 33 significant bits, so k SC_HI
// is exact and x - k SC_HI is exact (Sterbenz) for |k| < 2^20.  Then
//     sin h = h - h^3/3! + h^5/5!                    (next term < 2e-19 |h|)
//     cos h - 1 = -h^2/2! + h^4/4!                   (next term < 2e-18)
//     sin x = S_k + (C_k sin h + S_k (cos h - 1)),
//     cos x = C_k + (C_k (cos h - 1) - S_k sin h),
// with S_k, C_k = sin, cos (k pi/512) correctly rounded in a 1024-entry
// table (one period).  The corrections are small against S_k, C_k, so the
// result is within about one unit in the last place.  |x| >= 4096 and
// non-finite x fall back to CUDA's sincos.  16 FP64 operations.
constexpr double SC_INV = 0x1.45f306dc9c883p+7;   // 512/pi
constexpr double SC_HI = 0x1.921fb544p-8;         // pi/512 to 33 bits
constexpr double SC_LO = 0x1.0b4611a626331p-42;   // pi/512 - SC_HI
constexpr double SC_RND = 0x1.8p+52;              // adding it rounds to an integer, kept in the low bits
constexpr int SC_TAB = 1024;

__device__ __forceinline__ void sincos_tab(double x, const double2* __restrict__ tab, double& s, double& c) {
    if ((__double2hiint(x) & 0x7fffffff) < 0x40b00000) {   // |x| < 4096 (so |k| < 2^20), finite
        const double kr = fma(x, SC_INV, SC_RND);
        const int k = __double2loint(kr);
        const double kf = kr - SC_RND;
        const double h = fma(-kf, SC_LO, fma(-kf, SC_HI, x));
        const double h2 = h * h;
        const double sh = fma(h * h2, fma(h2, 1.0 / 120.0, -1.0 / 6.0), h);
        const double ch = h2 * fma(h2, 1.0 / 24.0, -0.5);
        const double2 t = tab[k & (SC_TAB - 1)];
        s = t.x + fma(t.x, ch, t.y * sh);
        c = t.y + fma(t.y, ch, -(t.x * sh));
    } else {
        sincos(x, &s, &c);
    }
}

// polynomial with N coefficients and its derivative (Horner, both at once)
template <int N>
__device__ __forceinline__ double horner64(const double* p, double u, double& dk) {
    if constexpr (N == 1) {
        dk = 0.0;
        return p[0];
    } else {
        double v = p[N - 1];
        double dv = v;
        v = fma(v, u, p[N - 2]);
#pragma unroll
        for (int i = N - 3; i >= 0; --i) {
            dv = fma(dv, u, v);
            v = fma(v, u, p[i]);
        }
        dk = dv;
        return v;
    }
}

// k(u) and k'(u) of law LAW; `tab` is the sine table (LAW_SIN only).
template <int LAW>
__device__ __forceinline__ double law64(const CoeffDev& c, double u, double& dk, const double2* tab) {
    if constexpr (LAW < LAW_SIN) {
        return horner64<LAW + 1>(c.p, u, dk);
    } else if constexpr (LAW == LAW_SIN) {
        double s, co;
        sincos_tab(c.p[2] * u, tab, s, co);
        dk = (c.p[1] * c.p[2]) * co;
        return fma(c.p[1], s, c.p[0]);
    } else {
        return k_eval<double>(c, u, dk);
    }
}

}  // namespace fem
