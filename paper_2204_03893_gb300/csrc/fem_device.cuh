// fem_device.cuh -- element-type traits, reference-table access and the
// conductivity law, shared by the device kernels of libfem.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fem {

// Element type (dimension D, Lagrange degree P) with the default quadrature
// rule of degree 2P.  Index conventions of the element product V = X Q:
//   sym(i,j), i<=j : row-major upper triangle of an n_p x n_p matrix
//                    (Section 7: only the distinct rows of Q are kept)
//   t(a,b),  a<=b  : upper triangle of the d x d matrix A_e
//   X_M[q]         = m w_q b_e                                  (Section 4.1)
//   X_K[q*NS+t]    = w_q b_e k(u_q) A_e[a][b]                   (Section 4.2)
//   X_T[q*D+a]     = w_q b_e k'(u_q) (A_e ghat_q)[a]           (Section 5.2 o_2 u)
//   Q_M[q][sym]    = phi_q[i] phi_q[j]
//   Q_K[q*NS+t][sym] = G_q[i][a] G_q[j][b] (+ G_q[i][b] G_q[j][a] if a != b)
//   Q_T[q*D+a][i*NP+j] = G_q[i][a] phi_q[j]
// with G_q the reference basis gradients (the paper's J_q) and ghat_q the
// reference gradient of u_h at x_q.
template <int D_, int P_>
struct ET {
    static constexpr int D = D_;
    static constexpr int P = P_;
    static constexpr int NP = (D == 2) ? (P + 1) * (P + 2) / 2 : (P + 1) * (P + 2) * (P + 3) / 6;
    static constexpr int NQ = (D == 2) ? (P == 1 ? 3 : P == 2 ? 6 : 12) : (P == 1 ? 4 : P == 2 ? 11 : 24);
    static constexpr int NS = D * (D + 1) / 2;
    static constexpr int NSYM = NP * (NP + 1) / 2;
    static constexpr int NT = NP * NP;
    static constexpr int KM = NQ;
    static constexpr int KK = NQ * NS;
    static constexpr int KT = NQ * D;
    static constexpr int TYPE = (D - 2) * 3 + (P - 1);   // 0..5
    static constexpr int NGEO = 1 + NS;                  // b_e, A_e (upper triangle)
};

__host__ __device__ constexpr int type_nq(int t) {
    return t == 0 ? 3 : t == 1 ? 6 : t == 2 ? 12 : t == 3 ? 4 : t == 4 ? 11 : 24;
}
__host__ __device__ constexpr int type_np(int t) {
    return t == 0 ? 3 : t == 1 ? 6 : t == 2 ? 10 : t == 3 ? 4 : t == 4 ? 10 : 20;
}
__host__ __device__ constexpr int type_d(int t) { return t < 3 ? 2 : 3; }
// per type: phi (NQ*NP), G (NQ*NP*D), w (NQ)
__host__ __device__ constexpr int type_tab_size(int t) {
    return type_nq(t) * type_np(t) * (1 + type_d(t)) + type_nq(t);
}
__host__ __device__ constexpr int type_tab_off(int t) {
    return t == 0 ? 0 : type_tab_off(t - 1) + type_tab_size(t - 1);
}
constexpr int TAB_TOTAL = type_tab_off(6);

__host__ __device__ constexpr int sym_index(int np, int i, int j) {
    // i <= j
    return i * np - (i * (i - 1)) / 2 + (j - i);
}

// Conductivity law (mirrors fem_coeff).
struct CoeffDev {
    int kind;
    int n;
    double p[16];
};

// An FP64 nodal value as two FP32 values with hi + lo = v to about 48 bits:
// hi is v with its mantissa cut to 23 bits, lo the cut-off bits.  Integer
// and FP32 instructions only (FP64 throughput is low on this part, and a
// conversion fallback, even when not taken, slowed the element kernels).
// Range: for 2^-74 <= |v| < 2^128 as stated; for 2^-126 <= |v| < 2^-74 lo
// is 0 (hi alone, 24 bits); |v| < 2^-126 gives (+-0, 0); larger values and
// infinities give +-inf, NaN gives NaN.  The FP32 element paths form the
// differences u_i - u_0 as (hi_i - hi_0) + (lo_i - lo_0), which keeps FP32
// relative accuracy where u varies little over an element.
__device__ __forceinline__ float2 split_f64_all(double v) {
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
    const uint32_t bh = static_cast<uint32_t>(bits >> 32), bl = static_cast<uint32_t>(bits);
    const uint32_t sign = bh & 0x80000000u;
    const uint32_t ex = (bh >> 20) & 0x7ffu;   // biased FP64 exponent
    if (ex - 897u < 254u) {
        // FP32 exponent ex - 1023 + 127; the top 23 of the 52 mantissa bits
        const uint32_t hi = sign | ((ex - 896u) << 23) | ((bh & 0xfffffu) << 3) | (bl >> 29);
        // the low 29 mantissa bits, worth 2^(ex - 1075) each (a normal FP32 scale for ex >= 949)
        const float scale = ex >= 949u ? __uint_as_float((ex - 948u) << 23) : 0.f;
        const float lo = static_cast<float>(bl & 0x1fffffffu) * scale;
        return make_float2(__uint_as_float(hi), sign ? -lo : lo);
    }
    const bool nan = ex == 0x7ffu && ((bh & 0xfffffu) | bl) != 0u;
    const uint32_t mag = nan ? 0x7fc00000u : ex > 1150u ? 0x7f800000u : 0u;
    return make_float2(__uint_as_float(sign | mag), 0.f);
}

// The same split with the values outside 2^-74 <= |v| < 2^126 handled out of
// line.  Same results as split_f64_all; the element tile kernels use this
// form (their code measured faster with the call than fully inline, by 25%
// for P1 tetrahedra), the chunked kernels the inline one.
static __device__ __noinline__ float2 split_f64_edge(double v) { return split_f64_all(v); }
__device__ __forceinline__ float2 split_f64(double v) {
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
    const uint32_t bh = static_cast<uint32_t>(bits >> 32), bl = static_cast<uint32_t>(bits);
    const uint32_t ex = (bh >> 20) & 0x7ffu;
    if (ex - 949u < 200u) {
        const uint32_t sign = bh & 0x80000000u;
        const uint32_t hi = sign | ((ex - 896u) << 23) | ((bh & 0xfffffu) << 3) | (bl >> 29);
        const float lo = static_cast<float>(bl & 0x1fffffffu) * __uint_as_float((ex - 948u) << 23);
        return make_float2(__uint_as_float(hi), sign ? -lo : lo);
    }
    return split_f64_edge(v);
}

// Horner for a polynomial with N coefficients and its derivative at once.
// It performs the same operations as the 8-coefficient loop below does on a
// polynomial whose leading 8 - N coefficients are zero (those steps only
// carry exact zeros), so both give the same bits for finite u.
template <typename T, int N>
__device__ __forceinline__ T horner_n(const CoeffDev& c, T u, T& dk) {
    if constexpr (N == 1) {
        dk = T(0);
        return T(c.p[0]);
    } else {
        T v = T(c.p[N - 1]);
        T dv = v;
        v = v * u + T(c.p[N - 2]);
#pragma unroll
        for (int i = N - 3; i >= 0; --i) {
            dv = dv * u + v;
            v = v * u + T(c.p[i]);
        }
        dk = dv;
        return v;
    }
}

// Law classes that formation code can be specialised for (the class is
// uniform over a launch, or over a batch work item, so the dispatch costs one
// branch outside the quadrature loops): polynomials with at most three
// coefficients, the sine law, and everything else.
enum : int { LC_ANY = 0, LC_POLY3 = 1, LC_SIN = 2 };
__host__ __device__ inline int law_class(const CoeffDev& c) {
    return c.kind == 0 && c.n <= 3 ? LC_POLY3 : c.kind == 1 ? LC_SIN : LC_ANY;
}

// k(u) and k'(u).  LC_POLY3 takes a 3-term Horner (unused coefficients are
// zero, so it gives the bits of the general loop below); LC_SIN the sine law
// alone; LC_ANY every law, with loops over the fixed maxima (8 polynomial
// coefficients, 8 knots) and predicates so that the parameters stay in the
// kernel-parameter space instead of being copied to local memory; unused
// parameters are zero.
template <typename T>
__device__ __forceinline__ T k_sin(const CoeffDev& c, T u, T& dk) {
    T g = T(c.p[2]);
    T s, co;
    if constexpr (sizeof(T) == 8) { sincos(g * u, &s, &co); }
    else { sincosf(g * u, &s, &co); }
    dk = T(c.p[1]) * g * co;
    return T(c.p[0]) + T(c.p[1]) * s;
}

template <typename T, int LC = LC_ANY>
__device__ __forceinline__ T k_eval(const CoeffDev& c, T u, T& dk) {
    if constexpr (LC == LC_POLY3) {
        return horner_n<T, 3>(c, u, dk);
    } else if constexpr (LC == LC_SIN) {
        return k_sin<T>(c, u, dk);
    } else if (c.kind == 0) {
        T v = T(0), dv = T(0);
#pragma unroll
        for (int i = 7; i >= 0; --i) {
            dv = dv * u + v;      // Horner for the derivative uses the running value
            v = v * u + T(c.p[i]);
        }
        dk = dv;
        return v;
    } else if (c.kind == 1) {
        return k_sin<T>(c, u, dk);
    } else {
        // device layout (set by the host): knots in p[0..7], values in p[8..15], m = n/2 knots
        const int m = c.n / 2;
        T val = T(0), slope = T(0), last = T(0);
        bool found = false;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i < m) last = T(c.p[8 + i]);
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            if (i + 1 < m && !found) {
                const T t0 = T(c.p[i]), t1 = T(c.p[i + 1]);
                // branch i covers (t_i, t_i+1]; the first one is closed on the left too
                const bool in = (i == 0) ? (u >= t0 && u <= t1) : (u > t0 && u <= t1);
                if (in) {
                    slope = T((c.p[8 + i + 1] - c.p[8 + i]) / (c.p[i + 1] - c.p[i]));
                    val = T(c.p[8 + i]) + slope * (u - t0);
                    found = true;
                }
            }
        }
        if (!found) {
            slope = T(0);
            val = (u < T(c.p[0])) ? T(c.p[8]) : last;
        }
        dk = slope;
        return val;
    }
}

}  // namespace fem
