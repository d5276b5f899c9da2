// element_simt.cu -- element products V = X Q on the SIMT pipes (FP64 and
// FP32), one thread per element.
//
// Algorithm 2, formation step: the coefficient evaluations S at the quadrature
// points (here k(u_q), k'(u_q) from u_q = phi_q . u_e), Lambda = S * (w b^T)
// (eq. def_lambda, computed as w_q S_qe b_e in place), X_m = Lambda and
// X_c = Lambda (.) W (Section 4.2), then V = Q X.  The tangent uses the same
// shape with X_T[q][a] = w_q b_e k'(u_q) (A_e ghat_q)[a], which contracts the
// Section 5.2 conductivity tensor with u in its second mode.  Only the
// n_p(n_p+1)/2 distinct entries of the symmetric M and K are formed
// (Section 7).  V is written element-major: V[e][n].
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "fem_internal.h"
#include "law64.cuh"
#include "refelem.h"

namespace fem {

namespace {

__host__ __device__ constexpr int q_size(int t) {
    return type_nq(t) * (type_np(t) * (type_np(t) + 1) / 2) * (1 + type_d(t) * (type_d(t) + 1) / 2) +
           type_nq(t) * type_d(t) * type_np(t) * type_np(t);
}
__host__ __device__ constexpr int q_off(int t) { return t == 0 ? 0 : q_off(t - 1) + q_size(t - 1); }
constexpr int Q_TOTAL = q_off(6);

__constant__ double c_ref64[TAB_TOTAL];
__constant__ float c_ref32[TAB_TOTAL];
__device__ double g_Q64[Q_TOTAL];
__device__ float g_Q32[Q_TOTAL];

template <typename T>
struct Tabs;
template <>
struct Tabs<double> {
    static __device__ __forceinline__ double ref(int i) { return c_ref64[i]; }
    static __device__ __forceinline__ const double* Q() { return g_Q64; }
};
template <>
struct Tabs<float> {
    static __device__ __forceinline__ float ref(int i) { return c_ref32[i]; }
    static __device__ __forceinline__ const float* Q() { return g_Q32; }
};

constexpr int BT = 64;   // elements (threads) per block

// FP64 P1 tables: the mass factor sum_q w_q phi_q[i] phi_q[j], which the
// rules (all symmetric in the vertices) make one value on the diagonal and
// one off it: c_p1m2 = (diagonal, off-diagonal) for triangles, then
// tetrahedra (checked at set-up); and the sine table of law64.cuh.
__constant__ double c_p1m2[4];
// A rule of n_p points, one per vertex, with equal weights w and basis
// values phi_q[j] = beta + gamma [j = vertex of q] (the degree-2 rules of
// both simplices): per simplex (beta, gamma, w, beta w, gamma w), used where
// c_p1q_on is set.  Then u at the point of vertex j is beta sum_i u_i +
// gamma u_j, and the sums over the points need no products by the basis.
__constant__ double c_p1q[10];
__constant__ int c_p1q_on[2];
__device__ double2 g_sincos_tab[SC_TAB];

// nodal values: FP64 as given; the FP32 path splits each gathered value
// as hi + lo (split_f64) so that the differences u_i - u_0 that carry the
// gradient keep FP32 relative accuracy.

// X row and V = X Q of element e (thread-private X row in shared memory).
template <typename ETy, typename T, bool PQ = false>
__device__ __forceinline__ void simt_element(int64_t e, const int* __restrict__ conn, const T* __restrict__ geo,
                                             int64_t gs, const double* __restrict__ u,
                                             const CoeffDev& k, T mass, T* __restrict__ VM, T* __restrict__ VK,
                                             T* __restrict__ VT, T* X) {
    constexpr int D = ETy::D, NP = ETy::NP, NQ = ETy::NQ, NS = ETy::NS;
    constexpr int KM = ETy::KM, KK = ETy::KK, KT = ETy::KT;
    constexpr int TO = type_tab_off(ETy::TYPE);
    constexpr int PHI = TO, GR = TO + NQ * NP, WQ = TO + NQ * NP * (1 + D);
    constexpr int QO = q_off(ETy::TYPE);
    constexpr int QM_O = QO, QK_O = QO + KM * ETy::NSYM, QT_O = QK_O + KK * ETy::NSYM;
    const T* Q = Tabs<T>::Q();
    const bool need_u = (VK != nullptr) | (VT != nullptr);
    // du[i] = u_i - u_0 and u_0 (u is only needed for K and T; mass-only calls pass NULL)
    T du[NP];
    T u0 = T(0);
    const int* ce = conn + e * NP;
    if (need_u) {
        if constexpr (sizeof(T) == 8) {
            u0 = u[ce[0]];
#pragma unroll
            for (int i = 0; i < NP; ++i) du[i] = u[ce[i]] - u0;
        } else {
            const float2 a = split_f64(u[ce[0]]);
            u0 = a.x + a.y;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const float2 b = split_f64(u[ce[i]]);
                du[i] = (b.x - a.x) + (b.y - a.y);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) du[i] = T(0);
    }
    // geometry: per element, or per quadrature point (PQ: the cache entry of
    // point q of element e at e n_q + q, Section 7 isoparametric mappings
    // and point-wise conductivity tensors)
    T b = T(0);
    T A[NS];
    if constexpr (!PQ) {
        b = geo[e];
#pragma unroll
        for (int t = 0; t < NS; ++t) A[t] = geo[(1 + t) * gs + e];
    }
    // --- X = Lambda, Lambda (.) W, tangent factors
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
        if constexpr (PQ) {
            const int64_t gi = e * NQ + q;
            b = geo[gi];
#pragma unroll
            for (int t = 0; t < NS; ++t) A[t] = geo[(1 + t) * gs + gi];
        }
        // u_q = u_0 + sum_i phi_i (u_i - u_0) (the basis sums to one); the
        // reference gradient uses the differences only (its rows sum to zero)
        T uq = T(0);
        T g[D];
#pragma unroll
        for (int a = 0; a < D; ++a) g[a] = T(0);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            uq += Tabs<T>::ref(PHI + q * NP + i) * du[i];
#pragma unroll
            for (int a = 0; a < D; ++a) g[a] += Tabs<T>::ref(GR + (q * NP + i) * D + a) * du[i];
        }
        uq += u0;
        T dk;
        T kq = k_eval<T>(k, uq, dk);
        T lam = Tabs<T>::ref(WQ + q) * b;
        X[q] = mass * lam;
        T lk = lam * kq;
#pragma unroll
        for (int t = 0; t < NS; ++t) X[KM + q * NS + t] = lk * A[t];
        // A ghat, A symmetric stored as upper triangle
        T ld = lam * dk;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            T s = T(0);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                int lo = a < c ? a : c, hi = a < c ? c : a;
                int t = lo * D - (lo * (lo - 1)) / 2 + (hi - lo);
                s += A[t] * g[c];
            }
            X[KM + KK + q * D + a] = ld * s;
        }
    }
    // --- V = X Q, chunks of CH outputs; entry n of the element at
    // V[(e N + n) CS] (CS = 2: M and K interleaved, K at VK = VM + 1)
    constexpr int CH = 8;
    auto product = [&](const T* Xs, int K, const T* Qm, int N, T* V, int CS) {
#pragma unroll 1
        for (int n0 = 0; n0 < N; n0 += CH) {
            T acc[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) acc[c] = T(0);
#pragma unroll 2
            for (int kk = 0; kk < K; ++kk) {
                T x = Xs[kk];
                const T* qrow = Qm + kk * N + n0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (n0 + c < N) acc[c] += x * qrow[c];
            }
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (n0 + c < N) V[(e * N + n0 + c) * CS] = acc[c];
        }
    };
    if (VM) product(X, KM, Q + QM_O, ETy::NSYM, VM, 2);
    if (VK) product(X + KM, KK, Q + QK_O, ETy::NSYM, VK, 2);
    if (VT) product(X + KM + KK, KT, Q + QT_O, ETy::NT, VT, 1);
}

template <typename ETy, typename T, bool PQ>
__global__ void __launch_bounds__(BT) element_simt_kernel(const int* __restrict__ conn, const T* __restrict__ geo,
                                                          int64_t E, int64_t gs,
                                                          const double* __restrict__ u,
                                                          CoeffDev k, T mass, T* __restrict__ VM, T* __restrict__ VK,
                                                          T* __restrict__ VT) {
    constexpr int KTOT = ETy::KM + ETy::KK + ETy::KT;
    constexpr int LD = KTOT | 1;   // odd row stride: conflict-free per-thread rows
    extern __shared__ unsigned char smem_raw[];
    T* X = reinterpret_cast<T*>(smem_raw) + threadIdx.x * LD;
    for (int64_t e0 = (int64_t)blockIdx.x * BT; e0 < E; e0 += (int64_t)gridDim.x * BT) {
        int64_t e = e0 + threadIdx.x;
        if (e >= E) continue;
        simt_element<ETy, T, PQ>(e, conn, geo, gs, u, k, mass, VM, VK, VT, X);
    }
}

// ------------------------------------------------------- P1 simplices in FP64
// For P1 the reference basis is the barycentric one, phi_0 = 1 - sum_a xhat_a
// and phi_a = xhat_a, whose gradients are constant: G = [-1 ... -1; I].  The
// rows of Q_K and Q_T then no longer depend on the quadrature point, so the
// products of Algorithm 2 can be summed over q first (Section 4.2 with X
// contracted over q before the product):
//     K_e = b_e (sum_q w_q k(u_q)) G A_e G^T,
//     T_e[i][j] = b_e (G A_e ghat)_i (sum_q w_q k'(u_q) phi_q[j]),
//     M_e = m b_e sum_q w_q phi_q phi_q^T,
// with ghat = G^T u_e = (u_1 - u_0, ..., u_d - u_0).  This is the same
// quadrature sum as the general path, regrouped, and every matrix is stored
// factored, for the CSR sum to multiply out as it adds (one fused
// multiply-add per contribution in place of its addition):
//   - K_e as its scalar factor b_e sum_q w_q k(u_q): the Gram matrix
//     G A_e G^T does not change with u and is kept per mesh (geometry.cu);
//   - T_e, an outer product, as its two factors t_e = b_e G A_e ghat and
//     s_e with s_e[j] = sum_q w_q k'(u_q) phi_q[j];
//   - M_e as its diagonal and off-diagonal value (the rules are symmetric in
//     the vertices, so sum_q w_q phi_q phi_q^T takes only these two).
// Tetrahedra need 114 FP64 operations per element with the sine law
// (mostly sin/cos at four points) against ~780 for the general product,
// which matters because the FP64 pipe, not HBM, bounds the FP64 path on
// this part.
//
// The element's values are written through `mk` (4 values: M's diagonal
// value, K's factor, M's off-diagonal value, K's factor again, so that the
// sum reads the pair it needs with one 16-byte load) and `tr` (2 n_p values:
// the factors of T_e), which point into shared memory in the single-mesh
// kernel and into V in the batched one.
template <int D, int LAW>
__device__ __forceinline__ void p1_element_fp64(int64_t e, const int* __restrict__ conn, const double* __restrict__ geo,
                                                int64_t gs, const double* __restrict__ u, const CoeffDev& k,
                                                double mass, const double2* tab, bool doM, bool doK, bool doT,
                                                double* mk, double* tr) {
    constexpr int NP = D + 1, NQ = D == 2 ? 3 : 4, NS = D * (D + 1) / 2;
    constexpr int TYPE = D == 2 ? 0 : 3;
    constexpr int PHI = type_tab_off(TYPE), WQ = PHI + NQ * NP * (1 + D);
    const double b = geo[e];
    if (doM) {   // M's diagonal and off-diagonal value
        const double mb = mass * b;
        mk[0] = mb * c_p1m2[2 * (D - 2)];
        mk[2] = mb * c_p1m2[2 * (D - 2) + 1];
    }
    if (!doK && !doT) return;
    double A[NS];
    if (doT) {
#pragma unroll
        for (int t = 0; t < NS; ++t) A[t] = geo[(1 + t) * gs + e];
    }
    const int* ce = conn + e * NP;
    double uv[NP], du[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) uv[i] = u[ce[i]];
    const double u0 = uv[0];
    du[0] = 0.0;
#pragma unroll
    for (int i = 1; i < NP; ++i) du[i] = uv[i] - u0;
    // sums over the quadrature points: s0 = sum w k(u_q), s1[j] = sum w k'(u_q) phi_q[j]
    double s0 = 0.0, s1[NP];
    if (NQ == NP && c_p1q_on[D - 2]) {
        // one point per vertex, equal weights (taken per vertex, so the
        // points' order does not matter): s0 = w sum k, s1[j] = beta w sum k'
        // + gamma w k'(point of vertex j)
        const double* cq = c_p1q + 5 * (D - 2);
        const double be = cq[0], ga = cq[1], w = cq[2], bw = cq[3], gw = cq[4];
        double su = uv[0];
#pragma unroll
        for (int i = 1; i < NP; ++i) su += uv[i];
        if constexpr (LAW == LAW_SIN) {
            // k = a + b sin(c u) is affine in sin and k' = b c cos(c u) linear
            // in cos, so the point sums are taken over sin and cos:
            // s0 = n_p a w + b w sum sin, s1[j] = b c (beta w sum cos + gamma w cos_j),
            // with the argument c u = (c beta) sum u + (c gamma) u_j
            const double ka = k.p[0], kb = k.p[1], kc = k.p[2];
            const double cga = kc * ga, xb = (kc * be) * su;
            double sn[NP], co[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) sincos_tab(fma(cga, uv[j], xb), tab, sn[j], co[j]);
            double ss = sn[0], sc = co[0];
#pragma unroll
            for (int j = 1; j < NP; ++j) {
                ss += sn[j];
                sc += co[j];
            }
            s0 = fma(w * kb, ss, (NP * w) * ka);
            const double bc = kb * kc, g1 = gw * bc, g0 = (bw * bc) * sc;
#pragma unroll
            for (int j = 0; j < NP; ++j) s1[j] = fma(g1, co[j], g0);
        } else {
            const double bsu = be * su;
            double kq[NP], dkq[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) kq[j] = law64<LAW>(k, fma(ga, uv[j], bsu), dkq[j], tab);
            double sk = kq[0], sd = dkq[0];
#pragma unroll
            for (int j = 1; j < NP; ++j) {
                sk += kq[j];
                sd += dkq[j];
            }
            s0 = w * sk;
            const double bws = bw * sd;
#pragma unroll
            for (int j = 0; j < NP; ++j) s1[j] = fma(gw, dkq[j], bws);
        }
    } else {
#pragma unroll
        for (int j = 0; j < NP; ++j) s1[j] = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double uq = u0;
#pragma unroll
            for (int i = 1; i < NP; ++i) uq = fma(c_ref64[PHI + q * NP + i], du[i], uq);
            double dk;
            const double kq = law64<LAW>(k, uq, dk, tab);
            const double w = c_ref64[WQ + q];
            s0 = fma(w, kq, s0);
            const double wd = w * dk;
#pragma unroll
            for (int j = 0; j < NP; ++j) s1[j] = fma(wd, c_ref64[PHI + q * NP + j], s1[j]);
        }
    }
    auto At = [&](int a, int c) {   // A[a][c] from the upper triangle
        const int lo = a < c ? a : c, hi = a < c ? c : a;
        return A[lo * D - (lo * (lo - 1)) / 2 + (hi - lo)];
    };
    if (doK) {   // K's factor (its Gram matrix G A_e G^T is cached per mesh)
        const double bs = b * s0;
        mk[1] = bs;
        mk[3] = bs;
    }
    if (doT) {
        double r[D];   // A ghat
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double v = At(a, 0) * du[1];
#pragma unroll
            for (int c = 1; c < D; ++c) v = fma(At(a, c), du[c + 1], v);
            r[a] = v;
        }
        double bt[NP];   // b (G A ghat)
        double r0 = r[0];
#pragma unroll
        for (int a = 1; a < D; ++a) r0 += r[a];
        bt[0] = -(b * r0);
#pragma unroll
        for (int a = 0; a < D; ++a) bt[a + 1] = b * r[a];
#pragma unroll
        for (int i = 0; i < NP; ++i) tr[i] = bt[i];
#pragma unroll
        for (int j = 0; j < NP; ++j) tr[NP + j] = s1[j];
    }
}

constexpr int P1_BT = 128;   // elements (threads) per block of the FP64 P1 kernel

template <int D>
__host__ __device__ constexpr int p1_ldmk() { return 5; }   // the 4-value M/K block, odd
template <int D>
__host__ __device__ constexpr int p1_ldt() { return 2 * (D + 1) | 1; }   // the two factors of T_e, odd

template <int D, int LAW>
__host__ __device__ constexpr size_t p1_smem() {
    return (LAW == LAW_SIN ? SC_TAB * sizeof(double2) : 0) + sizeof(double) * P1_BT * (p1_ldmk<D>() + p1_ldt<D>());
}

// One element per thread; each thread builds its element's rows in shared
// memory (odd row strides: no bank conflicts), then the block copies its
// P1_BT consecutive rows out with coalesced stores (the rows of consecutive
// elements are contiguous in V).
template <int D, int LAW>
__global__ void __launch_bounds__(P1_BT) element_p1_fp64_kernel(const int* __restrict__ conn,
                                                                const double* __restrict__ geo, int64_t E, int64_t gs,
                                                                const double* __restrict__ u, CoeffDev k, double mass,
                                                                double* __restrict__ VMK, bool doM, bool doK,
                                                                double* __restrict__ VT) {
    constexpr int NP = D + 1, NSYM = NP * (NP + 1) / 2, NT = 2 * NP;   // NT: T_e's factors
    constexpr int LDMK = p1_ldmk<D>(), LDT = p1_ldt<D>();
    extern __shared__ __align__(16) unsigned char p1_smem_raw[];
    const double2* tab = reinterpret_cast<const double2*>(p1_smem_raw);
    double* sMK = reinterpret_cast<double*>(p1_smem_raw + (LAW == LAW_SIN ? SC_TAB * sizeof(double2) : 0));
    double* sT = sMK + P1_BT * LDMK;
    if constexpr (LAW == LAW_SIN) {
        double2* t = reinterpret_cast<double2*>(p1_smem_raw);
        for (int i = threadIdx.x; i < SC_TAB; i += P1_BT) t[i] = g_sincos_tab[i];
        __syncthreads();
    }
    const bool doT = VT != nullptr;
    for (int64_t e0 = (int64_t)blockIdx.x * P1_BT; e0 < E; e0 += (int64_t)gridDim.x * P1_BT) {   // block-uniform
        const int64_t e = e0 + threadIdx.x;
        if (e < E)
            p1_element_fp64<D, LAW>(e, conn, geo, gs, u, k, mass, tab, doM, doK, doT, sMK + threadIdx.x * LDMK,
                                    sT + threadIdx.x * LDT);
        __syncthreads();
        const int rows = E - e0 < P1_BT ? (int)(E - e0) : P1_BT;
        if (doM || doK) {
            double* g = VMK + 4 * e0;   // the block's M/K blocks (two pairs each), contiguous
            if (doM && doK) {
                double2* g2 = reinterpret_cast<double2*>(g);
                for (int i = threadIdx.x; i < rows * 2; i += P1_BT) {
                    const double* r = sMK + (i / 2) * LDMK + 2 * (i % 2);
                    g2[i] = make_double2(r[0], r[1]);
                }
            } else {
                const int o = doM ? 0 : 1;
                for (int i = threadIdx.x; i < rows * 2; i += P1_BT)
                    g[2 * i + o] = sMK[(i / 2) * LDMK + 2 * (i % 2) + o];
            }
        }
        if (doT) {
            double* g = VT + e0 * NT;
            for (int i = threadIdx.x; i < rows * NT; i += P1_BT) g[i] = sT[(i / NT) * LDT + i % NT];
        }
        __syncthreads();
    }
}

template <int D, int LAW>
int launch_p1_law(const fem_mesh& m, const CoeffDev& k, const double* u, const double* geo, double* VMK, bool doM,
                  bool doK, double* VT, cudaStream_t s, int64_t e0, int64_t E) {
    constexpr size_t smem = p1_smem<D, LAW>();
    auto kern = element_p1_fp64_kernel<D, LAW>;
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, nsm = 0, per_sm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P1_BT, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = (E + P1_BT - 1) / P1_BT;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > tiles) grid = tiles;
    constexpr int NP = D + 1;
    cudaGetLastError();   // clear any stale error before the launch check
    kern<<<(unsigned)grid, P1_BT, smem, s>>>(m.conn.as<int>() + e0 * NP, geo + e0, E, m.E, u, k, m.m,
                                              VMK ? VMK + 4 * e0 : nullptr, doM, doK,
                                              VT ? VT + e0 * 2 * NP : nullptr);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

template <int D>
int launch_p1_fp64(const fem_mesh& m, const CoeffDev& k, const double* u, double* VM, double* VK, double* VT,
                   cudaStream_t s, int64_t e0, int64_t e1) {
    const int64_t E = e1 - e0;
    if (E <= 0) return FEM_OK;
    double* VMK = VM ? VM : VK ? VK - 1 : nullptr;
    const bool doM = VM != nullptr, doK = VK != nullptr;
    const double* geo = m.geo64.as<double>();
    const int law = (doK || VT) ? law_code(k) : 0;
    switch (law) {
#define FEM_P1_LAW(L) \
    case L: return launch_p1_law<D, L>(m, k, u, geo, VMK, doM, doK, VT, s, e0, E);
        FEM_P1_LAW(0) FEM_P1_LAW(1) FEM_P1_LAW(2) FEM_P1_LAW(3) FEM_P1_LAW(4)
        FEM_P1_LAW(5) FEM_P1_LAW(6) FEM_P1_LAW(7) FEM_P1_LAW(8) FEM_P1_LAW(9)
#undef FEM_P1_LAW
    }
    return fail(FEM_EINVAL, "conductivity law");
}

// The FP64 law on its own (fem_law_eval): k(u) and k'(u) at n values.
template <int LAW>
__global__ void __launch_bounds__(256) law_eval_kernel(CoeffDev k, const double* __restrict__ u, int64_t n,
                                                       double* __restrict__ kv, double* __restrict__ dkv) {
    __shared__ double2 tab[SC_TAB];
    if constexpr (LAW == LAW_SIN) {
        for (int i = threadIdx.x; i < SC_TAB; i += blockDim.x) tab[i] = g_sincos_tab[i];
        __syncthreads();
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double dk;
        const double v = law64<LAW>(k, u[i], dk, tab);
        if (kv) kv[i] = v;
        if (dkv) dkv[i] = dk;
    }
}

// FP64 P1 element with the law chosen at run time (batched kernel; the sine
// table is read from global memory there, the values are the same)
template <int D>
__device__ __forceinline__ void p1_element_fp64_any(const CoeffDev& k, int64_t e, const int* __restrict__ conn,
                                                    const double* __restrict__ geo, int64_t gs,
                                                    const double* __restrict__ u, double mass, bool doM, bool doK,
                                                    double* mk, double* tr) {
    const bool doT = tr != nullptr;
    switch (law_code(k)) {
#define FEM_P1_ANY(L) \
    case L: p1_element_fp64<D, L>(e, conn, geo, gs, u, k, mass, g_sincos_tab, doM, doK, doT, mk, tr); break;
        FEM_P1_ANY(0) FEM_P1_ANY(1) FEM_P1_ANY(2) FEM_P1_ANY(3) FEM_P1_ANY(4)
        FEM_P1_ANY(5) FEM_P1_ANY(6) FEM_P1_ANY(7) FEM_P1_ANY(8) FEM_P1_ANY(9)
#undef FEM_P1_ANY
        default: break;
    }
}

// Batched: the work list holds blocks of BT elements of many meshes.
template <typename T>
__global__ void __launch_bounds__(BT) batch_simt_kernel(const BatchItem* __restrict__ items, int nitems,
                                                        const BatchMesh* __restrict__ meshes) {
    extern __shared__ unsigned char smem_raw[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchMesh& bm = meshes[w.mesh];
        const int64_t e = w.first + threadIdx.x;
        if (!(bm.vM || bm.vK || bm.vT)) continue;   // mesh skipped in this launch
        if (threadIdx.x >= w.count || e >= bm.E) continue;
        const T* geo = static_cast<const T*>(sizeof(T) == 8 ? (const void*)bm.geo64 : (const void*)bm.geo32);
        const double* u = bm.u;
        T* VM = bm.vM ? static_cast<T*>(bm.VM) : nullptr;
        T* VK = bm.vK ? static_cast<T*>(bm.VK) : nullptr;
        T* VT = bm.vT ? static_cast<T*>(bm.VT) : nullptr;
        const T mass = (T)bm.mass;
        if constexpr (sizeof(T) == 8) {
            // FP64 P1: the same regrouped product as the single-mesh kernel
            // (same bits), rows written straight into V
            if (w.type == 0 || w.type == 3) {
                const int ntf = w.type == 0 ? 6 : 8;   // T_e's factors
                double* mk = (VM || VK) ? static_cast<double*>(bm.VM) + 4 * e : nullptr;   // the M/K block
                double* tr = VT ? VT + e * ntf : nullptr;
                if (w.type == 0)
                    p1_element_fp64_any<2>(bm.k, e, bm.conn, geo, bm.E, u, mass, VM != nullptr, VK != nullptr, mk, tr);
                else
                    p1_element_fp64_any<3>(bm.k, e, bm.conn, geo, bm.E, u, mass, VM != nullptr, VK != nullptr, mk, tr);
                continue;
            }
        }
        switch (w.type) {
#define FEM_BATCH_SIMT_CASE(TY, DD, PP)                                                                     \
    case TY: {                                                                                          \
        constexpr int LD = (ET<DD, PP>::KM + ET<DD, PP>::KK + ET<DD, PP>::KT) | 1;                      \
        simt_element<ET<DD, PP>, T>(e, bm.conn, geo, bm.E, u, bm.k, mass, VM, VK, VT,                   \
                                    reinterpret_cast<T*>(smem_raw) + threadIdx.x * LD);                 \
    } break;
            FEM_BATCH_SIMT_CASE(0, 2, 1)
            FEM_BATCH_SIMT_CASE(1, 2, 2)
            FEM_BATCH_SIMT_CASE(2, 2, 3)
            FEM_BATCH_SIMT_CASE(3, 3, 1)
            FEM_BATCH_SIMT_CASE(4, 3, 2)
            FEM_BATCH_SIMT_CASE(5, 3, 3)
#undef FEM_BATCH_SIMT_CASE
            default: break;
        }
    }
}

template <typename ETy, typename T, bool PQ>
int launch_simt(const fem_mesh& m, const CoeffDev& k, const double* u, const T* geo, T* VM, T* VK,
                T* VT, cudaStream_t s, int64_t e0, int64_t e1) {
    const int64_t E = e1 - e0;
    if (E <= 0) return FEM_OK;
    constexpr int KTOT = ETy::KM + ETy::KK + ETy::KT;
    constexpr int LD = KTOT | 1;
    size_t smem = sizeof(T) * (size_t)LD * BT;
    auto kern = element_simt_kernel<ETy, T, PQ>;
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    int dev = 0, nsm = 0, per_sm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t tiles = (E + BT - 1) / BT;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > tiles) grid = tiles;
    if (grid < 1) return FEM_OK;
    cudaGetLastError();   // clear any stale error before the launch check
    // per-point geometry: entries (e, q) at e n_q + q, SoA stride E n_q
    const T* g = PQ ? geo + e0 * ETy::NQ : geo + e0;
    const int64_t gs = PQ ? m.E * ETy::NQ : m.E;
    kern<<<(unsigned)grid, BT, smem, s>>>(m.conn.as<int>() + e0 * ETy::NP, g, E, gs, u, k, (T)m.m,
                                          VM ? VM + 2 * e0 * ETy::NSYM : nullptr, VK ? VK + 2 * e0 * ETy::NSYM : nullptr,
                                          VT ? VT + e0 * ETy::NT : nullptr);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

template <typename T>
int dispatch(const fem_mesh& m, const CoeffDev& k, const double* u, const T* geo, T* VM, T* VK,
             T* VT, cudaStream_t s, int64_t e0, int64_t e1) {
    if (e1 < 0) e1 = m.E;
    if (e0 < 0 || e0 > e1 || e1 > m.E) return fail(FEM_EINVAL, "element range out of bounds");
    if (m.perq) {   // per-point geometry: the general product, b and A read per point
        const T* gq = sizeof(T) == 8 ? reinterpret_cast<const T*>(m.geoq64.ptr) : reinterpret_cast<const T*>(m.geoq32.ptr);
        switch (m.type) {
            case 0: return launch_simt<ET<2, 1>, T, true>(m, k, u, gq, VM, VK, VT, s, e0, e1);
            case 1: return launch_simt<ET<2, 2>, T, true>(m, k, u, gq, VM, VK, VT, s, e0, e1);
            case 2: return launch_simt<ET<2, 3>, T, true>(m, k, u, gq, VM, VK, VT, s, e0, e1);
            case 3: return launch_simt<ET<3, 1>, T, true>(m, k, u, gq, VM, VK, VT, s, e0, e1);
            case 4: return launch_simt<ET<3, 2>, T, true>(m, k, u, gq, VM, VK, VT, s, e0, e1);
            case 5: return launch_simt<ET<3, 3>, T, true>(m, k, u, gq, VM, VK, VT, s, e0, e1);
        }
        return fail(FEM_EINVAL, "element type");
    }
    if constexpr (sizeof(T) == 8) {
        if (m.type == 0) return launch_p1_fp64<2>(m, k, u, VM, VK, VT, s, e0, e1);
        if (m.type == 3) return launch_p1_fp64<3>(m, k, u, VM, VK, VT, s, e0, e1);
    }
    switch (m.type) {
        case 0: return launch_simt<ET<2, 1>, T, false>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 1: return launch_simt<ET<2, 2>, T, false>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 2: return launch_simt<ET<2, 3>, T, false>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 3: return launch_simt<ET<3, 1>, T, false>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 4: return launch_simt<ET<3, 2>, T, false>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 5: return launch_simt<ET<3, 3>, T, false>(m, k, u, geo, VM, VK, VT, s, e0, e1);
    }
    return fail(FEM_EINVAL, "element type");
}

// The u-dependent mass (Section 2 with m = m(u_h)) and the Section 5.1 mass
// tensor multiplied by z = u - u^s in its second mode, both as products with
// the mass basis matrix Q_M (Section 4.1; the tensor's Q = Phi (.) Phi (.) Phi
// contracted with z_e over one factor leaves Q_M with z_q = phi_q . z_e in X):
//     X_u[q] = w_q b_e m(u_q),   X_t[q] = w_q b_e m'(u_q) z_q,   V = X Q_M,
// the n_sym distinct entries of each symmetric local matrix, M(u) at the even
// and the tensor term at the odd positions of the interleaved M/K storage.
// FP32 values take u through the (hi, lo) split as the other kernels, and z
// is formed in FP64 before it is rounded.  Where a block's rows fit
// (BT x (2 n_sym + 1) values, the odd row stride keeps the per-thread rows
// free of bank conflicts), each thread stores its element's row in shared
// memory and the block copies its BT consecutive rows out with coalesced
// stores; otherwise every thread stores its row directly.
template <typename ETy, typename T>
__host__ __device__ constexpr bool mass_u_staged() {
    return (BT * (2 * ETy::NSYM + 1) + ETy::NQ * ETy::NSYM) * sizeof(T) <= 48 * 1024;
}

template <typename ETy, typename T, bool PQ>
__global__ void __launch_bounds__(BT) mass_u_kernel(const int* __restrict__ conn, const T* __restrict__ geo,
                                                    int64_t E, const double* __restrict__ u,
                                                    const double* __restrict__ us, CoeffDev mk,
                                                    T* __restrict__ VMK, bool doMu, bool doMt) {
    constexpr int NP = ETy::NP, NQ = ETy::NQ, NSYM = ETy::NSYM, D = ETy::D;
    constexpr int TO = type_tab_off(ETy::TYPE);
    constexpr int PHI = TO, WQ = TO + NQ * NP * (1 + D);
    constexpr bool STAGED = mass_u_staged<ETy, T>();
    constexpr int LDS = 2 * NSYM + 1;
    extern __shared__ __align__(16) unsigned char mu_smem[];
    T* stage = reinterpret_cast<T*>(mu_smem);
    const T* Q = Tabs<T>::Q() + q_off(ETy::TYPE);   // Q_M, NQ x NSYM row-major
    if constexpr (STAGED) {   // Q_M to shared memory, after the staging rows
        T* sQ = stage + BT * LDS;
        for (int i = threadIdx.x; i < NQ * NSYM; i += BT) sQ[i] = Q[i];
        __syncthreads();
        Q = sQ;
    }
    for (int64_t e0 = (int64_t)blockIdx.x * BT; e0 < E; e0 += (int64_t)gridDim.x * BT) {   // block-uniform
        const int64_t e = e0 + threadIdx.x;
        if (e < E) {
            const int* ce = conn + e * NP;
            T du[NP], dz[NP];
            T u0;
            if constexpr (sizeof(T) == 8) {
                u0 = u[ce[0]];
#pragma unroll
                for (int i = 0; i < NP; ++i) du[i] = u[ce[i]] - u0;
            } else {
                const float2 a = split_f64(u[ce[0]]);
                u0 = a.x + a.y;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    const float2 c = split_f64(u[ce[i]]);
                    du[i] = (c.x - a.x) + (c.y - a.y);
                }
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) dz[i] = doMt ? (T)(u[ce[i]] - us[ce[i]]) : T(0);
            const T b0 = PQ ? T(0) : geo[e];
            T Xu[NQ], Xt[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const T b = PQ ? geo[e * NQ + q] : b0;   // |det B| per point (Section 7) or per element
                T uq = T(0), zq = T(0);
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    uq += Tabs<T>::ref(PHI + q * NP + i) * du[i];
                    zq += Tabs<T>::ref(PHI + q * NP + i) * dz[i];
                }
                uq += u0;
                T dm;
                const T mq = k_eval<T>(mk, uq, dm);
                const T lam = Tabs<T>::ref(WQ + q) * b;
                Xu[q] = lam * mq;
                Xt[q] = lam * dm * zq;
            }
#pragma unroll 1
            for (int n = 0; n < NSYM; ++n) {
                T au = T(0), at = T(0);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const T qv = Q[q * NSYM + n];
                    au += Xu[q] * qv;
                    at += Xt[q] * qv;
                }
                if constexpr (STAGED) {
                    stage[threadIdx.x * LDS + 2 * n] = au;
                    stage[threadIdx.x * LDS + 2 * n + 1] = at;
                } else {
                    if (doMu) VMK[2 * (e * NSYM + n)] = au;
                    if (doMt) VMK[2 * (e * NSYM + n) + 1] = at;
                }
            }
        }
        if constexpr (STAGED) {
            __syncthreads();
            const int rows = E - e0 < BT ? (int)(E - e0) : BT;
            T* g = VMK + 2 * e0 * NSYM;   // the block's rows are consecutive in V
            for (int i = threadIdx.x; i < rows * 2 * NSYM; i += BT)
                g[i] = stage[(i / (2 * NSYM)) * LDS + i % (2 * NSYM)];
            __syncthreads();
        }
    }
}

template <typename T, bool PQ>
int launch_mass_u(const fem_mesh& m, const CoeffDev& mk, const double* u, const double* us, const T* geo, T* VMK,
                  bool doMu, bool doMt, cudaStream_t s) {
    if (m.E <= 0) return FEM_OK;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = (m.E + BT - 1) / BT;
    if (grid > (int64_t)nsm * 16) grid = (int64_t)nsm * 16;
    cudaGetLastError();   // clear any stale error before the launch check
    switch (m.type) {
#define FEM_MASS_U_CASE(TY, DD, PP)                                                                          \
    case TY:                                                                                             \
        mass_u_kernel<ET<DD, PP>, T, PQ>                                                                 \
            <<<(unsigned)grid, BT,                                                                         \
               mass_u_staged<ET<DD, PP>, T>()                                                               \
                   ? (BT * (2 * ET<DD, PP>::NSYM + 1) + ET<DD, PP>::NQ * ET<DD, PP>::NSYM) * sizeof(T)      \
                   : 0,                                                                                     \
               s>>>(m.conn.as<int>(), geo, m.E, u, us, mk, VMK, doMu, doMt);                             \
        break;
        FEM_MASS_U_CASE(0, 2, 1)
        FEM_MASS_U_CASE(1, 2, 2)
        FEM_MASS_U_CASE(2, 2, 3)
        FEM_MASS_U_CASE(3, 3, 1)
        FEM_MASS_U_CASE(4, 3, 2)
        FEM_MASS_U_CASE(5, 3, 3)
#undef FEM_MASS_U_CASE
        default: return fail(FEM_EINVAL, "element type");
    }
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

std::mutex g_init_mu;
bool g_init_done[64] = {};

}  // namespace

int tables_init_simt() {
    int dev = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (dev < 64 && g_init_done[dev]) return FEM_OK;
    std::vector<double> ref64(TAB_TOTAL, 0.0), q64(Q_TOTAL, 0.0);
    for (int t = 0; t < 6; ++t) {
        const RefElem* R = refelem_for_type(t);
        if (!R) return fail(FEM_EINVAL, "reference element tables failed");
        int o = type_tab_off(t);
        int nq = R->nq, np = R->np, d = R->d;
        for (int i = 0; i < nq * np; ++i) ref64[o + i] = R->phi[i];
        for (int i = 0; i < nq * np * d; ++i) ref64[o + nq * np + i] = R->grad[i];
        for (int i = 0; i < nq; ++i) ref64[o + nq * np * (1 + d) + i] = R->wq[i];
        int qo = q_off(t);
        size_t a = R->QM.size(), b = R->QK.size(), c = R->QT.size();
        if ((int)(a + b + c) != q_size(t)) return fail(FEM_EINVAL, "Q size mismatch");
        std::copy(R->QM.begin(), R->QM.end(), q64.begin() + qo);
        std::copy(R->QK.begin(), R->QK.end(), q64.begin() + qo + a);
        std::copy(R->QT.begin(), R->QT.end(), q64.begin() + qo + a + b);
    }
    // FP64 P1 mass factors sum_q w_q phi_q[i] phi_q[j], i <= j (triangles, then tetrahedra)
    double p1m[16] = {};
    for (int t : {0, 3}) {
        const RefElem* R = refelem_for_type(t);
        const int np = R->np, o = t == 0 ? 0 : 6;
        for (int i = 0; i < np; ++i)
            for (int j = i; j < np; ++j) {
                double v = 0.0;
                for (int q = 0; q < R->nq; ++q) v += R->wq[q] * R->phi[q * np + i] * R->phi[q * np + j];
                p1m[o + sym_index(np, i, j)] = v;
            }
    }
    // sine table of the FP64 laws: (sin, cos)(k pi/512), k = 0..1023, from
    // the first quadrant by symmetry, so that the zeros and ones are exact:
    // s_j = sin(j pi/512), c_j = sin((256 - j) pi/512) for j < 256 from the
    // host's long double sine (arguments in [0, pi/2], rounded once), then
    // quadrant q = k / 256 maps (s_j, c_j) to (c_j, -s_j), (-s_j, -c_j), (-c_j, s_j)
    std::vector<double2> sct(SC_TAB);
    const long double pi_l = 3.14159265358979323846264338327950288L;
    for (int k = 0; k < SC_TAB; ++k) {
        const int q = k / 256, j = k % 256;
        const double sj = (double)sinl((long double)j * pi_l / 512.0L);
        const double cj = (double)sinl((long double)(256 - j) * pi_l / 512.0L);
        sct[k] = q == 0 ? make_double2(sj, cj) : q == 1 ? make_double2(cj, -sj)
               : q == 2 ? make_double2(-sj, -cj) : make_double2(-cj, sj);
    }
    // one diagonal and one off-diagonal value: every entry of each kind must
    // agree to within rounding (rules symmetric in the vertices)
    double p1m2[4] = {};
    for (int t : {0, 3}) {
        const int np = t == 0 ? 3 : 4, o = t == 0 ? 0 : 6, c = t == 0 ? 0 : 1;
        const double dg = p1m[o + sym_index(np, 0, 0)], od = p1m[o + sym_index(np, 0, 1)];
        bool same = dg > 0.0 && od > 0.0;
        for (int i = 0; i < np; ++i)
            for (int j = i; j < np; ++j) {
                const double v = p1m[o + sym_index(np, i, j)], ref = i == j ? dg : od;
                same = same && std::fabs(v - ref) <= 1e-14 * ref;
            }
        if (!same) return fail(FEM_EINVAL, "P1 mass factors of the quadrature rule are not symmetric in the vertices");
        p1m2[2 * c] = dg;
        p1m2[2 * c + 1] = od;
    }
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_p1m2, p1m2, sizeof(p1m2)));
    // rules of one point per vertex: every point has the basis value
    // beta + gamma at one vertex and beta at the others, each vertex has one
    // point, and all weights are equal
    double p1q[10] = {};
    int p1q_on[2] = {0, 0};
    for (int t : {0, 3}) {
        const RefElem* R = refelem_for_type(t);
        const int np = R->np, c = t == 0 ? 0 : 1;
        if (R->nq != np) continue;
        const double w = R->wq[0];
        double al = R->phi[0], be = R->phi[0];
        for (int j = 1; j < np; ++j) {
            al = std::max(al, R->phi[j]);
            be = std::min(be, R->phi[j]);
        }
        bool ok = al - be > 1e-3;
        std::vector<int> hits(np, 0);
        for (int q = 0; q < np && ok; ++q) {
            ok = std::fabs(R->wq[q] - w) <= 4e-16 * std::fabs(w);
            int nal = 0;
            for (int j = 0; j < np; ++j) {
                const double v = R->phi[q * np + j];
                if (std::fabs(v - al) <= 4e-16 * std::fabs(al)) {
                    ++nal;
                    ++hits[j];
                } else {
                    ok = ok && std::fabs(v - be) <= 4e-16 * std::fabs(be);
                }
            }
            ok = ok && nal == 1;
        }
        for (int j = 0; j < np; ++j) ok = ok && hits[j] == 1;
        if (!ok) continue;
        p1q[5 * c] = be;
        p1q[5 * c + 1] = al - be;
        p1q[5 * c + 2] = w;
        p1q[5 * c + 3] = be * w;
        p1q[5 * c + 4] = (al - be) * w;
        p1q_on[c] = 1;
    }
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_p1q, p1q, sizeof(p1q)));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_p1q_on, p1q_on, sizeof(p1q_on)));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(g_sincos_tab, sct.data(), sizeof(double2) * SC_TAB));
    std::vector<float> ref32(ref64.begin(), ref64.end()), q32(q64.begin(), q64.end());
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_ref64, ref64.data(), sizeof(double) * TAB_TOTAL));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_ref32, ref32.data(), sizeof(float) * TAB_TOTAL));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(g_Q64, q64.data(), sizeof(double) * Q_TOTAL));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(g_Q32, q32.data(), sizeof(float) * Q_TOTAL));
    if (dev < 64) g_init_done[dev] = true;
    return FEM_OK;
}

// The FP32 law code of the FP32 and tensor-core element kernels (class LC),
// at u rounded to FP32.
template <int LC>
__global__ void __launch_bounds__(256) law_eval32_kernel(CoeffDev k, const double* __restrict__ u, int64_t n,
                                                         float* __restrict__ kv, float* __restrict__ dkv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float dk;
        const float v = k_eval<float, LC>(k, (float)u[i], dk);
        if (kv) kv[i] = v;
        if (dkv) dkv[i] = dk;
    }
}

int law_eval_fp32(const CoeffDev& k, const double* u, int64_t n, float* kv, float* dkv, cudaStream_t s) {
    if (n <= 0) return FEM_OK;
    int rc = tables_init_simt();
    if (rc) return rc;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = (n + 255) / 256;
    if (grid > (int64_t)nsm * 8) grid = (int64_t)nsm * 8;
    cudaGetLastError();   // clear any stale error before the launch check
    switch (law_class(k)) {
        case LC_POLY3: law_eval32_kernel<LC_POLY3><<<(unsigned)grid, 256, 0, s>>>(k, u, n, kv, dkv); break;
        case LC_SIN: law_eval32_kernel<LC_SIN><<<(unsigned)grid, 256, 0, s>>>(k, u, n, kv, dkv); break;
        default: law_eval32_kernel<LC_ANY><<<(unsigned)grid, 256, 0, s>>>(k, u, n, kv, dkv); break;
    }
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

int law_eval_fp64(const CoeffDev& k, const double* u, int64_t n, double* kv, double* dkv, cudaStream_t s) {
    if (n <= 0) return FEM_OK;
    int rc = tables_init_simt();
    if (rc) return rc;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = (n + 255) / 256;
    if (grid > (int64_t)nsm * 8) grid = (int64_t)nsm * 8;
    cudaGetLastError();   // clear any stale error before the launch check
    switch (law_code(k)) {
#define FEM_LAW_EVAL(L) \
    case L: law_eval_kernel<L><<<(unsigned)grid, 256, 0, s>>>(k, u, n, kv, dkv); break;
        FEM_LAW_EVAL(0) FEM_LAW_EVAL(1) FEM_LAW_EVAL(2) FEM_LAW_EVAL(3) FEM_LAW_EVAL(4)
        FEM_LAW_EVAL(5) FEM_LAW_EVAL(6) FEM_LAW_EVAL(7) FEM_LAW_EVAL(8) FEM_LAW_EVAL(9)
#undef FEM_LAW_EVAL
        default: return fail(FEM_EINVAL, "conductivity law");
    }
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

int element_simt_fp64(const fem_mesh& m, const CoeffDev& k, const double* u, double* VM, double* VK, double* VT,
                      cudaStream_t s, int64_t e0, int64_t e1) {
    int rc = tables_init_simt();
    if (rc) return rc;
    return dispatch<double>(m, k, u, m.geo64.as<double>(), VM, VK, VT, s, e0, e1);
}

int batch_simt_smem(int type, int fp64) {
    const int ktot = type_nq(type) * (1 + type_d(type) * (type_d(type) + 1) / 2 + type_d(type));
    return (ktot | 1) * BT * (fp64 ? 8 : 4);
}

template <typename T>
int batch_simt_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, int max_type_smem, int grid,
                      cudaStream_t s) {
    if (nitems <= 0) return FEM_OK;
    int rc = tables_init_simt();
    if (rc) return rc;
    auto kern = batch_simt_kernel<T>;
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_type_smem));
    if (grid > nitems) grid = nitems;
    cudaGetLastError();   // clear any stale error before the launch check
    kern<<<grid, BT, max_type_smem, s>>>(items, nitems, meshes);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}
template int batch_simt_launch<float>(const BatchItem*, int, const BatchMesh*, int, int, cudaStream_t);
template int batch_simt_launch<double>(const BatchItem*, int, const BatchMesh*, int, int, cudaStream_t);

int element_simt_fp32(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                      cudaStream_t s, int64_t e0, int64_t e1) {
    int rc = tables_init_simt();
    if (rc) return rc;
    return dispatch<float>(m, k, u, m.geo32.as<float>(), VM, VK, VT, s, e0, e1);
}

int element_mass_u(const fem_mesh& m, const CoeffDev& mk, const double* u, const double* us, int fp64, void* VMK,
                   bool doMu, bool doMt, cudaStream_t s) {
    int rc = tables_init_simt();
    if (rc) return rc;
    if (m.perq) {
        if (fp64)
            return launch_mass_u<double, true>(m, mk, u, us, m.geoq64.as<double>(), static_cast<double*>(VMK), doMu,
                                               doMt, s);
        return launch_mass_u<float, true>(m, mk, u, us, m.geoq32.as<float>(), static_cast<float*>(VMK), doMu, doMt, s);
    }
    if (fp64)
        return launch_mass_u<double, false>(m, mk, u, us, m.geo64.as<double>(), static_cast<double*>(VMK), doMu, doMt,
                                            s);
    return launch_mass_u<float, false>(m, mk, u, us, m.geo32.as<float>(), static_cast<float*>(VMK), doMu, doMt, s);
}

}  // namespace fem
