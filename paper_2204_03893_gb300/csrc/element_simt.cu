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
#include <mutex>
#include <vector>

#include "fem_internal.h"
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

// nodal values: FP64 as given; the FP32 path splits each gathered value
// as hi + lo (split_f64) so that the differences u_i - u_0 that carry the
// gradient keep FP32 relative accuracy.

// X row and V = X Q of element e (thread-private X row in shared memory).
template <typename ETy, typename T>
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
    T b = geo[e];
    T A[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) A[t] = geo[(1 + t) * gs + e];
    // --- X = Lambda, Lambda (.) W, tangent factors
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
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

template <typename ETy, typename T>
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
        simt_element<ETy, T>(e, conn, geo, gs, u, k, mass, VM, VK, VT, X);
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
        if (threadIdx.x >= w.count || e >= bm.E) continue;
        const T* geo = static_cast<const T*>(sizeof(T) == 8 ? (const void*)bm.geo64 : (const void*)bm.geo32);
        const double* u = bm.u;
        T* VM = bm.vM ? static_cast<T*>(bm.VM) : nullptr;
        T* VK = bm.vK ? static_cast<T*>(bm.VK) : nullptr;
        T* VT = bm.vT ? static_cast<T*>(bm.VT) : nullptr;
        const T mass = (T)bm.mass;
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

template <typename ETy, typename T>
int launch_simt(const fem_mesh& m, const CoeffDev& k, const double* u, const T* geo, T* VM, T* VK,
                T* VT, cudaStream_t s, int64_t e0, int64_t e1) {
    const int64_t E = e1 - e0;
    if (E <= 0) return FEM_OK;
    constexpr int KTOT = ETy::KM + ETy::KK + ETy::KT;
    constexpr int LD = KTOT | 1;
    size_t smem = sizeof(T) * (size_t)LD * BT;
    auto kern = element_simt_kernel<ETy, T>;
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
    kern<<<(unsigned)grid, BT, smem, s>>>(m.conn.as<int>() + e0 * ETy::NP, geo + e0, E, m.E, u, k, (T)m.m,
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
    switch (m.type) {
        case 0: return launch_simt<ET<2, 1>, T>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 1: return launch_simt<ET<2, 2>, T>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 2: return launch_simt<ET<2, 3>, T>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 3: return launch_simt<ET<3, 1>, T>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 4: return launch_simt<ET<3, 2>, T>(m, k, u, geo, VM, VK, VT, s, e0, e1);
        case 5: return launch_simt<ET<3, 3>, T>(m, k, u, geo, VM, VK, VT, s, e0, e1);
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

template <typename ETy, typename T>
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
            const T b = geo[e];
            T Xu[NQ], Xt[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
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

template <typename T>
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
        mass_u_kernel<ET<DD, PP>, T>                                                                     \
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
    std::vector<float> ref32(ref64.begin(), ref64.end()), q32(q64.begin(), q64.end());
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_ref64, ref64.data(), sizeof(double) * TAB_TOTAL));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_ref32, ref32.data(), sizeof(float) * TAB_TOTAL));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(g_Q64, q64.data(), sizeof(double) * Q_TOTAL));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(g_Q32, q32.data(), sizeof(float) * Q_TOTAL));
    if (dev < 64) g_init_done[dev] = true;
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
    if (fp64) return launch_mass_u<double>(m, mk, u, us, m.geo64.as<double>(), static_cast<double*>(VMK), doMu, doMt, s);
    return launch_mass_u<float>(m, mk, u, us, m.geo32.as<float>(), static_cast<float*>(VMK), doMu, doMt, s);
}

}  // namespace fem
