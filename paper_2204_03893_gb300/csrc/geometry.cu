// geometry.cu -- per-element geometric factors, computed once per mesh.
//
// Section 3 step 3: x = a + B_e xhat with B_e = [x_1 - x_0, ..., x_d - x_0];
// the element integrals need b_e = |det B_e| and A_e = (B_e^T B_e)^-1 =
// B_e^-1 B_e^-T (the chain rule J_phi_e = J_phihat B_e^-1).  Algorithm 2
// takes b and W from the mesh alone, and Section 5 lists them among the
// quantities that never change with u.
//
// Output layout (structure of arrays, coalesced for one thread per element):
//   geo[0*E + e] = b_e,  geo[(1+t)*E + e] = A_e[a][b] for the t-th (a<=b).
// P1 simplices also keep the Gram matrix G A_e G^T of every element (G the
// constant reference gradients [-1 ... -1; I]; element-major, n_sym FP64
// values in symmetric storage): the part of K_e that does not change with u
// (K_e = b_e (sum_q w_q k(u_q)) G A_e G^T, Section 4.2 with the point sum
// taken first), so the FP64 element kernel forms only its scalar factor.
// geo64: everything in FP64.  geo32: edge vectors in FP64 (the coordinates
// are FP64 and nearby vertices cancel), det / inverse / A in FP32; elements
// whose condition estimate kappa = ||B||_F^d / |det B| exceeds 1e3 are
// recomputed in FP64 and rounded.
#include "fem_internal.h"
#include "refelem.h"

namespace fem {

namespace {

constexpr double KAPPA_MAX = 1e3;

template <int D, typename T>
__device__ __forceinline__ T det_inv(const T B[D][D], T Bi[D][D]) {
    T det;
    if constexpr (D == 2) {
        det = B[0][0] * B[1][1] - B[0][1] * B[1][0];
        T r = T(1) / det;
        Bi[0][0] = B[1][1] * r;
        Bi[0][1] = -B[0][1] * r;
        Bi[1][0] = -B[1][0] * r;
        Bi[1][1] = B[0][0] * r;
    } else {
        T c00 = B[1][1] * B[2][2] - B[1][2] * B[2][1];
        T c01 = B[1][2] * B[2][0] - B[1][0] * B[2][2];
        T c02 = B[1][0] * B[2][1] - B[1][1] * B[2][0];
        det = B[0][0] * c00 + B[0][1] * c01 + B[0][2] * c02;
        T r = T(1) / det;
        Bi[0][0] = c00 * r;
        Bi[1][0] = c01 * r;
        Bi[2][0] = c02 * r;
        Bi[0][1] = (B[0][2] * B[2][1] - B[0][1] * B[2][2]) * r;
        Bi[1][1] = (B[0][0] * B[2][2] - B[0][2] * B[2][0]) * r;
        Bi[2][1] = (B[0][1] * B[2][0] - B[0][0] * B[2][1]) * r;
        Bi[0][2] = (B[0][1] * B[1][2] - B[0][2] * B[1][1]) * r;
        Bi[1][2] = (B[0][2] * B[1][0] - B[0][0] * B[1][2]) * r;
        Bi[2][2] = (B[0][0] * B[1][1] - B[0][1] * B[1][0]) * r;
    }
    return det;
}

// the constant conductivity tensor c (3 x 3 row-major, entry (a, b) at
// 3a + b, whatever d; the identity for an isotropic conductivity)
struct Cond {
    double c[9];
};

// A = Bi c Bi^T (Section 7, anisotropic conductivity: A_e = B_e^-1 c B_e^-T;
// c = I gives Bi Bi^T), upper triangle in (a<=b) order
template <int D, typename T>
__device__ __forceinline__ void make_A(const T Bi[D][D], const Cond& cd, T* A) {
    T cb[D][D];   // c Bi^T
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            T s = T(0);
#pragma unroll
            for (int l = 0; l < D; ++l) s += (T)cd.c[k * 3 + l] * Bi[b][l];
            cb[k][b] = s;
        }
    int t = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) s += Bi[a][k] * cb[k][b];
            A[t++] = s;
        }
}

template <int D>
__global__ void geometry_kernel(const double* __restrict__ X, const int* __restrict__ conn, int64_t E, int np,
                                int64_t n, double* __restrict__ geo64, float* __restrict__ geo32, Cond cd,
                                unsigned long long* __restrict__ counters /* [0] bad index, [1] degenerate, [2] flagged */) {
    constexpr int NS = D * (D + 1) / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int* ce = conn + e * np;
        bool bad = false;
        for (int i = 0; i < np; ++i) {
            int v = ce[i];
            bad |= (v < 0) | ((int64_t)v >= n);
        }
        if (bad) {
            atomicAdd(&counters[0], 1ull);
            for (int t = 0; t <= NS; ++t) { geo64[t * E + e] = 0.0; geo32[t * E + e] = 0.0f; }
            continue;
        }
        double B[D][D];
        int v0 = ce[0];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            int vc = ce[c + 1];
#pragma unroll
            for (int r = 0; r < D; ++r) B[r][c] = X[(int64_t)vc * D + r] - X[(int64_t)v0 * D + r];
        }
        double Bi[D][D];
        double det = det_inv<D, double>(B, Bi);
        double nf = 0.0;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) nf += B[r][c] * B[r][c];
        double nfd = (D == 2) ? nf : nf * sqrt(nf);   // ||B||_F^d
        if (!(fabs(det) > 1e-14 * nfd)) {
            atomicAdd(&counters[1], 1ull);
            for (int t = 0; t <= NS; ++t) { geo64[t * E + e] = 0.0; geo32[t * E + e] = 0.0f; }
            continue;
        }
        double A[NS];
        make_A<D, double>(Bi, cd, A);
        geo64[e] = fabs(det);
#pragma unroll
        for (int t = 0; t < NS; ++t) geo64[(1 + t) * E + e] = A[t];

        // FP32 cache
        float Bf[D][D], Bif[D][D];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) Bf[r][c] = (float)B[r][c];
        float detf = det_inv<D, float>(Bf, Bif);
        float nff = 0.0f;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) nff += Bf[r][c] * Bf[r][c];
        float kappa = ((D == 2) ? nff : nff * sqrtf(nff)) / fabsf(detf);
        if (kappa > (float)KAPPA_MAX || !(kappa == kappa)) {
            atomicAdd(&counters[2], 1ull);
            geo32[e] = (float)fabs(det);
#pragma unroll
            for (int t = 0; t < NS; ++t) geo32[(1 + t) * E + e] = (float)A[t];
        } else {
            float Af[NS];
            make_A<D, float>(Bif, cd, Af);
            geo32[e] = fabsf(detf);
#pragma unroll
            for (int t = 0; t < NS; ++t) geo32[(1 + t) * E + e] = Af[t];
        }
    }
}

// ---------------------------------------------------- per-point geometry
// Section 7: with an isoparametric mapping x(xhat) = sum_i x_i phi_i(xhat)
// the Jacobian B_q = sum_i x_i (grad phi_i(xhat_q))^T depends on the
// quadrature point (n_q determinants and d^2 n_q Jacobian entries per
// element), and a conductivity tensor may vary over the points:
// A_q = B_q^-1 c_q B_q^-T.  One thread per (element, point); the cache is
// geoq[comp * E n_q + e n_q + q], comp 0 = |det B_q|, 1.. = A_q (upper
// triangle).  The FP32 cache holds the FP64 values rounded.
__constant__ double c_gq[2200];   // reference gradients at the points, per element type
struct GqType {
    int off[6];
};

template <int D>
__global__ void geometry_q_kernel(const double* __restrict__ X, const int* __restrict__ conn, int64_t E, int np,
                                  int nq, int goff, int iso, const double* __restrict__ cfield, Cond cd,
                                  double* __restrict__ g64, float* __restrict__ g32,
                                  unsigned long long* __restrict__ counters) {
    constexpr int NS = D * (D + 1) / 2;
    const int64_t m = E * nq;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k / nq;
        const int q = (int)(k - e * nq);
        const int* ce = conn + e * np;
        double B[D][D];
        if (iso) {
            const double* G = c_gq + goff + q * np * D;
#pragma unroll
            for (int r = 0; r < D; ++r)
#pragma unroll
                for (int c = 0; c < D; ++c) B[r][c] = 0.0;
            for (int i = 0; i < np; ++i) {
                const int vi = ce[i];
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    const double x = X[(int64_t)vi * D + r];
#pragma unroll
                    for (int c = 0; c < D; ++c) B[r][c] = fma(x, G[i * D + c], B[r][c]);
                }
            }
        } else {
            const int v0 = ce[0];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const int vc = ce[c + 1];
#pragma unroll
                for (int r = 0; r < D; ++r) B[r][c] = X[(int64_t)vc * D + r] - X[(int64_t)v0 * D + r];
            }
        }
        double Bi[D][D];
        const double det = det_inv<D, double>(B, Bi);
        double nf = 0.0;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) nf += B[r][c] * B[r][c];
        const double nfd = (D == 2) ? nf : nf * sqrt(nf);
        if (!(fabs(det) > 1e-14 * nfd)) {
            atomicAdd(&counters[1], 1ull);
            for (int t = 0; t <= NS; ++t) {
                g64[t * m + k] = 0.0;
                g32[t * m + k] = 0.0f;
            }
            continue;
        }
        Cond cq = cd;
        if (cfield) {
            const double* cf = cfield + k * D * D;
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) cq.c[a * 3 + b] = cf[a * D + b];
        }
        double A[NS];
        make_A<D, double>(Bi, cq, A);
        g64[k] = fabs(det);
        g32[k] = (float)fabs(det);
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            g64[(1 + t) * m + k] = A[t];
            g32[(1 + t) * m + k] = (float)A[t];
        }
    }
}

int gq_tables_init(GqType& out) {
    static bool done[64] = {};
    static GqType offs;
    int dev = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 64 && done[dev]) {
        out = offs;
        return FEM_OK;
    }
    std::vector<double> g;
    for (int t = 0; t < 6; ++t) {
        const RefElem* R = refelem_for_type(t);
        if (!R) return fail(FEM_EINVAL, "reference element tables failed");
        offs.off[t] = (int)g.size();
        g.insert(g.end(), R->grad.begin(), R->grad.end());
    }
    if (g.size() > sizeof(c_gq) / sizeof(double)) return fail(FEM_EINVAL, "gradient tables too large");
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_gq, g.data(), sizeof(double) * g.size()));
    if (dev < 64) done[dev] = true;
    out = offs;
    return FEM_OK;
}

// G A G^T needs no multiplications: entry (i, j), i, j >= 1, is A[i-1][j-1];
// entry (0, j) minus the (j-1)-th column sum of A; entry (0, 0) the sum of
// all of A (the column sums added in order).
template <int D>
__global__ void __launch_bounds__(256) p1_gram_kernel(const double* __restrict__ geo, int64_t E,
                                                      double* __restrict__ gram) {
    constexpr int NP = D + 1, NSYM = NP * (NP + 1) / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        double A[D * (D + 1) / 2];
#pragma unroll
        for (int t = 0; t < D * (D + 1) / 2; ++t) A[t] = geo[(1 + t) * E + e];
        auto At = [&](int a, int c) {   // A[a][c] from the upper triangle
            const int lo = a < c ? a : c, hi = a < c ? c : a;
            return A[lo * D - (lo * (lo - 1)) / 2 + (hi - lo)];
        };
        double g[NSYM];
        double tot = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            double v = At(0, c);
#pragma unroll
            for (int a = 1; a < D; ++a) v += At(a, c);
            g[sym_index(NP, 0, c + 1)] = -v;
            tot = c == 0 ? v : tot + v;
        }
        g[0] = tot;   // sym(0, 0) = 0
#pragma unroll
        for (int i = 1; i < NP; ++i)
#pragma unroll
            for (int j = i; j < NP; ++j) g[sym_index(NP, i, j)] = At(i - 1, j - 1);
        double* o = gram + e * NSYM;
#pragma unroll
        for (int t = 0; t < NSYM; ++t) o[t] = g[t];
    }
}

}  // namespace

// The per-point cache of a mesh in per-point mode (isoparametric and/or a
// conductivity field); FEM_EDEGENERATE if some det B_q vanishes.
int geometry_q_run(fem_mesh& m, cudaStream_t s) {
    GqType offs;
    int rc = gq_tables_init(offs);
    if (rc) return rc;
    const int ngeo = 1 + m.d * (m.d + 1) / 2;
    const size_t pts = (size_t)m.E * m.nq;
    if ((rc = buf_alloc(m.geoq64, sizeof(double) * ngeo * pts + 8, s))) return rc;
    if ((rc = buf_alloc(m.geoq32, sizeof(float) * ngeo * pts + 8, s))) return rc;
    DevBuf cnt;
    if ((rc = buf_alloc(cnt, 4 * sizeof(unsigned long long), s))) return rc;
    FEM_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, cnt.bytes, s));
    Cond cd;
    for (int i = 0; i < 9; ++i) cd.c[i] = m.cond[i];
    if (pts > 0) {
        cudaGetLastError();   // clear any stale error before the launch check
        int64_t blocks = ((int64_t)pts + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        const double* cf = m.cfield.ptr ? m.cfield.as<double>() : nullptr;
        if (m.d == 2)
            geometry_q_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(m.coords.as<double>(), m.conn.as<int>(), m.E, m.np,
                                                                  m.nq, offs.off[m.type], m.iso ? 1 : 0, cf, cd,
                                                                  m.geoq64.as<double>(), m.geoq32.as<float>(),
                                                                  cnt.as<unsigned long long>());
        else
            geometry_q_kernel<3><<<(unsigned)blocks, 256, 0, s>>>(m.coords.as<double>(), m.conn.as<int>(), m.E, m.np,
                                                                  m.nq, offs.off[m.type], m.iso ? 1 : 0, cf, cd,
                                                                  m.geoq64.as<double>(), m.geoq32.as<float>(),
                                                                  cnt.as<unsigned long long>());
        FEM_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long h[4] = {0, 0, 0, 0};
    FEM_CUDA_TRY(cudaMemcpyAsync(h, cnt.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    buf_free(cnt, s);
    if (h[1]) return fail(FEM_EDEGENERATE, std::to_string(h[1]) + " quadrature point(s) with a degenerate Jacobian");
    return FEM_OK;
}

int geometry_run(fem_mesh& m, cudaStream_t s) {
    int ngeo = 1 + m.d * (m.d + 1) / 2;
    int rc = buf_alloc(m.geo64, sizeof(double) * ngeo * (size_t)m.E, s);
    if (rc) return rc;
    rc = buf_alloc(m.geo32, sizeof(float) * ngeo * (size_t)m.E, s);
    if (rc) return rc;
    DevBuf cnt;
    rc = buf_alloc(cnt, 4 * sizeof(unsigned long long), s);
    if (rc) return rc;
    FEM_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, cnt.bytes, s));
    Cond cd;
    for (int i = 0; i < 9; ++i) cd.c[i] = m.cond[i];
    if (m.E > 0) {
        cudaGetLastError();   // clear any stale error before the launch check
        int threads = 256;
        int64_t blocks = (m.E + threads - 1) / threads;
        if (blocks > 152 * 64) blocks = 152 * 64;
        if (m.d == 2)
            geometry_kernel<2><<<(unsigned)blocks, threads, 0, s>>>(m.coords.as<double>(), m.conn.as<int>(), m.E, m.np,
                                                                    m.n, m.geo64.as<double>(), m.geo32.as<float>(),
                                                                    cd, cnt.as<unsigned long long>());
        else
            geometry_kernel<3><<<(unsigned)blocks, threads, 0, s>>>(m.coords.as<double>(), m.conn.as<int>(), m.E, m.np,
                                                                    m.n, m.geo64.as<double>(), m.geo32.as<float>(),
                                                                    cd, cnt.as<unsigned long long>());
        FEM_CUDA_TRY(cudaGetLastError());
    }
    if (m.type == 0 || m.type == 3) {   // P1: the elements' Gram matrices
        const size_t nsym = (size_t)m.np * (m.np + 1) / 2;
        if ((rc = buf_alloc(m.gram64, sizeof(double) * nsym * (size_t)(m.E > 0 ? m.E : 1), s))) return rc;
        if (m.E > 0) {
            int64_t blocks = (m.E + 255) / 256;
            if (blocks > 152 * 64) blocks = 152 * 64;
            if (m.d == 2)
                p1_gram_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(m.geo64.as<double>(), m.E, m.gram64.as<double>());
            else
                p1_gram_kernel<3><<<(unsigned)blocks, 256, 0, s>>>(m.geo64.as<double>(), m.E, m.gram64.as<double>());
            FEM_CUDA_TRY(cudaGetLastError());
        }
    }
    unsigned long long h[4] = {0, 0, 0, 0};
    FEM_CUDA_TRY(cudaMemcpyAsync(h, cnt.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    buf_free(cnt, s);
    if (h[0]) return fail(FEM_EINVAL, "connectivity index out of range in " + std::to_string(h[0]) + " element(s)");
    if (h[1]) return fail(FEM_EDEGENERATE, std::to_string(h[1]) + " degenerate element(s)");
    m.n_flagged = (int64_t)h[2];
    return FEM_OK;
}

}  // namespace fem
