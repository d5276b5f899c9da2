// scatter.cu -- global assembly of the element matrices into CSR values.
//
// Algorithm 2 line 12 ("form the matrices M and C from V_m and V_c and the
// set of indices of nonzero entries"); Section 3 step 2, eq. assemblage_1:
// M_ij = sum over elements of the element integrals.  Each CSR slot s sums
// its contributions contrib[seg_ptr[s] .. seg_ptr[s+1]) in ascending element
// entry order c = (e n_p + i) n_p + j, one thread per slot, with no atomics:
// the result is bit-reproducible run to run and the summation order is the
// element order of Algorithm 1.  M and K come from the symmetric element
// storage (entry (i,j) and (j,i) share V[e][sym(min,max)]), T from the full
// n_p x n_p storage.
#include "fem_internal.h"

namespace fem {

namespace {

template <typename T>
__device__ __forceinline__ void store_stream(T* p, T v) {
    __stcs(p, v);   // outputs are not re-read by this kernel: evict-first
}

// Each thread sums SPT slots spaced blockDim.x apart (coalesced across the
// warp) with independent load chains, so that several gathers are in flight.
constexpr int SPT = 4;

template <int NP, typename T>
__global__ void __launch_bounds__(256) scatter_kernel(const int* __restrict__ seg_ptr, const int* __restrict__ contrib,
                                                      int64_t nnz, const T* __restrict__ VM, const T* __restrict__ VK,
                                                      const T* __restrict__ VT, T* __restrict__ vM,
                                                      T* __restrict__ vK, T* __restrict__ vT) {
    constexpr int NT = NP * NP, NSYM = NP * (NP + 1) / 2;
    const bool dM = vM != nullptr, dK = vK != nullptr, dT = vT != nullptr;
    const int64_t chunk = (int64_t)blockDim.x * SPT;
    for (int64_t base = blockIdx.x * chunk; base < nnz; base += (int64_t)gridDim.x * chunk) {
        int a[SPT], b[SPT];
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int64_t s = base + k * blockDim.x + threadIdx.x;
            a[k] = s < nnz ? __ldg(seg_ptr + s) : 0;
            b[k] = s < nnz ? __ldg(seg_ptr + s + 1) : 0;
        }
        T am[SPT], ak[SPT], at[SPT];
#pragma unroll
        for (int k = 0; k < SPT; ++k) am[k] = ak[k] = at[k] = T(0);
        int len = 0;
#pragma unroll
        for (int k = 0; k < SPT; ++k) len = max(len, b[k] - a[k]);
        for (int p = 0; p < len; ++p) {
            int c[SPT];
#pragma unroll
            for (int k = 0; k < SPT; ++k) c[k] = (a[k] + p < b[k]) ? __ldg(contrib + a[k] + p) : -1;
#pragma unroll
            for (int k = 0; k < SPT; ++k) {
                if (c[k] < 0) continue;
                const int e = c[k] / NT;
                const int l = c[k] - e * NT;
                if (dT) at[k] += __ldg(VT + (int64_t)e * NT + l);
                if (dM | dK) {
                    const int i = l / NP, j = l - (l / NP) * NP;
                    const int lo = i < j ? i : j, hi = i < j ? j : i;
                    const int si = lo * NP - (lo * (lo - 1)) / 2 + (hi - lo);
                    if (dM) am[k] += __ldg(VM + (int64_t)e * NSYM + si);
                    if (dK) ak[k] += __ldg(VK + (int64_t)e * NSYM + si);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int64_t s = base + k * blockDim.x + threadIdx.x;
            if (s < nnz) {
                if (dM) store_stream(vM + s, am[k]);
                if (dK) store_stream(vK + s, ak[k]);
                if (dT) store_stream(vT + s, at[k]);
            }
        }
    }
}

template <typename T>
int run(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s) {
    if (m.nnz <= 0) return FEM_OK;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (m.nnz + 256 * SPT - 1) / (256 * SPT);
    if (blocks > (int64_t)nsm * 8) blocks = (int64_t)nsm * 8;
    const int* sp = m.seg_ptr.as<int>();
    const int* ct = m.contrib.as<int>();
    cudaGetLastError();   // clear any stale error before the launch check
    switch (m.np) {
        case 3: scatter_kernel<3, T><<<(unsigned)blocks, 256, 0, s>>>(sp, ct, m.nnz, VM, VK, VT, vM, vK, vT); break;
        case 4: scatter_kernel<4, T><<<(unsigned)blocks, 256, 0, s>>>(sp, ct, m.nnz, VM, VK, VT, vM, vK, vT); break;
        case 6: scatter_kernel<6, T><<<(unsigned)blocks, 256, 0, s>>>(sp, ct, m.nnz, VM, VK, VT, vM, vK, vT); break;
        case 10: scatter_kernel<10, T><<<(unsigned)blocks, 256, 0, s>>>(sp, ct, m.nnz, VM, VK, VT, vM, vK, vT); break;
        case 20: scatter_kernel<20, T><<<(unsigned)blocks, 256, 0, s>>>(sp, ct, m.nnz, VM, VK, VT, vM, vK, vT); break;
        default: return fail(FEM_EINVAL, "unsupported n_p");
    }
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // namespace

int scatter_fp64(const fem_mesh& m, const double* VM, const double* VK, const double* VT, double* vM, double* vK,
                 double* vT, cudaStream_t s) {
    return run<double>(m, VM, VK, VT, vM, vK, vT, s);
}

int scatter_fp32(const fem_mesh& m, const float* VM, const float* VK, const float* VT, float* vM, float* vK,
                 float* vT, cudaStream_t s) {
    return run<float>(m, VM, VK, VT, vM, vK, vT, s);
}

}  // namespace fem
