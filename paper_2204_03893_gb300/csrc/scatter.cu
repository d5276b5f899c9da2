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

template <int NP, typename T>
__global__ void __launch_bounds__(256) scatter_kernel(const int* __restrict__ seg_ptr, const int* __restrict__ contrib,
                                                      int64_t nnz, const T* __restrict__ VM, const T* __restrict__ VK,
                                                      const T* __restrict__ VT, T* __restrict__ vM,
                                                      T* __restrict__ vK, T* __restrict__ vT) {
    constexpr int NT = NP * NP, NSYM = NP * (NP + 1) / 2;
    const bool dM = vM != nullptr, dK = vK != nullptr, dT = vT != nullptr;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        const int a = seg_ptr[s], b = seg_ptr[s + 1];
        T am = T(0), ak = T(0), at = T(0);
        for (int p = a; p < b; ++p) {
            const int c = contrib[p];
            const int e = c / NT;
            const int l = c - e * NT;
            if (dT) at += VT[(int64_t)e * NT + l];
            if (dM | dK) {
                const int i = l / NP, j = l - (l / NP) * NP;
                const int lo = i < j ? i : j, hi = i < j ? j : i;
                const int si = lo * NP - (lo * (lo - 1)) / 2 + (hi - lo);
                if (dM) am += VM[(int64_t)e * NSYM + si];
                if (dK) ak += VK[(int64_t)e * NSYM + si];
            }
        }
        if (dM) vM[s] = am;
        if (dK) vK[s] = ak;
        if (dT) vT[s] = at;
    }
}

template <typename T>
int run(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s) {
    if (m.nnz <= 0) return FEM_OK;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (m.nnz + 255) / 256;
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
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
