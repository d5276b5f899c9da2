// csr_ops.cu -- Newton quantities from the assembled matrices, FP64, on the
// mesh's CSR pattern (Section 5, implicit Euler):
//   residual  F = M (u - u^s) + dt K u - dt b,  with ||F||_2 and ||F||_inf,
//   Jacobian  J = Mt + M + dt (K + T) - dt B,
//   y = alpha A x + beta y.
// Every reduction runs in one fixed order: a row's terms by ascending
// column; the norms by fixed chunks of 256 rows (a fixed tree in each), then
// the chunk partials in ascending order by one block -- results do not
// depend on the device or launch.
#include <cmath>

#include "fem_internal.h"

namespace fem {

namespace {

constexpr int ROWS = 256;   // rows per norm chunk (one block)

__global__ void __launch_bounds__(256) spmv_kernel(const int* __restrict__ rp, const int* __restrict__ ci, int64_t n,
                                                   const double* __restrict__ a, double alpha,
                                                   const double* __restrict__ x, double beta, double* __restrict__ y) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = rp[r]; k < rp[r + 1]; ++k) s = fma(a[k], x[ci[k]], s);
        y[r] = beta == 0.0 ? alpha * s : fma(beta, y[r], alpha * s);
    }
}

// One block per chunk of ROWS rows: F of each row, then the chunk's sum of
// squares and largest magnitude.
__global__ void __launch_bounds__(ROWS) residual_kernel(const int* __restrict__ rp, const int* __restrict__ ci,
                                                        int64_t n, const double* __restrict__ M,
                                                        const double* __restrict__ K, const double* __restrict__ b,
                                                        const double* __restrict__ u, const double* __restrict__ us,
                                                        double dt, double* __restrict__ F,
                                                        double2* __restrict__ part) {
    __shared__ double ss[ROWS / 32], sm[ROWS / 32];
    const int64_t r = blockIdx.x * (int64_t)ROWS + threadIdx.x;
    double f = 0.0;
    if (r < n) {
        double s = 0.0;
        for (int k = rp[r]; k < rp[r + 1]; ++k) {
            const int j = ci[k];
            const double uj = u[j];
            s += M[k] * (uj - us[j]) + dt * K[k] * uj;
        }
        f = s - (b ? dt * b[r] : 0.0);
        F[r] = f;
    }
    double q = f * f, mx = fabs(f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        q += __shfl_xor_sync(0xffffffffu, q, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = q;
        sm[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, m = 0.0;
        for (int w = 0; w < ROWS / 32; ++w) {
            t += ss[w];
            m = fmax(m, sm[w]);
        }
        part[blockIdx.x] = make_double2(t, m);
    }
}

__global__ void __launch_bounds__(1024) norms_kernel(const double2* __restrict__ part, int64_t nparts,
                                                     double* __restrict__ norms) {
    __shared__ double ss[32], sm[32];
    double t = 0.0, m = 0.0;
    for (int64_t i = threadIdx.x; i < nparts; i += 1024) {
        t += part[i].x;
        m = fmax(m, part[i].y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_xor_sync(0xffffffffu, t, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = t;
        sm[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 32; ++w) {
            a += ss[w];
            b = fmax(b, sm[w]);
        }
        norms[0] = sqrt(a);
        norms[1] = b;
    }
}

__global__ void __launch_bounds__(256) jacobian_kernel(int64_t nnz, double dt, const double* __restrict__ M,
                                                       const double* __restrict__ Mt, const double* __restrict__ K,
                                                       const double* __restrict__ T, const double* __restrict__ B,
                                                       double* __restrict__ J) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        const double kt = K[s] + (T ? T[s] : 0.0);
        J[s] = (Mt ? Mt[s] : 0.0) + M[s] + dt * kt - (B ? dt * B[s] : 0.0);
    }
}

int grid_for_rows(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

int csr_spmv(const fem_mesh& m, const double* vals, double alpha, const double* x, double beta, double* y,
             cudaStream_t s) {
    if (m.n <= 0) return FEM_OK;
    cudaGetLastError();   // clear any stale error before the launch check
    spmv_kernel<<<grid_for_rows(m.n, 256), 256, 0, s>>>(m.row_ptr.as<int>(), m.col_idx.as<int>(), m.n, vals, alpha,
                                                        x, beta, y);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

int csr_residual(fem_mesh& m, const double* vM, const double* vK, const double* b, const double* u, const double* us,
                 double dt, double* F, double* norms, cudaStream_t s) {
    const int64_t nb = (m.n + ROWS - 1) / ROWS;
    if (m.n <= 0) {
        if (norms) FEM_CUDA_TRY(cudaMemsetAsync(norms, 0, 2 * sizeof(double), s));
        return FEM_OK;
    }
    int rc = buf_alloc(m.npart, sizeof(double2) * (size_t)nb, s);
    if (rc) return rc;
    cudaGetLastError();   // clear any stale error before the launch checks
    residual_kernel<<<(unsigned)nb, ROWS, 0, s>>>(m.row_ptr.as<int>(), m.col_idx.as<int>(), m.n, vM, vK, b, u, us, dt,
                                                  F, m.npart.as<double2>());
    if (norms) norms_kernel<<<1, 1024, 0, s>>>(m.npart.as<double2>(), nb, norms);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

int csr_jacobian(const fem_mesh& m, double dt, const double* vM, const double* vMt, const double* vK,
                 const double* vT, const double* vB, double* vJ, cudaStream_t s) {
    if (m.nnz <= 0) return FEM_OK;
    cudaGetLastError();   // clear any stale error before the launch check
    jacobian_kernel<<<grid_for_rows(m.nnz, 256), 256, 0, s>>>(m.nnz, dt, vM, vMt, vK, vT, vB, vJ);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // namespace fem
