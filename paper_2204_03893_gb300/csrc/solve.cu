// solve.cu -- the linear and nonlinear solves of the heat problem, FP64:
// a Jacobi-preconditioned BiCGStab on the mesh's CSR pattern, and one
// implicit Euler step solved by Newton's method (Section 5: F(u) = M (u -
// u^s) + dt K(u) u - dt f(u), dF/du = M + dt (K + T) - dt B for a constant
// mass coefficient; Section 6, Experiment 2).  The paper solves the Newton
// systems with MATLAB's backslash or with GMRES; the linear solver is not
// part of its method.
//
// Every reduction runs in a fixed order (chunks of 256 entries, fixed trees,
// then the chunks in ascending order), and the scalars of the iteration stay
// on the device (computed by one thread from the reductions), so a solve
// gives the same bits run to run; the host reads one number per iteration to
// test convergence.
#include <cmath>

#include "fem_internal.h"

namespace fem {

namespace {

constexpr int RB = 256;   // entries per reduction chunk (one block)

// scalars of the iteration, in device memory
enum { S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_BETA, S_RV, S_TS, S_TT, S_RR, S_SS, S_BB, S_N };

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < RB / 32; ++w) t += sh[w];
    __syncthreads();
    return t;
}

// part[block][j] = sum over the block's chunk of x_j . y_j for up to two pairs
__global__ void __launch_bounds__(RB) dot2_partial(int64_t n, const double* __restrict__ x0,
                                                   const double* __restrict__ y0, const double* __restrict__ x1,
                                                   const double* __restrict__ y1, double2* __restrict__ part) {
    __shared__ double sh[RB / 32];
    const int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x;
    const double a = i < n ? x0[i] * y0[i] : 0.0;
    const double b = (x1 && i < n) ? x1[i] * y1[i] : 0.0;
    const double sa = block_sum(a, sh);
    const double sb = block_sum(b, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sa, sb);
}

// out[j0] = sum of the partials (.x), out[j1] = (.y) if j1 >= 0
__global__ void __launch_bounds__(1024) dot2_final(const double2* __restrict__ part, int64_t nb, double* __restrict__ sc,
                                                   int j0, int j1) {
    __shared__ double sa[32], sb[32];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < nb; i += 1024) {
        a += part[i].x;
        b += part[i].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < 32; ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        sc[j0] = ta;
        if (j1 >= 0) sc[j1] = tb;
    }
}

// dinv[r] = 1 / A[r][r] (the diagonal slot found by binary search in the row)
__global__ void jacobi_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ a,
                              int64_t n, double* __restrict__ dinv) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        int lo = rp[r], hi = rp[r + 1] - 1;
        double d = 0.0;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            if (ci[mid] == r) {
                d = a[mid];
                break;
            }
            if (ci[mid] < r) lo = mid + 1;
            else hi = mid - 1;
        }
        dinv[r] = d != 0.0 ? 1.0 / d : 1.0;
    }
}

// y = A x (row by ascending column)
__global__ void spmv_plain(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ a,
                           int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = rp[r]; k < rp[r + 1]; ++k) s = fma(a[k], x[ci[k]], s);
        y[r] = s;
    }
}

// r = b - A x, rhat = r, p = v = 0
__global__ void init_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ a,
                            int64_t n, const double* __restrict__ b, const double* __restrict__ x,
                            double* __restrict__ r, double* __restrict__ rh, double* __restrict__ p,
                            double* __restrict__ v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) s = fma(a[k], x[ci[k]], s);
        const double ri = b[i] - s;
        r[i] = ri;
        rh[i] = ri;
        p[i] = 0.0;
        v[i] = 0.0;
    }
}

__global__ void scalar_init(double* sc) {
    sc[S_RHO_OLD] = 1.0;
    sc[S_ALPHA] = 1.0;
    sc[S_OMEGA] = 1.0;
}

// beta = (rho / rho_old) (alpha / omega); p = r + beta (p - omega v); y = D^-1 p
__global__ void p_update(int64_t n, double* __restrict__ sc, const double* __restrict__ r, double* __restrict__ p,
                         const double* __restrict__ v, const double* __restrict__ dinv, double* __restrict__ y) {
    const double beta = (sc[S_RHO] / sc[S_RHO_OLD]) * (sc[S_ALPHA] / sc[S_OMEGA]);
    const double om = sc[S_OMEGA];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double pi = r[i] + beta * (p[i] - om * v[i]);
        p[i] = pi;
        y[i] = dinv[i] * pi;
    }
}

// alpha = rho / (rhat . v); s = r - alpha v (into r); x += alpha y; z = D^-1 s
__global__ void s_update(int64_t n, const double* __restrict__ sc, double* __restrict__ r,
                         const double* __restrict__ v, double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ dinv, double* __restrict__ z) {
    const double alpha = sc[S_RHO] / sc[S_RV];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double si = r[i] - alpha * v[i];
        r[i] = si;
        x[i] += alpha * y[i];
        z[i] = dinv[i] * si;
    }
}

__global__ void alpha_store(double* sc) { sc[S_ALPHA] = sc[S_RHO] / sc[S_RV]; }

// omega = (t . s) / (t . t); x += omega z; r = s - omega t
__global__ void x_update(int64_t n, double* __restrict__ sc, double* __restrict__ r, const double* __restrict__ t,
                         double* __restrict__ x, const double* __restrict__ z) {
    const double om = sc[S_TT] != 0.0 ? sc[S_TS] / sc[S_TT] : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += om * z[i];
        r[i] -= om * t[i];
    }
}

__global__ void omega_store(double* sc) {
    sc[S_OMEGA] = sc[S_TT] != 0.0 ? sc[S_TS] / sc[S_TT] : 0.0;
    sc[S_RHO_OLD] = sc[S_RHO];
}

// u -= du
__global__ void sub_kernel(int64_t n, double* __restrict__ u, const double* __restrict__ du) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] -= du[i];
}

int grid_n(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// Solver scratch of a mesh: 8 vectors of n and the reduction partials.
struct Scratch {
    double *r, *rh, *p, *v, *y, *z, *t, *dinv, *sc;
    double2* part;
};

int scratch(fem_mesh& m, Scratch& S, cudaStream_t s) {
    const size_t n = (size_t)m.n, nb = (n + RB - 1) / RB;
    // the partials are double2 (16-byte accesses): they start at an even
    // double offset from the (256-byte aligned) base
    const size_t poff = (8 * n + S_N + 1) & ~size_t(1);
    const size_t bytes = sizeof(double) * poff + sizeof(double2) * (nb + 1);
    int rc = buf_alloc(m.solve, bytes, s);
    if (rc) return rc;
    double* b = m.solve.as<double>();
    S.r = b;
    S.rh = b + n;
    S.p = b + 2 * n;
    S.v = b + 3 * n;
    S.y = b + 4 * n;
    S.z = b + 5 * n;
    S.t = b + 6 * n;
    S.dinv = b + 7 * n;
    S.sc = b + 8 * n;
    S.part = reinterpret_cast<double2*>(b + poff);
    return FEM_OK;
}

// sc[j0] = x0 . y0 (and sc[j1] = x1 . y1)
int dot2(int64_t n, const double* x0, const double* y0, const double* x1, const double* y1, const Scratch& S, int j0,
         int j1, cudaStream_t s) {
    const int64_t nb = (n + RB - 1) / RB;
    dot2_partial<<<(unsigned)nb, RB, 0, s>>>(n, x0, y0, x1, y1, S.part);
    dot2_final<<<1, 1024, 0, s>>>(S.part, nb, S.sc, j0, j1);
    return FEM_OK;
}

}  // namespace

int bicgstab(fem_mesh& m, const double* A, const double* b, double* x, double rtol, int maxit, int* iters,
             double* relres, cudaStream_t s) {
    Scratch S;
    int rc = scratch(m, S, s);
    if (rc) return rc;
    const int64_t n = m.n;
    const int* rp = m.row_ptr.as<int>();
    const int* ci = m.col_idx.as<int>();
    const int g = grid_n(n);
    cudaGetLastError();   // clear any stale error before the launch checks
    jacobi_kernel<<<g, 256, 0, s>>>(rp, ci, A, n, S.dinv);
    init_kernel<<<g, 256, 0, s>>>(rp, ci, A, n, b, x, S.r, S.rh, S.p, S.v);
    scalar_init<<<1, 1, 0, s>>>(S.sc);
    dot2(n, b, b, S.r, S.r, S, S_BB, S_RR, s);
    double h[2] = {0, 0};
    FEM_CUDA_TRY(cudaGetLastError());
    FEM_CUDA_TRY(cudaMemcpyAsync(h, S.sc + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    FEM_CUDA_TRY(cudaMemcpyAsync(h + 1, S.sc + S_BB, sizeof(double), cudaMemcpyDeviceToHost, s));
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(h[1]) > 0 ? std::sqrt(h[1]) : 1.0;
    double res = std::sqrt(h[0]) / bnorm;
    int it = 0;
    while (res > rtol && it < maxit) {
        ++it;
        dot2(n, S.rh, S.r, nullptr, nullptr, S, S_RHO, -1, s);                    // rho = rhat . r
        p_update<<<g, 256, 0, s>>>(n, S.sc, S.r, S.p, S.v, S.dinv, S.y);
        spmv_plain<<<g, 256, 0, s>>>(rp, ci, A, n, S.y, S.v);                    // v = A y
        dot2(n, S.rh, S.v, nullptr, nullptr, S, S_RV, -1, s);                     // rhat . v
        s_update<<<g, 256, 0, s>>>(n, S.sc, S.r, S.v, x, S.y, S.dinv, S.z);       // s in r, x += alpha y
        alpha_store<<<1, 1, 0, s>>>(S.sc);
        spmv_plain<<<g, 256, 0, s>>>(rp, ci, A, n, S.z, S.t);                    // t = A z
        dot2(n, S.t, S.r, S.t, S.t, S, S_TS, S_TT, s);                            // t . s, t . t
        x_update<<<g, 256, 0, s>>>(n, S.sc, S.r, S.t, x, S.z);                    // x += omega z, r = s - omega t
        omega_store<<<1, 1, 0, s>>>(S.sc);
        dot2(n, S.r, S.r, nullptr, nullptr, S, S_RR, -1, s);
        FEM_CUDA_TRY(cudaGetLastError());
        FEM_CUDA_TRY(cudaMemcpyAsync(h, S.sc + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
        FEM_CUDA_TRY(cudaStreamSynchronize(s));
        res = std::sqrt(h[0]) / bnorm;
        if (!std::isfinite(res)) break;
    }
    if (iters) *iters = it;
    if (relres) *relres = res;
    if (!std::isfinite(res)) return fail(FEM_ECUDA, "BiCGStab broke down (non-finite residual)");
    return FEM_OK;
}

int heat_step(fem_mesh& m, const fem_coeff* k, const CoeffDev& g, const unsigned char* mask, double dt,
              const double* us, double* u, double newton_rtol, int max_newton, double krylov_rtol, int max_krylov,
              fem_heat_report* rep, cudaStream_t s) {
    const size_t nnz = (size_t)m.nnz, n = (size_t)m.n;
    int rc = buf_alloc(m.newton, sizeof(double) * (5 * nnz + 2 * n + 2), s);
    if (rc) return rc;
    double* vM = m.newton.as<double>();
    double* vK = vM + nnz;
    double* vT = vK + nnz;
    double* vB = vT + nnz;
    double* vJ = vB + nnz;
    double* b = vJ + nnz;
    double* F = b + n;
    double* norms = F + n;
    fem_heat_report R = {};
    double r0 = -1.0;
    for (int it = 0; it <= max_newton; ++it) {
        if ((rc = fem_assemble_all(&m, k, u, FEM_FP64, vM, vK, vT, s))) return rc;
        if ((rc = boundary_assemble(m, g, u, mask, vB, b, s))) return rc;
        if ((rc = csr_residual(m, vM, vK, b, u, us, dt, F, norms, s))) return rc;
        double h[2];
        FEM_CUDA_TRY(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, s));
        FEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (r0 < 0) r0 = h[0];
        R.residual = h[0];
        if (!std::isfinite(h[0])) return fail(FEM_ECUDA, "Newton: non-finite residual");
        if (h[0] <= newton_rtol * (r0 > 0 ? r0 : 1.0) || it == max_newton) {
            R.converged = h[0] <= newton_rtol * (r0 > 0 ? r0 : 1.0);
            break;
        }
        if ((rc = csr_jacobian(m, dt, vM, nullptr, vK, vT, vB, vJ, s))) return rc;
        // J du = F, then u -= du (the Krylov solve starts from du = 0)
        double* du = vM;   // M is rebuilt at the next iteration; its space holds du
        FEM_CUDA_TRY(cudaMemsetAsync(du, 0, sizeof(double) * n, s));
        int kit = 0;
        double kres = 0.0;
        if ((rc = bicgstab(m, vJ, F, du, krylov_rtol, max_krylov, &kit, &kres, s))) return rc;
        R.krylov_iters += kit;
        R.max_krylov_relres = std::max(R.max_krylov_relres, kres);
        sub_kernel<<<grid_n(m.n), 256, 0, s>>>(m.n, u, du);
        FEM_CUDA_TRY(cudaGetLastError());
        ++R.newton_iters;
    }
    R.residual0 = r0;
    if (rep) *rep = R;
    return FEM_OK;
}

}  // namespace fem
