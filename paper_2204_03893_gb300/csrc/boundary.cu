// boundary.cu -- the boundary terms of the heat problem and the Newton
// quantities built from the assembled matrices, FP64.
//
// Section 5: the load vector holds b_i = int_{dOmega_N} g_N(u_h) phi_i dS and
// its derivative is the boundary matrix B_ik = int g_N'(u_h) phi_i phi_k dS;
// the implicit Euler residual is F(u) = M (u - u^s) + dt K(u) u - dt f(u) and
// its Jacobian Mt + M + dt (K + T) - dt B.  Section 6, Experiment 2: g_N is
// convection plus radiation, h_c (T_a - u) + h_r (T_a^4 - u^4), on the whole
// boundary -- a polynomial in u, given here as a conductivity-style law.
//
// Boundary facets (faces of exactly one element) are found once per mesh
// from the symbolic phase's node -> element incidences and listed in
// ascending (element, face) order.  B is formed per facet as the paper's
// mass-type product V = X Q on the facet (X[q] = w_q |J_f| g'(u_q), Q the
// products of the face nodes' basis values at the facet points), then summed
// into the volume pattern -- every facet pair (i, k) is also an element pair,
// so its CSR slot is the element entry's slot -- by one thread per boundary
// row, which adds its facets in ascending order: deterministic, no atomics.
#include "fem_internal.h"
#include "refelem.h"

namespace fem {

namespace {

constexpr int BMAX_NF = 10;      // face nodes of a P3 tetrahedron face
constexpr int BMAX_NQ = 12;      // points of the degree-6 triangle rule
constexpr int BSLOT = 16;        // incidence entry = facet * BSLOT + face-local node

struct FacetDev {
    int nf, nq, phi_off, pad;
    int fnode[4][BMAX_NF];
    double w[BMAX_NQ];
};
__constant__ FacetDev c_fac[6];
__constant__ double c_fphi[4 * BMAX_NQ * BMAX_NF * 6];

int facet_tables_init() {
    static bool done[64] = {};
    int dev = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 64 && done[dev]) return FEM_OK;
    FacetDev h[6] = {};
    std::vector<double> phi;
    for (int t = 0; t < 6; ++t) {
        const FacetTab* F = facets_for_type(t);
        if (!F || F->nf > BMAX_NF || F->nq > BMAX_NQ) return fail(FEM_EINVAL, "facet tables failed");
        h[t].nf = F->nf;
        h[t].nq = F->nq;
        h[t].phi_off = (int)phi.size();
        for (int f = 0; f < F->nfaces; ++f)
            for (int a = 0; a < F->nf; ++a) h[t].fnode[f][a] = F->fnode[f * F->nf + a];
        for (int q = 0; q < F->nq; ++q) h[t].w[q] = F->w[q];
        phi.insert(phi.end(), F->phi.begin(), F->phi.end());
    }
    if (phi.size() > sizeof(c_fphi) / sizeof(double)) return fail(FEM_EINVAL, "facet tables too large");
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_fac, h, sizeof(h)));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_fphi, phi.data(), sizeof(double) * phi.size()));
    if (dev < 64) done[dev] = true;
    return FEM_OK;
}

int grid1(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

// flag[e (d+1) + f] = 1 if face f of element e (the face opposite local
// vertex f) belongs to no other element: another element holding all its
// vertices must be incident to its first vertex.
__global__ void facet_flag_kernel(const int* __restrict__ conn, int np, int d, int64_t E,
                                  const int* __restrict__ inc_ptr, const int* __restrict__ inc, int* __restrict__ flag) {
    const int nv = d + 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < E * nv; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k / nv;
        const int f = (int)(k - e * nv);
        int fv[3], n = 0;
        for (int a = 0; a < nv; ++a)
            if (a != f) fv[n++] = conn[e * np + a];
        bool shared = false;
        for (int t = inc_ptr[fv[0]]; t < inc_ptr[fv[0] + 1] && !shared; ++t) {
            const int64_t e2 = inc[t] / np;
            if (e2 == e) continue;
            bool all = true;
            for (int i = 0; i < d && all; ++i) {
                bool found = false;
                for (int a = 0; a < nv; ++a) found |= conn[e2 * np + a] == fv[i];
                all = found;
            }
            shared = all;
        }
        flag[k] = shared ? 0 : 1;
    }
}

__global__ void facet_compact_kernel(const int* __restrict__ flag, const int* __restrict__ pos, int64_t m, int nv,
                                     int2* __restrict__ facets) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        if (flag[k]) facets[pos[k]] = make_int2((int)(k / nv), (int)(k % nv));
}

// node -> facet incidences (entries facet * BSLOT + face-local node)
__global__ void bnode_count_kernel(const int2* __restrict__ facets, int64_t nfb, const int* __restrict__ conn, int np,
                                   int type, int* __restrict__ cnt) {
    const int nf = c_fac[type].nf;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nfb; k += (int64_t)gridDim.x * blockDim.x) {
        const int2 fc = facets[k];
        for (int a = 0; a < nf; ++a) atomicAdd(&cnt[conn[(int64_t)fc.x * np + c_fac[type].fnode[fc.y][a]]], 1);
    }
}

__global__ void bnode_fill_kernel(const int2* __restrict__ facets, int64_t nfb, const int* __restrict__ conn, int np,
                                  int type, const int* __restrict__ ptr, int* __restrict__ fill, int* __restrict__ binc) {
    const int nf = c_fac[type].nf;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nfb; k += (int64_t)gridDim.x * blockDim.x) {
        const int2 fc = facets[k];
        for (int a = 0; a < nf; ++a) {
            const int r = conn[(int64_t)fc.x * np + c_fac[type].fnode[fc.y][a]];
            binc[ptr[r] + atomicAdd(&fill[r], 1)] = (int)k * BSLOT + a;
        }
    }
}

// each node's list ascending (the order its facets are added in)
__global__ void bnode_sort_kernel(const int* __restrict__ ptr, int64_t n, int* __restrict__ binc) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int a = ptr[r], b = ptr[r + 1];
        for (int i = a + 1; i < b; ++i) {
            const int v = binc[i];
            int j = i - 1;
            while (j >= a && binc[j] > v) {
                binc[j + 1] = binc[j];
                --j;
            }
            binc[j + 1] = v;
        }
    }
}

// Facet products: VB[f] = the n_f(n_f+1)/2 distinct entries of
// sum_q X[q] phi_q phi_q^T with X[q] = w_q |J_f| g'(u_q), then the n_f
// entries of the load, sum_q w_q |J_f| g(u_q) phi_q.  A facet outside the
// mask gets zeros.
template <int D>
__global__ void facet_form_kernel(const int2* __restrict__ facets, int64_t nfb, const int* __restrict__ conn, int np,
                                  int type, const double* __restrict__ X, const double* __restrict__ u, CoeffDev g,
                                  const unsigned char* __restrict__ mask, double* __restrict__ VB) {
    const FacetDev& T = c_fac[type];
    const int nf = T.nf, nq = T.nq, nsym = nf * (nf + 1) / 2, ld = nsym + nf;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nfb; k += (int64_t)gridDim.x * blockDim.x) {
        double* out = VB + k * ld;
        if (mask && !mask[k]) {
            for (int i = 0; i < ld; ++i) out[i] = 0.0;
            continue;
        }
        const int2 fc = facets[k];
        const int* ce = conn + (int64_t)fc.x * np;
        int wv[3], m = 0;
        for (int a = 0; a <= D; ++a)
            if (a != fc.y) wv[m++] = a;
        double e1[3], J;
        for (int a = 0; a < D; ++a) e1[a] = X[(int64_t)ce[wv[1]] * D + a] - X[(int64_t)ce[wv[0]] * D + a];
        if constexpr (D == 2) {
            J = sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
        } else {
            double e2[3];
            for (int a = 0; a < 3; ++a) e2[a] = X[(int64_t)ce[wv[2]] * 3 + a] - X[(int64_t)ce[wv[0]] * 3 + a];
            const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                         cz = e1[0] * e2[1] - e1[1] * e2[0];
            J = sqrt(cx * cx + cy * cy + cz * cz);
        }
        double uf[BMAX_NF];
        for (int a = 0; a < nf; ++a) uf[a] = u[ce[T.fnode[fc.y][a]]];
        const double* ph = c_fphi + T.phi_off + fc.y * nq * nf;
        double xb[BMAX_NQ], xg[BMAX_NQ];
        for (int q = 0; q < nq; ++q) {
            double uq = 0.0;
            for (int a = 0; a < nf; ++a) uq += ph[q * nf + a] * uf[a];
            double dg;
            const double gq = k_eval<double>(g, uq, dg);
            const double wj = T.w[q] * J;
            xb[q] = wj * dg;
            xg[q] = wj * gq;
        }
        int s = 0;
        for (int a = 0; a < nf; ++a)
            for (int b = a; b < nf; ++b, ++s) {
                double v = 0.0;
                for (int q = 0; q < nq; ++q) v += xb[q] * (ph[q * nf + a] * ph[q * nf + b]);
                out[s] = v;
            }
        for (int a = 0; a < nf; ++a) {
            double v = 0.0;
            for (int q = 0; q < nq; ++q) v += xg[q] * ph[q * nf + a];
            out[nsym + a] = v;
        }
    }
}

// One thread per boundary row r: its facets in ascending order, each adding
// its row of B into the row's slots (the element entries' slots) and its
// load entry into b[r].  vB must be zero on entry; b is written on every
// row (0 off the boundary).
__global__ void facet_rows_kernel(const int* __restrict__ ptr, const int* __restrict__ binc, int64_t n,
                                  const int2* __restrict__ facets, const int* __restrict__ slot, int np, int type,
                                  const double* __restrict__ VB, double* __restrict__ vB, double* __restrict__ b) {
    const FacetDev& T = c_fac[type];
    const int nf = T.nf, nsym = nf * (nf + 1) / 2, ld = nsym + nf;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double br = 0.0;
        for (int t = ptr[r]; t < ptr[r + 1]; ++t) {
            const int f = binc[t] / BSLOT, a = binc[t] % BSLOT;
            const int2 fc = facets[f];
            const double* v = VB + (int64_t)f * ld;
            br += v[nsym + a];
            if (vB) {
                const int64_t base = ((int64_t)fc.x * np + T.fnode[fc.y][a]) * np;
                for (int c = 0; c < nf; ++c) {
                    const int lo = a < c ? a : c, hi = a < c ? c : a;
                    const int s = lo * nf - (lo * (lo - 1)) / 2 + (hi - lo);
                    const int sl = slot[base + T.fnode[fc.y][c]];
                    vB[sl] += v[s];
                }
            }
        }
        if (b) b[r] = br;
    }
}

}  // namespace

int boundary_setup(fem_mesh& m, cudaStream_t s) {
    if (m.have_boundary) return FEM_OK;
    int rc = facet_tables_init();
    if (rc) return rc;
    if ((rc = slot_map_build(m, s))) return rc;   // the facet rows are scattered through it
    const int nv = m.d + 1;
    const int64_t mf = m.E * nv;
    DevBuf flag, pos, cnt, fill;
    if ((rc = buf_alloc(flag, sizeof(int) * (size_t)(mf + 1), s))) return rc;
    if ((rc = buf_alloc(pos, sizeof(int) * (size_t)(mf + 1), s))) return rc;
    cudaGetLastError();   // clear any stale error before the launch checks
    facet_flag_kernel<<<grid1(mf, 256), 256, 0, s>>>(m.conn.as<int>(), m.np, m.d, m.E, m.inc_ptr.as<int>(),
                                                     m.inc.as<int>(), flag.as<int>());
    FEM_CUDA_TRY(cudaGetLastError());
    if ((rc = scan_exclusive(flag.as<int>(), mf, pos.as<int>(), s))) return rc;
    int nfb = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&nfb, pos.as<int>() + mf, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    const int nf = facets_for_type(m.type)->nf;
    if ((rc = buf_alloc(m.bfacet, sizeof(int2) * (size_t)(nfb + 1), s))) return rc;
    if ((rc = buf_alloc(m.bnode_ptr, sizeof(int) * (size_t)(m.n + 1), s))) return rc;
    if ((rc = buf_alloc(m.bnode_inc, sizeof(int) * (size_t)nfb * nf + sizeof(int), s))) return rc;
    if ((rc = buf_alloc(cnt, sizeof(int) * (size_t)(m.n + 1), s))) return rc;
    if ((rc = buf_alloc(fill, sizeof(int) * (size_t)(m.n + 1), s))) return rc;
    facet_compact_kernel<<<grid1(mf, 256), 256, 0, s>>>(flag.as<int>(), pos.as<int>(), mf, nv, m.bfacet.as<int2>());
    FEM_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, cnt.bytes, s));
    FEM_CUDA_TRY(cudaMemsetAsync(fill.ptr, 0, fill.bytes, s));
    bnode_count_kernel<<<grid1(nfb, 256), 256, 0, s>>>(m.bfacet.as<int2>(), nfb, m.conn.as<int>(), m.np, m.type,
                                                       cnt.as<int>());
    FEM_CUDA_TRY(cudaGetLastError());
    if ((rc = scan_exclusive(cnt.as<int>(), m.n, m.bnode_ptr.as<int>(), s))) return rc;
    bnode_fill_kernel<<<grid1(nfb, 256), 256, 0, s>>>(m.bfacet.as<int2>(), nfb, m.conn.as<int>(), m.np, m.type,
                                                      m.bnode_ptr.as<int>(), fill.as<int>(), m.bnode_inc.as<int>());
    bnode_sort_kernel<<<grid1(m.n, 128), 128, 0, s>>>(m.bnode_ptr.as<int>(), m.n, m.bnode_inc.as<int>());
    FEM_CUDA_TRY(cudaGetLastError());
    buf_free(flag, s);
    buf_free(pos, s);
    buf_free(cnt, s);
    buf_free(fill, s);
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    m.n_bfacets = nfb;
    m.have_boundary = true;
    return FEM_OK;
}

int boundary_assemble(fem_mesh& m, const CoeffDev& g, const double* u, const unsigned char* mask, double* vB,
                      double* b, cudaStream_t s) {
    int rc = facet_tables_init();
    if (rc) return rc;
    const int nf = facets_for_type(m.type)->nf;
    const int ld = nf * (nf + 1) / 2 + nf;
    const int64_t nfb = m.n_bfacets;
    if ((rc = buf_alloc(m.bscratch, sizeof(double) * (size_t)(nfb * ld + 1), s))) return rc;
    if (vB) FEM_CUDA_TRY(cudaMemsetAsync(vB, 0, sizeof(double) * (size_t)m.nnz, s));
    cudaGetLastError();   // clear any stale error before the launch checks
    if (nfb > 0) {
        if (m.d == 2)
            facet_form_kernel<2><<<grid1(nfb, 128), 128, 0, s>>>(m.bfacet.as<int2>(), nfb, m.conn.as<int>(), m.np,
                                                                 m.type, m.coords.as<double>(), u, g, mask,
                                                                 m.bscratch.as<double>());
        else
            facet_form_kernel<3><<<grid1(nfb, 128), 128, 0, s>>>(m.bfacet.as<int2>(), nfb, m.conn.as<int>(), m.np,
                                                                 m.type, m.coords.as<double>(), u, g, mask,
                                                                 m.bscratch.as<double>());
        FEM_CUDA_TRY(cudaGetLastError());
    }
    facet_rows_kernel<<<grid1(m.n, 128), 128, 0, s>>>(m.bnode_ptr.as<int>(), m.bnode_inc.as<int>(), m.n,
                                                      m.bfacet.as<int2>(), m.slot.as<int>(), m.np, m.type,
                                                      m.bscratch.as<double>(), vB, b);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // namespace fem
