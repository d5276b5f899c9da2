// scatter.cu -- global assembly of the element matrices into CSR values.
//
// Algorithm 2 line 12 ("form the matrices M and C from V_m and V_c and the
// set of indices of nonzero entries"); Section 3 step 2, eq. assemblage_1:
// M_ij = sum over elements of the element integrals.  Deterministic, no
// atomics: every CSR slot adds its contributions in ascending element order,
// the order of Algorithm 1, so the result is bit-reproducible run to run.
// M and K come from the symmetric element storage (entry (i,j) and (j,i)
// share V[e][sym(min,max)]), T from the full n_p x n_p storage.
//
// One thread per CSR slot sums the slot's contributor list
// contrib[seg_ptr[s] .. seg_ptr[s+1]) (element entries, ascending).
#include <algorithm>
#include <vector>

#include "fem_internal.h"

namespace fem {

namespace {

__host__ __device__ constexpr int sym_idx(int np, int i, int j) {
    return i <= j ? i * np - (i * (i - 1)) / 2 + (j - i) : j * np - (j * (j - 1)) / 2 + (i - j);
}

// V entries of one element entry c = (e n_p + i) n_p + j: T from the full
// storage (its index is c itself), M and K from the symmetric storage at
// e n_p(n_p+1)/2 + sym[i n_p + j], with the local symmetric index from a
// small shared-memory table.
template <int NP, typename T>
struct Contribution {
    T m, k, t;
    // 32-bit unsigned index arithmetic (element entries, slots and V
    // offsets of a mesh are below 2^31)
    __device__ __forceinline__ void load(uint32_t c, const short* __restrict__ sym, const T* __restrict__ VM,
                                         const T* __restrict__ VK, const T* __restrict__ VT) {
        constexpr uint32_t NT = NP * NP, NSYM = NP * (NP + 1) / 2;
        t = VT ? __ldg(VT + c) : T(0);
        if (VM || VK) {
            const uint32_t e = c / NT;
            const uint32_t off = e * NSYM + (uint32_t)sym[c - e * NT];
            m = VM ? __ldg(VM + off) : T(0);
            k = VK ? __ldg(VK + off) : T(0);
        } else {
            m = k = T(0);
        }
    }
};

// the table sym[i n_p + j] of one element type, filled by the whole block
template <int NP>
__device__ __forceinline__ void fill_sym_table(short* sym) {
    for (int l = threadIdx.x; l < NP * NP; l += blockDim.x) sym[l] = (short)sym_idx(NP, l / NP, l % NP);
}

// Segment sum with the loads of consecutive grid-stride iterations
// overlapped: while slot s adds its V entries, the contributor indices of
// slot s+G and the segment bounds of slot s+2G are already in flight, so a
// slot costs about one memory round trip instead of three dependent ones.
// (A third stage, V of slot s+G, measured slower on GB300.)  The summation
// order per slot (ascending contributor) is unchanged.
template <int NP, typename T>
__global__ void __launch_bounds__(256) scatter_segments_kernel(const int* __restrict__ seg_ptr,
                                                               const int* __restrict__ contrib, int64_t nnz64,
                                                               const T* __restrict__ VM, const T* __restrict__ VK,
                                                               const T* __restrict__ VT, T* __restrict__ vM,
                                                               T* __restrict__ vK, T* __restrict__ vT) {
    __shared__ short sym[NP * NP];
    fill_sym_table<NP>(sym);
    __syncthreads();
    const T* vm_src = vM ? VM : nullptr;
    const T* vk_src = vK ? VK : nullptr;
    const T* vt_src = vT ? VT : nullptr;
    constexpr uint32_t NONE = 0xffffffffu;
    const uint32_t nnz = (uint32_t)nnz64;   // < 2^31 (int32 CSR)
    const uint32_t G = gridDim.x * blockDim.x;
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    const uint32_t* sp = reinterpret_cast<const uint32_t*>(seg_ptr);
    const uint32_t* cp = reinterpret_cast<const uint32_t*>(contrib);
    // pipeline registers: bounds of s and s+G, first two contributors of s
    uint32_t a0 = __ldg(sp + s), b0 = __ldg(sp + s + 1);
    uint32_t a1 = 0, b1 = 0;
    if (s + G < nnz) {
        a1 = __ldg(sp + s + G);
        b1 = __ldg(sp + s + G + 1);
    }
    uint32_t c0 = a0 < b0 ? __ldg(cp + a0) : NONE;
    uint32_t c1 = a0 + 1 < b0 ? __ldg(cp + a0 + 1) : NONE;
    while (true) {
        const uint32_t s1 = s + G, s2 = s + 2 * G;
        // in flight together: V of slot s, contributors of s+G, bounds of s+2G
        Contribution<NP, T> x0, x1;
        if (c0 != NONE) x0.load(c0, sym, vm_src, vk_src, vt_src);
        if (c1 != NONE) x1.load(c1, sym, vm_src, vk_src, vt_src);
        uint32_t n0 = NONE, n1 = NONE;
        if (s1 < nnz) {
            n0 = a1 < b1 ? __ldg(cp + a1) : NONE;
            n1 = a1 + 1 < b1 ? __ldg(cp + a1 + 1) : NONE;
        }
        uint32_t a2 = 0, b2 = 0;
        if (s2 < nnz) {
            a2 = __ldg(sp + s2);
            b2 = __ldg(sp + s2 + 1);
        }
        T am = T(0), ak = T(0), at = T(0);
        if (c0 != NONE) {
            am += x0.m;
            ak += x0.k;
            at += x0.t;
        }
        if (c1 != NONE) {
            am += x1.m;
            ak += x1.k;
            at += x1.t;
        }
        for (uint32_t p = a0 + 2; p < b0; ++p) {
            Contribution<NP, T> x;
            x.load(__ldg(cp + p), sym, vm_src, vk_src, vt_src);
            am += x.m;
            ak += x.k;
            at += x.t;
        }
        if (vM) vM[s] = am;
        if (vK) vK[s] = ak;
        if (vT) vT[s] = at;
        if (s1 >= nnz || s1 < s) break;
        s = s1;
        a0 = a1;
        b0 = b1;
        a1 = a2;
        b1 = b2;
        c0 = n0;
        c1 = n1;
    }
}

// One slot of the segment sum, contributions in ascending order (the same
// order as the single-mesh kernel, so batched sums carry the same bits).
template <int NP, typename T>
__device__ __forceinline__ void segment_slot(int64_t s, const int* __restrict__ seg_ptr,
                                             const int* __restrict__ contrib, const short* __restrict__ sym,
                                             const T* __restrict__ VM, const T* __restrict__ VK,
                                             const T* __restrict__ VT, T* __restrict__ vM, T* __restrict__ vK,
                                             T* __restrict__ vT) {
    const int a = __ldg(seg_ptr + s), b = __ldg(seg_ptr + s + 1);
    T am = T(0), ak = T(0), at = T(0);
    for (int p = a; p < b; ++p) {
        Contribution<NP, T> x;
        x.load((uint32_t)__ldg(contrib + p), sym, VM, VK, VT);
        am += x.m;
        ak += x.k;
        at += x.t;
    }
    if (vM) vM[s] = am;
    if (vK) vK[s] = ak;
    if (vT) vT[s] = at;
}

// offsets of the per-type symmetric-index tables in the batched kernel
__host__ __device__ constexpr int sym_tab_off(int np) {
    return np == 3 ? 0 : np == 4 ? 9 : np == 6 ? 25 : np == 10 ? 61 : 161;
}
constexpr int SYM_TAB_TOTAL = 561;

// Batched: the work list holds chunks of `count` slots of many meshes.
template <typename T>
__global__ void __launch_bounds__(512) batch_scatter_kernel(const BatchItem* __restrict__ items, int nitems,
                                                            const BatchMesh* __restrict__ meshes) {
    __shared__ short sym[SYM_TAB_TOTAL];
    fill_sym_table<3>(sym + sym_tab_off(3));
    fill_sym_table<4>(sym + sym_tab_off(4));
    fill_sym_table<6>(sym + sym_tab_off(6));
    fill_sym_table<10>(sym + sym_tab_off(10));
    fill_sym_table<20>(sym + sym_tab_off(20));
    __syncthreads();
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchMesh& bm = meshes[w.mesh];
        const T* VM = bm.vM ? static_cast<const T*>(bm.VM) : nullptr;
        const T* VK = bm.vK ? static_cast<const T*>(bm.VK) : nullptr;
        const T* VT = bm.vT ? static_cast<const T*>(bm.VT) : nullptr;
        T* vM = static_cast<T*>(bm.vM);
        T* vK = static_cast<T*>(bm.vK);
        T* vT = static_cast<T*>(bm.vT);
        const short* st = sym + sym_tab_off(bm.np);
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const int64_t s = w.first + k;
            if (s >= bm.nnz) break;
            switch (bm.np) {
                case 3: segment_slot<3, T>(s, bm.seg_ptr, bm.contrib, st, VM, VK, VT, vM, vK, vT); break;
                case 4: segment_slot<4, T>(s, bm.seg_ptr, bm.contrib, st, VM, VK, VT, vM, vK, vT); break;
                case 6: segment_slot<6, T>(s, bm.seg_ptr, bm.contrib, st, VM, VK, VT, vM, vK, vT); break;
                case 10: segment_slot<10, T>(s, bm.seg_ptr, bm.contrib, st, VM, VK, VT, vM, vK, vT); break;
                case 20: segment_slot<20, T>(s, bm.seg_ptr, bm.contrib, st, VM, VK, VT, vM, vK, vT); break;
                default: break;
            }
        }
    }
}

template <int NP, typename T>
int launch_np(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s,
              int nsm, int64_t s0, int64_t s1) {
    {
        // a slot range [s0, s1): the segment bounds and the outputs offset
        // by s0 (contributor indices address the whole V)
        const int B = m.sum_block >= 32 ? m.sum_block : 256;
        const int64_t ns = s1 - s0;
        if (ns <= 0) return FEM_OK;
        int64_t blocks = (ns + B - 1) / B;
        if (blocks > (int64_t)nsm * (4096 / B)) blocks = (int64_t)nsm * (4096 / B);
        cudaGetLastError();   // clear any stale error before the launch check
        scatter_segments_kernel<NP, T><<<(unsigned)blocks, B, 0, s>>>(
            m.seg_ptr.as<int>() + s0, m.contrib.as<int>(), ns, VM, VK, VT, vM ? vM + s0 : nullptr,
            vK ? vK + s0 : nullptr, vT ? vT + s0 : nullptr);
    }
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

template <typename T>
int run(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s, int64_t s0,
        int64_t s1) {
    if (s1 < 0) s1 = m.nnz;
    if (s0 < 0 || s0 > s1 || s1 > m.nnz) return fail(FEM_EINVAL, "slot range out of bounds");
    if (m.nnz <= 0 || s1 == s0) return FEM_OK;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    switch (m.np) {
        case 3: return launch_np<3, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
        case 4: return launch_np<4, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
        case 6: return launch_np<6, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
        case 10: return launch_np<10, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
        case 20: return launch_np<20, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
    }
    return fail(FEM_EINVAL, "unsupported n_p");
}

}  // namespace

template <typename T>
int batch_scatter_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, int block, cudaStream_t s) {
    if (nitems <= 0) return FEM_OK;
    if (block < 32 || block > 512) block = 256;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int grid = nsm * (2048 / block);
    if (grid > nitems) grid = nitems;
    cudaGetLastError();   // clear any stale error before the launch check
    batch_scatter_kernel<T><<<grid, block, 0, s>>>(items, nitems, meshes);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}
template int batch_scatter_launch<float>(const BatchItem*, int, const BatchMesh*, int, cudaStream_t);
template int batch_scatter_launch<double>(const BatchItem*, int, const BatchMesh*, int, cudaStream_t);

int scatter_fp64(const fem_mesh& m, const double* VM, const double* VK, const double* VT, double* vM, double* vK,
                 double* vT, cudaStream_t s, int64_t s0, int64_t s1) {
    return run<double>(m, VM, VK, VT, vM, vK, vT, s, s0, s1);
}

int scatter_fp32(const fem_mesh& m, const float* VM, const float* VK, const float* VT, float* vM, float* vK,
                 float* vT, cudaStream_t s, int64_t s0, int64_t s1) {
    return run<float>(m, VM, VK, VT, vM, vK, vT, s, s0, s1);
}


namespace {

// For every slot, the fine element chunk of its last (largest) contributor;
// per chunk, the smallest slot that needs it (block minimum in shared
// memory, then one atomic per block and chunk).
__global__ void slot_ready_kernel(const int* __restrict__ seg_ptr, const int* __restrict__ contrib, int64_t nnz,
                                  int nt, int64_t ec, int nfine, int* __restrict__ first_slot) {
    __shared__ int smin[PLAN_MAX_FINE];
    for (int i = threadIdx.x; i < nfine; i += blockDim.x) smin[i] = 0x7fffffff;
    __syncthreads();
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        const int b = seg_ptr[s + 1];
        if (b <= seg_ptr[s]) continue;
        const int64_t e = contrib[b - 1] / nt;
        const int j = (int)(e / ec);
        atomicMin(&smin[j < nfine ? j : nfine - 1], (int)s);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nfine; i += blockDim.x)
        if (smin[i] != 0x7fffffff) atomicMin(&first_slot[i], smin[i]);
}

}  // namespace

int chunk_plan_fine(fem_mesh& m, cudaStream_t s) {
    if (m.have_plan) return FEM_OK;
    const int64_t E = m.E;
    const int nt = m.np * m.np;
    int64_t ec = ((E + PLAN_MAX_FINE - 1) / PLAN_MAX_FINE + 127) / 128 * 128;
    if (ec < 128) ec = 128;
    const int nfine = E > 0 ? (int)((E + ec - 1) / ec) : 0;
    m.plan_e.assign(nfine + 1, 0);
    m.plan_s.assign(nfine + 1, 0);
    for (int j = 0; j <= nfine; ++j) m.plan_e[j] = std::min<int64_t>((int64_t)j * ec, E);
    if (nfine > 0) m.plan_s[nfine] = m.nnz;
    if (nfine > 1 && m.nnz > 0) {
        DevBuf fs;
        int rc = buf_alloc(fs, sizeof(int) * nfine, s);
        if (rc) return rc;
        std::vector<int> host(nfine, 0x7fffffff);
        FEM_CUDA_TRY(cudaMemcpyAsync(fs.ptr, host.data(), sizeof(int) * nfine, cudaMemcpyHostToDevice, s));
        int64_t blocks = (m.nnz + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        cudaGetLastError();   // clear any stale error before the launch check
        slot_ready_kernel<<<(unsigned)blocks, 256, 0, s>>>(m.seg_ptr.as<int>(), m.contrib.as<int>(), m.nnz, nt, ec,
                                                          nfine, fs.as<int>());
        FEM_CUDA_TRY(cudaGetLastError());
        FEM_CUDA_TRY(cudaMemcpyAsync(host.data(), fs.ptr, sizeof(int) * nfine, cudaMemcpyDeviceToHost, s));
        FEM_CUDA_TRY(cudaStreamSynchronize(s));
        buf_free(fs, s);
        // slots ready once chunks 0..j-1 are formed: those below the first
        // slot needing any chunk >= j (suffix minimum)
        int64_t run = m.nnz;
        for (int j = nfine - 1; j >= 0; --j) {
            run = std::min<int64_t>(run, host[j]);
            m.plan_s[j] = run;
        }
        m.plan_s[0] = 0;
    }
    m.have_plan = true;
    return FEM_OK;
}

}  // namespace fem
