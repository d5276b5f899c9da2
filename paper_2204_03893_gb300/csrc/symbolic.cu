// symbolic.cu -- CSR pattern and element-entry -> slot map, once per mesh.
//
// Section 3 step 2: the integral of an element contributes to (i, j) only if
// both nodes belong to the element (the index set N_e), which makes the
// matrix sparse; Algorithm 2 ends by summing V into the global matrix over
// the index set of its nonzero entries.  This module builds that set on the
// device by sorting the keys (row, col) = (conn[e][i], conn[e][j]) of every
// element entry c = (e n_p + i) n_p + j:
//   1. counting sort of the (e, i) incidences by row (integer atomics for
//      the counts, then each row's list sorted ascending, by ranks, so that
//      the order does not depend on atomic timing);
//   2. per row, a stable counting sort of its n_p * |incidences| entries by
//      column (ties keep ascending c), one warp per row: the row's distinct
//      columns by repeated warp minima, a count per column, then the entries
//      placed in order (very long rows fall back to a rank sort);
//   3. a scan of the per-row unique-column counts gives row_ptr;
//   4. per row, one warp walks the sorted entries and numbers the column
//      groups: col_idx and seg_ptr (first sorted position of each slot); the
//      slot map slot[c] is derived from the sorted list when first needed;
//   5. the same walk marks, for every group of 32 consecutive sorted
//      positions, which of them start a slot (a bit mask) and the slot of its
//      first position: what the CSR sum reads instead of seg_ptr.
// contrib[] holds the element entries sorted by (slot, c); seg_ptr[s] ..
// seg_ptr[s+1] is slot s's segment.  Everything is integer work and fully
// deterministic.
#include "fem_internal.h"

#include <climits>

namespace fem {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// block-wide exclusive scan of one int per thread; returns the block total
__device__ int block_exclusive_scan(int v, int& total) {
    __shared__ int warp_sums[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    int wprefix = w > 0 ? warp_sums[w - 1] : 0;
    total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return wprefix + x - v;
}

// pass 1: per-tile sums
__global__ void scan_tile_sums(const int* __restrict__ in, int64_t n, int* __restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + threadIdx.x * SCAN_ITEMS + k;
        if (i < n) s += in[i];
    }
    int total;
    block_exclusive_scan(s, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// pass 2: exclusive scan of the tile sums in one block (sequential chunks)
__global__ void scan_sums(int* __restrict__ sums, int nt) {
    int carry = 0;
    for (int base = 0; base < nt; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < nt ? sums[i] : 0;
        int total;
        int ex = block_exclusive_scan(v, total);
        if (i < nt) sums[i] = carry + ex;
        carry += total;
    }
}

// pass 3: out[i] = sum_{j<i} in[j] for i in [0, n]; out[n] is the total
__global__ void scan_apply(const int* __restrict__ in, int64_t n, const int* __restrict__ sums, int* __restrict__ out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + threadIdx.x * SCAN_ITEMS + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int total;
    int ex = block_exclusive_scan(s, total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + threadIdx.x * SCAN_ITEMS + k;
        if (i <= n) out[i] = ex;    // i == n receives the grand total
        ex += v[k];
    }
}

// ---------------------------------------------------------------- incidences
__global__ void inc_count(const int* __restrict__ conn, int64_t m, int* __restrict__ cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[conn[k]], 1);
}

__global__ void inc_fill(const int* __restrict__ conn, int64_t m, const int* __restrict__ inc_ptr,
                         int* __restrict__ fill, int* __restrict__ inc) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        int r = conn[k];
        int pos = inc_ptr[r] + atomicAdd(&fill[r], 1);
        inc[pos] = (int)k;   // k = e * n_p + i
    }
}

// Each row's incidences ascending, one warp per row: the keys (k = e n_p + i)
// are distinct, so an entry's position is the number of smaller keys.  The
// lanes hold up to IS_MAX / 32 keys each in registers, count their ranks
// against every key by shuffles, then store; longer rows (more than IS_MAX
// incident elements) fall back to an insertion sort by lane 0.
constexpr int IS_PER_LANE = 8, IS_MAX = 32 * IS_PER_LANE;

__global__ void __launch_bounds__(256) inc_sort(const int* __restrict__ inc_ptr, int64_t n, int* __restrict__ inc) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += nwarps) {
        const int a = inc_ptr[r], b = inc_ptr[r + 1], L = b - a;
        if (L <= 1) continue;
        if (L <= 32) {   // the common case: one key per lane
            const int v = lane < L ? inc[a + lane] : INT_MAX;
            int rank = 0;
            for (int m = 0; m < L; ++m) rank += __shfl_sync(0xffffffffu, v, m) < v ? 1 : 0;
            __syncwarp();
            if (lane < L) inc[a + rank] = v;
        } else if (L <= IS_MAX) {
            int v[IS_PER_LANE], rank[IS_PER_LANE];
#pragma unroll
            for (int t = 0; t < IS_PER_LANE; ++t) {
                const int i = t * 32 + lane;
                v[t] = i < L ? inc[a + i] : INT_MAX;
                rank[t] = 0;
            }
            const int chunks = (L + 31) >> 5;
#pragma unroll
            for (int c = 0; c < IS_PER_LANE; ++c) {
                if (c >= chunks) break;   // warp-uniform
                for (int m = 0; m < 32; ++m) {
                    const int o = __shfl_sync(0xffffffffu, v[c], m);
#pragma unroll
                    for (int t = 0; t < IS_PER_LANE; ++t) rank[t] += o < v[t] ? 1 : 0;
                }
            }
            __syncwarp();   // every key is in registers before any is stored
#pragma unroll
            for (int t = 0; t < IS_PER_LANE; ++t)
                if (t * 32 + lane < L) inc[a + rank[t]] = v[t];
        } else if (lane == 0) {
            for (int i = a + 1; i < b; ++i) {
                const int v = inc[i];
                int j = i - 1;
                while (j >= a && inc[j] > v) {
                    inc[j + 1] = inc[j];
                    --j;
                }
                inc[j + 1] = v;
            }
        }
    }
}

// ---------------------------------------------------------------- row sort
constexpr int RS_WARPS = 8;

// Row sort by counting: entries ordered by column, ties by ascending element
// entry (a stable sort by column).  One warp per row; the row's
// columns are staged in shared memory, then
//   1. its distinct columns U, ascending, by repeated warp minima (each pass
//      takes the smallest column above the last one found);
//   2. per entry the index of its column in U (binary search) and a count
//      per column (shared-memory atomics on integers: order-free);
//   3. exclusive offsets of the columns, then the entries placed in
//      ascending order, 32 at a time: lanes holding the same column rank
//      among themselves with __match_any_sync, after the entries of earlier
//      chunks (stable).
// Rows with more than RC_CAP entries or RC_UCAP distinct columns are left to
// a rank sort (row_sort_rest, the same order).  The staging takes shared
// memory per warp, and the sort waits on its gathers of conn: the launch
// picks the smallest staging that holds the mesh's longest row, so that
// more warps share an SM (a P1 tetrahedral mesh: rows of at most 4 x 24
// entries, 8 warps of 128 entries per block instead of 4 of 768).
template <int RC_WARPS, int RC_CAP, int RC_UCAP>
__global__ void __launch_bounds__(RC_WARPS * 32) row_sort_count(const int* __restrict__ conn, int np,
                                                                const int* __restrict__ inc_ptr,
                                                                const int* __restrict__ inc, int64_t n,
                                                                int* __restrict__ contrib, int* __restrict__ row_nnz,
                                                                int* __restrict__ overflow) {
    __shared__ int sc_all[RC_WARPS][RC_CAP];
    __shared__ short sb_all[RC_WARPS][RC_CAP];
    __shared__ int su_all[RC_WARPS][RC_UCAP];
    __shared__ int so_all[RC_WARPS][RC_UCAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* sc = sc_all[w];
    short* sb = sb_all[w];
    int* U = su_all[w];
    int* off = so_all[w];
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nwarps = (int64_t)gridDim.x * RC_WARPS;
    for (int64_t r = blockIdx.x * (int64_t)RC_WARPS + w; r < n; r += nwarps) {
        const int start = inc_ptr[r];
        const int L = np * (inc_ptr[r + 1] - start);
        if (L > RC_CAP) {   // left to the rank sort
            if (lane == 0) atomicAdd(overflow, 1);
            continue;
        }
        for (int k = lane; k < L; k += 32) {
            const int ei = inc[start + k / np];
            sc[k] = conn[(int64_t)(ei / np) * np + k % np];
        }
        __syncwarp();
        // 1. distinct columns, ascending
        int u = 0, last = INT_MIN;
        bool too_many = false;
        for (;;) {
            int m = INT_MAX;
            for (int k = lane; k < L; k += 32) {
                const int c = sc[k];
                if (c > last && c < m) m = c;
            }
            m = __reduce_min_sync(0xffffffffu, m);
            if (m == INT_MAX) break;
            if (u == RC_UCAP) {
                too_many = true;
                break;
            }
            if (lane == 0) U[u] = m;
            ++u;
            last = m;
        }
        if (too_many) {
            if (lane == 0) atomicAdd(overflow, 1);
            __syncwarp();
            continue;
        }
        for (int b = lane; b < u; b += 32) off[b] = 0;
        __syncwarp();
        // 2. bucket of every entry and the count per bucket
        for (int k = lane; k < L; k += 32) {
            const int c = sc[k];
            int lo = 0, hi = u - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (U[mid] < c) lo = mid + 1;
                else hi = mid;
            }
            sb[k] = (short)lo;
            atomicAdd(&off[lo], 1);
        }
        __syncwarp();
        // 3. exclusive offsets (lane l scans buckets l*chunk .. ), then stable placement
        {
            const int chunk = (u + 31) / 32;
            const int b0 = lane * chunk, b1 = min(b0 + chunk, u);
            int sum = 0;
            for (int b = b0; b < b1; ++b) sum += off[b];
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int run = incl - sum;
            __syncwarp();
            for (int b = b0; b < b1; ++b) {
                const int c = off[b];
                off[b] = run;
                run += c;
            }
        }
        __syncwarp();
        const int64_t base = (int64_t)np * start;
        for (int k0 = 0; k0 < L; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < L;
            const unsigned act = __ballot_sync(0xffffffffu, valid);
            if (valid) {
                const int b = sb[k];
                const unsigned peers = __match_any_sync(act, b);
                const int pos = off[b] + __popc(peers & lt);
                const int ei = inc[start + k / np];
                contrib[base + pos] = ei * np + (k % np);
                __syncwarp(act);
                if ((peers & lt) == 0) off[b] += __popc(peers);   // the lowest lane of the group
            }
            __syncwarp();
        }
        if (lane == 0) row_nnz[r] = u;
        __syncwarp();
    }
}

// The rank sort for the rows the counting sort left (row_nnz < 0 marks
// them): same result, O(L^2) per row.
__global__ void __launch_bounds__(RS_WARPS * 32) row_sort_rest(const int* __restrict__ conn, int np,
                                                               const int* __restrict__ inc_ptr,
                                                               const int* __restrict__ inc, int64_t n,
                                                               int* __restrict__ contrib, int* __restrict__ row_nnz) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * RS_WARPS;
    for (int64_t r = blockIdx.x * (int64_t)RS_WARPS + w; r < n; r += nwarps) {
        if (row_nnz[r] >= 0) continue;
        const int start = inc_ptr[r];
        const int L = np * (inc_ptr[r + 1] - start);
        const int64_t base = (int64_t)np * start;
        int heads = 0;
        for (int k = lane; k < L; k += 32) {
            const int ei = inc[start + k / np];
            const int ck = conn[(int64_t)(ei / np) * np + k % np];
            int rank = 0, head = 1;
            for (int k2 = 0; k2 < L; ++k2) {
                const int e2 = inc[start + k2 / np];
                const int c2 = conn[(int64_t)(e2 / np) * np + k2 % np];
                rank += (c2 < ck) | ((c2 == ck) & (k2 < k));
                head &= !((c2 == ck) & (k2 < k));
            }
            contrib[base + rank] = ei * np + (k % np);
            heads += head;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) heads += __shfl_xor_sync(0xffffffffu, heads, o);
        if (lane == 0) row_nnz[r] = heads;
    }
}

// ---------------------------------------------------------------- numbering
__global__ void __launch_bounds__(256) row_finish(const int* __restrict__ conn, int np,
                                                  const int* __restrict__ inc_ptr, const int* __restrict__ row_ptr,
                                                  const int* __restrict__ contrib, int64_t n,
                                                  int* __restrict__ col_idx, int* __restrict__ seg_ptr,
                                                  uint2* __restrict__ head) {
    int lane = threadIdx.x & 31;
    int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int np2 = np * np;
    unsigned le = (lane == 31) ? 0xffffffffu : ((1u << (lane + 1)) - 1u);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += nwarps) {
        int64_t start = (int64_t)np * inc_ptr[r], end = (int64_t)np * inc_ptr[r + 1];
        int slot0 = row_ptr[r];
        int carry = -1, count = 0;
        for (int64_t p0 = start; p0 < end; p0 += 32) {
            int64_t p = p0 + lane;
            bool valid = p < end;
            int c = valid ? contrib[p] : 0;
            int col = valid ? conn[(int64_t)(c / np2) * np + c % np] : INT_MAX;
            int prev = __shfl_up_sync(0xffffffffu, col, 1);
            if (lane == 0) prev = carry;
            bool is_head = valid && col != prev;
            unsigned mask = __ballot_sync(0xffffffffu, is_head);
            int idx = count + __popc(mask & le) - 1;
            if (valid && (p & 31) == 0) head[p >> 5].y = (unsigned)(slot0 + idx);
            if (is_head) {
                col_idx[slot0 + idx] = col;
                seg_ptr[slot0 + idx] = (int)p;
                atomicOr(&head[p >> 5].x, 1u << (p & 31));
            }
            count += __popc(mask);
            carry = __shfl_sync(0xffffffffu, col, 31);
        }
    }
}

__global__ void set_last(int* p, int64_t idx, int v) { p[idx] = v; }

// slot[c] for every element entry c: position p of the sorted list holds
// contrib[p]; its slot is the slot of the first position of its group of 32
// plus the heads after that position up to p
__global__ void slot_map_kernel(const int* __restrict__ contrib, const uint2* __restrict__ head, int64_t nc,
                                int* __restrict__ slot) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nc; p += (int64_t)gridDim.x * blockDim.x) {
        const uint2 h = head[p >> 5];
        const unsigned b = (unsigned)(p & 31);
        slot[contrib[p]] = (int)(h.y + __popc(h.x & ((2u << b) - 1u) & ~1u));
    }
}

// the largest incidence count of a row (warp maximum, one atomic per warp)
__global__ void inc_max(const int* __restrict__ inc_ptr, int64_t n, int* __restrict__ out) {
    int best = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        best = max(best, inc_ptr[r + 1] - inc_ptr[r]);
    best = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// longest segment seg_ptr[s+1] - seg_ptr[s] (warp maximum, one atomic per warp)
__global__ void seg_max(const int* __restrict__ seg_ptr, int64_t nnz, int* __restrict__ out) {
    int best = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x)
        best = max(best, seg_ptr[s + 1] - seg_ptr[s]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

int grid_for(int64_t work, int threads, int64_t cap = 152 * 32) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

// exclusive scan of n ints into n+1 outputs
int scan_exclusive(const int* in, int64_t n, int* out, cudaStream_t s) {
    int64_t nt = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
    DevBuf sums;
    int rc = buf_alloc(sums, sizeof(int) * (size_t)nt, s);
    if (rc) return rc;
    scan_tile_sums<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, sums.as<int>());
    scan_sums<<<1, 1024, 0, s>>>(sums.as<int>(), (int)nt);
    scan_apply<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, sums.as<int>(), out);
    cudaError_t e = cudaGetLastError();
    buf_free(sums, s);
    if (e != cudaSuccess) return cuda_fail(e, "scan");
    return FEM_OK;
}

// The element-entry -> slot map, built when first needed (the boundary
// terms and fem_get_slot_map read it; reassembly does not).
int slot_map_build(fem_mesh& m, cudaStream_t s) {
    if (m.have_slot) return FEM_OK;
    if (!m.have_pattern) return fail(FEM_ESTATE, "fem_symbolic has not run");
    const int64_t nc = m.E * m.np * m.np;
    int rc = buf_alloc(m.slot, sizeof(int) * (size_t)(nc + 1), s);
    if (rc) return rc;
    cudaGetLastError();   // clear any stale error before the launch check
    if (nc > 0)
        slot_map_kernel<<<grid_for(nc, 256, 152 * 64), 256, 0, s>>>(m.contrib.as<int>(), m.seg_head.as<uint2>(), nc,
                                                                    m.slot.as<int>());
    FEM_CUDA_TRY(cudaGetLastError());
    m.have_slot = true;
    return FEM_OK;
}

int symbolic_run(fem_mesh& m, cudaStream_t s) {
    const int np = m.np;
    const int64_t n = m.n, E = m.E;
    const int64_t m1 = E * np, m2 = E * np * np;
    int rc;
    DevBuf cnt, fill, row_nnz;
    if ((rc = buf_alloc(cnt, sizeof(int) * (size_t)(n + 1), s))) return rc;
    if ((rc = buf_alloc(m.inc_ptr, sizeof(int) * (size_t)(n + 1), s))) return rc;
    if ((rc = buf_alloc(m.inc, sizeof(int) * (size_t)(m1 + 1), s))) return rc;
    if ((rc = buf_alloc(fill, sizeof(int) * (size_t)(n + 1), s))) return rc;
    if ((rc = buf_alloc(m.contrib, sizeof(int) * (size_t)(m2 + 1), s))) return rc;
    if ((rc = buf_alloc(row_nnz, sizeof(int) * (size_t)(n + 1), s))) return rc;
    if ((rc = buf_alloc(m.row_ptr, sizeof(int) * (size_t)(n + 1), s))) return rc;
    FEM_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, cnt.bytes, s));
    FEM_CUDA_TRY(cudaMemsetAsync(fill.ptr, 0, fill.bytes, s));
    cudaGetLastError();   // clear any stale error before the launch checks
    const int* conn = m.conn.as<int>();
    inc_count<<<grid_for(m1, 256), 256, 0, s>>>(conn, m1, cnt.as<int>());
    if ((rc = scan_exclusive(cnt.as<int>(), n, m.inc_ptr.as<int>(), s))) return rc;
    inc_fill<<<grid_for(m1, 256), 256, 0, s>>>(conn, m1, m.inc_ptr.as<int>(), fill.as<int>(), m.inc.as<int>());
    inc_sort<<<grid_for(n * 32, 256, 152 * 64), 256, 0, s>>>(m.inc_ptr.as<int>(), n, m.inc.as<int>());
    // rows by counting sort; the few rows it leaves (marked -1) by rank sort
    FEM_CUDA_TRY(cudaMemsetAsync(row_nnz.ptr, 0xff, row_nnz.bytes, s));
    FEM_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, sizeof(int), s));   // overflow count (the incidence counts are scanned)
    {
        // the longest row (entries = n_p x incidences) picks the staging
        FEM_CUDA_TRY(cudaMemsetAsync(fill.ptr, 0, sizeof(int), s));
        inc_max<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(m.inc_ptr.as<int>(), n, fill.as<int>());
        FEM_CUDA_TRY(cudaGetLastError());
        int maxinc = 0;
        FEM_CUDA_TRY(cudaMemcpyAsync(&maxinc, fill.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        FEM_CUDA_TRY(cudaStreamSynchronize(s));
        const int64_t maxL = (int64_t)np * maxinc;
        auto sort_rows = [&](auto kern, int warps) {
            kern<<<grid_for(n, warps, 152 * 64), warps * 32, 0, s>>>(conn, np, m.inc_ptr.as<int>(), m.inc.as<int>(), n,
                                                                    m.contrib.as<int>(), row_nnz.as<int>(),
                                                                    cnt.as<int>());
        };
        if (maxL <= 128) sort_rows(row_sort_count<8, 128, 64>, 8);
        else if (maxL <= 256) sort_rows(row_sort_count<8, 256, 128>, 8);
        else sort_rows(row_sort_count<4, 768, 384>, 4);
    }
    FEM_CUDA_TRY(cudaGetLastError());
    int left = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&left, cnt.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (left > 0) {
        row_sort_rest<<<grid_for(n, RS_WARPS, 152 * 64), RS_WARPS * 32, 0, s>>>(
            conn, np, m.inc_ptr.as<int>(), m.inc.as<int>(), n, m.contrib.as<int>(), row_nnz.as<int>());
        FEM_CUDA_TRY(cudaGetLastError());
    }
    if ((rc = scan_exclusive(row_nnz.as<int>(), n, m.row_ptr.as<int>(), s))) return rc;
    int nnz = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&nnz, m.row_ptr.as<int>() + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    m.nnz = nnz;
    if ((rc = buf_alloc(m.col_idx, sizeof(int) * (size_t)(nnz + 1), s))) return rc;
    if ((rc = buf_alloc(m.seg_ptr, sizeof(int) * (size_t)(nnz + 1), s))) return rc;
    const int64_t ngroups = (m2 + 31) / 32;
    if ((rc = buf_alloc(m.seg_head, sizeof(uint2) * (size_t)(ngroups + 1), s))) return rc;
    FEM_CUDA_TRY(cudaMemsetAsync(m.seg_head.ptr, 0, m.seg_head.bytes, s));
    row_finish<<<grid_for(n, 8, 152 * 64), 256, 0, s>>>(conn, np, m.inc_ptr.as<int>(), m.row_ptr.as<int>(),
                                                        m.contrib.as<int>(), n, m.col_idx.as<int>(),
                                                        m.seg_ptr.as<int>(), m.seg_head.as<uint2>());
    set_last<<<1, 1, 0, s>>>(m.seg_ptr.as<int>(), nnz, (int)m2);
    FEM_CUDA_TRY(cudaGetLastError());
    // the longest segment bounds the steps of the CSR sum's warp scans
    int* dmax = cnt.as<int>();   // the incidence counts are no longer needed
    FEM_CUDA_TRY(cudaMemsetAsync(dmax, 0, sizeof(int), s));
    seg_max<<<grid_for(nnz, 256, 152 * 8), 256, 0, s>>>(m.seg_ptr.as<int>(), nnz, dmax);
    FEM_CUDA_TRY(cudaGetLastError());
    int maxseg = 0;
    FEM_CUDA_TRY(cudaMemcpyAsync(&maxseg, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    buf_free(cnt, s);
    buf_free(fill, s);
    buf_free(row_nnz, s);
    FEM_CUDA_TRY(cudaStreamSynchronize(s));
    m.max_seg = maxseg;
    m.have_pattern = true;
    return FEM_OK;
}

}  // namespace fem
