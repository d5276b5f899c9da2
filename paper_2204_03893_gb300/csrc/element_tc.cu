// element_tc.cu -- element products V = X Q on the tcgen05 tensor cores
// (TF32 x3 split precision, FP32 accumulation in tensor memory).
//
// The formation step of Algorithm 2 for a tile of 128 elements: every thread forms the
// X row of one element (Lambda = S * (w b^T) in place, eq. def_lambda;
// X_c = Lambda (.) W, Section 4.2; the tangent factors of the Section 5.2
// tensor multiplied by u) and stores it, split as X = Xhi + Xlo with Xhi,
// Xlo exact TF32 values, straight into the K-major shared-memory operand
// layout.  Q (reference element only, "computed and stored once and for
// all", Section 4.1) sits in shared memory for the whole persistent CTA,
// split the same way.  One thread issues, per K step of 8,
//     D += Xhi Qhi ; D += Xhi Qlo ; D += Xlo Qhi
// for M, K and T into separate TMEM column ranges (D: 128 lanes = elements,
// columns = entries), commits to an mbarrier, and the four warps read their
// 32 lanes back with tcgen05.ld into row-major blocks in shared memory that
// the copy engine writes to V (cp.async.bulk, one copy per warp and matrix).  Only the n_p(n_p+1)/2 distinct
// entries of M and K are formed (Section 7).
//
// Every mbarrier wait is bounded (~1 s of SM clocks); on timeout the kernel
// records an error word, stops, and releases its tensor memory.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "fem_internal.h"
#include "refelem.h"
#include "tc_ptx.cuh"

namespace fem {

namespace {

__host__ __device__ constexpr int ru(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int pow2_at_least(int x) {
    int p = 32;
    while (p < x) p *= 2;
    return p;
}

constexpr int TILE = 128;
constexpr int SMEM_MAX = 227 * 1024;
constexpr int STAGE_FLOATS = 4 * 32 * 33;   // epilogue_staged: 32 x 33 floats per warp
constexpr int IMG_SLOT_FLOATS = 24 * 1024;   // 96 KiB per element type

// Tile layout.  The X columns of M, K and T are packed into one K-major
// operand of KTOTp = ru(KM + KK + KT, 8) columns per element row (M at 0, K
// at KM, T at KM + KK).  Each matrix's MMAs run over the 8-wide K slices that
// overlap its own columns, and its Q image has zero rows at the columns of
// the neighbouring matrices, so the packing costs no extra products of any
// weight and saves the per-matrix padding (40 instead of 48 columns for P2
// triangles, which lets 4 CTAs share an SM).
template <typename ETy>
struct TcL {
    static constexpr int KM = ETy::KM, KK = ETy::KK, KT = ETy::KT;
    static constexpr int KTOT = KM + KK + KT, KTOTp = ru(KTOT, 8);
    static constexpr int OFF_M = 0, OFF_K = KM, OFF_T = KM + KK;
    // first slice and slice count of each matrix
    static constexpr int SM0 = 0, NSM = ru(KM, 8) / 8;
    static constexpr int SK0 = KM / 8, NSK = ru(KM + KK, 8) / 8 - KM / 8;
    static constexpr int ST0 = (KM + KK) / 8, NST = KTOTp / 8 - (KM + KK) / 8;
    static constexpr int NMp = ru(ETy::NSYM, 16), NTp = ru(ETy::NT, 16);
    static constexpr int COLM = 0, COLK = NMp, COLT = 2 * NMp, COLS = 2 * NMp + NTp;
    static constexpr int ALLOC = pow2_at_least(COLS);
    // shared-memory byte offsets: Q images (each matrix's slices), then X
    static constexpr int QMh = 0;
    static constexpr int QMl = QMh + NMp * NSM * 8 * 4;
    static constexpr int QKh = QMl + NMp * NSM * 8 * 4;
    static constexpr int QKl = QKh + NMp * NSK * 8 * 4;
    static constexpr int QTh = QKl + NMp * NSK * 8 * 4;
    static constexpr int QTl = QTh + NTp * NST * 8 * 4;
    static constexpr int QEND = QTl + NTp * NST * 8 * 4;
    static constexpr int XH = 0, XL = TILE * KTOTp * 4;
    static constexpr int XEND = 2 * TILE * KTOTp * 4;
    static constexpr uint32_t SBO_X = (KTOTp / 4) * 128;
    static constexpr int SMEM = QEND + XEND;
    // threads per element row in the single-mesh kernel, measured on GB300:
    // two (each forming half of the quadrature points) pay off for the
    // elements with many quadrature points (P3 triangles, P2 tetrahedra:
    // 0.76 vs 0.88 ms on tet_p2_64); P1/P2 triangles and P1 tetrahedra run
    // faster with one thread per row and 4 CTAs per SM (0.27 vs 0.29 ms on
    // tri_p2_1024, 0.73 vs 1.10 ms on tet_p1_128)
    static constexpr int TPR = ETy::NQ >= 11 ? 2 : 1;
    // CTAs per SM the tile fits (shared memory, TMEM; at most 3), the
    // register budget of __launch_bounds__ with two threads per row
    static constexpr int MINB_SMEM = (228 * 1024) / (SMEM + 1024), MINB_TMEM = 512 / ALLOC;
    static constexpr int MINB2 = MINB_SMEM < 1 ? 1 : MINB_SMEM < MINB_TMEM ? (MINB_SMEM < 3 ? MINB_SMEM : 3)
                                                                        : (MINB_TMEM < 3 ? MINB_TMEM : 3);
    // one thread per row: ask for the 4 CTAs per SM the tile fits, so that
    // the formation code specialised per law class stays within 128 registers
    static constexpr int MINB1 = MINB_SMEM < 4 || MINB_TMEM < 4 ? 1 : 4;
    static constexpr int MINB = TPR == 2 ? MINB2 : MINB1;
    // epilogue reads whole 32-column chunks: they must stay inside the allocation
    static constexpr bool FITS = NMp <= 256 && NTp <= 256 && ALLOC <= 512 && SMEM <= SMEM_MAX &&
                                 XEND >= 4 * 32 * ETy::NT * 4 && QEND <= IMG_SLOT_FLOATS * 4 &&
                                 COLM + ru(ETy::NSYM, 32) <= ALLOC && COLK + ru(ETy::NSYM, 32) <= ALLOC &&
                                 COLT + ru(ETy::NT, 32) <= ALLOC &&
                                 // packed order M, K, T; slices cover each matrix's columns
                                 OFF_M == 0 && SM0 == 0 && OFF_K <= OFF_T && SK0 * 8 <= OFF_K &&
                                 ST0 * 8 <= OFF_T && (SK0 + NSK) * 8 >= OFF_T && (ST0 + NST) * 8 == KTOTp &&
                                 XH == 0 && XL == XEND / 2 && SBO_X == (uint32_t)KTOTp * 32;
};

__constant__ float c_tcref[TAB_TOTAL];
__device__ float g_tcimg[6 * IMG_SLOT_FLOATS];
__device__ int g_tc_err;

constexpr long long WAIT_LIMIT = 2000000000LL;   // SM clocks (~1 s)

// Calls f(std::integral_constant<int, LC>) for the law class of k: the
// formation code is compiled once per class and the branch is taken once per
// tile, outside the quadrature loops.  SIN = false leaves the sine law to the
// generic code (one copy fewer where registers are tight).
template <bool SIN = true, typename F>
__device__ __forceinline__ void with_law(int lc, F&& f) {
    if (lc == LC_POLY3) f(std::integral_constant<int, LC_POLY3>{});
    else if (SIN && lc == LC_SIN) f(std::integral_constant<int, LC_SIN>{});
    else f(std::integral_constant<int, LC_ANY>{});
}

// Per-phase SM clock counters, compiled in only with -DFEM_PHASE_TIMERS (the
// default build has none): thread 0 of each CTA adds the clocks spent since
// its previous mark to a slot of g_phase (summed over CTAs), so a phase's
// share of a tile is read from thread 0's timeline.  Slots 0-4: tile kernel
// (formation incl. the barrier, MMA issue, MMA wait, epilogue, tiles);
// 8-14: chunked kernel (tile gathers, formation, copy wait, MMA issue, MMA
// wait, epilogue, tiles).
struct PhaseTimer {
#ifdef FEM_PHASE_TIMERS
    long long last = 0;
    __device__ __forceinline__ void start() {
        if (threadIdx.x == 0) last = clock64();
    }
    __device__ __forceinline__ void mark(int slot, long long add = -1);
#else
    __device__ __forceinline__ void start() {}
    __device__ __forceinline__ void mark(int, long long = -1) {}
#endif
};
#ifdef FEM_PHASE_TIMERS
__device__ unsigned long long g_phase[16];
__device__ __forceinline__ void PhaseTimer::mark(int slot, long long add) {
    if (threadIdx.x != 0) return;
    const long long t = clock64();
    atomicAdd(&g_phase[slot], (unsigned long long)(add >= 0 ? add : t - last));
    last = t;
}
#endif

// store one thread's X row (Kp values) as TF32 hi / lo parts
template <int Kp>
__device__ __forceinline__ void store_row(unsigned char* hi, unsigned char* lo, const float (&x)[Kp], int r) {
    constexpr uint32_t sbo = (Kp / 4) * 128;
    unsigned char* ph = hi + (r >> 3) * sbo + (r & 7) * 16;
    unsigned char* pl = lo + (r >> 3) * sbo + (r & 7) * 16;
#pragma unroll
    for (int c = 0; c < Kp / 4; ++c) {
        float4 h, l;
        h.x = tc::tf32_rna(x[4 * c + 0]);
        h.y = tc::tf32_rna(x[4 * c + 1]);
        h.z = tc::tf32_rna(x[4 * c + 2]);
        h.w = tc::tf32_rna(x[4 * c + 3]);
        l.x = tc::tf32_rna(x[4 * c + 0] - h.x);
        l.y = tc::tf32_rna(x[4 * c + 1] - h.y);
        l.z = tc::tf32_rna(x[4 * c + 2] - h.z);
        l.w = tc::tf32_rna(x[4 * c + 3] - h.w);
        *reinterpret_cast<float4*>(ph + c * 128) = h;
        *reinterpret_cast<float4*>(pl + c * 128) = l;
    }
}

// columns [c0, c0 + NC) of one X row of Kp columns (c0 and NC multiples of 4)
template <int Kp, int NC>
__device__ __forceinline__ void store_row_part(unsigned char* hi, unsigned char* lo, const float (&x)[NC], int r,
                                               int c0) {
    static_assert(NC % 4 == 0 && Kp % 4 == 0, "column groups of 4");
    constexpr uint32_t sbo = (Kp / 4) * 128;
    unsigned char* ph = hi + (r >> 3) * sbo + (r & 7) * 16 + (c0 >> 2) * 128;
    unsigned char* pl = lo + (r >> 3) * sbo + (r & 7) * 16 + (c0 >> 2) * 128;
#pragma unroll
    for (int c = 0; c < NC / 4; ++c) {
        float4 h, l;
        h.x = tc::tf32_rna(x[4 * c + 0]);
        h.y = tc::tf32_rna(x[4 * c + 1]);
        h.z = tc::tf32_rna(x[4 * c + 2]);
        h.w = tc::tf32_rna(x[4 * c + 3]);
        l.x = tc::tf32_rna(x[4 * c + 0] - h.x);
        l.y = tc::tf32_rna(x[4 * c + 1] - h.y);
        l.z = tc::tf32_rna(x[4 * c + 2] - h.z);
        l.w = tc::tf32_rna(x[4 * c + 3] - h.w);
        *reinterpret_cast<float4*>(ph + c * 128) = h;
        *reinterpret_cast<float4*>(pl + c * 128) = l;
    }
}

// D[dcol..] (+)= sum over K steps of (Xhi Qhi + Xhi Qlo + Xlo Qhi); with
// `acc` the first product also accumulates onto what D holds
template <int Kp>
__device__ __forceinline__ void issue_tf32x3(uint32_t tmem_d, uint32_t xh, uint32_t xl, uint32_t qh, uint32_t ql,
                                             uint32_t idesc, bool acc = false) {
    constexpr uint32_t sbo = (Kp / 4) * 128;
#pragma unroll
    for (int ks = 0; ks < Kp / 8; ++ks) {
        uint64_t ah = tc::smem_desc(xh + ks * 256, 128, sbo);
        uint64_t al = tc::smem_desc(xl + ks * 256, 128, sbo);
        uint64_t bh = tc::smem_desc(qh + ks * 256, 128, sbo);
        uint64_t bl = tc::smem_desc(ql + ks * 256, 128, sbo);
        tc::mma_tf32(tmem_d, ah, bh, idesc, (ks > 0 || acc) ? 1u : 0u);
        tc::mma_tf32(tmem_d, ah, bl, idesc, 1u);
        tc::mma_tf32(tmem_d, al, bh, idesc, 1u);
    }
}

// One matrix of the packed tile: D (+)= sum over its `ns` K slices of
// (Xhi Qhi + Xhi Qlo + Xlo Qhi), X slices s0 .. s0+ns-1 of the packed row
// (stride sbo_x), Q slices 0 .. ns-1 of the matrix's own image.
template <int NS_>
__device__ __forceinline__ void issue_packed(uint32_t tmem_d, uint32_t xh, uint32_t xl, uint32_t sbo_x, int s0,
                                             uint32_t qh, uint32_t ql, uint32_t idesc) {
    constexpr uint32_t sbo_q = (NS_ * 8 / 4) * 128;
#pragma unroll
    for (int ks = 0; ks < NS_; ++ks) {
        const uint32_t xo = (uint32_t)(s0 + ks) * 256, qo = (uint32_t)ks * 256;
        uint64_t ah = tc::smem_desc(xh + xo, 128, sbo_x);
        uint64_t al = tc::smem_desc(xl + xo, 128, sbo_x);
        uint64_t bh = tc::smem_desc(qh + qo, 128, sbo_q);
        uint64_t bl = tc::smem_desc(ql + qo, 128, sbo_q);
        tc::mma_tf32(tmem_d, ah, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32(tmem_d, ah, bl, idesc, 1u);
        tc::mma_tf32(tmem_d, al, bh, idesc, 1u);
    }
}

// The MMAs of one packed tile for the requested matrices (thread 0).
template <typename L>
__device__ __forceinline__ void issue_tile(uint32_t tmem, uint32_t sXu, uint32_t sQu, bool doM, bool doK, bool doT) {
    if (doM)
        issue_packed<L::NSM>(tmem + L::COLM, sXu + L::XH, sXu + L::XL, L::SBO_X, L::SM0, sQu + L::QMh, sQu + L::QMl,
                             tc::idesc_tf32(L::NMp));
    if (doK)
        issue_packed<L::NSK>(tmem + L::COLK, sXu + L::XH, sXu + L::XL, L::SBO_X, L::SK0, sQu + L::QKh, sQu + L::QKl,
                             tc::idesc_tf32(L::NMp));
    if (doT)
        issue_packed<L::NST>(tmem + L::COLT, sXu + L::XH, sXu + L::XL, L::SBO_X, L::ST0, sQu + L::QTh, sQu + L::QTl,
                             tc::idesc_tf32(L::NTp));
}

// The warp's block `blk` (32 rows of NF floats, the image of V rows
// row0..row0+31) -> V: lane 0 hands the whole block to one bulk copy
// (cp.async.bulk shared -> global; the block and V + row0 NF are 16-byte
// aligned since row0 is a multiple of 32).  The caller waits for the bulk
// reads before it reuses the block.  A partial last block (rows past E) is
// copied by the warp with plain stores.
template <int NF>
__device__ __forceinline__ void block_out(const float* blk, float* __restrict__ V, int64_t row0, int64_t E,
                                          int lane) {
    static_assert((32 * NF * 4) % 16 == 0, "bulk block size");
    if (E - row0 >= 32) {
        tc::fence_proxy_async_smem();   // this thread's row -> visible to the copy engine
        __syncwarp();
        if (lane == 0) tc::bulk_s2g(V + row0 * NF, tc::smem_u32(blk), 32u * NF * 4u);
    } else {
        __syncwarp();
        const int rows = E - row0 < 32 ? (int)(E - row0) : 32;
        const int nf = rows * NF, nv = nf >> 2;
        float* g = V + row0 * NF;   // 16-byte aligned (row0 is a multiple of 32)
        for (int i = lane; i < nv; i += 32) reinterpret_cast<float4*>(g)[i] = reinterpret_cast<const float4*>(blk)[i];
        for (int i = (nv << 2) + lane; i < nf; i += 32) g[i] = blk[i];
        __syncwarp();
    }
}

// TMEM (this warp's 32 lanes = 32 consecutive elements, columns col..col+N)
// -> V: every thread writes its row into the warp's block, then block_out.
template <int N, int W = 32>
__device__ __forceinline__ void epilogue_bulk(uint32_t tmem, int col, float* blk, float* __restrict__ V, int64_t row0,
                                              int64_t E, int warp, int lane) {
    if (row0 >= E) return;   // warp-uniform
    // W: columns per TMEM load (16 where registers are scarce)
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += W) {
        uint32_t r[W];
        tc::tmem_ld<W>(tmem + (static_cast<uint32_t>(warp * 32) << 16) + col + c0, r);
        float* dst = blk + lane * N + c0;
        if constexpr (N % 4 == 0) {
#pragma unroll
            for (int j = 0; j < W; j += 4)
                if (c0 + j < N)
                    *reinterpret_cast<float4*>(dst + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                                      __uint_as_float(r[j + 2]),
                                                                      __uint_as_float(r[j + 3]));
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j)
                if (c0 + j < N) dst[j] = __uint_as_float(r[j]);
        }
    }
    block_out<N>(blk, V, row0, E, lane);
}

// M and K (TMEM columns colM.., colK.., NS symmetric entries each) -> the
// interleaved V_MK rows (entry s of an element at 2s for M, 2s + 1 for K):
// each thread stores (M_s, K_s) pairs into its row of the warp's block (an
// unrequested matrix's half is written as 0), then block_out.  The 8-byte
// stores of a half-warp hit distinct bank pairs (row stride 2 NS floats,
// NS odd) or at worst two.
template <int NS, int WMAX = 32>
__device__ __forceinline__ void epilogue_mk_bulk(uint32_t tmem, int colM, int colK, float* blk,
                                                 float* __restrict__ VMK, bool doM, bool doK, int64_t row0, int64_t E,
                                                 int warp, int lane) {
    if (row0 >= E) return;   // warp-uniform
    // columns per TMEM load: the narrowest shape that covers a small NS
    constexpr int W = NS <= 8 ? 8 : NS <= 16 || WMAX == 16 ? 16 : 32;
    const uint32_t lanes = static_cast<uint32_t>(warp * 32) << 16;
#pragma unroll 1
    for (int c0 = 0; c0 < NS; c0 += W) {
        uint32_t rm[W], rk[W];
        if (doM) {
            tc::tmem_ld<W>(tmem + lanes + colM + c0, rm);
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j) rm[j] = 0u;
        }
        if (doK) {
            tc::tmem_ld<W>(tmem + lanes + colK + c0, rk);
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j) rk[j] = 0u;
        }
        float* dst = blk + lane * 2 * NS + 2 * c0;
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (c0 + j < NS)
                *reinterpret_cast<float2*>(dst + 2 * j) = make_float2(__uint_as_float(rm[j]), __uint_as_float(rk[j]));
    }
    block_out<2 * NS>(blk, VMK, row0, E, lane);
}

// The epilogue of one tile (M and K interleaved, T, as requested) through
// the X region of shared memory (`stage`, free once the MMAs are complete).
// Where both blocks fit side by side, both copies are in flight at once;
// otherwise the warp's one block is reused and the first copy's reads are
// waited for.  Returns with every bulk read of this warp complete, so the
// caller may overwrite the region after a block barrier.
template <typename ETy, int XEND, int W = 32>
__device__ __forceinline__ void epilogue_tile(uint32_t tmem, int colM, int colK, int colT, float* stage,
                                              float* __restrict__ VMK, float* __restrict__ VT, bool doM, bool doK,
                                              bool doT, int64_t row0, int64_t E, int warp, int lane) {
    constexpr int NMK = 2 * ETy::NSYM, NT = ETy::NT, NMAX = NMK > NT ? NMK : NT;
    constexpr bool DISJOINT = TILE * (NMK + NT) * 4 <= XEND;
    static_assert(TILE * NMAX * 4 <= XEND, "epilogue blocks do not fit the X region");
    float* bMK = DISJOINT ? stage + warp * 32 * NMK : stage + warp * 32 * NMAX;
    float* bT = DISJOINT ? stage + TILE * NMK + warp * 32 * NT : bMK;
    auto drain = [&]() {
        if (lane == 0) {
            tc::bulk_commit();
            tc::bulk_wait_read_all();
        }
        __syncwarp();
    };
    if (doM || doK) epilogue_mk_bulk<ETy::NSYM, W>(tmem, colM, colK, bMK, VMK, doM, doK, row0, E, warp, lane);
    if (!DISJOINT && (doM || doK)) drain();
    if (doT) epilogue_bulk<NT, W>(tmem, colT, bT, VT, row0, E, warp, lane);
    drain();
}

// TMEM (this warp's 32 lanes, columns col..col+N) -> V rows through a
// 32 x 33 staging tile per warp (stage + warp 32 x 33 floats): each store
// instruction writes one row.  Used where the whole-block staging of
// `epilogue` would not fit (the chunked product's 400-column T).
// Column c of a row lands at V[row LD + c_off + c CS].  The interleaved
// M/K storage (CS = 2) is written in two passes: M first as full (M, 0)
// pairs (PAIR: 8-byte stores, whole sectors, so L2 holds them without
// fetching the sectors from DRAM), then K into the odd positions of the
// same, still cached, sectors.
// The warp reads TMEM lane quadrant `quad` (its own: warp mod 4), stages
// through tile `slot`, and drains the 32-column chunks part, part + parts, ...
// (so two warps of one quadrant can split a block).
template <int N, int LD = N, int CS = 1, bool PAIR = false>
__device__ __forceinline__ void epilogue_staged(uint32_t tmem, int col, float* stage_base, float* __restrict__ V,
                                                int64_t row0, int64_t E, int quad, int lane, int c_off, int slot,
                                                int part, int parts) {
    float* stage = stage_base + slot * 32 * 33;
#pragma unroll 1
    for (int c0 = 32 * part; c0 < N; c0 += 32 * parts) {
        uint32_t r[32];
        tc::tmem_ld32(tmem + (static_cast<uint32_t>(quad * 32) << 16) + col + c0, r);
#pragma unroll
        for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            int64_t er = row0 + rr;
            int c = c0 + lane;
            if (er < E && c < N) {
                if constexpr (PAIR)
                    *reinterpret_cast<float2*>(V + er * LD + c * 2) = make_float2(stage[rr * 33 + lane], 0.f);
                else
                    V[er * LD + c_off + c * CS] = stage[rr * 33 + lane];
            }
        }
        __syncwarp();
    }
}

// X row of one element (Section 4: Lambda = S * (w b^T) in place; X_c =
// Lambda (.) W; the tangent factors), from its gathered nodal values (split
// as hi + lo) and its geometry (b_e, A_e upper triangle), packed as
// [X_M | X_K | X_T]; the padding columns stay as the caller set them (zero).
template <typename ETy, int KTOTp, int LC = LC_ANY>
__device__ __forceinline__ void form_x(const float2 (&pu)[ETy::NP], const float (&pgeo)[1 + ETy::NS], bool need_u,
                                       const CoeffDev& k, float mass, float (&x)[KTOTp]) {
    constexpr int OFF_K = ETy::KM, OFF_T = ETy::KM + ETy::KK;
    constexpr int D = ETy::D, NP = ETy::NP, NQ = ETy::NQ, NS = ETy::NS;
    constexpr int TO = type_tab_off(ETy::TYPE);
    constexpr int PHI = TO, GR = TO + NQ * NP, WQ = TO + NQ * NP * (1 + D);
    // du[i] = u_i - u_0 from the (hi, lo) split of u (exact differences of
    // the hi parts); u is only needed for K and T (mass-only calls pass NULL)
    float du[NP];
    float u0 = 0.f;
    if (need_u) {
        u0 = pu[0].x + pu[0].y;
#pragma unroll
        for (int i = 0; i < NP; ++i) du[i] = (pu[i].x - pu[0].x) + (pu[i].y - pu[0].y);
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) du[i] = 0.f;
    }
    const float b = pgeo[0];
    float A[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) A[t] = pgeo[1 + t];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float uq = 0.f, g[D];
#pragma unroll
        for (int a = 0; a < D; ++a) g[a] = 0.f;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            uq = fmaf(c_tcref[PHI + q * NP + i], du[i], uq);
#pragma unroll
            for (int a = 0; a < D; ++a) g[a] = fmaf(c_tcref[GR + (q * NP + i) * D + a], du[i], g[a]);
        }
        uq += u0;
        float dk;
        const float kq = k_eval<float, LC>(k, uq, dk);
        const float lam = c_tcref[WQ + q] * b;
        x[q] = mass * lam;
        const float lk = lam * kq;
#pragma unroll
        for (int t = 0; t < NS; ++t) x[OFF_K + q * NS + t] = lk * A[t];
        const float ld = lam * dk;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float sacc = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const int lo = a < c ? a : c, hi = a < c ? c : a;
                sacc = fmaf(A[lo * D - (lo * (lo - 1)) / 2 + (hi - lo)], g[c], sacc);
            }
            x[OFF_T + q * D + a] = ld * sacc;
        }
    }
}

// One half of an element's X row (Section 4 as in form_x), written straight
// into the K-major TF32 hi/lo operand: the columns of quadrature points
// [QLO, QHI) of every matrix, H = 0 for the first ceil(NQ/2) points, H = 1
// for the rest (which also zeroes the padding columns).  `valid` false (a
// row past E) writes zeros.  Scalar stores: a half's columns do not form
// whole 4-column groups.
template <typename ETy, int KTOTp, int H, int LC = LC_ANY>
__device__ __forceinline__ void form_x_half(const float2 (&pu)[ETy::NP], const float (&pgeo)[1 + ETy::NS],
                                            bool valid, bool need_u, const CoeffDev& k, float mass,
                                            unsigned char* xh, unsigned char* xl, int r) {
    constexpr int OFF_K = ETy::KM, OFF_T = ETy::KM + ETy::KK, KTOT = OFF_T + ETy::KT;
    constexpr int D = ETy::D, NP = ETy::NP, NQ = ETy::NQ, NS = ETy::NS;
    constexpr int QLO = H == 0 ? 0 : (NQ + 1) / 2, QHI = H == 0 ? (NQ + 1) / 2 : NQ;
    constexpr int TO = type_tab_off(ETy::TYPE);
    constexpr int PHI = TO, GR = TO + NQ * NP, WQ = TO + NQ * NP * (1 + D);
    constexpr uint32_t sbo = (KTOTp / 4) * 128;
    const uint32_t rowoff = (r >> 3) * sbo + (r & 7) * 16;
    auto put = [&](int c, float v) {
        const uint32_t o = rowoff + (c >> 2) * 128 + (c & 3) * 4;
        const float h = tc::tf32_rna(v);
        *reinterpret_cast<float*>(xh + o) = h;
        *reinterpret_cast<float*>(xl + o) = tc::tf32_rna(v - h);
    };
    float du[NP];
    float u0 = 0.f;
    if (valid && need_u) {
        u0 = pu[0].x + pu[0].y;
#pragma unroll
        for (int i = 0; i < NP; ++i) du[i] = (pu[i].x - pu[0].x) + (pu[i].y - pu[0].y);
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) du[i] = 0.f;
    }
    const float b = valid ? pgeo[0] : 0.f;
    float A[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) A[t] = valid ? pgeo[1 + t] : 0.f;
#pragma unroll
    for (int q = QLO; q < QHI; ++q) {
        float uq = 0.f, g[D];
#pragma unroll
        for (int a = 0; a < D; ++a) g[a] = 0.f;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            uq = fmaf(c_tcref[PHI + q * NP + i], du[i], uq);
#pragma unroll
            for (int a = 0; a < D; ++a) g[a] = fmaf(c_tcref[GR + (q * NP + i) * D + a], du[i], g[a]);
        }
        uq += u0;
        float dk;
        const float kq = k_eval<float, LC>(k, uq, dk);
        const float lam = c_tcref[WQ + q] * b;   // 0 for an invalid row, so every column is 0
        put(q, mass * lam);
        const float lk = lam * kq;
#pragma unroll
        for (int t = 0; t < NS; ++t) put(OFF_K + q * NS + t, lk * A[t]);
        const float ld = lam * dk;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float sacc = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const int lo = a < c ? a : c, hi = a < c ? c : a;
                sacc = fmaf(A[lo * D - (lo * (lo - 1)) / 2 + (hi - lo)], g[c], sacc);
            }
            put(OFF_T + q * D + a, ld * sacc);
        }
    }
    if constexpr (H == 1) {
#pragma unroll
        for (int c = KTOT; c < KTOTp; ++c) put(c, 0.f);
    }
}

// LC: the law class the formation is compiled for (the launch picks it from
// k; LC_ANY evaluates every law).
template <typename ETy, int LC>
__global__ void __launch_bounds__(TcL<ETy>::TPR * TILE, TcL<ETy>::MINB) element_tc_kernel(const int* __restrict__ conn, const float* __restrict__ geo,
                                                          int64_t E, int64_t gs, const double* __restrict__ u, CoeffDev k,
                                                          float mass, float* __restrict__ VM, float* __restrict__ VK,
                                                          float* __restrict__ VT, const float* __restrict__ img,
                                                          int* __restrict__ err) {
    using L = TcL<ETy>;
    constexpr int NP = ETy::NP, NS = ETy::NS;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;

    // TPR threads per element row.  With two: warps 0-3 form the first half
    // of each row's quadrature points and drain TMEM (they own its lanes),
    // warps 4-7 form the second half.
    constexpr int NTHR = L::TPR * TILE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = tid & (TILE - 1), half = tid / TILE;
    unsigned char* sQ = smem;
    unsigned char* sX = smem + L::QEND;

    {   // resident Q image
        const int4* src = reinterpret_cast<const int4*>(img);
        int4* dst = reinterpret_cast<int4*>(sQ);
        for (int i = tid; i < L::QEND / 16; i += NTHR) dst[i] = src[i];
    }
    const uint32_t mb = tc::smem_u32(&mbar);
    if (tid == 0) {
        tc::mbar_init(mb, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), L::ALLOC);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t sQu = tc::smem_u32(sQ), sXu = tc::smem_u32(sX);
    const bool doM = VM != nullptr, doK = VK != nullptr, doT = VT != nullptr;
    const bool need_u = doK | doT;
    float* VMK = doM ? VM : doK ? VK - 1 : nullptr;   // interleaved M/K storage (K at odd positions)
    float* stage = reinterpret_cast<float*>(sX);   // epilogue blocks (the X tile is consumed by then)
    uint32_t phase = 0;
    bool timed_out = false;

    const int64_t ntiles = (E + TILE - 1) / TILE;
    // Inputs of the next tile are prefetched into registers while the current
    // tile's MMAs and epilogue run: connectivity and geometry before the MMA
    // issue, the gathered u values right after it.
    int pidx[NP];
    double pu[NP];   // raw FP64 values: split at formation, so the loads stay in flight
    float pgeo[1 + NS];
    bool pvalid = false;
    auto fetch_meta = [&](int64_t t) {
        const int64_t e = t * TILE + r;
        pvalid = e < E;
        if (pvalid) {
            const int* ce = conn + e * NP;
#pragma unroll
            for (int i = 0; i < NP; ++i) pidx[i] = need_u ? __ldg(ce + i) : 0;
#pragma unroll
            for (int t2 = 0; t2 <= NS; ++t2) pgeo[t2] = __ldg(geo + t2 * gs + e);
        }
    };
    auto fetch_u = [&]() {
        if (pvalid && need_u) {
#pragma unroll
            for (int i = 0; i < NP; ++i) pu[i] = __ldg(u + pidx[i]);
        }
    };
    if ((int64_t)blockIdx.x < ntiles) {
        fetch_meta(blockIdx.x);
        fetch_u();
    }
    PhaseTimer pt;
    pt.start();
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // the whole packed row is written (unrequested parts too: every
        // matrix's slices overlap its neighbours' columns); with two threads
        // per row, half by each (warp-uniform branch)
        const int64_t next = tile + gridDim.x;
        {
            float2 su[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) su[i] = pvalid && need_u ? split_f64(pu[i]) : make_float2(0.f, 0.f);
            if constexpr (L::TPR == 1) {
                float x[L::KTOTp];
#pragma unroll
                for (int i = 0; i < L::KTOTp; ++i) x[i] = 0.f;
                if (pvalid) form_x<ETy, L::KTOTp, LC>(su, pgeo, need_u, k, mass, x);
                if (next < ntiles) fetch_meta(next);
                store_row<L::KTOTp>(sX + L::XH, sX + L::XL, x, r);
            } else {
                if (half == 0)
                    form_x_half<ETy, L::KTOTp, 0, LC>(su, pgeo, pvalid, need_u, k, mass, sX + L::XH, sX + L::XL, r);
                else
                    form_x_half<ETy, L::KTOTp, 1, LC>(su, pgeo, pvalid, need_u, k, mass, sX + L::XH, sX + L::XL, r);
                if (next < ntiles) fetch_meta(next);
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        pt.mark(0);
        if (tid == 0) {
            tc::fence_after_sync();
            issue_tile<L>(tmem, sXu, sQu, doM, doK, doT);
            tc::mma_commit(mb);
        }
        pt.mark(1);
        if (next < ntiles) fetch_u();
        // one thread waits (the other warps sleep at the barrier instead of
        // spinning on the mbarrier and taking issue slots from other CTAs)
        uint32_t ok = 1;
        if (tid == 0) ok = tc::mbar_wait_bounded(mb, phase, WAIT_LIMIT);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        pt.mark(2);
        tc::fence_after_sync();
        if (half == 0) {
            const int64_t row0 = tile * TILE + warp * 32;
            // narrower TMEM loads where two threads per row leave fewer registers
            epilogue_tile<ETy, L::XEND, L::TPR == 2 ? 16 : 32>(tmem, L::COLM, L::COLK, L::COLT, stage, VMK, VT, doM,
                                                               doK, doT, row0, E, warp, lane);
        }
        tc::fence_before_sync();
        __syncthreads();
        pt.mark(3);
        pt.mark(4, 1);
    }
    if (timed_out) {
        if (tid == 0) atomicExch(err, 1);
        // give in-flight tensor-core work one more bounded chance to drain
        tc::mbar_wait_bounded(mb, phase ^ 1u, WAIT_LIMIT);
    }
    if ((tid & 31) == 0) tc::bulk_wait_all();   // V copies of this warp are complete
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, L::ALLOC);
}

// One 128-element tile of one mesh in the batched kernel: the same steps as
// one iteration of element_tc_kernel (X rows -> shared memory, MMAs, bounded
// wait, epilogue), with the mesh's parameters from the batch table.  The
// type's Q image is already resident at smem[0, QEND).
template <typename ETy>
__device__ __forceinline__ bool batch_tc_tile(const BatchMesh& bm, int64_t first, unsigned char* smem,
                                              uint32_t tmem, uint32_t mb, uint32_t& phase) {
    using L = TcL<ETy>;
    constexpr int NP = ETy::NP, NS = ETy::NS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = tid & (TILE - 1), half = tid / TILE;   // two threads per element row, as in element_tc_kernel
    unsigned char* sX = smem + L::QEND;
    const uint32_t sQu = tc::smem_u32(smem), sXu = tc::smem_u32(sX);
    const bool doM = bm.vM != nullptr, doK = bm.vK != nullptr, doT = bm.vT != nullptr;
    if (!(doM | doK | doT)) return true;   // mesh skipped in this launch (uniform over the CTA)
    const bool need_u = doK | doT;
    const int64_t E = bm.E;
    const int64_t e = first + r;
    const bool valid = e < E;
    float2 pu[NP];
    float pgeo[1 + NS];
#pragma unroll
    for (int i = 0; i < NP; ++i) pu[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t <= NS; ++t) pgeo[t] = 0.f;
    if (valid) {
        const int* ce = bm.conn + e * NP;
        if (need_u) {
#pragma unroll
            for (int i = 0; i < NP; ++i) pu[i] = split_f64(__ldg(bm.u + __ldg(ce + i)));
        }
#pragma unroll
        for (int t = 0; t <= NS; ++t) pgeo[t] = __ldg(bm.geo32 + t * E + e);
    }
    with_law(law_class(bm.k), [&](auto lcv) {
        constexpr int LC = decltype(lcv)::value;
        if (half == 0)
            form_x_half<ETy, L::KTOTp, 0, LC>(pu, pgeo, valid, need_u, bm.k, (float)bm.mass, sX + L::XH, sX + L::XL, r);
        else
            form_x_half<ETy, L::KTOTp, 1, LC>(pu, pgeo, valid, need_u, bm.k, (float)bm.mass, sX + L::XH, sX + L::XL, r);
    });
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        issue_tile<L>(tmem, sXu, sQu, doM, doK, doT);
        tc::mma_commit(mb);
    }
    uint32_t ok = 1;
    if (tid == 0) ok = tc::mbar_wait_bounded(mb, phase, WAIT_LIMIT);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) return false;
    tc::fence_after_sync();
    // the epilogue stages through the X region (the MMAs are complete)
    float* stage = reinterpret_cast<float*>(sX);
    if (half == 0) {
        const int64_t row0 = first + warp * 32;
        epilogue_tile<ETy, L::XEND, 16>(tmem, L::COLM, L::COLK, L::COLT, stage, static_cast<float*>(bm.VM),
                                        static_cast<float*>(bm.VT), doM, doK, doT, row0, E, warp, lane);
    }
    tc::fence_before_sync();
    __syncthreads();
    return true;
}

__host__ __device__ constexpr int tc_qend(int t) {
    return t == 0 ? TcL<ET<2, 1>>::QEND : t == 1 ? TcL<ET<2, 2>>::QEND : t == 2 ? TcL<ET<2, 3>>::QEND
         : t == 3 ? TcL<ET<3, 1>>::QEND : t == 4 ? TcL<ET<3, 2>>::QEND : 0;
}

// Persistent batched kernel: 256-thread CTAs (two threads per row) walk the work list
// (tiles of all meshes, grouped by element type) and reloads the resident Q
// image whenever the type changes.
__global__ void __launch_bounds__(2 * TILE, 1) batch_tc_kernel(const BatchItem* __restrict__ items, int nitems,
                                                        const BatchMesh* __restrict__ meshes,
                                                        const float* __restrict__ img_all, uint32_t talloc,
                                                        int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mb = tc::smem_u32(&mbar);
    if (tid == 0) {
        tc::mbar_init(mb, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), talloc);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    uint32_t phase = 0;
    int cur = -1;
    bool timed_out = false;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        if (w.type != cur) {
            const int4* src = reinterpret_cast<const int4*>(img_all + (size_t)w.type * IMG_SLOT_FLOATS);
            int4* dst = reinterpret_cast<int4*>(smem);
            const int n16 = tc_qend(w.type) / 16;
            for (int i = tid; i < n16; i += 2 * TILE) dst[i] = src[i];
            __syncthreads();
            cur = w.type;
        }
        const BatchMesh& bm = meshes[w.mesh];
        bool ok = true;
        switch (w.type) {
            case 0: ok = batch_tc_tile<ET<2, 1>>(bm, w.first, smem, tmem, mb, phase); break;
            case 1: ok = batch_tc_tile<ET<2, 2>>(bm, w.first, smem, tmem, mb, phase); break;
            case 2: ok = batch_tc_tile<ET<2, 3>>(bm, w.first, smem, tmem, mb, phase); break;
            case 3: ok = batch_tc_tile<ET<3, 1>>(bm, w.first, smem, tmem, mb, phase); break;
            case 4: ok = batch_tc_tile<ET<3, 2>>(bm, w.first, smem, tmem, mb, phase); break;
            default: break;
        }
        if (!ok) {   // uniform: decided by __syncthreads_or inside the tile
            timed_out = true;
            break;
        }
    }
    if (timed_out) {
        if (tid == 0) atomicExch(err, 1);
        tc::mbar_wait_bounded(mb, phase ^ 1u, WAIT_LIMIT);
    }
    if ((tid & 31) == 0) tc::bulk_wait_all();   // V copies of this warp are complete
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, talloc);
}

// ---------------------------------------------------------------------------
// Chunked tensor-core product for element types whose Q does not fit in
// shared memory (P3 tetrahedra: Q_M, Q_K and Q_T are 541 KB as TF32 hi/lo
// parts, the X rows of a 128-element tile 245 KB).  The contraction index
// K = (q, a<=b) (or (q), (q, a)) runs over quadrature points, so it is cut
// into chunks of whole quadrature points: per chunk, the CTA forms the X
// columns of those points in shared memory while one bulk copy brings the
// matching rows of Q (a precomputed operand image in global memory, resident
// in L2), then thread 0 issues the TF32x3 MMAs that accumulate into TMEM.
// M and K accumulate side by side (224 + 224 columns), are drained, then T
// (400 columns, issued as two MMAs of N = 208 and 192) reuses the columns.
template <typename ETy>
struct ChL {
    static constexpr int NQ = ETy::NQ, NS = ETy::NS, D = ETy::D;
    static constexpr int QCM = 8, QCK = 4, QCT = 8;                      // quadrature points per chunk
    static constexpr int KcM = QCM, KcK = QCK * NS, KcT = QCT * D;       // chunk widths (multiples of 8)
    static constexpr int NCM = NQ / QCM, NCK = NQ / QCK, NCT = NQ / QCT;
    // four passes, each accumulating at TMEM column 0 and drained before the
    // next: M, K, T rows [0, NTa), T rows [NTa, NTp)
    static constexpr int NSTEP = NCM + NCK + 2 * NCT;
    static constexpr int NMp = ru(ETy::NSYM, 16), NTp = ru(ETy::NT, 16);
    static constexpr int NTa = NTp > 256 ? ru(NTp / 2, 16) : NTp, NTb = NTp - NTa;
    static constexpr int NMAXp = NMp > NTa ? NMp : NTa;
    static constexpr int ALLOC = pow2_at_least(ru(NMAXp, 32));
    static constexpr int KcMax = KcK > KcT ? (KcK > KcM ? KcK : KcM) : (KcT > KcM ? KcT : KcM);
    static constexpr int XBYTES = TILE * KcMax * 8;                      // X chunk, hi + lo
    static constexpr int QB_M = NMp * KcM * 8, QB_K = NMp * KcK * 8, QB_Ta = NTa * KcT * 8, QB_Tb = NTb * KcT * 8;
    static constexpr int QBMAX = QB_K > QB_M ? (QB_K > QB_Ta ? QB_K : QB_Ta) : (QB_M > QB_Ta ? QB_M : QB_Ta);
    static constexpr int IMG_BYTES = NCM * QB_M + NCK * QB_K + NCT * (QB_Ta + QB_Tb);
    // reference tables in shared memory, read with 16-byte broadcast loads:
    // {phi_i, d phi_i / d xhat_0..2} at (q, i), then phi rows (NP floats per
    // point), then the weights
    static constexpr int NP = ETy::NP;
    static constexpr int TAB_PG = XBYTES + QBMAX, TAB_P = TAB_PG + NQ * NP * 16, TAB_W = TAB_P + NQ * NP * 4;
    static constexpr int SMEM = TAB_W + ru(NQ * 4, 16);                  // X chunk + Q chunk + tables
    // the epilogue of all eight warps stages through the X and Q chunks
    static constexpr int STAGE8_BYTES = 8 * 32 * 33 * 4;
    static constexpr bool OK = NQ % QCM == 0 && NQ % QCK == 0 && NQ % QCT == 0 && KcK % 8 == 0 && KcT % 8 == 0 &&
                               D == 3 && NP % 4 == 0 && STAGE8_BYTES <= TAB_PG &&
                               NMp <= 256 && NTa <= 256 && NTb <= 256 && NTb % 16 == 0 && NTb > 0 &&
                               QB_Tb <= QBMAX && ALLOC <= 256 && ru(ETy::NSYM, 32) <= ALLOC &&
                               ru(NTa, 32) <= ALLOC && ru(NTb, 32) <= ALLOC && XBYTES >= STAGE_FLOATS * 4 &&
                               SMEM <= SMEM_MAX;
    // step s -> (pass 0/1/2/3 = M/K/Ta/Tb, chunk index)
    __host__ __device__ static constexpr int kind(int s) {
        return s < NCM ? 0 : s < NCM + NCK ? 1 : s < NCM + NCK + NCT ? 2 : 3;
    }
    __host__ __device__ static constexpr int chunk(int s) {
        return s < NCM ? s : s < NCM + NCK ? s - NCM : s < NCM + NCK + NCT ? s - NCM - NCK : s - NCM - NCK - NCT;
    }
    __host__ __device__ static constexpr int qbytes(int s) {
        return kind(s) == 0 ? QB_M : kind(s) == 1 ? QB_K : kind(s) == 2 ? QB_Ta : QB_Tb;
    }
    __host__ __device__ static constexpr int img_off(int s) {
        return s <= NCM ? s * QB_M
             : s <= NCM + NCK ? NCM * QB_M + (s - NCM) * QB_K
             : s <= NCM + NCK + NCT ? NCM * QB_M + NCK * QB_K + (s - NCM - NCK) * QB_Ta
                                    : NCM * QB_M + NCK * QB_K + NCT * QB_Ta + (s - NCM - NCK - NCT) * QB_Tb;
    }
    __host__ __device__ static constexpr bool last_of_pass(int s) {
        return s == NCM - 1 || s == NCM + NCK - 1 || s == NCM + NCK + NCT - 1 || s == NSTEP - 1;
    }
};

constexpr int CHUNK_IMG_BYTES = ChL<ET<3, 3>>::IMG_BYTES;
__device__ __align__(128) unsigned char g_tcbig[CHUNK_IMG_BYTES];

// X columns of quadrature points q0 .. q0+QC-1 for one matrix: the same
// quantities as form_x, restricted to a chunk, in the same operations and
// order.  The reference values come from the shared-memory tables
// (ChL::TAB_*): a chunk's point index is not a compile-time constant, so
// constant-bank reads would each be a separate load, while a 16-byte shared
// load brings four values at once.
template <typename ETy, int QC>
__device__ __forceinline__ void form_chunk_m_s(int q0, float b, float mass, const float* __restrict__ tw,
                                               float (&x)[QC]) {
#pragma unroll
    for (int j = 0; j < QC; ++j) x[j] = mass * (tw[q0 + j] * b);
}

template <typename ETy, int QC, int LC = LC_ANY>
__device__ __forceinline__ void form_chunk_k_s(int q0, const float (&du)[ETy::NP], float u0, float b,
                                               const float (&A)[ETy::NS], const CoeffDev& k,
                                               const float* __restrict__ tp, const float* __restrict__ tw,
                                               float (&x)[QC * ETy::NS]) {
    constexpr int NP = ETy::NP, NS = ETy::NS;
#pragma unroll
    for (int j = 0; j < QC; ++j) {
        const int q = q0 + j;
        const float4* prow = reinterpret_cast<const float4*>(tp + q * NP);
        float uq = 0.f;
#pragma unroll
        for (int i4 = 0; i4 < NP / 4; ++i4) {
            const float4 p = prow[i4];
            uq = fmaf(p.x, du[4 * i4 + 0], uq);
            uq = fmaf(p.y, du[4 * i4 + 1], uq);
            uq = fmaf(p.z, du[4 * i4 + 2], uq);
            uq = fmaf(p.w, du[4 * i4 + 3], uq);
        }
        uq += u0;
        float dk;
        const float kq = k_eval<float, LC>(k, uq, dk);
        const float lk = (tw[q] * b) * kq;
#pragma unroll
        for (int t = 0; t < NS; ++t) x[j * NS + t] = lk * A[t];
    }
}

template <typename ETy, int QC, int LC = LC_ANY>
__device__ __forceinline__ void form_chunk_t_s(int q0, const float (&du)[ETy::NP], float u0, float b,
                                               const float (&A)[ETy::NS], const CoeffDev& k,
                                               const float4* __restrict__ tpg, const float* __restrict__ tw,
                                               float (&x)[QC * ETy::D]) {
    constexpr int NP = ETy::NP, D = ETy::D;
    static_assert(D == 3, "one 16-byte entry holds phi and a 3-component gradient");
#pragma unroll
    for (int j = 0; j < QC; ++j) {
        const int q = q0 + j;
        float uq = 0.f, g[D];
#pragma unroll
        for (int a = 0; a < D; ++a) g[a] = 0.f;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const float4 t = tpg[q * NP + i];
            uq = fmaf(t.x, du[i], uq);
            g[0] = fmaf(t.y, du[i], g[0]);
            g[1] = fmaf(t.z, du[i], g[1]);
            g[2] = fmaf(t.w, du[i], g[2]);
        }
        uq += u0;
        float dk;
        k_eval<float, LC>(k, uq, dk);
        const float ld = (tw[q] * b) * dk;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            float sacc = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const int lo = a < c ? a : c, hi = a < c ? c : a;
                sacc = fmaf(A[lo * D - (lo * (lo - 1)) / 2 + (hi - lo)], g[c], sacc);
            }
            x[j * D + a] = ld * sacc;
        }
    }
}

// Fills the chunked kernel's shared-memory tables from the constant bank
// (all threads; once per CTA, before the CTA's first barrier).
template <typename ETy>
__device__ __forceinline__ void chunk_tables_fill(unsigned char* smem) {
    using L = ChL<ETy>;
    constexpr int NP = ETy::NP, NQ = ETy::NQ, D = ETy::D;
    constexpr int TO = type_tab_off(ETy::TYPE);
    constexpr int PHI = TO, GR = TO + NQ * NP, WQ = TO + NQ * NP * (1 + D);
    float4* pg = reinterpret_cast<float4*>(smem + L::TAB_PG);
    float* p = reinterpret_cast<float*>(smem + L::TAB_P);
    float* w = reinterpret_cast<float*>(smem + L::TAB_W);
    for (int i = threadIdx.x; i < NQ * NP; i += blockDim.x) {
        pg[i] = make_float4(c_tcref[PHI + i], c_tcref[GR + i * D + 0], c_tcref[GR + i * D + 1], c_tcref[GR + i * D + 2]);
        p[i] = c_tcref[PHI + i];
    }
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) w[q] = c_tcref[WQ + q];
}

// Threads of a chunked-product CTA: two per element row.  Thread tid works
// on row tid mod 128 and forms half of each chunk's quadrature points
// (half tid / 128), so the serial formation of a chunk is split in two;
// warps 0-3 (the TMEM lane owners of the 128 rows) drain the accumulators.
constexpr int CT = 2 * TILE;

// One 128-element tile of the chunked product (all CT threads; uniform
// control).  Returns false if a bounded wait gave up; *pend_q / *pend_mma
// then tell which barrier still has an operation in flight.
template <typename ETy>
__device__ __forceinline__ bool chunked_tile(const int* __restrict__ conn, const float* __restrict__ geo, int64_t E,
                                             int64_t gs,
                                             const double* __restrict__ u, const CoeffDev& k, float mass,
                                             float* __restrict__ VM, float* __restrict__ VK, float* __restrict__ VT,
                                             const unsigned char* __restrict__ img, int64_t first,
                                             unsigned char* smem, uint32_t tmem, uint32_t mb_mma, uint32_t mb_q,
                                             uint32_t& ph_mma, uint32_t& ph_q, bool& pend_q, bool& pend_mma) {
    using L = ChL<ETy>;
    constexpr int NP = ETy::NP, NS = ETy::NS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = tid & (TILE - 1), half = tid / TILE;   // element row, half of each chunk
    const bool doM = VM != nullptr, doK = VK != nullptr, doT = VT != nullptr;
    float* VMK = doM ? VM : doK ? VK - 1 : nullptr;   // interleaved M/K storage (K at odd positions)
    const bool need_u = doK | doT;
    const int64_t e = first + r;
    PhaseTimer pt;
    pt.start();
    // element data for the whole tile: u differences (hi/lo split, as in
    // form_x) and the geometry
    float du[NP], A[NS];
    float u0 = 0.f, b = 0.f;
#pragma unroll
    for (int i = 0; i < NP; ++i) du[i] = 0.f;
#pragma unroll
    for (int t = 0; t < NS; ++t) A[t] = 0.f;
    if (e < E) {
        b = __ldg(geo + e);
#pragma unroll
        for (int t = 0; t < NS; ++t) A[t] = __ldg(geo + (int64_t)(1 + t) * gs + e);
        if (need_u) {
            const int* ce = conn + e * NP;
            const float2 p0 = split_f64_all(__ldg(u + __ldg(ce)));
            u0 = p0.x + p0.y;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const float2 pi = split_f64_all(__ldg(u + __ldg(ce + i)));
                du[i] = (pi.x - p0.x) + (pi.y - p0.y);
            }
        }
    }
    unsigned char* sX = smem;
    unsigned char* sQ = smem + L::XBYTES;
    const uint32_t sXu = tc::smem_u32(sX), sQu = tc::smem_u32(sQ);
    const float4* tpg = reinterpret_cast<const float4*>(smem + L::TAB_PG);
    const float* tp = reinterpret_cast<const float*>(smem + L::TAB_P);
    const float* tw = reinterpret_cast<const float*>(smem + L::TAB_W);
    // epilogue: warp w drains lane quadrant w mod 4, every other 32-column chunk
    const int quad = warp & 3, part = warp >> 2;
    const int64_t row0 = first + quad * 32;
    float* stage = reinterpret_cast<float*>(smem);
    pt.mark(8);
#pragma unroll 1
    for (int s = 0; s < L::NSTEP; ++s) {
        const int kd = L::kind(s), c = L::chunk(s);
        const bool active = kd == 0 ? doM : kd == 1 ? doK : doT;
        if (active) {
            const int qb = L::qbytes(s);
            if (tid == 0) {
                tc::mbar_arrive_expect_tx(mb_q, (uint32_t)qb);
                for (int o = 0; o < qb; o += 32768) {
                    const int n = qb - o < 32768 ? qb - o : 32768;
                    tc::bulk_g2s(sQu + o, img + L::img_off(s) + o, (uint32_t)n, mb_q);
                }
            }
            pend_q = true;
            // this thread's half of the chunk: quadrature points
            // c QC + half QC/2 .., i.e. columns half Kc/2 .. of the X chunk
            if (kd == 0) {
                constexpr int QH = L::QCM / 2, KH = L::KcM / 2;
                float x[KH];
                form_chunk_m_s<ETy, QH>(c * L::QCM + half * QH, b, mass, tw, x);
                store_row_part<L::KcM, KH>(sX, sX + TILE * L::KcM * 4, x, r, half * KH);
            } else if (kd == 1) {
                constexpr int QH = L::QCK / 2, KH = L::KcK / 2;
                float x[KH];
                // generic law code: the chunk loop is not unrolled, and three
                // specialised copies cost the kernel registers (it runs at 128)
                form_chunk_k_s<ETy, QH>(c * L::QCK + half * QH, du, u0, b, A, k, tp, tw, x);
                store_row_part<L::KcK, KH>(sX, sX + TILE * L::KcK * 4, x, r, half * KH);
            } else {   // both halves of T use the same X columns
                constexpr int QH = L::QCT / 2, KH = L::KcT / 2;
                float x[KH];
                form_chunk_t_s<ETy, QH>(c * L::QCT + half * QH, du, u0, b, A, k, tpg, tw, x);
                store_row_part<L::KcT, KH>(sX, sX + TILE * L::KcT * 4, x, r, half * KH);
            }
            tc::fence_proxy_async_smem();
            pt.mark(9);
            uint32_t okq = 1;
            if (tid == 0) okq = tc::mbar_wait_bounded(mb_q, ph_q, WAIT_LIMIT);
            tc::fence_before_sync();
            if (__syncthreads_or(!okq)) return false;
            pt.mark(10);
            ph_q ^= 1u;
            pend_q = false;
            if (tid == 0) {
                tc::fence_after_sync();
                // every pass accumulates at TMEM column 0
                if (kd == 0) {
                    constexpr int Kc = L::KcM;
                    issue_tf32x3<Kc>(tmem, sXu, sXu + TILE * Kc * 4, sQu, sQu + L::NMp * Kc * 4,
                                     tc::idesc_tf32(L::NMp), c > 0);
                } else if (kd == 1) {
                    constexpr int Kc = L::KcK;
                    issue_tf32x3<Kc>(tmem, sXu, sXu + TILE * Kc * 4, sQu, sQu + L::NMp * Kc * 4,
                                     tc::idesc_tf32(L::NMp), c > 0);
                } else if (kd == 2) {
                    constexpr int Kc = L::KcT;
                    issue_tf32x3<Kc>(tmem, sXu, sXu + TILE * Kc * 4, sQu, sQu + L::NTa * Kc * 4,
                                     tc::idesc_tf32(L::NTa), c > 0);
                } else {
                    constexpr int Kc = L::KcT;
                    issue_tf32x3<Kc>(tmem, sXu, sXu + TILE * Kc * 4, sQu, sQu + L::NTb * Kc * 4,
                                     tc::idesc_tf32(L::NTb), c > 0);
                }
                tc::mma_commit(mb_mma);
            }
            pt.mark(11);
            pend_mma = true;
            uint32_t okm = 1;
            if (tid == 0) okm = tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_LIMIT);
            if (__syncthreads_or(!okm)) return false;
            pt.mark(12);
            ph_mma ^= 1u;
            pend_mma = false;
            tc::fence_after_sync();
        }
        // drain the pass's accumulator once its last chunk is in (the stage
        // tiles alias the X and Q chunks, which the completed MMAs no longer
        // read and the next step's copy only overwrites after the barrier
        // below); all eight warps, two per TMEM lane quadrant
        if (active && L::last_of_pass(s)) {
            if (kd == 0)
                epilogue_staged<ETy::NSYM, 2 * ETy::NSYM, 2, true>(tmem, 0, stage, VMK, row0, E, quad, lane, 0, warp,
                                                                   part, 2);
            else if (kd == 1)
                epilogue_staged<ETy::NSYM, 2 * ETy::NSYM, 2>(tmem, 0, stage, VMK, row0, E, quad, lane, 1, warp, part,
                                                             2);
            else if (kd == 2)
                epilogue_staged<L::NTa, ETy::NT>(tmem, 0, stage, VT, row0, E, quad, lane, 0, warp, part, 2);
            else
                epilogue_staged<ETy::NT - L::NTa, ETy::NT>(tmem, 0, stage, VT, row0, E, quad, lane, L::NTa, warp, part,
                                                           2);
            tc::fence_proxy_async_smem();   // stage writes before the next bulk copy into the Q chunk
            tc::fence_before_sync();
            __syncthreads();
            pt.mark(13);
        }
    }
    pt.mark(14, 1);
    return true;
}

template <typename ETy>
__global__ void __launch_bounds__(CT, 2) element_tc_chunked_kernel(
    const int* __restrict__ conn, const float* __restrict__ geo, int64_t E, int64_t gs, const double* __restrict__ u,
    CoeffDev k, float mass, float* __restrict__ VM, float* __restrict__ VK, float* __restrict__ VT,
    const unsigned char* __restrict__ img, int* __restrict__ err) {
    using L = ChL<ETy>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_mma, bar_q;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mb_mma = tc::smem_u32(&bar_mma), mb_q = tc::smem_u32(&bar_q);
    if (tid == 0) {
        tc::mbar_init(mb_mma, 1);
        tc::mbar_init(mb_q, 1);
        tc::fence_mbar_init();
    }
    chunk_tables_fill<ETy>(smem);
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), L::ALLOC);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    uint32_t ph_mma = 0, ph_q = 0;
    bool pend_q = false, pend_mma = false, ok = true;
    const int64_t ntiles = (E + TILE - 1) / TILE;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
        ok = chunked_tile<ETy>(conn, geo, E, gs, u, k, mass, VM, VK, VT, img, tile * TILE, smem, tmem, mb_mma, mb_q,
                               ph_mma, ph_q, pend_q, pend_mma);
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // give the copy or the MMAs still in flight one more bounded chance to finish
        if (pend_q) tc::mbar_wait_bounded(mb_q, ph_q, WAIT_LIMIT);
        if (pend_mma) tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_LIMIT);
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, L::ALLOC);
}

// Batched chunked product: a persistent walk over the 128-element tiles of
// every P3-tetrahedron mesh of a batch (the same tile code as the
// single-mesh kernel, so the bits are the same).
__global__ void __launch_bounds__(CT, 2) batch_tc_chunked_kernel(const BatchItem* __restrict__ items, int nitems,
                                                                   const BatchMesh* __restrict__ meshes,
                                                                   const unsigned char* __restrict__ img,
                                                                   int* __restrict__ err) {
    using ETy = ET<3, 3>;
    using L = ChL<ETy>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_mma, bar_q;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mb_mma = tc::smem_u32(&bar_mma), mb_q = tc::smem_u32(&bar_q);
    if (tid == 0) {
        tc::mbar_init(mb_mma, 1);
        tc::mbar_init(mb_q, 1);
        tc::fence_mbar_init();
    }
    chunk_tables_fill<ETy>(smem);
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), L::ALLOC);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    uint32_t ph_mma = 0, ph_q = 0;
    bool pend_q = false, pend_mma = false, ok = true;
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchMesh& bm = meshes[w.mesh];
        if (w.type != ETy::TYPE) continue;
        float* VM = bm.vM ? static_cast<float*>(bm.VM) : nullptr;
        float* VK = bm.vK ? static_cast<float*>(bm.VK) : nullptr;
        float* VT = bm.vT ? static_cast<float*>(bm.VT) : nullptr;
        if (!(VM || VK || VT)) continue;   // mesh skipped in this launch
        ok = chunked_tile<ETy>(bm.conn, bm.geo32, bm.E, bm.E, bm.u, bm.k, (float)bm.mass, VM, VK, VT, img, w.first, smem,
                               tmem, mb_mma, mb_q, ph_mma, ph_q, pend_q, pend_mma);
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        if (pend_q) tc::mbar_wait_bounded(mb_q, ph_q, WAIT_LIMIT);
        if (pend_mma) tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_LIMIT);
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, L::ALLOC);
}

// ------------------------------------------------ u-dependent mass, TF32x3
// M(u) and the mass tensor times z = u - u^s (Sections 2, 5, 5.1) as two
// products with Q_M: the packed row [X_u | X_t] with X_u[q] = w_q b_e m(u_q)
// and X_t[q] = w_q b_e m'(u_q) z_q feeds the tile layout with the K product
// replaced by the second Q_M product and no T, so the MMA issue and the
// interleaved M/K epilogue of the tile kernel serve unchanged.
template <typename ETy>
struct MUET {
    static constexpr int D = ETy::D, P = ETy::P, NP = ETy::NP, NQ = ETy::NQ, NS = ETy::NS, NSYM = ETy::NSYM;
    static constexpr int NT = 0, KM = NQ, KK = NQ, KT = 0, TYPE = ETy::TYPE, NGEO = ETy::NGEO;
};

// its fit: the interleaved epilogue reads W columns per step (8, 16 or 32,
// as epilogue_mk_bulk chooses them), which must stay inside each product's
// columns and the allocation; both products' X columns are covered by their
// slices; X tile, then the epilogue blocks, in the X region
template <typename ETy>
struct MuL {
    using L = TcL<MUET<ETy>>;
    static constexpr int NQ = ETy::NQ, NSYM = ETy::NSYM;
    static constexpr int W = NSYM <= 8 ? 8 : NSYM <= 16 ? 16 : 32;
    static constexpr int XREG = L::XEND > TILE * 2 * NSYM * 4 ? L::XEND : TILE * 2 * NSYM * 4;
    static constexpr int SMEM = L::QEND + XREG;
    static constexpr bool FITS = L::NMp <= 256 && L::ALLOC <= 512 && SMEM <= SMEM_MAX &&
                                 L::QEND <= IMG_SLOT_FLOATS * 4 && L::COLM + ru(NSYM, W) <= L::COLK &&
                                 L::COLK + ru(NSYM, W) <= L::ALLOC && L::OFF_M == 0 && L::SM0 == 0 &&
                                 L::NSM * 8 >= NQ && L::OFF_K == NQ && L::SK0 * 8 <= NQ &&
                                 (L::SK0 + L::NSK) * 8 >= 2 * NQ && L::XEND == 2 * TILE * L::KTOTp * 4;
};

__device__ float g_tcimg_mu[6 * IMG_SLOT_FLOATS];

template <typename ETy>
__global__ void __launch_bounds__(TILE) mass_u_tc_kernel(const int* __restrict__ conn, const float* __restrict__ geo,
                                                         int64_t E, const double* __restrict__ u,
                                                         const double* __restrict__ us, CoeffDev mk,
                                                         float* __restrict__ VMK, bool doMu, bool doMt,
                                                         const float* __restrict__ img, int* __restrict__ err) {
    using L = TcL<MUET<ETy>>;
    constexpr int NP = ETy::NP, NQ = ETy::NQ, D = ETy::D;
    constexpr int TO = type_tab_off(ETy::TYPE);
    constexpr int PHI = TO, WQ = TO + NQ * NP * (1 + D);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* sQ = smem;
    unsigned char* sX = smem + L::QEND;
    {   // resident Q_M images
        const int4* src = reinterpret_cast<const int4*>(img);
        int4* dst = reinterpret_cast<int4*>(sQ);
        for (int i = tid; i < L::QEND / 16; i += TILE) dst[i] = src[i];
    }
    const uint32_t mb = tc::smem_u32(&mbar);
    if (tid == 0) {
        tc::mbar_init(mb, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), L::ALLOC);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t sQu = tc::smem_u32(sQ), sXu = tc::smem_u32(sX);
    float* stage = reinterpret_cast<float*>(sX);   // epilogue blocks (the X tile is consumed by then)
    uint32_t phase = 0;
    bool timed_out = false;
    const int64_t ntiles = (E + TILE - 1) / TILE;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e = tile * TILE + tid;
        float x[L::KTOTp];
#pragma unroll
        for (int i = 0; i < L::KTOTp; ++i) x[i] = 0.f;
        if (e < E) {
            const int* ce = conn + e * NP;
            double uv[NP];
            float du[NP], dz[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) uv[i] = __ldg(u + __ldg(ce + i));
            const float2 a = split_f64(uv[0]);
            const float u0 = a.x + a.y;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const float2 c = split_f64(uv[i]);
                du[i] = (c.x - a.x) + (c.y - a.y);
                dz[i] = doMt ? (float)(uv[i] - __ldg(us + __ldg(ce + i))) : 0.f;
            }
            const float b = __ldg(geo + e);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                float uq = 0.f, zq = 0.f;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    uq = fmaf(c_tcref[PHI + q * NP + i], du[i], uq);
                    zq = fmaf(c_tcref[PHI + q * NP + i], dz[i], zq);
                }
                uq += u0;
                float dm;
                const float mq = k_eval<float>(mk, uq, dm);
                const float lam = c_tcref[WQ + q] * b;
                x[q] = lam * mq;
                x[NQ + q] = lam * dm * zq;
            }
        }
        store_row<L::KTOTp>(sX + L::XH, sX + L::XL, x, tid);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_tile<L>(tmem, sXu, sQu, true, true, false);
            tc::mma_commit(mb);
        }
        uint32_t ok = 1;
        if (tid == 0) ok = tc::mbar_wait_bounded(mb, phase, WAIT_LIMIT);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        tc::fence_after_sync();
        const int64_t row0 = tile * TILE + warp * 32;
        epilogue_tile<MUET<ETy>, MuL<ETy>::XREG, 32>(tmem, L::COLM, L::COLK, L::COLT, stage, VMK, nullptr, doMu, doMt,
                                                     false, row0, E, warp, lane);
        tc::fence_before_sync();
        __syncthreads();
    }
    if (timed_out) {
        if (tid == 0) atomicExch(err, 1);
        tc::mbar_wait_bounded(mb, phase ^ 1u, WAIT_LIMIT);
    }
    if ((tid & 31) == 0) tc::bulk_wait_all();   // V copies of this warp are complete
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, L::ALLOC);
}

// ------------------------------------------------------ BF16 x3 / x6 tiles
// The split-precision product in BF16 (Section 4's V = X Q, as the TF32 tile
// above): X and Q are split into NPART BF16 parts (x = x0 + x1 (+ x2), each
// part the round-to-nearest BF16 of what the earlier parts leave), and
// kind::f16 MMAs accumulate the products of total part order below NPART in
// FP32 in TMEM: NPART = 2 (BF16x3) x0 q0 + x0 q1 + x1 q0, NPART = 3
// (BF16x6) adds x0 q2 + x1 q1 + x2 q0.  Same packed operand [X_M | X_K |
// X_T] in K steps of 16 (one MMA), same TMEM columns and epilogue; the core
// matrices hold 8 BF16 per 16-byte row, the byte geometry of the TF32 tile.
constexpr int BF_IMG_SLOT = 72 * 1024;   // bytes of Q parts per element type and scheme

template <typename ETy, int NPART>
struct TbL {
    static constexpr int KM = ETy::KM, KK = ETy::KK, KT = ETy::KT;
    static constexpr int KTOT = KM + KK + KT, KTOTp = ru(KTOT, 16);
    static constexpr int OFF_M = 0, OFF_K = KM, OFF_T = KM + KK;
    static constexpr int SM0 = 0, NSM = ru(KM, 16) / 16;
    static constexpr int SK0 = KM / 16, NSK = ru(KM + KK, 16) / 16 - KM / 16;
    static constexpr int ST0 = (KM + KK) / 16, NST = KTOTp / 16 - (KM + KK) / 16;
    static constexpr int NMp = ru(ETy::NSYM, 16), NTp = ru(ETy::NT, 16);
    static constexpr int COLM = 0, COLK = NMp, COLT = 2 * NMp, COLS = 2 * NMp + NTp;
    static constexpr int ALLOC = pow2_at_least(COLS);
    // Q parts: per matrix NPART images of N x (slices x 16) BF16, K-major
    static constexpr int QM_B = NMp * NSM * 32, QK_B = NMp * NSK * 32, QT_B = NTp * NST * 32;
    static constexpr int QM0 = 0, QK0 = NPART * QM_B, QT0 = QK0 + NPART * QK_B, QEND = QT0 + NPART * QT_B;
    static constexpr int XPART = TILE * KTOTp * 2;   // one BF16 part of the X tile
    static constexpr int XEND = NPART * XPART;
    static constexpr int NMK = 2 * ETy::NSYM, NMAXE = NMK > ETy::NT ? NMK : ETy::NT;
    static constexpr int XREG = XEND > TILE * NMAXE * 4 ? XEND : TILE * NMAXE * 4;   // X tile, then epilogue blocks
    static constexpr uint32_t SBO_X = (KTOTp / 8) * 128;
    static constexpr int SMEM = QEND + XREG;
    static constexpr bool FITS = NMp <= 256 && NTp <= 256 && ALLOC <= 512 && SMEM <= SMEM_MAX &&
                                 QEND <= BF_IMG_SLOT && COLM + ru(ETy::NSYM, 32) <= ALLOC &&
                                 COLK + ru(ETy::NSYM, 32) <= ALLOC && COLT + ru(ETy::NT, 32) <= ALLOC;
};

__device__ __align__(128) unsigned char g_tbimg[2 * 6 * BF_IMG_SLOT];

// one thread's X row (Kp values) as NPART BF16 parts, 8 values per 16-byte store
template <int Kp, int NPART>
__device__ __forceinline__ void store_row_bf(unsigned char* x0, const float (&x)[Kp], int r) {
    constexpr uint32_t sbo = (Kp / 8) * 128, part = TILE * Kp * 2;
    unsigned char* base = x0 + (r >> 3) * sbo + (r & 7) * 16;
#pragma unroll
    for (int c = 0; c < Kp / 8; ++c) {
        uint32_t w[NPART][4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            uint32_t pk[NPART];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float rem = x[8 * c + j + h];
#pragma unroll
                for (int q = 0; q < NPART; ++q) {
                    const __nv_bfloat16 b = __float2bfloat16_rn(rem);
                    rem = rem - __bfloat162float(b);
                    const uint32_t bits = __bfloat16_as_ushort(b);
                    pk[q] = h == 0 ? bits : (pk[q] | (bits << 16));
                }
            }
#pragma unroll
            for (int q = 0; q < NPART; ++q) w[q][j / 2] = pk[q];
        }
#pragma unroll
        for (int q = 0; q < NPART; ++q)
            *reinterpret_cast<uint4*>(base + q * part + c * 128) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

// One matrix: D (+)= sum over its `ns` K slices of the products of the
// parts of total order below NPART (X slices s0.., Q slices 0..).
template <int NS_, int NPART>
__device__ __forceinline__ void issue_bf_matrix(uint32_t tmem_d, uint32_t x0, uint32_t xpart, uint32_t sbo_x, int s0,
                                                uint32_t q0, uint32_t qpart, uint32_t idesc) {
    constexpr uint32_t sbo_q = NS_ * 256;
#pragma unroll
    for (int ks = 0; ks < NS_; ++ks) {
        const uint32_t xo = (uint32_t)(s0 + ks) * 256, qo = (uint32_t)ks * 256;
#pragma unroll
        for (int i = 0; i < NPART; ++i)
#pragma unroll
            for (int j = 0; i + j < NPART; ++j) {
                const uint64_t a = tc::smem_desc(x0 + i * xpart + xo, 128, sbo_x);
                const uint64_t b = tc::smem_desc(q0 + j * qpart + qo, 128, sbo_q);
                tc::mma_bf16(tmem_d, a, b, idesc, (ks > 0 || i > 0 || j > 0) ? 1u : 0u);
            }
    }
}

template <typename L, int NPART>
__device__ __forceinline__ void issue_tile_bf(uint32_t tmem, uint32_t sXu, uint32_t sQu, bool doM, bool doK,
                                              bool doT) {
    if (doM)
        issue_bf_matrix<L::NSM, NPART>(tmem + L::COLM, sXu, L::XPART, L::SBO_X, L::SM0, sQu + L::QM0, L::QM_B,
                                       tc::idesc_bf16(L::NMp));
    if (doK)
        issue_bf_matrix<L::NSK, NPART>(tmem + L::COLK, sXu, L::XPART, L::SBO_X, L::SK0, sQu + L::QK0, L::QK_B,
                                       tc::idesc_bf16(L::NMp));
    if (doT)
        issue_bf_matrix<L::NST, NPART>(tmem + L::COLT, sXu, L::XPART, L::SBO_X, L::ST0, sQu + L::QT0, L::QT_B,
                                       tc::idesc_bf16(L::NTp));
}

// The BF16 tile kernel: the structure of element_tc_kernel with one thread
// per element row (persistent CTAs, resident Q parts, next-tile prefetch,
// one waiting thread, bulk-copy epilogue).
template <typename ETy, int NPART, int LC>
__global__ void __launch_bounds__(TILE) element_bf_kernel(const int* __restrict__ conn, const float* __restrict__ geo,
                                                          int64_t E, int64_t gs, const double* __restrict__ u,
                                                          CoeffDev k, float mass, float* __restrict__ VM,
                                                          float* __restrict__ VK, float* __restrict__ VT,
                                                          const unsigned char* __restrict__ img,
                                                          int* __restrict__ err) {
    using L = TbL<ETy, NPART>;
    constexpr int NP = ETy::NP, NS = ETy::NS;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* sQ = smem;
    unsigned char* sX = smem + L::QEND;
    {   // resident Q parts
        const int4* src = reinterpret_cast<const int4*>(img);
        int4* dst = reinterpret_cast<int4*>(sQ);
        for (int i = tid; i < L::QEND / 16; i += TILE) dst[i] = src[i];
    }
    const uint32_t mb = tc::smem_u32(&mbar);
    if (tid == 0) {
        tc::mbar_init(mb, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_slot), L::ALLOC);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t sQu = tc::smem_u32(sQ), sXu = tc::smem_u32(sX);
    const bool doM = VM != nullptr, doK = VK != nullptr, doT = VT != nullptr;
    const bool need_u = doK | doT;
    float* VMK = doM ? VM : doK ? VK - 1 : nullptr;   // interleaved M/K storage (K at odd positions)
    float* stage = reinterpret_cast<float*>(sX);      // epilogue blocks (the X tile is consumed by then)
    uint32_t phase = 0;
    bool timed_out = false;
    const int64_t ntiles = (E + TILE - 1) / TILE;
    int pidx[NP];
    double pu[NP];
    float pgeo[1 + NS];
    bool pvalid = false;
    auto fetch_meta = [&](int64_t t) {
        const int64_t e = t * TILE + tid;
        pvalid = e < E;
        if (pvalid) {
            const int* ce = conn + e * NP;
#pragma unroll
            for (int i = 0; i < NP; ++i) pidx[i] = need_u ? __ldg(ce + i) : 0;
#pragma unroll
            for (int t2 = 0; t2 <= NS; ++t2) pgeo[t2] = __ldg(geo + t2 * gs + e);
        }
    };
    auto fetch_u = [&]() {
        if (pvalid && need_u) {
#pragma unroll
            for (int i = 0; i < NP; ++i) pu[i] = __ldg(u + pidx[i]);
        }
    };
    if ((int64_t)blockIdx.x < ntiles) {
        fetch_meta(blockIdx.x);
        fetch_u();
    }
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        float x[L::KTOTp];
#pragma unroll
        for (int i = 0; i < L::KTOTp; ++i) x[i] = 0.f;
        if (pvalid) {
            float2 su[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) su[i] = need_u ? split_f64(pu[i]) : make_float2(0.f, 0.f);
            form_x<ETy, L::KTOTp, LC>(su, pgeo, need_u, k, mass, x);
        }
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) fetch_meta(next);
        store_row_bf<L::KTOTp, NPART>(sX, x, tid);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_tile_bf<L, NPART>(tmem, sXu, sQu, doM, doK, doT);
            tc::mma_commit(mb);
        }
        if (next < ntiles) fetch_u();
        uint32_t ok = 1;
        if (tid == 0) ok = tc::mbar_wait_bounded(mb, phase, WAIT_LIMIT);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        tc::fence_after_sync();
        const int64_t row0 = tile * TILE + warp * 32;
        epilogue_tile<ETy, L::XREG>(tmem, L::COLM, L::COLK, L::COLT, stage, VMK, VT, doM, doK, doT, row0, E, warp,
                                    lane);
        tc::fence_before_sync();
        __syncthreads();
    }
    if (timed_out) {
        if (tid == 0) atomicExch(err, 1);
        tc::mbar_wait_bounded(mb, phase ^ 1u, WAIT_LIMIT);
    }
    if ((tid & 31) == 0) tc::bulk_wait_all();   // V copies of this warp are complete
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, L::ALLOC);
}

// host-side TF32 rounding, nearest with ties away from zero (matches cvt.rna)
float tf32_rna_host(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    if ((b & 0x7F800000u) != 0x7F800000u) {
        b += 0x1000u;
        b &= 0xFFFFE000u;
    }
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

// Q (K x N, FP64, row-major) -> B operand image (N x Kp, K-major core matrices), hi and lo
void put_operand(std::vector<float>& img, int off_hi, int off_lo, const double* Q, int K, int N, int Kp) {
    const int sbo = (Kp / 4) * 128;
    for (int n = 0; n < N; ++n)
        for (int kk = 0; kk < K; ++kk) {
            double v = Q[(size_t)kk * N + n];
            float hi = tf32_rna_host((float)v);
            float lo = tf32_rna_host((float)(v - (double)hi));
            int byte = (n >> 3) * sbo + (kk >> 2) * 128 + (n & 7) * 16 + (kk & 3) * 4;
            img[(off_hi + byte) / 4] = hi;
            img[(off_lo + byte) / 4] = lo;
        }
}

template <typename ETy>
void build_image(std::vector<float>& all, const RefElem& R) {
    using L = TcL<ETy>;
    std::vector<float> img(IMG_SLOT_FLOATS, 0.f);
    if constexpr (L::FITS) {
        // rows of each matrix's slices: its own Q rows at their packed
        // columns, zero rows at the neighbours' columns
        auto slices = [](const std::vector<double>& Q, int K, int N, int off, int s0, int ns) {
            std::vector<double> P((size_t)ns * 8 * N, 0.0);
            for (int kk = 0; kk < ns * 8; ++kk) {
                const int own = s0 * 8 + kk - off;
                if (own >= 0 && own < K)
                    for (int n = 0; n < N; ++n) P[(size_t)kk * N + n] = Q[(size_t)own * N + n];
            }
            return P;
        };
        const auto PM = slices(R.QM, ETy::KM, ETy::NSYM, L::OFF_M, L::SM0, L::NSM);
        const auto PK = slices(R.QK, ETy::KK, ETy::NSYM, L::OFF_K, L::SK0, L::NSK);
        const auto PT = slices(R.QT, ETy::KT, ETy::NT, L::OFF_T, L::ST0, L::NST);
        put_operand(img, L::QMh, L::QMl, PM.data(), L::NSM * 8, ETy::NSYM, L::NSM * 8);
        put_operand(img, L::QKh, L::QKl, PK.data(), L::NSK * 8, ETy::NSYM, L::NSK * 8);
        put_operand(img, L::QTh, L::QTl, PT.data(), L::NST * 8, ETy::NT, L::NST * 8);
    }
    std::copy(img.begin(), img.end(), all.begin() + (size_t)ETy::TYPE * IMG_SLOT_FLOATS);
}

// Q_M images of the u-dependent mass tile: the M product over the X_u
// columns, the second product over the X_t columns (both Q_M; zero rows
// at the neighbours' columns, as in build_image)
template <typename ETy>
void build_image_mu(std::vector<float>& all, const RefElem& R) {
    using L = TcL<MUET<ETy>>;
    std::vector<float> img(IMG_SLOT_FLOATS, 0.f);
    if constexpr (MuL<ETy>::FITS) {
        auto slices = [](const std::vector<double>& Q, int K, int N, int off, int s0, int ns) {
            std::vector<double> P((size_t)ns * 8 * N, 0.0);
            for (int kk = 0; kk < ns * 8; ++kk) {
                const int own = s0 * 8 + kk - off;
                if (own >= 0 && own < K)
                    for (int n = 0; n < N; ++n) P[(size_t)kk * N + n] = Q[(size_t)own * N + n];
            }
            return P;
        };
        const auto PU = slices(R.QM, ETy::NQ, ETy::NSYM, L::OFF_M, L::SM0, L::NSM);
        const auto PT = slices(R.QM, ETy::NQ, ETy::NSYM, L::OFF_K, L::SK0, L::NSK);
        put_operand(img, L::QMh, L::QMl, PU.data(), L::NSM * 8, ETy::NSYM, L::NSM * 8);
        put_operand(img, L::QKh, L::QKl, PT.data(), L::NSK * 8, ETy::NSYM, L::NSK * 8);
    }
    std::copy(img.begin(), img.end(), all.begin() + (size_t)ETy::TYPE * IMG_SLOT_FLOATS);
}

// host-side BF16 rounding to nearest even (matches cvt.rn.bf16.f32)
uint16_t bf16_rn_host(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    if ((b & 0x7F800000u) == 0x7F800000u) return static_cast<uint16_t>((b >> 16) | ((b & 0xFFFFu) ? 0x40u : 0u));
    b += 0x7FFFu + ((b >> 16) & 1u);
    return static_cast<uint16_t>(b >> 16);
}
float bf16_to_float_host(uint16_t h) {
    const uint32_t b = static_cast<uint32_t>(h) << 16;
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

// Q (K x N, FP64, row-major) -> NPART BF16 parts of the B operand (N x Kp,
// K-major core matrices of 8 rows x 8 values), part q at byte off + q * pstride
void put_operand_bf(std::vector<unsigned char>& img, int off, int pstride, int npart, const double* Q, int K, int N,
                    int Kp) {
    const int sbo = (Kp / 8) * 128;
    for (int n = 0; n < N; ++n)
        for (int kk = 0; kk < K; ++kk) {
            double rem = Q[(size_t)kk * N + n];
            const int byte = (n >> 3) * sbo + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2;
            for (int q = 0; q < npart; ++q) {
                const uint16_t h = bf16_rn_host(static_cast<float>(rem));
                rem -= static_cast<double>(bf16_to_float_host(h));
                std::memcpy(&img[(size_t)off + (size_t)q * pstride + byte], &h, 2);
            }
        }
}

template <typename ETy, int NPART>
void build_image_bf(std::vector<unsigned char>& all, const RefElem& R) {
    using L = TbL<ETy, NPART>;
    std::vector<unsigned char> img(BF_IMG_SLOT, 0);
    if constexpr (L::FITS) {
        // each matrix's slices: its own Q rows at their packed columns, zero
        // rows at the neighbours' columns (as in build_image)
        auto slices = [](const std::vector<double>& Q, int K, int N, int off, int s0, int ns) {
            std::vector<double> P((size_t)ns * 16 * N, 0.0);
            for (int kk = 0; kk < ns * 16; ++kk) {
                const int own = s0 * 16 + kk - off;
                if (own >= 0 && own < K)
                    for (int n = 0; n < N; ++n) P[(size_t)kk * N + n] = Q[(size_t)own * N + n];
            }
            return P;
        };
        const auto PM = slices(R.QM, ETy::KM, ETy::NSYM, L::OFF_M, L::SM0, L::NSM);
        const auto PK = slices(R.QK, ETy::KK, ETy::NSYM, L::OFF_K, L::SK0, L::NSK);
        const auto PT = slices(R.QT, ETy::KT, ETy::NT, L::OFF_T, L::ST0, L::NST);
        put_operand_bf(img, L::QM0, L::QM_B, NPART, PM.data(), L::NSM * 16, ETy::NSYM, L::NSM * 16);
        put_operand_bf(img, L::QK0, L::QK_B, NPART, PK.data(), L::NSK * 16, ETy::NSYM, L::NSK * 16);
        put_operand_bf(img, L::QT0, L::QT_B, NPART, PT.data(), L::NST * 16, ETy::NT, L::NST * 16);
    }
    const size_t slot = (size_t)(NPART - 2) * 6 + ETy::TYPE;
    std::copy(img.begin(), img.end(), all.begin() + slot * BF_IMG_SLOT);
}

// Operand images of the Q chunks of the chunked product, step after step:
// rows k0 .. k0+Kc of Q (K x N, row-major) as an N x Kc K-major operand,
// hi part then lo part, N padded with zero rows.
template <typename ETy>
void build_chunk_image(std::vector<float>& img, const RefElem& R) {
    using L = ChL<ETy>;
    img.assign(L::IMG_BYTES / 4, 0.f);
    for (int st = 0; st < L::NSTEP; ++st) {
        const int kd = L::kind(st), c = L::chunk(st);
        const int Kc = kd == 0 ? L::KcM : kd == 1 ? L::KcK : L::KcT;
        const int N = kd >= 2 ? ETy::NT : ETy::NSYM;
        // the pass's output columns [n0, n0 + nw) and their padded row count
        const int n0 = kd == 3 ? L::NTa : 0;
        const int nw = kd == 2 ? std::min(L::NTa, N) : kd == 3 ? N - L::NTa : N;
        const int Np = kd == 2 ? L::NTa : kd == 3 ? L::NTb : L::NMp;
        const std::vector<double>& Q = kd == 0 ? R.QM : kd == 1 ? R.QK : R.QT;
        std::vector<double> sub((size_t)Kc * nw);
        for (int kk = 0; kk < Kc; ++kk)
            for (int n = 0; n < nw; ++n) sub[(size_t)kk * nw + n] = Q[((size_t)c * Kc + kk) * N + n0 + n];
        const int off = L::img_off(st);
        put_operand(img, off, off + Np * Kc * 4, sub.data(), Kc, nw, Kc);
    }
}

std::mutex g_mu;
bool g_done[64] = {};
std::atomic<bool> g_ready[64];   // lock-free fast path of tables_init_tc

// Launch shape of a tensor-core kernel on one device: computed (and the
// kernel's shared-memory attributes set) on first use, then cached.
struct LaunchShape {
    int nsm = 0, smem = 0, occ = 0;
    const void* img = nullptr;
    int* err = nullptr;
};

template <typename F>
int cached_shape(std::atomic<int>* have, LaunchShape* cache, std::mutex& mu, F compute, LaunchShape& out) {
    int dev = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    const bool slot = dev >= 0 && dev < 64;
    if (slot && have[dev].load(std::memory_order_acquire)) {
        out = cache[dev];
        return FEM_OK;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (slot && have[dev].load(std::memory_order_relaxed)) {
        out = cache[dev];
        return FEM_OK;
    }
    LaunchShape sh;
    const int rc = compute(dev, sh);
    if (rc) return rc;
    if (slot) {
        cache[dev] = sh;
        have[dev].store(1, std::memory_order_release);
    }
    out = sh;
    return FEM_OK;
}

template <typename ETy>
int launch_tc_chunked(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                      cudaStream_t s, int64_t e0, int64_t e1) {
    using L = ChL<ETy>;
    const int64_t E = e1 - e0;
    if (E <= 0) return FEM_OK;
    auto kern = element_tc_chunked_kernel<ETy>;
    static std::atomic<int> have[64];
    static LaunchShape cache[64];
    static std::mutex mu;
    LaunchShape sh;
    int rc = cached_shape(have, cache, mu, [&](int dev, LaunchShape& o) -> int {
        int optin = 0, per_sm = 0, occ = 0;
        FEM_CUDA_TRY(cudaDeviceGetAttribute(&o.nsm, cudaDevAttrMultiProcessorCount, dev));
        FEM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        FEM_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        cudaFuncAttributes fa;
        FEM_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
        const int dyn_max = optin - (int)fa.sharedSizeBytes;
        // at most 512 / ALLOC CTAs per SM (each holds ALLOC TMEM columns):
        // ask for enough shared memory that no more fit
        const int cmax = 512 / L::ALLOC;
        o.smem = std::min(dyn_max, std::max(L::SMEM, per_sm / (cmax + 1) + 1));
        if (o.smem < L::SMEM) return fail(FEM_EINVAL, "chunked tensor-core tile does not fit in shared memory");
        FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, o.smem));
        FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
        FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, CT, o.smem));
        if (occ > cmax) return fail(FEM_ECUDA, "cannot bound CTAs per SM for tensor memory");
        o.occ = std::max(1, std::min(cmax, ctas_per_sm(fa, CT, o.smem, dev)));
        void* img = nullptr;
        FEM_CUDA_TRY(cudaGetSymbolAddress(&img, g_tcbig));
        o.img = img;
        FEM_CUDA_TRY(cudaGetSymbolAddress((void**)&o.err, g_tc_err));
        return FEM_OK;
    }, sh);
    if (rc) return rc;
    const int64_t ntiles = (E + TILE - 1) / TILE;
    int64_t grid = (int64_t)sh.nsm * sh.occ;
    if (grid > ntiles) grid = ntiles;
    trace_launch("element_tc_chunked_kernel", grid, CT, sh.smem, sh.occ);
    cudaGetLastError();   // clear any stale error before the launch check
    kern<<<(unsigned)grid, CT, sh.smem, s>>>(m.conn.as<int>() + e0 * ETy::NP, m.geo32.as<float>() + e0, E, m.E, u, k,
                                               (float)m.m, VM ? VM + 2 * e0 * ETy::NSYM : nullptr,
                                               VK ? VK + 2 * e0 * ETy::NSYM : nullptr, VT ? VT + e0 * ETy::NT : nullptr,
                                               static_cast<const unsigned char*>(sh.img), sh.err);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

template <typename ETy, int LC>
int launch_tc(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
              cudaStream_t s, int64_t e0, int64_t e1) {
    using L = TcL<ETy>;
    if constexpr (!L::FITS) {
        if constexpr (ChL<ETy>::OK && ChL<ETy>::IMG_BYTES == CHUNK_IMG_BYTES)
            return launch_tc_chunked<ETy>(m, k, u, VM, VK, VT, s, e0, e1);
        else
            return fail(FEM_EINVAL, "FEM_TF32X3 is not available for this element type (tile does not fit)");
    } else {
        const int64_t E = e1 - e0;
        if (E <= 0) return FEM_OK;
        auto kern = element_tc_kernel<ETy, LC>;
        constexpr int SMEM0 = L::SMEM;
        constexpr int ALLOC0 = L::ALLOC;
        static std::atomic<int> have[64];
        static LaunchShape cache[64];
        static std::mutex mu;
        LaunchShape sh;
        int rc = cached_shape(have, cache, mu, [&](int dev, LaunchShape& o) -> int {
            int optin = 0, occ = 0;
            FEM_CUDA_TRY(cudaDeviceGetAttribute(&o.nsm, cudaDevAttrMultiProcessorCount, dev));
            FEM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            cudaFuncAttributes fa;
            FEM_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
            const int dyn_max = optin - (int)fa.sharedSizeBytes;   // static shared memory counts against the limit
            int smem = SMEM0;
            if (smem > dyn_max) return fail(FEM_EINVAL, "tensor-core tile does not fit in shared memory");
            FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            // the whole unified L1/shared array as shared memory, so that
            // several CTAs (each with its own TMEM columns) overlap their load,
            // MMA and epilogue phases on one SM
            FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared));
            FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, L::TPR * TILE, smem));
            const int occ_max = 512 / ALLOC0;   // co-resident CTAs must fit their TMEM columns
            if (occ > occ_max) {
                // ask for enough shared memory that at most occ_max CTAs fit on an SM
                int per_sm = 0;
                FEM_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
                smem = per_sm / (occ_max + 1) + 1;
                if (smem > dyn_max) smem = dyn_max;
                FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, L::TPR * TILE, smem));
                if (occ > occ_max) return fail(FEM_ECUDA, "cannot bound CTAs per SM for tensor memory");
            }
            if (occ < 1) return fail(FEM_ECUDA, "tensor-core kernel does not fit on an SM");
            // the occupancy query can under-report with the carveout
            // preference; the register / shared-memory budget (bounded by
            // TMEM) decides, and a persistent grid larger than what is
            // co-resident stays correct
            o.occ = std::max(occ, std::min(occ_max, ctas_per_sm(fa, L::TPR * TILE, smem, dev)));
            o.smem = smem;
            void* img = nullptr;
            FEM_CUDA_TRY(cudaGetSymbolAddress(&img, g_tcimg));
            o.img = static_cast<const float*>(img) + (size_t)ETy::TYPE * IMG_SLOT_FLOATS;
            FEM_CUDA_TRY(cudaGetSymbolAddress((void**)&o.err, g_tc_err));
            return FEM_OK;
        }, sh);
        if (rc) return rc;
        const int64_t ntiles = (E + TILE - 1) / TILE;
        int64_t grid = (int64_t)sh.nsm * sh.occ;
        if (grid > ntiles) grid = ntiles;
        trace_launch("element_tc_kernel", grid, L::TPR * TILE, sh.smem, sh.occ);
        cudaGetLastError();   // clear any stale error before the launch check
        kern<<<(unsigned)grid, L::TPR * TILE, sh.smem, s>>>(m.conn.as<int>() + e0 * ETy::NP, m.geo32.as<float>() + e0, E, m.E, u,
                                                   k, (float)m.m, VM ? VM + 2 * e0 * ETy::NSYM : nullptr,
                                                   VK ? VK + 2 * e0 * ETy::NSYM : nullptr,
                                                   VT ? VT + e0 * ETy::NT : nullptr, static_cast<const float*>(sh.img),
                                                   sh.err);
        FEM_CUDA_TRY(cudaGetLastError());
        return FEM_OK;
    }
}

// The tile kernel compiled for k's law class (one formation copy per kernel;
// every class gives the same bits).
template <typename ETy>
int launch_tc_law(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                  cudaStream_t s, int64_t e0, int64_t e1) {
    if constexpr (!TcL<ETy>::FITS) {
        return launch_tc<ETy, LC_ANY>(m, k, u, VM, VK, VT, s, e0, e1);
    } else {
        switch (law_class(k)) {
            case LC_POLY3: return launch_tc<ETy, LC_POLY3>(m, k, u, VM, VK, VT, s, e0, e1);
            case LC_SIN: return launch_tc<ETy, LC_SIN>(m, k, u, VM, VK, VT, s, e0, e1);
            default: return launch_tc<ETy, LC_ANY>(m, k, u, VM, VK, VT, s, e0, e1);
        }
    }
}

}  // namespace

int tables_init_tc() {
    int dev = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && g_ready[dev].load(std::memory_order_acquire)) return FEM_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 64 && g_done[dev]) return FEM_OK;
    std::vector<float> ref(TAB_TOTAL, 0.f), img((size_t)6 * IMG_SLOT_FLOATS, 0.f);
    for (int t = 0; t < 6; ++t) {
        const RefElem* R = refelem_for_type(t);
        if (!R) return fail(FEM_EINVAL, "reference element tables failed");
        int o = type_tab_off(t);
        for (int i = 0; i < R->nq * R->np; ++i) ref[o + i] = (float)R->phi[i];
        for (int i = 0; i < R->nq * R->np * R->d; ++i) ref[o + R->nq * R->np + i] = (float)R->grad[i];
        for (int i = 0; i < R->nq; ++i) ref[o + R->nq * R->np * (1 + R->d) + i] = (float)R->wq[i];
        switch (t) {
            case 0: build_image<ET<2, 1>>(img, *R); break;
            case 1: build_image<ET<2, 2>>(img, *R); break;
            case 2: build_image<ET<2, 3>>(img, *R); break;
            case 3: build_image<ET<3, 1>>(img, *R); break;
            case 4: build_image<ET<3, 2>>(img, *R); break;
            case 5: build_image<ET<3, 3>>(img, *R); break;
        }
    }
    FEM_CUDA_TRY(cudaMemcpyToSymbol(c_tcref, ref.data(), sizeof(float) * TAB_TOTAL));
    FEM_CUDA_TRY(cudaMemcpyToSymbol(g_tcimg, img.data(), sizeof(float) * img.size()));
    {
        std::vector<float> mimg((size_t)6 * IMG_SLOT_FLOATS, 0.f);
        for (int t = 0; t < 5; ++t) {
            const RefElem* R = refelem_for_type(t);
            switch (t) {
                case 0: build_image_mu<ET<2, 1>>(mimg, *R); break;
                case 1: build_image_mu<ET<2, 2>>(mimg, *R); break;
                case 2: build_image_mu<ET<2, 3>>(mimg, *R); break;
                case 3: build_image_mu<ET<3, 1>>(mimg, *R); break;
                case 4: build_image_mu<ET<3, 2>>(mimg, *R); break;
            }
        }
        FEM_CUDA_TRY(cudaMemcpyToSymbol(g_tcimg_mu, mimg.data(), sizeof(float) * mimg.size()));
    }
    {
        std::vector<unsigned char> bimg((size_t)2 * 6 * BF_IMG_SLOT, 0);
        for (int t = 0; t < 6; ++t) {
            const RefElem* R = refelem_for_type(t);
            switch (t) {
                case 0: build_image_bf<ET<2, 1>, 2>(bimg, *R); build_image_bf<ET<2, 1>, 3>(bimg, *R); break;
                case 1: build_image_bf<ET<2, 2>, 2>(bimg, *R); build_image_bf<ET<2, 2>, 3>(bimg, *R); break;
                case 2: build_image_bf<ET<2, 3>, 2>(bimg, *R); build_image_bf<ET<2, 3>, 3>(bimg, *R); break;
                case 3: build_image_bf<ET<3, 1>, 2>(bimg, *R); build_image_bf<ET<3, 1>, 3>(bimg, *R); break;
                case 4: build_image_bf<ET<3, 2>, 2>(bimg, *R); build_image_bf<ET<3, 2>, 3>(bimg, *R); break;
                case 5: build_image_bf<ET<3, 3>, 2>(bimg, *R); build_image_bf<ET<3, 3>, 3>(bimg, *R); break;
            }
        }
        FEM_CUDA_TRY(cudaMemcpyToSymbol(g_tbimg, bimg.data(), bimg.size()));
    }
    {
        std::vector<float> big;
        const RefElem* R5 = refelem_for_type(5);
        if (!R5) return fail(FEM_EINVAL, "reference element tables failed");
        build_chunk_image<ET<3, 3>>(big, *R5);
        FEM_CUDA_TRY(cudaMemcpyToSymbol(g_tcbig, big.data(), sizeof(float) * big.size()));
    }
    int zero = 0;
    FEM_CUDA_TRY(cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(int)));
    if (dev >= 0 && dev < 64) {
        g_done[dev] = true;
        g_ready[dev].store(true, std::memory_order_release);
    }
    return FEM_OK;
}

int tc_type_supported(int type) {
    switch (type) {
        case 0: return TcL<ET<2, 1>>::FITS;
        case 1: return TcL<ET<2, 2>>::FITS;
        case 2: return TcL<ET<2, 3>>::FITS;
        case 3: return TcL<ET<3, 1>>::FITS;
        case 4: return TcL<ET<3, 2>>::FITS;
        case 5: return TcL<ET<3, 3>>::FITS;
    }
    return 0;
}
int tc_type_smem(int type) {
    switch (type) {
        case 0: return TcL<ET<2, 1>>::SMEM;
        case 1: return TcL<ET<2, 2>>::SMEM;
        case 2: return TcL<ET<2, 3>>::SMEM;
        case 3: return TcL<ET<3, 1>>::SMEM;
        case 4: return TcL<ET<3, 2>>::SMEM;
    }
    return 0;
}
int tc_type_alloc(int type) {
    switch (type) {
        case 0: return TcL<ET<2, 1>>::ALLOC;
        case 1: return TcL<ET<2, 2>>::ALLOC;
        case 2: return TcL<ET<2, 3>>::ALLOC;
        case 3: return TcL<ET<3, 1>>::ALLOC;
        case 4: return TcL<ET<3, 2>>::ALLOC;
    }
    return 0;
}

int batch_tc_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, int talloc, int smem, int grid,
                    cudaStream_t s) {
    if (nitems <= 0) return FEM_OK;
    int rc = tables_init_tc();
    if (rc) return rc;
    if (talloc < 32 || talloc > 512 || (talloc & (talloc - 1))) return fail(FEM_EINVAL, "bad TMEM allocation");
    auto kern = batch_tc_kernel;
    int dev = 0, optin = 0, occ = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    FEM_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    if (smem > optin - (int)fa.sharedSizeBytes) return fail(FEM_EINVAL, "batched tile does not fit in shared memory");
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 2 * TILE, smem));
    if (occ < 1) return fail(FEM_ECUDA, "batched tensor-core kernel does not fit on an SM");
    // co-resident CTAs must fit their TMEM columns: ask for enough shared
    // memory that at most 512 / talloc CTAs fit on an SM
    const int occ_max = 512 / talloc;
    if (occ > occ_max) {
        int per_sm = 0;
        FEM_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        smem = std::min(per_sm / (occ_max + 1) + 1, optin - (int)fa.sharedSizeBytes);
        FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 2 * TILE, smem));
        if (occ > occ_max) return fail(FEM_ECUDA, "cannot bound CTAs per SM for tensor memory");
    }
    occ = std::max(occ, std::min(occ_max, ctas_per_sm(fa, 2 * TILE, smem, dev)));
    grid *= occ;
    float* img = nullptr;
    int* err = nullptr;
    FEM_CUDA_TRY(cudaGetSymbolAddress((void**)&img, g_tcimg));
    FEM_CUDA_TRY(cudaGetSymbolAddress((void**)&err, g_tc_err));
    if (grid > nitems) grid = nitems;
    trace_launch("batch_tc_kernel", grid, 2 * TILE, smem, occ);
    cudaGetLastError();   // clear any stale error before the launch check
    kern<<<grid, 2 * TILE, smem, s>>>(items, nitems, meshes, img, (uint32_t)talloc, err);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

int batch_tc_chunked_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, cudaStream_t s) {
    if (nitems <= 0) return FEM_OK;
    int rc = tables_init_tc();
    if (rc) return rc;
    using L = ChL<ET<3, 3>>;
    auto kern = batch_tc_chunked_kernel;
    int dev = 0, nsm = 0, optin = 0, per_sm = 0, occ = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    cudaFuncAttributes fa;
    FEM_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    const int cmax = 512 / L::ALLOC;
    const int smem = std::min(optin - (int)fa.sharedSizeBytes, std::max(L::SMEM, per_sm / (cmax + 1) + 1));
    if (smem < L::SMEM) return fail(FEM_EINVAL, "chunked tensor-core tile does not fit in shared memory");
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, CT, smem));
    if (occ > cmax) return fail(FEM_ECUDA, "cannot bound CTAs per SM for tensor memory");
    const int per = std::max(1, std::min(cmax, ctas_per_sm(fa, CT, smem, dev)));
    const int grid = nitems < nsm * per ? nitems : nsm * per;
    unsigned char* img = nullptr;
    int* err = nullptr;
    FEM_CUDA_TRY(cudaGetSymbolAddress((void**)&img, g_tcbig));
    FEM_CUDA_TRY(cudaGetSymbolAddress((void**)&err, g_tc_err));
    trace_launch("batch_tc_chunked_kernel", grid, CT, smem, per);
    cudaGetLastError();   // clear any stale error before the launch check
    kern<<<grid, CT, smem, s>>>(items, nitems, meshes, img, err);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

int tc_chunked_supported(int type) { return type == 5 && ChL<ET<3, 3>>::OK; }

#ifdef FEM_PHASE_TIMERS
// Reads (and optionally clears) the 16 phase counters of a timer build.
extern "C" int fem_debug_phase_cycles(unsigned long long* out, int clear) {
    if (cudaMemcpyFromSymbol(out, g_phase, sizeof(unsigned long long) * 16) != cudaSuccess) return FEM_ECUDA;
    if (clear) {
        unsigned long long z[16] = {};
        if (cudaMemcpyToSymbol(g_phase, z, sizeof z) != cudaSuccess) return FEM_ECUDA;
    }
    return FEM_OK;
}
#endif

int tc_error_flag(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_err, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        int zero = 0;
        cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(int));
    }
    return v;
}

template <typename ETy, int NPART, int LC>
int launch_bf(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT, cudaStream_t s,
              int64_t e0, int64_t e1) {
    using L = TbL<ETy, NPART>;
    if constexpr (!L::FITS) {
        return fail(FEM_EINVAL, "FEM_BF16X3 / FEM_BF16X6 are not available for this element type (tile does not fit)");
    } else {
        const int64_t E = e1 - e0;
        if (E <= 0) return FEM_OK;
        auto kern = element_bf_kernel<ETy, NPART, LC>;
        static std::atomic<int> have[64];
        static LaunchShape cache[64];
        static std::mutex mu;
        LaunchShape sh;
        int rc = cached_shape(have, cache, mu, [&](int dev, LaunchShape& o) -> int {
            int optin = 0, occ = 0;
            FEM_CUDA_TRY(cudaDeviceGetAttribute(&o.nsm, cudaDevAttrMultiProcessorCount, dev));
            FEM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            cudaFuncAttributes fa;
            FEM_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
            const int dyn_max = optin - (int)fa.sharedSizeBytes;
            int smem = L::SMEM;
            if (smem > dyn_max) return fail(FEM_EINVAL, "BF16 tensor-core tile does not fit in shared memory");
            FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared));
            FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TILE, smem));
            const int occ_max = 512 / L::ALLOC;   // co-resident CTAs must fit their TMEM columns
            if (occ > occ_max) {
                int per_sm = 0;
                FEM_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
                smem = per_sm / (occ_max + 1) + 1;
                if (smem > dyn_max) smem = dyn_max;
                FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TILE, smem));
                if (occ > occ_max) return fail(FEM_ECUDA, "cannot bound CTAs per SM for tensor memory");
            }
            if (occ < 1) return fail(FEM_ECUDA, "BF16 tensor-core kernel does not fit on an SM");
            o.occ = std::max(occ, std::min(occ_max, ctas_per_sm(fa, TILE, smem, dev)));
            o.smem = smem;
            void* img = nullptr;
            FEM_CUDA_TRY(cudaGetSymbolAddress(&img, g_tbimg));
            o.img = static_cast<const unsigned char*>(img) + ((size_t)(NPART - 2) * 6 + ETy::TYPE) * BF_IMG_SLOT;
            FEM_CUDA_TRY(cudaGetSymbolAddress((void**)&o.err, g_tc_err));
            return FEM_OK;
        }, sh);
        if (rc) return rc;
        const int64_t ntiles = (E + TILE - 1) / TILE;
        int64_t grid = (int64_t)sh.nsm * sh.occ;
        if (grid > ntiles) grid = ntiles;
        trace_launch("element_bf_kernel", grid, TILE, sh.smem, sh.occ);
        cudaGetLastError();   // clear any stale error before the launch check
        kern<<<(unsigned)grid, TILE, sh.smem, s>>>(m.conn.as<int>() + e0 * ETy::NP, m.geo32.as<float>() + e0, E, m.E, u,
                                                   k, (float)m.m, VM ? VM + 2 * e0 * ETy::NSYM : nullptr,
                                                   VK ? VK + 2 * e0 * ETy::NSYM : nullptr,
                                                   VT ? VT + e0 * ETy::NT : nullptr,
                                                   static_cast<const unsigned char*>(sh.img), sh.err);
        FEM_CUDA_TRY(cudaGetLastError());
        return FEM_OK;
    }
}

template <typename ETy, int NPART>
int launch_bf_law(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                  cudaStream_t s, int64_t e0, int64_t e1) {
    if constexpr (!TbL<ETy, NPART>::FITS) {
        return launch_bf<ETy, NPART, LC_ANY>(m, k, u, VM, VK, VT, s, e0, e1);
    } else {
        switch (law_class(k)) {
            case LC_POLY3: return launch_bf<ETy, NPART, LC_POLY3>(m, k, u, VM, VK, VT, s, e0, e1);
            case LC_SIN: return launch_bf<ETy, NPART, LC_SIN>(m, k, u, VM, VK, VT, s, e0, e1);
            default: return launch_bf<ETy, NPART, LC_ANY>(m, k, u, VM, VK, VT, s, e0, e1);
        }
    }
}

template <int NPART>
int dispatch_bf(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                cudaStream_t s, int64_t e0, int64_t e1) {
    switch (m.type) {
        case 0: return launch_bf_law<ET<2, 1>, NPART>(m, k, u, VM, VK, VT, s, e0, e1);
        case 1: return launch_bf_law<ET<2, 2>, NPART>(m, k, u, VM, VK, VT, s, e0, e1);
        case 2: return launch_bf_law<ET<2, 3>, NPART>(m, k, u, VM, VK, VT, s, e0, e1);
        case 3: return launch_bf_law<ET<3, 1>, NPART>(m, k, u, VM, VK, VT, s, e0, e1);
        case 4: return launch_bf_law<ET<3, 2>, NPART>(m, k, u, VM, VK, VT, s, e0, e1);
        case 5: return launch_bf_law<ET<3, 3>, NPART>(m, k, u, VM, VK, VT, s, e0, e1);
    }
    return fail(FEM_EINVAL, "element type");
}

template <typename ETy>
int launch_mu(const fem_mesh& m, const CoeffDev& mk, const double* u, const double* us, float* VMK, bool doMu,
              bool doMt, cudaStream_t s) {
    using L = TcL<MUET<ETy>>;
    if constexpr (!MuL<ETy>::FITS) {
        return fail(FEM_EINVAL, "the TF32x3 u-dependent mass is not available for this element type");
    } else {
        const int64_t E = m.E;
        if (E <= 0) return FEM_OK;
        auto kern = mass_u_tc_kernel<ETy>;
        static std::atomic<int> have[64];
        static LaunchShape cache[64];
        static std::mutex mu;
        LaunchShape sh;
        int rc = cached_shape(have, cache, mu, [&](int dev, LaunchShape& o) -> int {
            int optin = 0, occ = 0;
            FEM_CUDA_TRY(cudaDeviceGetAttribute(&o.nsm, cudaDevAttrMultiProcessorCount, dev));
            FEM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            cudaFuncAttributes fa;
            FEM_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
            const int dyn_max = optin - (int)fa.sharedSizeBytes;
            int smem = MuL<ETy>::SMEM;
            if (smem > dyn_max) return fail(FEM_EINVAL, "u-dependent mass tile does not fit in shared memory");
            FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared));
            FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TILE, smem));
            const int occ_max = 512 / L::ALLOC;   // co-resident CTAs must fit their TMEM columns
            if (occ > occ_max) {
                int per_sm = 0;
                FEM_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
                smem = per_sm / (occ_max + 1) + 1;
                if (smem > dyn_max) smem = dyn_max;
                FEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TILE, smem));
                if (occ > occ_max) return fail(FEM_ECUDA, "cannot bound CTAs per SM for tensor memory");
            }
            if (occ < 1) return fail(FEM_ECUDA, "u-dependent mass tile does not fit on an SM");
            o.occ = std::max(occ, std::min(occ_max, ctas_per_sm(fa, TILE, smem, dev)));
            o.smem = smem;
            void* img = nullptr;
            FEM_CUDA_TRY(cudaGetSymbolAddress(&img, g_tcimg_mu));
            o.img = static_cast<const float*>(img) + (size_t)ETy::TYPE * IMG_SLOT_FLOATS;
            FEM_CUDA_TRY(cudaGetSymbolAddress((void**)&o.err, g_tc_err));
            return FEM_OK;
        }, sh);
        if (rc) return rc;
        const int64_t ntiles = (E + TILE - 1) / TILE;
        int64_t grid = (int64_t)sh.nsm * sh.occ;
        if (grid > ntiles) grid = ntiles;
        trace_launch("mass_u_tc_kernel", grid, TILE, sh.smem, sh.occ);
        cudaGetLastError();   // clear any stale error before the launch check
        kern<<<(unsigned)grid, TILE, sh.smem, s>>>(m.conn.as<int>(), m.geo32.as<float>(), E, u, us, mk, VMK, doMu,
                                                    doMt, static_cast<const float*>(sh.img), sh.err);
        FEM_CUDA_TRY(cudaGetLastError());
        return FEM_OK;
    }
}

int element_mass_u_tc(const fem_mesh& m, const CoeffDev& mk, const double* u, const double* us, float* VMK, bool doMu,
                      bool doMt, cudaStream_t s) {
    int rc = tables_init_tc();
    if (rc) return rc;
    switch (m.type) {
        case 0: return launch_mu<ET<2, 1>>(m, mk, u, us, VMK, doMu, doMt, s);
        case 1: return launch_mu<ET<2, 2>>(m, mk, u, us, VMK, doMu, doMt, s);
        case 2: return launch_mu<ET<2, 3>>(m, mk, u, us, VMK, doMu, doMt, s);
        case 3: return launch_mu<ET<3, 1>>(m, mk, u, us, VMK, doMu, doMt, s);
        case 4: return launch_mu<ET<3, 2>>(m, mk, u, us, VMK, doMu, doMt, s);
    }
    return fail(FEM_EINVAL, "the TF32x3 u-dependent mass is not available for P3 tetrahedra");
}

int element_tc_bf16(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                    int nparts, cudaStream_t s, int64_t e0, int64_t e1) {
    if (e1 < 0) e1 = m.E;
    if (e0 < 0 || e0 > e1 || e1 > m.E) return fail(FEM_EINVAL, "element range out of bounds");
    int rc = tables_init_tc();
    if (rc) return rc;
    if (nparts == 2) return dispatch_bf<2>(m, k, u, VM, VK, VT, s, e0, e1);
    if (nparts == 3) return dispatch_bf<3>(m, k, u, VM, VK, VT, s, e0, e1);
    return fail(FEM_EINVAL, "BF16 split into 2 or 3 parts");
}

int element_tc_tf32x3(const fem_mesh& m, const CoeffDev& k, const double* u, float* VM, float* VK, float* VT,
                      cudaStream_t s, int64_t e0, int64_t e1) {
    if (e1 < 0) e1 = m.E;
    if (e0 < 0 || e0 > e1 || e1 > m.E) return fail(FEM_EINVAL, "element range out of bounds");
    int rc = tables_init_tc();
    if (rc) return rc;
    switch (m.type) {
        case 0: return launch_tc_law<ET<2, 1>>(m, k, u, VM, VK, VT, s, e0, e1);
        case 1: return launch_tc_law<ET<2, 2>>(m, k, u, VM, VK, VT, s, e0, e1);
        case 2: return launch_tc_law<ET<2, 3>>(m, k, u, VM, VK, VT, s, e0, e1);
        case 3: return launch_tc_law<ET<3, 1>>(m, k, u, VM, VK, VT, s, e0, e1);
        case 4: return launch_tc_law<ET<3, 2>>(m, k, u, VM, VK, VT, s, e0, e1);
        case 5: return launch_tc_law<ET<3, 3>>(m, k, u, VM, VK, VT, s, e0, e1);
    }
    return fail(FEM_EINVAL, "element type");
}

}  // namespace fem
