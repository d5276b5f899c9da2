// scatter.cu -- global assembly of the element matrices into CSR values.
//
// The last step of Algorithm 2 (the global matrices from V and the index set
// of nonzero entries); Section 3 step 2, eq. assemblage_1: M_ij = sum over
// elements of the element integrals.  Deterministic, no atomics: every CSR
// slot adds its contributions in a fixed order given by the mesh alone, so
// the result is bit-reproducible run to run.
// M and K come from the symmetric element storage (entry (i,j) and (j,i)
// share V[e][sym(min,max)]; M and K interleaved), T from the full n_p x n_p
// storage.
//
// A warp sums 64 consecutive contributions at a time (two per lane) with a
// segmented scan over the lanes; the slot boundaries come from the head
// masks of the groups of 32 contributions built by the symbolic phase.
#include <algorithm>
#include <vector>

#include "fem_internal.h"

namespace fem {

namespace {

__host__ __device__ constexpr int sym_idx(int np, int i, int j) {
    return i <= j ? i * np - (i * (i - 1)) / 2 + (j - i) : j * np - (j * (j - 1)) / 2 + (i - j);
}

// V entries of one element entry c = (e n_p + i) n_p + j: T from the full
// storage (its index is c itself), M and K from the interleaved symmetric
// storage (M at 2 off, K at 2 off + 1, off = e n_p(n_p+1)/2 + sym[i n_p +
// j]), with the local symmetric index from a small shared-memory table.
// VK is VM + 1 when both are requested: one 8- or 16-byte load reads both.
template <typename T>
struct Pair;
template <>
struct Pair<float> { using type = float2; };
template <>
struct Pair<double> { using type = double2; };

// F: the element matrices of a P1 simplex in FP64 as the P1 kernel stores
// them (element_simt.cu): per element the block (m_d, b s0, m_o, b s0) --
// M's diagonal and off-diagonal value and K's factor, K_e = b s0 Gram_e
// with the element's Gram matrix G A_e G^T from the geometry cache -- and
// T_e as its two factors (t_e then s_e, 2 n_p values).  A contribution
// then carries m, the pair (k, g) whose product is K's entry and the pair
// (t, s) whose product is T's.
template <int NP, typename T, bool F = false>
struct Contribution {
    T m, k, t, s, g;   // s, g: the second factors (F only)
    // 32-bit unsigned index arithmetic (element entries, slots and V
    // offsets of a mesh are below 2^31)
    __device__ __forceinline__ void load(uint32_t c, const short* __restrict__ sym, const T* __restrict__ VM,
                                         const T* __restrict__ VK, const T* __restrict__ VT,
                                         const T* __restrict__ gram) {
        constexpr uint32_t NT = NP * NP, NSYM = NP * (NP + 1) / 2;
        if constexpr (F) {
            const uint32_t e = c / NT, l = c - e * NT;
            if (VT) {
                const T* f = VT + e * (2 * NP);
                t = __ldg(f + l / NP);
                s = __ldg(f + NP + l % NP);
            } else {
                t = s = T(0);
            }
            if (VM || VK) {
                const T* base = VM ? VM : VK - 1;
                const uint32_t i = l / NP, j = l - i * NP;
                const typename Pair<T>::type mb =
                    __ldg(reinterpret_cast<const typename Pair<T>::type*>(base) + 2 * e + (i == j ? 0u : 1u));
                m = VM ? mb.x : T(0);
                k = VK ? mb.y : T(0);
                g = VK ? __ldg(gram + e * NSYM + (uint32_t)sym[l]) : T(0);
            } else {
                m = k = g = T(0);
            }
            return;
        }
        t = VT ? __ldg(VT + c) : T(0);
        if (VM || VK) {
            const uint32_t e = c / NT;
            const uint32_t off = e * NSYM + (uint32_t)sym[c - e * NT];
            if (VM && VK) {
                const typename Pair<T>::type mk = __ldg(reinterpret_cast<const typename Pair<T>::type*>(VM) + off);
                m = mk.x;
                k = mk.y;
            } else {
                m = VM ? __ldg(VM + 2 * off) : T(0);
                k = VK ? __ldg(VK + 2 * off) : T(0);
            }
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

// ------------------------------------------------------------ segment sum
// The contributions, sorted by slot, are cut into groups of 64 consecutive
// positions; a warp takes one group per step, a lane two adjacent
// contributions.  The group's head mask (bit j: position 64k+j starts a
// slot, from two of the symbolic phase's 32-bit words) and the slot of its
// first position give every lane its slots without reading seg_ptr.  Each
// lane loads its V entries and adds them within the lane, then a segmented
// inclusive scan over the lanes (shuffles) leaves every segment's total in
// the lane of its last contribution, which stores it.  A segment that runs
// past position 63 is carried into the warp's next group.
//
// Ownership: a warp task is a run of TASK groups; it writes the slots whose
// first contribution lies in its run, reading on past the run's end until
// its last slot closes.  The additions for a slot follow the fixed pattern
// of each aligned 64-group (in-lane pairs, then the lane tree), groups in
// ascending order, so the bits depend only on the mesh: run to run, across
// launch shapes, slot ranges and the batched kernel.
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ void put3(uint32_t slot, T m, T k, T t, T* __restrict__ vM, T* __restrict__ vK,
                                     T* __restrict__ vT) {
    if (vM) vM[slot] = m;
    if (vK) vK[slot] = k;
    if (vT) vT[slot] = t;
}

// A warp step covers 64 consecutive contributions (a "pair group": two of
// the symbolic phase's 32-groups, read as one 16-byte word pair), lane l the
// positions q0 = 2l and q1 = 2l + 1.  Within the lane: if q1 starts a slot,
// q0 ends one (the "first" piece, stored by this lane) and the lane's
// running piece is V[q1] alone; otherwise the running piece is V[q0] + V[q1].
// A segmented inclusive scan of the running pieces over the lanes (lane
// heads: a slot starting at q0 or q1) gives every lane the sum of its
// running segment so far; a first piece adds the scanned value of the lane
// before it.  Positions nc and beyond act as the start of a slot, so values
// loaded for them (indices clamped into the array) never reach a stored sum.
//
// Pair groups [k0, k1) of a mesh with `nc` contributions; only slots in
// [s0, s1) are written.  STEPS lane-scan strides must cover the lanes one
// slot's running piece spans within a pair group (2 for segments of at
// most 8 contributions, 4 for at most 32, else 5); more steps than needed
// leave the sums unchanged.
//
// Ownership: the warp writes the slots whose first contribution lies in its
// pair groups: in the first group the positions from its first head on, in
// its own groups all positions, and past its last group the positions that
// continue its last slot (up to the next head).
//
// Software pipeline: while pair group k is summed, the V entries of group
// k+1 and the head words and contributor indices of group k+2 are in flight
// (V and indices only up to group k1, where a carried slot usually ends).
template <int NP, typename T, int STEPS>
__device__ __forceinline__ void segsum_warp(uint32_t k0, uint32_t k1, uint32_t nc, uint32_t s0, uint32_t s1,
                                            const uint4* __restrict__ head2, const uint32_t* __restrict__ contrib,
                                            const short* __restrict__ sym, const T* __restrict__ VM,
                                            const T* __restrict__ VK, const T* __restrict__ VT, T* __restrict__ vM,
                                            T* __restrict__ vK, T* __restrict__ vT, int lane) {
    const uint32_t glast = (nc - 1) >> 6;        // last pair group
    const uint32_t qmax = (nc - 1) & ~1u;        // last even position (pairs are read from an even index)
    const uint32_t j0 = 2u * lane;               // q0 within the pair group
    auto hword = [&](uint32_t k) { return __ldg(head2 + (k < glast ? k : glast)); };
    auto cpair = [&](uint32_t k) {
        const uint32_t q = (k << 6) + j0, qc = q < qmax ? q : qmax;
        uint2 c = __ldg(reinterpret_cast<const uint2*>(contrib + qc));
        if (qc + 1 >= nc) c.y = c.x;   // odd nc: the entry past the end is not a contributor index
        return c;
    };
    uint4 h0 = hword(k0), h1 = hword(k0 + 1);
    Contribution<NP, T> a0, b0;
    {
        const uint2 c = cpair(k0);
        a0.load(c.x, sym, VM, VK, VT, nullptr);
        b0.load(c.y, sym, VM, VK, VT, nullptr);
    }
    uint2 c1 = cpair(k0 + 1);
    uint32_t lo;   // first owned position of the pair group
    {
        const uint64_t H = (static_cast<uint64_t>(h0.z) << 32) | h0.x;
        lo = H ? __ffsll(H) - 1 : 64u;
    }
    T cm = T(0), ck = T(0), ct = T(0);   // running sum carried past position 63
    for (uint32_t k = k0;; ++k) {
        // prefetch (warp-uniform): V of k+1 while k+1 <= k1 (k1 itself is
        // the usual continuation group), indices of k+2 while k+2 <= k1;
        // groups further on are loaded when the carry actually reaches them
        Contribution<NP, T> a1, b1;
        if (k + 1 <= k1) {
            a1.load(c1.x, sym, VM, VK, VT, nullptr);
            b1.load(c1.y, sym, VM, VK, VT, nullptr);
        }
        const uint4 h2 = hword(k + 2);
        const uint2 c2 = k + 2 <= k1 ? cpair(k + 2) : make_uint2(0u, 0u);

        const uint64_t H = (static_cast<uint64_t>(h0.z) << 32) | h0.x;
        const uint32_t hi = k < k1 ? 64u : (H ? __ffsll(H) - 1 : 64u);   // past k1: up to the next head
        const uint32_t q0 = (k << 6) + j0, q1 = q0 + 1;
        const uint32_t two = static_cast<uint32_t>(H >> j0) & 3u;
        const bool rB = two >> 1;                         // real head at q1
        const bool hA = (two & 1u) || q0 == nc, hB = rB || q1 == nc;
        const uint32_t slotA = h0.y + __popcll(H & ((2ull << j0) - 1) & ~1ull);
        const uint32_t slotB = slotA + (rB ? 1u : 0u);
        T rm = hB ? b0.m : a0.m + b0.m;
        T rk = hB ? b0.k : a0.k + b0.k;
        T rt = hB ? b0.t : a0.t + b0.t;
        const uint32_t lup = __ballot_sync(FULL, hA || hB) & (FULL >> (31 - lane));
        const int run = lane - (lup ? 31 - __clz(lup) : 0);
#pragma unroll
        for (int i = 0; i < STEPS; ++i) {
            const int d = 1 << i;
            const T ym = __shfl_up_sync(FULL, rm, d);
            const T yk = __shfl_up_sync(FULL, rk, d);
            const T yt = __shfl_up_sync(FULL, rt, d);
            if (run >= d) {
                rm = ym + rm;
                rk = yk + rk;
                rt = yt + rt;
            }
        }
        if (lup == 0) {   // continues the running sum of the previous pair group
            rm = cm + rm;
            rk = ck + rk;
            rt = ct + rt;
        }
        // the sum before q0 within its segment (lane 0: the carried sum)
        T pm = __shfl_up_sync(FULL, rm, 1), pk = __shfl_up_sync(FULL, rk, 1), pt = __shfl_up_sync(FULL, rt, 1);
        if (lane == 0) {
            pm = cm;
            pk = ck;
            pt = ct;
        }
        const bool own0 = j0 >= lo && j0 < hi, own1 = j0 + 1 >= lo && j0 + 1 < hi;
        if (hB && q0 < nc && own0 && slotA >= s0 && slotA < s1) {
            const bool alone = two & 1u;   // a head at q0 too: V[q0] is the whole slot
            put3(slotA, alone ? a0.m : pm + a0.m, alone ? a0.k : pk + a0.k, alone ? a0.t : pt + a0.t, vM, vK, vT);
        }
        const uint32_t nxt = lane < 31 ? static_cast<uint32_t>(H >> (lane < 31 ? j0 + 2 : 0)) & 1u : (h1.x & 1u);
        if ((nxt || q1 + 1 == nc) && q1 < nc && own1 && slotB >= s0 && slotB < s1) put3(slotB, rm, rk, rt, vM, vK, vT);
        // does position 63's slot (this warp's, in range) go on into pair group k+1?
        const uint32_t q63 = (k << 6) + 63;
        const uint32_t slot63 = h0.y + __popcll(H & ~1ull);
        const bool carry = q63 + 1 < nc && !(h1.x & 1u) && hi == 64u && lo <= 63u && slot63 >= s0 && slot63 < s1;
        cm = __shfl_sync(FULL, rm, 31);
        ck = __shfl_sync(FULL, rk, 31);
        ct = __shfl_sync(FULL, rt, 31);
        if (k >= glast || (k + 1 >= k1 && !carry)) break;
        lo = 0;
        h0 = h1;
        h1 = h2;
        if (k + 1 <= k1) {
            a0 = a1;
            b0 = b1;
        } else {   // the carry runs past the prefetched continuation group
            const uint2 c = cpair(k + 1);
            a0.load(c.x, sym, VM, VK, VT, nullptr);
            b0.load(c.y, sym, VM, VK, VT, nullptr);
        }
        c1 = c2;
    }
}

// ------------------------------------------------------- FP64 octet sum
// FP64 values take a different grouping, because FP64 additions, not memory,
// bound the pair-group sum in FP64 on this part (about 2 FP64 operations per
// clock and SM: the pair-group scan spends ~10.5 additions per contribution,
// most of them on scan steps whose result is discarded).  Here a warp step
// covers 256 consecutive contributions, lane l the eight positions
// 256k + 8l .. 256k + 8l + 7, added in order inside the lane (a segment that
// starts and ends inside the lane is complete there); only the piece open at
// the lane's end takes part in a segmented inclusive scan over the lanes
// (STEPS strides cover a segment of up to 8 (2^STEPS - 1) + 1 contributions
// within one step: 1 step for 9, 2 for 25, 3 for 57, 5 for any), and the
// piece before the lane's first head adds the scanned value of the lane
// before it.  About 4 additions per contribution (7 in-lane and ~6 scan and
// carry additions per matrix and 256 contributions, for 2 scan steps).
//
// Stores: a slot's total is stored by the lane holding its last
// contribution: inside the loop when the lane meets the next head, after the
// scan when the lane's first head closes a slot begun in earlier lanes, or
// when the position after the lane is a head (or the end).  Positions nc and
// beyond act as heads; lanes wholly past nc store nothing.
//
// Ownership: a warp task covers steps [k0, k1) and writes the slots whose
// first contribution lies in [256 k0, 256 k1) (and in [s0, s1)), going on
// past k1 while its last slot is open.  The order of additions for a slot
// depends only on the positions (eight per lane, the fixed scan tree, steps
// in ascending order), so the bits are the same for every task shape, slot
// range and the batched kernel.
// PART selects the matrices a call sums: 0 all three, 1 M and K (the
// interleaved pairs), 2 T; the split form runs a task twice with fewer
// values live per lane (more resident warps).  The additions per matrix are
// the same in every form, so are the bits.
// F: the P1 factored element matrices (see Contribution); each K and T
// contribution is added as a fused multiply-add of its two factors.
template <int NP, int STEPS, int PART, typename T, bool F = false, int LAF = 4>
__device__ __forceinline__ void segsum8_warp(uint32_t k0, uint32_t k1, uint32_t nc, uint32_t s0, uint32_t s1,
                                             const uint2* __restrict__ head, const uint32_t* __restrict__ contrib,
                                             const short* __restrict__ sym, const T* __restrict__ VM,
                                             const T* __restrict__ VK, const T* __restrict__ VT,
                                             const T* __restrict__ gram, T* __restrict__ vM, T* __restrict__ vK,
                                             T* __restrict__ vT, int lane) {
    constexpr bool MK = PART != 2, TT = PART != 1;
    if constexpr (!MK) { VM = VK = nullptr; vM = vK = nullptr; }
    if constexpr (!TT) { VT = nullptr; vT = nullptr; }
    const uint32_t nwords = (nc + 31) >> 5;
    auto word = [&](uint32_t w) { return __ldg(head + (w < nwords ? w : nwords - 1)); };
    // first slot whose first contribution is at or after position p (p a multiple of 256)
    auto first_slot_from = [&](uint32_t p) -> uint32_t {
        if (p >= nc) return 0xffffffffu;
        const uint2 h = word(p >> 5);
        return h.y + ((h.x & 1u) ? 0u : 1u);
    };
    const uint32_t slo = max(first_slot_from(k0 << 8), s0);
    const uint32_t shi = min(first_slot_from(k1 << 8), s1);
    T cm = T(0), ck = T(0), ct = T(0);   // running sum carried into the step
    const int sh = (lane & 3) * 8;
    for (uint32_t k = k0;; ++k) {
        const uint32_t p0 = (k << 8) + 8u * lane;
        const bool live = p0 < nc;
        const uint2 hw = word((k << 3) + (lane >> 2));
        uint32_t bits = (hw.x >> sh) & 0xffu;
        if (p0 + 8 > nc) bits |= nc > p0 ? (0xffu << (nc - p0)) & 0xffu : 0xffu;   // positions >= nc: heads
        // slot of position p0 (the word's slot plus the heads after its first position)
        const uint32_t slot0 = hw.y + __popc(hw.x & ((2u << sh) - 1u) & ~1u);
        // the lane's eight contributors and their V entries
        uint32_t c[8];
        if (p0 + 8 <= nc) {
            const uint4 a = __ldg(reinterpret_cast<const uint4*>(contrib + p0));
            const uint4 b = __ldg(reinterpret_cast<const uint4*>(contrib + p0 + 4));
            c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
            c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) c[i] = p0 + i < nc ? __ldg(contrib + p0 + i) : 0u;
        }
        // the lane's V entries: all eight in flight at once, or, for the
        // factored M/K pass (three values per entry), four at a time, each
        // next one issued as the oldest is added (64 registers either way)
        constexpr int LA = (F && MK) ? LAF : 8;
        Contribution<NP, T, F> v[8];
        auto fetch = [&](int i) {
            if (p0 + i < nc) v[i].load(c[i], sym, VM, VK, VT, gram);
            else v[i].m = v[i].k = v[i].t = v[i].s = v[i].g = T(0);
        };
#pragma unroll
        for (int i = 0; i < LA; ++i) fetch(i);
        auto own = [&](uint32_t sl) { return live && sl >= slo && sl < shi; };
        // in-lane pass: a* = the open piece, p* = the piece before the first head
        const bool h0 = bits & 1u;
        T am = T(0), ak = T(0), at = T(0), pm = T(0), pk = T(0), pt = T(0);
        if constexpr (MK) { am = v[0].m; ak = F ? v[0].k * v[0].g : v[0].k; }
        if constexpr (TT) at = F ? v[0].t * v[0].s : v[0].t;
        bool seen = h0;
        uint32_t cur = slot0;   // slot of the open piece once a head was seen
#pragma unroll
        for (int i = 1; i < 8; ++i) {
            if (i + LA - 1 < 8 && i + LA - 1 >= LA) fetch(i + LA - 1);
            const bool h = (bits >> i) & 1u;
            if (h && seen && own(cur)) put3(cur, am, ak, at, vM, vK, vT);   // a slot complete in the lane
            if (h && !seen) {
                if constexpr (MK) { pm = am; pk = ak; }
                if constexpr (TT) pt = at;
            }
            cur += h ? 1u : 0u;   // the first head opens slot0 + 1, each later one the next slot
            seen = seen || h;
            if constexpr (MK) {
                am = h ? v[i].m : am + v[i].m;
                if constexpr (F) ak = fma(v[i].k, v[i].g, h ? T(0) : ak);
                else ak = h ? v[i].k : ak + v[i].k;
            }
            if constexpr (TT) {
                if constexpr (F) at = fma(v[i].t, v[i].s, h ? T(0) : at);
                else at = h ? v[i].t : at + v[i].t;
            }
        }
        // segmented inclusive scan of the open pieces over the lanes
        const uint32_t lup = __ballot_sync(FULL, seen) & (FULL >> (31 - lane));
        const int run = lane - (lup ? 31 - __clz(lup) : 0);
#pragma unroll
        for (int i = 0; i < STEPS; ++i) {
            const int d = 1 << i;
            T ym = T(0), yk = T(0), yt = T(0);
            if constexpr (MK) { ym = __shfl_up_sync(FULL, am, d); yk = __shfl_up_sync(FULL, ak, d); }
            if constexpr (TT) yt = __shfl_up_sync(FULL, at, d);
            if (run >= d) {
                if constexpr (MK) { am = ym + am; ak = yk + ak; }
                if constexpr (TT) at = yt + at;
            }
        }
        if (lup == 0) {   // continues the piece carried from the previous step
            if constexpr (MK) { am = cm + am; ak = ck + ak; }
            if constexpr (TT) at = ct + at;
        }
        // the lane's first head closes the slot begun before the lane
        T qm = T(0), qk = T(0), qt = T(0);
        if constexpr (MK) { qm = __shfl_up_sync(FULL, am, 1); qk = __shfl_up_sync(FULL, ak, 1); }
        if constexpr (TT) qt = __shfl_up_sync(FULL, at, 1);
        if (lane == 0) {
            qm = cm;
            qk = ck;
            qt = ct;
        }
        if (seen && !h0 && own(slot0)) {
            if constexpr (MK) { qm = qm + pm; qk = qk + pk; }
            if constexpr (TT) qt = qt + pt;
            put3(slot0, qm, qk, qt, vM, vK, vT);
        }
        // the position after the lane starts a slot (or is the end): the open piece is complete
        const uint32_t nb = __shfl_down_sync(FULL, bits, 1);
        const bool next_head = lane < 31 ? (nb & 1u) != 0u
                                         : ((k + 1) << 8) >= nc || (word((k + 1) << 3).x & 1u) != 0u;
        if (next_head && own(cur)) put3(cur, am, ak, at, vM, vK, vT);
        if constexpr (MK) { cm = __shfl_sync(FULL, am, 31); ck = __shfl_sync(FULL, ak, 31); }
        if constexpr (TT) ct = __shfl_sync(FULL, at, 31);
        // go on past k1 only while the slot open at the step's end is this warp's
        if (k + 1 >= k1) {
            const uint32_t pn = (k + 1) << 8;
            if (pn >= nc) break;
            const uint2 hn = word(pn >> 5);
            if ((hn.x & 1u) || hn.y >= shi || hn.y < slo) break;
        }
    }
}

// Launch shape, measured on GB300: FP32 values run best with registers
// capped for 5 blocks of 256 threads per SM (tri_p2_1024: 0.390 ms vs 0.434
// with 6 blocks and 0.398 with 4; the tetrahedral meshes lose 5-20% with 4
// or 6), FP64 values with 4; warp tasks of 32 pair groups (tri_p2_1024:
// 0.382 ms vs 0.389 with 16 and 0.412 with 8; the tetrahedral meshes are
// flat from 32 to 48).
template <int STEPS, typename T>
struct SegShape {
    static constexpr int MIN_BLOCKS = sizeof(T) == 8 ? 4 : 5;
    static constexpr uint32_t TASK = 32;   // pair groups per warp task (at most)
};

// Slots [s0, s1) of one mesh; the warps take tasks grid-stride, so the
// pair groups in flight form one moving window over the slot order
// (elements shared by nearby rows are re-read from L2).
template <int NP, typename T, int STEPS>
__global__ void __launch_bounds__(256, SegShape<STEPS, T>::MIN_BLOCKS)
    segsum_kernel(const uint4* __restrict__ head2, const uint32_t* __restrict__ contrib, uint32_t nc,
                  const int* __restrict__ seg_ptr, uint32_t s0, uint32_t s1, uint32_t task, const T* __restrict__ VM,
                  const T* __restrict__ VK, const T* __restrict__ VT, T* __restrict__ vM, T* __restrict__ vK,
                  T* __restrict__ vT) {
    __shared__ short sym[NP * NP];
    fill_sym_table<NP>(sym);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t a = (uint32_t)__ldg(seg_ptr + s0), b = (uint32_t)__ldg(seg_ptr + s1);
    const uint32_t g0 = a >> 6, g1 = (b + 63) >> 6;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const T* vm_src = vM ? VM : nullptr;
    const T* vk_src = vK ? VK : nullptr;
    const T* vt_src = vT ? VT : nullptr;
    for (uint32_t t = g0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * task; t < g1; t += nw * task)
        segsum_warp<NP, T, STEPS>(t, t + task < g1 ? t + task : g1, nc, s0, s1, head2, contrib, sym, vm_src, vk_src,
                                  vt_src, vM, vK, vT, lane);
}

// FP64: steps of 256 contributions (eight per lane), warps take tasks of up
// to TASK8 steps grid-stride
constexpr uint32_t TASK8 = 8;

template <int NP, int STEPS, int MINB, bool SPLIT, typename T, bool F>
__global__ void __launch_bounds__(256, MINB) segsum8_kernel(const uint2* __restrict__ head,
                                                      const uint32_t* __restrict__ contrib, uint32_t nc,
                                                      const int* __restrict__ seg_ptr, uint32_t s0, uint32_t s1,
                                                      uint32_t task, const T* __restrict__ VM,
                                                      const T* __restrict__ VK, const T* __restrict__ VT,
                                                      const T* __restrict__ gram, T* __restrict__ vM,
                                                      T* __restrict__ vK, T* __restrict__ vT) {
    __shared__ short sym[NP * NP];
    fill_sym_table<NP>(sym);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t a = (uint32_t)__ldg(seg_ptr + s0), b = (uint32_t)__ldg(seg_ptr + s1);
    const uint32_t g0 = a >> 8, g1 = (b + 255) >> 8;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const T* vm_src = vM ? VM : nullptr;
    const T* vk_src = vK ? VK : nullptr;
    const T* vt_src = vT ? VT : nullptr;
    for (uint32_t t = g0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * task; t < g1; t += nw * task) {
        const uint32_t t1 = t + task < g1 ? t + task : g1;
        if constexpr (SPLIT) {
            if (vM || vK)
                segsum8_warp<NP, STEPS, 1, T, F, (MINB >= 4 ? 4 : 8)>(t, t1, nc, s0, s1, head, contrib, sym, vm_src,
                                                                      vk_src, vt_src, gram, vM, vK, vT, lane);
            if (vT)
                segsum8_warp<NP, STEPS, 2, T, F>(t, t1, nc, s0, s1, head, contrib, sym, vm_src, vk_src, vt_src, gram,
                                                 vM, vK, vT, lane);
        } else {
            segsum8_warp<NP, STEPS, 0, T, F>(t, t1, nc, s0, s1, head, contrib, sym, vm_src, vk_src, vt_src, gram, vM,
                                             vK, vT, lane);
        }
    }
}

template <int NP, int STEPS, int MINB, bool SPLIT, typename T, bool F>
int launch_steps8_b(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s,
                    int nsm, int64_t s0, int64_t s1) {
    static int occ = 0;   // blocks per SM (the same on every device of the pool)
    if (!occ) {
        int o = 0;
        FEM_CUDA_TRY(
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, segsum8_kernel<NP, STEPS, MINB, SPLIT, T, F>, 256, 0));
        occ = o > 0 ? o : 1;
    }
    const int64_t nc = m.E * m.np * m.np;
    const int64_t steps = ((nc + 255) / 256) * (s1 - s0) / (m.nnz > 0 ? m.nnz : 1) + 1;
    const int64_t warps = (int64_t)nsm * occ * 8;
    int64_t task = (steps + warps - 1) / warps;
    if (task > TASK8) task = TASK8;
    if (task < 1) task = 1;
    int64_t blocks = ((steps + task - 1) / task + 7) / 8;
    if (blocks > (int64_t)nsm * occ) blocks = (int64_t)nsm * occ;
    if (blocks < 1) blocks = 1;
    cudaGetLastError();   // clear any stale error before the launch check
    segsum8_kernel<NP, STEPS, MINB, SPLIT, T, F><<<(unsigned)blocks, 256, 0, s>>>(
        m.seg_head.as<uint2>(), reinterpret_cast<const uint32_t*>(m.contrib.as<int>()), (uint32_t)nc,
        m.seg_ptr.as<int>(), (uint32_t)s0, (uint32_t)s1, (uint32_t)task, VM, VK, VT,
        F ? reinterpret_cast<const T*>(m.gram64.ptr) : nullptr, vM, vK, vT);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

// The sum is bound by the latency of its gathers (ncu: long-scoreboard
// stalls, FP64 pipe half busy at two blocks per SM).  Summing a task twice,
// the M/K pairs and then T, keeps fewer values live per lane: 64 registers,
// four blocks of 256 per SM.  Measured on GB300 (FP64): tet_p1_128 1.89 ms
// against 2.02 with three blocks and 2.75 for the single pass at two blocks
// (116 registers); tri_p2_1024 0.96 vs 1.17 ms; tet_p2_64 1.70 vs 2.46 ms.
// Prefetching the next step's V lines into L2 was slower (3.47 vs 3.01 ms
// for the single pass).  Every form adds the same terms in the same order.
template <int NP, int STEPS, typename T>
int launch_steps8(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s,
                  int nsm, int64_t s0, int64_t s1, bool p1f) {
    if constexpr (NP == 3 || NP == 4) {
        if (p1f) return launch_steps8_b<NP, STEPS, 4, true, T, true>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
    }
    return launch_steps8_b<NP, STEPS, 4, true, T, false>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
}


// Batched: one warp per work item (a run of `count` groups of one mesh),
// the same per-warp sum as the single-mesh kernels, so a mesh's CSR values
// carry the same bits alone and in a batch.  The items are grouped by n_p
// and each group has its own launch, compiled for its n_p and scan depth
// (the deepest any of its meshes needs; deeper scans leave the sums
// unchanged), with its registers capped so that 3 (FP64) or 4 (FP32) blocks
// of 256 threads share an SM.
// One block per SM fewer than the single-mesh sums: the per-item mesh
// parameters take registers, and at the single-mesh cap the loop spills.
template <typename T>
constexpr int batch_sum_blocks() { return SegShape<1, T>::MIN_BLOCKS - 1; }

template <int NP, typename T, int STEPS>
__global__ void __launch_bounds__(256, batch_sum_blocks<T>())
    batch_segsum_kernel(const BatchItem* __restrict__ items, int nitems, const BatchMesh* __restrict__ meshes) {
    __shared__ short sym[NP * NP];
    fill_sym_table<NP>(sym);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < nitems; it += nw) {
        const BatchItem w = items[it];
        const BatchMesh& bm = meshes[w.mesh];
        T* vM = static_cast<T*>(bm.vM);
        T* vK = static_cast<T*>(bm.vK);
        T* vT = static_cast<T*>(bm.vT);
        if (!(vM || vK || vT)) continue;   // mesh skipped in this launch (warp-uniform)
        const T* VM = vM ? static_cast<const T*>(bm.VM) : nullptr;
        const T* VK = vK ? static_cast<const T*>(bm.VK) : nullptr;
        const T* VT = vT ? static_cast<const T*>(bm.VT) : nullptr;
        const uint32_t k0 = (uint32_t)w.first, k1 = k0 + (uint32_t)w.count;
        const uint32_t nc = (uint32_t)(bm.E * bm.np * bm.np), s1 = (uint32_t)bm.nnz;
        const uint32_t* cp = reinterpret_cast<const uint32_t*>(bm.contrib);
        if constexpr (sizeof(T) == 8) {   // the single-mesh FP64 form: M/K pairs, then T
            bool f = false;   // P1 simplices: the factored element matrices
            if constexpr (NP == 3 || NP == 4) f = bm.type == 0 || bm.type == 3;
            const double* gram = bm.gram64;
            if (f) {
                if (vM || vK)
                    segsum8_warp<NP, STEPS, 1, double, true>(k0, k1, nc, 0u, s1, bm.seg_head, cp, sym, VM, VK, VT,
                                                             gram, vM, vK, vT, lane);
                if (vT)
                    segsum8_warp<NP, STEPS, 2, double, true>(k0, k1, nc, 0u, s1, bm.seg_head, cp, sym, VM, VK, VT,
                                                             gram, vM, vK, vT, lane);
            } else {
                if (vM || vK)
                    segsum8_warp<NP, STEPS, 1, double, false>(k0, k1, nc, 0u, s1, bm.seg_head, cp, sym, VM, VK, VT,
                                                              nullptr, vM, vK, vT, lane);
                if (vT)
                    segsum8_warp<NP, STEPS, 2, double, false>(k0, k1, nc, 0u, s1, bm.seg_head, cp, sym, VM, VK, VT,
                                                              nullptr, vM, vK, vT, lane);
            }
        } else {
            segsum_warp<NP, T, STEPS>(k0, k1, nc, 0u, s1, reinterpret_cast<const uint4*>(bm.seg_head), cp, sym, VM,
                                      VK, VT, vM, vK, vT, lane);
        }
    }
}

template <int NP, typename T, int STEPS>
int batch_segsum_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, int nsm, cudaStream_t s) {
    const int wpb = 8;
    int grid = nsm * batch_sum_blocks<T>();
    if ((int64_t)grid * wpb > nitems) grid = (nitems + wpb - 1) / wpb;
    cudaGetLastError();   // clear any stale error before the launch check
    batch_segsum_kernel<NP, T, STEPS><<<grid, 256, 0, s>>>(items, nitems, meshes);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

template <int NP, typename T>
int batch_segsum_np(const BatchItem* items, int nitems, const BatchMesh* meshes, int max_seg, int nsm,
                    cudaStream_t s) {
    if constexpr (sizeof(T) == 8) {
        if (max_seg <= 9) return batch_segsum_launch<NP, T, 1>(items, nitems, meshes, nsm, s);
        if (max_seg <= 25) return batch_segsum_launch<NP, T, 2>(items, nitems, meshes, nsm, s);
        if (max_seg <= 57) return batch_segsum_launch<NP, T, 3>(items, nitems, meshes, nsm, s);
        return batch_segsum_launch<NP, T, 5>(items, nitems, meshes, nsm, s);
    } else {
        if (max_seg <= 8) return batch_segsum_launch<NP, T, 2>(items, nitems, meshes, nsm, s);
        if (max_seg <= 32) return batch_segsum_launch<NP, T, 4>(items, nitems, meshes, nsm, s);
        return batch_segsum_launch<NP, T, 5>(items, nitems, meshes, nsm, s);
    }
}

template <int NP, typename T, int STEPS>
int launch_steps(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s,
                 int nsm, int64_t s0, int64_t s1) {
    // persistent: as many 256-thread blocks as fit on the GPU at once
    static int occ = 0;   // blocks per SM (the same on every device of the pool)
    if (!occ) {
        int o = 0;
        FEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, segsum_kernel<NP, T, STEPS>, 256, 0));
        occ = o > 0 ? o : 1;
    }
    const int64_t nc = m.E * m.np * m.np;
    // tasks of up to TASK pair groups; fewer for small meshes or slot ranges
    // (groups estimated in proportion to the slots), so that every resident
    // warp gets work (the sums do not depend on the task size)
    const int64_t groups = ((nc + 63) / 64) * (s1 - s0) / (m.nnz > 0 ? m.nnz : 1) + 1;
    const int64_t warps = (int64_t)nsm * occ * 8;
    int64_t task = (groups + warps - 1) / warps;
    if (task > SegShape<STEPS, T>::TASK) task = SegShape<STEPS, T>::TASK;
    if (task < 1) task = 1;
    int64_t blocks = ((groups + task - 1) / task + 7) / 8;
    if (blocks > (int64_t)nsm * occ) blocks = (int64_t)nsm * occ;
    if (blocks < 1) blocks = 1;
    cudaGetLastError();   // clear any stale error before the launch check
    segsum_kernel<NP, T, STEPS><<<(unsigned)blocks, 256, 0, s>>>(
        reinterpret_cast<const uint4*>(m.seg_head.as<uint2>()), reinterpret_cast<const uint32_t*>(m.contrib.as<int>()),
        (uint32_t)nc,
        m.seg_ptr.as<int>(), (uint32_t)s0, (uint32_t)s1, (uint32_t)task, VM, VK, VT, vM, vK, vT);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

// lane-scan steps: 2 cover segments of up to 8 contributions (every
// triangle mesh), 4 up to 32 (the tetrahedral meshes), 5 any
template <int NP, typename T>
int launch_np(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s,
              int nsm, int64_t s0, int64_t s1, bool p1f) {
    if constexpr (sizeof(T) == 8) {
        // eight contributions per lane: scan strides for the longest segment
        if (m.max_seg <= 9) return launch_steps8<NP, 1>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
        if (m.max_seg <= 25) return launch_steps8<NP, 2>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
        if (m.max_seg <= 57) return launch_steps8<NP, 3>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
        return launch_steps8<NP, 5>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
    }
    if (m.max_seg <= 8) return launch_steps<NP, T, 2>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
    if (m.max_seg <= 32) return launch_steps<NP, T, 4>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
    return launch_steps<NP, T, 5>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1);
}

template <typename T>
int run(const fem_mesh& m, const T* VM, const T* VK, const T* VT, T* vM, T* vK, T* vT, cudaStream_t s, int64_t s0,
        int64_t s1, bool p1f) {
    if (s1 < 0) s1 = m.nnz;
    if (s0 < 0 || s0 > s1 || s1 > m.nnz) return fail(FEM_EINVAL, "slot range out of bounds");
    if (m.nnz <= 0 || s1 == s0) return FEM_OK;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    switch (m.np) {
        case 3: return launch_np<3, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
        case 4: return launch_np<4, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
        case 6: return launch_np<6, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
        case 10: return launch_np<10, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
        case 20: return launch_np<20, T>(m, VM, VK, VT, vM, vK, vT, s, nsm, s0, s1, p1f);
    }
    return fail(FEM_EINVAL, "unsupported n_p");
}

}  // namespace

template <typename T>
int batch_scatter_launch(const BatchItem* items, int nitems, const BatchMesh* meshes, int np, int max_seg,
                         cudaStream_t s) {
    if (nitems <= 0) return FEM_OK;
    int dev = 0, nsm = 0;
    FEM_CUDA_TRY(cudaGetDevice(&dev));
    FEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    switch (np) {
        case 3: return batch_segsum_np<3, T>(items, nitems, meshes, max_seg, nsm, s);
        case 4: return batch_segsum_np<4, T>(items, nitems, meshes, max_seg, nsm, s);
        case 6: return batch_segsum_np<6, T>(items, nitems, meshes, max_seg, nsm, s);
        case 10: return batch_segsum_np<10, T>(items, nitems, meshes, max_seg, nsm, s);
        case 20: return batch_segsum_np<20, T>(items, nitems, meshes, max_seg, nsm, s);
        default: return fail(FEM_EINVAL, "element type");
    }
}
template int batch_scatter_launch<float>(const BatchItem*, int, const BatchMesh*, int, int, cudaStream_t);
template int batch_scatter_launch<double>(const BatchItem*, int, const BatchMesh*, int, int, cudaStream_t);

int scatter_fp64(const fem_mesh& m, const double* VM, const double* VK, const double* VT, double* vM, double* vK,
                 double* vT, bool p1f, cudaStream_t s, int64_t s0, int64_t s1) {
    if (p1f && !p1_factored(m)) return fail(FEM_EINVAL, "factored element matrices of a mesh that has none");
    return run<double>(m, VM, VK, VT, vM, vK, vT, s, s0, s1, p1f);
}

int scatter_fp32(const fem_mesh& m, const float* VM, const float* VK, const float* VT, float* vM, float* vK,
                 float* vT, cudaStream_t s, int64_t s0, int64_t s1) {
    return run<float>(m, VM, VK, VT, vM, vK, vT, s, s0, s1, false);
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
