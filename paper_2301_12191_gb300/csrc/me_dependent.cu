// me_dependent.cu -- dependent analysis of ladder rungs (inter-resolution
// analysis sharing with refinement, Sec. 4.3 / 6.3; reuse and refinement
// controls, App. A.1 / A.2), in three kernels over a whole batch:
//
//   1. rules (one CTA per CTU): every CU maps its centre to the reference
//      rung, takes the co-located leaf's depth and scaled vector (search
//      centre) and its depth window; reachability through the ancestors'
//      split permissions; the evaluated CUs are appended to one task list
//      per CU size, the CTU's argmin keys are reset.
//   2. search (persistent grid over the task lists): lane task = one CU x
//      one horizontal offset dx x a band of TY vertical offsets; the lane
//      walks every 8x8 block of its CU and accumulates the CU's SAD for its
//      TY candidates.  Reference rows are read straight from L1: three (8-bit)
//      or five (10-bit) aligned words, shifted to the lane's start with two
//      multiply-adds per word (FMA pipe; the ALU pipe does the SADs).  8-bit
//      SADs use vabsdiff4 .add; 10-bit SADs use sum(a) + sum(b) -
//      2 sum(min(a, b)) on packed halfword pairs (see me_full.cu).  The
//      lanes of a CU are contiguous in a warp: a segmented min over the
//      keys SAD * 2^RB + code (code orders (|dx|+|dy|, dy, dx)) leaves one
//      atomicMin per CU and warp on the CU's global key.  CUs of 32x32 and
//      up are split into 16x16 ranges (one task each, so no warp walks more
//      than four blocks); their candidate SADs add up in a per-CU table.
//   3. decide (one CTA per CTU): vectors from the keys (or the argmin over
//      a CU's table), then SATD, cost, split and leaf maps.
#include "common.cuh"

#include <algorithm>
#include <type_traits>

namespace ladder_impl {
namespace {

__constant__ int c_lambda_q16[52] = {
#include "lambda_table.inc"
};

constexpr int kSearchThreads = 256;
constexpr int kDecideThreads = 128;

__device__ __forceinline__ int item_of(const DependentBatch &b) { return dev::item_of_cta(b.item, b.n); }

__device__ __forceinline__ int depth_of(int i, int dmax)
{
    int d = 0;
    while (d < dmax && i >= key_offset(d + 1)) ++d;
    return d;
}

// ---- 1. rules ---------------------------------------------------------------
// One CTA per CTU, one thread per CU: the rule, reachability and flags, the
// CU's place in its size class's task list (one global atomic per class and
// CTA), and zeroed sum tables for the CUs searched in pieces.
constexpr int kRulesThreads = 128;

template <int CTU>
__global__ void __launch_bounds__(kRulesThreads) k_dep_rules(const __grid_constant__ DependentBatch b)
{
    dev::chain_entry();
    using C = dev::Ctu<CTU>;
    constexpr int NK = C::NKEY;
    static_assert(NK <= kRulesThreads, "one thread per CU");
    static_assert(((kRuleEvaluated | kRuleCanSplit | kRuleReachable | kRuleInherited) & dev::kPresent) == 0,
                  "rule flags and the present flag share one byte");
    constexpr int NBIG = key_offset(C::DMAX - kFirstSummedClass + 1);  // CUs of 32x32 and up
    const int tid = threadIdx.x;
    const bool mine = tid < NK;

    __shared__ uint8_t s_leaf[NK], s_splitok[NK], s_ev[NK], s_inh[NK];
    __shared__ uint32_t s_ctr[NK];  // centres, cx | cy << 16
    __shared__ int s_pos[NK];       // list places (searched) or table slots (inherited), -1: none
    __shared__ unsigned int s_cnt[2 * kSizeClasses], s_base[2 * kSizeClasses];
    __shared__ int s_big[NBIG > 0 ? NBIG : 1];  // list places of CUs searched in pieces (-1: none)
    if (tid < 2 * kSizeClasses) s_cnt[tid] = 0;

    const int ri = item_of(b);
    const DependentItem &a = b.item[ri];
    const RungInfo &rinf = b.rung[a.rung];
    const RungInfo &rref = b.rung[a.parent];  // the rung whose decisions this one refines
    const RungGeom &g = rinf.g;
    const int ctu_idx = static_cast<int>(blockIdx.x) - a.cta_begin;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const long kbase = static_cast<long>(ctu_idx) * NK;

    // the rule of CU tid
    const int d = mine ? depth_of(tid, C::DMAX) : 0;
    const int li = tid - key_offset(d), n = 1 << d, S = CTU >> d;
    const int cu_x = x0 + (li % n) * S, cu_y = y0 + (li / n) * S;
    const bool present = mine && cu_x < g.W8 && cu_y < g.H8;
    uint8_t leaf = 0, splitok = 0;
    int16_t cx = 0, cy = 0;
    if (present) {
        DepRefs refs;
        refs.Wr = rref.g.W;
        refs.Hr = rref.g.H;
        refs.cols8_r = rref.g.cols8;
        refs.leaf_depth = reinterpret_cast<const uint8_t *>(a.ref_block + rref.off.leaf_depth);
        refs.leaf_mvx = reinterpret_cast<const int16_t *>(a.ref_block + rref.off.leaf_mvx);
        refs.leaf_mvy = reinterpret_cast<const int16_t *>(a.ref_block + rref.off.leaf_mvy);
        refs.depth_lo = b.depth_lo;
        refs.depth_hi = b.depth_hi;
        refs.use_ref_mv = b.use_ref_mv;
        refs.div_2wr = rref.g.div_2w;
        refs.div_2hr = rref.g.div_2h;
        refs.n8_r = static_cast<long>(rref.g.cols8) * rref.g.rows8;
        refs.status = b.status;
        const bool inside = cu_x + S <= g.W8 && cu_y + S <= g.H8;
        const dev::Rule ru = dev::derive_rule(g, refs, d, cu_x, cu_y);
        cx = static_cast<int16_t>(ru.cx);
        cy = static_cast<int16_t>(ru.cy);
        leaf = inside && ru.allowed_leaf;
        splitok = d < C::DMAX && (!inside || ru.allowed_split);
    }
    if (mine) {
        s_leaf[tid] = leaf;
        s_splitok[tid] = splitok;
    }
    __syncthreads();

    // reachability (every ancestor may split) and the rule flags
    uint8_t f = 0;
    const int cxl = li % n, cyl = li / n;
    if (present) {
        f = dev::kPresent;
        bool reach = true;
        for (int e = 0; e < d; ++e)
            reach = reach && s_splitok[dev::key_index(e, (cyl >> (d - e)) * (1 << e) + (cxl >> (d - e)))];
        if (reach) f |= kRuleReachable;
        if (reach && s_leaf[tid]) f |= kRuleEvaluated;
        if (reach && s_splitok[tid]) f |= kRuleCanSplit;
    }
    const uint32_t ctr = static_cast<uint32_t>(static_cast<uint16_t>(cx)) |
                         (static_cast<uint32_t>(static_cast<uint16_t>(cy)) << 16);
    if (mine) {
        s_ev[tid] = f & kRuleEvaluated;
        s_ctr[tid] = ctr;
    }
    __syncthreads();
    // a CU searched in pieces whose four sub-CUs are evaluated around its own
    // centre: its SADs are the sums of theirs (the same candidates over four
    // disjoint quarters of its samples)
    if (b.inherit && (f & kRuleEvaluated) && S > b.range && d < C::DMAX) {
        bool all = true;
        for (int q = 0; q < 4; ++q) {
            const int ci = dev::key_index(d + 1, (2 * cyl + (q >> 1)) * (2 * n) + 2 * cxl + (q & 1));
            all = all && s_ev[ci] && s_ctr[ci] == ctr;
        }
        if (all) f |= kRuleInherited;
    }
    const int c = C::DMAX - d;  // size class: CU size 8 << c
    // an inherited CU whose sub-CUs are single pieces takes a table that their
    // lanes add into; one whose sub-CUs have tables of their own has none: the
    // decisions add the four sub-CUs' tables entry by entry
    const bool inh_table = (f & kRuleInherited) && (S >> 1) <= b.range;
    if ((f & kRuleEvaluated) && (!(f & kRuleInherited) || inh_table))
        atomicAdd(&s_cnt[(f & kRuleInherited) ? kSizeClasses + c : c], 1u);
    const long nk_frame = static_cast<long>(g.ctu_cols) * g.ctu_rows * NK;  // key slots of the frame
    if (mine && in_range(b.status, kbase + tid, nk_frame)) {
        reinterpret_cast<int16_t *>(a.block + rinf.off.dep_cx)[kbase + tid] = cx;
        reinterpret_cast<int16_t *>(a.block + rinf.off.dep_cy)[kbase + tid] = cy;
        reinterpret_cast<uint8_t *>(a.block + rinf.off.dep_flags)[kbase + tid] = f;
        reinterpret_cast<unsigned long long *>(a.block + rinf.off.keys)[kbase + tid] = ~0ull;
    }
    __syncthreads();
    if (tid < 2 * kSizeClasses) {
        const int cl = tid % kSizeClasses;
        const unsigned int cnt = s_cnt[tid];
        unsigned int base = 0;
        if (cnt) base = atomicAdd(&b.counts[tid], cnt);
        if (cnt && base + cnt > b.cap[cl]) atomicExch(b.status, kStatusTaskOverflow);
        s_base[tid] = base;
        s_cnt[tid] = 0;
        // the SAD-candidate evaluations (8x8 blocks x candidates) searched for
        // this CTU's tasks of class tid
        if (tid < kSizeClasses && cnt && b.evals) {
            const unsigned long long K = 2 * b.r + 1;
            atomicAdd(b.evals, (static_cast<unsigned long long>(cnt) << (2 * tid)) * K * K);
        }
    }
    __syncthreads();

    // a searched CU's task: item | key slot << 8, centre in the high word; its
    // origin.  An inherited CU with a table: a slot from the top of the class's
    // room (without one: none, -1).
    int pos = -1;
    if (f & kRuleEvaluated) {
        if (f & kRuleInherited) {
            if (inh_table) {
                const unsigned int k = s_base[kSizeClasses + c] + atomicAdd(&s_cnt[kSizeClasses + c], 1u);
                if (k < b.cap[c]) pos = static_cast<int>(b.cap[c] - 1 - k);
            }
        } else {
            const unsigned int p = s_base[c] + atomicAdd(&s_cnt[c], 1u);
            if (p < b.cap[c]) {
                const uint32_t lo = static_cast<uint32_t>(ri) | (static_cast<uint32_t>(kbase + tid) << 8);
                b.tasks[c][p] = (static_cast<unsigned long long>(ctr) << 32) | lo;
                b.pos[c][p] = static_cast<unsigned int>(cu_x) | (static_cast<unsigned int>(cu_y) << 16);
                pos = static_cast<int>(p);
            }
        }
    }
    if (mine && in_range(b.status, kbase + tid, nk_frame)) reinterpret_cast<int *>(a.block + rinf.off.dep_slot)[kbase + tid] = pos;
    if (mine) {
        s_pos[tid] = pos;
        s_inh[tid] = (f & kRuleInherited) ? 1 : 0;
    }
    __syncthreads();
    // a searched CU's inherited parent with a table: its lanes add their SADs
    // into that table too.  Only single-piece CUs have one (an inherited
    // parent of CUs with tables has none), and the chain ends there: an
    // inherited CU has a table, so an inherited grandparent has none.
    if ((f & kRuleEvaluated) && !(f & kRuleInherited) && pos >= 0 && c >= kFirstUpClass && c < kSizeClasses - 1 &&
        c < C::DMAX) {
        uint32_t up = kNoUp;
        const int pi = dev::key_index(d - 1, (cyl >> 1) * (n >> 1) + (cxl >> 1));
        if (s_inh[pi] && s_pos[pi] >= 0) up = static_cast<uint32_t>(s_pos[pi]);
        b.up[c][pos] = up;
    }
    if (tid < NBIG) s_big[tid] = S > b.range ? pos : -1;
    __syncthreads();
    // zeroed sum tables of the CUs searched in pieces and of the inherited ones
    const int KK = (2 * b.r + 1) * (2 * b.r + 1);
    for (int i = 0; i < NBIG; ++i) {
        if (s_big[i] < 0) continue;
        const int cls = C::DMAX - depth_of(i, C::DMAX);
        if (!in_range(b.status, s_big[i], b.cap[cls])) continue;
        unsigned int *sum = b.sums[cls] + static_cast<long>(s_big[i]) * KK;
        for (int k = tid; k < KK; k += kRulesThreads) sum[k] = 0;
    }
}

// ---- 2. search --------------------------------------------------------------
__device__ __forceinline__ uint32_t umad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t umulhi(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// (hi:lo) >> (32 - log2(m)) for m = 2^(32 - s), s in {8, 16, 24, 32}: the
// word that starts s bits into lo, on the multiply-add pipe.
__device__ __forceinline__ uint32_t shift_in(uint32_t lo, uint32_t hi, uint32_t m)
{
    return umad(hi, m, umulhi(lo, m));
}

__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// ---- block SADs --------------------------------------------------------------
// A lane's work per column of NBV stacked 8x8 current blocks: the SADs of the
// TY candidates (x, y + i), i < TY, in row-major order over the window rows
// y .. y + 8 NBV + TY - 2, so each reference row is fetched once and used by
// every candidate it overlaps.  The row fetch is a functor: the fast one reads
// aligned words and shifts them on the multiply-add pipe; the frame-edge one
// clamps every sample position into the frame.

// 8-bit: acc[i] += sum over the column of |cur - ref| at candidate i.
template <int TY, int NBV, typename RowFn>
__device__ __forceinline__ void sads_core_u8(const uint2 (&c)[8 * NBV], RowFn row, uint32_t (&acc)[TY])
{
    constexpr int CR = 8 * NBV, NR = CR + TY - 1;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        uint32_t w0, w1;
        row(r, w0, w1);
        // all candidates on word 0, then on word 1: no back-to-back dependence
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < CR) acc[i] = dev::sad_acc<4>(c[j].x, w0, acc[i]);
        }
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < CR) acc[i] = dev::sad_acc<4>(c[j].y, w1, acc[i]);
        }
    }
}

// 10-bit, one block: SAD = sum(a) + sum(b) - 2 sum(min(a, b)) per packed
// half; sa = packed sums of the current block's (even, odd) columns.
template <int TY, typename RowFn>
__device__ __forceinline__ void sads_core_u16(const uint4 (&c)[8], uint32_t sa, uint32_t one, RowFn row,
                                              uint32_t (&acc)[TY])
{
    constexpr int NR = 8 + TY - 1;
    uint32_t mn[TY];
#pragma unroll
    for (int i = 0; i < TY; ++i) mn[i] = 0;
    uint32_t rs[NR];
    uint32_t sb = 0;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        uint32_t w0, w1, w2, w3;
        row(r, w0, w1, w2, w3);
        rs[r] = umad(w0, one, w1) + umad(w2, one, w3);
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < 8) mn[i] = umad(min_u16x2(c[j].x, w0), one, mn[i]);
        }
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < 8) mn[i] = umad(min_u16x2(c[j].y, w1), one, mn[i]);
        }
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < 8) mn[i] = umad(min_u16x2(c[j].z, w2), one, mn[i]);
        }
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < 8) mn[i] = umad(min_u16x2(c[j].w, w3), one, mn[i]);
        }
        if (r < 8) sb += rs[r];
        else sb = sb + rs[r] - rs[r - 8];
        if (r >= 7) {
            const int i = r - 7;  // candidate i is complete
            const uint32_t d = umad(mn[i], 0xfffffffeu, sa + sb);
            acc[i] += (d & 0xffffu) + (d >> 16);
        }
    }
}

// Frame-edge columns (8-bit).  Reference: the clamped positions
// p_e = clamp(x + e, 0, W - 1), e < 8, lie within 8 bytes of p_0, so each
// row is three aligned words (word indices capped at the row's last
// sample), one funnel shift to p_0 and a byte permute.  Rows clamp into
// [0, H).  Current: rows and columns clamp into the frame (replication
// into the 8-aligned pad).  Writes the column's SADs to out[i].
template <int TY, int NBV>
__device__ __noinline__ void column_sads_edge_u8(const char *cur, const char *ref, long pitch, int W, int H, int bx,
                                                 int by, int x, int y, uint32_t *out)
{
    constexpr int CR = 8 * NBV;
    const int p0 = min(max(x, 0), W - 1);
    const int q = p0 >> 2, qmax = (W - 1) >> 2, q1 = min(q + 1, qmax), q2 = min(q + 2, qmax);
    const uint32_t sh = 8u * static_cast<uint32_t>(p0 & 3);
    uint32_t rsel0 = 0, rsel1 = 0, csel0 = 0, csel1 = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        rsel0 |= static_cast<uint32_t>(min(max(x + e, 0), W - 1) - p0) << (4 * e);
        rsel1 |= static_cast<uint32_t>(min(max(x + 4 + e, 0), W - 1) - p0) << (4 * e);
        csel0 |= static_cast<uint32_t>(min(bx + e, W - 1) - bx) << (4 * e);
        csel1 |= static_cast<uint32_t>(min(bx + 4 + e, W - 1) - bx) << (4 * e);
    }
    uint2 c[CR];
#pragma unroll
    for (int j = 0; j < CR; ++j) {
        // bx + 8 <= W8 <= pitch: the aligned 8-byte load stays inside the row
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(cur + static_cast<long>(min(by + j, H - 1)) * pitch + bx));
        c[j].x = __byte_perm(v.x, v.y, csel0);
        c[j].y = __byte_perm(v.x, v.y, csel1);
    }
    uint32_t acc[TY];
#pragma unroll
    for (int i = 0; i < TY; ++i) acc[i] = 0;
    sads_core_u8<TY, NBV>(c, [&](int r, uint32_t &w0, uint32_t &w1) {
        const uint32_t *rp = reinterpret_cast<const uint32_t *>(ref + static_cast<long>(min(max(y + r, 0), H - 1)) * pitch);
        const uint32_t a0 = __ldg(rp + q), a1 = __ldg(rp + q1), a2 = __ldg(rp + q2);
        const uint32_t v0 = __funnelshift_r(a0, a1, sh), v1 = __funnelshift_r(a1, a2, sh);
        w0 = __byte_perm(v0, v1, rsel0);
        w1 = __byte_perm(v0, v1, rsel1);
    }, acc);
#pragma unroll
    for (int i = 0; i < TY; ++i) out[i] = acc[i];
}

// Frame-edge blocks (10-bit): samples gathered one by one at clamped
// positions (columns once per block, rows once per row).
template <int TY>
__device__ __noinline__ void block_sads_edge_u16(const char *cur, const char *ref, long pitch, int W, int H, int bx,
                                                 int by, int x, int y, uint32_t one, uint32_t *out)
{
    int cc[8], rc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        cc[e] = min(bx + e, W - 1);
        rc[e] = min(max(x + e, 0), W - 1);
    }
    uint4 c[8];
    uint32_t sa = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint16_t *row = reinterpret_cast<const uint16_t *>(cur + static_cast<long>(min(by + j, H - 1)) * pitch);
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            w[k] = static_cast<uint32_t>(__ldg(row + cc[2 * k])) | (static_cast<uint32_t>(__ldg(row + cc[2 * k + 1])) << 16);
        c[j] = make_uint4(w[0], w[1], w[2], w[3]);
        sa += (w[0] + w[1]) + (w[2] + w[3]);
    }
    uint32_t acc[TY];
#pragma unroll
    for (int i = 0; i < TY; ++i) acc[i] = 0;
    sads_core_u16<TY>(c, sa, one, [&](int r, uint32_t &w0, uint32_t &w1, uint32_t &w2, uint32_t &w3) {
        const uint16_t *row = reinterpret_cast<const uint16_t *>(ref + static_cast<long>(min(max(y + r, 0), H - 1)) * pitch);
        w0 = static_cast<uint32_t>(__ldg(row + rc[0])) | (static_cast<uint32_t>(__ldg(row + rc[1])) << 16);
        w1 = static_cast<uint32_t>(__ldg(row + rc[2])) | (static_cast<uint32_t>(__ldg(row + rc[3])) << 16);
        w2 = static_cast<uint32_t>(__ldg(row + rc[4])) | (static_cast<uint32_t>(__ldg(row + rc[5])) << 16);
        w3 = static_cast<uint32_t>(__ldg(row + rc[6])) | (static_cast<uint32_t>(__ldg(row + rc[7])) << 16);
    }, acc);
#pragma unroll
    for (int i = 0; i < TY; ++i) out[i] = acc[i];
}

// Adds the SADs of the 8-wide, 8*NBV-high column of current blocks at
// (bx, by) for the TY candidates (x, y + i), i < TY, to acc (8-bit samples).
template <int TY, int NBV>
__device__ __forceinline__ void block_sads_u8(const char *cur, const char *ref, long pitch, int W, int H, int bx,
                                              int by, int x, int y, uint32_t (&acc)[TY])
{
    constexpr int CR = 8 * NBV, NR = CR + TY - 1;
    const int q = (x - 1) >> 2;  // words q .. q+2 hold samples x .. x+7
    const bool fast = bx + 8 <= W && x >= 1 && 4 * q + 12 <= W && y >= 0 && y + NR <= H;
    if (!fast) {
        uint32_t e[TY];
        column_sads_edge_u8<TY, NBV>(cur, ref, pitch, W, H, bx, by, x, y, e);
#pragma unroll
        for (int i = 0; i < TY; ++i) acc[i] += e[i];
        return;
    }
    uint2 c[CR];
#pragma unroll
    for (int j = 0; j < CR; ++j)
        c[j] = __ldg(reinterpret_cast<const uint2 *>(cur + static_cast<long>(min(by + j, H - 1)) * pitch + bx));
    const uint32_t m = 1u << (32 - 8 * (x - 4 * q));  // x - 4q in 1..4
    const uint32_t *rp = reinterpret_cast<const uint32_t *>(ref + static_cast<long>(y) * pitch) + q;
    const long wp = pitch / 4;
    sads_core_u8<TY, NBV>(c, [&](int r, uint32_t &w0, uint32_t &w1) {
        const uint32_t a0 = __ldg(rp + r * wp), a1 = __ldg(rp + r * wp + 1), a2 = __ldg(rp + r * wp + 2);
        w0 = shift_in(a0, a1, m);
        w1 = shift_in(a1, a2, m);
    }, acc);
}

// 10-bit samples, one 8x8 block.
template <int TY>
__device__ __forceinline__ void block_sads_u16(const char *cur, const char *ref, long pitch, int W, int H, int bx,
                                               int by, int x, int y, uint32_t one, uint32_t (&acc)[TY])
{
    constexpr int NR = 8 + TY - 1;
    const int q = (x - 1) >> 1;  // words q .. q+4 hold samples x .. x+7
    const bool fast = bx + 8 <= W && x >= 1 && 2 * q + 10 <= W && y >= 0 && y + NR <= H;
    if (!fast) {
        uint32_t e[TY];
        block_sads_edge_u16<TY>(cur, ref, pitch, W, H, bx, by, x, y, one, e);
#pragma unroll
        for (int i = 0; i < TY; ++i) acc[i] += e[i];
        return;
    }
    uint4 c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        c[j] = __ldg(reinterpret_cast<const uint4 *>(cur + static_cast<long>(min(by + j, H - 1)) * pitch + 2 * bx));
    uint32_t sa = 0;  // packed sums of the current block's even / odd columns
#pragma unroll
    for (int j = 0; j < 8; ++j) sa += (c[j].x + c[j].y) + (c[j].z + c[j].w);
    const uint32_t m = (x - 2 * q == 1) ? (1u << 16) : 1u;
    const uint32_t *rp = reinterpret_cast<const uint32_t *>(ref + static_cast<long>(y) * pitch) + q;
    const long wp = pitch / 4;
    sads_core_u16<TY>(c, sa, one, [&](int r, uint32_t &w0, uint32_t &w1, uint32_t &w2, uint32_t &w3) {
        const uint32_t a0 = __ldg(rp + r * wp), a1 = __ldg(rp + r * wp + 1), a2 = __ldg(rp + r * wp + 2),
                       a3 = __ldg(rp + r * wp + 3), a4 = __ldg(rp + r * wp + 4);
        w0 = shift_in(a0, a1, m);
        w1 = shift_in(a1, a2, m);
        w2 = shift_in(a2, a3, m);
        w3 = shift_in(a3, a4, m);
    }, acc);
}

// Bits of the largest SAD of an S x S CU.
__device__ __forceinline__ int sad_bits(int S, int bit_depth)
{
    return (S == 8 ? 6 : S == 16 ? 8 : S == 32 ? 10 : 12) + bit_depth;
}

// The table slot of the inherited parent of task u of class c (kNoUp: none;
// kRuleInherited).
__device__ __forceinline__ uint32_t parent_slot(const DependentBatch &b, int c, unsigned int u)
{
    return (c >= kFirstUpClass && c < kSizeClasses - 1 && b.inherit) ? __ldcg(b.up[c] + u) : kNoUp;
}

// A searched CU's lane adds its candidates' SADs into the table of the CU's
// inherited parent (slot from parent_slot), every candidate once: no padding
// lanes (the caller's), no rows a clamped band shares with the band before
// it, no rows past +r.
template <int TY>
__device__ __forceinline__ void add_to_parent(const DependentBatch &b, int c, uint32_t slot, int dxi, int dy0, int b0,
                                              const uint32_t (&acc)[TY])
{
    if (slot == kNoUp || !in_range(b.status, slot, b.cap[c + 1])) return;
    const int r = b.r, K = 2 * r + 1;
    unsigned int *sum = b.sums[c + 1] + static_cast<long>(slot) * (K * K);
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        const int dyo = dy0 + i;
        if (dyo >= b0 && dyo <= r && in_range(b.status, (dyo + r) * K + dxi, K * K))
            atomicAdd(sum + (dyo + r) * K + dxi, acc[i]);
    }
}

template <typename T, int TY>
__device__ __forceinline__ void search_tile(const DependentBatch &b, int c, int lt, unsigned int ncu, int per_cu,
                                            const FastDiv &div_cu, const FastDiv &div_k, int rb, int lane)
{
    const int r = b.r, K = 2 * r + 1;
    // CUs larger than the range are searched as range x range pieces
    const int S = 8 << c, RS = S < b.range ? S : b.range;
    const int nrs = S / RS, nr = nrs * nrs;
    const int per_task = nr * per_cu;  // lanes of one CU
    const long ntask = static_cast<long>(ncu) * per_task;
    const long traw = static_cast<long>(lt) * 32 + lane;
    const long t = min(traw, ntask - 1);
    // lane t of the class = ((CU u, piece rg), band, dxi): t / per_cu = u * nr + rg (nr a power of 4)
    const uint32_t q = t <= 0xffffffffL ? fast_div(static_cast<uint32_t>(t), div_cu)
                                        : static_cast<uint32_t>(t / per_cu);
    const unsigned int u = q >> (2 * (31 - __clz(nrs)));
    const int rg = static_cast<int>(q & static_cast<uint32_t>(nr - 1));
    const int rem = static_cast<int>(t - static_cast<long>(q) * per_cu);
    const int band = static_cast<int>(fast_div(static_cast<uint32_t>(rem), div_k)), dxi = rem - band * K;
    if (!in_range(b.status, u, b.cap[c])) return;  // (debug builds) a lane's CU lies in its task list
    const unsigned long long task = __ldcg(b.tasks[c] + u);
    const uint32_t lo = static_cast<uint32_t>(task), hi = static_cast<uint32_t>(task >> 32);
    const DependentItem &a = b.item[lo & 0xffu];
    const RungInfo &rinf = b.rung[a.rung];
    const RungGeom &g = rinf.g;
    const unsigned int p = __ldcg(b.pos[c] + u);
    const int cu_x = static_cast<int>(p & 0xffffu) + (rg % nrs) * RS;  // this piece's origin
    const int cu_y = static_cast<int>(p >> 16) + (rg / nrs) * RS;
    const int cx = static_cast<int16_t>(hi & 0xffffu), cy = static_cast<int16_t>(hi >> 16);
    const int dxo = dxi - r;  // offsets from the centre
    const int b0 = band * TY - r;
    const int dy0 = K >= TY ? min(b0, r - TY + 1) : b0;

    uint32_t acc[TY];
#pragma unroll
    for (int i = 0; i < TY; ++i) acc[i] = 0;
    const char *cur = static_cast<const char *>(a.cur), *ref = static_cast<const char *>(a.ref);
    const int nb = RS / 8;
    if constexpr (sizeof(T) == 1) {
        if (nb >= 2) {
            // columns of two stacked blocks: the candidate rows they share are read once
#pragma unroll 1
            for (int col = 0; col < nb * nb / 2; ++col) {
                const int bx = cu_x + 8 * (col % nb), by = cu_y + 16 * (col / nb);
                block_sads_u8<TY, 2>(cur, ref, a.pitch_bytes, g.W, g.H, bx, by, bx + cx + dxo, by + cy + dy0, acc);
            }
        } else {
            block_sads_u8<TY, 1>(cur, ref, a.pitch_bytes, g.W, g.H, cu_x, cu_y, cu_x + cx + dxo, cu_y + cy + dy0, acc);
        }
    } else {
#pragma unroll 1
        for (int blk = 0; blk < nb * nb; ++blk) {
            const int bx = cu_x + 8 * (blk % nb), by = cu_y + 8 * (blk / nb);
            block_sads_u16<TY>(cur, ref, a.pitch_bytes, g.W, g.H, bx, by, bx + cx + dxo, by + cy + dy0, b.one, acc);
        }
    }

    if (traw < ntask) add_to_parent<TY>(b, c, parent_slot(b, c, u), dxi, dy0, b0, acc);
    if (nr > 1) {
        // add this range's SADs to the CU's table; every candidate exactly
        // once: no padding lanes, no rows a clamped band shares with the
        // band before it, no rows past +r
        if (traw < ntask) {
            unsigned int *sum = b.sums[c] + static_cast<long>(u) * (K * K);
#pragma unroll
            for (int i = 0; i < TY; ++i) {
                const int dyo = dy0 + i;
                if (dyo >= b0 && dyo <= r && in_range(b.status, (dyo + r) * K + dxi, K * K))
                    atomicAdd(sum + (dyo + r) * K + dxi, acc[i]);
            }
        }
        return;
    }

    // keys; candidate rows past +r (only when 2r + 1 < TY) never win.
    // code = (|dx|+|dy|) 2K + 2 (dy + r) + [dx > 0]
    const int bits = sad_bits(S, sizeof(T) == 1 ? 8 : 10);
    const uint32_t cbase = static_cast<uint32_t>(abs(dxo) * 2 * K + 2 * (dy0 + r) + (dxo > 0));
    unsigned long long best = ~0ull;
    if (bits + rb <= 32) {
        uint32_t k = 0xffffffffu;
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int dyo = dy0 + i;
            const bool ok = dyo <= r;
            const uint32_t code = umad(static_cast<uint32_t>(abs(dyo)), 2u * K, cbase + 2u * i);
            k = min(k, umad(acc[i], ok ? (1u << rb) : 0u, ok ? code : 0xffffffffu));
        }
        best = k == 0xffffffffu ? ~0ull : k;
    } else {
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int dyo = dy0 + i;
            if (dyo > r) continue;
            const uint32_t code = umad(static_cast<uint32_t>(abs(dyo)), 2u * K, cbase + 2u * i);
            const unsigned long long key = (static_cast<unsigned long long>(acc[i]) << rb) | code;
            best = key < best ? key : best;
        }
    }
    // segmented min over the lanes of this CU (contiguous: first .. last)
    const long cu_first = static_cast<long>(u) * per_task - static_cast<long>(lt) * 32;
    const int first = static_cast<int>(max(cu_first, 0L));
    const int last = static_cast<int>(min(cu_first + per_task - 1, ntask - 1 - static_cast<long>(lt) * 32));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_down_sync(0xffffffffu, best, o);
        if (lane + o <= last) best = v < best ? v : best;
    }
    if (lane == first && best != ~0ull) {
        const uint32_t sad = static_cast<uint32_t>(best >> rb);
        const int code = static_cast<int>(best & ((1ull << rb) - 1));
        const int l1 = code / (2 * K), rr = code - l1 * 2 * K;
        const int dyv = (rr >> 1) - r;
        const int adx = l1 - abs(dyv);
        const int dxv = (rr & 1) ? adx : -adx;
        const uint32_t tb = static_cast<uint32_t>(l1 * K * K + (dyv + r) * K + (dxv + r));
        unsigned long long *keys = reinterpret_cast<unsigned long long *>(a.block + rinf.off.keys);
        const long nk = static_cast<long>(rinf.g.ctu_cols) * rinf.g.ctu_rows * keys_per_ctu(rinf.g.dmax);
        if (in_range(b.status, lo >> 8, nk)) atomicMin(keys + (lo >> 8), (static_cast<unsigned long long>(sad) << 32) | tb);
    }
}

template <typename T, int TY>
__global__ void __launch_bounds__(kSearchThreads, 2)
    k_dep_search(const __grid_constant__ DependentBatch b, const FastDiv div_cu, const FastDiv div_k)
{
    dev::chain_entry();
    const int lane = threadIdx.x & 31;
    const int r = b.r, K = 2 * r + 1;
    const int per_cu = K * ((K + TY - 1) / TY);
    const int code_max = 4 * r * K + 4 * r + 1;
    const int rb = 32 - __clz(code_max);
    // per size class: CUs and warp tiles (scalars: no local-memory arrays)
    const unsigned int n0 = min(__ldcg(b.counts + 0), b.cap[0]), n1 = min(__ldcg(b.counts + 1), b.cap[1]),
                       n2 = min(__ldcg(b.counts + 2), b.cap[2]), n3 = min(__ldcg(b.counts + 3), b.cap[3]);
    // lanes per CU: per_cu per piece (pieces of 32x32 / 64x64 CUs: (S / range)^2)
    const long p2 = b.range >= 32 ? 1 : 4, p3 = b.range >= 32 ? 4 : 16;
    const long t0 = (static_cast<long>(n0) * per_cu + 31) / 32, t1 = (static_cast<long>(n1) * per_cu + 31) / 32,
               t2 = (static_cast<long>(n2) * p2 * per_cu + 31) / 32, t3 = (static_cast<long>(n3) * p3 * per_cu + 31) / 32;
    const long total = t0 + t1 + t2 + t3;
    const long nwarps = static_cast<long>(gridDim.x) * (kSearchThreads / 32);
#pragma unroll 1
    // consecutive tiles go to different CTAs (SMs): the long tiles of large
    // CUs come first and spread over the whole GPU
    for (long w = static_cast<long>(threadIdx.x >> 5) * gridDim.x + blockIdx.x; w < total; w += nwarps) {
        long lt = w;
        int c;
        unsigned int ncu;
        if (lt < t3) {
            c = 3;
            ncu = n3;
        } else if ((lt -= t3) < t2) {
            c = 2;
            ncu = n2;
        } else if ((lt -= t2) < t1) {
            c = 1;
            ncu = n1;
        } else {
            lt -= t1;
            c = 0;
            ncu = n0;
        }
        search_tile<T, TY>(b, c, static_cast<int>(lt), ncu, per_cu, div_cu, div_k, rb, lane);
    }
}

// ---- 2b. staged search ------------------------------------------------------
// A CTA takes tiles of kStageThreads consecutive lane tasks of one size
// class.  The lanes of a CU piece are contiguous, so a tile touches a few
// pieces.  Each piece's reference window (every row and column its
// candidates read) and its current samples are staged in shared memory
// first, with the frame-edge rules applied there once (reference rows and
// columns clamped into the frame, current samples replicated into the
// 8-aligned pad).  10-bit (ES = 2):
//   raw0  the window's rows from an 8-sample-aligned column ax, sample
//         pairs (s[ax + 2m], s[ax + 2m + 1]) per word (16-byte async copies
//         of whole row chunks when the window lies inside the frame);
//   raw1  the same rows shifted by one sample, (s[ax + 2m + 1], s[ax + 2m + 2]),
//         built from raw0 in shared memory;
//   cur   the piece's current rows, sample pairs per word.
// A lane whose candidate column starts at an even offset from ax reads its 8
// samples of a row as 4 aligned words of raw0, an odd one as 4 aligned words
// of raw1: no shifts, no frame-edge path and no divergence in the candidate
// loop.  8-bit (ES = 1): raw0 only, from a 16-sample-aligned column ax that
// lies 1..16 samples left of the window; a lane reads 3 aligned words per
// row and shifts them on the multiply-add pipe (as the L1 form does), which
// leaves the ALU pipe to the packed absolute differences.  By default a CTA
// stages into one buffer (several CTAs per SM overlap one another's staging);
// dep_staged = 2 gives it two, the next tile's copies in flight while the
// current tile is computed.
constexpr int kStageThreads = 128;  // small tiles: several CTAs per SM, staging overlaps compute
constexpr int kMaxStageSlots = 32;  // pieces one tile may touch (lanes per piece >= 9)

// Shared-memory layout of one staged piece (words).
struct StageShape {
    int RS;    // piece side
    int WR;    // window rows
    int WW;    // samples a candidate column may start at past the window's first column, + 1
    int NC;    // 16-byte chunks per raw row
    int RW;    // words per raw row (at least 4 NC, a multiple of 4: rows stay 16-byte aligned)
    int CNC;   // 16-byte chunks per current row
    int CW;    // words per current row (4 CNC)
    int O1;    // offset of raw1 (10-bit)
    int OC;    // offset of the current rows
    int PW;    // words per piece slot (a multiple of 4)
};

template <int ES>
__host__ __device__ inline StageShape stage_shape(int RS, int r, int TY)
{
    StageShape s;
    s.RS = RS;
    // candidate rows reach RS - 1 + r below the piece; a single band taller
    // than 2r + 1 reads TY - 1 - r rows further (those candidates are dropped)
    s.WR = RS + (2 * r > TY - 1 ? 2 * r : TY - 1);
    s.WW = RS + 2 * r - 1;
    if (ES == 2) {
        // the window's first column lies up to 7 samples past ax
        s.NC = (s.WW + 15) / 8;
        // Banks: a warp's lanes read consecutive words, the even-offset ones in
        // raw0, the odd-offset ones in raw1 (16 banks away); with several bands
        // (2r + 1 > TY) a warp also holds a band TY rows lower, and a row stride
        // of 8 (mod 16) words puts its words beside the first band's.
        s.RW = 2 * r + 1 > TY ? ((4 * s.NC + 7) & ~15) + 8 : 4 * s.NC;
        s.CNC = RS / 8;
        s.CW = RS / 2;
        s.O1 = ((s.WR * s.RW + 15) & ~31) + 16;
        s.OC = (s.O1 + s.WR * s.RW + 3) & ~3;
        s.PW = (s.OC + RS * s.CW + 3) & ~3;
    } else {
        // the window's first column lies 1..16 samples past ax; a lane's last
        // word of a row ends at most RS + 2r + 18 samples past ax
        s.NC = (RS + 2 * r + 19 + 15) / 16;
        s.RW = 2 * r + 1 > TY ? ((4 * s.NC + 7) & ~15) + 8 : 4 * s.NC;
        // current rows from a 16-sample-aligned column (an 8x8 CU's 8 samples
        // lie in the first or second half of its chunk)
        s.CNC = (RS + 15) / 16;
        s.CW = 4 * s.CNC;
        s.O1 = 0;
        s.OC = (s.WR * s.RW + 3) & ~3;
        // slots 8 (mod 32) words apart: the (up to four) pieces a warp holds
        // read different banks
        s.PW = ((s.OC + RS * s.CW + 23) & ~31) + 8;
    }
    return s;
}

// Pieces a tile of kStageThreads lane tasks may touch, per_cu lanes each.
__host__ __device__ inline int stage_slots(int per_cu) { return (kStageThreads - 1) / per_cu + 2; }

// Divisors of the staging loops, one per size class (host-made).
struct StageDivs {
    FastDiv cps[kSizeClasses];   // copy columns per slot: row groups x (reference + current chunks per row)
    FastDiv c1[kSizeClasses];    // shift columns per slot: row groups x reference chunks per row
};

__device__ __forceinline__ void cp_async16(uint32_t *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dev::smem_addr(dst)), "l"(src) : "memory");
}

// 10-bit SADs of one 8x8 current block for the TY candidates of a lane over
// its staged window rows: sum(a) + sum(b) - 2 sum(min(a, b)) per packed half
// (see sads_core_u16).  Candidate i's word starts at sum(a) and takes
// -2 min(a, b) per sample pair on the multiply-add pipe (m2 = -2, a runtime
// value); sum(b) over its rows i..i+7 is the difference of two prefixes P of
// the packed row sums, added at its last row; one dp2a folds the halves.
// Everything is modulo 2^32: each half of the final word is that half's
// sum of |a - b| (at most 32 * 1023), so the wrap-arounds in between cancel.
// ep: the lane's first word of its first row; words 0, 1, 2, 3 hold its 8
// samples.
template <int TY>
__device__ __forceinline__ void sads_staged_u16(const uint4 (&c)[8], uint32_t sa, uint32_t m2, const uint32_t *ep,
                                                int rw, uint32_t (&acc)[TY])
{
    constexpr int NR = 8 + TY - 1;
    uint32_t x[TY];
#pragma unroll
    for (int i = 0; i < TY; ++i) x[i] = sa;
    uint32_t pf[NR + 1];  // pf[r + 1]: packed sum of rows 0..r
    pf[0] = 0;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const uint32_t *q = ep + r * rw;
        const uint32_t w0 = q[0], w1 = q[1], w2 = q[2], w3 = q[3];
        pf[r + 1] = (pf[r] + w0 + w1) + (w2 + w3);
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < 8) x[i] = umad(min_u16x2(c[j].x, w0), m2, x[i]);
        }
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < 8) x[i] = umad(min_u16x2(c[j].y, w1), m2, x[i]);
        }
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < 8) x[i] = umad(min_u16x2(c[j].z, w2), m2, x[i]);
        }
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = r - i;
            if (j >= 0 && j < 8) x[i] = umad(min_u16x2(c[j].w, w3), m2, x[i]);
        }
        if (r >= 7) {
            const int i = r - 7;  // candidate i is complete
            acc[i] = __dp2a_lo(x[i] + (pf[r + 1] - pf[i]), 0x0101u, acc[i]);
        }
    }
}

// One tile of the staged search: its size class, its lane tasks and the
// pieces they touch.
struct StageTile {
    int c;          // size class
    long tf, ntask; // first lane task of the tile, lane tasks of the class
    uint32_t q0;    // first piece
    int nslots;     // pieces touched
    int RS, nrs, nr, lg;
    StageShape sh;
};

// Per-slot parameters of the pieces staged in one buffer.
struct StageSlots {
    const char *ref[kMaxStageSlots], *cur[kMaxStageSlots];
    long pitch[kMaxStageSlots];
    int W[kMaxStageSlots], H[kMaxStageSlots], wy0[kMaxStageSlots], ax[kMaxStageSlots];
    int off[kMaxStageSlots], cux[kMaxStageSlots], cuy[kMaxStageSlots], edge[kMaxStageSlots];
    int coff[kMaxStageSlots];  // the piece's first current column past its staged chunk (8-bit: 0 or 8)
    int any_edge;  // some slot needs the frame-edge fix-up
};

template <int ES, int TY>
__device__ __forceinline__ StageTile stage_tile(const DependentBatch &b, long tile, int per_cu, const FastDiv &div_cu,
                                                const long *ln, const long *tn)
{
    StageTile t;
    long lt = tile;
    int c = 3;
    while (c > 0 && lt >= tn[c]) lt -= tn[c--];  // largest CUs first
    t.c = c;
    t.ntask = ln[c];
    t.tf = lt * kStageThreads;
    const int S = 8 << c;
    t.RS = S < b.range ? S : b.range;
    t.nrs = S / t.RS;
    t.nr = t.nrs * t.nrs;
    t.lg = 31 - __clz(t.nrs);
    t.sh = stage_shape<ES>(t.RS, b.r, TY);
    const long tl = min(t.tf + kStageThreads - 1, t.ntask - 1);
    t.q0 = fast_div(static_cast<uint32_t>(t.tf), div_cu);
    t.nslots = static_cast<int>(fast_div(static_cast<uint32_t>(tl), div_cu) - t.q0) + 1;
    return t;
}

// The tile's pieces: planes, window origin, frame-edge flags (threads
// below nslots, one piece each).
template <int ES>
__device__ __forceinline__ void stage_slots_setup(const DependentBatch &b, const StageTile &t, StageSlots &ss)
{
    constexpr int CS = 16 / ES;  // samples per 16-byte chunk
    const int tid = threadIdx.x;
    if (tid == 0) ss.any_edge = 0;
    __syncthreads();
    if (tid < t.nslots) {
        const uint32_t q = t.q0 + tid;
        const unsigned int u = q >> (2 * t.lg);
        const int rg = static_cast<int>(q & static_cast<uint32_t>(t.nr - 1));
        const unsigned long long task = __ldcg(b.tasks[t.c] + u);
        const uint32_t hi = static_cast<uint32_t>(task >> 32);
        const unsigned int p = __ldcg(b.pos[t.c] + u);
        const DependentItem &a = b.item[static_cast<uint32_t>(task) & 0xffu];
        const RungGeom &g = b.rung[a.rung].g;
        const int cux = static_cast<int>(p & 0xffffu) + (rg % t.nrs) * t.RS;
        const int cuy = static_cast<int>(p >> 16) + (rg / t.nrs) * t.RS;
        const int wx0 = cux + static_cast<int16_t>(hi & 0xffffu) - b.r;
        // 10-bit: the 8-aligned column at or left of the window; 8-bit: the
        // 16-aligned column 1..16 samples left of it (a lane's first word
        // then starts left of its first sample)
        const int ax = ES == 2 ? (wx0 & ~7) : ((wx0 - 1) & ~15);
        const int cx0 = cux & ~(CS - 1);
        ss.ref[tid] = static_cast<const char *>(a.ref);
        ss.cur[tid] = static_cast<const char *>(a.cur);
        ss.pitch[tid] = a.pitch_bytes;
        ss.W[tid] = g.W;
        ss.H[tid] = g.H;
        ss.wy0[tid] = cuy + static_cast<int16_t>(hi >> 16) - b.r;
        ss.ax[tid] = ax;
        ss.off[tid] = wx0 - ax;
        ss.cux[tid] = cux;
        ss.cuy[tid] = cuy;
        ss.coff[tid] = cux - cx0;
        // bit 0: a raw word holds a sample outside the frame's columns;
        // bit 1: a staged current word passes the frame's right edge
        const int e = ((ax < 0 || ax + CS * t.sh.NC > g.W) ? 1 : 0) | (cx0 + CS * t.sh.CNC > g.W ? 2 : 0);
        ss.edge[tid] = e;
        if (e) ss.any_edge = 1;
    }
}

// Issues the async copies of every 16-byte chunk of the tile's raw0 and
// current rows that lies inside its frame (rows clamped into the frame);
// chunks outside are left to the fix-up.  A thread takes one column of
// chunks (slot, chunk, every fourth row from its row group) and walks its
// rows.  Interleaved rows put the four row groups of a chunk column
// RW, 2 RW and 3 RW words apart, in different banks for the row pitches
// the shapes give (a contiguous quarter of the rows each would put them a
// multiple of 32 words apart: four-way bank conflicts).
constexpr int kStageRowGroups = 4;

template <int ES>
__device__ __forceinline__ void stage_copy(const StageTile &t, const StageSlots &ss, uint32_t *buf,
                                           const FastDiv &div_cps)
{
    constexpr int CS = 16 / ES;  // samples per 16-byte chunk
    const StageShape &sh = t.sh;
    const int cps = kStageRowGroups * (sh.NC + sh.CNC);  // columns per slot
#pragma unroll 1
    for (int col = threadIdx.x; col < t.nslots * cps; col += kStageThreads) {
        const int slot = static_cast<int>(fast_div(static_cast<uint32_t>(col), div_cps));
        const int k = col - slot * cps;
        const int grp = k & (kStageRowGroups - 1), ch = k / kStageRowGroups;
        const int W = ss.W[slot], H = ss.H[slot];
        const long pitch = ss.pitch[slot];
        const bool ref = ch < sh.NC;
        const int x = ref ? ss.ax[slot] + CS * ch : ss.cux[slot] - ss.coff[slot] + CS * (ch - sh.NC);
        if (x < 0 || x >= W) continue;  // x is a multiple of CS: a chunk that starts in the row ends in its pitch
        const int rows = ref ? sh.WR : t.RS;
        const int y0 = (ref ? ss.wy0[slot] : ss.cuy[slot]) + grp;
        const char *src = (ref ? ss.ref[slot] : ss.cur[slot]) + ES * static_cast<long>(x);
        const int stride = ref ? sh.RW : sh.CW;
        uint32_t *dst = buf + slot * sh.PW + (ref ? 0 : sh.OC) + grp * stride + 4 * (ref ? ch : ch - sh.NC);
#pragma unroll 1
        for (int i = 0; grp + i < rows; i += kStageRowGroups, dst += kStageRowGroups * stride)
            cp_async16(dst, src + static_cast<long>(min(max(y0 + i, 0), H - 1)) * pitch);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Frame edges: every raw0 word with a sample outside the frame's columns,
// and every current word past its right edge, from clamped samples (edge
// slots only; one warp per row).
template <int ES>
__device__ __forceinline__ void stage_fixup(const StageTile &t, const StageSlots &ss, uint32_t *buf)
{
    using T = typename std::conditional<ES == 1, uint8_t, uint16_t>::type;
    constexpr int SPW = 4 / ES;  // samples per word
    const StageShape &sh = t.sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kStageThreads / 32;
#pragma unroll 1
    for (int slot = 0; slot < t.nslots; ++slot) {
        const int e = ss.edge[slot];
        if (!e) continue;
        const int W = ss.W[slot];
#pragma unroll 1
        for (int row = warp; row < sh.WR + t.RS; row += kWarps) {
            const bool ref_row = row < sh.WR;
            if (ref_row ? !(e & 1) : !(e & 2)) continue;
            const int y = ref_row ? min(max(ss.wy0[slot] + row, 0), ss.H[slot] - 1)
                                  : min(ss.cuy[slot] + row - sh.WR, ss.H[slot] - 1);
            const T *src = reinterpret_cast<const T *>((ref_row ? ss.ref[slot] : ss.cur[slot]) +
                                                       static_cast<long>(y) * ss.pitch[slot]);
            uint32_t *dst = buf + slot * sh.PW + (ref_row ? row * sh.RW : sh.OC + (row - sh.WR) * sh.CW);
            const int x0 = ref_row ? ss.ax[slot] : ss.cux[slot] - ss.coff[slot];
            const int nw = ref_row ? 4 * sh.NC : sh.CW;
            for (int m = lane; m < nw; m += 32) {
                const int p = x0 + SPW * m;
                if (p >= 0 && p + SPW - 1 < W) continue;  // copied as it stands
                uint32_t v = 0;
#pragma unroll
                for (int e2 = 0; e2 < SPW; ++e2)
                    v |= static_cast<uint32_t>(__ldg(src + min(max(p + e2, 0), W - 1))) << (8 * ES * e2);
                dst[m] = v;
            }
        }
    }
}

// raw1: every raw row shifted by one sample, four words at a time; a
// thread takes one column (slot, four words, every fourth row from its row
// group, as in the copies).
__device__ __forceinline__ void stage_raw1(const StageTile &t, uint32_t *buf, const FastDiv &div_c1)
{
    const StageShape &sh = t.sh;
    const int cps = kStageRowGroups * sh.NC;
#pragma unroll 1
    for (int col = threadIdx.x; col < t.nslots * cps; col += kStageThreads) {
        const int slot = static_cast<int>(fast_div(static_cast<uint32_t>(col), div_c1));
        const int k = col - slot * cps;
        const int grp = k / kStageRowGroups, row0 = k & (kStageRowGroups - 1);
        const bool last = grp + 1 >= sh.NC;  // the row's last word: never read shifted
        const uint32_t *src = buf + slot * sh.PW + row0 * sh.RW + 4 * grp;
        uint32_t *dst = buf + slot * sh.PW + sh.O1 + row0 * sh.RW + 4 * grp;
        const int step = kStageRowGroups * sh.RW;
#pragma unroll 1
        for (int i = row0; i < sh.WR; i += kStageRowGroups, src += step, dst += step) {
            const uint4 a4 = *reinterpret_cast<const uint4 *>(src);
            const uint32_t e = last ? 0u : src[4];
            uint4 o;
            o.x = __byte_perm(a4.x, a4.y, 0x5432);
            o.y = __byte_perm(a4.y, a4.z, 0x5432);
            o.z = __byte_perm(a4.z, a4.w, 0x5432);
            o.w = __byte_perm(a4.w, e, 0x5432);
            *reinterpret_cast<uint4 *>(dst) = o;
        }
    }
}

// The SADs of one lane's task over the staged tile, into its CU's key or
// sum table.
template <int ES, int TY>
__device__ __forceinline__ void stage_compute(const DependentBatch &b, const StageTile &t, const StageSlots &ss,
                                              const uint32_t *buf, int per_cu, const FastDiv &div_cu,
                                              const FastDiv &div_k, int rb)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = b.r, K = 2 * r + 1;
    const StageShape &sh = t.sh;
    const long traw = t.tf + tid;
    const long tt = min(traw, t.ntask - 1);
    const uint32_t q = fast_div(static_cast<uint32_t>(tt), div_cu);
    const int slot = static_cast<int>(q - t.q0);
    const int rem = static_cast<int>(tt - static_cast<long>(q) * per_cu);
    const int band = static_cast<int>(fast_div(static_cast<uint32_t>(rem), div_k)), dxi = rem - band * K;
    const int dxo = dxi - r;
    const int b0 = band * TY - r;
    const int dy0 = K >= TY ? min(b0, r - TY + 1) : b0;
    // the lane's first sample of a block row, counted from the raw rows' column ax
    const int xs = ss.off[slot] + dxo + r;
    // 10-bit: its first word in raw0 or raw1; 8-bit: the word before the one
    // holding its first sample (q = (xs - 1) / 4, xs >= 1), shifted by m
    const int wq = ES == 2 ? (xs >> 1) : ((xs - 1) >> 2);
    const uint32_t *win = buf + slot * sh.PW + ((ES == 2 && (xs & 1)) ? sh.O1 : 0) + wq;
    const uint32_t *curw = buf + slot * sh.PW + sh.OC + (ES == 2 ? 0 : ss.coff[slot] / 4);
    // debug builds: the lane's slot is staged, and its last window word lies
    // in its raw rows (else it reads the slot's first words; recorded)
    if (!in_range(b.status, slot, t.nslots) ||
        !in_range(b.status, (t.RS - 8 + dy0 + r + TY + 6) * sh.RW + wq + (t.RS - 8) * ES / 4 + (ES == 2 ? 3 : 2),
                  sh.WR * sh.RW)) {
        win = buf;
        curw = buf;
    }
    // the CU's task word and inherited parent, loaded before the SADs (used
    // after them)
    const unsigned int ucu = q >> (2 * t.lg);
    const unsigned long long task = __ldcg(b.tasks[t.c] + ucu);
    const uint32_t up = parent_slot(b, t.c, ucu);
    uint32_t acc[TY];
#pragma unroll
    for (int i = 0; i < TY; ++i) acc[i] = 0;
    const int nb = t.RS / 8;
    if constexpr (ES == 2) {
        const uint32_t m2 = 0u - 2u * b.one;  // -2, unknown to the compiler: kept on the multiply-add pipe
#pragma unroll 1
        for (int blk = 0; blk < nb * nb; ++blk) {
            const int bx = 8 * (blk % nb), by = 8 * (blk / nb);
            uint4 cv[8];
            uint32_t sa = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                cv[j] = *reinterpret_cast<const uint4 *>(curw + (by + j) * sh.CW + bx / 2);
                sa += (cv[j].x + cv[j].y) + (cv[j].z + cv[j].w);
            }
            sads_staged_u16<TY>(cv, sa, m2, win + (by + dy0 + r) * sh.RW + bx / 2, sh.RW, acc);
        }
    } else {
        const uint32_t m = 1u << (32 - 8 * (xs - 4 * wq));  // xs - 4 wq in 1..4
#pragma unroll 1
        for (int blk = 0; blk < nb * nb; ++blk) {
            const int bx = 8 * (blk % nb), by = 8 * (blk / nb);
            uint2 cv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) cv[j] = *reinterpret_cast<const uint2 *>(curw + (by + j) * sh.CW + bx / 4);
            const uint32_t *rp = win + (by + dy0 + r) * sh.RW + bx / 4;
            const int rw = sh.RW;
            sads_core_u8<TY, 1>(cv, [&](int row, uint32_t &w0, uint32_t &w1) {
                const uint32_t a0 = rp[row * rw], a1 = rp[row * rw + 1], a2 = rp[row * rw + 2];
                w0 = shift_in(a0, a1, m);
                w1 = shift_in(a1, a2, m);
            }, acc);
        }
    }

    if (traw < t.ntask) add_to_parent<TY>(b, t.c, up, dxi, dy0, b0, acc);
    const uint32_t lo = static_cast<uint32_t>(task);
    const DependentItem &a = b.item[lo & 0xffu];
    const RungInfo &rinf = b.rung[a.rung];
    if (t.nr > 1) {
        // this piece's SADs into the CU's table, every candidate once
        if (traw < t.ntask && in_range(b.status, ucu, b.cap[t.c])) {
            unsigned int *sum = b.sums[t.c] + static_cast<long>(ucu) * (K * K);
#pragma unroll
            for (int i = 0; i < TY; ++i) {
                const int dyo = dy0 + i;
                if (dyo >= b0 && dyo <= r && in_range(b.status, (dyo + r) * K + dxi, K * K))
                    atomicAdd(sum + (dyo + r) * K + dxi, acc[i]);
            }
        }
        return;
    }
    const uint32_t cbase = static_cast<uint32_t>(abs(dxo) * 2 * K + 2 * (dy0 + r) + (dxo > 0));
    unsigned long long best = ~0ull;
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        const int dyo = dy0 + i;
        if (dyo > r) continue;
        const uint32_t code = umad(static_cast<uint32_t>(abs(dyo)), 2u * K, cbase + 2u * i);
        const unsigned long long key = (static_cast<unsigned long long>(acc[i]) << rb) | code;
        best = key < best ? key : best;
    }
    // segmented min over the lanes of this CU in the warp
    const long wfirst = t.tf + 32 * warp;  // the warp's first task
    const long cu_first = static_cast<long>(q) * per_cu - wfirst;
    const int first = static_cast<int>(max(cu_first, 0L));
    const int last = static_cast<int>(min(cu_first + per_cu - 1, t.ntask - 1 - wfirst));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_down_sync(0xffffffffu, best, o);
        if (lane + o <= last) best = v < best ? v : best;
    }
    if (lane == first && best != ~0ull) {
        const uint32_t sad = static_cast<uint32_t>(best >> rb);
        const int code = static_cast<int>(best & ((1ull << rb) - 1));
        const int l1 = code / (2 * K), rr = code - l1 * 2 * K;
        const int dyv = (rr >> 1) - r;
        const int adx = l1 - abs(dyv);
        const int dxv = (rr & 1) ? adx : -adx;
        const uint32_t tb = static_cast<uint32_t>(l1 * K * K + (dyv + r) * K + (dxv + r));
        unsigned long long *keys = reinterpret_cast<unsigned long long *>(a.block + rinf.off.keys);
        const long nk = static_cast<long>(rinf.g.ctu_cols) * rinf.g.ctu_rows * keys_per_ctu(rinf.g.dmax);
        if (in_range(b.status, lo >> 8, nk)) atomicMin(keys + (lo >> 8), (static_cast<unsigned long long>(sad) << 32) | tb);
    }
}

// pipelined = 1: two buffers of staged pieces, the next tile's async copies
// filling one while the current tile is computed from the other; 0: one
// buffer (less shared memory: more CTAs per SM overlap one another's
// staging instead).  `half`: words of one buffer.
// Four CTAs per SM (at most 128 registers a thread): with fewer, the
// staging of one CTA's tile is not hidden behind the others' compute.
template <typename T, int TY>
__global__ void __launch_bounds__(kStageThreads, 4)
    k_dep_search_staged(const __grid_constant__ DependentBatch b, const FastDiv div_cu, const FastDiv div_k,
                        const __grid_constant__ StageDivs dv, int half, int pipelined)
{
    constexpr int ES = sizeof(T);
    dev::chain_entry();
    extern __shared__ __align__(16) uint32_t s_win[];
    __shared__ StageSlots s_slots[2];
    __shared__ long s_ln[kSizeClasses], s_tn[kSizeClasses];  // lane tasks and tiles per size class
    __shared__ long s_next;  // this CTA's next tile
    const int r = b.r, K = 2 * r + 1;
    const int per_cu = K * ((K + TY - 1) / TY);
    const int code_max = 4 * r * K + 4 * r + 1;
    const int rb = 32 - __clz(code_max);
    if (threadIdx.x < kSizeClasses) {
        const int c = threadIdx.x;
        const long pieces = c < 2 ? 1 : (b.range >= 32 ? (c == 2 ? 1 : 4) : (c == 2 ? 4 : 16));
        s_ln[c] = static_cast<long>(min(__ldcg(b.counts + c), b.cap[c])) * pieces * per_cu;
        s_tn[c] = (s_ln[c] + kStageThreads - 1) / kStageThreads;
    }
    __syncthreads();
    const long total = s_tn[0] + s_tn[1] + s_tn[2] + s_tn[3];
    long tile = blockIdx.x;
    if (tile >= total) return;  // the whole CTA: nothing to do
    int bi = 0;
    StageTile t = stage_tile<ES, TY>(b, tile, per_cu, div_cu, s_ln, s_tn);
    stage_slots_setup<ES>(b, t, s_slots[0]);
    __syncthreads();
    stage_copy<ES>(t, s_slots[0], s_win, dv.cps[t.c]);
#pragma unroll 1
    for (;;) {
        uint32_t *buf = s_win + bi * half;
        // tiles after the first of each CTA are handed out in order as CTAs
        // free up (the tiles of the largest CUs come first): the grid's
        // tail is one tile of the smallest CUs
        if (threadIdx.x == 0) s_next = gridDim.x + static_cast<long>(atomicAdd(b.counts + kTileCounter, 1u));
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        if (s_slots[bi].any_edge) {
            stage_fixup<ES>(t, s_slots[bi], buf);
            __syncthreads();
        }
        if constexpr (ES == 2) {
            stage_raw1(t, buf, dv.c1[t.c]);
            __syncthreads();
        }
        // the next tile of this CTA into the other buffer, in flight during this one
        const long next = s_next;
        if (pipelined && next < total) {
            const StageTile tnext = stage_tile<ES, TY>(b, next, per_cu, div_cu, s_ln, s_tn);
            stage_slots_setup<ES>(b, tnext, s_slots[bi ^ 1]);
            __syncthreads();
            stage_copy<ES>(tnext, s_slots[bi ^ 1], s_win + (bi ^ 1) * half, dv.cps[tnext.c]);
        }
        stage_compute<ES, TY>(b, t, s_slots[bi], buf, per_cu, div_cu, div_k, rb);
        if (next >= total) break;
        __syncthreads();  // the buffer and its slots are restaged (now, or by the tile after next)
        t = stage_tile<ES, TY>(b, next, per_cu, div_cu, s_ln, s_tn);  // recomputed: nothing held across the compute
        tile = next;
        if (pipelined) {
            bi ^= 1;
        } else {
            stage_slots_setup<ES>(b, t, s_slots[0]);
            __syncthreads();
            stage_copy<ES>(t, s_slots[0], s_win, dv.cps[t.c]);
        }
    }
}

// ---- 3. decide --------------------------------------------------------------
template <typename T, int CTU>
__global__ void __launch_bounds__(kDecideThreads, 10) k_dep_decide(const __grid_constant__ DependentBatch b)
{
    dev::chain_entry();
    // the search has completed: its task counters go back to zero for the
    // next batch (they rest at zero between batches)
    if (blockIdx.x == 0 && threadIdx.x < kDepCounters) b.counts[threadIdx.x] = 0;
    using C = dev::Ctu<CTU>;
    const DependentItem &a = b.item[item_of(b)];
    const RungInfo &rinf = b.rung[a.rung];
    const RungGeom &g = rinf.g;
    __shared__ dev::CtuState<CTU> st;
    const int tid = threadIdx.x;
    const int ctu_idx = blockIdx.x - a.cta_begin;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    long kbase = static_cast<long>(ctu_idx) * C::NKEY;
    // debug builds: the CTU's key slots lie in the frame's
    if (!in_range(b.status, kbase + C::NKEY - 1, static_cast<long>(g.ctu_cols) * g.ctu_rows * C::NKEY)) kbase = 0;
    const int r = b.r, K = 2 * r + 1;
    const int16_t *in_cx = reinterpret_cast<const int16_t *>(a.block + rinf.off.dep_cx) + kbase;
    const int16_t *in_cy = reinterpret_cast<const int16_t *>(a.block + rinf.off.dep_cy) + kbase;
    const uint8_t *in_fl = reinterpret_cast<const uint8_t *>(a.block + rinf.off.dep_flags) + kbase;
    const unsigned long long *keys = reinterpret_cast<const unsigned long long *>(a.block + rinf.off.keys) + kbase;
    const int *in_slot = reinterpret_cast<const int *>(a.block + rinf.off.dep_slot) + kbase;
    // rule flags and list places of the CTU's CUs, one round of L2 loads
    constexpr int NBIG = key_offset(C::DMAX - kFirstSummedClass + 1);  // CUs of 32x32 and up
    __shared__ uint8_t s_fl[C::NKEY];
    __shared__ int s_slot[NBIG > 0 ? NBIG : 1];  // 16x16 CTUs have no CU of 32x32
    __shared__ unsigned long long s_best[NBIG > 0 ? NBIG : 1];
    // a 64x64 CTU whose SADs are its four sub-CUs' sums: their tables added
    // up entry by entry, (2r + 1)^2 entries, r <= 32
    __shared__ unsigned int s_ctu_sum[CTU == 64 ? 65 * 65 : 1];
    for (int i = tid; i < C::NKEY; i += kDecideThreads) {
        s_fl[i] = __ldcg(in_fl + i);
        if (i < NBIG) {
            s_slot[i] = __ldcg(in_slot + i);
            s_best[i] = ~0ull;
        }
    }
    __syncthreads();
    // CUs searched in pieces: argmin of (SAD, |dx|+|dy|, dy, dx) over the
    // CU's sum table, 16 lanes per CU.  A lane loads kScanBatch entries
    // before it uses any (one L2 round trip per batch, two for r = 8).  An
    // inherited CU whose sub-CUs have tables of their own (only the CTU can
    // be one: a 64x64 CU with 32x32 sub-CUs) has none: the sub-CUs' lanes add
    // the entries they load into a shared copy, which the whole CTA then scans.
    auto own_table = [&](int i) { return i < NBIG && s_slot[i] >= 0 && (CTU >> depth_of(i, C::DMAX)) > b.range; };
    const bool ctu_kids = CTU == 64 && NBIG > 0 && (s_fl[0] & kRuleInherited) && (CTU >> 1) > b.range;
    auto summed = [&](int i) { return own_table(i) || (i == 0 && ctu_kids); };
    {
        constexpr int kScanBatch = 10;
        const int hl = tid & 15;
        const unsigned hmask = 0xffffu << (tid & 16);
        const int KK = K * K;
        // candidate row of entry k: (k + 1/2) / K in fp32 is at least 1/(2K)
        // from an integer for k < 2^16, so the truncation is exact
        const float inv_k = 1.0f / static_cast<float>(K);
        auto key_of = [&](int k, unsigned int v) {
            const int dy = static_cast<int>((static_cast<float>(k) + 0.5f) * inv_k);
            const int dxo = k - dy * K - r, dyo = dy - r;
            const uint32_t tb = static_cast<uint32_t>((abs(dxo) + abs(dyo)) * KK + k);
            return (static_cast<unsigned long long>(v) << 32) | tb;
        };
        if (ctu_kids) {  // the same for the whole CTA
            for (int k = tid; k < KK; k += kDecideThreads) s_ctu_sum[k] = 0;
            __syncthreads();
        }
        for (int i = tid >> 4; i < NBIG; i += kDecideThreads / 16) {
            if (!own_table(i) || !(s_fl[i] & kRuleEvaluated)) continue;  // the same for the 16 lanes
            if (!in_range(b.status, s_slot[i], b.cap[C::DMAX - depth_of(i, C::DMAX)])) continue;
            const unsigned int *sum = b.sums[C::DMAX - depth_of(i, C::DMAX)] + static_cast<long>(s_slot[i]) * KK;
            const bool feed = ctu_kids && i >= 1 && i <= 4;  // a sub-CU of the CTU
            unsigned long long best = ~0ull;
            for (int k0 = hl; k0 < KK; k0 += 16 * kScanBatch) {
                unsigned int v[kScanBatch];
#pragma unroll
                for (int u = 0; u < kScanBatch; ++u) v[u] = k0 + 16 * u < KK ? __ldcg(sum + k0 + 16 * u) : 0u;
#pragma unroll
                for (int u = 0; u < kScanBatch; ++u) {
                    const int k = k0 + 16 * u;
                    if (k >= KK) break;
                    if constexpr (CTU == 64)
                        if (feed) atomicAdd(&s_ctu_sum[k], v[u]);
                    const unsigned long long key = key_of(k, v[u]);
                    best = key < best ? key : best;
                }
            }
#pragma unroll
            for (int o = 8; o >= 1; o >>= 1) {
                const unsigned long long v = __shfl_xor_sync(hmask, best, o);
                best = v < best ? v : best;
            }
            if (hl == 0) s_best[i] = best;
        }
        if constexpr (CTU == 64) {
            if (ctu_kids) {
                __syncthreads();
                unsigned long long best = ~0ull;
                for (int k = tid; k < KK; k += kDecideThreads) {
                    const unsigned long long key = key_of(k, s_ctu_sum[k]);
                    best = key < best ? key : best;
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
                    best = v < best ? v : best;
                }
                if ((tid & 31) == 0) atomicMin(&s_best[0], best);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < C::NKEY; i += kDecideThreads) {
        const uint8_t f = s_fl[i];
        st.flags[i] = f;
        st.satd[i] = 0;
        if (f & kRuleEvaluated) {
            const unsigned long long key = summed(i) ? s_best[i] : __ldcg(keys + i);
            const int rem = static_cast<int>(static_cast<uint32_t>(key & 0xffffffffu) % static_cast<uint32_t>(K * K));
            st.mvx[i] = static_cast<int16_t>(__ldcg(in_cx + i) + rem % K - r);
            st.mvy[i] = static_cast<int16_t>(__ldcg(in_cy + i) + rem / K - r);
            st.sad[i] = static_cast<int32_t>(key >> 32);
        } else {
            st.mvx[i] = INT16_MIN;
            st.mvy[i] = INT16_MIN;
            st.sad[i] = INT32_MAX;
        }
    }
    __syncthreads();
    // keys back to ~0 for the next search of this rung
    for (int i = tid; i < C::NKEY; i += kDecideThreads)
        const_cast<unsigned long long *>(keys)[i] = ~0ull;
    dev::DecideIOT<OffDecisions> io{a.cur, a.ref, a.pitch_bytes, &rinf.g, a.qp, b.satd_mode, c_lambda_q16,
                     OffDecisions{a.block, &rinf.off}, b.status};
    dev::ctu_decide<T, CTU>(st, io, x0, y0);
}

// ---- launches ---------------------------------------------------------------
template <typename T, int TY> int search_ctas_per_sm()
{
    static int n = 0;
    if (n == 0) {
        int v = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_dep_search<T, TY>, kSearchThreads, 0) != cudaSuccess ||
            v < 1)
            v = 1;
        n = v;
    }
    return n;
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 1;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess)
            v = 1;
        n = v;
    }
    return n;
}

template <typename T, int TY> cudaError_t search_t(const DependentBatch &b, cudaStream_t s)
{
    const int fit = search_ctas_per_sm<T, TY>();
    const int grid = sm_count() * (b.ctas_per_sm > 0 ? std::min(b.ctas_per_sm, fit) : fit);
    // divisors of the lane decode: lanes per CU piece, candidate columns
    const uint32_t K = 2 * b.r + 1, per_cu = K * ((K + TY - 1) / TY);
    return launch_chained(k_dep_search<T, TY>, dim3(grid), dim3(kSearchThreads), 0, s, b, make_fastdiv(per_cu),
                          make_fastdiv(K));
}

// Dynamic shared memory a staged-search CTA may take: the device's opt-in
// limit less the kernel's static shared memory.
int smem_optin()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 48 << 10;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            v = 48 << 10;
        cudaFuncAttributes fa{};
        size_t fixed = 1024;
        if (cudaFuncGetAttributes(&fa, k_dep_search_staged<uint16_t, kDepBand>) == cudaSuccess)
            fixed = fa.sharedSizeBytes;
        n = v - static_cast<int>(fixed);
    }
    return n;
}

// Dynamic shared memory of a staged search: the most pieces a tile touches
// times the largest piece of any size class (0 if it does not fit a CTA).
// (one buffer for b.staged == 1, two for 2; 0 if they do not fit a CTA).
template <typename T, int TY> size_t staged_smem_bytes(const DependentBatch &b)
{
    const int K = 2 * b.r + 1, per_cu = K * ((K + TY - 1) / TY);
    const int slots = stage_slots(per_cu);
    if (slots > kMaxStageSlots) return 0;
    int pw = 0;
    for (int S = 8; S <= 64; S <<= 1)
        pw = std::max(pw, stage_shape<sizeof(T)>(S < b.range ? S : b.range, b.r, TY).PW);
    const size_t bytes = (b.staged == 2 ? 2 : 1) * static_cast<size_t>(slots) * pw * 4;
    return bytes <= static_cast<size_t>(smem_optin()) ? bytes : 0;
}

template <typename T, int TY> cudaError_t search_staged(const DependentBatch &b, size_t smem, cudaStream_t s)
{
    int fit = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_dep_search_staged<T, TY>, kStageThreads, smem) !=
            cudaSuccess ||
        fit < 1)
        fit = 1;
    const int grid = sm_count() * (b.ctas_per_sm > 0 ? std::min(b.ctas_per_sm, fit) : fit);
    const uint32_t K = 2 * b.r + 1, per_cu = K * ((K + TY - 1) / TY);
    StageDivs dv{};
    for (int c = 0; c < kSizeClasses; ++c) {
        const int S = 8 << c;
        const StageShape sh = stage_shape<sizeof(T)>(S < b.range ? S : b.range, b.r, TY);
        dv.cps[c] = make_fastdiv(static_cast<uint32_t>(kStageRowGroups * (sh.NC + sh.CNC)));
        dv.c1[c] = make_fastdiv(static_cast<uint32_t>(kStageRowGroups * sh.NC));
    }
    const int pipelined = b.staged == 2 ? 1 : 0;
    const int half = static_cast<int>(smem / (pipelined ? 8 : 4));  // words of one buffer
    return launch_chained(k_dep_search_staged<T, TY>, dim3(grid), dim3(kStageThreads), smem, s, b, make_fastdiv(per_cu),
                          make_fastdiv(K), dv, half, pipelined);
}

template <typename T> cudaError_t search_bd(const DependentBatch &b, cudaStream_t s)
{
    // bands of 9 rows when 2r + 1 <= 9 or when asked for; 10-bit bodies are
    // twice as long per row, so 10-bit takes 9 unless asked for 17
    const bool nine = 2 * b.r + 1 <= 9 || b.band == 9 || (sizeof(T) == 2 && b.band != kDepBand);
    if (b.staged && b.r >= 4) {
        // staged windows (refinement ranges of 4 and more: at least 9 lanes
        // per piece, so a tile touches few pieces), when they fit a CTA
        const size_t smem = nine ? staged_smem_bytes<T, 9>(b) : staged_smem_bytes<T, kDepBand>(b);
        if (smem > 0) return nine ? search_staged<T, 9>(b, smem, s) : search_staged<T, kDepBand>(b, smem, s);
    }
    if (nine) return search_t<T, 9>(b, s);
    return search_t<T, kDepBand>(b, s);
}

}  // namespace

cudaError_t launch_dependent_rules(int ctu, const DependentBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxDepItems || b.total_ctas <= 0) return cudaErrorInvalidValue;
    auto kern = ctu == 64 ? k_dep_rules<64> : ctu == 32 ? k_dep_rules<32> : k_dep_rules<16>;
    return launch_chained(kern, dim3(b.total_ctas), dim3(kRulesThreads), 0, s, b);
}

cudaError_t launch_dependent_search(int bit_depth, const DependentBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxDepItems) return cudaErrorInvalidValue;
    return bit_depth == 8 ? search_bd<uint8_t>(b, s) : search_bd<uint16_t>(b, s);
}

cudaError_t launch_dependent_decide(int bit_depth, int ctu, const DependentBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxDepItems || b.total_ctas <= 0) return cudaErrorInvalidValue;
    auto kern = bit_depth == 8 ? (ctu == 64 ? k_dep_decide<uint8_t, 64>
                                            : ctu == 32 ? k_dep_decide<uint8_t, 32> : k_dep_decide<uint8_t, 16>)
                               : (ctu == 64 ? k_dep_decide<uint16_t, 64>
                                            : ctu == 32 ? k_dep_decide<uint16_t, 32> : k_dep_decide<uint16_t, 16>);
    return launch_chained(kern, dim3(b.total_ctas), dim3(kDecideThreads), 0, s, b);
}

cudaError_t prepare_kernels(int bit_depth, int ctu, int R, int r)
{
    cudaError_t e = prepare_full_search(bit_depth, ctu, R);
    if (e != cudaSuccess) return e;
    sm_count();
    // the staged search sizes its shared memory per launch, up to the opt-in limit
    if (bit_depth == 8) {
        search_ctas_per_sm<uint8_t, 9>();
        search_ctas_per_sm<uint8_t, kDepBand>();
        e = cudaFuncSetAttribute(k_dep_search_staged<uint8_t, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_optin());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_dep_search_staged<uint8_t, kDepBand>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
    } else {
        search_ctas_per_sm<uint16_t, 9>();
        search_ctas_per_sm<uint16_t, kDepBand>();
        e = cudaFuncSetAttribute(k_dep_search_staged<uint16_t, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_optin());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_dep_search_staged<uint16_t, kDepBand>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
    }
    if (e != cudaSuccess) return e;
    (void)r;
    return cudaGetLastError();
}

}  // namespace ladder_impl
