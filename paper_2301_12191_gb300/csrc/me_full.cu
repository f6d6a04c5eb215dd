// me_full.cu -- independent analysis, step 1: integer full-search block
// matching (SAD, Sec. 5.4.1) for every CU of every depth of a CTU at once.
//
// SAD is additive at a fixed vector, so one pass over the candidates yields
// the SAD of every 8x8 block, and sums of 4 / 16 / 64 of them give the 16x16,
// 32x32 and 64x64 CUs (the "SAD tree").  Per CTU the kernel keeps, for each
// of its CUs, the argmin of the key (SAD, |dx|+|dy|, dy, dx) over the
// (2R+1)^2 candidates.
//
// Layout of the work:
//   * Lane task = one dx and TY consecutive dy (a "band" of candidate rows);
//     a warp tile = 32 lane tasks (consecutive dx, wrapping into the next
//     band).  CTA = one CTU x one warp tile, 4 warps: warp q searches the
//     q-th quadrant of the CTU for the same 32 x TY candidates; several CTAs
//     per SM hide each other's copies and barriers.
//   * The reference window rows those candidates need and the current CTU
//     arrive by TMA tile copies.  The window is expanded
//     in place to one 32-bit word per sample position (8-bit: samples
//     p..p+3; 10-bit: p, p+1), taking the clamped sample wherever the window
//     leaves the frame, so the 32 lanes (consecutive dx) read 32 consecutive
//     words: conflict-free, with compile-time row offsets.  The current CTU
//     is read by broadcast.
//   * 8-bit: packed absdiff-accumulate (vabsdiff4 .add), 4 samples per ALU
//     instruction.  10-bit: SAD = sum(a) + sum(b) - 2 sum(min(a, b)) on
//     packed halfword pairs: one min.u16x2 (ALU) and one multiply-add
//     accumulate (FMA pipe) per two samples; sum(b) comes from row sums
//     slid over the candidate rows, sum(a) is per block.  Each half of a
//     packed 8x8 sum stays below 2^16, so nothing carries across halves.
//   * Keys: SAD * 2^16 + code, code = L1 * 2K + 2 (dy + R) + [dx > 0] (K =
//     2R + 1), which orders candidates of equal SAD by (|dx|+|dy|, dy, dx).
//     Per CU each lane takes the min over its TY candidates, one warp min
//     (redux.sync) gives the tile's best, and lane 0 folds it into the CTA's
//     keys with a shared atomicMin.  8x8 (and 8-bit 16x16) keys fit in 32
//     bits; larger CUs use 64-bit keys.  The 64x64 sums add the quadrants'
//     sums through shared memory.
//   * The CTA's keys are re-encoded as (SAD << 32) | tie-break and merged
//     into the global per-CTU keys with atomicMin (warp tiles of one CTU run
//     in different CTAs).  Integer min is order-independent, so the result
//     is deterministic.
#include "common.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

namespace ladder_impl {
namespace {

using dev::mbar_arrive_expect_tx;
using dev::mbar_init;
using dev::mbar_wait_bounded;
using dev::sad_acc;
using dev::tma_load_2d;

template <typename T, int CTU, int RP, int BAND> struct Shape {
    static constexpr int ES = sizeof(T);
    static constexpr int TY = BAND;
    static constexpr int P4 = CTU + 2 * RP;       // window positions (= expanded words) per row
    static constexpr int NT = 128;                // 4 warps, one per quadrant
    static constexpr int Q = CTU / 2;             // quadrant side
    static constexpr int QB = Q / 8;              // 8x8 blocks per quadrant side
    static constexpr int NBQ = QB * QB;           // 8x8 blocks per quadrant
    static constexpr int DMAX = CTU == 64 ? 3 : (CTU == 32 ? 2 : 1);
    static constexpr int NKEY = keys_per_ctu(DMAX);
    static constexpr int NB8 = (CTU / 8) * (CTU / 8);
    static constexpr int MAX_ROWS = CTU + 4 * TY - 1;  // a CTA's warp tiles span at most 4 bands
    static constexpr int CPR = P4 / 4;            // 16-byte chunks of expanded words per row
    // phase 2 of the in-place expansion covers at most box_h * ES / 4 + 2 rows
    static constexpr int MAXC = (((MAX_ROWS * ES + 3) / 4 + 2) * CPR + NT - 1) / NT;
    static constexpr int NW = ES == 1 ? 2 : 3;    // staged words behind one chunk
    static constexpr bool K16_32 = ES == 1;       // 16x16 keys fit 32 bits (8-bit samples)
};

__device__ __forceinline__ uint32_t umad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ unsigned long long umad_wide(uint32_t a, uint32_t b, uint32_t c)
{
    unsigned long long d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(static_cast<unsigned long long>(c)));
    return d;
}

__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
    const uint32_t hi = static_cast<uint32_t>(v >> 32), lo = static_cast<uint32_t>(v);
    const uint32_t mh = __reduce_min_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_min_sync(0xffffffffu, hi == mh ? lo : 0xffffffffu);
    return (static_cast<unsigned long long>(mh) << 32) | ml;
}

// Min over the lane's candidates of the 32-bit key SAD * 2^16 + code (m16 =
// 2^16 as an operand the compiler cannot fold, so the products stay on the
// multiply-add pipe).  Candidate rows past +R (only when 2R + 1 < TY, i.e.
// !all_valid) never win.  Tree order: the mins do not form one long chain.
template <int TY>
__device__ __forceinline__ uint32_t lane_key32(const uint32_t (&s)[TY], const uint32_t (&code)[TY], uint32_t m16,
                                               bool all_valid, int dy0, int R)
{
    uint32_t k[TY];
#pragma unroll
    for (int i = 0; i < TY; ++i) k[i] = umad(s[i], m16, code[i]);
    if (!all_valid) {
#pragma unroll
        for (int i = 0; i < TY; ++i)
            if (dy0 + i > R) k[i] = 0xffffffffu;
    }
#pragma unroll
    for (int w = 1; w < TY; w *= 2)
#pragma unroll
        for (int i = 0; i + w < TY; i += 2 * w) k[i] = min(k[i], k[i + w]);
    return k[0];
}

template <int TY>
__device__ __forceinline__ unsigned long long lane_key64(const uint32_t (&s)[TY], const uint32_t (&code)[TY],
                                                         uint32_t m16, bool all_valid, int dy0, int R)
{
    unsigned long long k[TY];
#pragma unroll
    for (int i = 0; i < TY; ++i) k[i] = (all_valid || dy0 + i <= R) ? umad_wide(s[i], m16, code[i]) : ~0ull;
#pragma unroll
    for (int w = 1; w < TY; w *= 2)
#pragma unroll
        for (int i = 0; i + w < TY; i += 2 * w) k[i] = k[i + w] < k[i] ? k[i + w] : k[i];
    return k[0];
}

// Staged words behind expanded chunk m (positions 4m .. 4m+3) of a window
// row: 8-bit samples 4m .. 4m+7, 10-bit samples 4m .. 4m+5.  `srow` is the
// staged row (already clamped to the frame); columns left or right of the
// frame take the clamped sample.
template <typename T, int P4>
__device__ __forceinline__ void fetch_chunk(const T *srow, int m, int gx0, int W, uint32_t (&w)[sizeof(T) == 1 ? 2 : 3])
{
    constexpr int ES = sizeof(T);
    constexpr int NW = ES == 1 ? 2 : 3;
    constexpr int NS = ES == 1 ? 8 : 6;  // samples behind the chunk
    const int c0 = 4 * m;
    if (gx0 + c0 >= 0 && gx0 + c0 + NS <= W && c0 + NS <= P4) {
        const uint32_t *sw = reinterpret_cast<const uint32_t *>(srow);
#pragma unroll
        for (int k = 0; k < NW; ++k) w[k] = sw[c0 * ES / 4 + k];
    } else {
#pragma unroll
        for (int k = 0; k < NW; ++k) w[k] = 0;
#pragma unroll
        for (int e = 0; e < NS; ++e) {
            const int c = min(max(gx0 + c0 + e, 0), W - 1) - gx0;  // inside the staged row
            if (c0 + e < P4) w[e * ES / 4] |= static_cast<uint32_t>(srow[c]) << ((e * ES * 8) & 31);
        }
    }
}

template <int ES>
__device__ __forceinline__ void emit_chunk(const uint32_t (&w)[ES == 1 ? 2 : 3], uint32_t *dst)
{
    uint4 v;
    if constexpr (ES == 1) {
        v.x = w[0];
        v.y = __funnelshift_r(w[0], w[1], 8);
        v.z = __funnelshift_r(w[0], w[1], 16);
        v.w = __funnelshift_r(w[0], w[1], 24);
    } else {
        v.x = w[0];
        v.y = __funnelshift_r(w[0], w[1], 16);
        v.z = w[1];
        v.w = __funnelshift_r(w[1], w[2], 16);
    }
    *reinterpret_cast<uint4 *>(dst) = v;
}

__constant__ int c_lambda_q16[52] = {
#include "lambda_table.inc"
};

static_assert(sizeof(FullSearchBatch) <= 32764, "full-search batch exceeds the kernel parameter space");

// The decisions of one CTU after its search (fuse_decide): decode the keys
// (and reset them to ~0 for the next search), then SATD, cost, split and
// leaf maps.  `st` lies in the CTA's shared memory.
template <typename T, int CTU>
__device__ __forceinline__ void decide_ctu(const FullSearchBatch &b, const FullSearchItem &a, int ctu_idx, int x0,
                                           int y0, dev::CtuState<CTU> &st)
{
    using C = dev::Ctu<CTU>;
    const RungInfo &ri = b.rung[a.rung];
    const RungGeom &g = ri.g;
    const int K = 2 * b.R + 1;
    unsigned long long *keys = a.keys + static_cast<long>(ctu_idx) * C::NKEY;
    for (int i = threadIdx.x; i < C::NKEY; i += blockDim.x) {
        int d = 0;
        while (d < C::DMAX && i >= key_offset(d + 1)) ++d;
        const int li = i - key_offset(d), n = 1 << d, S = CTU >> d;
        const int fx = x0 / S + li % n, fy = y0 / S + li / n;
        uint8_t flags = 0;
        if (fx * S < g.W8 && fy * S < g.H8) {
            const bool inside = fx * S + S <= g.W8 && fy * S + S <= g.H8;
            flags = dev::kPresent | kRuleReachable | (inside ? kRuleEvaluated : 0) | (d < C::DMAX ? kRuleCanSplit : 0);
        }
        st.flags[i] = flags;
        st.satd[i] = 0;
        const unsigned long long key = __ldcg(keys + i);
        __stcg(keys + i, ~0ull);
        if (flags & kRuleEvaluated) {
            const int rem = static_cast<int>(static_cast<uint32_t>(key & 0xffffffffu) % static_cast<uint32_t>(K * K));
            st.mvx[i] = static_cast<int16_t>(rem % K - b.R);
            st.mvy[i] = static_cast<int16_t>(rem / K - b.R);
            st.sad[i] = static_cast<int32_t>(key >> 32);
        } else {
            st.mvx[i] = INT16_MIN;
            st.mvy[i] = INT16_MIN;
            st.sad[i] = INT32_MAX;
        }
    }
    __syncthreads();
    dev::DecideIO io{a.cur, a.ref, a.pitch_bytes, &g, a.qp, b.satd_mode, c_lambda_q16, decisions_at(a.block, ri.off),
                     b.status};
    dev::ctu_decide<T, CTU>(st, io, x0, y0);
}

// 8-bit: four CTAs per SM; 10-bit: three (at most 168 registers), which
// the shared memory allows with bands of 9, or with bands of 13 when the
// current CTU is read through L1 (CL: frames of whole 8x8 blocks, so no
// current sample needs the edge replication of the staged copy).
template <typename T, int CTU, int RP, int BAND, bool CL>
__global__ void __launch_bounds__(128, sizeof(T) == 1 ? 4 : 3) k_full_search(const __grid_constant__ FullSearchBatch b)
{
    using S = Shape<T, CTU, RP, BAND>;
    constexpr int TY = S::TY, P4 = S::P4, ES = S::ES, NT = S::NT;
    constexpr int NR = 8 + TY - 1;  // window rows read per 8x8 block
    dev::chain_entry();

    extern __shared__ __align__(128) uint8_t smem_raw[];
    // 128-byte aligned base by pointer arithmetic on the shared array (the
    // compiler keeps every derived pointer in the shared window)
    uint8_t *const sm = smem_raw + ((128u - (dev::smem_addr(smem_raw) & 127u)) & 127u);
    uint32_t *const E = reinterpret_cast<uint32_t *>(sm);             // box_h rows x P4 words
    T *const stage = reinterpret_cast<T *>(sm + b.stage_off);         // box_h rows x P4 samples, inside E
    T *const curs = reinterpret_cast<T *>(sm + b.e_bytes);            // CTU x CTU samples (not with CL)
    uint32_t *const a8 = reinterpret_cast<uint32_t *>(sm + b.e_bytes + (CL ? 0 : CTU * CTU * ES));  // 10-bit block sums
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_k8[S::NB8];                          // 8x8 keys
    __shared__ unsigned long long s_kup[keys_per_ctu(S::DMAX - 1)];  // larger CUs
    // quadrant sums per candidate and lane for the CTU level: in E when the
    // CTA has one warp tile (E is then free), else after the current CTU
    uint32_t *const s_xch = b.group > 1 ? a8 + (ES == 2 ? S::NB8 : 0) : E;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = b.R, K = 2 * R + 1;
    const int ii = dev::item_of_cta(b.item, b.n);  // the frame of this CTA
    const FullSearchItem &a = b.item[ii];
    const int local = blockIdx.x - a.cta_begin;
    // this CTA: warp tiles wt0 .. wt1-1 of one CTU, over one staged window
    const int ngroups = (b.warp_tiles + b.group - 1) / b.group;
    const int ctu_idx = local / ngroups, grp = local - ctu_idx * ngroups;
    const int wt0 = grp * b.group, wt1 = min(wt0 + b.group, b.warp_tiles);
    const int W8 = (a.W + 7) & ~7, H8 = (a.H + 7) & ~7;
    const int ctu_cols = (W8 + CTU - 1) / CTU;
    const int x0 = (ctu_idx % ctu_cols) * CTU, y0 = (ctu_idx / ctu_cols) * CTU;
    auto band_dy0 = [&](int t) {
        int v = (t / K) * TY - R;
        if (K >= TY) v = min(v, R - TY + 1);
        return v;
    };
    const int tf = wt0 * 32, tl = min(wt1 * 32 - 1, b.ntasks - 1);
    const int rlo = band_dy0(tf) + R;                   // first window row, relative to y0 - R
    const int rows = band_dy0(tl) + R + TY - 1 + CTU - rlo;
    const int gy0 = y0 - R + rlo;                       // frame row of window row 0
    const int sy0 = min(max(gy0, 0), a.H - 1);          // window rows clamp into staged rows [sy0, sy0 + box_h)

    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&b.map[ii])) : "memory");
    }
    for (int i = tid; i < S::NB8; i += NT) s_k8[i] = 0xffffffffu;
    for (int i = tid; i < keys_per_ctu(S::DMAX - 1); i += NT) s_kup[i] = ~0ull;
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, static_cast<uint32_t>((b.box_h * P4 + (CL ? 0 : CTU * CTU)) * ES));
        tma_load_2d(stage, &b.map[ii], &bar, x0 - b.Rp, sy0);
        if constexpr (!CL) tma_load_2d(curs, &b.cur_map[ii], &bar, x0, y0);
    }

    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(b.status, kStatusTimeout);
        if (!ok) mbar_wait_bounded(&bar, 0);
        return;
    }

    // CL: the current CTU's samples, row pitch cps (read through L1)
    const long cps = a.pitch_bytes / ES;
    const T *const curg = static_cast<const T *>(a.cur) + static_cast<long>(y0) * cps + x0;
    // Current CTU: edge replication into the 8-aligned pad.
    if (!CL && (x0 + CTU > a.W || y0 + CTU > a.H)) {
        for (int i = tid; i < CTU * CTU; i += NT) {
            const int row = i / CTU, col = i - row * CTU;
            const int gx = x0 + col, gy = y0 + row;
            if (gx < W8 && gy < H8 && (gx >= a.W || gy >= a.H))
                curs[i] = curs[(min(gy, a.H - 1) - y0) * CTU + (min(gx, a.W - 1) - x0)];
        }
    }
    // In-place expansion of the window (the staged rows sit at the end of
    // E).  Phase 1: rows of E that end before the staged rows; phase 2: the
    // staged words of the remaining rows go to registers first.  Window row
    // r is staged row clamp(gy0 + r) - sy0 <= r.
    {
        const int gx0 = x0 - b.Rp;
        auto srow_of = [&](int r) { return stage + (min(max(gy0 + r, 0), a.H - 1) - sy0) * P4; };
        const int r1 = min(b.phase1_rows, rows);
        // phase 1: one warp per row (row clamp once), one chunk per lane
        constexpr int LPR = (S::CPR + 31) / 32;
#pragma unroll 1
        for (int r = warp; r < r1; r += NT / 32) {
            const T *srow = srow_of(r);
            uint32_t *erow = E + r * P4;
#pragma unroll
            for (int k = 0; k < LPR; ++k) {
                const int m = lane + 32 * k;
                if (S::CPR % 32 == 0 || m < S::CPR) {
                    uint32_t w[S::NW];
                    fetch_chunk<T, P4>(srow, m, gx0, a.W, w);
                    emit_chunk<ES>(w, erow + 4 * m);
                }
            }
        }
        const int n2 = (rows - r1) * S::CPR;
        uint32_t hold[S::MAXC][S::NW];
#pragma unroll
        for (int c = 0; c < S::MAXC; ++c) {
            const int i = tid + c * NT;
            if (i < n2) fetch_chunk<T, P4>(srow_of(r1 + i / S::CPR), i % S::CPR, gx0, a.W, hold[c]);
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < S::MAXC; ++c) {
            const int i = tid + c * NT;
            if (i < n2) emit_chunk<ES>(hold[c], E + (r1 + i / S::CPR) * P4 + 4 * (i % S::CPR));
        }
    }
    if constexpr (ES == 2) {
        // packed (even, odd) sample sums of every 8x8 block of the CTU
        for (int blk = tid; blk < S::NB8; blk += NT) {
            const int bx = (blk % (CTU / 8)) * 8, by = (blk / (CTU / 8)) * 8;
            uint32_t s = 0;
            if (CL && (x0 + bx >= W8 || y0 + by >= H8)) {  // outside the frame: never read
                a8[blk] = 0;
                continue;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint4 v = CL ? __ldg(reinterpret_cast<const uint4 *>(curg + (by + j) * cps + bx))
                                   : *reinterpret_cast<const uint4 *>(curs + (by + j) * CTU + bx);
                s += v.x + v.y + v.z + v.w;
            }
            a8[blk] = s;
        }
    }
    __syncthreads();

    // ---- search: per warp tile, warp = quadrant, its 8x8 blocks in Z order ----
    const int qx = (warp & 1) * S::Q, qy = (warp >> 1) * S::Q;
    const uint32_t one = b.one, m16 = b.one << 16;
    const uint32_t m2 = 0u - 2u * b.one;  // -2, unknown to the compiler: kept on the multiply-add pipe
    const bool all_valid = K >= TY;  // else rows past +R exist and never win
#pragma unroll 1
    for (int wt = wt0; wt < wt1; ++wt) {
        const int t = min(wt * 32 + lane, b.ntasks - 1);
        const int dx = t % K - R, dy0 = band_dy0(t);
        uint32_t code[TY];  // (|dx|+|dy|) 2K + 2 (dy + R) + [dx > 0]
    #pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int dy = dy0 + i;
            code[i] = static_cast<uint32_t>((abs(dx) + abs(dy)) * 2 * K + 2 * (dy + R) + (dx > 0));
        }
        const uint32_t *lp = E + (dy0 + R - rlo + qy) * P4 + (dx + b.Rp + qx);
        // debug builds: the lane's first and last window words lie in the
        // staged window (else it reads from the window's origin: the failure
        // is recorded; the CTA's barriers below still run)
        if (!in_range(b.status, (dy0 + R - rlo + qy) * P4 + (dx + b.Rp + qx), b.e_bytes / 4) ||
            !in_range(b.status, (dy0 + R - rlo + qy + S::Q - 8 + NR - 1) * P4 + (dx + b.Rp + qx + S::Q - 8) +
                                    (ES == 1 ? 4 : 6),
                      b.e_bytes / 4))
            lp = E;
        uint32_t s16[TY], s32[TY];
    #pragma unroll
        for (int i = 0; i < TY; ++i) {
            s16[i] = 0;
            s32[i] = 0;
        }
        // SADs of the lane's candidates for the 8x8 block at (bx, by) of the
        // quadrant (acc starts at zero), and the block's 8x8 key
        auto block_sads = [&](int bx, int by, uint32_t(&acc)[TY]) {
            const uint32_t *bp = lp + by * P4 + bx;
            const T *cp = CL ? curg + (qy + by) * cps + qx + bx : curs + (qy + by) * CTU + qx + bx;
            const long cstride = CL ? cps : CTU;
            if constexpr (ES == 1) {
                uint2 c[8];
    #pragma unroll
                for (int j = 0; j < 8; ++j) c[j] = *reinterpret_cast<const uint2 *>(cp + j * cstride);
    #pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t w0 = bp[r * P4], w1 = bp[r * P4 + 4];
                    // all candidates on word 0, then on word 1: no back-to-back dependence
    #pragma unroll
                    for (int i = 0; i < TY; ++i) {
                        const int j = r - i;
                        if (j >= 0 && j < 8) acc[i] = sad_acc<4>(c[j].x, w0, acc[i]);
                    }
    #pragma unroll
                    for (int i = 0; i < TY; ++i) {
                        const int j = r - i;
                        if (j >= 0 && j < 8) acc[i] = sad_acc<4>(c[j].y, w1, acc[i]);
                    }
                }
            } else {
                uint4 c[8];
    #pragma unroll
                for (int j = 0; j < 8; ++j)
                    c[j] = CL ? __ldg(reinterpret_cast<const uint4 *>(cp + j * cstride))
                              : *reinterpret_cast<const uint4 *>(cp + j * CTU);
                const uint32_t sa = a8[((qy + by) / 8) * (CTU / 8) + (qx + bx) / 8];
                // SAD = sum(a) + sum(b) - 2 sum(min), per packed half, modulo
                // 2^32 (each half of the final word is at most 32 * 1023):
                // candidate i's word starts at sum(a) and takes -2 min per
                // sample pair; at its last row i + 7 it takes sum(b) as the
                // difference of two prefixes of the packed row sums, and one
                // dp2a adds its halves
    #pragma unroll
                for (int i = 0; i < TY; ++i) acc[i] = sa;
                uint32_t pf[NR + 1];  // pf[r + 1]: packed sum of window rows 0..r
                pf[0] = 0;
    #pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t w0 = bp[r * P4], w1 = bp[r * P4 + 2], w2 = bp[r * P4 + 4], w3 = bp[r * P4 + 6];
                    pf[r + 1] = (pf[r] + w0 + w1) + (w2 + w3);
    #pragma unroll
                    for (int i = 0; i < TY; ++i) {
                        const int j = r - i;
                        if (j >= 0 && j < 8) acc[i] = umad(min_u16x2(c[j].x, w0), m2, acc[i]);
                    }
    #pragma unroll
                    for (int i = 0; i < TY; ++i) {
                        const int j = r - i;
                        if (j >= 0 && j < 8) acc[i] = umad(min_u16x2(c[j].y, w1), m2, acc[i]);
                    }
    #pragma unroll
                    for (int i = 0; i < TY; ++i) {
                        const int j = r - i;
                        if (j >= 0 && j < 8) acc[i] = umad(min_u16x2(c[j].z, w2), m2, acc[i]);
                    }
    #pragma unroll
                    for (int i = 0; i < TY; ++i) {
                        const int j = r - i;
                        if (j >= 0 && j < 8) acc[i] = umad(min_u16x2(c[j].w, w3), m2, acc[i]);
                    }
                    if (r >= 7) {
                        const int i = r - 7;  // candidate i is complete
                        acc[i] = __dp2a_lo(acc[i] + (pf[r + 1] - pf[i]), 0x0101u, 0u);
                    }
                }
            }
            const uint32_t key = __reduce_min_sync(0xffffffffu, lane_key32<TY>(acc, code, m16, all_valid, dy0, R));
            if (lane == 0) atomicMin(&s_k8[((qy + by) / 8) * (CTU / 8) + (qx + bx) / 8], key);
        };
        auto key16 = [&](int cx, int cy) {  // 16x16 CU (cx, cy) of the CTU complete in s16
            if (x0 + cx * 16 < W8 && y0 + cy * 16 < H8) {
                unsigned long long key;
                if constexpr (S::K16_32) key = __reduce_min_sync(0xffffffffu, lane_key32<TY>(s16, code, m16, all_valid, dy0, R));
                else key = warp_min_u64(lane_key64<TY>(s16, code, m16, all_valid, dy0, R));
                if (lane == 0) atomicMin(&s_kup[key_offset(S::DMAX - 1) + cy * (CTU / 16) + cx], key);
            }
    #pragma unroll
            for (int i = 0; i < TY; ++i) {
                s32[i] = umad(s16[i], one, s32[i]);
                s16[i] = 0;
            }
        };
        auto key32 = [&]() {  // the quadrant's 32x32 CU complete in s32
            const int cx = qx / 32, cy = qy / 32;
            if (x0 + cx * 32 < W8 && y0 + cy * 32 < H8) {
                const unsigned long long key = warp_min_u64(lane_key64<TY>(s32, code, m16, all_valid, dy0, R));
                if (lane == 0) atomicMin(&s_kup[key_offset(S::DMAX - 2) + cy * (CTU / 32) + cx], key);
            }
        };
        // blocks in Z order.  8-bit: 16x16 CUs of 4 blocks as an inner loop;
        // 10-bit (longer block bodies): one loop over the quadrant's blocks
        if constexpr (ES == 1) {
            constexpr int B16 = S::NBQ >= 4 ? 4 : S::NBQ;  // 8x8 blocks per 16x16 CU inside a quadrant
            constexpr int N16 = S::NBQ / B16;
    #pragma unroll 1
            for (int q16 = 0; q16 < N16; ++q16) {
    #pragma unroll 1
                for (int b4 = 0; b4 < B16; ++b4) {
                    const int bq = q16 * B16 + b4;
                    const int bx = ((bq & 1) | ((bq >> 1) & 2)) * 8, by = (((bq >> 1) & 1) | ((bq >> 2) & 2)) * 8;
                    if (x0 + qx + bx >= W8 || y0 + qy + by >= H8) continue;  // block outside the frame: adds 0
                    uint32_t acc[TY];
    #pragma unroll
                    for (int i = 0; i < TY; ++i) acc[i] = 0;
                    block_sads(bx, by, acc);
    #pragma unroll
                    for (int i = 0; i < TY; ++i) s16[i] = umad(acc[i], one, s16[i]);
                }
                if constexpr (S::Q >= 16) key16((qx + 16 * (q16 & 1)) / 16, (qy + 16 * (q16 >> 1)) / 16);
            }
        } else {
    #pragma unroll 1
            for (int bq = 0; bq < S::NBQ; ++bq) {
                const int bx = ((bq & 1) | ((bq >> 1) & 2)) * 8, by = (((bq >> 1) & 1) | ((bq >> 2) & 2)) * 8;
                uint32_t acc[TY];
    #pragma unroll
                for (int i = 0; i < TY; ++i) acc[i] = 0;
                if (x0 + qx + bx < W8 && y0 + qy + by < H8) block_sads(bx, by, acc);
    #pragma unroll
                for (int i = 0; i < TY; ++i) s16[i] = umad(acc[i], one, s16[i]);
                if constexpr (S::Q >= 16)
                    if ((bq & 3) == 3) key16((qx + bx) / 16, (qy + by) / 16);
            }
        }
        if constexpr (S::Q >= 32) key32();

        // CTU level: the four quadrants' sums; warps 1-3 pass theirs to warp
        // 0 (which has read the previous tile's exchange once every warp
        // passes the first barrier)
        __syncthreads();
        const uint32_t(&top)[TY] = (S::Q >= 16) ? s32 : s16;
        if (warp > 0) {
    #pragma unroll
            for (int i = 0; i < TY; ++i) s_xch[((warp - 1) * TY + i) * 32 + lane] = top[i];
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t tot[TY];
    #pragma unroll
            for (int i = 0; i < TY; ++i)
                tot[i] = top[i] + s_xch[i * 32 + lane] + s_xch[(TY + i) * 32 + lane] + s_xch[(2 * TY + i) * 32 + lane];
            const unsigned long long key = warp_min_u64(lane_key64<TY>(tot, code, m16, all_valid, dy0, R));
            if (lane == 0) atomicMin(&s_kup[0], key);
        }
    }  // warp tiles
    __syncthreads();

    // Re-encode (SAD << 16 | code) as (SAD << 32 | tie-break) and merge.
    unsigned long long *out = a.keys + static_cast<long>(ctu_idx) * S::NKEY;
    const long nkeys = static_cast<long>(ctu_cols) * ((H8 + CTU - 1) / CTU) * S::NKEY;  // the frame's keys
    constexpr int NUP = keys_per_ctu(S::DMAX - 1);
    for (int i = tid; i < S::NKEY; i += NT) {
        const unsigned long long v = i < NUP ? s_kup[i] : static_cast<unsigned long long>(s_k8[i - NUP]);
        if (i < NUP ? v == ~0ull : v == 0xffffffffull) continue;
        const uint32_t sad = static_cast<uint32_t>(v >> 16);
        const int c = static_cast<int>(v & 0xffffu);
        const int l1 = c / (2 * K), rem = c - l1 * 2 * K;
        const int dyv = (rem >> 1) - R;
        const int adx = l1 - abs(dyv);
        const int dxv = (rem & 1) ? adx : -adx;
        const uint32_t tb = static_cast<uint32_t>(l1 * K * K + (dyv + R) * K + (dxv + R));
        if (in_range(b.status, static_cast<long>(ctu_idx) * S::NKEY + i, nkeys))
            atomicMin(out + i, (static_cast<unsigned long long>(sad) << 32) | tb);
    }
    if (b.fuse_decide) {
        // the last CTA of this CTU to finish takes its decisions
        __shared__ int s_last;
        __threadfence();  // this CTA's key updates before its count
        __syncthreads();
        unsigned int *done = a.done + ctu_idx;
        if (tid == 0) s_last = atomicAdd(done, 1u) == static_cast<unsigned int>(ngroups - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();  // every other CTA's key updates before the reads
        if (tid == 0) *done = 0;  // zero for the next search of this block
        decide_ctu<T, CTU>(b, a, ctu_idx, x0, y0, *reinterpret_cast<dev::CtuState<CTU> *>(sm));
    }
}

// Largest dynamic shared memory already granted to a kernel instance.
template <typename T, int CTU, int RP, int BAND, bool CL> int &granted_smem()
{
    static int bytes = -1;
    return bytes;
}

template <typename T, int CTU, int RP, int BAND, bool CL> cudaError_t ensure_smem(int smem)
{
    if (granted_smem<T, CTU, RP, BAND, CL>() >= smem) return cudaSuccess;
    cudaError_t e =
        cudaFuncSetAttribute(k_full_search<T, CTU, RP, BAND, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) granted_smem<T, CTU, RP, BAND, CL>() = smem;
    return e;
}

template <typename T, int CTU, int RP, int BAND, bool CL> int occupancy_t(int smem)
{
    if (ensure_smem<T, CTU, RP, BAND, CL>(smem) != cudaSuccess) return 1;
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_full_search<T, CTU, RP, BAND, CL>, Shape<T, CTU, RP, BAND>::NT,
                                                      smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <typename T, int CTU, int RP, int BAND, bool CL>
cudaError_t launch_t(const FullSearchBatch &b, int smem, cudaStream_t s)
{
    using S = Shape<T, CTU, RP, BAND>;
    cudaError_t e = ensure_smem<T, CTU, RP, BAND, CL>(smem);
    if (e != cudaSuccess) return e;
    const int n2 = (b.box_h - std::min(b.phase1_rows, b.box_h)) * S::CPR;
    if (n2 > S::MAXC * S::NT || b.box_h > S::MAX_ROWS || 3 * S::TY * 32 * 4 > b.e_bytes) return cudaErrorInvalidValue;
    return launch_chained(k_full_search<T, CTU, RP, BAND, CL>, dim3(b.total), dim3(S::NT), smem, s, b);
}

// Dispatch on (bit depth, CTU, window margin class, band, current CTU
// through L1): 64x64 CTUs have bands of 13 (default) and 9 candidate rows,
// smaller CTUs only 13; the L1 form exists for 10-bit only.
template <typename T, int CTU, int RP, int BAND, typename F> cudaError_t dispatch_cl(bool cl, F &&f)
{
    if constexpr (sizeof(T) == 2) {
        if (cl) return f.template run<T, CTU, RP, BAND, true>();
    }
    return f.template run<T, CTU, RP, BAND, false>();
}

template <typename F> cudaError_t dispatch(int bit_depth, int ctu, int Rp, int band, bool cl, F &&f)
{
    const bool wide = Rp > 32, b9 = band == 9;
    if (bit_depth == 8) {
        if (ctu == 64) {
            if (wide) return b9 ? dispatch_cl<uint8_t, 64, 64, 9>(false, f) : dispatch_cl<uint8_t, 64, 64, 13>(false, f);
            return b9 ? dispatch_cl<uint8_t, 64, 32, 9>(false, f) : dispatch_cl<uint8_t, 64, 32, 13>(false, f);
        }
        if (ctu == 32) return dispatch_cl<uint8_t, 32, 64, 13>(false, f);
        return dispatch_cl<uint8_t, 16, 64, 13>(false, f);
    }
    if (ctu == 64) {
        if (wide) return b9 ? dispatch_cl<uint16_t, 64, 64, 9>(cl, f) : dispatch_cl<uint16_t, 64, 64, 13>(cl, f);
        return b9 ? dispatch_cl<uint16_t, 64, 32, 9>(cl, f) : dispatch_cl<uint16_t, 64, 32, 13>(cl, f);
    }
    if (ctu == 32) return dispatch_cl<uint16_t, 32, 64, 13>(cl, f);
    return dispatch_cl<uint16_t, 16, 64, 13>(cl, f);
}

int rp_class(int ctu, int Rp) { return (ctu == 64 && Rp <= 32) ? 32 : 64; }

struct OccupancyOp {
    int smem, n;
    template <typename T, int CTU, int RP, int BAND, bool CL> cudaError_t run()
    {
        n = occupancy_t<T, CTU, RP, BAND, CL>(smem);
        return cudaSuccess;
    }
};

struct LaunchOp {
    const FullSearchBatch &b;
    int smem;
    cudaStream_t s;
    template <typename T, int CTU, int RP, int BAND, bool CL> cudaError_t run()
    {
        return launch_t<T, CTU, RP, BAND, CL>(b, smem, s);
    }
};

}  // namespace

FullSearchPlan full_search_plan(int bit_depth, int ctu, int R, int band, int group, int cur_l1)
{
    if (ctu != 64 || band != 9) band = kFsBand;  // the compiled bands
    FullSearchPlan p{};
    p.cur_l1 = bit_depth == 10 && cur_l1 ? 1 : 0;  // the L1 form exists for 10-bit only
    const int es = bit_depth == 8 ? 1 : 2;
    const int K = 2 * R + 1;
    p.Rp = (R + 15) / 16 * 16;
    const int RPc = rp_class(ctu, p.Rp);
    p.band = band;
    p.nbands = (K + band - 1) / band;
    p.ntasks = K * p.nbands;
    p.warp_tiles = (p.ntasks + 31) / 32;
    auto dy0 = [&](int t) {
        int v = (t / K) * band - R;
        if (K >= band) v = std::min(v, R - band + 1);
        return v;
    };
    // window rows of a CTA holding `g` consecutive warp tiles
    auto rows_for = [&](int g) {
        int rows = 0;
        for (int w0 = 0; w0 < p.warp_tiles; w0 += g) {
            const int tf = w0 * 32, tl = std::min((w0 + g) * 32 - 1, p.ntasks - 1);
            rows = std::max(rows, dy0(tl) - dy0(tf) + band - 1 + ctu);
        }
        return rows;
    };
    group = std::max(1, std::min(group, p.warp_tiles));
    while (group > 1 && rows_for(group) > ctu + 4 * band - 1) --group;  // the kernels' window bound
    p.group = group;
    p.ctas_per_ctu = (p.warp_tiles + group - 1) / group;
    const int rows = rows_for(group);
    p.P4 = ctu + 2 * RPc;
    p.box_w = p.P4;
    p.box_h = rows;
    p.e_bytes = (rows * p.P4 * 4 + 127) / 128 * 128;
    const int stage_bytes = rows * p.P4 * es;
    p.stage_off = (p.e_bytes - stage_bytes) / 128 * 128;
    p.phase1_rows = p.stage_off / (4 * p.P4);
    const int cur_bytes = p.cur_l1 ? 0 : ctu * ctu * es;
    const int a8_bytes = es == 2 ? (ctu / 8) * (ctu / 8) * 4 : 0;
    const int xch_bytes = group > 1 ? 3 * band * 32 * 4 : 0;  // else the exchange reuses the window
    p.buf_bytes = (p.e_bytes + cur_bytes + a8_bytes + xch_bytes + 127) / 128 * 128;
    p.smem_bytes = p.buf_bytes + 128;  // + alignment slack
    return p;
}

void fill_full_search_batch(FullSearchBatch &b, const FullSearchPlan &p, int R)
{
    b.R = R;
    b.band = p.band;
    b.group = p.group;
    b.Rp = p.Rp;
    b.ntasks = p.ntasks;
    b.warp_tiles = p.warp_tiles;
    b.box_h = p.box_h;
    b.e_bytes = p.e_bytes;
    b.stage_off = p.stage_off;
    b.phase1_rows = p.phase1_rows;
    b.buf_bytes = p.buf_bytes;
    b.cur_l1 = p.cur_l1;
    b.one = 1;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

int encode_plane_map(CUtensorMap *map, const void *plane, int W, int H, long pitch_bytes, int bit_depth, int box_w,
                     int box_h)
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return -1;
    const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H)};
    const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(pitch_bytes)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h)};
    const cuuint32_t estride[2] = {1, 1};
    const CUtensorMapDataType dt = bit_depth == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    return static_cast<int>(g_encode(map, dt, 2, const_cast<void *>(plane), gdim, gstride, box, estride,
                                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE));
}

int encode_item_maps(FullSearchBatch &b, int k, const void *cur, const void *ref, int W, int H, long pitch_bytes,
                     int bit_depth, int ctu, const FullSearchPlan &p)
{
    const int r = encode_plane_map(&b.map[k], ref, W, H, pitch_bytes, bit_depth, p.box_w, p.box_h);
    if (r != 0) return r;
    return encode_plane_map(&b.cur_map[k], cur, W, H, pitch_bytes, bit_depth, ctu, ctu);
}

cudaError_t prepare_full_search(int bit_depth, int ctu, int R)
{
    // raises the shared-memory attributes (largest: the widest group) outside any capture
    for (int g = 1; g <= kFsMaxGroup; ++g)
        for (int cl = 0; cl <= (bit_depth == 10 ? 1 : 0); ++cl) {
            full_search_ctas_per_sm(bit_depth, ctu, R, kFsBand, g, cl);
            if (ctu == 64) full_search_ctas_per_sm(bit_depth, ctu, R, 9, g, cl);
        }
    return cudaGetLastError();
}

int full_search_ctas_per_sm(int bit_depth, int ctu, int R, int band, int group, int cur_l1)
{
    const FullSearchPlan p = full_search_plan(bit_depth, ctu, R, band, group, cur_l1);
    OccupancyOp f{p.smem_bytes, 1};
    dispatch(bit_depth, ctu, p.Rp, p.band, p.cur_l1 != 0, f);
    return f.n;
}

cudaError_t launch_full_search(int bit_depth, int ctu, const FullSearchBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxItems || b.total <= 0) return cudaErrorInvalidValue;
    const FullSearchPlan p = full_search_plan(bit_depth, ctu, b.R, b.band, b.group, b.cur_l1);
    if (p.cur_l1) {
        // every frame of whole 8x8 blocks: no current sample needs replication
        for (int k = 0; k < b.n; ++k)
            if ((b.item[k].W & 7) || (b.item[k].H & 7)) return cudaErrorInvalidValue;
    }
    LaunchOp f{b, p.smem_bytes, s};
    return dispatch(bit_depth, ctu, p.Rp, p.band, p.cur_l1 != 0, f);
}

}  // namespace ladder_impl
