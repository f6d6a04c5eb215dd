// me_dependent.cu -- dependent analysis of one rung in one kernel (one CTA
// per CTU): constraint derivation from the resident reference-rung leaves,
// refinement search around the scaled reference vectors, SATD, cost, split
// and leaf maps (inter-resolution analysis sharing with refinement,
// Sec. 4.3 / 6.3; reuse and refinement controls, App. A.1 / A.2).
//
// Search layout.  The CTA lists the evaluated CUs of every depth, then
// spreads (CU, 8x8 block, candidate-row tile, candidate-column chunk) items
// over its threads.  An item holds the block's 8 current rows in registers,
// walks the 8 + TY - 1 reference rows it needs once each (aligned 32-bit
// loads through L1, one funnel shift to the row start, SPW-1 more for the
// sub-word candidate offsets), and accumulates a TY x KC tile of packed
// absdiff sums: every reference row feeds up to 8 x KC x (8/SPW) packed
// instructions.  Block sums are added into a per-CU candidate table in
// shared memory (integer reductions, so the order is free); one warp per CU
// then takes the argmin of (SAD, |dx|+|dy|, dy, dx).
#include "common.cuh"

#include <algorithm>
#include <cstdlib>
#include <vector>

namespace ladder_impl {
namespace {

using dev::Traits;

__constant__ int c_lambda_q16[52] = {
#include "lambda_table.inc"
};

// SADs of the 8x8 block at (bx, by) for the TY x KC candidates whose
// reference block starts at (xs + j, ys + i).
template <typename T, int KC, int TY>
__device__ __forceinline__ void block_tile_sads(const char *cb, const char *rb, long pitch, int W, int H, int bx,
                                                int by, int xs, int ys, uint32_t (&acc)[TY * KC])
{
    constexpr int SPW = Traits<T>::SPW, BITS = 32 / SPW, WPR = 8 / SPW;
    constexpr int NWN = (8 + KC - 1 + SPW - 1) / SPW;  // words of a reference row segment
    uint32_t cw[8][WPR];
    if (bx + 8 <= W) {
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const char *row = cb + static_cast<long>(min(by + y, H - 1)) * pitch + static_cast<long>(bx) * sizeof(T);
            if constexpr (WPR == 2) {
                const uint2 v = __ldg(reinterpret_cast<const uint2 *>(row));
                cw[y][0] = v.x;
                cw[y][1] = v.y;
            } else {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(row));
                cw[y][0] = v.x;
                cw[y][1] = v.y;
                cw[y][2] = v.z;
                cw[y][3] = v.w;
            }
        }
    } else {
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int cy = min(by + y, H - 1);
#pragma unroll
            for (int m = 0; m < WPR; ++m) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < SPW; ++e)
                    w |= static_cast<uint32_t>(dev::ld_sample<T>(cb, pitch, min(bx + m * SPW + e, W - 1), cy))
                         << (e * BITS);
                cw[y][m] = w;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < TY * KC; ++c) acc[c] = 0;

    const bool xfast = xs >= 0 && (xs / SPW + NWN + 1) * SPW <= W;
    const int sh = (xs & (SPW - 1)) * BITS;
#pragma unroll
    for (int rr = 0; rr < 8 + TY - 1; ++rr) {
        const int ry = min(max(ys + rr, 0), H - 1);
        const char *rowb = rb + static_cast<long>(ry) * pitch;
        uint32_t nw[NWN];
        if (xfast) {
            const uint32_t *rp = reinterpret_cast<const uint32_t *>(rowb) + xs / SPW;
            uint32_t raw[NWN + 1];
#pragma unroll
            for (int m = 0; m <= NWN; ++m) raw[m] = __ldg(rp + m);
#pragma unroll
            for (int m = 0; m < NWN; ++m) nw[m] = __funnelshift_r(raw[m], raw[m + 1], sh);
        } else {
#pragma unroll
            for (int m = 0; m < NWN; ++m) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < SPW; ++e)
                    w |= static_cast<uint32_t>(dev::ld_sample<T>(rb, pitch, min(max(xs + m * SPW + e, 0), W - 1), ry))
                         << (e * BITS);
                nw[m] = w;
            }
        }
        // shw[k][m]: samples starting at sub-word offset k of word m
        uint32_t shw[SPW][NWN];
#pragma unroll
        for (int m = 0; m < NWN; ++m) shw[0][m] = nw[m];
#pragma unroll
        for (int k = 1; k < SPW; ++k)
#pragma unroll
            for (int m = 0; m + 1 < NWN; ++m) shw[k][m] = __funnelshift_r(nw[m], nw[m + 1], k * BITS);
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            const int j = rr - i;  // current row j meets reference row rr at candidate row i
            if (j < 0 || j >= 8) continue;
#pragma unroll
            for (int jx = 0; jx < KC; ++jx) {
                const int q = jx / SPW, k = jx % SPW;
#pragma unroll
                for (int m = 0; m < WPR; ++m)
                    acc[i * KC + jx] = dev::sad_acc<SPW>(cw[j][m], shw[k][q + m], acc[i * KC + jx]);
            }
        }
    }
}

constexpr int kDepThreads = 128;  // 4 warps per CTU

// Reduce-scatter of the candidate tables of the lanes that differ in the
// low LG lane bits (the 8x8 blocks of one CU).  The table has N entries,
// padded with zeros to NCP (a multiple of 32); afterwards each lane holds
// NCP >> LG summed entries in s[0..], candidates off .. off + (NCP >> LG) - 1.
template <int N, int NCP, int LG>
__device__ __forceinline__ int scatter_tables(uint32_t (&s)[N], int lane)
{
    int off = 0;
#pragma unroll
    for (int b = 0; b < LG; ++b) {
        const int half = NCP >> (b + 1);
        const bool up = (lane >> b) & 1;
#pragma unroll
        for (int m = 0; m < half; ++m) {
            if (m >= N) break;
            const uint32_t lo = s[m];
            const uint32_t hi = (m + half < N && (b > 0 || m + half < N)) ? s[m + half] : 0u;
            const uint32_t send = up ? lo : hi;
            const uint32_t keep = up ? hi : lo;
            s[m] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << b);
        }
        off += up ? half : 0;
    }
    return off;
}

// Best key among the held candidates, as SAD << 32 | rank (rank = position
// of the candidate in the (|dx|+|dy|, dy, dx) order).  Candidate c of a
// (ty, dc) job is (dyi, dxi) = (ty*TY + c / KC, dc*KC + c % KC).  The min is
// taken on 32-bit keys SAD << RB | rank when SB + RB <= 32 (SB = bits of the
// CU's largest SAD), else on 64-bit keys.
template <int TY, int KC, int N, int CNT, int SB>
__device__ __forceinline__ unsigned long long held_best(const uint32_t (&s)[N], int off, int ty, int dc, int K,
                                                        const uint16_t *rank, int rb)
{
    const int base = ty * TY * K + dc * KC;
    if (SB + rb <= 32) {
        uint32_t best = 0xffffffffu;
        const uint32_t mul = 1u << rb;
#pragma unroll
        for (int m = 0; m < CNT; ++m) {
            const int c = off + m;
            const int dyi = ty * TY + c / KC, dxi = dc * KC + c % KC;
            if (c < TY * KC && dyi < K && dxi < K) {
                const uint32_t key = s[m] * mul + rank[base + (c / KC) * K + c % KC];
                best = key < best ? key : best;
            }
        }
        if (best == 0xffffffffu) return ~0ull;
        return (static_cast<unsigned long long>(best >> rb) << 32) | (best & (mul - 1u));
    }
    unsigned long long best = ~0ull;
#pragma unroll
    for (int m = 0; m < CNT; ++m) {
        const int c = off + m;
        const int dyi = ty * TY + c / KC, dxi = dc * KC + c % KC;
        if (c < TY * KC && dyi < K && dxi < K) {
            const unsigned long long key =
                (static_cast<unsigned long long>(s[m]) << 32) | rank[base + (c / KC) * K + c % KC];
            best = key < best ? key : best;
        }
    }
    return best;
}

// Bits of the largest SAD of an S x S CU of B-bit samples.
template <typename T> __host__ __device__ constexpr int sad_bits(int S)
{
    return (S == 8 ? 6 : S == 16 ? 8 : S == 32 ? 10 : 12) + (sizeof(T) == 1 ? 8 : 10);
}

template <typename T, int CTU, int KC, int TY>
__global__ void __launch_bounds__(kDepThreads, 4) k_dependent(const __grid_constant__ DependentBatch b)
{
    int ri = 0;  // the batch item of this CTA
    while (ri + 1 < b.n && static_cast<int>(blockIdx.x) >= b.item[ri + 1].cta_begin) ++ri;
    const DependentItem &a = b.item[ri];
    const RungInfo &rinf = b.rung[a.rung];
    const RungInfo &rref = b.rung[b.ref_rung];
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
    using C = dev::Ctu<CTU>;
    constexpr int NT = kDepThreads, NWARP = NT / 32;
    constexpr int NCAND = TY * KC;
    constexpr int NCP = (NCAND + 31) / 32 * 32;  // padded so that 5 halvings stay whole
    __shared__ dev::CtuState<CTU> st;
    __shared__ int16_t s_cx[C::NKEY], s_cy[C::NKEY];
    __shared__ uint8_t s_leaf[C::NKEY], s_splitok[C::NKEY];
    __shared__ unsigned long long s_key[C::NKEY];
    __shared__ int s_list[C::NKEY];       // evaluated CUs (key index), grouped by depth
    __shared__ int s_cnt[C::DMAX + 1];
    __shared__ int s_base[C::DMAX + 2];
    __shared__ int s_wpre[C::DMAX + 2];   // warp-job prefix per depth
    extern __shared__ uint32_t s_dyn[];   // 64x64 CU sums, then rank / unrank tables
    uint32_t *const s_sum = s_dyn;
    uint16_t *const s_rank = reinterpret_cast<uint16_t *>(s_dyn + (2 * b.r + 1) * (2 * b.r + 1));
    uint16_t *const s_unrank = s_rank + (2 * b.r + 1) * (2 * b.r + 1);

    const RungGeom &g = rinf.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ctu_idx = blockIdx.x - a.cta_begin;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const int r = b.r, K = 2 * r + 1, KK = K * K;
    const char *cb = static_cast<const char *>(a.cur);
    const char *rb = static_cast<const char *>(a.ref);

    // 1. local rule of every present CU
    for (int i = tid; i < C::NKEY; i += NT) {
        int d = 0;
        while (d < C::DMAX && i >= key_offset(d + 1)) ++d;
        const int li = i - key_offset(d), n = 1 << d, S = CTU >> d;
        const int cu_x = x0 + (li % n) * S, cu_y = y0 + (li / n) * S;
        const bool present = cu_x < g.W8 && cu_y < g.H8;
        uint8_t leaf = 0, splitok = 0;
        int16_t cx = 0, cy = 0;
        if (present) {
            const bool inside = cu_x + S <= g.W8 && cu_y + S <= g.H8;
            const dev::Rule ru = dev::derive_rule(g, refs, d, cu_x, cu_y);
            cx = static_cast<int16_t>(ru.cx);
            cy = static_cast<int16_t>(ru.cy);
            leaf = inside && ru.allowed_leaf;
            splitok = d < C::DMAX && (!inside || ru.allowed_split);
        }
        s_cx[i] = cx;
        s_cy[i] = cy;
        s_leaf[i] = leaf;
        s_splitok[i] = splitok;
        s_key[i] = ~0ull;
        st.flags[i] = present ? dev::kPresent : 0;
    }
    if (tid <= C::DMAX) s_cnt[tid] = 0;
    for (int x = tid; x < KK; x += NT) {
        s_sum[x] = 0;
        s_rank[x] = b.rank[x];
        s_unrank[x] = b.unrank[x];
    }
    __syncthreads();

    // 2. reachability (every ancestor may split) and the decision flags
    for (int i = tid; i < C::NKEY; i += NT) {
        st.satd[i] = 0;
        st.mvx[i] = INT16_MIN;
        st.mvy[i] = INT16_MIN;
        st.sad[i] = INT32_MAX;
        if (!(st.flags[i] & dev::kPresent)) continue;
        int d = 0;
        while (d < C::DMAX && i >= key_offset(d + 1)) ++d;
        const int li = i - key_offset(d), n = 1 << d;
        const int cxl = li % n, cyl = li / n;
        bool reach = true;
        for (int e = 0; e < d; ++e)
            reach = reach && s_splitok[dev::key_index(e, (cyl >> (d - e)) * (1 << e) + (cxl >> (d - e)))];
        uint8_t f = dev::kPresent;
        if (reach) f |= kRuleReachable;
        if (reach && s_leaf[i]) f |= kRuleEvaluated;
        if (reach && s_splitok[i]) f |= kRuleCanSplit;
        st.flags[i] = f;
        if (f & kRuleEvaluated) atomicAdd(&s_cnt[d], 1);
    }
    __syncthreads();
    const int n_ty = (K + TY - 1) / TY, n_dc = (K + KC - 1) / KC;
    if (tid == 0) {
        s_base[0] = 0;
        s_wpre[0] = 0;
        for (int d = 0; d <= C::DMAX; ++d) {
            s_base[d + 1] = s_base[d] + s_cnt[d];
            const int nblk = ((CTU >> d) / 8) * ((CTU >> d) / 8);
            const int groups = nblk >= 32 ? s_cnt[d] * (nblk / 32) : (s_cnt[d] * nblk + 31) / 32;
            s_wpre[d + 1] = s_wpre[d] + groups * n_ty * n_dc;
            s_cnt[d] = 0;
        }
    }
    __syncthreads();
    for (int i = tid; i < C::NKEY; i += NT) {
        if (!(st.flags[i] & kRuleEvaluated)) continue;
        int d = 0;
        while (d < C::DMAX && i >= key_offset(d + 1)) ++d;
        s_list[s_base[d] + atomicAdd(&s_cnt[d], 1)] = i;
    }
    __syncthreads();

    // 3. refinement search: warp jobs of 32 lanes = 8x8 blocks of CUs of one
    //    depth (the blocks of a CU on consecutive lanes), one (ty, dc) tile.
    const int n_wjobs = s_wpre[C::DMAX + 1];
    for (int wj = warp; wj < n_wjobs; wj += NWARP) {
        int d = 0;
        while (d < C::DMAX && wj >= s_wpre[d + 1]) ++d;
        const int S = CTU >> d, nb = S / 8, nblk = nb * nb;
        int loc = wj - s_wpre[d];
        const int dc = loc % n_dc;
        loc /= n_dc;
        const int ty = loc % n_ty;
        const int grp = loc / n_ty;
        int e, blk;
        if (nblk >= 32) {
            e = grp / (nblk / 32);
            blk = (grp % (nblk / 32)) * 32 + lane;
        } else {
            e = (grp * 32 + lane) / nblk;
            blk = lane % nblk;
        }
        const bool valid = e < s_cnt[d];
        const int i = s_list[s_base[d] + (valid ? e : 0)];
        const int li = i - key_offset(d), n = 1 << d;
        const int bx = x0 + (li % n) * S + (blk % nb) * 8;
        const int by = y0 + (li / n) * S + (blk / nb) * 8;
        uint32_t t[NCAND];
        block_tile_sads<T, KC, TY>(cb, rb, a.pitch_bytes, g.W, g.H, bx, by, bx + s_cx[i] - r + dc * KC,
                                   by + s_cy[i] - r + ty * TY, t);
        if (nblk == 1) {
            const unsigned long long best =
                held_best<TY, KC, NCAND, NCAND, sad_bits<T>(8)>(t, 0, ty, dc, K, s_rank, b.rank_bits);
            if (valid) atomicMin(&s_key[i], best);
        } else if (nblk == 4) {
            const int off = scatter_tables<NCAND, NCP, 2>(t, lane);
            unsigned long long best =
                held_best<TY, KC, NCAND, NCP / 4, sad_bits<T>(16)>(t, off, ty, dc, K, s_rank, b.rank_bits);
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, 1 << b);
                best = o < best ? o : best;
            }
            if (valid && (lane & 3) == 0) atomicMin(&s_key[i], best);
        } else if (nblk == 16) {
            const int off = scatter_tables<NCAND, NCP, 4>(t, lane);
            unsigned long long best =
                held_best<TY, KC, NCAND, NCP / 16, sad_bits<T>(32)>(t, off, ty, dc, K, s_rank, b.rank_bits);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, 1 << b);
                best = o < best ? o : best;
            }
            if (valid && (lane & 15) == 0) atomicMin(&s_key[i], best);
        } else {
            // 64x64: the 64 blocks span two warp jobs; add both halves' sums
            const int off = scatter_tables<NCAND, NCP, 5>(t, lane);
#pragma unroll
            for (int m = 0; m < NCP / 32; ++m) {
                const int c = off + m;
                const int dyi = ty * TY + c / KC, dxi = dc * KC + c % KC;
                if (valid && c < NCAND && dyi < K && dxi < K) atomicAdd(&s_sum[dyi * K + dxi], t[m]);
            }
        }
    }
    __syncthreads();
    if (CTU == 64 && warp == 0 && (st.flags[0] & kRuleEvaluated)) {
        unsigned long long best = ~0ull;
        for (int c = lane; c < KK; c += 32) {
            const unsigned long long key = (static_cast<unsigned long long>(s_sum[c]) << 32) | s_rank[c];
            best = key < best ? key : best;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            best = v < best ? v : best;
        }
        if (lane == 0) s_key[0] = best;
    }
    __syncthreads();
    for (int i = tid; i < C::NKEY; i += NT) {
        if (!(st.flags[i] & kRuleEvaluated)) continue;
        const unsigned long long best = s_key[i];
        const int c = s_unrank[static_cast<uint32_t>(best & 0xffffffffu)];
        st.mvx[i] = static_cast<int16_t>(s_cx[i] + c % K - r);
        st.mvy[i] = static_cast<int16_t>(s_cy[i] + c / K - r);
        st.sad[i] = static_cast<int32_t>(best >> 32);
    }
    __syncthreads();

    // 4. SATD, cost, split, leaf maps
    dev::DecideIO io{a.cur, a.ref, a.pitch_bytes, &rinf.g, a.qp, b.satd_mode, c_lambda_q16,
                     decisions_at(a.block, rinf.off)};
    dev::ctu_decide<T, CTU>(st, io, x0, y0);
}

template <typename T, int CTU, int KC, int TY> cudaError_t ensure_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_dependent<T, CTU, KC, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         65 * 65 * 8);
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T, int CTU> cudaError_t prepare_dependent_t(int r)
{
    if (2 * r + 1 <= 9) return ensure_attr<T, CTU, 9, sizeof(T) == 1 ? 5 : 3>();
    return ensure_attr<T, CTU, 17, sizeof(T) == 1 ? 2 : 1>();
}

template <typename T, int CTU, int KC, int TY>
cudaError_t dependent_t(int r, const DependentBatch &b, cudaStream_t s)
{
    const int K = 2 * r + 1;
    const int smem = K * K * 8;
    auto kern = k_dependent<T, CTU, KC, TY>;
    cudaError_t e = ensure_attr<T, CTU, KC, TY>();
    if (e != cudaSuccess) return e;
    kern<<<b.total_ctas, kDepThreads, smem, s>>>(b);
    return cudaGetLastError();
}

template <typename T, int CTU>
cudaError_t dependent_ctu(int r, const DependentBatch &b, cudaStream_t s)
{
    if (2 * r + 1 <= 9) return dependent_t<T, CTU, 9, sizeof(T) == 1 ? 5 : 3>(r, b, s);
    return dependent_t<T, CTU, 17, sizeof(T) == 1 ? 2 : 1>(r, b, s);
}

}  // namespace

void refine_rank_tables(int r, uint16_t *rank, uint16_t *unrank)
{
    const int K = 2 * r + 1, KK = K * K;
    std::vector<int> order(KK);
    for (int c = 0; c < KK; ++c) order[c] = c;
    // (|dx|+|dy|, dy, dx) with dx = c % K - r, dy = c / K - r
    std::sort(order.begin(), order.end(), [&](int p, int q) {
        const int px = p % K - r, py = p / K - r, qx = q % K - r, qy = q / K - r;
        const int lp = std::abs(px) + std::abs(py), lq = std::abs(qx) + std::abs(qy);
        if (lp != lq) return lp < lq;
        if (py != qy) return py < qy;
        return px < qx;
    });
    for (int k = 0; k < KK; ++k) {
        rank[order[k]] = static_cast<uint16_t>(k);
        unrank[k] = static_cast<uint16_t>(order[k]);
    }
}

cudaError_t prepare_kernels(int bit_depth, int ctu, int R, int r)
{
    cudaError_t e = prepare_full_search(bit_depth, ctu, R);
    if (e != cudaSuccess) return e;
    if (bit_depth == 8)
        return ctu == 64 ? prepare_dependent_t<uint8_t, 64>(r)
                         : (ctu == 32 ? prepare_dependent_t<uint8_t, 32>(r) : prepare_dependent_t<uint8_t, 16>(r));
    return ctu == 64 ? prepare_dependent_t<uint16_t, 64>(r)
                     : (ctu == 32 ? prepare_dependent_t<uint16_t, 32>(r) : prepare_dependent_t<uint16_t, 16>(r));
}

cudaError_t launch_dependent(int bit_depth, int ctu, int r, const DependentBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxDepItems || b.total_ctas <= 0) return cudaErrorInvalidValue;
    if (bit_depth == 8) {
        if (ctu == 64) return dependent_ctu<uint8_t, 64>(r, b, s);
        if (ctu == 32) return dependent_ctu<uint8_t, 32>(r, b, s);
        return dependent_ctu<uint8_t, 16>(r, b, s);
    }
    if (ctu == 64) return dependent_ctu<uint16_t, 64>(r, b, s);
    if (ctu == 32) return dependent_ctu<uint16_t, 32>(r, b, s);
    return dependent_ctu<uint16_t, 16>(r, b, s);
}

}  // namespace ladder_impl
