// me_refine.cu -- dependent analysis, motion step: for every CU the
// constraint pass marked "evaluated", the argmin of (SAD, |dx|+|dy|, dy, dx)
// over the (2r+1)^2 candidates centre + (dx, dy) (Sec. 4.3 / 6.3: the reused,
// scaled vector is refined in a small window).
//
// CTA = one CTU.  Depth by depth, the CTA lists its evaluated CUs, then
// spreads (CU, 8x8 block, candidate row) items over its threads; each item
// accumulates the SADs of one 8x8 block for a chunk of KC candidate columns
// in registers (packed absdiff-accumulate on a register copy of the
// reference row, shifted per column with funnel shifts) and adds them into a
// per-CU candidate table in shared memory (integer atomics: order-free).
// One warp per CU then reduces the table to the best 64-bit key.
#include "ladder_internal.h"

#include <algorithm>

namespace ladder_impl {
namespace {

template <typename T> struct Traits;
template <> struct Traits<uint8_t> { static constexpr int SPW = 4; };
template <> struct Traits<uint16_t> { static constexpr int SPW = 2; };

template <int SPW> __device__ __forceinline__ uint32_t sad_acc(uint32_t a, uint32_t b, uint32_t c);
template <> __device__ __forceinline__ uint32_t sad_acc<4>(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
template <> __device__ __forceinline__ uint32_t sad_acc<2>(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("vabsdiff2.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

template <typename T>
__device__ __forceinline__ uint32_t sample(const char *base, long pitch, int x, int y)
{
    return static_cast<uint32_t>(__ldg(reinterpret_cast<const T *>(base + static_cast<long>(y) * pitch) + x));
}

// SADs of the 8x8 block at (bx, by) against reference columns rx0 + c,
// c = 0..KC-1 (only the first kc are stored), reference rows by + mvy + y.
template <typename T, int KC>
__device__ __forceinline__ void block_row_sads(const RefineArgs &a, int bx, int by, int rx0, int mvy, int kc,
                                               uint32_t *dst)
{
    constexpr int SPW = Traits<T>::SPW;
    constexpr int BITS = 32 / SPW;
    constexpr int WPR = 8 / SPW;                     // words per 8-sample row
    constexpr int NRW = (8 + KC - 1 + SPW - 1) / SPW + 1;  // reference words held
    const char *cb = static_cast<const char *>(a.cur);
    const char *rb = static_cast<const char *>(a.ref);
    const int W = a.g.W, H = a.g.H;
    uint32_t acc[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] = 0;
#pragma unroll 1
    for (int y = 0; y < 8; ++y) {
        const int cy = min(by + y, H - 1);
        const int ry = min(max(by + mvy + y, 0), H - 1);
        uint32_t cw[WPR];
#pragma unroll
        for (int m = 0; m < WPR; ++m) {
            uint32_t w = 0;
#pragma unroll
            for (int e = 0; e < SPW; ++e)
                w |= sample<T>(cb, a.pitch_bytes, min(bx + m * SPW + e, W - 1), cy) << (e * BITS);
            cw[m] = w;
        }
        uint32_t rw[NRW];
#pragma unroll
        for (int m = 0; m < NRW; ++m) {
            uint32_t w = 0;
#pragma unroll
            for (int e = 0; e < SPW; ++e) {
                const int x = min(max(rx0 + m * SPW + e, 0), W - 1);
                w |= sample<T>(rb, a.pitch_bytes, x, ry) << (e * BITS);
            }
            rw[m] = w;
        }
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            const int q = c / SPW, sh = (c % SPW) * BITS;
#pragma unroll
            for (int m = 0; m < WPR; ++m) {
                const uint32_t r = sh ? __funnelshift_r(rw[q + m], rw[q + m + 1], sh) : rw[q + m];
                acc[c] = sad_acc<SPW>(cw[m], r, acc[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < KC; ++c)
        if (c < kc) atomicAdd(dst + c, acc[c]);
}

template <typename T, int CTU, int KC>
__global__ void __launch_bounds__(kThreads) k_refine(const RefineArgs a, const int batch)
{
    constexpr int DMAX = CTU == 64 ? 3 : (CTU == 32 ? 2 : 1);
    constexpr int NKEY = keys_per_ctu(DMAX);
    extern __shared__ uint32_t s_sum[];
    __shared__ int s_list[64];
    __shared__ int s_n;

    const RungGeom &g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ctu_idx = blockIdx.x;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const int r = a.r, K = 2 * r + 1, KK = K * K;

    for (int d = 0; d <= DMAX; ++d) {
        const int n = 1 << d, S = CTU >> d, nb = S / 8, NBLK = nb * nb;
        if (tid == 0) s_n = 0;
        __syncthreads();
        for (int li = tid; li < n * n; li += kThreads) {
            const int fx = x0 / S + li % n, fy = y0 / S + li / n;
            if (fx * S < g.W8 && fy * S < g.H8 &&
                (a.rules.flags[d][static_cast<long>(fy) * g.cols[d] + fx] & kRuleEvaluated))
                s_list[atomicAdd(&s_n, 1)] = li;
        }
        __syncthreads();
        const int ncu = s_n;
        for (int b0 = 0; b0 < ncu; b0 += batch) {
            const int nbat = min(batch, ncu - b0);
            for (int i = tid; i < nbat * KK; i += kThreads) s_sum[i] = 0;
            __syncthreads();
            const int nchunk = (K + KC - 1) / KC;
            const long items = static_cast<long>(nbat) * NBLK * K * nchunk;
            for (long it = tid; it < items; it += kThreads) {
                long rem = it;
                const int ch = static_cast<int>(rem % nchunk);
                rem /= nchunk;
                const int dyi = static_cast<int>(rem % K);
                rem /= K;
                const int blk = static_cast<int>(rem % NBLK);
                const int cu = static_cast<int>(rem / NBLK);
                const int li = s_list[b0 + cu];
                const int cux = x0 + (li % n) * S, cuy = y0 + (li / n) * S;
                const long gi = static_cast<long>(cuy / S) * g.cols[d] + cux / S;
                const int cx = a.rules.cx[d][gi], cy = a.rules.cy[d][gi];
                const int bx = cux + (blk % nb) * 8, by = cuy + (blk / nb) * 8;
                const int dx0 = ch * KC;
                const int kc = min(KC, K - dx0);
                block_row_sads<T, KC>(a, bx, by, bx + cx - r + dx0, cy - r + dyi, kc,
                                      s_sum + cu * KK + dyi * K + dx0);
            }
            __syncthreads();
            for (int cu = warp; cu < nbat; cu += kThreads / 32) {
                unsigned long long best = ~0ull;
                for (int c = lane; c < KK; c += 32) {
                    const int dxi = c % K, dyi = c / K;
                    const uint32_t tb = static_cast<uint32_t>((abs(dxi - r) + abs(dyi - r)) * KK + dyi * K + dxi);
                    const unsigned long long key = (static_cast<unsigned long long>(s_sum[cu * KK + c]) << 32) | tb;
                    best = key < best ? key : best;
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
                    best = other < best ? other : best;
                }
                if (lane == 0) {
                    const int li = s_list[b0 + cu];
                    a.keys[static_cast<long>(ctu_idx) * NKEY + key_offset(d) + li] = best;
                }
            }
            __syncthreads();
        }
    }
}

constexpr int kSumBudgetBytes = 48 * 1024;

template <typename T, int CTU>
cudaError_t refine_t(const RefineArgs &a, cudaStream_t s)
{
    const int K = 2 * a.r + 1, KK = K * K;
    const int batch = std::max(1, std::min(64, kSumBudgetBytes / (4 * KK)));
    const int smem = batch * KK * 4;
    const int nctu = a.g.ctu_cols * a.g.ctu_rows;
    if (K <= 9) {
        auto kern = k_refine<T, CTU, 9>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSumBudgetBytes);
        kern<<<nctu, kThreads, smem, s>>>(a, batch);
    } else {
        auto kern = k_refine<T, CTU, 17>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSumBudgetBytes);
        kern<<<nctu, kThreads, smem, s>>>(a, batch);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refine(int bit_depth, const RefineArgs &a, cudaStream_t s)
{
    if (bit_depth == 8) {
        if (a.g.ctu == 64) return refine_t<uint8_t, 64>(a, s);
        if (a.g.ctu == 32) return refine_t<uint8_t, 32>(a, s);
        return refine_t<uint8_t, 16>(a, s);
    }
    if (a.g.ctu == 64) return refine_t<uint16_t, 64>(a, s);
    if (a.g.ctu == 32) return refine_t<uint16_t, 32>(a, s);
    return refine_t<uint16_t, 16>(a, s);
}

}  // namespace ladder_impl
