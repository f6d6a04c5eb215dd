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
//   * CTA = one CTU x one slice of candidate tiles (grid.x = slices,
//     grid.y = CTUs); 256 threads.
//   * The reference window (CTU + 2R rows, CTU + 2Rp samples) is loaded by
//     one TMA tile copy into shared memory (zero fill out of the frame, then
//     the out-of-frame samples are replaced by the clamped ones).  It is then
//     expanded into SPW byte-shifted copies (SPW = samples per 32-bit word)
//     so that every candidate reads whole, aligned words.
//   * Thread = one "unit" of the current CTU held in registers (16x16 samples
//     for 8-bit, 8 wide x 16 high for 10-bit: 16 rows x 4 words either way)
//     x one group of candidate tiles.  A tile is TY consecutive dy by NX
//     consecutive dx of one word class (dx = base + SPW*n): each shared
//     memory row load feeds TY*NX*4 packed absdiff-accumulate instructions
//     (vabsdiff4/vabsdiff2 .add).
//   * 16 / 32 / 64 sums across threads use reduce-scatter shuffles inside a
//     warp (units of a CTU are Z-ordered across lanes), so each level costs
//     a few shuffles per tile instead of one per candidate.
//   * Per-thread running bests are merged with shared-memory atomicMin on the
//     64-bit keys, then into the global per-CTU keys with global atomicMin
//     (slices of the same CTU run in different CTAs).  Integer min is
//     order-independent, so the result is deterministic.
#include "common.cuh"

#include <algorithm>

namespace ladder_impl {
namespace {

using dev::mbar_arrive_expect_tx;
using dev::mbar_init;
using dev::mbar_wait_bounded;
using dev::sad_acc;
using dev::tma_load_2d;
using dev::Traits;

// Origin (in samples, inside the CTU) of unit u.  Units are Z-ordered so
// that lanes sharing a 16x16 / 32x32 / 64x64 CU differ only in low lane bits.
template <int SPW>
__device__ __forceinline__ void unit_origin(int u, int &ux, int &uy)
{
    const int q = (SPW == 4) ? u : (u >> 1);
    const int h = (SPW == 4) ? 0 : (u & 1);
    const int x16 = (q & 1) | ((q >> 1) & 2);
    const int y16 = ((q >> 1) & 1) | ((q >> 2) & 2);
    ux = x16 * 16 + h * 8;
    uy = y16 * 16;
}

// Candidate (dx, dy) of tile-local index c.
template <int SPW, int NX>
__device__ __forceinline__ void cand_of(int c, int dxb, int dyb, int &dx, int &dy)
{
    dx = dxb + SPW * (c % NX);
    dy = dyb + c / NX;
}

// Folds a tile's best 32-bit key (SAD << KS | L1 << LNC | c) into a running
// 64-bit best (SAD << 32 | global tie-break).  The 32-bit key already orders
// the tile's candidates by (SAD, L1, dy, dx); the global tie-break is only
// computed when the tile can win.
template <int SPW, int NX, int KS, int LNC>
__device__ __forceinline__ void fold_key32(unsigned long long &best, uint32_t kmin, int dxb, int dyb, int R, int K)
{
    const uint32_t sad = kmin >> KS;
    if (sad <= static_cast<uint32_t>(best >> 32)) {
        int dx, dy;
        cand_of<SPW, NX>(static_cast<int>(kmin & ((1u << LNC) - 1)), dxb, dyb, dx, dy);
        const uint32_t tb = static_cast<uint32_t>((abs(dx) + abs(dy)) * K * K + (dy + R) * K + (dx + R));
        const unsigned long long key = (static_cast<unsigned long long>(sad) << 32) | tb;
        best = key < best ? key : best;
    }
}

template <int SPW, int NX>
__device__ __forceinline__ void fold_sum(unsigned long long &best, uint32_t sad, int c, int dxb, int dyb, int R,
                                         int K)
{
    if (sad <= static_cast<uint32_t>(best >> 32)) {
        int dx, dy;
        cand_of<SPW, NX>(c, dxb, dyb, dx, dy);
        const uint32_t tb = static_cast<uint32_t>((abs(dx) + abs(dy)) * K * K + (dy + R) * K + (dx + R));
        const unsigned long long key = (static_cast<unsigned long long>(sad) << 32) | tb;
        best = key < best ? key : best;
    }
}

// One reduce-scatter step over lane bit `bit` on the CNT held sums: the lane
// keeps half of them, summed with its partner's copy of that half.
template <int NC, int CNT>
__device__ __forceinline__ void scatter_step(uint32_t (&s)[NC], int &off, int lane, int bit)
{
    if constexpr (CNT >= 2) {
        const bool up = (lane >> bit) & 1;
#pragma unroll
        for (int m = 0; m < CNT / 2; ++m) {
            const uint32_t send = up ? s[m] : s[m + CNT / 2];
            const uint32_t keep = up ? s[m + CNT / 2] : s[m];
            s[m] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << bit);
        }
        off += up ? CNT / 2 : 0;
    } else {
        s[0] += __shfl_xor_sync(0xffffffffu, s[0], 1 << bit);
    }
}

template <int CNT> __host__ __device__ constexpr int after_step() { return CNT >= 2 ? CNT / 2 : 1; }

// Argmin over the CNT held candidates (indices off .. off+CNT-1) of one level.
template <int SPW, int NX, int NC, int CNT, int KS, int LNC>
__device__ __forceinline__ void level_argmin(unsigned long long &best, const uint32_t (&s)[NC],
                                             const uint32_t (&code)[NC], int off, int dxb, int dyb, int R,
                                             int K)
{
    if constexpr (CNT == 1) {
        fold_sum<SPW, NX>(best, s[0], off, dxb, dyb, R, K);
    } else {
        uint32_t kmin = 0xffffffffu;
#pragma unroll
        for (int m = 0; m < CNT; ++m) {
            // code[] is indexed by the tile-local candidate; off is a
            // multiple of CNT, so select with a short unrolled search.
            uint32_t cd = 0;
#pragma unroll
            for (int c = 0; c < NC; c += CNT) cd = (off == c) ? code[c + m] : cd;
            const uint32_t k = (s[m] << KS) | cd;
            kmin = k < kmin ? k : kmin;
        }
        fold_key32<SPW, NX, KS, LNC>(best, kmin, dxb, dyb, R, K);
    }
}

// Min of a 64-bit key over the lanes that differ only in the bits of `mask`.
__device__ __forceinline__ unsigned long long warp_min_over(unsigned long long v, unsigned mask)
{
#pragma unroll
    for (int b = 0; b < 5; ++b)
        if (mask & (1u << b)) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, 1 << b);
            v = o < v ? o : v;
        }
    return v;
}

// Word offset of window row `row`, word `w` in a shifted copy: rows are
// `pw` words apart plus one pad word every 16 rows, so that the lanes of a
// warp (units 16 rows apart, 4 words apart) hit distinct banks.
__device__ __forceinline__ int copy_off(int row, int w, int pw) { return row * pw + (row >> 4) + w; }

template <typename T, int CTU, int TY, int NX>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 1 ? 2 : 1)
    k_full_search(const __grid_constant__ FullSearchBatch b, const int box_h, const int pw, const int cstride)
{
    constexpr int SPW = Traits<T>::SPW;
    constexpr int UW = 4 * SPW;                 // unit width in samples
    constexpr int NU = (CTU / UW) * (CTU / 16); // units per CTU
    constexpr int G = 32 / NU;                  // candidate groups per warp
    constexpr int NG = kThreads / NU;           // candidate groups per CTA
    constexpr int WPB = 8 / SPW;                // words per 8-sample block row
    constexpr int NBH = 4 / WPB;                // 8x8 blocks across a unit
    constexpr int NB = 2 * NBH;                 // 8x8 blocks in a unit
    constexpr int NC = TY * NX;                 // candidates per tile
    constexpr int LNC = NC == 16 ? 4 : (NC == 8 ? 3 : (NC == 4 ? 2 : (NC == 2 ? 1 : 0)));
    constexpr int KS = 8 + LNC;                 // L1 < 256 takes 8 bits
    constexpr int DMAX = CTU == 64 ? 3 : (CTU == 32 ? 2 : 1);
    constexpr int NKEY = keys_per_ctu(DMAX);
    constexpr int B0 = SPW == 4 ? 0 : 1;        // lane bits already spent inside a 16x16
    static_assert((1 << LNC) == NC, "tile size must be a power of two");
    static_assert(NU <= 32 && 32 % NU == 0, "a CTU's units must tile a warp");
    // Key widths: SAD < 2^(32-KS) wherever a level holds >= 2 candidates
    // (8-bit 32x32 <= 261120, 10-bit 32x32 <= 1047552, 10-bit 16x16 <= 261888);
    // single-candidate levels fold the sum directly into 64 bits.

    extern __shared__ __align__(128) uint8_t smem_raw[];
    // staging: the TMA box, dense (box_h rows x pw words); then SPW shifted copies
    uint32_t *const stage =
        reinterpret_cast<uint32_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint32_t *const copies = stage + box_h * pw;
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned long long cta_keys[NKEY];
    __shared__ unsigned long long *s_out_keys;  // this CTU's global keys (read after the main loop)
    // 8-bit: running best keys live in shared memory ([slot][thread], conflict-free)
    // to keep the main loop within 128 registers
    constexpr bool kSmemBest = SPW == 4;
    __shared__ unsigned long long s_best[kSmemBest ? NB + DMAX : 1][kSmemBest ? kThreads : 1];

    int ii = 0;  // the batch item of this CTA row
    while (ii + 1 < b.n && static_cast<int>(blockIdx.y) >= b.item[ii + 1].cta_begin) ++ii;
    const FullSearchItem &a = b.item[ii];
    const CUtensorMap *ref_map = &b.map[ii];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int u = lane % NU;
    const int g = lane / NU;
    const int ctu_idx = blockIdx.y - a.cta_begin;
    const int W8 = (a.W + 7) & ~7;
    const int ctu_cols = (W8 + CTU - 1) / CTU;
    const int x0 = (ctu_idx % ctu_cols) * CTU;
    const int y0 = (ctu_idx / ctu_cols) * CTU;
    const int R = b.R, K = 2 * R + 1;

    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(ref_map)) : "memory");
    }
    for (int i = tid; i < NKEY; i += kThreads) cta_keys[i] = ~0ull;
    if (tid == 0) s_out_keys = a.keys + static_cast<long>(ctu_idx) * NKEY;
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(box_h * pw) * 4u);
        tma_load_2d(stage, ref_map, &bar, x0 - b.Rp, y0 - R);
    }

    // Current unit -> registers while the window is in flight.
    int ux, uy;
    unit_origin<SPW>(u, ux, uy);
    uint32_t cur[16][4];
    {
        const char *base = static_cast<const char *>(a.cur);
        const int gx = x0 + ux;
        const bool full = gx + UW <= a.W;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int gy = min(y0 + uy + j, a.H - 1);
            const char *row = base + static_cast<long>(gy) * a.pitch_bytes;
            if (full) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(row + static_cast<long>(gx) * sizeof(T)));
                cur[j][0] = v.x;
                cur[j][1] = v.y;
                cur[j][2] = v.z;
                cur[j][3] = v.w;
            } else {
                const T *rp = reinterpret_cast<const T *>(row);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    uint32_t w = 0;
#pragma unroll
                    for (int e = 0; e < SPW; ++e) {
                        const int x = min(gx + c * SPW + e, a.W - 1);
                        w |= static_cast<uint32_t>(rp[x]) << (e * (32 / SPW));
                    }
                    cur[j][c] = w;
                }
            }
        }
    }

    // Tiles of this slice; tiles are ordered by candidate row, so the slice
    // needs window rows [r_lo, r_hi) only.
    const int tile_begin = blockIdx.x * b.tiles_per_slice;
    const int tile_end = min(tile_begin + b.tiles_per_slice, b.ntiles);
    const int n_iter = (tile_end - tile_begin + NG - 1) / NG;  // uniform across the CTA
    const int r_lo = (__ldg(b.tiles + tile_begin) >> 16) + R;
    const int r_hi = min(box_h, (__ldg(b.tiles + tile_end - 1) >> 16) + R + TY - 1 + CTU);

    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(b.status, kStatusTimeout);
        if (!ok) mbar_wait_bounded(&bar, 0);
        return;
    }

    // Out-of-frame samples of the window take the clamped sample.
    {
        const int gx0 = x0 - b.Rp, gy0 = y0 - R;
        const int ww = pw * SPW;
        if (gx0 < 0 || gy0 < 0 || gx0 + ww > a.W || gy0 + box_h > a.H) {
            T *w0 = reinterpret_cast<T *>(stage);
            for (int i = r_lo * ww + tid; i < r_hi * ww; i += kThreads) {
                const int row = i / ww, col = i - row * ww;
                const int gx = gx0 + col, gy = gy0 + row;
                const int cx = min(max(gx, 0), a.W - 1), cy = min(max(gy, 0), a.H - 1);
                if (cx != gx || cy != gy) w0[i] = w0[(cy - gy0) * ww + (cx - gx0)];
            }
            __syncthreads();
        }
    }
    // Shifted copies: copy k word w of a row = samples [SPW*w + k, SPW*w + k + SPW).
    {
        const int nw = (r_hi - r_lo) * pw;
        for (int i = tid; i < SPW * nw; i += kThreads) {
            const int k = i / nw, rem = i - k * nw;
            const int row = r_lo + rem / pw, w = rem % pw;
            const uint32_t lo = stage[row * pw + w];
            const uint32_t hi = (w + 1 < pw) ? stage[row * pw + w + 1] : 0u;
            copies[k * cstride + copy_off(row, w, pw)] = __funnelshift_r(lo, hi, k * (32 / SPW));
        }
    }
    __syncthreads();

    // Running bests: 8x8 blocks of the unit, then one per coarser depth.
    unsigned long long rbest[kSmemBest ? 1 : NB + DMAX];
#pragma unroll
    for (int q = 0; q < NB + DMAX; ++q) {
        if constexpr (kSmemBest) s_best[q][tid] = ~0ull;
        else rbest[q] = ~0ull;
    }
    auto best_ref = [&](int q) -> unsigned long long & {
        if constexpr (kSmemBest) return s_best[q][tid];
        else return rbest[q];
    };

    for (int it = 0; it < n_iter; ++it) {
        // the G groups of a warp take G consecutive tiles (paired word classes)
        int t = tile_begin + G * (warp + (kThreads / 32) * it) + g;
        if (t >= tile_end) t = tile_begin;  // a duplicate tile cannot change a min
        const int packed = __ldg(b.tiles + t);
        const int dxb = static_cast<int>(static_cast<short>(packed & 0xffff));
        const int dyb = packed >> 16;
        const int k = dxb & (SPW - 1);
        const uint32_t *cp = copies + k * cstride + (ux + dxb + b.Rp - k) / SPW;
        const int row0 = uy + dyb + R;

        uint32_t acc[NB][NC];
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[b][c] = 0;

#pragma unroll
        for (int rr = 0; rr < 16 + TY - 1; ++rr) {
            uint32_t w[NX + 3];
            const uint32_t *rowp = cp + copy_off(row0 + rr, 0, pw);
#pragma unroll
            for (int c = 0; c < NX + 3; ++c) w[c] = rowp[c];
#pragma unroll
            for (int i = 0; i < TY; ++i) {
                const int j = rr - i;  // current row paired with ref row rr at dy index i
                if (j < 0 || j >= 16) continue;
                const int bv = j >> 3;
#pragma unroll
                for (int n = 0; n < NX; ++n)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int bb = bv * NBH + c / WPB;
                        acc[bb][i * NX + n] = sad_acc<SPW>(cur[j][c], w[n + c], acc[bb][i * NX + n]);
                    }
            }
        }

        // Tile-local tie-break codes: (L1 << LNC) | c orders the tile's
        // candidates by (L1, dy, dx) because dy, dx grow with c.
        uint32_t code[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            int dx, dy;
            cand_of<SPW, NX>(c, dxb, dyb, dx, dy);
            code[c] = (static_cast<uint32_t>(abs(dx) + abs(dy)) << LNC) | static_cast<uint32_t>(c);
        }

        // depth DMAX: the unit's own 8x8 blocks
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            uint32_t kmin = 0xffffffffu;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const uint32_t kk = (acc[b][c] << KS) | code[c];
                kmin = kk < kmin ? kk : kmin;
            }
            fold_key32<SPW, NX, KS, LNC>(best_ref(b), kmin, dxb, dyb, R, K);
        }

        // unit sums
        uint32_t s[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            uint32_t v = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b) v += acc[b][c];
            s[c] = v;
        }
        int off = 0;
        // depth DMAX-1 (16x16)
        if constexpr (B0 == 0) {
            level_argmin<SPW, NX, NC, NC, KS, LNC>(best_ref(NB + DMAX - 1), s, code, off, dxb, dyb, R, K);
        } else {
            scatter_step<NC, NC>(s, off, lane, 0);
            level_argmin<SPW, NX, NC, after_step<NC>(), KS, LNC>(best_ref(NB + DMAX - 1), s, code, off, dxb, dyb, R,
                                                                 K);
        }
        // depth DMAX-2 (32x32)
        if constexpr (DMAX >= 2) {
            constexpr int C0 = (B0 == 0) ? NC : after_step<NC>();
            constexpr int C1 = after_step<C0>();
            constexpr int C2 = after_step<C1>();
            scatter_step<NC, C0>(s, off, lane, B0);
            scatter_step<NC, C1>(s, off, lane, B0 + 1);
            level_argmin<SPW, NX, NC, C2, KS, LNC>(best_ref(NB + DMAX - 2), s, code, off, dxb, dyb, R, K);
            // depth DMAX-3 (64x64)
            if constexpr (DMAX >= 3) {
                constexpr int C3 = after_step<C2>();
                constexpr int C4 = after_step<C3>();
                scatter_step<NC, C2>(s, off, lane, B0 + 2);
                scatter_step<NC, C3>(s, off, lane, B0 + 3);
                level_argmin<SPW, NX, NC, C4, KS, LNC>(best_ref(NB + DMAX - 3), s, code, off, dxb, dyb, R, K);
            }
        }
    }

    // Merge: per-thread bests -> min over the lanes of a warp that share the
    // CU -> CTA keys (shared atomics) -> global keys (atomics across slices).
    // Lane bits: unit bits below log2(NU) (Z-order: 8-bit 2 per level from
    // 32x32 up; 10-bit one for the 16x16 half, then 2 per level), group bits above.
    constexpr int LNU = NU == 32 ? 5 : (NU == 16 ? 4 : (NU == 8 ? 3 : (NU == 4 ? 2 : (NU == 2 ? 1 : 0))));
    constexpr unsigned GROUP_BITS = 0x1fu & ~((1u << LNU) - 1u);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const unsigned long long v = warp_min_over(best_ref(b), GROUP_BITS);
        if ((lane & GROUP_BITS) == 0) {
            const int bx = ux + 8 * (b % NBH), by = uy + 8 * (b / NBH);
            const int li = (by / 8) * (CTU / 8) + bx / 8;
            atomicMin(&cta_keys[key_offset(DMAX) + li], v);
        }
    }
#pragma unroll
    for (int d = 0; d < DMAX; ++d) {
        // unit bits inside a depth-d CU: 8-bit 2*(DMAX-1-d), 10-bit 2*(DMAX-1-d)+1
        const int inner = 2 * (DMAX - 1 - d) + B0;
        const unsigned m = GROUP_BITS | ((1u << inner) - 1u);
        const unsigned long long v = warp_min_over(best_ref(NB + d), m);
        if ((lane & m) == 0) {
            const int S = CTU >> d;
            const int li = (uy / S) * (CTU / S) + ux / S;
            atomicMin(&cta_keys[key_offset(d) + li], v);
        }
    }
    __syncthreads();
    for (int i = tid; i < NKEY; i += kThreads) {
        const unsigned long long v = cta_keys[i];
        if (v != ~0ull) atomicMin(s_out_keys + i, v);
    }
}

constexpr int kTileDY = 4;
constexpr int kTileNX = 2;

// Largest dynamic shared memory already granted to k_full_search<T, CTU>.
template <typename T, int CTU> int &granted_smem()
{
    static int bytes = -1;
    return bytes;
}

template <typename T, int CTU> cudaError_t ensure_smem(int smem)
{
    if (granted_smem<T, CTU>() >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_full_search<T, CTU, kTileDY, kTileNX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) granted_smem<T, CTU>() = smem;
    return e;
}

template <typename T, int CTU>
cudaError_t launch_t(const FullSearchBatch &b, const FullSearchPlan &p, int nslices, int total_ctus, cudaStream_t s)
{
    auto kern = k_full_search<T, CTU, kTileDY, kTileNX>;
    cudaError_t e = ensure_smem<T, CTU>(p.smem_bytes);
    if (e != cudaSuccess) return e;
    dim3 grid(nslices, total_ctus);
    kern<<<grid, kThreads, p.smem_bytes, s>>>(b, p.box_h, p.pitch_words, p.copy_stride);
    return cudaGetLastError();
}

template <typename T, int CTU>
int occupancy_t(int smem)
{
    auto kern = k_full_search<T, CTU, kTileDY, kTileNX>;
    if (ensure_smem<T, CTU>(smem) != cudaSuccess) return 1;
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace

cudaError_t prepare_full_search(int bit_depth, int ctu, int R)
{
    const FullSearchPlan p = full_search_plan(bit_depth, ctu, R);
    // launch_t raises the attribute on first use; doing it here keeps the
    // attribute call out of any later stream capture
    int n = bit_depth == 8 ? (ctu == 64 ? occupancy_t<uint8_t, 64>(p.smem_bytes)
                                        : (ctu == 32 ? occupancy_t<uint8_t, 32>(p.smem_bytes)
                                                     : occupancy_t<uint8_t, 16>(p.smem_bytes)))
                           : (ctu == 64 ? occupancy_t<uint16_t, 64>(p.smem_bytes)
                                        : (ctu == 32 ? occupancy_t<uint16_t, 32>(p.smem_bytes)
                                                     : occupancy_t<uint16_t, 16>(p.smem_bytes)));
    (void)n;
    return cudaGetLastError();
}

int full_search_ctas_per_sm(int bit_depth, int ctu, int R)
{
    const FullSearchPlan p = full_search_plan(bit_depth, ctu, R);
    if (bit_depth == 8)
        return ctu == 64 ? occupancy_t<uint8_t, 64>(p.smem_bytes)
                         : (ctu == 32 ? occupancy_t<uint8_t, 32>(p.smem_bytes) : occupancy_t<uint8_t, 16>(p.smem_bytes));
    return ctu == 64 ? occupancy_t<uint16_t, 64>(p.smem_bytes)
                     : (ctu == 32 ? occupancy_t<uint16_t, 32>(p.smem_bytes) : occupancy_t<uint16_t, 16>(p.smem_bytes));
}

FullSearchPlan full_search_plan(int bit_depth, int ctu, int R)
{
    FullSearchPlan p{};
    const int spw = bit_depth == 8 ? 4 : 2;
    const int Rp = (R + 15) / 16 * 16;
    p.tile_dy = kTileDY;
    p.tile_nx = kTileNX;
    p.pitch_words = (ctu + 2 * Rp) / spw;   // words per window row (a multiple of 4)
    p.box_w = p.pitch_words * spw;
    p.box_h = ctu + 2 * R;
    const int raw = p.box_h * p.pitch_words + (p.box_h >> 4) + 1;
    p.copy_stride = (raw + 31) / 32 * 32 + 16;  // copies of paired word classes 16 banks apart
    p.smem_bytes = (p.box_h * p.pitch_words + spw * p.copy_stride) * 4 + 128;  // + alignment slack
    const int unit_w = 4 * spw;
    const int nu = (ctu / unit_w) * (ctu / 16);
    p.groups = kThreads / nu;
    return p;
}

// Candidate tiles, ordered by candidate row (dy), then by pairs of word
// classes (0,1), (2,3): the two lane groups of a warp take the two tiles of a
// pair, which read the same rows and columns of copies k and k+1.
int full_search_tiles(int bit_depth, int R, int *out, int cap)
{
    const int spw = bit_depth == 8 ? 4 : 2;
    const int n_ty = (2 * R + 1 + kTileDY - 1) / kTileDY;
    int first[4], last[4], ntx[4];
    for (int k = 0; k < spw; ++k) {
        first[k] = -R + (((k + R) % spw) + spw) % spw;
        last[k] = R - (((R - k) % spw) + spw) % spw;
        const int cnt = (last[k] - first[k]) / spw + 1;
        ntx[k] = (cnt + kTileNX - 1) / kTileNX;
    }
    int n = 0;
    auto emit = [&](int dxb, int dyb) {
        if (n < cap && out) out[n] = (dxb & 0xffff) | (dyb << 16);
        ++n;
    };
    for (int ty = 0; ty < n_ty; ++ty) {
        const int dyb = std::min(-R + kTileDY * ty, R - kTileDY + 1);
        for (int k0 = 0; k0 < spw; k0 += 2) {
            const int m = std::max(ntx[k0], ntx[k0 + 1]);
            for (int tx = 0; tx < m; ++tx)
                for (int k = k0; k < k0 + 2; ++k) {
                    const int t = std::min(tx, ntx[k] - 1);
                    emit(std::min(first[k] + spw * kTileNX * t, last[k] - spw * (kTileNX - 1)), dyb);
                }
        }
    }
    return n;
}

cudaError_t launch_full_search(int bit_depth, int ctu, const FullSearchBatch &b, int nslices, int total_ctus,
                               cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxItems || total_ctus <= 0 || nslices <= 0) return cudaErrorInvalidValue;
    const FullSearchPlan p = full_search_plan(bit_depth, ctu, b.R);
    if (bit_depth == 8) {
        if (ctu == 64) return launch_t<uint8_t, 64>(b, p, nslices, total_ctus, s);
        if (ctu == 32) return launch_t<uint8_t, 32>(b, p, nslices, total_ctus, s);
        return launch_t<uint8_t, 16>(b, p, nslices, total_ctus, s);
    }
    if (ctu == 64) return launch_t<uint16_t, 64>(b, p, nslices, total_ctus, s);
    if (ctu == 32) return launch_t<uint16_t, 32>(b, p, nslices, total_ctus, s);
    return launch_t<uint16_t, 16>(b, p, nslices, total_ctus, s);
}

}  // namespace ladder_impl
