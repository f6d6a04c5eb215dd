// subpel.cu -- quarter-pel refinement with SATD of an analysed rung (SATD
// finds the quarter-pel vectors, Sec. 5.4.1; the interpolation filters are
// among the encoder's accelerated kernels, Sec. 6.6).
//
// Every evaluated CU starts at its integer vector (in quarter-pel units,
// 4 mv) and cost J = SATD + lambda * se-bits; a half-pel round tries the 8
// neighbours at +-2 quarter units, a quarter-pel round the 8 neighbours at
// +-1 of the best so far; a candidate replaces the best only with a
// strictly lower cost (candidates in raster order).  The split is then
// decided again over the refined costs (ctu_split).
//
// Prediction (reading: the 8-tap luma filters of HEVC for the phases 0,
// 1/4, 1/2, 3/4): P = clip(floor((sum_j f_fy[j] sum_i f_fx[i] Ref(X + i - 3,
// Y + j - 3) + 2^11) / 2^12)) with the reference clamped to the frame.  The
// two sums are exact in fp32 (|sum| <= 112^2 x 1023 < 2^24), so the
// filtering runs as fp32 multiply-adds.
//
// Two launches.  k_interp writes the 16 phase planes of the reference once
// (as an encoder interpolates its reference frames once); k_subpel, one CTA
// per CTU, evaluates (CU, 8x8 block, candidate) work items, one thread each,
// as the SATD of the current block against a block of one plane, and sums
// the block SATDs per CU and candidate in shared memory.
#include "common.cuh"

namespace ladder_impl {
namespace {

constexpr int kSubpelThreads = 256;

__constant__ int c_lambda_q16_sp[52] = {
#include "lambda_table.inc"
};

__device__ __forceinline__ int floor4(int v) { return v >> 2; }  // arithmetic shift: floor(v / 4)

// ---- interpolated planes --------------------------------------------------
// P_(fx,fy)(X, Y) for every phase and every position -4 <= X <= W+3,
// -4 <= Y <= H+3, stored at plane column X + 4, row Y + 4.  Past those
// bounds every tap of the filter reads a clamped edge sample, so the value
// no longer changes: a position outside the plane reads the nearest stored
// one.  The filter runs as two exact fp32 passes over a tile staged in
// shared memory (a horizontal pass for the 4 x phases, then a vertical
// pass for the 4 y phases) and the sum is rounded once.

constexpr int kInterpTW = 32, kInterpTH = 64, kInterpThreads = 256;
constexpr int kInterpSP = kInterpTW + 12;  // staged row: TW + 7 samples, padded (conflict-free float4 reads)
constexpr int kInterpHP = kInterpTW + 4;   // horizontal-pass row, padded
constexpr int kInterpRows = kInterpTH + 7;
constexpr int kInterpSmem = (kInterpRows * kInterpSP + 4 * kInterpRows * kInterpHP) * 4;

// Tap i of the HEVC luma filter of phase f / 4 (a constant wherever f and i are)
__device__ __forceinline__ constexpr float qtap(int f, int i)
{
    constexpr float t[4][8] = {
        {0.f, 0.f, 0.f, 64.f, 0.f, 0.f, 0.f, 0.f},
        {-1.f, 4.f, -10.f, 58.f, 17.f, -5.f, 1.f, 0.f},
        {-1.f, 4.f, -11.f, 40.f, 40.f, -11.f, 4.f, -1.f},
        {0.f, 1.f, -5.f, 17.f, 58.f, -10.f, 4.f, -1.f},
    };
    return t[f][i];
}

// Index of the job whose CTA range (interpolation or refinement) holds this CTA.
__device__ __forceinline__ int job_of_cta(const SubpelBatch &bb, bool interp)
{
    int lo = 0, hi = bb.n - 1;
    const int c = static_cast<int>(blockIdx.x);
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (c >= (interp ? bb.item[mid].icta_begin : bb.item[mid].cta_begin)) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(kInterpThreads, 3) k_interp(const __grid_constant__ SubpelBatch bb)
{
    dev::chain_entry();
    extern __shared__ __align__(16) float interp_smem[];
    float *const s_in = interp_smem;                         // [kInterpRows][kInterpSP]
    float *const s_h = interp_smem + kInterpRows * kInterpSP;  // [4][kInterpRows][kInterpHP]
    const SubpelItem &b = bb.item[job_of_cta(bb, true)];
    const int W = b.g.W, H = b.g.H, Wp = W + 8, Hp = H + 8;
    const int tile = static_cast<int>(blockIdx.x) - b.icta_begin;
    const int u0 = (tile % b.icols) * kInterpTW, v0 = (tile / b.icols) * kInterpTH;
    const int Xs = u0 - 4, Ys = v0 - 4;  // frame position of the tile's first output
    const T *ref = static_cast<const T *>(b.ref);
    const long rpitch = b.pitch_bytes / static_cast<long>(sizeof(T));
    // staged reference: rows Ys-3 .. Ys+TH+3, columns Xs-3 .. Xs+TW+3, clamped
    constexpr int kStaged = kInterpRows * (kInterpTW + 7);
    constexpr int kPer = (kStaged + kInterpThreads - 1) / kInterpThreads;
    T sv[kPer];
#pragma unroll
    for (int n = 0; n < kPer; ++n) {  // every load in flight before the first store
        const int k = min(static_cast<int>(threadIdx.x) + n * kInterpThreads, kStaged - 1);
        const int r = k / (kInterpTW + 7), c = k - r * (kInterpTW + 7);
        const int y = min(max(Ys - 3 + r, 0), H - 1), x = min(max(Xs - 3 + c, 0), W - 1);
        sv[n] = __ldg(ref + static_cast<long>(y) * rpitch + x);
    }
#pragma unroll
    for (int n = 0; n < kPer; ++n) {
        const int k = threadIdx.x + n * kInterpThreads;
        if (k < kStaged) {
            const int r = k / (kInterpTW + 7), c = k - r * (kInterpTW + 7);
            s_in[r * kInterpSP + c] = static_cast<float>(sv[n]);
        }
    }
    __syncthreads();
    // horizontal pass: 8 outputs of one staged row for the 4 x phases
    for (int k = threadIdx.x; k < kInterpRows * (kInterpTW / 8); k += kInterpThreads) {
        const int r = k >> 2, xg = (k & 3) * 8;
        float s[16];
        const float4 *src = reinterpret_cast<const float4 *>(s_in + r * kInterpSP + xg);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float4 q = src[m];
            s[4 * m] = q.x;
            s[4 * m + 1] = q.y;
            s[4 * m + 2] = q.z;
            s[4 * m + 3] = q.w;
        }
#pragma unroll
        for (int fx = 0; fx < 4; ++fx) {
            float h[8];
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                float t = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (qtap(fx, i) != 0.f) t = fmaf(qtap(fx, i), s[x + i], t);
                h[x] = t;
            }
            float4 *dst = reinterpret_cast<float4 *>(s_h + (fx * kInterpRows + r) * kInterpHP + xg);
            dst[0] = make_float4(h[0], h[1], h[2], h[3]);
            dst[1] = make_float4(h[4], h[5], h[6], h[7]);
        }
    }
    __syncthreads();
    // vertical pass: 8 rows x 4 columns of one x phase for the 4 y phases
    const int xq = threadIdx.x & 7, yg = (threadIdx.x >> 3) & 7, fx = threadIdx.x >> 6;
    float4 col[15];
#pragma unroll
    for (int j = 0; j < 15; ++j)
        col[j] = *reinterpret_cast<const float4 *>(s_h + (fx * kInterpRows + yg * 8 + j) * kInterpHP + xq * 4);
    const int u = u0 + xq * 4;
    // Rounding: the accumulator starts at 2^11, and one multiply-add rounded
    // toward -inf gives 1.5 * 2^23 + floor(sum / 2^12) exactly (the result
    // stays in [2^23, 2^24), where the spacing of floats is 1), so the
    // sample is the low bits of the float's pattern after clamping.
    constexpr float kBias = 12582912.f;  // 1.5 * 2^23
    constexpr float kMax = kBias + (sizeof(T) == 1 ? 255.f : 1023.f);
#pragma unroll
    for (int fy = 0; fy < 4; ++fy) {
        char *plane = b.planes + static_cast<long>(fy * 4 + fx) * b.plane_bytes;
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            float a[4] = {2048.f, 2048.f, 2048.f, 2048.f};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (qtap(fy, j) == 0.f) continue;
                const float f = qtap(fy, j);
                a[0] = fmaf(f, col[y + j].x, a[0]);
                a[1] = fmaf(f, col[y + j].y, a[1]);
                a[2] = fmaf(f, col[y + j].z, a[2]);
                a[3] = fmaf(f, col[y + j].w, a[3]);
            }
            uint32_t q[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                q[e] = __float_as_uint(fminf(fmaxf(__fmaf_rd(a[e], 1.f / 4096.f, kBias), kBias), kMax));
            const int v = v0 + yg * 8 + y;
            if (v >= Hp || u >= Wp) continue;
            char *row = plane + static_cast<long>(v) * b.plane_pitch;
            if constexpr (sizeof(T) == 1) {
                const uint32_t lo = __byte_perm(q[0], q[1], 0x0040u), hi = __byte_perm(q[2], q[3], 0x0040u);
                *reinterpret_cast<uint32_t *>(row + u) = __byte_perm(lo, hi, 0x5410u);
            } else {
                *reinterpret_cast<uint2 *>(row + 2 * u) =
                    make_uint2(__byte_perm(q[0], q[1], 0x5410u), __byte_perm(q[2], q[3], 0x5410u));
            }
        }
    }
}

// SATD of the 8x8 block at (px, py) of cur against the block of an
// interpolated plane whose first sample is at plane column pu, row pv, by
// one thread.  Plane rows and columns are clamped to the plane.
template <typename T>
__device__ int satd8_plane(const char *cur, long pitch, int W, int H, int px, int py, const char *plane, long ppitch,
                           int Wp, int Hp, int pu, int pv, int mode)
{
    constexpr int SPW = dev::Traits<T>::SPW, BITS = 32 / SPW, WPR = 8 / SPW;
    const bool cur_fast = px + 8 <= W;
    const bool pl_fast = pu >= 0 && pu + 8 <= Wp;
    const uint32_t sh = static_cast<uint32_t>((pu & (SPW - 1)) * BITS);
    float v[64];
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const int cy = min(py + y, H - 1);
        const char *crow = cur + static_cast<long>(cy) * pitch;
        const char *prow = plane + static_cast<long>(min(max(pv + y, 0), Hp - 1)) * ppitch;
        uint32_t cw[WPR], pw[WPR];
        if (cur_fast) {  // px is a multiple of 8: aligned vector loads
            if constexpr (WPR == 2) {
                const uint2 q = __ldg(reinterpret_cast<const uint2 *>(crow + px));
                cw[0] = q.x;
                cw[1] = q.y;
            } else {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(crow + 2 * px));
                cw[0] = q.x;
                cw[1] = q.y;
                cw[2] = q.z;
                cw[3] = q.w;
            }
        } else {
#pragma unroll
            for (int m = 0; m < WPR; ++m) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < SPW; ++e)
                    w |= static_cast<uint32_t>(__ldg(reinterpret_cast<const T *>(crow) + min(px + m * SPW + e, W - 1)))
                         << (e * BITS);
                cw[m] = w;
            }
        }
        // The planes were written by the previous launch: plain (coherent,
        // L1-cached) loads after the grid dependency wait, never the
        // non-coherent path.
        if (pl_fast) {  // aligned words + one funnel shift
            const uint32_t *rp = reinterpret_cast<const uint32_t *>(prow) + pu / SPW;
            uint32_t raw[WPR + 1];
#pragma unroll
            for (int m = 0; m <= WPR; ++m) raw[m] = rp[m];
#pragma unroll
            for (int m = 0; m < WPR; ++m) pw[m] = __funnelshift_r(raw[m], raw[m + 1], sh);
        } else {
#pragma unroll
            for (int m = 0; m < WPR; ++m) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < SPW; ++e)
                    w |= static_cast<uint32_t>(reinterpret_cast<const T *>(prow)[min(max(pu + m * SPW + e, 0), Wp - 1)])
                         << (e * BITS);
                pw[m] = w;
            }
        }
#pragma unroll
        for (int x = 0; x < 8; ++x)
            v[8 * y + x] = dev::sample_f<T>(cw[x / SPW], x % SPW) - dev::sample_f<T>(pw[x / SPW], x % SPW);
    }
    return dev::satd8_transform(v, mode);
}

// Work list of a CTU: one entry per distinct (8x8 block, centre) among the
// evaluated CUs covering the block (a CU and its sub-CUs often share a
// centre): block | (depths sharing it) << 8.  Block SATDs are exact
// integers, so the order of the additions over entries does not matter.
// *ne must be zero (and visible) before the call.
template <int CTU>
__device__ __forceinline__ void centre_entries(const dev::CtuState<CTU> &st, uint16_t *ent, int *ne)
{
    using C = dev::Ctu<CTU>;
    for (int blk = threadIdx.x; blk < C::NB8; blk += blockDim.x) {
        const int bx = blk % C::N8, by = blk / C::N8;
        int ci[C::DMAX + 1];
        unsigned left = 0;
#pragma unroll
        for (int d = 0; d <= C::DMAX; ++d) {
            ci[d] = dev::key_of_block<CTU>(d, bx, by);
            if (st.flags[ci[d]] & kRuleEvaluated) left |= 1u << d;
        }
#pragma unroll
        for (int d = 0; d <= C::DMAX; ++d) {
            if (!((left >> d) & 1u)) continue;
            unsigned mask = 1u << d;
#pragma unroll
            for (int e = d + 1; e <= C::DMAX; ++e)
                if (((left >> e) & 1u) && st.mvx[ci[e]] == st.mvx[ci[d]] && st.mvy[ci[e]] == st.mvy[ci[d]])
                    mask |= 1u << e;
            left &= ~mask;
            ent[atomicAdd(ne, 1)] = static_cast<uint16_t>(blk | (mask << 8));
        }
    }
}

__device__ __forceinline__ int32_t rate_q(int lam, int qx, int qy)
{
    const long long bits = dev::se_bits(qx) + dev::se_bits(qy);
    return static_cast<int32_t>((static_cast<long long>(lam) * bits + 32768) >> 16);
}

// The CTU's flags (a dependent rung's rules, else its geometry), every
// evaluated CU's integer vector in quarter units and its SATD in st, and
// its cost with the predictor (0, 0) in j (when j is not null).
template <int CTU>
__device__ __forceinline__ void integer_state(const SubpelItem &b, int ctu_idx, int x0, int y0, int lam,
                                              dev::CtuState<CTU> &st, int32_t *j)
{
    using C = dev::Ctu<CTU>;
    const RungGeom &g = b.g;
    const uint8_t *dep_flags = reinterpret_cast<const uint8_t *>(b.block + b.off.dep_flags) +
                               static_cast<long>(ctu_idx) * C::NKEY;
    for (int i = threadIdx.x; i < C::NKEY; i += blockDim.x) {
        int d = 0;
        while (d < C::DMAX && i >= key_offset(d + 1)) ++d;
        const int li = i - key_offset(d), n = 1 << d, S = CTU >> d;
        const int fx = x0 / S + li % n, fy = y0 / S + li / n;
        const bool present = fx * S < g.W8 && fy * S < g.H8;
        uint8_t flags = 0;
        if (b.dependent) {
            flags = __ldcg(dep_flags + i);
        } else if (present) {
            const bool inside = fx * S + S <= g.W8 && fy * S + S <= g.H8;
            flags = dev::kPresent | kRuleReachable | (inside ? kRuleEvaluated : 0) | (d < C::DMAX ? kRuleCanSplit : 0);
        }
        st.flags[i] = flags;
        st.mvx[i] = INT16_MIN;
        st.mvy[i] = INT16_MIN;
        st.satd[i] = INT32_MAX;
        if (flags & kRuleEvaluated) {
            const long gi = static_cast<long>(fy) * g.cols[d] + fx;
            const int qx = 4 * __ldcg(reinterpret_cast<const int16_t *>(b.block + b.off.mvx[d]) + gi);
            const int qy = 4 * __ldcg(reinterpret_cast<const int16_t *>(b.block + b.off.mvy[d]) + gi);
            const int32_t sd = __ldcg(reinterpret_cast<const int32_t *>(b.block + b.off.satd[d]) + gi);
            st.mvx[i] = static_cast<int16_t>(qx);
            st.mvy[i] = static_cast<int16_t>(qy);
            st.satd[i] = sd;
            if (j) j[i] = sd + rate_q(lam, qx, qy);
        }
    }
}

template <typename T, int CTU>
__global__ void __launch_bounds__(kSubpelThreads, 3) k_subpel(const __grid_constant__ SubpelBatch bb)
{
    dev::chain_entry();
    using C = dev::Ctu<CTU>;
    __shared__ dev::CtuState<CTU> st;
    __shared__ int32_t s_j[C::NKEY];
    __shared__ int32_t s_cand[C::NKEY][8];
    __shared__ uint16_t s_ent[(C::DMAX + 1) * C::NB8];
    __shared__ int s_ne;
    const SubpelItem &b = bb.item[job_of_cta(bb, false)];
    const RungGeom &g = b.g;
    const int tid = threadIdx.x;
    const int ctu_idx = static_cast<int>(blockIdx.x) - b.cta_begin;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const int lam = c_lambda_q16_sp[b.qp];
    integer_state<CTU>(b, ctu_idx, x0, y0, lam, st, s_j);
    __syncthreads();
    const char *cur = static_cast<const char *>(b.cur);
#pragma unroll 1
    for (int step = 2; step >= 1; --step) {
        if (tid == 0) s_ne = 0;
        for (int k = tid; k < C::NKEY * 8; k += kSubpelThreads) (&s_cand[0][0])[k] = 0;
        __syncthreads();
        centre_entries<CTU>(st, s_ent, &s_ne);
        __syncthreads();
        const int ne = s_ne;
        // the 8 candidates of one entry in neighbouring threads: their plane
        // reads overlap in L1
        for (int w = tid; w < ne * 8; w += kSubpelThreads) {
            const unsigned e = s_ent[w >> 3];
            const int c = w & 7, blk = e & 0xff, bx = blk % C::N8, by = blk / C::N8;
            const int i0 = dev::key_of_block<CTU>(__ffs(e >> 8) - 1, bx, by);
            const int cc = c < 4 ? c : c + 1;  // raster 3x3 without the centre
            const int qx = st.mvx[i0] + step * (cc % 3 - 1), qy = st.mvy[i0] + step * (cc / 3 - 1);
            const int px = x0 + 8 * bx, py = y0 + 8 * by;
            const char *plane = b.planes + static_cast<long>((qy & 3) * 4 + (qx & 3)) * b.plane_bytes;
            const int v = satd8_plane<T>(cur, b.pitch_bytes, g.W, g.H, px, py, plane, b.plane_pitch, g.W + 8,
                                         g.H + 8, px + floor4(qx) + 4, py + floor4(qy) + 4, bb.satd_mode);
#pragma unroll
            for (int d = 0; d <= C::DMAX; ++d)
                if ((e >> (8 + d)) & 1u) atomicAdd(&s_cand[dev::key_of_block<CTU>(d, bx, by)][c], v);
        }
        __syncthreads();
        for (int i = tid; i < C::NKEY; i += kSubpelThreads) {
            if (!(st.flags[i] & kRuleEvaluated)) continue;
            const int cx = st.mvx[i], cy = st.mvy[i];
            int bx = cx, by = cy;
            int32_t bj = s_j[i], bs = st.satd[i];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int cc = c < 4 ? c : c + 1;
                const int qx = cx + step * (cc % 3 - 1), qy = cy + step * (cc / 3 - 1);
                const int32_t J = s_cand[i][c] + rate_q(lam, qx, qy);
                if (J < bj) {
                    bj = J;
                    bs = s_cand[i][c];
                    bx = qx;
                    by = qy;
                }
            }
            st.mvx[i] = static_cast<int16_t>(bx);
            st.mvy[i] = static_cast<int16_t>(by);
            st.satd[i] = bs;
            s_j[i] = bj;
        }
        __syncthreads();
    }
    dev::ctu_split<CTU>(st, lam, g, b.out, dev::kSplitWriteVectors, x0, y0, true);
}

// ---- spatial MV predictor in the refinement -------------------------------
// Reading: the predictor of the integer decisions (the component-wise median
// of the leaf vectors at A1, B1, B0, available only outside the CU's CTU and
// in an earlier CTU of the WPP wavefront, Sec. 2.2), formed from the refined
// quarter-pel leaf vectors; every candidate's rate, the integer start
// included, is taken against it.  A CU's path through the two rounds
// depends on its predictor (the quarter-pel round centres on the half-pel
// best), and the predictor on the refined vectors of earlier CTUs.  So the
// SATDs of every position the rounds can visit are computed first, in
// parallel (k_subpel_table: the 48 quarter-pel positions within +-3 of
// 4 mv), and one more launch walks the CTUs in wavefront order
// (k_subpel_mvp), choosing each CU's path from its table with its
// predictor and deciding the split.

// One CTA per CTU: the 48 SATDs of every evaluated CU, one thread per
// (entry, position), summed per CU in shared memory.
template <typename T, int CTU>
__global__ void __launch_bounds__(kSubpelThreads, 3) k_subpel_table(const __grid_constant__ SubpelBatch bb)
{
    dev::chain_entry();
    using C = dev::Ctu<CTU>;
    __shared__ dev::CtuState<CTU> st;
    __shared__ int32_t s_tab[C::NKEY][kSubpelTab];
    __shared__ uint16_t s_ent[(C::DMAX + 1) * C::NB8];
    __shared__ int s_ne;
    const SubpelItem &b = bb.item[job_of_cta(bb, false)];
    const RungGeom &g = b.g;
    const int tid = threadIdx.x;
    const int ctu_idx = static_cast<int>(blockIdx.x) - b.cta_begin;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    if (tid == 0) s_ne = 0;
    for (int k = tid; k < C::NKEY * kSubpelTab; k += kSubpelThreads) (&s_tab[0][0])[k] = 0;
    integer_state<CTU>(b, ctu_idx, x0, y0, 0, st, nullptr);
    __syncthreads();
    centre_entries<CTU>(st, s_ent, &s_ne);
    __syncthreads();
    const int ne = s_ne;
    const char *cur = static_cast<const char *>(b.cur);
    // the positions of one entry in neighbouring threads: their plane reads overlap in L1
    for (int w = tid; w < ne * kSubpelTab; w += kSubpelThreads) {
        const int en = w / kSubpelTab, c = w - en * kSubpelTab;
        const unsigned e = s_ent[en];
        const int blk = e & 0xff, bx = blk % C::N8, by = blk / C::N8;
        const int i0 = dev::key_of_block<CTU>(__ffs(e >> 8) - 1, bx, by);
        const int pos = c < 24 ? c : c + 1;  // raster 7x7 without the centre
        const int qx = st.mvx[i0] + pos % 7 - 3, qy = st.mvy[i0] + pos / 7 - 3;
        const int px = x0 + 8 * bx, py = y0 + 8 * by;
        const char *plane = b.planes + static_cast<long>((qy & 3) * 4 + (qx & 3)) * b.plane_bytes;
        const int v = satd8_plane<T>(cur, b.pitch_bytes, g.W, g.H, px, py, plane, b.plane_pitch, g.W + 8, g.H + 8,
                                     px + floor4(qx) + 4, py + floor4(qy) + 4, bb.satd_mode);
#pragma unroll
        for (int d = 0; d <= C::DMAX; ++d)
            if ((e >> (8 + d)) & 1u) atomicAdd(&s_tab[dev::key_of_block<CTU>(d, bx, by)][c], v);
    }
    __syncthreads();
    int32_t *tab = b.table + static_cast<long>(ctu_idx) * C::NKEY * kSubpelTab;
    for (int k = tid; k < C::NKEY * kSubpelTab; k += kSubpelThreads)
        if (st.flags[k / kSubpelTab] & kRuleEvaluated) tab[k] = (&s_tab[0][0])[k];
}

// Wavefront: one CTA walks one CTU row left to right (kMvpThreads threads,
// one per CU key); rows hand their bottom row's refined leaf vectors to the
// row below through generation-tagged words, as the integer decisions'
// wavefront does (same words, later generation).
constexpr int kSpMvpThreads = 128;

template <int CTU>
__global__ void __launch_bounds__(kSpMvpThreads, 8) k_subpel_mvp(const __grid_constant__ SubpelMvpBatch b)
{
    using C = dev::Ctu<CTU>;
    constexpr int N8 = C::N8;
    __shared__ dev::CtuState<CTU> st;
    __shared__ int16_t s_pmx[C::NKEY], s_pmy[C::NKEY];
    __shared__ uint32_t s_left[N8];       // refined right column of the left CTU
    __shared__ uint32_t s_above[N8 + 1];  // refined bottom row of the CTU above, first bottom block of the one above-right
    __shared__ int s_stop;
    const SubpelMvpItem &it = b.item[dev::item_of_cta(b.item, b.n)];
    const RungInfo &ri = b.rung[it.rung];
    const RungGeom &g = ri.g;
    const DevDecisions res = decisions_at(it.block, ri.off);  // the integer vectors and SATDs
    const int nctu = g.ctu_cols * g.ctu_rows;
    unsigned long long *hand = reinterpret_cast<unsigned long long *>(it.block + ri.off.mvp_flag);  // [CTU][N8]
    unsigned *gen = reinterpret_cast<unsigned *>(hand + static_cast<long>(nctu) * N8), *rows_done = gen + 1;
    const uint8_t *dep_flags = reinterpret_cast<const uint8_t *>(it.block + ri.off.dep_flags);
    const int tid = threadIdx.x;
    const int cy = static_cast<int>(blockIdx.x) - it.cta_begin;
    const int lam = c_lambda_q16_sp[it.qp];
    const unsigned target = __ldcg(gen) + 1u;  // published by the previous wavefront launch on this block
    const unsigned want = target + (b.lost_handoff ? 1u : 0u);
    static_assert(C::NKEY <= kSpMvpThreads, "one key per thread");
    const int ki = tid;
    int kd = 0;
    while (kd < C::DMAX && ki >= key_offset(kd + 1)) ++kd;
    const int kli = ki - key_offset(kd), kn = 1 << kd, kS = CTU >> kd;
    // this key's state in CTU column cx and its 8 half-pel SATDs, as loads
    // into registers issued one CTU ahead
    uint8_t p_flags = 0;
    int16_t p_mvx = 0, p_mvy = 0;
    int32_t p_satd = 0;
    int32_t p_half[8];
    auto fetch = [&](int cx) {
        p_flags = 0;
        if (ki >= C::NKEY) return;
        const int fx = cx * kn + kli % kn, fy = cy * kn + kli / kn;
        const bool present = fx * kS < g.W8 && fy * kS < g.H8;
        if (it.dependent) {
            p_flags = __ldcg(dep_flags + static_cast<long>(cy * g.ctu_cols + cx) * C::NKEY + ki);
        } else if (present) {
            const bool inside = fx * kS + kS <= g.W8 && fy * kS + kS <= g.H8;
            p_flags = dev::kPresent | kRuleReachable | (inside ? kRuleEvaluated : 0) | (kd < C::DMAX ? kRuleCanSplit : 0);
        }
        if (p_flags & kRuleEvaluated) {
            const long gi = static_cast<long>(fy) * g.cols[kd] + fx;
            p_mvx = static_cast<int16_t>(4 * __ldcg(res.mvx[kd] + gi));
            p_mvy = static_cast<int16_t>(4 * __ldcg(res.mvy[kd] + gi));
            p_satd = __ldcg(res.satd[kd] + gi);
            const int32_t *row = it.table + (static_cast<long>(cy * g.ctu_cols + cx) * C::NKEY + ki) * kSubpelTab;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int cc = c < 4 ? c : c + 1;
                p_half[c] = __ldcg(row + subpel_tab_index(2 * (cc % 3 - 1), 2 * (cc / 3 - 1)));
            }
        }
    };
    if (tid == 0) s_stop = 0;
    fetch(0);
    for (int cx = 0; cx < g.ctu_cols; ++cx) {
        const int ctu_idx = cy * g.ctu_cols + cx;
        const int x0 = cx * CTU, y0 = cy * CTU;
        // this CTU's state (fetched one CTU ahead)
        const uint8_t flags = p_flags;
        const int mx4 = p_mvx, my4 = p_mvy;
        const int32_t satd0 = p_satd;
        int32_t half[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) half[c] = p_half[c];
        if (cx + 1 < g.ctu_cols) fetch(cx + 1);
        // the refined vectors this CTU reads from the row above (threads 0..N8)
        if (cy > 0 && tid <= N8) {
            const int qcx = tid < N8 ? cx : cx + 1, qb = tid < N8 ? tid : 0;
            uint32_t v = 0;
            if (qcx < g.ctu_cols && qcx * CTU + 8 * qb < g.W8) {
                const unsigned long long *w = hand + (static_cast<long>(cy - 1) * g.ctu_cols + qcx) * N8 + qb;
                bool ok = false;
                for (int n = 0; n < b.spin; ++n) {
                    const unsigned long long x = dev::ld_relaxed64(w);
                    if (static_cast<unsigned>(x >> 32) == want) {
                        v = static_cast<uint32_t>(x);
                        ok = true;
                        break;
                    }
                    if ((n & 255) == 255 && *reinterpret_cast<volatile int *>(b.status) != kStatusOk) break;
                }
                if (!ok) {
                    atomicCAS(b.status, kStatusOk, kStatusTimeout);
                    s_stop = 1;
                }
            }
            s_above[tid] = v;
        }
        __syncthreads();
        if (s_stop) break;
        // predictor and the two rounds of this thread's CU
        if (ki < C::NKEY) {
            st.flags[ki] = flags;
            st.mvx[ki] = INT16_MIN;
            st.mvy[ki] = INT16_MIN;
            st.satd[ki] = INT32_MAX;
            s_pmx[ki] = s_pmy[ki] = 0;
            if (flags & kRuleEvaluated) {
                const int lx = (kli % kn) * kS, ly = (kli / kn) * kS;  // CU position inside the CTU
                const uint32_t a1 = (lx == 0 && cx > 0) ? s_left[(ly + kS - 1) >> 3] : 0u;
                const bool top = ly == 0 && cy > 0;
                const uint32_t b1 = top ? s_above[(lx + kS - 1) >> 3] : 0u;
                uint32_t b0 = 0u;
                if (top && x0 + lx + kS < g.W8) b0 = lx + kS < CTU ? s_above[(lx + kS) >> 3] : s_above[N8];
                const int pqx = dev::median3(dev::mv_x(a1), dev::mv_x(b1), dev::mv_x(b0));
                const int pqy = dev::median3(dev::mv_y(a1), dev::mv_y(b1), dev::mv_y(b0));
                s_pmx[ki] = static_cast<int16_t>(pqx);
                s_pmy[ki] = static_cast<int16_t>(pqy);
                int bx = mx4, by = my4;
                int32_t bs = satd0, bj = satd0 + rate_q(lam, bx - pqx, by - pqy);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int cc = c < 4 ? c : c + 1;
                    const int qx = mx4 + 2 * (cc % 3 - 1), qy = my4 + 2 * (cc / 3 - 1);
                    const int32_t J = half[c] + rate_q(lam, qx - pqx, qy - pqy);
                    if (J < bj) {
                        bj = J;
                        bs = half[c];
                        bx = qx;
                        by = qy;
                    }
                }
                // quarter-pel round around the half-pel best: its 8 SATDs
                // from the table (one more round of loads)
                const int32_t *row = it.table + (static_cast<long>(ctu_idx) * C::NKEY + ki) * kSubpelTab;
                int32_t quarter[8];
                const int hx = bx - mx4, hy = by - my4;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int cc = c < 4 ? c : c + 1;
                    const int ox = hx + cc % 3 - 1, oy = hy + cc / 3 - 1;
                    quarter[c] = (ox == 0 && oy == 0) ? satd0 : __ldcg(row + subpel_tab_index(ox, oy));
                }
                const int cxq = bx, cyq = by;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int cc = c < 4 ? c : c + 1;
                    const int qx = cxq + cc % 3 - 1, qy = cyq + cc / 3 - 1;
                    const int32_t J = quarter[c] + rate_q(lam, qx - pqx, qy - pqy);
                    if (J < bj) {
                        bj = J;
                        bs = quarter[c];
                        bx = qx;
                        by = qy;
                    }
                }
                st.mvx[ki] = static_cast<int16_t>(bx);
                st.mvy[ki] = static_cast<int16_t>(by);
                st.satd[ki] = bs;
            }
        }
        __syncthreads();
        dev::ctu_split<CTU>(st, lam, g, it.out, dev::kSplitWriteVectors, x0, y0, true, s_pmx, s_pmy, b.status);
        __syncthreads();
        // publish the refined bottom row for the row below; keep the right column
        if (tid < N8) {
            if (cy + 1 < g.ctu_rows && x0 + 8 * tid < g.W8)
                dev::st_relaxed64(hand + static_cast<long>(ctu_idx) * N8 + tid,
                                  (static_cast<unsigned long long>(target) << 32) | dev::leaf_mv<CTU>(st, tid, N8 - 1));
        } else if (tid < 2 * N8) {
            s_left[tid - N8] = dev::leaf_mv<CTU>(st, N8 - 1, tid - N8);
        }
        __syncthreads();
    }
    // the last row to finish (decided or given up) publishes the generation
    if (tid == 0 && atomicAdd(rows_done, 1u) == static_cast<unsigned>(g.ctu_rows) - 1u) {
        *rows_done = 0;
        dev::st_release32(gen, target);
    }
}

}  // namespace

long subpel_workspace_layout(int bit_depth, int W, int H, long *plane_pitch, long *plane_bytes)
{
    const long ss = bit_depth == 8 ? 1 : 2;
    // W + 8 stored columns, 8 more for the word loads past a row's last block
    const long pitch = ((static_cast<long>(W) + 16) * ss + 63) / 64 * 64;
    const long bytes = (pitch * (H + 8) + 255) / 256 * 256;
    if (plane_pitch) *plane_pitch = pitch;
    if (plane_bytes) *plane_bytes = bytes;
    return 16 * bytes;
}

template <typename T> cudaError_t interp_smem_attr()
{
    static const cudaError_t e =
        cudaFuncSetAttribute(k_interp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInterpSmem);
    return e;
}

void subpel_interp_tiles(int W, int H, int *cols, int *rows)
{
    *cols = (W + 8 + kInterpTW - 1) / kInterpTW;
    *rows = (H + 8 + kInterpTH - 1) / kInterpTH;
}

cudaError_t launch_subpel(int bit_depth, int ctu, const SubpelBatch &b, int ctas, int interp_ctas, cudaStream_t s)
{
    cudaError_t e;
    if (bit_depth == 8) {
        if ((e = interp_smem_attr<uint8_t>()) != cudaSuccess) return e;
        if ((e = launch_chained(k_interp<uint8_t>, dim3(interp_ctas), dim3(kInterpThreads), kInterpSmem, s, b)) !=
            cudaSuccess)
            return e;
        auto kern = ctu == 64 ? k_subpel<uint8_t, 64> : ctu == 32 ? k_subpel<uint8_t, 32> : k_subpel<uint8_t, 16>;
        return launch_chained(kern, dim3(ctas), dim3(kSubpelThreads), 0, s, b);
    }
    if ((e = interp_smem_attr<uint16_t>()) != cudaSuccess) return e;
    if ((e = launch_chained(k_interp<uint16_t>, dim3(interp_ctas), dim3(kInterpThreads), kInterpSmem, s, b)) !=
        cudaSuccess)
        return e;
    auto kern = ctu == 64 ? k_subpel<uint16_t, 64> : ctu == 32 ? k_subpel<uint16_t, 32> : k_subpel<uint16_t, 16>;
    return launch_chained(kern, dim3(ctas), dim3(kSubpelThreads), 0, s, b);
}

cudaError_t launch_subpel_table(int bit_depth, int ctu, const SubpelBatch &b, int ctas, int interp_ctas,
                                cudaStream_t s)
{
    cudaError_t e;
    if (bit_depth == 8) {
        if ((e = interp_smem_attr<uint8_t>()) != cudaSuccess) return e;
        if ((e = launch_chained(k_interp<uint8_t>, dim3(interp_ctas), dim3(kInterpThreads), kInterpSmem, s, b)) !=
            cudaSuccess)
            return e;
        auto kern = ctu == 64 ? k_subpel_table<uint8_t, 64>
                              : ctu == 32 ? k_subpel_table<uint8_t, 32> : k_subpel_table<uint8_t, 16>;
        return launch_chained(kern, dim3(ctas), dim3(kSubpelThreads), 0, s, b);
    }
    if ((e = interp_smem_attr<uint16_t>()) != cudaSuccess) return e;
    if ((e = launch_chained(k_interp<uint16_t>, dim3(interp_ctas), dim3(kInterpThreads), kInterpSmem, s, b)) !=
        cudaSuccess)
        return e;
    auto kern = ctu == 64 ? k_subpel_table<uint16_t, 64>
                          : ctu == 32 ? k_subpel_table<uint16_t, 32> : k_subpel_table<uint16_t, 16>;
    return launch_chained(kern, dim3(ctas), dim3(kSubpelThreads), 0, s, b);
}

cudaError_t launch_subpel_mvp(int ctu, const SubpelMvpBatch &b, int ctas, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxSubpelItems || ctas < 1) return cudaErrorInvalidValue;
    auto kern = ctu == 64 ? k_subpel_mvp<64> : ctu == 32 ? k_subpel_mvp<32> : k_subpel_mvp<16>;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every row resident: rows wait on the row above
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kSpMvpThreads);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, b);
}

int subpel_mvp_capacity(int ctu, int sm_count)
{
    auto kern = ctu == 64 ? k_subpel_mvp<64> : ctu == 32 ? k_subpel_mvp<32> : k_subpel_mvp<16>;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kSpMvpThreads, 0) != cudaSuccess) return 0;
    return n * sm_count;
}

}  // namespace ladder_impl
