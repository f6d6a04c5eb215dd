// subpel.cu -- quarter-pel refinement with SATD of an analysed rung (SATD
// finds the quarter-pel vectors, Sec. 5.4.1; the interpolation filters are
// among the encoder's accelerated kernels, Sec. 6.6).
//
// One CTA per CTU.  Every evaluated CU starts at its integer vector (in
// quarter-pel units, 4 mv) and cost J = SATD + lambda * se-bits; a half-pel
// round tries the 8 neighbours at +-2 quarter units, a quarter-pel round
// the 8 neighbours at +-1 of the best so far; a candidate replaces the best
// only with a strictly lower cost (candidates in raster order).  The split
// is then decided again over the refined costs (ctu_split).
//
// Prediction (reading: the 8-tap luma filters of HEVC for the phases 0,
// 1/4, 1/2, 3/4): P = clip(floor((sum_j f_fy[j] sum_i f_fx[i] Ref(X + i - 3,
// Y + j - 3) + 2^11) / 2^12)) with the reference clamped to the frame.  The
// two sums are exact in fp32 (|sum| <= 112^2 x 1023 < 2^24), so the
// filtering runs as fp32 multiply-adds.  Work items are (CU, 8x8 block,
// candidate) triples, one thread each; block SATDs are summed per CU and
// candidate in shared memory.
#include "common.cuh"

namespace ladder_impl {
namespace {

constexpr int kSubpelThreads = 256;

__constant__ float c_qfilt[4][8] = {
    {0.f, 0.f, 0.f, 64.f, 0.f, 0.f, 0.f, 0.f},
    {-1.f, 4.f, -10.f, 58.f, 17.f, -5.f, 1.f, 0.f},
    {-1.f, 4.f, -11.f, 40.f, 40.f, -11.f, 4.f, -1.f},
    {0.f, 1.f, -5.f, 17.f, 58.f, -10.f, 4.f, -1.f},
};

__constant__ int c_lambda_q16_sp[52] = {
#include "lambda_table.inc"
};

__device__ __forceinline__ int floor4(int v) { return v >> 2; }  // arithmetic shift: floor(v / 4)

// Sample k of a packed word as a float: its bits placed under the exponent
// of 2^23 by a byte permute, then 2^23 subtracted (exact, no conversion).
template <typename T>
__device__ __forceinline__ float word_sample(uint32_t w, int k)
{
    const uint32_t sel = sizeof(T) == 1 ? 0x7540u + static_cast<uint32_t>(k)
                                        : 0x7400u + static_cast<uint32_t>(2 * k) + (static_cast<uint32_t>(2 * k + 1) << 4);
    return __int_as_float(static_cast<int>(__byte_perm(w, 0x4b000000u, sel))) - 8388608.f;
}

// 16 consecutive samples X0 .. X0+15 of row y as floats (2^23 + sample
// would lose nothing, but plain values are exact too: samples < 2^10).
template <typename T>
__device__ __forceinline__ void ref_row16(const char *ref, long pitch, int W, int H, int X0, int y, float (&s)[16])
{
    constexpr int SPW = dev::Traits<T>::SPW;
    const char *row = ref + static_cast<long>(min(max(y, 0), H - 1)) * pitch;
    if constexpr (SPW == 4) {
        const int q = X0 >> 2;
        if (X0 >= 0 && 4 * q + 20 <= W) {
            const uint32_t *rp = reinterpret_cast<const uint32_t *>(row) + q;
            uint32_t w[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) w[m] = __ldg(rp + m);
            const uint32_t sh = 8u * static_cast<uint32_t>(X0 & 3);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint32_t a = __funnelshift_r(w[m], w[m + 1], sh);
#pragma unroll
                for (int e = 0; e < 4; ++e) s[4 * m + e] = word_sample<T>(a, e);
            }
            return;
        }
    } else {
        const int q = X0 >> 1;
        if (X0 >= 0 && 2 * q + 18 <= W) {
            const uint32_t *rp = reinterpret_cast<const uint32_t *>(row) + q;
            uint32_t w[9];
#pragma unroll
            for (int m = 0; m < 9; ++m) w[m] = __ldg(rp + m);
            const uint32_t sh = 16u * static_cast<uint32_t>(X0 & 1);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const uint32_t a = __funnelshift_r(w[m], w[m + 1], sh);
                s[2 * m] = word_sample<T>(a, 0);
                s[2 * m + 1] = word_sample<T>(a, 1);
            }
            return;
        }
    }
    const T *rt = reinterpret_cast<const T *>(row);
#pragma unroll
    for (int k = 0; k < 16; ++k) s[k] = static_cast<float>(__ldg(rt + min(max(X0 + k, 0), W - 1)));
}

// SATD of the 8x8 block at (px, py) against the quarter-pel prediction at
// (qx, qy), by one thread.
template <typename T>
__device__ int satd8_qpel(const char *cur, const char *ref, long pitch, int W, int H, int px, int py, int qx, int qy,
                          int mode)
{
    const int X0 = px + floor4(qx) - 3, Y0 = py + floor4(qy) - 3;
    const int fx = qx & 3, fy = qy & 3;
    float hf[8], vf[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        hf[i] = c_qfilt[fx][i];
        vf[i] = c_qfilt[fy][i];
    }
    float acc[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) acc[i] = 0.f;
#pragma unroll
    for (int r = 0; r < 15; ++r) {
        float s[16];
        ref_row16<T>(ref, pitch, W, H, X0, Y0 + r, s);
        float h[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            float t = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) t = fmaf(hf[i], s[x + i], t);
            h[x] = t;
        }
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int j = r - y;
            if (j >= 0 && j < 8) {
#pragma unroll
                for (int x = 0; x < 8; ++x) acc[8 * y + x] = fmaf(vf[j], h[x], acc[8 * y + x]);
            }
        }
    }
    // prediction = clip(floor(acc / 4096 + 1/2)) (exact: acc is an integer, the scaling a power of 2)
    const float maxv = sizeof(T) == 1 ? 255.f : 1023.f;
    const bool cur_fast = px + 8 <= W;
    constexpr int SPW = dev::Traits<T>::SPW, WPR = 8 / SPW;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const int cy = min(py + y, H - 1);
        const char *crow = cur + static_cast<long>(cy) * pitch;
        uint32_t cw[WPR];
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
                         << (e * 32 / SPW);
                cw[m] = w;
            }
        }
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const float p = fminf(fmaxf(floorf(fmaf(acc[8 * y + x], 1.f / 4096.f, 0.5f)), 0.f), maxv);
            acc[8 * y + x] = word_sample<T>(cw[x / SPW], x % SPW) - p;
        }
    }
    return dev::satd8_transform(acc, mode);
}

__device__ __forceinline__ int32_t rate_q(int lam, int qx, int qy)
{
    const long long bits = dev::se_bits(qx) + dev::se_bits(qy);
    return static_cast<int32_t>((static_cast<long long>(lam) * bits + 32768) >> 16);
}

template <typename T, int CTU>
__global__ void __launch_bounds__(kSubpelThreads, 1) k_subpel(const __grid_constant__ SubpelBatch b)
{
    dev::chain_entry();
    using C = dev::Ctu<CTU>;
    __shared__ dev::CtuState<CTU> st;
    __shared__ int32_t s_j[C::NKEY];
    __shared__ int32_t s_cand[C::NKEY][8];
    __shared__ uint16_t s_ent[(C::DMAX + 1) * C::NB8];
    __shared__ int s_ne;
    const RungGeom &g = b.g;
    const int tid = threadIdx.x;
    const int ctu_idx = blockIdx.x;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const int lam = c_lambda_q16_sp[b.qp];
    const uint8_t *dep_flags = reinterpret_cast<const uint8_t *>(b.block + b.off.dep_flags) +
                               static_cast<long>(ctu_idx) * C::NKEY;
    if (tid == 0) s_ne = 0;
    // the CU's flags, its integer vector in quarter units and its cost
    for (int i = tid; i < C::NKEY; i += kSubpelThreads) {
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
            s_j[i] = sd + rate_q(lam, qx, qy);
        }
    }
    __syncthreads();
    // (CU, 8x8 block) entries of the evaluated CUs: CU | block << 7
    for (int i = tid; i < C::NKEY; i += kSubpelThreads) {
        if (!(st.flags[i] & kRuleEvaluated)) continue;
        int d = 0;
        while (d < C::DMAX && i >= key_offset(d + 1)) ++d;
        const int li = i - key_offset(d), n = 1 << d, S = CTU >> d, nb = S / 8;
        const int bx0 = (li % n) * nb, by0 = (li / n) * nb;
        const int base = atomicAdd(&s_ne, nb * nb);
        for (int k = 0; k < nb * nb; ++k) {
            const int blk = (by0 + k / nb) * C::N8 + bx0 + k % nb;
            s_ent[base + k] = static_cast<uint16_t>(i | (blk << 7));
        }
    }
    __syncthreads();
    const int ne = s_ne;
    const char *cur = static_cast<const char *>(b.cur), *ref = static_cast<const char *>(b.ref);
#pragma unroll 1
    for (int step = 2; step >= 1; --step) {
        for (int k = tid; k < C::NKEY * 8; k += kSubpelThreads) (&s_cand[0][0])[k] = 0;
        __syncthreads();
        // the 8 candidates of one (CU, block) in neighbouring threads: their
        // reference windows overlap in L1
        for (int w = tid; w < ne * 8; w += kSubpelThreads) {
            const unsigned e = s_ent[w >> 3];
            const int c = w & 7, i = e & 127, blk = e >> 7;
            const int cc = c < 4 ? c : c + 1;  // raster 3x3 without the centre
            const int qx = st.mvx[i] + step * (cc % 3 - 1), qy = st.mvy[i] + step * (cc / 3 - 1);
            const int v = satd8_qpel<T>(cur, ref, b.pitch_bytes, g.W, g.H, x0 + 8 * (blk % C::N8),
                                        y0 + 8 * (blk / C::N8), qx, qy, b.satd_mode);
            atomicAdd(&s_cand[i][c], v);
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

}  // namespace

cudaError_t launch_subpel(int bit_depth, int ctu, const SubpelBatch &b, cudaStream_t s)
{
    const dim3 grid(b.g.ctu_cols * b.g.ctu_rows);
    if (bit_depth == 8) {
        auto kern = ctu == 64 ? k_subpel<uint8_t, 64> : ctu == 32 ? k_subpel<uint8_t, 32> : k_subpel<uint8_t, 16>;
        return launch_chained(kern, grid, dim3(kSubpelThreads), 0, s, b);
    }
    auto kern = ctu == 64 ? k_subpel<uint16_t, 64> : ctu == 32 ? k_subpel<uint16_t, 32> : k_subpel<uint16_t, 16>;
    return launch_chained(kern, grid, dim3(kSubpelThreads), 0, s, b);
}

}  // namespace ladder_impl
