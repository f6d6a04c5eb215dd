// decide.cu -- SATD at the chosen vectors, rate-distortion cost, bottom-up
// quadtree split decision and leaf maps (one CTA per CTU); the dependent-mode
// constraint derivation (one thread per CU); key initialisation.
//
//   SATD  -- Sec. 5.4.1, SATD equation (sum of |Hadamard coefficients| of the
//            residual, normalised); Sec. 5.4.2, satd8 / satd_8x4 listings
//            for the two-4x4-per-8x4 mode.
//   cost  -- J = SATD + ((lambdaQ16[qp] * bits(mv) + 2^15) >> 16), bits =
//            signed Exp-Golomb lengths of the quarter-pel components
//            (predictor (0,0)); lambda is the integer table below.
//   split -- Sec. 2.1: a CU splits iff it must (partial CU at the frame
//            edge) or may, and its children's best sum is strictly lower
//            than its own J, or it may not be a leaf.
//   reuse -- Sec. 4.3 / 6.3 and App. A.1-A.2: a dependent CU takes the
//            co-located reference leaf's depth (bounding its own depth to
//            n, n+1 of the projected size) and its MV scaled by the
//            resolution ratio as the search centre.
#include "ladder_internal.h"

#include <algorithm>

namespace ladder_impl {
namespace {

__constant__ int c_lambda_q16[52] = {
#include "lambda_table.inc"
};

__device__ __forceinline__ int se_bits(int v)
{
    const unsigned k = v > 0 ? 2u * static_cast<unsigned>(v) - 1u : static_cast<unsigned>(-2 * v);
    return 2 * (31 - __clz(static_cast<int>(k + 1))) + 1;
}

// In-place unnormalised Walsh-Hadamard transform of N values (natural order).
template <int N>
__device__ __forceinline__ void fwht(int (&v)[N])
{
#pragma unroll
    for (int s = N / 2; s >= 1; s >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((i & s) == 0) {
                const int a = v[i], b = v[i + s];
                v[i] = a + b;
                v[i + s] = a - b;
            }
}

template <typename T>
__device__ __forceinline__ int load_sample(const char *base, long pitch, int x, int y)
{
    return static_cast<int>(__ldg(reinterpret_cast<const T *>(base + static_cast<long>(y) * pitch) + x));
}

// SATD of the 8x8 block at (px, py) against the reference at (px+mvx, py+mvy).
template <typename T>
__device__ int satd8(const DecideArgs &a, int px, int py, int mvx, int mvy)
{
    const char *cb = static_cast<const char *>(a.cur);
    const char *rb = static_cast<const char *>(a.ref);
    const int W = a.g.W, H = a.g.H;
    int d[8][8];
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const int cy = min(py + y, H - 1);
        const int ry = min(max(py + y + mvy, 0), H - 1);
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int cx = min(px + x, W - 1);
            const int rx = min(max(px + x + mvx, 0), W - 1);
            d[y][x] = load_sample<T>(cb, a.pitch_bytes, cx, cy) - load_sample<T>(rb, a.pitch_bytes, rx, ry);
        }
    }
    if (a.satd_mode == 0) {
        // 8x8 Hadamard: rows, then columns; (sum |T|) >> 2
#pragma unroll
        for (int y = 0; y < 8; ++y) fwht<8>(d[y]);
        int sum = 0;
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            int col[8];
#pragma unroll
            for (int y = 0; y < 8; ++y) col[y] = d[y][x];
            fwht<8>(col);
#pragma unroll
            for (int y = 0; y < 8; ++y) sum += abs(col[y]);
        }
        return sum >> 2;
    }
    // two 4x4 Hadamards per 8x4 half, (sum of both) >> 1, halves added
    int total = 0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        int s = 0;
#pragma unroll
        for (int bx = 0; bx < 8; bx += 4) {
            int blk[4][4];
#pragma unroll
            for (int y = 0; y < 4; ++y) {
#pragma unroll
                for (int x = 0; x < 4; ++x) blk[y][x] = d[4 * half + y][bx + x];
                fwht<4>(blk[y]);
            }
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                int col[4];
#pragma unroll
                for (int y = 0; y < 4; ++y) col[y] = blk[y][x];
                fwht<4>(col);
#pragma unroll
                for (int y = 0; y < 4; ++y) s += abs(col[y]);
            }
        }
        total += s >> 1;
    }
    return total;
}

template <typename T, int CTU>
__global__ void __launch_bounds__(kThreads) k_decide(const DecideArgs a)
{
    constexpr int DMAX = CTU == 64 ? 3 : (CTU == 32 ? 2 : 1);
    constexpr int NKEY = keys_per_ctu(DMAX);
    constexpr int N8 = CTU / 8;
    constexpr int NB8 = N8 * N8;
    constexpr uint8_t kPresent = 8;

    __shared__ int32_t s_satd[NKEY], s_sad[NKEY], s_best[NKEY];
    __shared__ int16_t s_mvx[NKEY], s_mvy[NKEY];
    __shared__ uint8_t s_flags[NKEY], s_split[NKEY];

    const RungGeom &g = a.g;
    const int tid = threadIdx.x;
    const int ctu_idx = blockIdx.x;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const int K = 2 * a.range + 1;

    // 1. flags, vectors and SADs of every CU of the CTU
    for (int i = tid; i < NKEY; i += kThreads) {
        int d = 0;
        while (d < DMAX && i >= key_offset(d + 1)) ++d;
        const int li = i - key_offset(d), n = 1 << d, S = CTU >> d;
        const int fx = x0 / S + li % n, fy = y0 / S + li / n;
        const bool present = fx * S < g.W8 && fy * S < g.H8;
        uint8_t flags = 0;
        int cx = 0, cy = 0;
        if (present) {
            if (a.dependent) {
                const long gi = static_cast<long>(fy) * g.cols[d] + fx;
                flags = a.rules.flags[d][gi];
                cx = a.rules.cx[d][gi];
                cy = a.rules.cy[d][gi];
            } else {
                const bool inside = fx * S + S <= g.W8 && fy * S + S <= g.H8;
                flags = kRuleReachable | (inside ? kRuleEvaluated : 0) | (d < DMAX ? kRuleCanSplit : 0);
            }
            flags |= kPresent;
        }
        s_flags[i] = flags;
        s_satd[i] = 0;
        if (flags & kRuleEvaluated) {
            const unsigned long long key = a.keys[static_cast<long>(ctu_idx) * NKEY + i];
            const uint32_t tb = static_cast<uint32_t>(key & 0xffffffffu);
            const int rem = static_cast<int>(tb % static_cast<uint32_t>(K * K));
            s_mvx[i] = static_cast<int16_t>(cx + rem % K - a.range);
            s_mvy[i] = static_cast<int16_t>(cy + rem / K - a.range);
            s_sad[i] = static_cast<int32_t>(key >> 32);
        } else {
            s_mvx[i] = INT16_MIN;
            s_mvy[i] = INT16_MIN;
            s_sad[i] = INT32_MAX;
        }
    }
    __syncthreads();

    // 2. SATD of every (depth, 8x8 block) pair whose CU is evaluated
    for (int t = tid; t < (DMAX + 1) * NB8; t += kThreads) {
        const int d = t / NB8, b = t % NB8;
        const int bx = b % N8, by = b / N8;
        const int S = CTU >> d;
        const int i = key_offset(d) + ((by * 8) / S) * (1 << d) + (bx * 8) / S;
        if (!(s_flags[i] & kRuleEvaluated)) continue;
        const int v = satd8<T>(a, x0 + 8 * bx, y0 + 8 * by, s_mvx[i], s_mvy[i]);
        atomicAdd(&s_satd[i], v);
    }
    __syncthreads();

    // 3. cost and bottom-up split, finest depth first
    const int lam = c_lambda_q16[a.qp];
    for (int d = DMAX; d >= 0; --d) {
        const int n = 1 << d, S = CTU >> d;
        for (int li = tid; li < n * n; li += kThreads) {
            const int i = key_offset(d) + li;
            const uint8_t f = s_flags[i];
            if (!(f & kPresent)) continue;
            const bool ev = f & kRuleEvaluated;
            int32_t J = INT32_MAX;
            if (ev) {
                const long long bits = se_bits(4 * s_mvx[i]) + se_bits(4 * s_mvy[i]);
                J = s_satd[i] + static_cast<int32_t>((static_cast<long long>(lam) * bits + 32768) >> 16);
            }
            int32_t best = J;
            uint8_t split = 0;
            if (d < DMAX) {
                const bool can_split = f & kRuleCanSplit;
                int32_t children = 0;
                if (can_split) {
                    const int cxl = li % n, cyl = li / n;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ci = key_offset(d + 1) + (2 * cyl + (q >> 1)) * (2 * n) + 2 * cxl + (q & 1);
                        if (s_flags[ci] & kPresent) children += s_best[ci];
                    }
                }
                split = can_split && (!ev || children < J);
                best = !(f & kRuleReachable) ? INT32_MAX : (split ? children : J);
            }
            s_best[i] = best;
            s_split[i] = split;
            const long gi = static_cast<long>(y0 / S + li / n) * g.cols[d] + x0 / S + li % n;
            a.out.mvx[d][gi] = s_mvx[i];
            a.out.mvy[d][gi] = s_mvy[i];
            a.out.sad[d][gi] = s_sad[i];
            a.out.satd[d][gi] = ev ? s_satd[i] : INT32_MAX;
            a.out.cost[d][gi] = J;
            a.out.best[d][gi] = best;
            a.out.split[d][gi] = split;
            a.out.evaluated[d][gi] = ev ? 1 : 0;
        }
        __syncthreads();
    }

    // 4. leaf depth and vector of every present 8x8
    for (int b = tid; b < NB8; b += kThreads) {
        const int bx = b % N8, by = b / N8;
        const int px = x0 + 8 * bx, py = y0 + 8 * by;
        if (px >= g.W8 || py >= g.H8) continue;
        int d = 0, i = 0;
        for (;;) {
            const int S = CTU >> d;
            i = key_offset(d) + ((by * 8) / S) * (1 << d) + (bx * 8) / S;
            if (d == DMAX || !s_split[i]) break;
            ++d;
        }
        const long li = static_cast<long>(py / 8) * g.cols8 + px / 8;
        a.out.leaf_depth[li] = static_cast<uint8_t>(d);
        a.out.leaf_mvx[li] = s_mvx[i];
        a.out.leaf_mvy[li] = s_mvy[i];
    }
}

// ---- dependent-mode constraint derivation --------------------------------
struct Rule {
    int cx, cy;
    bool allowed_leaf, allowed_split;
};

__device__ __forceinline__ int scale_component(int v, int to, int from)
{
    const long long av = v < 0 ? -static_cast<long long>(v) : v;
    const long long s = (2 * av * to + from) / (2LL * from);  // round half away from zero
    const int r = static_cast<int>(v < 0 ? -s : s);
    return min(max(r, -256), 256);
}

__device__ Rule derive(const RuleArgs &a, int d, int x0, int y0)
{
    const RungGeom &g = a.g;
    const int S = g.ctu >> d;
    // co-located point of the CU centre in the reference rung
    long long xm = (static_cast<long long>(2 * x0 + S) * a.Wr) / (2LL * g.W);
    long long ym = (static_cast<long long>(2 * y0 + S) * a.Hr) / (2LL * g.H);
    xm = xm > a.Wr - 1 ? a.Wr - 1 : xm;
    ym = ym > a.Hr - 1 ? a.Hr - 1 : ym;
    const long li = (ym >> 3) * a.cols8_r + (xm >> 3);
    const int depth_r = a.ref_leaf_depth[li];
    Rule r;
    if (a.use_ref_mv) {
        r.cx = scale_component(a.ref_leaf_mvx[li], g.W, a.Wr);
        r.cy = scale_component(a.ref_leaf_mvy[li], g.H, a.Hr);
    } else {
        r.cx = r.cy = 0;
    }
    // Deq: deepest depth whose CU still covers the projected reference leaf
    const long long proj = static_cast<long long>(g.ctu >> depth_r) * g.W;
    int deq = 0;
    for (int dd = 0; dd <= g.dmax; ++dd)
        if (static_cast<long long>(g.ctu >> dd) * a.Wr >= proj) deq = dd;
    r.allowed_split = d < g.dmax && d < deq + a.depth_hi;
    r.allowed_leaf = (deq + a.depth_lo <= d && d <= deq + a.depth_hi) || d == g.dmax || !r.allowed_split;
    return r;
}

__global__ void k_rules(const RuleArgs a)
{
    const RungGeom &g = a.g;
    long t = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
    int d = 0;
    while (d <= g.dmax && t >= static_cast<long>(g.cols[d]) * g.rows[d]) {
        t -= static_cast<long>(g.cols[d]) * g.rows[d];
        ++d;
    }
    if (d > g.dmax) return;
    const int S = g.ctu >> d;
    const int fx = static_cast<int>(t % g.cols[d]), fy = static_cast<int>(t / g.cols[d]);
    const int x0 = fx * S, y0 = fy * S;
    bool reachable = true;
    for (int e = 0; e < d; ++e) {  // every ancestor must be able to split
        const int Se = g.ctu >> e;
        const int ax = x0 / Se * Se, ay = y0 / Se * Se;
        const bool forced = ax + Se > g.W8 || ay + Se > g.H8;
        if (!forced && !derive(a, e, ax, ay).allowed_split) {
            reachable = false;
            break;
        }
    }
    const Rule r = derive(a, d, x0, y0);
    const bool inside = x0 + S <= g.W8 && y0 + S <= g.H8;
    uint8_t flags = 0;
    if (reachable) flags |= kRuleReachable;
    if (reachable && inside && r.allowed_leaf) flags |= kRuleEvaluated;
    if (reachable && (!inside || r.allowed_split) && d < g.dmax) flags |= kRuleCanSplit;
    a.rules.cx[d][t] = static_cast<int16_t>(r.cx);
    a.rules.cy[d][t] = static_cast<int16_t>(r.cy);
    a.rules.flags[d][t] = flags;
}

__global__ void k_fill_keys(unsigned long long *keys, long n)
{
    for (long i = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x)
        keys[i] = ~0ull;
}

template <typename T, int CTU>
cudaError_t decide_t(const DecideArgs &a, cudaStream_t s)
{
    k_decide<T, CTU><<<a.g.ctu_cols * a.g.ctu_rows, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decide(int bit_depth, const DecideArgs &a, cudaStream_t s)
{
    if (bit_depth == 8) {
        if (a.g.ctu == 64) return decide_t<uint8_t, 64>(a, s);
        if (a.g.ctu == 32) return decide_t<uint8_t, 32>(a, s);
        return decide_t<uint8_t, 16>(a, s);
    }
    if (a.g.ctu == 64) return decide_t<uint16_t, 64>(a, s);
    if (a.g.ctu == 32) return decide_t<uint16_t, 32>(a, s);
    return decide_t<uint16_t, 16>(a, s);
}

cudaError_t launch_rules(const RuleArgs &a, cudaStream_t s)
{
    long n = 0;
    for (int d = 0; d <= a.g.dmax; ++d) n += static_cast<long>(a.g.cols[d]) * a.g.rows[d];
    const int blocks = static_cast<int>((n + kThreads - 1) / kThreads);
    k_rules<<<blocks, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fill_keys(unsigned long long *keys, long n, cudaStream_t s)
{
    const int blocks = static_cast<int>(std::min<long>((n + kThreads - 1) / kThreads, 1024));
    k_fill_keys<<<blocks > 0 ? blocks : 1, kThreads, 0, s>>>(keys, n);
    return cudaGetLastError();
}

}  // namespace ladder_impl
