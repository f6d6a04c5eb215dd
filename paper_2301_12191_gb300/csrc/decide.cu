// decide.cu -- independent analysis, step 2: decode the per-CTU argmin keys
// of the full search, then SATD at the chosen vectors, rate-distortion cost,
// bottom-up quadtree split and leaf maps (one CTA per CTU, for every frame
// of a batch); the decisions at further QPs; the decisions with the spatial
// MV predictor in wavefront order; and the key initialisation kernel.
#include "common.cuh"

#include <algorithm>

namespace ladder_impl {
namespace {

__constant__ int c_lambda_q16[52] = {
#include "lambda_table.inc"
};

template <typename T, int CTU>
__global__ void __launch_bounds__(kThreads) k_decide(const __grid_constant__ DecideBatch b)
{
    dev::chain_entry();
    using C = dev::Ctu<CTU>;
    __shared__ dev::CtuState<CTU> st;
    const int ii = dev::item_of_cta(b.item, b.n);  // the batch item of this CTA
    const DecideItem &item = b.item[ii];
    const RungInfo &ri = b.rung[item.rung];
    const RungGeom &g = ri.g;
    const unsigned long long *keys = reinterpret_cast<const unsigned long long *>(array_at(item.block, ri.off.keys));
    const int tid = threadIdx.x;
    const int ctu_idx = blockIdx.x - item.cta_begin;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const int K = 2 * b.range + 1;

    for (int i = tid; i < C::NKEY; i += kThreads) {
        int d = 0;
        while (d < C::DMAX && i >= key_offset(d + 1)) ++d;
        const int li = i - key_offset(d), n = 1 << d, S = CTU >> d;
        const int fx = x0 / S + li % n, fy = y0 / S + li / n;
        uint8_t flags = 0;
        if (fx * S < g.W8 && fy * S < g.H8) {
            const bool inside = fx * S + S <= g.W8 && fy * S + S <= g.H8;
            flags = dev::kPresent | kRuleReachable | (inside ? kRuleEvaluated : 0) |
                    (d < C::DMAX ? kRuleCanSplit : 0);
        }
        st.flags[i] = flags;
        st.satd[i] = 0;
        // read the key and reset it to ~0 for the next search
        const long ki = static_cast<long>(ctu_idx) * C::NKEY + i;
        const bool kin = in_range(b.status, ki, static_cast<long>(g.ctu_cols) * g.ctu_rows * C::NKEY);
        unsigned long long *kp = const_cast<unsigned long long *>(keys) + (kin ? ki : 0);
        const unsigned long long key = __ldcg(kp);
        if (kin) *kp = ~0ull;
        if (flags & kRuleEvaluated) {
            const int rem = static_cast<int>(static_cast<uint32_t>(key & 0xffffffffu) % static_cast<uint32_t>(K * K));
            st.mvx[i] = static_cast<int16_t>(rem % K - b.range);
            st.mvy[i] = static_cast<int16_t>(rem / K - b.range);
            st.sad[i] = static_cast<int32_t>(key >> 32);
        } else {
            st.mvx[i] = INT16_MIN;
            st.mvy[i] = INT16_MIN;
            st.sad[i] = INT32_MAX;
        }
    }
    __syncthreads();
    dev::DecideIO io{item.cur, item.ref, item.pitch_bytes, &g, item.qp, b.satd_mode, c_lambda_q16,
                     decisions_at(item.block, ri.off), b.status};
    dev::ctu_decide<T, CTU>(st, io, x0, y0);
}

// Further-QP decisions (intra-resolution sharing, Sec. 4.2): CTU blockIdx.x
// of the rung at QP b.qp[blockIdx.y], from the resident vectors and SATDs.
template <int CTU>
__global__ void __launch_bounds__(kThreads) k_decide_qps(const __grid_constant__ QpBatch b)
{
    dev::chain_entry();
    using C = dev::Ctu<CTU>;
    __shared__ dev::CtuState<CTU> st;
    const RungGeom &g = b.g;
    const int ctu_idx = blockIdx.x;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const uint8_t *dep_flags = reinterpret_cast<const uint8_t *>(b.block + b.off.dep_flags) +
                               static_cast<long>(ctu_idx) * C::NKEY;
    for (int i = threadIdx.x; i < C::NKEY; i += kThreads) {
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
        if (flags & dev::kPresent) {
            const long gi = static_cast<long>(fy) * g.cols[d] + fx;
            st.mvx[i] = __ldcg(reinterpret_cast<const int16_t *>(b.block + b.off.mvx[d]) + gi);
            st.mvy[i] = __ldcg(reinterpret_cast<const int16_t *>(b.block + b.off.mvy[d]) + gi);
            st.satd[i] = __ldcg(reinterpret_cast<const int32_t *>(b.block + b.off.satd[d]) + gi);
        }
    }
    __syncthreads();
    dev::ctu_split<CTU>(st, c_lambda_q16[b.qp[blockIdx.y]], g, b.out[blockIdx.y], 0, x0, y0);
}

// ---- spatial MV predictor ---------------------------------------------------
// Reading for the wavefront CTU order of WPP (Sec. 2.2: a CTU starts once the
// CTU above and to its right is done): the predictor of a CU of size S at
// (x, y) is the component-wise median of the leaf vectors at A1 = (x-1,
// y+S-1), B1 = (x+S-1, y-1) and B0 = (x+S, y-1), as HEVC's spatial AMVP
// candidates.  A position counts as (0, 0) unless it lies inside the
// 8-aligned frame, outside the CU's own CTU (one motion estimation region,
// its CUs analysed in parallel) and in an earlier CTU of the wavefront: to
// the left in the same row, or in the row above at most one column right.
// Only the rate term changes (the search is by SAD, the SATD is at the
// found vector), so the kernel decides cost, split and leaf maps again from
// the resident vectors and SATDs: one CTA walks one CTU row left to right.
//
// The positions a CTU reads are the right column of its left neighbour
// (decided by the same CTA: kept in shared memory), the bottom row of the
// CTU above and the first bottom block of the CTU above-right.  Each CTU
// publishes its bottom-row leaf vectors as 64-bit words (generation << 32 |
// vector), one store each: a reader polls the words it needs until they
// carry this launch's generation, which also delivers the vector (no fence,
// no second read).  The generation is read from the block at the start and
// published by the last row to finish, so words of earlier launches (a
// replayed graph's included) never pass for this one.

constexpr int kMvpThreads = 128;

template <int CTU>
__global__ void __launch_bounds__(kMvpThreads, 12) k_decide_mvp(const __grid_constant__ MvpBatch b)
{
    using C = dev::Ctu<CTU>;
    constexpr int N8 = C::N8;
    __shared__ dev::CtuState<CTU> st;
    __shared__ int16_t s_pmx[C::NKEY], s_pmy[C::NKEY];
    __shared__ uint32_t s_left[N8];       // right column of the left CTU
    __shared__ uint32_t s_above[N8 + 1];  // bottom row of the CTU above, first bottom block of the one above-right
    __shared__ int s_stop;
    const MvpItem &it = b.item[dev::item_of_cta(b.item, b.n)];
    const RungInfo &ri = b.rung[it.rung];
    const RungGeom &g = ri.g;
    const DevDecisions res = decisions_at(it.block, ri.off);  // the resident vectors and SATDs
    const DevDecisions out = b.use_out ? b.out : res;           // where the decisions go
    const int nctu = g.ctu_cols * g.ctu_rows;
    unsigned long long *hand = reinterpret_cast<unsigned long long *>(it.block + ri.off.mvp_flag);  // [CTU][N8]
    unsigned *gen = reinterpret_cast<unsigned *>(hand + static_cast<long>(nctu) * N8), *rows_done = gen + 1;
    const uint8_t *dep_flags = reinterpret_cast<const uint8_t *>(it.block + ri.off.dep_flags);
    const int tid = threadIdx.x;
    const int cy = static_cast<int>(blockIdx.x) - it.cta_begin;
    const int lam = c_lambda_q16[it.qp];
    const unsigned target = __ldcg(gen) + 1u;  // published by the previous launch on this block
    // the generation a reader waits for: this launch's, unless a test asks
    // for one that no row publishes (every wait then runs out)
    const unsigned want = target + (b.lost_handoff ? 1u : 0u);
    // this thread's CU key (NKEY <= threads): its depth and place in the CTU
    static_assert(C::NKEY <= kMvpThreads, "one key per thread");
    const int ki = tid;
    int kd = 0;
    while (kd < C::DMAX && ki >= key_offset(kd + 1)) ++kd;
    const int kli = ki - key_offset(kd), kn = 1 << kd, kS = CTU >> kd;
    // resident state of key ki of CTU column cx, as loads into registers
    // (issued one CTU ahead: their latency hides behind the current CTU)
    uint8_t p_flags = 0;
    int16_t p_mvx = 0, p_mvy = 0;
    int32_t p_satd = 0;
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
        if (present) {
            const long gi = static_cast<long>(fy) * g.cols[kd] + fx;
            p_mvx = __ldcg(res.mvx[kd] + gi);
            p_mvy = __ldcg(res.mvy[kd] + gi);
            p_satd = __ldcg(res.satd[kd] + gi);
        }
    };
    auto stage = [&]() {
        if (ki >= C::NKEY) return;
        st.flags[ki] = p_flags;
        st.mvx[ki] = p_mvx;
        st.mvy[ki] = p_mvy;
        st.satd[ki] = p_satd;
    };
    if (tid == 0) s_stop = 0;
    fetch(0);
    stage();
    __syncthreads();
    for (int cx = 0; cx < g.ctu_cols; ++cx) {
        const int ctu_idx = cy * g.ctu_cols + cx;
        const int x0 = cx * CTU, y0 = cy * CTU;
        if (cx + 1 < g.ctu_cols) fetch(cx + 1);
        // the vectors this CTU reads from the row above (threads 0..N8)
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
                    // another row gave up (checked now and then: each check is a round trip)
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
        // predictors of the evaluated CUs (an evaluated CU lies inside the
        // 8-aligned frame, so A1 and B1 do whenever they are outside its CTU)
        if (ki < C::NKEY) {
            s_pmx[ki] = s_pmy[ki] = 0;
            if (st.flags[ki] & kRuleEvaluated) {
                const int lx = (kli % kn) * kS, ly = (kli / kn) * kS;  // CU position inside the CTU
                const uint32_t a1 = (lx == 0 && cx > 0) ? s_left[(ly + kS - 1) >> 3] : 0u;
                const bool top = ly == 0 && cy > 0;
                const uint32_t b1 = top ? s_above[(lx + kS - 1) >> 3] : 0u;
                uint32_t b0 = 0u;
                if (top && x0 + lx + kS < g.W8) b0 = lx + kS < CTU ? s_above[(lx + kS) >> 3] : s_above[N8];
                s_pmx[ki] = static_cast<int16_t>(dev::median3(dev::mv_x(a1), dev::mv_x(b1), dev::mv_x(b0)));
                s_pmy[ki] = static_cast<int16_t>(dev::median3(dev::mv_y(a1), dev::mv_y(b1), dev::mv_y(b0)));
            }
        }
        __syncthreads();
        dev::ctu_split<CTU>(st, lam, g, out, 0, x0, y0, false, s_pmx, s_pmy);
        __syncthreads();
        // publish the bottom row for the row below; keep the right column
        if (tid < N8) {
            if (cy + 1 < g.ctu_rows && x0 + 8 * tid < g.W8)
                dev::st_relaxed64(hand + static_cast<long>(ctu_idx) * N8 + tid,
                             (static_cast<unsigned long long>(target) << 32) | dev::leaf_mv<CTU>(st, tid, N8 - 1));
        } else if (tid < 2 * N8) {
            s_left[tid - N8] = dev::leaf_mv<CTU>(st, N8 - 1, tid - N8);
        }
        __syncthreads();
        if (cx + 1 < g.ctu_cols) stage();  // the next CTU's state
        __syncthreads();
    }
    // the last row to finish (decided or given up) publishes the generation
    if (tid == 0 && atomicAdd(rows_done, 1u) == static_cast<unsigned>(g.ctu_rows) - 1u) {
        *rows_done = 0;
        dev::st_release32(gen, target);
    }
}

__global__ void k_fill_keys(const __grid_constant__ FillBatch b)
{
    dev::chain_entry();
    for (int k = 0; k < b.n; ++k)
        for (long i = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x; i < b.item[k].n;
             i += static_cast<long>(gridDim.x) * blockDim.x)
            b.item[k].keys[i] = ~0ull;
}

template <typename T, int CTU>
cudaError_t decide_t(const DecideBatch &b, cudaStream_t s)
{
    return launch_chained(k_decide<T, CTU>, dim3(b.total_ctas), dim3(kThreads), 0, s, b);
}

}  // namespace

cudaError_t launch_decide(int bit_depth, int ctu, const DecideBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxItems || b.total_ctas <= 0) return cudaErrorInvalidValue;
    if (bit_depth == 8) {
        if (ctu == 64) return decide_t<uint8_t, 64>(b, s);
        if (ctu == 32) return decide_t<uint8_t, 32>(b, s);
        return decide_t<uint8_t, 16>(b, s);
    }
    if (ctu == 64) return decide_t<uint16_t, 64>(b, s);
    if (ctu == 32) return decide_t<uint16_t, 32>(b, s);
    return decide_t<uint16_t, 16>(b, s);
}

cudaError_t launch_decide_qps(int ctu, const QpBatch &b, cudaStream_t s)
{
    if (b.n_qps < 1 || b.n_qps > kMaxQps) return cudaErrorInvalidValue;
    const dim3 grid(b.g.ctu_cols * b.g.ctu_rows, b.n_qps);
    auto kern = ctu == 64 ? k_decide_qps<64> : ctu == 32 ? k_decide_qps<32> : k_decide_qps<16>;
    return launch_chained(kern, grid, dim3(kThreads), 0, s, b);
}

cudaError_t launch_decide_mvp(int ctu, const MvpBatch &b, int ctas, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxMvpItems || ctas < 1) return cudaErrorInvalidValue;
    auto kern = ctu == 64 ? k_decide_mvp<64> : ctu == 32 ? k_decide_mvp<32> : k_decide_mvp<16>;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every row resident: rows wait on the row above
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kMvpThreads);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, b);
}

int decide_mvp_capacity(int ctu, int sm_count)
{
    auto kern = ctu == 64 ? k_decide_mvp<64> : ctu == 32 ? k_decide_mvp<32> : k_decide_mvp<16>;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kMvpThreads, 0) != cudaSuccess) return 0;
    return n * sm_count;
}

cudaError_t launch_fill_keys(const FillBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxItems) return cudaErrorInvalidValue;
    long most = 0;
    for (int k = 0; k < b.n; ++k) most = std::max(most, b.item[k].n);
    const int blocks = static_cast<int>(std::max<long>(1, std::min<long>((most + kThreads - 1) / kThreads, 1024)));
    return launch_chained(k_fill_keys, dim3(blocks), dim3(kThreads), 0, s, b);
}

}  // namespace ladder_impl
