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
    const unsigned long long *keys = reinterpret_cast<const unsigned long long *>(item.block + ri.off.keys);
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
        unsigned long long *kp = const_cast<unsigned long long *>(keys) + static_cast<long>(ctu_idx) * C::NKEY + i;
        const unsigned long long key = __ldcg(kp);
        *kp = ~0ull;
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
                     decisions_at(item.block, ri.off)};
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
// the resident vectors and SATDs: one CTA walks one CTU row left to right,
// each CTU waiting for the row above to have finished the CTU above-right.
// Every launch decides a new generation of the block (read from the block
// at the start, published by the last row to finish), and a CTU's flag holds
// the generation that decided it: flags of earlier launches, a replayed
// graph's included, never pass for this one.

constexpr int kMvpThreads = 128;
constexpr int kMvpSpin = 1 << 22;  // polls (about 0.2 us each) before a wait gives up

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int median3(int a, int b, int c) { return max(min(a, b), min(max(a, b), c)); }

template <int CTU>
__global__ void __launch_bounds__(kMvpThreads) k_decide_mvp(const __grid_constant__ MvpBatch b)
{
    using C = dev::Ctu<CTU>;
    constexpr int kLog2Ctu = CTU == 64 ? 6 : (CTU == 32 ? 5 : 4);
    __shared__ dev::CtuState<CTU> st;
    __shared__ int16_t s_pmx[C::NKEY], s_pmy[C::NKEY];
    __shared__ int s_stop;
    const MvpItem &it = b.item[dev::item_of_cta(b.item, b.n)];
    const RungInfo &ri = b.rung[it.rung];
    const RungGeom &g = ri.g;
    const DevDecisions out = decisions_at(it.block, ri.off);
    unsigned *done = reinterpret_cast<unsigned *>(it.block + ri.off.mvp_flag);
    unsigned *gen = done + g.ctu_cols * g.ctu_rows, *rows_done = gen + 1;
    const uint8_t *dep_flags = reinterpret_cast<const uint8_t *>(it.block + ri.off.dep_flags);
    const int tid = threadIdx.x;
    const int cy = static_cast<int>(blockIdx.x) - it.cta_begin;
    const int lam = c_lambda_q16[it.qp];
    const unsigned target = __ldcg(gen) + 1u;  // published by the previous launch on this block
    if (tid == 0) s_stop = 0;
    for (int cx = 0; cx < g.ctu_cols; ++cx) {
        const int ctu_idx = cy * g.ctu_cols + cx;
        const int x0 = cx * CTU, y0 = cy * CTU;
        // wait for the row above to have decided the CTU above-right (the
        // rest of this CTU's neighbours are before it in one of the rows)
        if (tid == 0 && cy > 0) {
            const unsigned *f = done + (cy - 1) * g.ctu_cols + min(cx + 1, g.ctu_cols - 1);
            int ok = 0;
            for (int n = 0; n < kMvpSpin; ++n) {
                if (ld_acquire(f) == target) {
                    ok = 1;
                    break;
                }
                if (*reinterpret_cast<volatile int *>(b.status) != kStatusOk) break;  // another row gave up
                __nanosleep(128);
            }
            if (!ok) {
                atomicCAS(b.status, kStatusOk, kStatusTimeout);
                s_stop = 1;
            }
        }
        __syncthreads();
        if (s_stop) break;
        for (int i = tid; i < C::NKEY; i += kMvpThreads) {
            int d = 0;
            while (d < C::DMAX && i >= key_offset(d + 1)) ++d;
            const int li = i - key_offset(d), n = 1 << d, S = CTU >> d;
            const int fx = (x0 >> (kLog2Ctu - d)) + li % n, fy = (y0 >> (kLog2Ctu - d)) + li / n;
            const bool present = fx * S < g.W8 && fy * S < g.H8;
            uint8_t flags = 0;
            if (it.dependent) {
                flags = __ldcg(dep_flags + static_cast<long>(ctu_idx) * C::NKEY + i);
            } else if (present) {
                const bool inside = fx * S + S <= g.W8 && fy * S + S <= g.H8;
                flags = dev::kPresent | kRuleReachable | (inside ? kRuleEvaluated : 0) |
                        (d < C::DMAX ? kRuleCanSplit : 0);
            }
            st.flags[i] = flags;
            s_pmx[i] = s_pmy[i] = 0;
            if (flags & dev::kPresent) {
                const long gi = static_cast<long>(fy) * g.cols[d] + fx;
                st.mvx[i] = __ldcg(out.mvx[d] + gi);
                st.mvy[i] = __ldcg(out.mvy[d] + gi);
                st.satd[i] = __ldcg(out.satd[d] + gi);
            }
            if (flags & kRuleEvaluated) {
                const int x = fx * S, y = fy * S;
                const int px[3] = {x - 1, x + S - 1, x + S}, py[3] = {y + S - 1, y - 1, y - 1};
                int vx[3], vy[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int qx = px[k] >> kLog2Ctu, qy = py[k] >> kLog2Ctu;  // CTU of the position
                    const bool in_frame = px[k] >= 0 && py[k] >= 0 && px[k] < g.W8 && py[k] < g.H8;
                    const bool before = (qy == cy && qx < cx) || (qy == cy - 1 && qx <= cx + 1);
                    vx[k] = vy[k] = 0;
                    if (in_frame && before) {
                        const long l8 = static_cast<long>(py[k] >> 3) * g.cols8 + (px[k] >> 3);
                        vx[k] = __ldcg(out.leaf_mvx + l8);
                        vy[k] = __ldcg(out.leaf_mvy + l8);
                    }
                }
                s_pmx[i] = static_cast<int16_t>(median3(vx[0], vx[1], vx[2]));
                s_pmy[i] = static_cast<int16_t>(median3(vy[0], vy[1], vy[2]));
            }
        }
        __syncthreads();
        dev::ctu_split<CTU>(st, lam, g, out, 0, x0, y0, false, s_pmx, s_pmy);
        __threadfence();  // this CTU's decisions, before its flag
        __syncthreads();
        if (tid == 0) st_release(done + ctu_idx, target);
    }
    // the last row to finish (decided or given up) publishes the generation
    if (tid == 0 && atomicAdd(rows_done, 1u) == static_cast<unsigned>(g.ctu_rows) - 1u) {
        *rows_done = 0;
        st_release(gen, target);
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
