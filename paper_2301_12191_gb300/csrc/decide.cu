// decide.cu -- independent analysis, step 2: decode the per-CTU argmin keys
// of the full search, then SATD at the chosen vectors, rate-distortion cost,
// bottom-up quadtree split and leaf maps (one CTA per CTU, for every frame
// of a batch); and the key initialisation kernel.
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

cudaError_t launch_fill_keys(const FillBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kMaxItems) return cudaErrorInvalidValue;
    long most = 0;
    for (int k = 0; k < b.n; ++k) most = std::max(most, b.item[k].n);
    const int blocks = static_cast<int>(std::max<long>(1, std::min<long>((most + kThreads - 1) / kThreads, 1024)));
    return launch_chained(k_fill_keys, dim3(blocks), dim3(kThreads), 0, s, b);
}

}  // namespace ladder_impl
