// decide.cu -- independent analysis, step 2: decode the per-CTU argmin keys
// of the full search, then SATD at the chosen vectors, rate-distortion cost,
// bottom-up quadtree split and leaf maps (one CTA per CTU); and the key
// initialisation kernel.
#include "common.cuh"

#include <algorithm>

namespace ladder_impl {
namespace {

__constant__ int c_lambda_q16[52] = {
#include "lambda_table.inc"
};

template <typename T, int CTU>
__global__ void __launch_bounds__(kThreads) k_decide(const DecideArgs a)
{
    using C = dev::Ctu<CTU>;
    __shared__ dev::CtuState<CTU> st;
    const RungGeom &g = a.g;
    const int tid = threadIdx.x;
    const int ctu_idx = blockIdx.x;
    const int x0 = (ctu_idx % g.ctu_cols) * CTU, y0 = (ctu_idx / g.ctu_cols) * CTU;
    const int K = 2 * a.range + 1;

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
        if (flags & kRuleEvaluated) {
            const unsigned long long key = a.keys[static_cast<long>(ctu_idx) * C::NKEY + i];
            const int rem = static_cast<int>(static_cast<uint32_t>(key & 0xffffffffu) % static_cast<uint32_t>(K * K));
            st.mvx[i] = static_cast<int16_t>(rem % K - a.range);
            st.mvy[i] = static_cast<int16_t>(rem / K - a.range);
            st.sad[i] = static_cast<int32_t>(key >> 32);
        } else {
            st.mvx[i] = INT16_MIN;
            st.mvy[i] = INT16_MIN;
            st.sad[i] = INT32_MAX;
        }
    }
    __syncthreads();
    dev::DecideIO io{a.cur, a.ref, a.pitch_bytes, &a.g, a.qp, a.satd_mode, c_lambda_q16, a.out};
    dev::ctu_decide<T, CTU>(st, io, x0, y0);
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

cudaError_t launch_fill_keys(unsigned long long *keys, long n, cudaStream_t s)
{
    const int blocks = static_cast<int>(std::min<long>((n + kThreads - 1) / kThreads, 1024));
    k_fill_keys<<<blocks > 0 ? blocks : 1, kThreads, 0, s>>>(keys, n);
    return cudaGetLastError();
}

}  // namespace ladder_impl
