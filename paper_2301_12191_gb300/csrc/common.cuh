// common.cuh -- device helpers shared by the kernels of libladder.so:
// packed absdiff-accumulate, TMA / mbarrier wrappers with bounded waits,
// the integer rate term, and the CTU decision step (SATD at the chosen
// vectors, cost, bottom-up split, leaf maps).
#pragma once

#include "ladder_internal.h"

namespace ladder_impl {
namespace dev {

template <typename T> struct Traits;
template <> struct Traits<uint8_t> { static constexpr int SPW = 4; };   // samples per 32-bit word
template <> struct Traits<uint16_t> { static constexpr int SPW = 2; };

template <int CTU> struct Ctu {
    static constexpr int DMAX = CTU == 64 ? 3 : (CTU == 32 ? 2 : 1);
    static constexpr int NKEY = keys_per_ctu(DMAX);
    static constexpr int N8 = CTU / 8;
    static constexpr int NB8 = N8 * N8;
};

// d = c + sum of |a_i - b_i| over the packed samples of a and b.
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

// First statement of every kernel of this library (launched by
// launch_chained): wait until the previous kernel in the stream has
// completed and its writes are visible, then let the next kernel be
// scheduled.  Every CTA passes the wait before it can finish, so each kernel
// completes only after its predecessor, and at most one kernel waits behind
// a running one.  Data written by earlier kernels is read with L2 loads
// (__ldcg) or atomics, never through the non-coherent read-only path.
__device__ __forceinline__ void chain_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^22 polls (over a second with the
// back-off), so a lost completion cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 32) __nanosleep(256);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// Length of the signed Exp-Golomb code se(v).
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
__device__ __forceinline__ int ld_sample(const char *base, long pitch, int x, int y)
{
    return static_cast<int>(__ldg(reinterpret_cast<const T *>(base + static_cast<long>(y) * pitch) + x));
}

// Sample k of a packed word as the float 2^23 + sample (a byte permute
// into the bit pattern of 2^23): exact, and the difference of two such
// floats is the exact integer difference of the samples.
template <typename T>
__device__ __forceinline__ float sample_f(uint32_t w, int k)
{
    // selector: sample bytes into bytes 0 (and 1), zero, 0x4b (byte 7 of the pair)
    const uint32_t sel = sizeof(T) == 1 ? 0x7540u + static_cast<uint32_t>(k)
                                        : 0x7400u + static_cast<uint32_t>(2 * k) + (static_cast<uint32_t>(2 * k + 1) << 4);
    return __int_as_float(static_cast<int>(__byte_perm(w, 0x4b000000u, sel)));
}

__device__ __forceinline__ int satd8_transform(float (&v)[64], int mode);

// SATD of the 8x8 block at (px, py) against the reference displaced by
// (mvx, mvy), by one thread.  Samples are read with clamping (current:
// replicate to the 8-aligned size; reference: frame edge).  The residual
// and every butterfly sum are integers below 2^24 in magnitude, so they are
// exact in fp32: the transform runs as fp32 adds on the FMA pipes.
//   mode 0: 8x8 Hadamard T = H8 D H8^T, (sum |T|) >> 2
//   mode 1: two 4x4 Hadamards per 8x4 half, (sum of both) >> 1, halves added
template <typename T>
__device__ __forceinline__ int satd8_thread(const void *cur, const void *ref, long pitch, int W, int H, int px, int py,
                                            int mvx, int mvy, int mode, int *status = nullptr)
{
    const char *cb = static_cast<const char *>(cur);
    const char *rb = static_cast<const char *>(ref);
    constexpr int SPW = Traits<T>::SPW, BITS = 32 / SPW, WPR = 8 / SPW;
    const int rx0 = px + mvx;
    const bool cur_fast = px + 8 <= W;
    const bool ref_fast = rx0 >= 0 && (rx0 / SPW + WPR + 1) * SPW <= W;
    const int sh = (rx0 & (SPW - 1)) * BITS;
    // debug builds: the rows are clamped into [0, H); the fast paths' row
    // spans (8 current samples from px, WPR + 1 reference words from
    // rx0 / SPW) must end inside the row's pitch
    if ((cur_fast && !in_range(status, static_cast<long>(px + 8) * sizeof(T) - 1, pitch)) ||
        (ref_fast && !in_range(status, static_cast<long>(rx0 / SPW + WPR + 1) * 4 - 1, pitch)) ||
        !in_range(status, px, W))
        return 0;
    float v[64];
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const int cy = min(py + y, H - 1);
        const int ry = min(max(py + y + mvy, 0), H - 1);
        uint32_t cw[WPR], rw[WPR];
        if (cur_fast) {  // one aligned vector load
            const char *row = cb + static_cast<long>(cy) * pitch + static_cast<long>(px) * sizeof(T);
            if constexpr (WPR == 2) {
                const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row));
                cw[0] = q.x;
                cw[1] = q.y;
            } else {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(row));
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
                    w |= static_cast<uint32_t>(ld_sample<T>(cb, pitch, min(px + m * SPW + e, W - 1), cy)) << (e * BITS);
                cw[m] = w;
            }
        }
        if (ref_fast) {  // aligned words + one funnel shift
            const uint32_t *rp = reinterpret_cast<const uint32_t *>(rb + static_cast<long>(ry) * pitch) + rx0 / SPW;
            uint32_t raw[WPR + 1];
#pragma unroll
            for (int m = 0; m <= WPR; ++m) raw[m] = __ldg(rp + m);
#pragma unroll
            for (int m = 0; m < WPR; ++m) rw[m] = __funnelshift_r(raw[m], raw[m + 1], sh);
        } else {
#pragma unroll
            for (int m = 0; m < WPR; ++m) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < SPW; ++e)
                    w |= static_cast<uint32_t>(ld_sample<T>(rb, pitch, min(max(rx0 + m * SPW + e, 0), W - 1), ry))
                         << (e * BITS);
                rw[m] = w;
            }
        }
#pragma unroll
        for (int x = 0; x < 8; ++x) v[8 * y + x] = sample_f<T>(cw[x / SPW], x % SPW) - sample_f<T>(rw[x / SPW], x % SPW);
    }
    return satd8_transform(v, mode);
}

// The SATD of the 8x8 block at (px, py) by a pair of lanes (lane ^ 1, both
// in `mask`): this lane loads and transforms rows 4h .. 4h + 3 (h = lane &
// 1), so a lane keeps 32 values and issues half the loads of satd8_thread,
// all of them before its first transform.  The butterflies and the exact
// sums are those of satd8_thread; mode 0's vertical stage that pairs rows y
// and y + 4 exchanges values between the two lanes.  Both lanes return the
// block's SATD.
template <typename T>
__device__ __forceinline__ int satd8_pair(const void *cur, const void *ref, long pitch, int W, int H, int px, int py,
                                          int mvx, int mvy, int mode, unsigned mask, int *status = nullptr)
{
    const char *cb = static_cast<const char *>(cur);
    const char *rb = static_cast<const char *>(ref);
    constexpr int SPW = Traits<T>::SPW, BITS = 32 / SPW, WPR = 8 / SPW;
    const int h = threadIdx.x & 1;
    int rx0 = px + mvx;
    bool cur_fast = px + 8 <= W;
    bool ref_fast = rx0 >= 0 && (rx0 / SPW + WPR + 1) * SPW <= W;
    // debug builds: as satd8_thread, but a failed check only zeroes the
    // result (both lanes still reach the exchange)
    const bool ok = !((cur_fast && !in_range(status, static_cast<long>(px + 8) * sizeof(T) - 1, pitch)) ||
                      (ref_fast && !in_range(status, static_cast<long>(rx0 / SPW + WPR + 1) * 4 - 1, pitch)) ||
                      !in_range(status, px, W));
    if (!ok) {  // read the frame's first block instead
        px = 0;
        rx0 = 0;
        cur_fast = ref_fast = false;
    }
    const int sh = (rx0 & (SPW - 1)) * BITS;
    float v[32];
    uint32_t cw[4][WPR], rw[4][WPR];
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int cy = min(py + 4 * h + y, H - 1);
        const int ry = min(max(py + 4 * h + y + mvy, 0), H - 1);
        if (cur_fast) {
            const char *row = cb + static_cast<long>(cy) * pitch + static_cast<long>(px) * sizeof(T);
            if constexpr (WPR == 2) {
                const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row));
                cw[y][0] = q.x;
                cw[y][1] = q.y;
            } else {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(row));
                cw[y][0] = q.x;
                cw[y][1] = q.y;
                cw[y][2] = q.z;
                cw[y][3] = q.w;
            }
        } else {
#pragma unroll
            for (int m = 0; m < WPR; ++m) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < SPW; ++e)
                    w |= static_cast<uint32_t>(ld_sample<T>(cb, pitch, min(px + m * SPW + e, W - 1), cy)) << (e * BITS);
                cw[y][m] = w;
            }
        }
        if (ref_fast) {
            const uint32_t *rp = reinterpret_cast<const uint32_t *>(rb + static_cast<long>(ry) * pitch) + rx0 / SPW;
            uint32_t raw[WPR + 1];
#pragma unroll
            for (int m = 0; m <= WPR; ++m) raw[m] = __ldg(rp + m);
#pragma unroll
            for (int m = 0; m < WPR; ++m) rw[y][m] = __funnelshift_r(raw[m], raw[m + 1], sh);
        } else {
#pragma unroll
            for (int m = 0; m < WPR; ++m) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < SPW; ++e)
                    w |= static_cast<uint32_t>(ld_sample<T>(rb, pitch, min(max(rx0 + m * SPW + e, 0), W - 1), ry))
                         << (e * BITS);
                rw[y][m] = w;
            }
        }
    }
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 8; ++x)
            v[8 * y + x] = sample_f<T>(cw[y][x / SPW], x % SPW) - sample_f<T>(rw[y][x / SPW], x % SPW);
    auto bfly = [&](int i, int j) {
        const float a = v[i], b = v[j];
        v[i] = a + b;
        v[j] = a - b;
    };
    const int top = mode == 0 ? 4 : 2;  // horizontal stages: the row, or each 4-wide half
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int s = 4; s >= 1; s >>= 1)
            if (s <= top) {
#pragma unroll
                for (int x = 0; x < 8; ++x)
                    if (!(x & s)) bfly(8 * y + x, 8 * y + x + s);
            }
    if (mode == 0) {  // rows y and y + 4: lane 0 keeps the sums, lane 1 the differences
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float o = __shfl_xor_sync(mask, v[k], 1);
            v[k] = h ? o - v[k] : v[k] + o;
        }
    }
#pragma unroll
    for (int x = 0; x < 8; ++x)  // the remaining vertical stages, inside this lane's 4 rows
#pragma unroll
        for (int s = 2; s >= 1; s >>= 1)
#pragma unroll
            for (int y = 0; y < 4; ++y)
                if (!(y & s)) bfly(8 * y + x, 8 * (y + s) + x);
    float part[4];
#pragma unroll
    for (int y = 0; y < 4; ++y)
        part[y] = (fabsf(v[8 * y]) + fabsf(v[8 * y + 1])) + (fabsf(v[8 * y + 2]) + fabsf(v[8 * y + 3])) +
                  ((fabsf(v[8 * y + 4]) + fabsf(v[8 * y + 5])) + (fabsf(v[8 * y + 6]) + fabsf(v[8 * y + 7])));
    const float half_sum = (part[0] + part[1]) + (part[2] + part[3]);  // exact: integers below 2^24
    int r;
    if (mode == 0) {
        r = __float2int_rn(half_sum + __shfl_xor_sync(mask, half_sum, 1)) >> 2;
    } else {
        const int mine = __float2int_rn(half_sum) >> 1;  // this 8x4 half
        r = mine + __shfl_xor_sync(mask, mine, 1);
    }
    return ok ? r : 0;
}

// The Hadamard part of the SATD of an 8x8 residual held in fp32 (integers
// below 2^24 in magnitude, so every add is exact).
//   mode 0: 8x8 Hadamard T = H8 D H8^T, (sum |T|) >> 2
//   mode 1: two 4x4 Hadamards per 8x4 half, (sum of both) >> 1, halves added
__device__ __forceinline__ int satd8_transform(float (&v)[64], int mode)
{
    auto bfly = [&](int i, int j) {
        const float a = v[i], b = v[j];
        v[i] = a + b;
        v[j] = a - b;
    };
    if (mode == 0) {
#pragma unroll
        for (int y = 0; y < 8; ++y)  // rows
#pragma unroll
            for (int s = 4; s >= 1; s >>= 1)
#pragma unroll
                for (int x = 0; x < 8; ++x)
                    if (!(x & s)) bfly(8 * y + x, 8 * y + x + s);
#pragma unroll
        for (int x = 0; x < 8; ++x)  // columns
#pragma unroll
            for (int s = 4; s >= 1; s >>= 1)
#pragma unroll
                for (int y = 0; y < 8; ++y)
                    if (!(y & s)) bfly(8 * y + x, 8 * (y + s) + x);
        // exact sums (integers below 2^24): any order, here a short tree
        float part[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            part[y] = (fabsf(v[8 * y]) + fabsf(v[8 * y + 1])) + (fabsf(v[8 * y + 2]) + fabsf(v[8 * y + 3])) +
                      ((fabsf(v[8 * y + 4]) + fabsf(v[8 * y + 5])) + (fabsf(v[8 * y + 6]) + fabsf(v[8 * y + 7])));
        }
        const float sum = ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
        return __float2int_rn(sum) >> 2;
    }
#pragma unroll
    for (int y = 0; y < 8; ++y)  // rows of each 4-wide half
#pragma unroll
        for (int s = 2; s >= 1; s >>= 1)
#pragma unroll
            for (int x = 0; x < 8; ++x)
                if (!(x & s)) bfly(8 * y + x, 8 * y + x + s);
#pragma unroll
    for (int x = 0; x < 8; ++x)  // columns of each 4-row half
#pragma unroll
        for (int s = 2; s >= 1; s >>= 1)
#pragma unroll
            for (int y = 0; y < 8; ++y)
                if (!(y & s)) bfly(8 * y + x, 8 * (y + s) + x);
    float part[8];  // rows; rows 0-3 and 4-7 are the two 8x4 halves
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        part[y] = (fabsf(v[8 * y]) + fabsf(v[8 * y + 1])) + (fabsf(v[8 * y + 2]) + fabsf(v[8 * y + 3])) +
                  ((fabsf(v[8 * y + 4]) + fabsf(v[8 * y + 5])) + (fabsf(v[8 * y + 6]) + fabsf(v[8 * y + 7])));
    }
    const float top = (part[0] + part[1]) + (part[2] + part[3]), bottom = (part[4] + part[5]) + (part[6] + part[7]);
    return (__float2int_rn(top) >> 1) + (__float2int_rn(bottom) >> 1);
}

// Index of the batch item whose CTA range holds this CTA (items in order of
// cta_begin): a binary search over the item table in parameter space.
template <typename Item>
__device__ __forceinline__ int item_of_cta(const Item *item, int n)
{
    int lo = 0, hi = n - 1;
    const int c = static_cast<int>(blockIdx.x);
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (c >= item[mid].cta_begin) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr uint8_t kPresent = 8;  // CU lies (at least partly) inside the 8-aligned frame

// Per-CTU state of the decision step, in shared memory.
template <int CTU>
struct CtuState {
    int32_t satd[Ctu<CTU>::NKEY], sad[Ctu<CTU>::NKEY], best[Ctu<CTU>::NKEY];
    int16_t mvx[Ctu<CTU>::NKEY], mvy[Ctu<CTU>::NKEY];
    uint8_t flags[Ctu<CTU>::NKEY], split[Ctu<CTU>::NKEY];
    uint16_t pairs[(Ctu<CTU>::DMAX + 1) * Ctu<CTU>::NB8];  // distinct (8x8 block, vector): block | depths << 8
    int npairs;
};

template <typename O>
struct DecideIOT {
    const void *cur, *ref;
    long pitch_bytes;
    const RungGeom *g;
    int qp, satd_mode;
    const int *lambda_q16;  // 52 entries
    O out;                  // DevDecisions or OffDecisions
    int *status;            // debug builds record failed bounds checks here (may be null)
};
using DecideIO = DecideIOT<DevDecisions>;

// Index of CU (d, local raster li) in the per-CTU key layout.
__device__ __forceinline__ int key_index(int d, int li) { return key_offset(d) + li; }

// Key of the depth-d CU that covers 8x8 block (bx, by) of a CTU: the block
// coordinates shifted by log2 of the CU's size in blocks (no division).
template <int CTU>
__device__ __forceinline__ int key_of_block(int d, int bx, int by)
{
    constexpr int kLog2N8 = CTU == 64 ? 3 : (CTU == 32 ? 2 : 1);
    const int sh = kLog2N8 - d;
    return key_index(d, ((by >> sh) << d) + (bx >> sh));
}

// ---- wavefront hand-off (the spatial MV predictor's CTU order) ----------------
// Words a CTU row publishes for the row below (generation << 32 | packed
// vector), relaxed 64-bit loads and stores, and the median of the three
// predictor candidates.
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int median3(int a, int b, int c) { return max(min(a, b), min(max(a, b), c)); }

__device__ __forceinline__ uint32_t pack_mv(int mvx, int mvy)
{
    return static_cast<uint32_t>(static_cast<uint16_t>(mvx)) | (static_cast<uint32_t>(static_cast<uint16_t>(mvy)) << 16);
}
__device__ __forceinline__ int mv_x(uint32_t v) { return static_cast<int16_t>(v & 0xffffu); }
__device__ __forceinline__ int mv_y(uint32_t v) { return static_cast<int16_t>(v >> 16); }

// Leaf vector of 8x8 block (bx, by) of the CTU in st (split flags decided).
template <int CTU>
__device__ __forceinline__ uint32_t leaf_mv(const CtuState<CTU> &st, int bx, int by)
{
    using C = Ctu<CTU>;
    int d = 0, i = 0;
    for (;;) {
        i = key_of_block<CTU>(d, bx, by);
        if (d == C::DMAX || !st.split[i]) break;
        ++d;
    }
    return pack_mv(st.mvx[i], st.mvy[i]);
}

// What ctu_split writes besides cost, best, split and the leaf maps.
enum : int {
    kSplitWriteVectors = 1,  // mvx, mvy and SATD per CU
    kSplitWriteAll = 3,      // also SAD and the evaluated flags
};

// Cost, bottom-up split and leaf maps of one CTU at lambda lam (Q16), from
// st: flags, vectors and, for evaluated CUs, SADs and SATDs.  All threads
// of the CTA take part.  Writes cost, best and split per CU, the leaf maps
// and the fields `write` names.  `qpel`: the vectors are in quarter-pel
// units (the rate term takes them as they are), else in integer samples.
// pmx / pmy: per-CU predictors (shared memory, the vectors' units), or
// null for the predictor (0, 0).
//   cost   -- J = SATD + ((lambdaQ16[qp] * bits + 2^15) >> 16), bits = se()
//             lengths of the quarter-pel components of vector - predictor
//   split  -- Sec. 2.1: split iff it may and (it is not a leaf candidate or
//             the children's best sum is strictly lower), or it must
template <int CTU, typename O>
__device__ void ctu_split(CtuState<CTU> &st, int lam, const RungGeom &g, const O &out, int write, int x0,
                          int y0, bool qpel = false, const int16_t *pmx = nullptr, const int16_t *pmy = nullptr,
                          int *status = nullptr)
{
    using C = Ctu<CTU>;
    const int tid = threadIdx.x, nthr = blockDim.x;
#pragma unroll
    for (int d = C::DMAX; d >= 0; --d) {  // unrolled: n and S are constants, the index math shifts
        const int n = 1 << d, S = CTU >> d;
        for (int li = tid; li < n * n; li += nthr) {
            const int i = key_index(d, li);
            const uint8_t f = st.flags[i];
            if (!(f & kPresent)) continue;
            const bool ev = f & kRuleEvaluated;
            int32_t J = INT32_MAX;
            if (ev) {
                const int u = qpel ? 1 : 4;
                const int px = pmx ? pmx[i] : 0, py = pmy ? pmy[i] : 0;
                const long long bits = se_bits(u * (st.mvx[i] - px)) + se_bits(u * (st.mvy[i] - py));
                J = st.satd[i] + static_cast<int32_t>((static_cast<long long>(lam) * bits + 32768) >> 16);
            }
            int32_t best = J;
            uint8_t split = 0;
            if (d < C::DMAX) {
                const bool can_split = f & kRuleCanSplit;
                int32_t children = 0;
                if (can_split) {
                    const int cxl = li % n, cyl = li / n;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ci = key_index(d + 1, (2 * cyl + (q >> 1)) * (2 * n) + 2 * cxl + (q & 1));
                        if (st.flags[ci] & kPresent) children += st.best[ci];
                    }
                }
                split = can_split && (!ev || children < J);
                best = !(f & kRuleReachable) ? INT32_MAX : (split ? children : J);
            }
            st.best[i] = best;
            st.split[i] = split;
            const long gi = static_cast<long>(y0 / S + li / n) * g.cols[d] + x0 / S + li % n;
            if (!in_range(status, gi, static_cast<long>(g.cols[d]) * g.rows[d])) continue;
            if (write & kSplitWriteVectors) {
                out.at_mvx(d)[gi] = st.mvx[i];
                out.at_mvy(d)[gi] = st.mvy[i];
                out.at_satd(d)[gi] = ev ? st.satd[i] : INT32_MAX;
            }
            if ((write & kSplitWriteAll) == kSplitWriteAll) {
                out.at_sad(d)[gi] = st.sad[i];
                out.at_evaluated(d)[gi] = ev ? 1 : 0;
            }
            out.at_cost(d)[gi] = J;
            out.at_best(d)[gi] = best;
            out.at_split(d)[gi] = split;
        }
        __syncthreads();
    }

    for (int b = tid; b < C::NB8; b += nthr) {
        const int bx = b % C::N8, by = b / C::N8;
        const int px = x0 + 8 * bx, py = y0 + 8 * by;
        if (px >= g.W8 || py >= g.H8) continue;
        int d = 0, i = 0;
        for (;;) {
            i = key_of_block<CTU>(d, bx, by);
            if (d == C::DMAX || !st.split[i]) break;
            ++d;
        }
        const long li = static_cast<long>(py / 8) * g.cols8 + px / 8;
        if (!in_range(status, li, static_cast<long>(g.cols8) * g.rows8)) continue;
        out.at_leaf_depth()[li] = static_cast<uint8_t>(d);
        out.at_leaf_mvx()[li] = st.mvx[i];
        out.at_leaf_mvy()[li] = st.mvy[i];
    }
}

// The decision step for one CTU, given flags / vectors / SADs in `st`
// (satd[] must be zero): SATD at the chosen vectors, then ctu_split.  All
// threads of the CTA take part.
//   SATD   -- Sec. 5.4.1 SATD equation; Sec. 5.4.2 satd8 / satd_8x4 listings
template <typename T, int CTU, typename O>
__device__ void ctu_decide(CtuState<CTU> &st, const DecideIOT<O> &io, int x0, int y0)
{
    using C = Ctu<CTU>;
    const RungGeom &g = *io.g;
    const int tid = threadIdx.x, nthr = blockDim.x;

    // SATD.  Every evaluated CU covering an 8x8 block needs that block's
    // SATD at the CU's vector; a CU and its sub-CUs often keep the same
    // vector, so the list holds one entry per distinct (block, vector):
    // block | (depths sharing the vector) << 8.  SATD sums are exact, so the
    // order of the additions does not matter.
    if (tid == 0) st.npairs = 0;
    __syncthreads();
    for (int b = tid; b < C::NB8; b += nthr) {
        const int bx = b % C::N8, by = b / C::N8;
        int ci[C::DMAX + 1];
        unsigned left = 0;
#pragma unroll
        for (int d = 0; d <= C::DMAX; ++d) {
            ci[d] = key_of_block<CTU>(d, bx, by);
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
            const int slot = atomicAdd(&st.npairs, 1);
            if (in_range(io.status, slot, (C::DMAX + 1) * C::NB8)) st.pairs[slot] = static_cast<uint16_t>(b | (mask << 8));
        }
    }
    __syncthreads();
    // two lanes per entry (satd8_pair): every thread runs the same number of
    // rounds, so the pair mask is taken with the whole warp present
    const int nwork = 2 * min(st.npairs, (C::DMAX + 1) * C::NB8);
    const int rounds = (nwork + nthr - 1) / nthr;
    for (int it = 0; it < rounds; ++it) {
        const int w = tid + it * nthr;
        const unsigned mask = __ballot_sync(0xffffffffu, w < nwork);  // whole pairs: nwork and nthr are even
        if (w < nwork) {
            const unsigned ent = st.pairs[w >> 1];
            const int b = ent & 0xff, bx = b % C::N8, by = b / C::N8;
            const int i0 = key_of_block<CTU>(__ffs(ent >> 8) - 1, bx, by);
            const int v = satd8_pair<T>(io.cur, io.ref, io.pitch_bytes, g.W, g.H, x0 + 8 * bx, y0 + 8 * by,
                                        st.mvx[i0], st.mvy[i0], io.satd_mode, mask, io.status);
            if (!(w & 1)) {
#pragma unroll
                for (int d = 0; d <= C::DMAX; ++d) {
                    if (!((ent >> (8 + d)) & 1u)) continue;
                    atomicAdd(&st.satd[key_of_block<CTU>(d, bx, by)], v);
                }
            }
        }
    }
    __syncthreads();

    ctu_split<CTU>(st, io.lambda_q16[io.qp], *io.g, io.out, kSplitWriteAll, x0, y0, false, nullptr, nullptr, io.status);
}

// ---- dependent-mode constraint derivation --------------------------------
// Sec. 4.3 / 6.3 and App. A.1-A.2: a dependent CU maps its centre to the
// reference rung, takes the co-located reference leaf's depth and vector,
// scales the vector by the resolution ratio (round half away from zero,
// clamped to +-256) as its search centre, and bounds its own depth around
// Deq, the deepest depth whose CU still covers the projected reference leaf.
struct Rule {
    int cx, cy;
    bool allowed_leaf, allowed_split;
};

__device__ __forceinline__ int scale_component(int v, int to, int from, const FastDiv &div_2from)
{
    // |v| <= 32768 and sizes <= 8192: 2|v|*to + from < 2^31
    const unsigned av = static_cast<unsigned>(v < 0 ? -v : v);
    const int s = static_cast<int>(fast_div(2u * av * static_cast<unsigned>(to) + static_cast<unsigned>(from), div_2from));
    const int r = v < 0 ? -s : s;
    return min(max(r, -256), 256);
}

__device__ __forceinline__ Rule derive_rule(const RungGeom &g, const DepRefs &rf, int d, int x0, int y0)
{
    // sizes are <= 8192, so the products below stay inside 32 bits
    const int S = g.ctu >> d;
    const int xm = min(static_cast<int>(fast_div(static_cast<unsigned>((2 * x0 + S) * rf.Wr), g.div_2w)), rf.Wr - 1);
    const int ym = min(static_cast<int>(fast_div(static_cast<unsigned>((2 * y0 + S) * rf.Hr), g.div_2h)), rf.Hr - 1);
    int li = (ym >> 3) * rf.cols8_r + (xm >> 3);
    if (!in_range(rf.status, li, rf.n8_r)) li = 0;
    const int depth_r = __ldcg(rf.leaf_depth + li);
    Rule r;
    if (rf.use_ref_mv) {
        r.cx = scale_component(__ldcg(rf.leaf_mvx + li), g.W, rf.Wr, rf.div_2wr);
        r.cy = scale_component(__ldcg(rf.leaf_mvy + li), g.H, rf.Hr, rf.div_2hr);
    } else {
        r.cx = r.cy = 0;
    }
    const int proj = (g.ctu >> depth_r) * g.W;
    int deq = 0;
    for (int dd = 0; dd <= g.dmax; ++dd)
        if ((g.ctu >> dd) * rf.Wr >= proj) deq = dd;
    r.allowed_split = d < g.dmax && d < deq + rf.depth_hi;
    r.allowed_leaf = (deq + rf.depth_lo <= d && d <= deq + rf.depth_hi) || d == g.dmax || !r.allowed_split;
    return r;
}

}  // namespace dev
}  // namespace ladder_impl
