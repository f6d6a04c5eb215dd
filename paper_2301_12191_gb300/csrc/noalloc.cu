// noalloc.cu -- independent analysis of one frame pair that allocates no
// memory at all.
//
// Who needs it: code that is not allowed to call cudaMalloc, e.g. an encoder
// plugin hosted by an application that owns every device allocation through
// its own pool, a real-time pipeline that forbids allocations (and the device
// synchronisation cudaMalloc may cause) after start-up, or a caller that only
// hands us device buffers it already has.  The caller passes the input planes
// and the output decision arrays (all device memory it owns); the scratch
// the search needs lives in the fixed array below, which the module creates
// when the library is loaded.
//
// Scratch: g_noalloc_scratch holds the device status word and the per-CTU
// argmin keys.  Its size caps the frame: at most kNoallocMaxKeyBytes /
// (8 * keys per CTU) CTUs (3083 CTUs of 64x64; a 3840x2160 frame has 2040).
// Every call reuses the same array and leaves its contents behind; the keys
// are reset at the start of each call.  The status word is not: a bounded
// wait that runs out sets it and it stays set until
// analyze_reference_noalloc_status reads and clears it.  Two calls whose
// work overlaps on the GPU (different streams, no ordering) race on the
// array: order them.
#include "../../include/ladder.h"
#include "ladder_internal.h"

#include <cudaTypedefs.h>

using namespace ladder_impl;

namespace {

constexpr size_t kNoallocScratchBytes = 2u << 20;               // 2 MiB, every device that loads the library
constexpr size_t kNoallocStatusBytes = 256;
constexpr size_t kNoallocMaxKeyBytes = kNoallocScratchBytes - kNoallocStatusBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the scratch array in the current device's context (host
// code may not use the symbol itself, which is only a host-side stand-in for
// the device array).  Looked up on every call: the address belongs to the
// context, and a context that was reset and created again (cudaDeviceReset)
// loads the module anew, possibly elsewhere.  The first lookup in a context
// loads the module there.
ladder_status scratch_for_current_device(unsigned char **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return LADDER_E_CUDA;
    }
    *out = static_cast<unsigned char *>(p);
    return LADDER_OK;
}

}  // namespace

extern "C" ladder_status analyze_reference_noalloc_status(void *cuda_stream)
{
    unsigned char *scratch = nullptr;
    ladder_status st = scratch_for_current_device(&scratch);
    if (st != LADDER_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, scratch, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && status != kStatusOk) {
        e = cudaMemsetAsync(scratch, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LADDER_E_CUDA;
    }
    if (status == kStatusOk) return LADDER_OK;
    return status == kStatusBounds ? LADDER_E_BOUNDS : LADDER_E_TIMEOUT;
}

extern "C" ladder_status analyze_reference_noalloc(const void *cur, const void *ref, int width, int height,
                                                   long pitch_bytes, int bit_depth, int ctu_size, int search_range,
                                                   int qp, int satd_mode, const ladder_decisions *out,
                                                   void *cuda_stream)
{
    // argument checks (the same limits as ladder_init / analyze_reference)
    if (!cur || !ref || !out) return LADDER_E_INVAL;
    if (bit_depth != 8 && bit_depth != 10) return LADDER_E_INVAL;
    if (ctu_size != 16 && ctu_size != 32 && ctu_size != 64) return LADDER_E_INVAL;
    if (search_range < 4 || search_range > 64 || qp < 0 || qp > 51) return LADDER_E_INVAL;
    if (satd_mode != 0 && satd_mode != 1) return LADDER_E_INVAL;
    if (width < 16 || height < 16 || width > 8192 || height > 8192 || (width & 1) || (height & 1))
        return LADDER_E_INVAL;
    const int ss = bit_depth == 8 ? 1 : 2;
    if (pitch_bytes <= 0 || (pitch_bytes & 15) || pitch_bytes < static_cast<long>(width) * ss) return LADDER_E_INVAL;
    if ((reinterpret_cast<uintptr_t>(cur) & 15) || (reinterpret_cast<uintptr_t>(ref) & 15)) return LADDER_E_INVAL;

    RungGeom g{};
    g.W = width;
    g.H = height;
    g.W8 = (width + 7) / 8 * 8;
    g.H8 = (height + 7) / 8 * 8;
    g.ctu = ctu_size;
    g.dmax = ctu_size == 64 ? 3 : (ctu_size == 32 ? 2 : 1);
    g.ctu_cols = (g.W8 + ctu_size - 1) / ctu_size;
    g.ctu_rows = (g.H8 + ctu_size - 1) / ctu_size;
    for (int d = 0; d <= g.dmax; ++d) {
        const int S = ctu_size >> d;
        g.cols[d] = (g.W8 + S - 1) / S;
        g.rows[d] = (g.H8 + S - 1) / S;
    }
    g.cols8 = g.W8 / 8;
    g.rows8 = g.H8 / 8;
    // sizes beyond the scratch array are refused
    const int nctus = g.ctu_cols * g.ctu_rows;
    const long nkeys = static_cast<long>(nctus) * keys_per_ctu(g.dmax);
    if (static_cast<size_t>(nkeys) * 8 > kNoallocMaxKeyBytes) return LADDER_E_INVAL;
    DevDecisions dec{};
    for (int d = 0; d <= g.dmax; ++d) {
        if (!out->mvx[d] || !out->mvy[d] || !out->sad[d] || !out->satd[d] || !out->cost[d] || !out->best[d] ||
            !out->split[d] || !out->evaluated[d])
            return LADDER_E_INVAL;
        dec.mvx[d] = out->mvx[d];
        dec.mvy[d] = out->mvy[d];
        dec.sad[d] = out->sad[d];
        dec.satd[d] = out->satd[d];
        dec.cost[d] = out->cost[d];
        dec.best[d] = out->best[d];
        dec.split[d] = out->split[d];
        dec.evaluated[d] = out->evaluated[d];
    }
    if (!out->leaf_depth || !out->leaf_mvx || !out->leaf_mvy) return LADDER_E_INVAL;
    dec.leaf_depth = out->leaf_depth;
    dec.leaf_mvx = out->leaf_mvx;
    dec.leaf_mvy = out->leaf_mvy;

    unsigned char *scratch = nullptr;
    ladder_status st = scratch_for_current_device(&scratch);
    if (st != LADDER_OK) return st;
    int *d_status = reinterpret_cast<int *>(scratch);
    unsigned long long *d_keys = reinterpret_cast<unsigned long long *>(scratch + kNoallocStatusBytes);

    const FullSearchPlan plan = full_search_plan(bit_depth, ctu_size, search_range);
    FullSearchBatch fb{};
    fb.n = 1;
    fill_full_search_batch(fb, plan, search_range);
    fb.status = d_status;
    fb.total = nctus * plan.ctas_per_ctu;
    fb.item[0] = FullSearchItem{width, height, d_keys, 0};
    if (encode_item_maps(fb, 0, cur, ref, width, height, pitch_bytes, bit_depth, ctu_size, plan) != 0)
        return LADDER_E_CUDA;

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    FillBatch fill{};
    fill.n = 1;
    fill.item[0] = FillItem{d_keys, nkeys};
    cudaError_t e = launch_fill_keys(fill, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LADDER_E_CUDA;
    }
    e = launch_full_search(bit_depth, ctu_size, fb, s);
    if (e == cudaSuccess) {
        // the decision kernel reads its arrays as offsets from a block base;
        // here every array is the caller's (or the scratch's), so there is
        // no block: a null base makes the offsets the arrays' addresses
        DecideBatch db{};
        db.n = 1;
        db.range = search_range;
        db.satd_mode = satd_mode;
        db.total_ctas = nctus;
        db.status = d_status;
        RungInfo &ri = db.rung[0];
        ri.g = g;
        for (int d = 0; d <= g.dmax; ++d) {
            ri.off.mvx[d] = reinterpret_cast<long>(dec.mvx[d]);
            ri.off.mvy[d] = reinterpret_cast<long>(dec.mvy[d]);
            ri.off.sad[d] = reinterpret_cast<long>(dec.sad[d]);
            ri.off.satd[d] = reinterpret_cast<long>(dec.satd[d]);
            ri.off.cost[d] = reinterpret_cast<long>(dec.cost[d]);
            ri.off.best[d] = reinterpret_cast<long>(dec.best[d]);
            ri.off.split[d] = reinterpret_cast<long>(dec.split[d]);
            ri.off.evaluated[d] = reinterpret_cast<long>(dec.evaluated[d]);
        }
        ri.off.leaf_depth = reinterpret_cast<long>(dec.leaf_depth);
        ri.off.leaf_mvx = reinterpret_cast<long>(dec.leaf_mvx);
        ri.off.leaf_mvy = reinterpret_cast<long>(dec.leaf_mvy);
        ri.off.keys = reinterpret_cast<long>(d_keys);
        db.item[0] = DecideItem{cur, ref, pitch_bytes, nullptr, 0, qp, 0};
        e = launch_decide(bit_depth, ctu_size, db, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LADDER_E_CUDA;
    }
    return LADDER_OK;
}
