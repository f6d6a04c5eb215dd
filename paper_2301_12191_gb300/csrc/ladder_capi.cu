// ladder_capi.cu -- host side of the C ABI declared in include/ladder.h:
// geometry validation, frame slots, one device arena per handle, TMA
// descriptor encoding and the launch sequence of each analysis.
#include "../../include/ladder.h"
#include "ladder_internal.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace ladder_impl;

namespace {

struct RungBuffers {
    DevDecisions dec;
    char *dec_base;     // the decision arrays form one contiguous block
    size_t dec_bytes;
    unsigned long long *keys;
    int analysed;  // 0: nothing, 1: independent, 2: dependent
};

struct Slot {
    int used;
    int frame_id;
    int ref_done;
    std::vector<RungBuffers> rungs;
};

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

constexpr int kKinds = 4;  // full search, decide, dependent, fill keys

struct ProfEvent {
    int kind;
    cudaEvent_t start, stop;
};

struct ladder {
    ladder_geometry geo;
    std::vector<ladder_rung> rungs;
    std::vector<RungGeom> rg;
    std::vector<Slot> slots;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    int *d_status = nullptr;
    int *d_tiles = nullptr;
    int ntiles = 0;
    uint16_t *d_rank = nullptr, *d_unrank = nullptr;  // refinement candidate order
    int rank_bits = 0;
    std::string err;
    int sm_count = 0;
    int fs_ctas_per_sm = 1;  // resident full-search CTAs per SM
    char *host_stage = nullptr;  // pinned staging for fetch_decisions
    size_t host_stage_bytes = 0;
    // tracing
    int prof_on = 0;
    long launches[kKinds] = {};
    double total_ms[kKinds] = {};
    std::vector<ProfEvent> pending;
    std::vector<cudaEvent_t> spare;
};

namespace {

ladder_status fail(ladder_t *l, ladder_status st, const char *fmt, ...)
{
    if (l) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        l->err = buf;
    }
    return st;
}

ladder_status cuda_fail(ladder_t *l, cudaError_t e, const char *what)
{
    return fail(l, LADDER_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaEvent_t take_event(ladder_t *l)
{
    if (!l->spare.empty()) {
        cudaEvent_t e = l->spare.back();
        l->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs one launch, counting it and, when timing is on, bracketing it with
// events on its stream.
template <typename F>
cudaError_t traced(ladder_t *l, int kind, cudaStream_t s, F &&launch)
{
    ++l->launches[kind];
    if (!l->prof_on) return launch();
    ProfEvent pe{kind, take_event(l), take_event(l)};
    cudaEventRecord(pe.start, s);
    cudaError_t e = launch();
    cudaEventRecord(pe.stop, s);
    l->pending.push_back(pe);
    return e;
}

void drain_events(ladder_t *l)
{
    for (auto &pe : l->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(pe.stop) == cudaSuccess && cudaEventElapsedTime(&ms, pe.start, pe.stop) == cudaSuccess)
            l->total_ms[pe.kind] += ms;
        l->spare.push_back(pe.start);
        l->spare.push_back(pe.stop);
    }
    l->pending.clear();
}

RungGeom make_geom(int W, int H, int ctu)
{
    RungGeom g{};
    g.W = W;
    g.H = H;
    g.W8 = (W + 7) / 8 * 8;
    g.H8 = (H + 7) / 8 * 8;
    g.ctu = ctu;
    g.dmax = ctu == 64 ? 3 : (ctu == 32 ? 2 : 1);
    g.ctu_cols = (g.W8 + ctu - 1) / ctu;
    g.ctu_rows = (g.H8 + ctu - 1) / ctu;
    for (int d = 0; d <= g.dmax; ++d) {
        const int S = ctu >> d;
        g.cols[d] = (g.W8 + S - 1) / S;
        g.rows[d] = (g.H8 + S - 1) / S;
    }
    g.cols8 = g.W8 / 8;
    g.rows8 = g.H8 / 8;
    return g;
}

// Bytes of one (slot, rung) buffer set; carves it when base != nullptr.
size_t carve(const RungGeom &g, char *base, RungBuffers *rb)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align_up(bytes, 256);
        return p;
    };
    for (int d = 0; d <= g.dmax; ++d) {
        const size_t n = static_cast<size_t>(g.cols[d]) * g.rows[d];
        char *p;
        p = take(n * 2); if (rb) rb->dec.mvx[d] = reinterpret_cast<int16_t *>(p);
        p = take(n * 2); if (rb) rb->dec.mvy[d] = reinterpret_cast<int16_t *>(p);
        p = take(n * 4); if (rb) rb->dec.sad[d] = reinterpret_cast<int32_t *>(p);
        p = take(n * 4); if (rb) rb->dec.satd[d] = reinterpret_cast<int32_t *>(p);
        p = take(n * 4); if (rb) rb->dec.cost[d] = reinterpret_cast<int32_t *>(p);
        p = take(n * 4); if (rb) rb->dec.best[d] = reinterpret_cast<int32_t *>(p);
        p = take(n); if (rb) rb->dec.split[d] = reinterpret_cast<uint8_t *>(p);
        p = take(n); if (rb) rb->dec.evaluated[d] = reinterpret_cast<uint8_t *>(p);
    }
    const size_t n8 = static_cast<size_t>(g.cols8) * g.rows8;
    char *p;
    p = take(n8); if (rb) rb->dec.leaf_depth = reinterpret_cast<uint8_t *>(p);
    p = take(n8 * 2); if (rb) rb->dec.leaf_mvx = reinterpret_cast<int16_t *>(p);
    p = take(n8 * 2); if (rb) rb->dec.leaf_mvy = reinterpret_cast<int16_t *>(p);
    if (rb) {
        rb->dec_base = base;
        rb->dec_bytes = off;
    }
    const size_t nk = static_cast<size_t>(g.ctu_cols) * g.ctu_rows * keys_per_ctu(g.dmax);
    p = take(nk * 8); if (rb) rb->keys = reinterpret_cast<unsigned long long *>(p);
    return off;
}

ladder_status validate_geometry(const ladder_geometry *g)
{
    if (!g || !g->rungs) return LADDER_E_INVAL;
    if (g->n_rungs < 1 || g->n_rungs > 16) return LADDER_E_INVAL;
    if (g->ref_rung < 0 || g->ref_rung >= g->n_rungs) return LADDER_E_INVAL;
    if (g->bit_depth != 8 && g->bit_depth != 10) return LADDER_E_INVAL;
    if (g->ctu_size != 16 && g->ctu_size != 32 && g->ctu_size != 64) return LADDER_E_INVAL;
    if (g->ref_search_range < 4 || g->ref_search_range > 64) return LADDER_E_INVAL;
    if (g->dep_refine_range < 0 || g->dep_refine_range > 32) return LADDER_E_INVAL;
    if (g->dep_depth_lo < -3 || g->dep_depth_lo > 3 || g->dep_depth_hi < -3 || g->dep_depth_hi > 3 ||
        g->dep_depth_lo > g->dep_depth_hi)
        return LADDER_E_INVAL;
    if (g->dep_use_ref_mv != 0 && g->dep_use_ref_mv != 1) return LADDER_E_INVAL;
    if (g->satd_mode != 0 && g->satd_mode != 1) return LADDER_E_INVAL;
    if (g->max_frames < 1 || g->max_frames > 64) return LADDER_E_INVAL;
    for (int i = 0; i < g->n_rungs; ++i) {
        const ladder_rung &r = g->rungs[i];
        if (r.width < 16 || r.height < 16 || r.width > 8192 || r.height > 8192) return LADDER_E_INVAL;
        if ((r.width & 1) || (r.height & 1)) return LADDER_E_INVAL;
    }
    return LADDER_OK;
}

Slot *find_slot(ladder_t *l, int frame_id)
{
    for (auto &s : l->slots)
        if (s.used && s.frame_id == frame_id) return &s;
    return nullptr;
}

Slot *claim_slot(ladder_t *l, int frame_id)
{
    if (Slot *s = find_slot(l, frame_id)) return s;
    for (auto &s : l->slots)
        if (!s.used) {
            s.used = 1;
            s.frame_id = frame_id;
            s.ref_done = 0;
            for (auto &r : s.rungs) r.analysed = 0;
            return &s;
        }
    return nullptr;
}

ladder_status check_planes(ladder_t *l, int rung, const void *cur, const void *ref, long pitch, int qp)
{
    if (rung < 0 || rung >= l->geo.n_rungs) return fail(l, LADDER_E_INVAL, "rung %d out of range", rung);
    if (!cur || !ref) return fail(l, LADDER_E_INVAL, "null plane");
    if ((reinterpret_cast<uintptr_t>(cur) & 15) || (reinterpret_cast<uintptr_t>(ref) & 15))
        return fail(l, LADDER_E_INVAL, "planes must be 16-byte aligned");
    const int ss = l->geo.bit_depth == 8 ? 1 : 2;
    if (pitch <= 0 || (pitch & 15) || pitch < static_cast<long>(l->rungs[rung].width) * ss)
        return fail(l, LADDER_E_INVAL, "pitch %ld must be a multiple of 16 and >= width * %d", pitch, ss);
    if (qp < 0 || qp > 51) return fail(l, LADDER_E_INVAL, "qp %d outside 0..51", qp);
    return LADDER_OK;
}

bool encode_ref_map(ladder_t *l, CUtensorMap *map, const void *ref, const RungGeom &g, long pitch,
                    const FullSearchPlan &p)
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) {
        fail(l, LADDER_E_CUDA, "cuTensorMapEncodeTiled unavailable");
        return false;
    }
    const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(g.W), static_cast<cuuint64_t>(g.H)};
    const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(pitch)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(p.box_w), static_cast<cuuint32_t>(p.box_h)};
    const cuuint32_t estride[2] = {1, 1};
    const CUtensorMapDataType dt =
        l->geo.bit_depth == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    CUresult r = g_encode(map, dt, 2, const_cast<void *>(ref), gdim, gstride, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        fail(l, LADDER_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
        return false;
    }
    return true;
}

// Candidate slices per CTU: whole group-iterations per slice (no duplicate
// tiles), about two waves of CTAs at one resident CTA per SM.
int choose_tiles_per_slice(const ladder_t *l, int nctus, int ntiles, int groups)
{
    const int target = 2 * std::max(1, l->sm_count) * std::max(1, l->fs_ctas_per_sm);
    const int slices = std::max(1, (target + nctus - 1) / nctus);
    int tps = (ntiles + slices - 1) / slices;
    tps = (tps + groups - 1) / groups * groups;
    return std::max(groups, tps);
}

ladder_status run_independent(ladder_t *l, Slot *slot, int rung, const void *cur, const void *ref, long pitch,
                              int qp, cudaStream_t s)
{
    const RungGeom &g = l->rg[rung];
    RungBuffers &rb = slot->rungs[rung];
    const int nctus = g.ctu_cols * g.ctu_rows;
    const int R = l->geo.ref_search_range;
    const FullSearchPlan plan = full_search_plan(l->geo.bit_depth, g.ctu, R);
    CUtensorMap map;
    if (!encode_ref_map(l, &map, ref, g, pitch, plan)) return LADDER_E_CUDA;
    cudaError_t e = traced(l, 3, s, [&] {
        return launch_fill_keys(rb.keys, static_cast<long>(nctus) * keys_per_ctu(g.dmax), s);
    });
    if (e != cudaSuccess) return cuda_fail(l, e, "fill keys");
    const int tps = choose_tiles_per_slice(l, nctus, l->ntiles, plan.groups);
    const int slices = (l->ntiles + tps - 1) / tps;
    FullSearchArgs fa{};
    fa.cur = cur;
    fa.pitch_bytes = pitch;
    fa.W = g.W;
    fa.H = g.H;
    fa.R = R;
    fa.Rp = (R + 15) / 16 * 16;
    fa.ntiles = l->ntiles;
    fa.tiles_per_slice = tps;
    fa.tiles = l->d_tiles;
    fa.keys = rb.keys;
    fa.status = l->d_status;
    e = traced(l, 0, s, [&] { return launch_full_search(l->geo.bit_depth, g.ctu, fa, map, slices, nctus, s); });
    if (e != cudaSuccess) return cuda_fail(l, e, "full search launch");
    DecideArgs da{};
    da.cur = cur;
    da.ref = ref;
    da.pitch_bytes = pitch;
    da.g = g;
    da.range = R;
    da.keys = rb.keys;
    da.qp = qp;
    da.satd_mode = l->geo.satd_mode;
    da.out = rb.dec;
    e = traced(l, 1, s, [&] { return launch_decide(l->geo.bit_depth, da, s); });
    if (e != cudaSuccess) return cuda_fail(l, e, "decide launch");
    rb.analysed = 1;
    return LADDER_OK;
}

}  // namespace

extern "C" {

const char *ladder_version(void) { return "ladder 0.1 (sm_103a)"; }

ladder_status ladder_init(const ladder_geometry *geometry, void *cuda_stream, ladder_t **out)
{
    if (!out) return LADDER_E_INVAL;
    *out = nullptr;
    ladder_status st = validate_geometry(geometry);
    if (st != LADDER_OK) return st;
    ladder_t *l = new (std::nothrow) ladder();
    if (!l) return LADDER_E_NOMEM;
    l->geo = *geometry;
    l->rungs.assign(geometry->rungs, geometry->rungs + geometry->n_rungs);
    l->geo.rungs = l->rungs.data();
    for (const auto &r : l->rungs) l->rg.push_back(make_geom(r.width, r.height, geometry->ctu_size));
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l->sm_count, cudaDevAttrMultiProcessorCount, dev);
    l->fs_ctas_per_sm = full_search_ctas_per_sm(geometry->bit_depth, geometry->ctu_size, geometry->ref_search_range);

    size_t per_slot = 0;
    for (const auto &g : l->rg) per_slot += carve(g, nullptr, nullptr);
    const int ntiles = full_search_tiles(geometry->bit_depth, geometry->ref_search_range, nullptr, 0);
    l->ntiles = ntiles;
    const int Kr = 2 * geometry->dep_refine_range + 1;
    const size_t rank_bytes = align_up(static_cast<size_t>(Kr) * Kr * 2, 256);
    const size_t fixed = align_up(256, 256) + align_up(static_cast<size_t>(ntiles) * 4, 256) + 2 * rank_bytes;
    l->arena_bytes = fixed + per_slot * geometry->max_frames;
    cudaError_t e = cudaMalloc(&l->arena, l->arena_bytes);
    if (e != cudaSuccess) {
        delete l;
        cudaGetLastError();
        return LADDER_E_NOMEM;
    }
    char *base = static_cast<char *>(l->arena);
    l->d_status = reinterpret_cast<int *>(base);
    l->d_tiles = reinterpret_cast<int *>(base + 256);
    l->d_rank = reinterpret_cast<uint16_t *>(base + 256 + align_up(static_cast<size_t>(ntiles) * 4, 256));
    l->d_unrank = reinterpret_cast<uint16_t *>(reinterpret_cast<char *>(l->d_rank) + rank_bytes);
    while ((1 << l->rank_bits) < Kr * Kr) ++l->rank_bits;
    char *p = base + fixed;
    l->slots.resize(geometry->max_frames);
    for (auto &s : l->slots) {
        s.used = 0;
        s.frame_id = 0;
        s.ref_done = 0;
        s.rungs.resize(l->rg.size());
        for (size_t r = 0; r < l->rg.size(); ++r) {
            p += carve(l->rg[r], p, &s.rungs[r]);
            s.rungs[r].analysed = 0;
        }
    }
    for (const auto &r : l->slots[0].rungs) l->host_stage_bytes = std::max(l->host_stage_bytes, r.dec_bytes);
    if (cudaMallocHost(&l->host_stage, l->host_stage_bytes) != cudaSuccess) {
        cudaFree(l->arena);
        delete l;
        cudaGetLastError();
        return LADDER_E_NOMEM;
    }
    std::vector<int> tiles(ntiles);
    full_search_tiles(geometry->bit_depth, geometry->ref_search_range, tiles.data(), ntiles);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    e = cudaMemsetAsync(l->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(l->d_tiles, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice, s);
    std::vector<uint16_t> rank(static_cast<size_t>(Kr) * Kr), unrank(rank.size());
    refine_rank_tables(geometry->dep_refine_range, rank.data(), unrank.data());
    if (e == cudaSuccess) e = cudaMemcpyAsync(l->d_rank, rank.data(), rank.size() * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(l->d_unrank, unrank.data(), unrank.size() * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFreeHost(l->host_stage);
        cudaFree(l->arena);
        delete l;
        return LADDER_E_CUDA;
    }
    *out = l;
    return LADDER_OK;
}

ladder_status analyze_independent(ladder_t *l, int rung, int frame_id, const void *cur, const void *ref,
                                  long pitch_bytes, int qp, void *cuda_stream)
{
    if (!l) return LADDER_E_INVAL;
    ladder_status st = check_planes(l, rung, cur, ref, pitch_bytes, qp);
    if (st != LADDER_OK) return st;
    Slot *slot = claim_slot(l, frame_id);
    if (!slot) return fail(l, LADDER_E_BUSY, "no free frame slot for frame %d", frame_id);
    st = run_independent(l, slot, rung, cur, ref, pitch_bytes, qp, static_cast<cudaStream_t>(cuda_stream));
    if (st == LADDER_OK && rung == l->geo.ref_rung) slot->ref_done = 1;
    return st;
}

ladder_status analyze_reference(ladder_t *l, int frame_id, const void *cur, const void *ref, long pitch_bytes,
                                int qp, void *cuda_stream)
{
    if (!l) return LADDER_E_INVAL;
    return analyze_independent(l, l->geo.ref_rung, frame_id, cur, ref, pitch_bytes, qp, cuda_stream);
}

ladder_status analyze_dependents(ladder_t *l, int frame_id, int n, const int *rungs, const void *const *cur,
                                 const void *const *ref, const long *pitch_bytes, int qp, void *cuda_stream)
{
    if (!l) return LADDER_E_INVAL;
    if (n < 1 || n > kMaxBatch || !rungs || !cur || !ref || !pitch_bytes)
        return fail(l, LADDER_E_INVAL, "dependent batch of %d rungs (1..%d)", n, kMaxBatch);
    for (int k = 0; k < n; ++k) {
        ladder_status st = check_planes(l, rungs[k], cur[k], ref[k], pitch_bytes[k], qp);
        if (st != LADDER_OK) return st;
        if (rungs[k] == l->geo.ref_rung) return fail(l, LADDER_E_INVAL, "rung %d is the reference rung", rungs[k]);
        for (int j = 0; j < k; ++j)
            if (rungs[j] == rungs[k]) return fail(l, LADDER_E_INVAL, "rung %d appears twice", rungs[k]);
    }
    Slot *slot = find_slot(l, frame_id);
    if (!slot || !slot->ref_done)
        return fail(l, LADDER_E_NOREF, "frame %d has no reference analysis", frame_id);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const RungGeom &gr = l->rg[l->geo.ref_rung];
    const RungBuffers &ref_rb = slot->rungs[l->geo.ref_rung];
    DependentBatch batch{};
    batch.n = n;
    batch.cta_begin[0] = 0;
    for (int k = 0; k < n; ++k) {
        const RungGeom &g = l->rg[rungs[k]];
        DependentArgs &da = batch.rung[k];
        da.cur = cur[k];
        da.ref = ref[k];
        da.pitch_bytes = pitch_bytes[k];
        da.g = g;
        da.r = l->geo.dep_refine_range;
        da.rank = l->d_rank;
        da.unrank = l->d_unrank;
        da.rank_bits = l->rank_bits;
        da.refs.Wr = gr.W;
        da.refs.Hr = gr.H;
        da.refs.cols8_r = gr.cols8;
        da.refs.leaf_depth = ref_rb.dec.leaf_depth;
        da.refs.leaf_mvx = ref_rb.dec.leaf_mvx;
        da.refs.leaf_mvy = ref_rb.dec.leaf_mvy;
        da.refs.depth_lo = l->geo.dep_depth_lo;
        da.refs.depth_hi = l->geo.dep_depth_hi;
        da.refs.use_ref_mv = l->geo.dep_use_ref_mv;
        da.qp = qp;
        da.satd_mode = l->geo.satd_mode;
        da.out = slot->rungs[rungs[k]].dec;
        da.status = l->d_status;
        batch.cta_begin[k + 1] = batch.cta_begin[k] + g.ctu_cols * g.ctu_rows;
    }
    cudaError_t e = traced(l, 2, s, [&] {
        return launch_dependent(l->geo.bit_depth, l->geo.ctu_size, l->geo.dep_refine_range, batch, s);
    });
    if (e != cudaSuccess) return cuda_fail(l, e, "dependent launch");
    for (int k = 0; k < n; ++k) slot->rungs[rungs[k]].analysed = 2;
    return LADDER_OK;
}

ladder_status analyze_dependent(ladder_t *l, int rung, int frame_id, const void *cur, const void *ref,
                                long pitch_bytes, int qp, void *cuda_stream)
{
    return analyze_dependents(l, frame_id, 1, &rung, &cur, &ref, &pitch_bytes, qp, cuda_stream);
}

ladder_status ladder_grid(const ladder_t *l, int rung, int *dims, int *n_depths)
{
    if (!l || !dims || rung < 0 || rung >= l->geo.n_rungs) return LADDER_E_INVAL;
    const RungGeom &g = l->rg[rung];
    for (int d = 0; d <= g.dmax; ++d) {
        dims[2 * d] = g.cols[d];
        dims[2 * d + 1] = g.rows[d];
    }
    dims[2 * (g.dmax + 1)] = g.cols8;
    dims[2 * (g.dmax + 1) + 1] = g.rows8;
    if (n_depths) *n_depths = g.dmax + 1;
    return LADDER_OK;
}

ladder_status ladder_sync(ladder_t *l, void *cuda_stream)
{
    if (!l) return LADDER_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, l->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(l, e, "sync");
    if (status != 0) {
        cudaMemsetAsync(l->d_status, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        return fail(l, LADDER_E_TIMEOUT, "a bounded device wait ran out");
    }
    return LADDER_OK;
}

ladder_status fetch_decisions(ladder_t *l, int rung, int frame_id, ladder_decisions *out, void *cuda_stream)
{
    if (!l || !out) return LADDER_E_INVAL;
    if (rung < 0 || rung >= l->geo.n_rungs) return fail(l, LADDER_E_INVAL, "rung %d out of range", rung);
    Slot *slot = find_slot(l, frame_id);
    if (!slot || !slot->rungs[rung].analysed)
        return fail(l, LADDER_E_STATE, "rung %d of frame %d has not been analysed", rung, frame_id);
    const RungGeom &g = l->rg[rung];
    const RungBuffers &rb = slot->rungs[rung];
    const DevDecisions &dec = rb.dec;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // one copy of the rung's whole decision block into pinned memory, then
    // host copies into the caller's arrays
    cudaError_t e = cudaMemcpyAsync(l->host_stage, rb.dec_base, rb.dec_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(l, e, "fetch copy");
    auto copy = [&](void *dst, const void *src, size_t bytes) {
        if (dst) memcpy(dst, l->host_stage + (static_cast<const char *>(src) - rb.dec_base), bytes);
    };
    for (int d = 0; d <= g.dmax; ++d) {
        const size_t n = static_cast<size_t>(g.cols[d]) * g.rows[d];
        copy(out->mvx[d], dec.mvx[d], n * 2);
        copy(out->mvy[d], dec.mvy[d], n * 2);
        copy(out->sad[d], dec.sad[d], n * 4);
        copy(out->satd[d], dec.satd[d], n * 4);
        copy(out->cost[d], dec.cost[d], n * 4);
        copy(out->best[d], dec.best[d], n * 4);
        copy(out->split[d], dec.split[d], n);
        copy(out->evaluated[d], dec.evaluated[d], n);
    }
    const size_t n8 = static_cast<size_t>(g.cols8) * g.rows8;
    copy(out->leaf_depth, dec.leaf_depth, n8);
    copy(out->leaf_mvx, dec.leaf_mvx, n8 * 2);
    copy(out->leaf_mvy, dec.leaf_mvy, n8 * 2);
    return ladder_sync(l, cuda_stream);
}

ladder_status ladder_release_frame(ladder_t *l, int frame_id)
{
    if (!l) return LADDER_E_INVAL;
    Slot *slot = find_slot(l, frame_id);
    if (!slot) return fail(l, LADDER_E_STATE, "frame %d holds no slot", frame_id);
    slot->used = 0;
    slot->ref_done = 0;
    for (auto &r : slot->rungs) r.analysed = 0;
    return LADDER_OK;
}

ladder_status ladder_profile_enable(ladder_t *l, int enable)
{
    if (!l) return LADDER_E_INVAL;
    l->prof_on = enable != 0;
    return LADDER_OK;
}

ladder_status ladder_profile_read(ladder_t *l, int kind, long *launches, double *total_ms, int reset)
{
    if (!l || kind < 0 || kind >= kKinds) return LADDER_E_INVAL;
    drain_events(l);
    if (launches) *launches = l->launches[kind];
    if (total_ms) *total_ms = l->total_ms[kind];
    if (reset) {
        l->launches[kind] = 0;
        l->total_ms[kind] = 0.0;
    }
    return LADDER_OK;
}

void ladder_destroy(ladder_t *l)
{
    if (!l) return;
    cudaDeviceSynchronize();
    drain_events(l);
    for (cudaEvent_t e : l->spare) cudaEventDestroy(e);
    cudaFreeHost(l->host_stage);
    cudaFree(l->arena);
    delete l;
}

const char *ladder_last_error(const ladder_t *l) { return l ? l->err.c_str() : "null handle"; }

}  // extern "C"
