// ladder_capi.cu -- host side of the C ABI declared in include/ladder.h:
// geometry validation, frame slots, one device arena per handle, TMA
// descriptor encoding, batched launch descriptors, CUDA-graph capture of a
// batch, and per-kernel tracing.
#include "../../include/ladder.h"
#include "ladder_internal.h"

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

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
    char *block;   // decision arrays [0, dec_bytes) then the argmin keys
    int analysed;  // 0: nothing, 1: independent, 2: dependent
};

struct Slot {
    int used;
    int frame_id;
    int ref_done;
    std::vector<RungBuffers> rungs;
};


size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr int kKinds = 9;  // full search, decide, dependent search, fill keys, dependent rules, dependent decide,
                           // further-QP decisions, quarter-pel refinement, spatial-predictor decisions

struct ProfEvent {
    int kind;
    cudaEvent_t start, stop;
};

// The last work a handle enqueued on one stream: ladder_destroy waits for
// these events (the handle's own work) rather than for the whole device.
struct StreamMark {
    cudaStream_t stream;
    cudaEvent_t done;
};
constexpr size_t kMaxMarks = 16;

}  // namespace

// One set of dependent task lists: the counters, tasks, positions and sum
// tables a dependent batch fills and consumes.  A batch takes the set its
// stream used last (no wait: one stream is ordered), else a set not used
// yet, else the least recently used one, waiting for that set's last batch.
struct DepSet {
    unsigned int *counts = nullptr;  // kDepCounters: tasks and inherited CUs per CU size class, next tile
    unsigned long long *tasks[kSizeClasses] = {};
    unsigned int *pos[kSizeClasses] = {};
    unsigned int *sums[kSizeClasses] = {};
    unsigned int *up[kSizeClasses] = {};  // classes kFirstUpClass .. kSizeClasses - 2
    bool counts_dirty = false;  // counters not known to be zero (zeroed with the arena at init)
    cudaEvent_t done = nullptr;
    bool recorded = false;
    cudaStream_t stream = nullptr;  // stream of the set's last recorded batch
    unsigned long long last_use = 0;
};
constexpr int kDepSets = 3;

struct ladder {
    ladder_geometry geo;
    std::vector<ladder_rung> rungs;
    std::vector<RungInfo> info;  // geometry + block layout per rung
    std::vector<Slot> slots;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    int *d_status = nullptr;
    // dependent launches share the task lists: each waits for the one
    // before it (on whatever stream that ran)
    std::vector<int> parent;  // per rung: the rung whose decisions a dependent analysis refines (-1: reference)
    std::vector<int> tier;    // per rung: steps from the reference rung along the parents
    // every argmin key is ~0 at rest (searches reset them after use); after a
    // failed launch that may not hold, and the next launch fills them first
    bool keys_dirty = true;
    // dependent task lists: kDepSets sets taken in turn by dependent batches,
    // so batches on different streams (consecutive frames) run side by side
    DepSet dep[kDepSets];
    unsigned long long dep_clock = 0;
    unsigned int task_cap[kSizeClasses] = {};  // entries per list (every set)
    std::string err;
    int sm_count = 0;
    int fs_ctas_per_sm = 1;      // resident full-search CTAs per SM
    // kernel shapes (ladder_set_tuning): results never depend on them
    int tune_fs_band = kFsBand, tune_fs_group = 0, tune_fs_fuse = 1, tune_dep_band = 0, tune_dep_range = 16,
        tune_dep_ctas = 0, tune_dep_staged = 1, tune_dep_inherit = 1;
    unsigned long long *d_evals = nullptr;  // running count of the dependent searches' SAD-candidate evaluations
    int mv_predictor = 0;  // 0: (0, 0); 1: spatial, decided in wavefront order (ladder_set_mv_predictor)
    // test controls (ladder_set_debug)
    int dbg_wait_polls = 0;   // 0: kMvpSpinDefault
    int dbg_lost_handoff = 0;
    int mvp_capacity = 0;  // resident CTAs of the wavefront kernel
    int subpel_mvp_capacity = 0;  // resident CTAs of the refinement's wavefront kernel
    char *host_stage = nullptr;  // pinned staging for fetch_decisions
    size_t host_stage_bytes = 0;
    // tracing
    int prof_on = 0;
    long launches[kKinds] = {};
    double total_ms[kKinds] = {};
    std::vector<ProfEvent> pending;
    std::vector<cudaEvent_t> spare;
    // streams the handle's calls enqueued work on (not inside a capture, nor
    // a pipeline's own streams, which the pipeline waits for itself)
    std::vector<StreamMark> marks;
    int quiet = 0;
};

struct ladder_graph {
    ladder_t *l = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// An NVTX range around a public call (no cost without an attached tool):
// profilers show each call's host span beside its kernels.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
};

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

// Error of a non-zero device status word.
ladder_status device_status_error(ladder_t *l, int status)
{
    if (status == kStatusTaskOverflow) return fail(l, LADDER_E_STATE, "a dependent task list overflowed");
    if (status == kStatusBounds) return fail(l, LADDER_E_BOUNDS, "a device-side bounds check failed");
    return fail(l, LADDER_E_TIMEOUT, "a bounded device wait ran out");
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

// Records, after a public call's work on stream s, an event that
// ladder_destroy waits for.
void mark_stream(ladder_t *l, cudaStream_t s)
{
    if (l->quiet) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cap != cudaStreamCaptureStatusNone) return;  // a graph: its launches are marked instead
    for (auto &m : l->marks)
        if (m.stream == s) {
            cudaEventRecord(m.done, s);
            return;
        }
    if (l->marks.size() >= kMaxMarks) {  // the oldest stream: wait for it now
        cudaEventSynchronize(l->marks.front().done);
        cudaEventDestroy(l->marks.front().done);
        l->marks.erase(l->marks.begin());
    }
    StreamMark m{s, nullptr};
    if (cudaEventCreateWithFlags(&m.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(m.done, s);
    l->marks.push_back(m);
}

// The status of a call that enqueued work on s: marks the stream on success.
ladder_status marked(ladder_t *l, cudaStream_t s, ladder_status st)
{
    if (st == LADDER_OK) mark_stream(l, s);
    return st;
}

void drain_events(ladder_t *l)
{
    for (auto &pe : l->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(pe.stop) == cudaSuccess &&
            cudaEventElapsedTime(&ms, pe.start, pe.stop) == cudaSuccess)
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
    g.div_2w = make_fastdiv(2u * static_cast<uint32_t>(W));
    g.div_2h = make_fastdiv(2u * static_cast<uint32_t>(H));
    return g;
}

// Layout of one (slot, rung) block: the decision arrays, each 256-byte
// aligned, then the argmin keys.  Returns the block's bytes.
size_t layout(const RungGeom &g, DecOffsets &o)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const long at = static_cast<long>(off);
        off += align_up(bytes, 256);
        return at;
    };
    o = DecOffsets{};
    for (int d = 0; d <= g.dmax; ++d) {
        const size_t n = static_cast<size_t>(g.cols[d]) * g.rows[d];
        o.mvx[d] = take(n * 2);
        o.mvy[d] = take(n * 2);
        o.sad[d] = take(n * 4);
        o.satd[d] = take(n * 4);
        o.cost[d] = take(n * 4);
        o.best[d] = take(n * 4);
        o.split[d] = take(n);
        o.evaluated[d] = take(n);
    }
    const size_t n8 = static_cast<size_t>(g.cols8) * g.rows8;
    o.leaf_depth = take(n8);
    o.leaf_mvx = take(n8 * 2);
    o.leaf_mvy = take(n8 * 2);
    o.dec_bytes = static_cast<long>(off);
    const size_t nk = static_cast<size_t>(g.ctu_cols) * g.ctu_rows * keys_per_ctu(g.dmax);
    o.keys = take(nk * 8);
    o.dep_cx = take(nk * 2);
    o.dep_cy = take(nk * 2);
    o.dep_flags = take(nk);
    o.dep_slot = take(nk * 4);
    o.done = take(static_cast<size_t>(g.ctu_cols) * g.ctu_rows * 4);
    // per CTU one word per bottom-row 8x8 block (ctu / 8 of them), then 2 counters
    o.mvp_flag = take(static_cast<size_t>(g.ctu_cols) * g.ctu_rows * g.ctu + 8);
    return off;
}

ladder_status validate_geometry(const ladder_geometry *g)
{
    if (!g || !g->rungs) return LADDER_E_INVAL;
    if (g->n_rungs < 1 || g->n_rungs > kMaxRungs) return LADDER_E_INVAL;
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
    if (g->max_frames < 1 || g->max_frames > 256) return LADDER_E_INVAL;
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

// One rung of one frame and its planes.
struct Job {
    Slot *slot;
    int rung;
    const void *cur, *ref;
    long pitch;
    int qp;
};

// Decisions with the spatial MV predictor of analysed jobs (their vectors
// and SATDs resident): cooperative launches of one CTA per CTU row, as many
// jobs per launch as fit on the device at once.
ladder_status launch_mvp(ladder_t *l, const Job *jobs, int n, int dependent, cudaStream_t s)
{
    if (l->mvp_capacity <= 0) l->mvp_capacity = decide_mvp_capacity(l->geo.ctu_size, l->sm_count);
    auto *b = new (std::nothrow) MvpBatch{};
    if (!b) return fail(l, LADDER_E_NOMEM, "wavefront batch table");
    for (int r = 0; r < l->geo.n_rungs; ++r) b->rung[r] = l->info[r];
    b->status = l->d_status;
    b->spin = l->dbg_wait_polls > 0 ? l->dbg_wait_polls : kMvpSpinDefault;
    b->lost_handoff = l->dbg_lost_handoff;
    int k = 0;
    while (k < n) {
        int m = 0, ctas = 0;
        while (k + m < n && m < kMaxMvpItems) {
            const Job &jb = jobs[k + m];
            const int rows = l->info[jb.rung].g.ctu_rows;
            if (m > 0 && ctas + rows > l->mvp_capacity) break;
            RungBuffers &rb = jb.slot->rungs[jb.rung];
            b->item[m] = MvpItem{rb.block, jb.rung, jb.qp, dependent, ctas};
            ctas += rows;
            ++m;
        }
        if (ctas > l->mvp_capacity) {
            delete b;
            return fail(l, LADDER_E_INVAL, "%d CTU rows exceed the %d resident wavefront CTAs", ctas, l->mvp_capacity);
        }
        b->n = m;
        const cudaError_t e = traced(l, 8, s, [&] { return launch_decide_mvp(l->geo.ctu_size, *b, ctas, s); });
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(l, e, "spatial-predictor decisions");
        }
        k += m;
    }
    delete b;
    return LADDER_OK;
}

// Full search + decisions of independently analysed jobs, in batched
// launches of at most kMaxItems jobs.
ladder_status launch_independent(ladder_t *l, const Job *jobs, int n, cudaStream_t s)
{
    const int R = l->geo.ref_search_range;
    // warp tiles per CTA: the knob, or automatically 1 (many small CTAs for
    // the tail of a small launch) unless the launch has several waves of
    // tiles, where sharing one staged window between 2 tiles saves work
    int group = l->tune_fs_group;
    // 10-bit frames of whole 8x8 blocks read their current CTUs through L1
    // (no shared copy: room for a third CTA per SM)
    int cur_l1 = l->geo.bit_depth == 10 ? 1 : 0;
    for (int k = 0; k < n; ++k)
        if ((l->info[jobs[k].rung].g.W & 7) || (l->info[jobs[k].rung].g.H & 7)) cur_l1 = 0;
    if (group <= 0) {
        const FullSearchPlan p1 =
            full_search_plan(l->geo.bit_depth, l->geo.ctu_size, R, l->tune_fs_band, 1, cur_l1);
        long tiles = 0;
        for (int k = 0; k < n; ++k)
            tiles += static_cast<long>(l->info[jobs[k].rung].g.ctu_cols) * l->info[jobs[k].rung].g.ctu_rows *
                     p1.warp_tiles;
        group = tiles >= 6L * l->sm_count * std::max(1, l->fs_ctas_per_sm) ? 2 : 1;
    }
    const FullSearchPlan plan =
        full_search_plan(l->geo.bit_depth, l->geo.ctu_size, R, l->tune_fs_band, group, cur_l1);
    for (int j0 = 0; j0 < n; j0 += kMaxItems) {
        const int m = std::min(kMaxItems, n - j0);
        FillBatch fill{};
        FullSearchBatch fb{};
        DecideBatch db{};
        fill.n = m;
        fb.n = m;
        fill_full_search_batch(fb, plan, R);
        fb.status = l->d_status;
        for (int r = 0; r < l->geo.n_rungs; ++r) fb.rung[r] = l->info[r];
        db.n = m;
        db.range = R;
        db.satd_mode = l->geo.satd_mode;
        db.status = l->d_status;
        for (int r = 0; r < l->geo.n_rungs; ++r) db.rung[r] = l->info[r];
        int total = 0, total_ctas = 0;
        for (int k = 0; k < m; ++k) {
            const Job &jb = jobs[j0 + k];
            const RungInfo &ri = l->info[jb.rung];
            char *block = jb.slot->rungs[jb.rung].block;
            auto *keys = reinterpret_cast<unsigned long long *>(block + ri.off.keys);
            const int nctus = ri.g.ctu_cols * ri.g.ctu_rows;
            fill.item[k] = FillItem{keys, static_cast<long>(nctus) * keys_per_ctu(ri.g.dmax)};
            const int er = encode_item_maps(fb, k, jb.cur, jb.ref, ri.g.W, ri.g.H, jb.pitch, l->geo.bit_depth,
                                            l->geo.ctu_size, plan);
            if (er != 0) return fail(l, LADDER_E_CUDA, "tensor map encoding failed (%d)", er);
            fb.item[k] = FullSearchItem{ri.g.W,   ri.g.H, keys,   total_ctas, jb.cur,
                                        jb.ref,   jb.pitch, block, jb.rung,   jb.qp,
                                        reinterpret_cast<unsigned int *>(block + ri.off.done)};
            db.item[k] = DecideItem{jb.cur, jb.ref, jb.pitch, block, jb.rung, jb.qp, total};
            total += nctus;
            total_ctas += nctus * plan.ctas_per_ctu;
        }
        db.total_ctas = total;
        fb.total = total_ctas;
        // fused: keys are ~0 at rest and the last CTA of each CTU takes its
        // decisions (and resets its keys); otherwise fill + search + decide
        const bool fuse = !l->keys_dirty && l->tune_fs_fuse;
        fb.fuse_decide = fuse ? 1 : 0;
        fb.satd_mode = l->geo.satd_mode;
        cudaError_t e = cudaSuccess;
        if (!fuse) {
            // after a failed launch: counters back to zero, keys to ~0
            for (int k = 0; k < m && e == cudaSuccess; ++k) {
                const RungInfo &ri = l->info[jobs[j0 + k].rung];
                e = cudaMemsetAsync(fb.item[k].done, 0, static_cast<size_t>(ri.g.ctu_cols) * ri.g.ctu_rows * 4, s);
            }
            if (e == cudaSuccess) e = traced(l, 3, s, [&] { return launch_fill_keys(fill, s); });
            if (e != cudaSuccess) {
                l->keys_dirty = true;
                return cuda_fail(l, e, "fill keys");
            }
        }
        e = traced(l, 0, s, [&] { return launch_full_search(l->geo.bit_depth, l->geo.ctu_size, fb, s); });
        if (e != cudaSuccess) {
            l->keys_dirty = true;
            return cuda_fail(l, e, "full search launch");
        }
        if (!fuse) {
            e = traced(l, 1, s, [&] { return launch_decide(l->geo.bit_depth, l->geo.ctu_size, db, s); });
            if (e != cudaSuccess) {
                l->keys_dirty = true;
                return cuda_fail(l, e, "decide launch");
            }
        }
    }
    l->keys_dirty = false;  // every search above left its keys at ~0
    if (l->mv_predictor) {
        const ladder_status st = launch_mvp(l, jobs, n, 0, s);
        if (st != LADDER_OK) return st;
    }
    for (int k = 0; k < n; ++k) jobs[k].slot->rungs[jobs[k].rung].analysed = 1;
    return LADDER_OK;
}

// Dependent analyses of one tier (no job's parent among them) in batched
// launches of at most kMaxDepItems jobs: rules + task lists, search,
// decisions.
ladder_status launch_dependent_tier(ladder_t *l, const Job *jobs, int n, cudaStream_t s)
{
    // the task lists come in sets: the stream's own set, else a fresh one,
    // else the least recently used, whose last batch this one waits for (not
    // inside a graph capture: a captured batch is one ordered stream)
    int pick = -1;
    for (int k = 0; k < kDepSets && pick < 0; ++k)
        if (l->dep[k].recorded && l->dep[k].stream == s) pick = k;
    for (int k = 0; k < kDepSets && pick < 0; ++k)
        if (!l->dep[k].recorded) pick = k;
    if (pick < 0) {
        pick = 0;
        for (int k = 1; k < kDepSets; ++k)
            if (l->dep[k].last_use < l->dep[pick].last_use) pick = k;
    }
    DepSet &ds = l->dep[pick];
    ds.last_use = ++l->dep_clock;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    const bool chain = cap == cudaStreamCaptureStatusNone;
    if (chain && ds.recorded && ds.stream != s) {  // same stream: ordered already
        const cudaError_t e = cudaStreamWaitEvent(s, ds.done, 0);
        if (e != cudaSuccess) return cuda_fail(l, e, "dependent ordering");
    }
    for (int j0 = 0; j0 < n; j0 += kMaxDepItems) {
        const int m = std::min(kMaxDepItems, n - j0);
        DependentBatch b{};
        b.n = m;
        b.r = l->geo.dep_refine_range;
        b.range = l->tune_dep_range;
        b.band = l->tune_dep_band;
        b.ctas_per_sm = l->tune_dep_ctas;
        b.staged = l->tune_dep_staged;
        b.inherit = l->tune_dep_inherit;
        b.evals = l->d_evals;
        b.satd_mode = l->geo.satd_mode;
        b.depth_lo = l->geo.dep_depth_lo;
        b.depth_hi = l->geo.dep_depth_hi;
        b.use_ref_mv = l->geo.dep_use_ref_mv;
        b.status = l->d_status;
        b.counts = ds.counts;
        b.one = 1;
        for (int c = 0; c < kSizeClasses; ++c) {
            b.tasks[c] = ds.tasks[c];
            b.pos[c] = ds.pos[c];
            b.sums[c] = ds.sums[c];
            b.up[c] = ds.up[c];
            b.cap[c] = l->task_cap[c];
        }
        for (int r = 0; r < l->geo.n_rungs; ++r) b.rung[r] = l->info[r];
        int total = 0;
        for (int k = 0; k < m; ++k) {
            const Job &jb = jobs[j0 + k];
            const RungGeom &g = l->info[jb.rung].g;
            const int par = l->parent[jb.rung];
            b.item[k] = DependentItem{jb.cur, jb.ref, jb.pitch, jb.slot->rungs[jb.rung].block,
                                      jb.slot->rungs[par].block, jb.rung, par, jb.qp, total};
            total += g.ctu_cols * g.ctu_rows;
        }
        b.total_ctas = total;
        // the counters rest at zero (each batch's decision kernel resets them)
        // unless a launch of an earlier batch failed
        cudaError_t e = cudaSuccess;
        if (ds.counts_dirty) {
            e = cudaMemsetAsync(ds.counts, 0, kDepCounters * sizeof(unsigned int), s);
            if (e != cudaSuccess) return cuda_fail(l, e, "task counters");
        }
        ds.counts_dirty = true;
        e = traced(l, 4, s, [&] { return launch_dependent_rules(l->geo.ctu_size, b, s); });
        if (e == cudaSuccess) e = traced(l, 2, s, [&] { return launch_dependent_search(l->geo.bit_depth, b, s); });
        if (e == cudaSuccess)
            e = traced(l, 5, s, [&] { return launch_dependent_decide(l->geo.bit_depth, l->geo.ctu_size, b, s); });
        if (e != cudaSuccess) {
            l->keys_dirty = true;
            return cuda_fail(l, e, "dependent launch");
        }
        ds.counts_dirty = false;
    }
    if (chain) {
        const cudaError_t e = cudaEventRecord(ds.done, s);
        if (e != cudaSuccess) return cuda_fail(l, e, "dependent ordering");
        ds.recorded = true;
        ds.stream = s;
    }
    if (l->mv_predictor) {  // before the next tier reads these leaf maps
        const ladder_status st = launch_mvp(l, jobs, n, 1, s);
        if (st != LADDER_OK) return st;
    }
    for (int k = 0; k < n; ++k) jobs[k].slot->rungs[jobs[k].rung].analysed = 2;
    return LADDER_OK;
}

// Dependent analyses, tier by tier along the parents (a cascaded chain
// refines a dependent rung's decisions at the next tier): each tier's
// launches follow the previous tier's on the stream.
ladder_status launch_dependents(ladder_t *l, const Job *jobs, int n, cudaStream_t s)
{
    int top = 0;
    for (int k = 0; k < n; ++k) top = std::max(top, l->tier[jobs[k].rung]);
    if (top <= 1) return launch_dependent_tier(l, jobs, n, s);
    std::vector<Job> tier_jobs;
    for (int t = 1; t <= top; ++t) {
        tier_jobs.clear();
        for (int k = 0; k < n; ++k)
            if (l->tier[jobs[k].rung] == t) tier_jobs.push_back(jobs[k]);
        if (tier_jobs.empty()) continue;
        const ladder_status st = launch_dependent_tier(l, tier_jobs.data(), static_cast<int>(tier_jobs.size()), s);
        if (st != LADDER_OK) return st;
    }
    return LADDER_OK;
}

}  // namespace

extern "C" {

const char *ladder_version(void)
{
    return LADDER_BOUNDS_CHECK ? "ladder 0.3 (sm_103a, bounds-checked debug build)" : "ladder 0.3 (sm_103a)";
}

ladder_status ladder_init(const ladder_geometry *geometry, void *cuda_stream, ladder_t **out)
{
    TraceRange trace("ladder_init");
    if (!out) return LADDER_E_INVAL;
    *out = nullptr;
    ladder_status st = validate_geometry(geometry);
    if (st != LADDER_OK) return st;
    ladder_t *l = new (std::nothrow) ladder();
    if (!l) return LADDER_E_NOMEM;
    l->geo = *geometry;
    l->rungs.assign(geometry->rungs, geometry->rungs + geometry->n_rungs);
    l->geo.rungs = l->rungs.data();
    size_t per_slot = 0;
    for (const auto &r : l->rungs) {
        RungInfo ri{};
        ri.g = make_geom(r.width, r.height, geometry->ctu_size);
        per_slot += layout(ri.g, ri.off);
        l->info.push_back(ri);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (prepare_kernels(geometry->bit_depth, geometry->ctu_size, geometry->ref_search_range,
                        geometry->dep_refine_range) != cudaSuccess) {
        cudaGetLastError();
        delete l;
        return LADDER_E_CUDA;
    }
    l->fs_ctas_per_sm = full_search_ctas_per_sm(geometry->bit_depth, geometry->ctu_size, geometry->ref_search_range);

    // dependent task lists: room for every CU of every size class of every
    // dependent rung of every frame slot (a launch never holds more)
    size_t dep_ctus = 0;
    for (int r = 0; r < geometry->n_rungs; ++r)
        if (r != geometry->ref_rung)
            dep_ctus += static_cast<size_t>(l->info[r].g.ctu_cols) * l->info[r].g.ctu_rows;
    const size_t kr2 = static_cast<size_t>(2 * geometry->dep_refine_range + 1) * (2 * geometry->dep_refine_range + 1);
    size_t task_bytes = 0;
    for (int c = 0; c < kSizeClasses; ++c) {
        const int S = 8 << c;
        const size_t per_ctu = S <= geometry->ctu_size ? static_cast<size_t>(geometry->ctu_size / S) *
                                                             (geometry->ctu_size / S)
                                                       : 0;
        const size_t cap = dep_ctus * per_ctu * geometry->max_frames;
        l->task_cap[c] = static_cast<unsigned int>(std::min<size_t>(cap, 0xffffffffu));
        task_bytes += kDepSets * (align_up(cap * 8, 256) + align_up(cap * 4, 256));
        if (c >= kFirstSummedClass) task_bytes += kDepSets * align_up(cap * kr2 * 4, 256);
        if (c >= kFirstUpClass && c < kSizeClasses - 1) task_bytes += kDepSets * align_up(cap * 4, 256);
    }
    const size_t fixed = 256 + task_bytes;
    l->arena_bytes = fixed + per_slot * geometry->max_frames;
    cudaError_t e = cudaMalloc(&l->arena, l->arena_bytes);
    if (e != cudaSuccess) {
        delete l;
        cudaGetLastError();
        return LADDER_E_NOMEM;
    }
    char *base = static_cast<char *>(l->arena);
    l->d_status = reinterpret_cast<int *>(base);
    l->d_evals = reinterpret_cast<unsigned long long *>(base + 8);
    static_assert(64 + kDepSets * 64 <= 256 && kDepCounters * sizeof(unsigned int) <= 64,
                  "counters inside the arena header");
    {
        char *tp = base + 256;
        for (int k = 0; k < kDepSets; ++k) {
            DepSet &ds = l->dep[k];
            ds.counts = reinterpret_cast<unsigned int *>(base + 64 + 64 * k);
            for (int c = 0; c < kSizeClasses; ++c) {
                ds.tasks[c] = reinterpret_cast<unsigned long long *>(tp);
                tp += align_up(static_cast<size_t>(l->task_cap[c]) * 8, 256);
                ds.pos[c] = reinterpret_cast<unsigned int *>(tp);
                tp += align_up(static_cast<size_t>(l->task_cap[c]) * 4, 256);
                if (c >= kFirstSummedClass) {
                    ds.sums[c] = reinterpret_cast<unsigned int *>(tp);
                    tp += align_up(static_cast<size_t>(l->task_cap[c]) * kr2 * 4, 256);
                }
                if (c >= kFirstUpClass && c < kSizeClasses - 1) {
                    ds.up[c] = reinterpret_cast<unsigned int *>(tp);
                    tp += align_up(static_cast<size_t>(l->task_cap[c]) * 4, 256);
                }
            }
        }
    }
    char *p = base + fixed;
    l->parent.assign(geometry->n_rungs, geometry->ref_rung);
    l->parent[geometry->ref_rung] = -1;
    l->tier.assign(geometry->n_rungs, 1);
    l->tier[geometry->ref_rung] = 0;
    l->slots.resize(geometry->max_frames);
    for (auto &sl : l->slots) {
        sl.used = 0;
        sl.frame_id = 0;
        sl.ref_done = 0;
        sl.rungs.resize(l->info.size());
        for (size_t r = 0; r < l->info.size(); ++r) {
            DecOffsets o;
            sl.rungs[r].block = p;
            sl.rungs[r].analysed = 0;
            p += layout(l->info[r].g, o);
        }
    }
    for (const auto &ri : l->info)
        l->host_stage_bytes = std::max(l->host_stage_bytes, static_cast<size_t>(ri.off.dec_bytes));
    if (cudaMallocHost(&l->host_stage, l->host_stage_bytes) != cudaSuccess) {
        cudaFree(l->arena);
        delete l;
        cudaGetLastError();
        return LADDER_E_NOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    e = cudaMemsetAsync(l->arena, 0, l->arena_bytes, s);  // counters and per-CTU done counts at zero
    for (auto &ds : l->dep)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ds.done, cudaEventDisableTiming);
    // every key of every slot to ~0 (searches keep that at rest)
    if (e == cudaSuccess) {
        FillBatch fill{};
        for (auto &sl : l->slots)
            for (size_t r = 0; r < l->info.size() && e == cudaSuccess; ++r) {
                const RungInfo &ri = l->info[r];
                fill.item[fill.n++] = FillItem{reinterpret_cast<unsigned long long *>(sl.rungs[r].block + ri.off.keys),
                                               static_cast<long>(ri.g.ctu_cols) * ri.g.ctu_rows * keys_per_ctu(ri.g.dmax)};
                if (fill.n == kMaxItems) {
                    e = launch_fill_keys(fill, s);
                    fill.n = 0;
                }
            }
        if (e == cudaSuccess && fill.n > 0) e = launch_fill_keys(fill, s);
    }
    if (e == cudaSuccess) {
        e = cudaStreamSynchronize(s);
        l->keys_dirty = e != cudaSuccess;
    }
    if (e != cudaSuccess) {
        for (auto &ds : l->dep)
            if (ds.done) cudaEventDestroy(ds.done);
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
    TraceRange trace("analyze_independent");
    if (!l) return LADDER_E_INVAL;
    ladder_status st = check_planes(l, rung, cur, ref, pitch_bytes, qp);
    if (st != LADDER_OK) return st;
    Slot *slot = claim_slot(l, frame_id);
    if (!slot) return fail(l, LADDER_E_BUSY, "no free frame slot for frame %d", frame_id);
    Job job{slot, rung, cur, ref, pitch_bytes, qp};
    st = launch_independent(l, &job, 1, static_cast<cudaStream_t>(cuda_stream));
    if (st == LADDER_OK && rung == l->geo.ref_rung) slot->ref_done = 1;
    return marked(l, static_cast<cudaStream_t>(cuda_stream), st);
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
    TraceRange trace("analyze_dependents");
    if (!l) return LADDER_E_INVAL;
    if (n < 1 || n > kMaxRungs || !rungs || !cur || !ref || !pitch_bytes)
        return fail(l, LADDER_E_INVAL, "dependent batch of %d rungs (1..%d)", n, kMaxRungs);
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
    // each rung's parent: analysed for this frame, or in this call
    for (int k = 0; k < n; ++k) {
        const int p = l->parent[rungs[k]];
        bool ok = slot->rungs[p].analysed != 0;
        for (int j = 0; j < n && !ok; ++j) ok = rungs[j] == p;
        if (!ok) return fail(l, LADDER_E_NOREF, "rung %d: its parent rung %d has no analysis of frame %d", rungs[k], p, frame_id);
    }
    std::vector<Job> jobs;
    for (int k = 0; k < n; ++k) jobs.push_back(Job{slot, rungs[k], cur[k], ref[k], pitch_bytes[k], qp});
    return marked(l, static_cast<cudaStream_t>(cuda_stream),
                  launch_dependents(l, jobs.data(), n, static_cast<cudaStream_t>(cuda_stream)));
}

ladder_status analyze_dependent(ladder_t *l, int rung, int frame_id, const void *cur, const void *ref,
                                long pitch_bytes, int qp, void *cuda_stream)
{
    return analyze_dependents(l, frame_id, 1, &rung, &cur, &ref, &pitch_bytes, qp, cuda_stream);
}

ladder_status ladder_analyze_batch(ladder_t *l, const ladder_request *reqs, int n, void *cuda_stream)
{
    TraceRange trace("ladder_analyze_batch");
    if (!l) return LADDER_E_INVAL;
    const int nd = l->geo.n_rungs - 1;
    if (!reqs || n < 1 || n > kMaxItems || n * nd > kMaxDepItems)
        return fail(l, LADDER_E_INVAL, "batch of %d frames (1..%d, and frames x dependent rungs <= %d)", n,
                    kMaxItems, kMaxDepItems);
    for (int k = 0; k < n; ++k) {
        if (!reqs[k].cur || !reqs[k].ref || !reqs[k].pitch_bytes)
            return fail(l, LADDER_E_INVAL, "request %d has null plane arrays", k);
        for (int r = 0; r < l->geo.n_rungs; ++r) {
            ladder_status st =
                check_planes(l, r, reqs[k].cur[r], reqs[k].ref[r], reqs[k].pitch_bytes[r], reqs[k].qp);
            if (st != LADDER_OK) return st;
        }
        for (int j = 0; j < k; ++j)
            if (reqs[j].frame_id == reqs[k].frame_id)
                return fail(l, LADDER_E_INVAL, "frame %d appears twice in the batch", reqs[k].frame_id);
    }
    int free_slots = 0, needed = 0;
    for (auto &sl : l->slots) free_slots += !sl.used;
    for (int k = 0; k < n; ++k) needed += find_slot(l, reqs[k].frame_id) == nullptr;
    if (needed > free_slots)
        return fail(l, LADDER_E_BUSY, "batch needs %d free frame slots, %d free", needed, free_slots);
    std::vector<Slot *> slots(n);
    for (int k = 0; k < n; ++k) slots[k] = claim_slot(l, reqs[k].frame_id);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int rr = l->geo.ref_rung;
    std::vector<Job> ij, dj;
    for (int k = 0; k < n; ++k) {
        ij.push_back(Job{slots[k], rr, reqs[k].cur[rr], reqs[k].ref[rr], reqs[k].pitch_bytes[rr], reqs[k].qp});
        for (int r = 0; r < l->geo.n_rungs; ++r)
            if (r != rr)
                dj.push_back(Job{slots[k], r, reqs[k].cur[r], reqs[k].ref[r], reqs[k].pitch_bytes[r], reqs[k].qp});
    }
    ladder_status st = launch_independent(l, ij.data(), n, s);
    if (st != LADDER_OK) return st;
    for (int k = 0; k < n; ++k) slots[k]->ref_done = 1;
    if (!dj.empty()) st = launch_dependents(l, dj.data(), static_cast<int>(dj.size()), s);
    return marked(l, s, st);
}

ladder_status ladder_analyze_batch_independent(ladder_t *l, const ladder_request *reqs, int n, void *cuda_stream)
{
    TraceRange trace("ladder_analyze_batch_independent");
    if (!l) return LADDER_E_INVAL;
    if (!reqs || n < 1 || n > kMaxItems) return fail(l, LADDER_E_INVAL, "batch of %d frames (1..%d)", n, kMaxItems);
    for (int k = 0; k < n; ++k) {
        if (!reqs[k].cur || !reqs[k].ref || !reqs[k].pitch_bytes)
            return fail(l, LADDER_E_INVAL, "request %d has null plane arrays", k);
        for (int r = 0; r < l->geo.n_rungs; ++r) {
            ladder_status st =
                check_planes(l, r, reqs[k].cur[r], reqs[k].ref[r], reqs[k].pitch_bytes[r], reqs[k].qp);
            if (st != LADDER_OK) return st;
        }
        for (int j = 0; j < k; ++j)
            if (reqs[j].frame_id == reqs[k].frame_id)
                return fail(l, LADDER_E_INVAL, "frame %d appears twice in the batch", reqs[k].frame_id);
    }
    int free_slots = 0, needed = 0;
    for (auto &sl : l->slots) free_slots += !sl.used;
    for (int k = 0; k < n; ++k) needed += find_slot(l, reqs[k].frame_id) == nullptr;
    if (needed > free_slots)
        return fail(l, LADDER_E_BUSY, "batch needs %d free frame slots, %d free", needed, free_slots);
    std::vector<Job> jobs;
    std::vector<Slot *> slots(n);
    for (int k = 0; k < n; ++k) {
        slots[k] = claim_slot(l, reqs[k].frame_id);
        for (int r = 0; r < l->geo.n_rungs; ++r)
            jobs.push_back(Job{slots[k], r, reqs[k].cur[r], reqs[k].ref[r], reqs[k].pitch_bytes[r], reqs[k].qp});
    }
    ladder_status st = launch_independent(l, jobs.data(), static_cast<int>(jobs.size()),
                                          static_cast<cudaStream_t>(cuda_stream));
    if (st == LADDER_OK)
        for (int k = 0; k < n; ++k) slots[k]->ref_done = 1;
    return marked(l, static_cast<cudaStream_t>(cuda_stream), st);
}

ladder_status ladder_analyze_jobs(ladder_t *l, const ladder_job *jobs, int n, void *cuda_stream)
{
    TraceRange trace("ladder_analyze_jobs");
    if (!l) return LADDER_E_INVAL;
    if (!jobs || n < 0) return fail(l, LADDER_E_INVAL, "bad job list");
    if (n == 0) return LADDER_OK;
    std::vector<Job> ij, dj;
    // validate everything before touching any slot
    for (int k = 0; k < n; ++k) {
        const ladder_job &jb = jobs[k];
        ladder_status st = check_planes(l, jb.rung, jb.cur, jb.ref, jb.pitch_bytes, jb.qp);
        if (st != LADDER_OK) return st;
        if (jb.kind != 0 && jb.kind != 1) return fail(l, LADDER_E_INVAL, "job %d: kind %d", k, jb.kind);
        if (jb.kind == 1 && jb.rung == l->geo.ref_rung)
            return fail(l, LADDER_E_INVAL, "job %d: the reference rung cannot be dependent", k);
        for (int j = 0; j < k; ++j)
            if (jobs[j].frame_id == jb.frame_id && jobs[j].rung == jb.rung)
                return fail(l, LADDER_E_INVAL, "job %d repeats (frame %d, rung %d)", k, jb.frame_id, jb.rung);
    }
    int free_slots = 0;
    for (auto &sl : l->slots) free_slots += !sl.used;
    std::vector<int> new_frames;
    for (int k = 0; k < n; ++k)
        if (!find_slot(l, jobs[k].frame_id) &&
            std::find(new_frames.begin(), new_frames.end(), jobs[k].frame_id) == new_frames.end())
            new_frames.push_back(jobs[k].frame_id);
    if (static_cast<int>(new_frames.size()) > free_slots)
        return fail(l, LADDER_E_BUSY, "jobs need %zu free frame slots, %d free", new_frames.size(), free_slots);
    // a dependent needs its parent rung's decisions of its frame: already
    // resident, or a job of this same call
    for (int k = 0; k < n; ++k) {
        if (jobs[k].kind != 1) continue;
        const int p = l->parent[jobs[k].rung];
        Slot *sl = find_slot(l, jobs[k].frame_id);
        bool ok = sl && sl->rungs[p].analysed != 0;
        for (int j = 0; j < n && !ok; ++j) ok = jobs[j].rung == p && jobs[j].frame_id == jobs[k].frame_id;
        if (!ok)
            return fail(l, LADDER_E_NOREF, "job %d: parent rung %d has no analysis of frame %d", k, p, jobs[k].frame_id);
    }
    for (int k = 0; k < n; ++k) {
        const ladder_job &jb = jobs[k];
        Slot *sl = claim_slot(l, jb.frame_id);
        (jb.kind == 0 ? ij : dj).push_back(Job{sl, jb.rung, jb.cur, jb.ref, jb.pitch_bytes, jb.qp});
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!ij.empty()) {
        ladder_status st = launch_independent(l, ij.data(), static_cast<int>(ij.size()), s);
        if (st != LADDER_OK) return st;
        for (const Job &jb : ij)
            if (jb.rung == l->geo.ref_rung) jb.slot->ref_done = 1;
    }
    if (!dj.empty()) return marked(l, s, launch_dependents(l, dj.data(), static_cast<int>(dj.size()), s));
    return marked(l, s, LADDER_OK);
}

ladder_status ladder_capture_batch(ladder_t *l, const ladder_request *reqs, int n, void *cuda_stream,
                                   ladder_graph_t **out)
{
    TraceRange trace("ladder_capture_batch");
    if (!l || !out) return LADDER_E_INVAL;
    *out = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!s) return fail(l, LADDER_E_INVAL, "capture needs a non-default stream");
    const int prof = l->prof_on;
    l->prof_on = 0;  // no event records inside the graph
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        l->prof_on = prof;
        return cuda_fail(l, e, "begin capture");
    }
    ladder_status st = ladder_analyze_batch(l, reqs, n, cuda_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    l->prof_on = prof;
    if (st != LADDER_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(l, e, "end capture");
    ladder_graph_t *g = new (std::nothrow) ladder_graph();
    if (!g) {
        cudaGraphDestroy(graph);
        return LADDER_E_NOMEM;
    }
    g->l = l;
    g->graph = graph;
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete g;
        return cuda_fail(l, e, "graph instantiate");
    }
    *out = g;
    return LADDER_OK;
}

ladder_status ladder_graph_launch(ladder_graph_t *g, void *cuda_stream)
{
    TraceRange trace("ladder_graph_launch");
    if (!g || !g->exec) return LADDER_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGraphLaunch(g->exec, s) != cudaSuccess) return LADDER_E_CUDA;
    if (g->l) mark_stream(g->l, s);
    return LADDER_OK;
}

void ladder_graph_destroy(ladder_graph_t *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}


ladder_status ladder_grid(const ladder_t *l, int rung, int *dims, int *n_depths)
{
    if (!l || !dims || rung < 0 || rung >= l->geo.n_rungs) return LADDER_E_INVAL;
    const RungGeom &g = l->info[rung].g;
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
    TraceRange trace("ladder_sync");
    if (!l) return LADDER_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, l->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(l, e, "sync");
    if (status != 0) {
        cudaMemsetAsync(l->d_status, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        return device_status_error(l, status);
    }
    return LADDER_OK;
}

ladder_status ladder_set_parents(ladder_t *l, const int *parent)
{
    if (!l || !parent) return LADDER_E_INVAL;
    const int n = l->geo.n_rungs, rr = l->geo.ref_rung;
    std::vector<int> tier(n, -1);
    for (int r = 0; r < n; ++r) {
        if (r == rr) {
            if (parent[r] != -1) return fail(l, LADDER_E_INVAL, "the reference rung %d takes parent -1", rr);
            continue;
        }
        if (parent[r] < 0 || parent[r] >= n || parent[r] == r)
            return fail(l, LADDER_E_INVAL, "rung %d: parent %d", r, parent[r]);
    }
    // tiers: steps to the reference rung; a cycle never reaches it
    for (int r = 0; r < n; ++r) {
        int t = 0, x = r;
        while (x != rr && t <= n) {
            x = parent[x];
            ++t;
        }
        if (t > n) return fail(l, LADDER_E_INVAL, "the parents of rung %d form a cycle", r);
        tier[r] = t;
    }
    l->parent.assign(parent, parent + n);
    l->tier = tier;
    return LADDER_OK;
}

ladder_status ladder_set_mv_predictor(ladder_t *l, int mode)
{
    if (!l) return LADDER_E_INVAL;
    if (mode != 0 && mode != 1) return fail(l, LADDER_E_INVAL, "mv predictor mode %d: 0 or 1", mode);
    l->mv_predictor = mode;
    return LADDER_OK;
}

ladder_status ladder_decide_qps(ladder_t *l, int rung, int frame_id, int n, const int *qps,
                                const ladder_qp_decisions *out, void *cuda_stream)
{
    TraceRange trace("ladder_decide_qps");
    if (!l || !qps || !out) return LADDER_E_INVAL;
    if (rung < 0 || rung >= l->geo.n_rungs) return fail(l, LADDER_E_INVAL, "rung %d out of range", rung);
    if (n < 1 || n > kMaxQps) return fail(l, LADDER_E_INVAL, "%d QPs (1..%d)", n, kMaxQps);
    Slot *slot = find_slot(l, frame_id);
    if (!slot || !slot->rungs[rung].analysed)
        return fail(l, LADDER_E_STATE, "rung %d of frame %d has not been analysed", rung, frame_id);
    const RungGeom &g = l->info[rung].g;
    QpBatch b{};
    b.n_qps = n;
    b.g = g;
    b.off = l->info[rung].off;
    b.block = slot->rungs[rung].block;
    b.dependent = slot->rungs[rung].analysed == 2;
    for (int k = 0; k < n; ++k) {
        if (qps[k] < 0 || qps[k] > 51) return fail(l, LADDER_E_INVAL, "qp %d outside 0..51", qps[k]);
        b.qp[k] = qps[k];
        const ladder_qp_decisions &o = out[k];
        if (!o.leaf_depth || !o.leaf_mvx || !o.leaf_mvy)
            return fail(l, LADDER_E_INVAL, "qp %d: leaf arrays missing", qps[k]);
        for (int d = 0; d <= g.dmax; ++d) {
            if (!o.cost[d] || !o.best[d] || !o.split[d])
                return fail(l, LADDER_E_INVAL, "qp %d: depth %d arrays missing", qps[k], d);
            b.out[k].cost[d] = o.cost[d];
            b.out[k].best[d] = o.best[d];
            b.out[k].split[d] = o.split[d];
        }
        b.out[k].leaf_depth = o.leaf_depth;
        b.out[k].leaf_mvx = o.leaf_mvx;
        b.out[k].leaf_mvy = o.leaf_mvy;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (l->mv_predictor) {
        // spatial predictor: one wavefront launch per QP, in order on the
        // stream (each takes a new generation of the block's hand-off area)
        if (l->mvp_capacity <= 0) l->mvp_capacity = decide_mvp_capacity(l->geo.ctu_size, l->sm_count);
        if (g.ctu_rows > l->mvp_capacity)
            return fail(l, LADDER_E_INVAL, "%d CTU rows exceed the %d resident wavefront CTAs", g.ctu_rows,
                        l->mvp_capacity);
        auto *mb = new (std::nothrow) MvpBatch{};
        if (!mb) return fail(l, LADDER_E_NOMEM, "wavefront batch table");
        for (int r = 0; r < l->geo.n_rungs; ++r) mb->rung[r] = l->info[r];
        mb->status = l->d_status;
        mb->spin = l->dbg_wait_polls > 0 ? l->dbg_wait_polls : kMvpSpinDefault;
        mb->lost_handoff = l->dbg_lost_handoff;
        mb->n = 1;
        mb->use_out = 1;
        for (int k = 0; k < n; ++k) {
            mb->item[0] = MvpItem{slot->rungs[rung].block, rung, qps[k], b.dependent, 0};
            mb->out = b.out[k];
            const cudaError_t e =
                traced(l, 8, s, [&] { return launch_decide_mvp(l->geo.ctu_size, *mb, g.ctu_rows, s); });
            if (e != cudaSuccess) {
                delete mb;
                return cuda_fail(l, e, "further-QP decisions with the spatial predictor");
            }
        }
        delete mb;
        return marked(l, s, LADDER_OK);
    }
    const cudaError_t e = traced(l, 6, s, [&] { return launch_decide_qps(l->geo.ctu_size, b, s); });
    if (e != cudaSuccess) return cuda_fail(l, e, "further-QP decisions");
    return marked(l, s, LADDER_OK);
}

ladder_status fetch_decisions(ladder_t *l, int rung, int frame_id, ladder_decisions *out, void *cuda_stream)
{
    TraceRange trace("fetch_decisions");
    if (!l || !out) return LADDER_E_INVAL;
    if (rung < 0 || rung >= l->geo.n_rungs) return fail(l, LADDER_E_INVAL, "rung %d out of range", rung);
    Slot *slot = find_slot(l, frame_id);
    if (!slot || !slot->rungs[rung].analysed)
        return fail(l, LADDER_E_STATE, "rung %d of frame %d has not been analysed", rung, frame_id);
    const RungGeom &g = l->info[rung].g;
    const DecOffsets &o = l->info[rung].off;
    const char *block = slot->rungs[rung].block;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // one copy of the rung's whole decision block into pinned memory, then
    // host copies into the caller's arrays
    cudaError_t e =
        cudaMemcpyAsync(l->host_stage, block, static_cast<size_t>(o.dec_bytes), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(l, e, "fetch copy");
    auto copy = [&](void *dst, long off, size_t bytes) {
        if (dst) memcpy(dst, l->host_stage + off, bytes);
    };
    for (int d = 0; d <= g.dmax; ++d) {
        const size_t n = static_cast<size_t>(g.cols[d]) * g.rows[d];
        copy(out->mvx[d], o.mvx[d], n * 2);
        copy(out->mvy[d], o.mvy[d], n * 2);
        copy(out->sad[d], o.sad[d], n * 4);
        copy(out->satd[d], o.satd[d], n * 4);
        copy(out->cost[d], o.cost[d], n * 4);
        copy(out->best[d], o.best[d], n * 4);
        copy(out->split[d], o.split[d], n);
        copy(out->evaluated[d], o.evaluated[d], n);
    }
    const size_t n8 = static_cast<size_t>(g.cols8) * g.rows8;
    copy(out->leaf_depth, o.leaf_depth, n8);
    copy(out->leaf_mvx, o.leaf_mvx, n8 * 2);
    copy(out->leaf_mvy, o.leaf_mvy, n8 * 2);
    return ladder_sync(l, cuda_stream);
}

ladder_status ladder_load_reference(ladder_t *l, int frame_id, const ladder_decisions *in, void *cuda_stream)
{
    TraceRange trace("ladder_load_reference");
    if (!l || !in) return LADDER_E_INVAL;
    const int rung = l->geo.ref_rung;
    const RungGeom &g = l->info[rung].g;
    const DecOffsets &o = l->info[rung].off;
    for (int d = 0; d <= g.dmax; ++d)
        if (!in->mvx[d] || !in->mvy[d] || !in->sad[d] || !in->satd[d] || !in->cost[d] || !in->best[d] ||
            !in->split[d] || !in->evaluated[d])
            return fail(l, LADDER_E_INVAL, "depth %d arrays missing", d);
    if (!in->leaf_depth || !in->leaf_mvx || !in->leaf_mvy) return fail(l, LADDER_E_INVAL, "leaf arrays missing");
    Slot *slot = claim_slot(l, frame_id);
    if (!slot) return fail(l, LADDER_E_BUSY, "no free frame slot for frame %d", frame_id);
    // the caller's arrays into the pinned staging buffer in the block's
    // layout, then one copy into the frame's reference-rung block
    auto put = [&](long off, const void *src, size_t bytes) { memcpy(l->host_stage + off, src, bytes); };
    for (int d = 0; d <= g.dmax; ++d) {
        const size_t n = static_cast<size_t>(g.cols[d]) * g.rows[d];
        put(o.mvx[d], in->mvx[d], n * 2);
        put(o.mvy[d], in->mvy[d], n * 2);
        put(o.sad[d], in->sad[d], n * 4);
        put(o.satd[d], in->satd[d], n * 4);
        put(o.cost[d], in->cost[d], n * 4);
        put(o.best[d], in->best[d], n * 4);
        put(o.split[d], in->split[d], n);
        put(o.evaluated[d], in->evaluated[d], n);
    }
    const size_t n8 = static_cast<size_t>(g.cols8) * g.rows8;
    put(o.leaf_depth, in->leaf_depth, n8);
    put(o.leaf_mvx, in->leaf_mvx, n8 * 2);
    put(o.leaf_mvy, in->leaf_mvy, n8 * 2);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemcpyAsync(slot->rungs[rung].block, l->host_stage, static_cast<size_t>(o.dec_bytes),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the staging buffer is free again
    if (e != cudaSuccess) return cuda_fail(l, e, "reference load copy");
    slot->rungs[rung].analysed = 1;
    slot->ref_done = 1;
    return LADDER_OK;
}

long ladder_subpel_workspace_bytes(const ladder_t *l, int rung)
{
    if (!l || rung < 0 || rung >= l->geo.n_rungs) return 0;
    const RungGeom &g = l->info[rung].g;
    // the 16 phase planes, then the SATD table of the refinement with the
    // spatial predictor (always counted: the mode may change between calls)
    return subpel_workspace_layout(l->geo.bit_depth, g.W, g.H, nullptr, nullptr) +
           subpel_table_bytes(g.ctu_cols, g.ctu_rows, g.dmax);
}

namespace {

// Validates one refinement job and fills its launch item (CTA ranges unset).
ladder_status subpel_item(ladder_t *l, const ladder_subpel_job &j, SubpelItem &it)
{
    ladder_status st = check_planes(l, j.rung, j.cur, j.ref, j.pitch_bytes, j.qp);
    if (st != LADDER_OK) return st;
    const ladder_subpel_decisions *out = j.out;
    if (!out) return fail(l, LADDER_E_INVAL, "null output arrays");
    const long need = ladder_subpel_workspace_bytes(l, j.rung);
    if (!j.workspace || (reinterpret_cast<uintptr_t>(j.workspace) & 255) || j.workspace_bytes < need)
        return fail(l, LADDER_E_INVAL, "workspace must be 256-byte aligned and hold %ld bytes (got %ld)", need,
                    j.workspace_bytes);
    Slot *slot = find_slot(l, j.frame_id);
    if (!slot || !slot->rungs[j.rung].analysed)
        return fail(l, LADDER_E_STATE, "rung %d of frame %d has not been analysed", j.rung, j.frame_id);
    const RungGeom &g = l->info[j.rung].g;
    it = SubpelItem{};
    it.rung = j.rung;
    it.g = g;
    it.off = l->info[j.rung].off;
    it.block = slot->rungs[j.rung].block;
    it.dependent = slot->rungs[j.rung].analysed == 2;
    it.qp = j.qp;
    it.cur = j.cur;
    it.ref = j.ref;
    it.pitch_bytes = j.pitch_bytes;
    it.planes = static_cast<char *>(j.workspace);
    const long planes_bytes = subpel_workspace_layout(l->geo.bit_depth, g.W, g.H, &it.plane_pitch, &it.plane_bytes);
    it.table = reinterpret_cast<int32_t *>(it.planes + planes_bytes);  // 256-byte aligned: planes_bytes is
    if (!out->leaf_depth || !out->leaf_qmvx || !out->leaf_qmvy)
        return fail(l, LADDER_E_INVAL, "leaf arrays missing");
    for (int d = 0; d <= g.dmax; ++d) {
        if (!out->qmvx[d] || !out->qmvy[d] || !out->satd[d] || !out->cost[d] || !out->best[d] || !out->split[d])
            return fail(l, LADDER_E_INVAL, "depth %d arrays missing", d);
        it.out.mvx[d] = out->qmvx[d];
        it.out.mvy[d] = out->qmvy[d];
        it.out.satd[d] = out->satd[d];
        it.out.cost[d] = out->cost[d];
        it.out.best[d] = out->best[d];
        it.out.split[d] = out->split[d];
    }
    it.out.leaf_depth = out->leaf_depth;
    it.out.leaf_mvx = out->leaf_qmvx;
    it.out.leaf_mvy = out->leaf_qmvy;
    return LADDER_OK;
}

// The refinement with the spatial predictor: the interpolation and every
// job's SATD table in one pair of launches, then cooperative wavefront
// launches of one CTA per CTU row, as many jobs per launch as fit on the
// device at once (rows wait on the row above).
ladder_status refine_subpel_mvp(ladder_t *l, const SubpelBatch &b, int ctas, int ictas, cudaStream_t s)
{
    if (l->subpel_mvp_capacity <= 0) l->subpel_mvp_capacity = subpel_mvp_capacity(l->geo.ctu_size, l->sm_count);
    for (int k = 0; k < b.n; ++k)
        if (b.item[k].g.ctu_rows > l->subpel_mvp_capacity)
            return fail(l, LADDER_E_INVAL, "%d CTU rows exceed the %d resident wavefront CTAs", b.item[k].g.ctu_rows,
                        l->subpel_mvp_capacity);
    cudaError_t e = traced(l, 7, s, [&] {
        return launch_subpel_table(l->geo.bit_depth, l->geo.ctu_size, b, ctas, ictas, s);
    });
    if (e != cudaSuccess) return cuda_fail(l, e, "quarter-pel SATD tables");
    auto *mb = new (std::nothrow) SubpelMvpBatch{};
    if (!mb) return fail(l, LADDER_E_NOMEM, "wavefront batch table");
    for (int r = 0; r < l->geo.n_rungs; ++r) mb->rung[r] = l->info[r];
    mb->status = l->d_status;
    mb->spin = l->dbg_wait_polls > 0 ? l->dbg_wait_polls : kMvpSpinDefault;
    mb->lost_handoff = l->dbg_lost_handoff;
    int k = 0;
    while (k < b.n) {
        int m = 0, rows = 0;
        while (k + m < b.n && m < kMaxSubpelItems) {
            const SubpelItem &it = b.item[k + m];
            if (m > 0 && rows + it.g.ctu_rows > l->subpel_mvp_capacity) break;
            mb->item[m] = SubpelMvpItem{const_cast<char *>(it.block), it.rung, it.qp, it.dependent, rows, it.table,
                                        it.out};
            rows += it.g.ctu_rows;
            ++m;
        }
        mb->n = m;
        e = traced(l, 7, s, [&] { return launch_subpel_mvp(l->geo.ctu_size, *mb, rows, s); });
        if (e != cudaSuccess) {
            delete mb;
            return cuda_fail(l, e, "quarter-pel refinement wavefront");
        }
        k += m;
    }
    delete mb;
    return LADDER_OK;
}

}  // namespace

ladder_status ladder_refine_subpel_batch(ladder_t *l, int n, const ladder_subpel_job *jobs, void *cuda_stream)
{
    TraceRange trace("ladder_refine_subpel_batch");
    if (!l || !jobs) return LADDER_E_INVAL;
    if (n < 1 || n > LADDER_MAX_SUBPEL_JOBS)
        return fail(l, LADDER_E_INVAL, "%d jobs: 1 .. %d per call", n, LADDER_MAX_SUBPEL_JOBS);
    static_assert(LADDER_MAX_SUBPEL_JOBS == kMaxSubpelItems, "job table size");
    static_assert(sizeof(SubpelBatch) <= 32000, "kernel parameter space");
    auto *b = new (std::nothrow) SubpelBatch{};
    if (!b) return fail(l, LADDER_E_NOMEM, "batch table");
    // independently analysed jobs (every depth evaluated: the longest CTAs) first
    int order[LADDER_MAX_SUBPEL_JOBS], m = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < n; ++k) {
            const Slot *slot = find_slot(l, jobs[k].frame_id);
            const bool indep = slot && jobs[k].rung >= 0 && jobs[k].rung < l->geo.n_rungs &&
                               slot->rungs[jobs[k].rung].analysed == 1;
            if (indep == (pass == 0)) order[m++] = k;
        }
    int ctas = 0, ictas = 0;
    for (int k = 0; k < n; ++k) {
        SubpelItem &it = b->item[k];
        const ladder_status st = subpel_item(l, jobs[order[k]], it);
        if (st != LADDER_OK) {
            delete b;
            return st;
        }
        int rows = 0;
        subpel_interp_tiles(it.g.W, it.g.H, &it.icols, &rows);
        it.cta_begin = ctas;
        it.icta_begin = ictas;
        ctas += it.g.ctu_cols * it.g.ctu_rows;
        ictas += it.icols * rows;
    }
    b->n = n;
    b->satd_mode = l->geo.satd_mode;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (l->mv_predictor) {
        const ladder_status st = refine_subpel_mvp(l, *b, ctas, ictas, s);
        delete b;
        return st == LADDER_OK ? marked(l, s, LADDER_OK) : st;
    }
    const cudaError_t e =
        traced(l, 7, s, [&] { return launch_subpel(l->geo.bit_depth, l->geo.ctu_size, *b, ctas, ictas, s); });
    delete b;
    if (e != cudaSuccess) return cuda_fail(l, e, "quarter-pel refinement");
    return marked(l, s, LADDER_OK);
}

ladder_status ladder_refine_subpel(ladder_t *l, int rung, int frame_id, const void *cur, const void *ref,
                                   long pitch_bytes, int qp, const ladder_subpel_decisions *out, void *workspace,
                                   long workspace_bytes, void *cuda_stream)
{
    const ladder_subpel_job j{frame_id, rung, qp, cur, ref, pitch_bytes, out, workspace, workspace_bytes};
    return ladder_refine_subpel_batch(l, 1, &j, cuda_stream);
}

long ladder_frame_bytes(const ladder_t *l)
{
    if (!l) return 0;
    long total = 0;
    for (int r = 0; r < l->geo.n_rungs; ++r) total += l->info[r].off.dec_bytes;
    return total;
}

ladder_status ladder_decision_offsets(const ladder_t *l, int rung, long *offsets)
{
    if (!l || !offsets) return LADDER_E_INVAL;
    if (rung < 0 || rung >= l->geo.n_rungs) return LADDER_E_INVAL;
    long base = 0;
    for (int r = 0; r < rung; ++r) base += l->info[r].off.dec_bytes;
    const DecOffsets &o = l->info[rung].off;
    for (int d = 0; d < kMaxDepths; ++d) {
        const bool has = d <= l->info[rung].g.dmax;
        const long f[8] = {o.mvx[d], o.mvy[d], o.sad[d], o.satd[d], o.cost[d], o.best[d], o.split[d], o.evaluated[d]};
        for (int k = 0; k < 8; ++k) offsets[8 * d + k] = has ? base + f[k] : -1;
    }
    offsets[32] = base + o.leaf_depth;
    offsets[33] = base + o.leaf_mvx;
    offsets[34] = base + o.leaf_mvy;
    return LADDER_OK;
}

ladder_status ladder_fetch_frame_async(ladder_t *l, int frame_id, void *host_dst, long bytes, void *cuda_stream)
{
    TraceRange trace("ladder_fetch_frame_async");
    if (!l || !host_dst) return LADDER_E_INVAL;
    if (bytes < ladder_frame_bytes(l)) return fail(l, LADDER_E_INVAL, "%ld bytes, the frame needs %ld", bytes, ladder_frame_bytes(l));
    Slot *slot = find_slot(l, frame_id);
    if (!slot) return fail(l, LADDER_E_STATE, "frame %d holds no slot", frame_id);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    char *dst = static_cast<char *>(host_dst);
    for (int r = 0; r < l->geo.n_rungs; ++r) {
        const long n = l->info[r].off.dec_bytes;
        const cudaError_t e = cudaMemcpyAsync(dst, slot->rungs[r].block, static_cast<size_t>(n), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(l, e, "frame fetch copy");
        dst += n;
    }
    return marked(l, s, LADDER_OK);
}

struct ladder_pipeline {
    ladder_t *l = nullptr;
    int depth = 0, base = 0;
    long in_bytes = 0, out_bytes = 0;
    std::vector<long> cur_off, ref_off, pitch;
    std::vector<char *> dev_in;
    std::vector<cudaStream_t> comp;  // one analysis stream per slot
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_comp, ev_out;
    std::vector<long> slot_ticket;  // the last ticket of each slot (-1: none yet)
    long next = 0;
    // per slot: the device status word as read back after the slot's last
    // frame (pinned), and whether it has been reported yet
    int *h_status = nullptr;
    std::vector<char> reported;
    int pending = 0;  // a non-zero status of a frame whose ticket was not waited for
};

namespace {

void pipeline_free(ladder_pipeline *p)
{
    if (!p) return;
    for (cudaStream_t s : p->comp)
        if (s) cudaStreamSynchronize(s);
    if (p->s_in) cudaStreamSynchronize(p->s_in);
    if (p->s_out) cudaStreamSynchronize(p->s_out);
    for (char *b : p->dev_in) cudaFree(b);
    if (p->h_status) cudaFreeHost(p->h_status);
    for (cudaStream_t s : p->comp)
        if (s) cudaStreamDestroy(s);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    for (auto *v : {&p->ev_in, &p->ev_comp, &p->ev_out})
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    delete p;
}

}  // namespace

ladder_status ladder_pipeline_create(ladder_t *l, int depth, int base_frame_id, long in_bytes, const long *cur_off,
                                     const long *ref_off, const long *pitch, ladder_pipeline_t **out)
{
    if (!l || !out || !cur_off || !ref_off || !pitch) return LADDER_E_INVAL;
    *out = nullptr;
    if (depth < 1 || depth > 8) return fail(l, LADDER_E_INVAL, "pipeline depth %d: 1 .. 8", depth);
    if (in_bytes <= 0) return fail(l, LADDER_E_INVAL, "input bytes %ld", in_bytes);
    const int ss = l->geo.bit_depth == 8 ? 1 : 2;
    for (int r = 0; r < l->geo.n_rungs; ++r) {
        const long w = l->rungs[r].width, h = l->rungs[r].height;
        if (pitch[r] < w * ss || (pitch[r] & 15))
            return fail(l, LADDER_E_INVAL, "rung %d: pitch %ld (multiple of 16, >= %ld)", r, pitch[r], w * ss);
        for (const long o : {cur_off[r], ref_off[r]})
            if (o < 0 || (o & 15) || o + pitch[r] * h > in_bytes)
                return fail(l, LADDER_E_INVAL, "rung %d: plane at %ld outside the %ld-byte input", r, o, in_bytes);
    }
    auto *p = new (std::nothrow) ladder_pipeline();
    if (!p) return LADDER_E_NOMEM;
    p->l = l;
    p->depth = depth;
    p->base = base_frame_id;
    p->in_bytes = in_bytes;
    p->out_bytes = ladder_frame_bytes(l);
    p->cur_off.assign(cur_off, cur_off + l->geo.n_rungs);
    p->ref_off.assign(ref_off, ref_off + l->geo.n_rungs);
    p->pitch.assign(pitch, pitch + l->geo.n_rungs);
    p->slot_ticket.assign(depth, -1);
    p->reported.assign(depth, 1);
    p->dev_in.assign(depth, nullptr);
    p->comp.assign(depth, nullptr);
    for (auto *v : {&p->ev_in, &p->ev_comp, &p->ev_out}) v->assign(depth, nullptr);
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < depth && e == cudaSuccess; ++j) {
        e = cudaMalloc(&p->dev_in[j], static_cast<size_t>(in_bytes));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->comp[j], cudaStreamNonBlocking);
        for (auto *v : {&p->ev_in, &p->ev_comp, &p->ev_out})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&(*v)[j], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&p->h_status, sizeof(int) * depth);
    if (e == cudaSuccess) memset(p->h_status, 0, sizeof(int) * depth);
    if (e != cudaSuccess) {
        pipeline_free(p);
        return cuda_fail(l, e, "pipeline buffers and streams");
    }
    *out = p;
    return LADDER_OK;
}

namespace {

// Status read back with slot j's last frame (complete): a non-zero word is
// kept to be reported once, and the device word is cleared.
void pipeline_collect(ladder_pipeline *p, int j)
{
    if (p->reported[j]) return;
    p->reported[j] = 1;
    if (p->h_status[j] == kStatusOk) return;
    if (!p->pending) p->pending = p->h_status[j];
    cudaMemsetAsync(p->l->d_status, 0, sizeof(int), p->s_out);
    cudaStreamSynchronize(p->s_out);
}

// Reports (once) a device status that frames of the pipeline read back.
ladder_status pipeline_take_pending(ladder_pipeline *p)
{
    if (!p->pending) return LADDER_OK;
    const int st = p->pending;
    p->pending = 0;
    return device_status_error(p->l, st);
}

}  // namespace

ladder_status ladder_pipeline_submit(ladder_pipeline_t *p, const void *host_in, int qp, void *host_out, long *ticket)
{
    TraceRange trace("ladder_pipeline_submit");
    if (!p || !host_in || !host_out) return LADDER_E_INVAL;
    ladder_t *l = p->l;
    const int j = static_cast<int>(p->next % p->depth), frame_id = p->base + j;
    cudaError_t e = cudaSuccess;
    if (p->slot_ticket[j] >= 0) {
        e = cudaEventSynchronize(p->ev_out[j]);  // the slot's previous frame is home
        if (e != cudaSuccess) return cuda_fail(l, e, "pipeline slot");
        pipeline_collect(p, j);
    }
    // a bounded device wait that ran out in an earlier frame: report it
    // before taking more work (nothing of this frame is enqueued)
    ladder_status pst = pipeline_take_pending(p);
    if (pst != LADDER_OK) return pst;
    e = cudaMemcpyAsync(p->dev_in[j], host_in, static_cast<size_t>(p->in_bytes), cudaMemcpyHostToDevice, p->s_in);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[j], p->s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->comp[j], p->ev_in[j], 0);
    if (e != cudaSuccess) return cuda_fail(l, e, "pipeline upload");
    const int rr = l->geo.ref_rung, n = l->geo.n_rungs;
    char *in = p->dev_in[j];
    struct Quiet {  // the pipeline waits for its own streams: no per-call marks
        ladder_t *l;
        explicit Quiet(ladder_t *x) : l(x) { ++l->quiet; }
        ~Quiet() { --l->quiet; }
    } quiet(l);
    ladder_status st = analyze_reference(l, frame_id, in + p->cur_off[rr], in + p->ref_off[rr], p->pitch[rr], qp,
                                         p->comp[j]);
    if (st != LADDER_OK) return st;
    if (n > 1) {
        std::vector<int> rungs;
        std::vector<const void *> curs, refs;
        std::vector<long> pitches;
        for (int r = 0; r < n; ++r) {
            if (r == rr) continue;
            rungs.push_back(r);
            curs.push_back(in + p->cur_off[r]);
            refs.push_back(in + p->ref_off[r]);
            pitches.push_back(p->pitch[r]);
        }
        st = analyze_dependents(l, frame_id, static_cast<int>(rungs.size()), rungs.data(), curs.data(), refs.data(),
                                pitches.data(), qp, p->comp[j]);
        if (st != LADDER_OK) return st;
    }
    e = cudaEventRecord(p->ev_comp[j], p->comp[j]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_out, p->ev_comp[j], 0);
    if (e != cudaSuccess) return cuda_fail(l, e, "pipeline ordering");
    st = ladder_fetch_frame_async(l, frame_id, host_out, p->out_bytes, p->s_out);
    if (st != LADDER_OK) return st;
    // the status word after this frame's analyses, read back with its decisions
    e = cudaMemcpyAsync(&p->h_status[j], l->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->s_out);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_out[j], p->s_out);
    if (e != cudaSuccess) return cuda_fail(l, e, "pipeline read-back");
    p->reported[j] = 0;
    p->slot_ticket[j] = p->next;
    if (ticket) *ticket = p->next;
    ++p->next;
    return LADDER_OK;
}

ladder_status ladder_pipeline_wait(ladder_pipeline_t *p, long ticket)
{
    TraceRange trace("ladder_pipeline_wait");
    if (!p) return LADDER_E_INVAL;
    if (ticket < 0 || ticket >= p->next) return fail(p->l, LADDER_E_INVAL, "ticket %ld not submitted", ticket);
    const int j = static_cast<int>(ticket % p->depth);
    if (p->slot_ticket[j] == ticket) {  // else a later frame of the slot waited for it already
        const cudaError_t e = cudaEventSynchronize(p->ev_out[j]);
        if (e != cudaSuccess) return cuda_fail(p->l, e, "pipeline wait");
        pipeline_collect(p, j);
    }
    return pipeline_take_pending(p);
}

void ladder_pipeline_destroy(ladder_pipeline_t *p) { pipeline_free(p); }

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

ladder_status ladder_set_tuning(ladder_t *l, int knob, int value)
{
    if (!l) return LADDER_E_INVAL;
    switch (knob) {
    case LADDER_TUNE_FS_BAND:
        if (value != 9 && value != 13) return fail(l, LADDER_E_INVAL, "full-search band %d (9 or 13)", value);
        if (value == 9 && l->geo.ctu_size != 64) return fail(l, LADDER_E_INVAL, "band 9 needs 64x64 CTUs");
        l->tune_fs_band = value;
        return LADDER_OK;
    case LADDER_TUNE_DEP_BAND:
        if (value != 0 && value != 9 && value != 17) return fail(l, LADDER_E_INVAL, "dependent band %d", value);
        l->tune_dep_band = value;
        return LADDER_OK;
    case LADDER_TUNE_DEP_RANGE:
        if (value != 16 && value != 32) return fail(l, LADDER_E_INVAL, "dependent range %d (16 or 32)", value);
        l->tune_dep_range = value;
        return LADDER_OK;
    case LADDER_TUNE_DEP_CTAS_PER_SM:
        if (value < 0 || value > 8) return fail(l, LADDER_E_INVAL, "CTAs per SM %d (0..8)", value);
        l->tune_dep_ctas = value;
        return LADDER_OK;
    case LADDER_TUNE_FS_GROUP:
        if (value < 0 || value > kFsMaxGroup) return fail(l, LADDER_E_INVAL, "tiles per CTA %d (0..%d)", value, kFsMaxGroup);
        l->tune_fs_group = value;
        return LADDER_OK;
    case LADDER_TUNE_FS_FUSE:
        if (value != 0 && value != 1) return fail(l, LADDER_E_INVAL, "fuse %d (0 or 1)", value);
        l->tune_fs_fuse = value;
        return LADDER_OK;
    case LADDER_TUNE_DEP_STAGED:
        if (value < 0 || value > 2) return fail(l, LADDER_E_INVAL, "staged %d (0, 1 or 2)", value);
        l->tune_dep_staged = value;
        return LADDER_OK;
    case LADDER_TUNE_DEP_INHERIT:
        if (value != 0 && value != 1) return fail(l, LADDER_E_INVAL, "inherit %d (0 or 1)", value);
        l->tune_dep_inherit = value;
        return LADDER_OK;
    default:
        return fail(l, LADDER_E_INVAL, "unknown tuning knob %d", knob);
    }
}

ladder_status ladder_set_debug(ladder_t *l, int control, int value)
{
    if (!l) return LADDER_E_INVAL;
    switch (control) {
    case LADDER_DEBUG_WAIT_POLLS:
        if (value != 0 && (value < 64 || value > kMvpSpinDefault))
            return fail(l, LADDER_E_INVAL, "wait polls %d (0, or 64 .. %d)", value, kMvpSpinDefault);
        l->dbg_wait_polls = value;
        return LADDER_OK;
    case LADDER_DEBUG_LOST_HANDOFF:
        if (value != 0 && value != 1) return fail(l, LADDER_E_INVAL, "lost hand-off %d (0 or 1)", value);
        l->dbg_lost_handoff = value;
        return LADDER_OK;
    default:
        return fail(l, LADDER_E_INVAL, "unknown debug control %d", control);
    }
}

ladder_status ladder_get_tuning(const ladder_t *l, int knob, int *value)
{
    if (!l || !value) return LADDER_E_INVAL;
    switch (knob) {
    case LADDER_TUNE_FS_BAND: *value = l->tune_fs_band; return LADDER_OK;
    case LADDER_TUNE_DEP_BAND: *value = l->tune_dep_band; return LADDER_OK;
    case LADDER_TUNE_DEP_RANGE: *value = l->tune_dep_range; return LADDER_OK;
    case LADDER_TUNE_DEP_CTAS_PER_SM: *value = l->tune_dep_ctas; return LADDER_OK;
    case LADDER_TUNE_FS_GROUP: *value = l->tune_fs_group; return LADDER_OK;
    case LADDER_TUNE_FS_FUSE: *value = l->tune_fs_fuse; return LADDER_OK;
    case LADDER_TUNE_DEP_STAGED: *value = l->tune_dep_staged; return LADDER_OK;
    case LADDER_TUNE_DEP_INHERIT: *value = l->tune_dep_inherit; return LADDER_OK;
    default: return LADDER_E_INVAL;
    }
}

ladder_status ladder_dependent_evals(ladder_t *l, void *cuda_stream, unsigned long long *evals)
{
    if (!l || !evals) return LADDER_E_INVAL;
    TraceRange tr("ladder_dependent_evals");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, l->d_evals, sizeof v, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(l->d_evals, 0, sizeof v, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(l, e, "dependent evaluation count");
    *evals = v;
    return LADDER_OK;
}

long ladder_device_bytes(const ladder_t *l) { return l ? static_cast<long>(l->arena_bytes) : 0; }

void ladder_destroy(ladder_t *l)
{
    TraceRange trace("ladder_destroy");
    if (!l) return;
    // the handle's own work only: other handles' streams keep running
    for (auto &m : l->marks) {
        cudaEventSynchronize(m.done);
        cudaEventDestroy(m.done);
    }
    l->marks.clear();
    for (auto &ds : l->dep)
        if (ds.done && ds.recorded) cudaEventSynchronize(ds.done);
    drain_events(l);
    for (cudaEvent_t e : l->spare) cudaEventDestroy(e);
    for (auto &ds : l->dep)
        if (ds.done) cudaEventDestroy(ds.done);
    cudaFreeHost(l->host_stage);
    cudaFree(l->arena);
    delete l;
}

const char *ladder_last_error(const ladder_t *l) { return l ? l->err.c_str() : "null handle"; }

}  // extern "C"
