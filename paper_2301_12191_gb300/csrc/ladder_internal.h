// ladder_internal.h -- declarations shared by the translation units of
// libladder.so (kernels + host C ABI).  Not a public header.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ladder_impl {

constexpr int kMaxDepths = 4;
constexpr int kThreads = 256;  // every analysis kernel runs 256-thread CTAs

// Launches a kernel of this library on stream s as a programmatic dependent
// of the kernel before it in the stream: its CTAs may be scheduled while
// that kernel drains.  Every kernel starts with dev::chain_entry(), which
// waits for the previous kernel to complete (its memory operations visible)
// before anything touches global memory, so stream order is kept.
template <typename... Params, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                  Args &&...args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// Device status word values (mirror ladder_status).
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = -6;
constexpr int kStatusTaskOverflow = -7;  // a dependent task list ran out of room (sized so it cannot)
constexpr int kStatusBounds = -8;        // debug builds: an index failed its bounds check (the access was skipped)

// Debug builds (compiled with LADDER_BOUNDS_CHECK=1) check array indexes and
// plane offsets on the device: a failed check records kStatusBounds in the
// launch's status word (first failure wins) and the caller skips the
// access.  Release builds compile every check to `true`.
#ifndef LADDER_BOUNDS_CHECK
#define LADDER_BOUNDS_CHECK 0
#endif
#ifdef __CUDACC__
__device__ __forceinline__ bool in_range(int *status, long i, long n)
{
#if LADDER_BOUNDS_CHECK
    if (i >= 0 && i < n) return true;
    if (status) atomicCAS(status, kStatusOk, kStatusBounds);
    return false;
#else
    (void)status;
    (void)i;
    (void)n;
    return true;
#endif
}
#endif

// Per-CTU layout of the candidate keys written by the motion search and read
// by the decision kernel: depth d occupies (4^d - 1) / 3 ... (4^(d+1) - 1) / 3,
// CUs of a depth in raster order inside the CTU.  A key is
// (SAD << 32) | tb, tb = L1 * K^2 + (dy + r) * K + (dx + r) with K = 2r + 1 and
// (dx, dy) the offset from the CU's search centre: the unsigned order of keys
// is the (SAD, |dx|+|dy|, dy, dx) order of the tie-break.
__host__ __device__ constexpr int key_offset(int d) { return ((1 << (2 * d)) - 1) / 3; }
__host__ __device__ constexpr int keys_per_ctu(int dmax) { return key_offset(dmax + 1); }

// Dependent-mode rule of one CU, written by the constraint-derivation kernel.
enum : uint8_t {
    kRuleEvaluated = 1,  // reachable, inside the 8-aligned frame, allowed as a leaf
    kRuleCanSplit = 2,   // reachable and (forced or allowed to split)
    kRuleReachable = 4,  // every ancestor may split
    // (8 is dev::kPresent)
    kRuleInherited = 16,  // evaluated, searched in pieces, and its four sub-CUs are evaluated around the same
                          // centre: its candidate SADs are their sums (the sub-CUs' lanes add into its table)
};

// Division by a divisor fixed for a whole launch as a multiply-high, an
// add and two shifts (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994, Sec. 4): exact for every 32-bit
// numerator and every divisor >= 1.  make_fastdiv runs on the host,
// fast_div on the device.
struct FastDiv {
    uint32_t m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    int l = 0;  // ceil(log2 d)
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.m = static_cast<uint32_t>((((1ull << l) - d) << 32) / d + 1);
    f.s1 = l > 0 ? 1 : 0;
    f.s2 = l > 0 ? l - 1 : 0;
    return f;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fast_div(uint32_t x, const FastDiv &f)
{
    const uint32_t t = __umulhi(f.m, x);
    return (t + ((x - t) >> f.s1)) >> f.s2;
}
#endif

// Geometry of one rung (host and device).
struct RungGeom {
    int W, H, W8, H8;
    int ctu, dmax;
    int ctu_cols, ctu_rows;
    int cols[kMaxDepths], rows[kMaxDepths];
    int cols8, rows8;
    FastDiv div_2w, div_2h;  // division by 2W, 2H
};

// Device decision arrays of one (rung, frame slot).  The at_* accessors are
// the interface the decision step writes through (OffDecisions has the same).
struct DevDecisions {
    int16_t *mvx[kMaxDepths], *mvy[kMaxDepths];
    int32_t *sad[kMaxDepths], *satd[kMaxDepths], *cost[kMaxDepths], *best[kMaxDepths];
    uint8_t *split[kMaxDepths], *evaluated[kMaxDepths];
    uint8_t *leaf_depth;
    int16_t *leaf_mvx, *leaf_mvy;
    __host__ __device__ int16_t *at_mvx(int d) const { return mvx[d]; }
    __host__ __device__ int16_t *at_mvy(int d) const { return mvy[d]; }
    __host__ __device__ int32_t *at_sad(int d) const { return sad[d]; }
    __host__ __device__ int32_t *at_satd(int d) const { return satd[d]; }
    __host__ __device__ int32_t *at_cost(int d) const { return cost[d]; }
    __host__ __device__ int32_t *at_best(int d) const { return best[d]; }
    __host__ __device__ uint8_t *at_split(int d) const { return split[d]; }
    __host__ __device__ uint8_t *at_evaluated(int d) const { return evaluated[d]; }
    __host__ __device__ uint8_t *at_leaf_depth() const { return leaf_depth; }
    __host__ __device__ int16_t *at_leaf_mvx() const { return leaf_mvx; }
    __host__ __device__ int16_t *at_leaf_mvy() const { return leaf_mvy; }
};

// Byte offsets of the decision arrays (and the per-CTU argmin keys) inside
// one (frame slot, rung) block; the same for every slot of a rung.
struct DecOffsets {
    long mvx[kMaxDepths], mvy[kMaxDepths], sad[kMaxDepths], satd[kMaxDepths], cost[kMaxDepths], best[kMaxDepths];
    long split[kMaxDepths], evaluated[kMaxDepths];
    long leaf_depth, leaf_mvx, leaf_mvy;
    long keys;
    long done;  // per CTU: full-search CTAs finished (zero at rest)
    // spatial-predictor decisions: per CTU its bottom-row leaf vectors as
    // (generation << 32 | vector) words, then the block's generation and its
    // count of finished rows
    long mvp_flag;
    // dependent rungs: per CTU and key slot, the search centre, rule flags
    // and (CUs of 32x32 and up) the CU's place in its task list
    long dep_cx, dep_cy, dep_flags, dep_slot;
    long dec_bytes;  // the decision arrays span [0, dec_bytes)
};

struct RungInfo {
    RungGeom g;
    DecOffsets off;
};

// Address of the array at `off` in a block; a null base means the offsets
// are the arrays' own device addresses (caller-owned arrays that live in no
// block, as with the allocation-free entry point).
__host__ __device__ inline char *array_at(char *base, long off)
{
    return base ? base + off : reinterpret_cast<char *>(static_cast<uintptr_t>(off));
}

__host__ __device__ inline DevDecisions decisions_at(char *base, const DecOffsets &o)
{
    DevDecisions d{};
    for (int k = 0; k < kMaxDepths; ++k) {
        d.mvx[k] = reinterpret_cast<int16_t *>(array_at(base, o.mvx[k]));
        d.mvy[k] = reinterpret_cast<int16_t *>(array_at(base, o.mvy[k]));
        d.sad[k] = reinterpret_cast<int32_t *>(array_at(base, o.sad[k]));
        d.satd[k] = reinterpret_cast<int32_t *>(array_at(base, o.satd[k]));
        d.cost[k] = reinterpret_cast<int32_t *>(array_at(base, o.cost[k]));
        d.best[k] = reinterpret_cast<int32_t *>(array_at(base, o.best[k]));
        d.split[k] = reinterpret_cast<uint8_t *>(array_at(base, o.split[k]));
        d.evaluated[k] = reinterpret_cast<uint8_t *>(array_at(base, o.evaluated[k]));
    }
    d.leaf_depth = reinterpret_cast<uint8_t *>(array_at(base, o.leaf_depth));
    d.leaf_mvx = reinterpret_cast<int16_t *>(array_at(base, o.leaf_mvx));
    d.leaf_mvy = reinterpret_cast<int16_t *>(array_at(base, o.leaf_mvy));
    return d;
}

// The same arrays as a block and its offsets, for a kernel whose offsets sit
// in its parameters: each address is formed where it is used, so no table
// of pointers is held per thread (a kernel at 64 registers kept that table
// in local memory).  `base` is a rung block (never null here).
struct OffDecisions {
    char *base;
    const DecOffsets *off;
    template <typename P> __device__ P *at(long o) const { return reinterpret_cast<P *>(base + o); }
    __device__ int16_t *at_mvx(int d) const { return at<int16_t>(off->mvx[d]); }
    __device__ int16_t *at_mvy(int d) const { return at<int16_t>(off->mvy[d]); }
    __device__ int32_t *at_sad(int d) const { return at<int32_t>(off->sad[d]); }
    __device__ int32_t *at_satd(int d) const { return at<int32_t>(off->satd[d]); }
    __device__ int32_t *at_cost(int d) const { return at<int32_t>(off->cost[d]); }
    __device__ int32_t *at_best(int d) const { return at<int32_t>(off->best[d]); }
    __device__ uint8_t *at_split(int d) const { return at<uint8_t>(off->split[d]); }
    __device__ uint8_t *at_evaluated(int d) const { return at<uint8_t>(off->evaluated[d]); }
    __device__ uint8_t *at_leaf_depth() const { return at<uint8_t>(off->leaf_depth); }
    __device__ int16_t *at_leaf_mvx() const { return at<int16_t>(off->leaf_mvx); }
    __device__ int16_t *at_leaf_mvy() const { return at<int16_t>(off->leaf_mvy); }
};

constexpr int kMaxRungs = 16;
constexpr int kMaxItems = 64;                    // frames per batched launch
constexpr int kMaxDepItems = kMaxItems * 3;      // dependent (frame, rung) pairs per batched launch

// ---- full search (independent analysis) --------------------------------
// One item = one frame's independently analysed rung.  One CTA per (CTU,
// warp tile of candidates); kernel parameters are grid-constant (CUDA 12.1+
// allows 32 KB), the tensor maps included.
constexpr int kFsBand = 13;    // candidate rows (dy) per lane task
constexpr int kFsMaxGroup = 4;  // warp tiles one full-search CTA may take

struct FullSearchItem {
    int W, H;
    unsigned long long *keys;  // per CTU keys_per_ctu(dmax), ~0 before the search
    int cta_begin;             // first CTA of this frame: CTUs x ctas_per_ctu CTAs, CTU-major
    // the decisions, when the search takes them too (fuse_decide)
    const void *cur, *ref;
    long pitch_bytes;
    char *block;               // the (slot, rung) block
    int rung, qp;
    unsigned int *done;        // per CTU: CTAs finished (fuse_decide; zero before and after)
};

struct FullSearchBatch {
    int n;
    int R;            // search range
    int band;         // candidate rows per lane task (13, or 9 for 64x64 CTUs)
    int group;        // consecutive warp tiles of one CTU per CTA (one staged window)
    int Rp;           // left window margin: R rounded up to 16 samples
    int ntasks;       // lane tasks (dx, band of kFsBand dy) per CTU
    int warp_tiles;   // warp tiles per CTU: ceil(ntasks / 32)
    int box_h;        // rows of the TMA box (the most any warp tile needs)
    int e_bytes;      // shared bytes of the expanded window (box_h x positions x 4)
    int stage_off;    // byte offset of the staged rows inside the expanded window
    int phase1_rows;  // expanded rows that end before the staged rows
    int buf_bytes;    // shared bytes of the expanded window + current CTU + block sums
    int cur_l1;       // 10-bit: current CTU through L1 (every item's W and H multiples of 8)
    int total;        // CTAs of the batch
    uint32_t one;     // 1, as an operand the compiler cannot fold
    int *status;
    // fuse_decide: the last CTA to finish a CTU also takes the CTU's
    // decisions (SATD, cost, split, leaf maps) and resets its keys to ~0
    int fuse_decide;
    int satd_mode;
    RungInfo rung[kMaxRungs];
    FullSearchItem item[kMaxItems];
    CUtensorMap map[kMaxItems];      // reference plane of each item (box: window positions x box_h rows)
    CUtensorMap cur_map[kMaxItems];  // current plane of each item (box: CTU x CTU)
};

struct FullSearchPlan {
    int Rp;
    int band, nbands, ntasks, warp_tiles;
    int group, ctas_per_ctu;  // warp tiles per CTA, CTAs per CTU
    int P4;           // window positions per row
    int box_w, box_h; // TMA box (samples x rows)
    int e_bytes, stage_off, phase1_rows, buf_bytes;
    int smem_bytes;   // dynamic shared memory of one CTA (two buffers)
    int cur_l1;       // 10-bit: the current CTU read through L1 (no shared copy)
};

// Returns the plan for bit depth / CTU / R / band (13 or 9 candidate rows
// per lane task; 9 only with 64x64 CTUs).
// `group` warp tiles share one CTA and its window (reduced while the window
// would exceed the kernels' bound).
// cur_l1 (10-bit, frames of whole 8x8 blocks): the current CTU is read
// through L1 instead of a shared copy, which frees its shared memory.
FullSearchPlan full_search_plan(int bit_depth, int ctu, int R, int band = kFsBand, int group = 1, int cur_l1 = 0);
// Tiled 2-D tensor map of a W x H plane (8-bit: uint8, 10-bit: uint16
// samples), box box_w x box_h samples, zero fill outside the plane.
// Returns 0 on success, else the driver's error (or -1: encoder unavailable).
int encode_plane_map(CUtensorMap *map, const void *plane, int W, int H, long pitch_bytes, int bit_depth, int box_w,
                     int box_h);
// Both maps of one full-search item: the reference window and the current CTU.
int encode_item_maps(FullSearchBatch &b, int k, const void *cur, const void *ref, int W, int H, long pitch_bytes,
                     int bit_depth, int ctu, const FullSearchPlan &p);
// Copies the plan's launch constants into a batch.
void fill_full_search_batch(FullSearchBatch &b, const FullSearchPlan &p, int R);
// Resident full-search CTAs per SM for this plan (occupancy calculator).
int full_search_ctas_per_sm(int bit_depth, int ctu, int R, int band = kFsBand, int group = 1, int cur_l1 = 0);
// One CTA per work item: b.total = sum over frames of CTUs x ceil(warp_tiles / group).
cudaError_t launch_full_search(int bit_depth, int ctu, const FullSearchBatch &b, cudaStream_t s);

// ---- decision step of independently analysed rungs -------------------------
struct DecideItem {
    const void *cur, *ref;
    long pitch_bytes;
    char *block;          // the (slot, rung) block: decisions + keys (null: the offsets are addresses)
    int rung;
    int qp;
    int cta_begin;        // first CTA of this item (one CTA per CTU)
};

struct DecideBatch {
    int n;
    int range;            // R: decodes the keys
    int satd_mode;
    int total_ctas;
    int *status;          // device status word (debug builds record failed bounds checks)
    RungInfo rung[kMaxRungs];
    DecideItem item[kMaxItems];
};
cudaError_t launch_decide(int bit_depth, int ctu, const DecideBatch &b, cudaStream_t s);

// ---- dependent analysis: rules, refinement search, decisions --------------
// Reference-rung state a dependent rung reads.
struct DepRefs {
    int Wr, Hr, cols8_r;     // reference rung size and 8x8 grid width
    const uint8_t *leaf_depth;
    const int16_t *leaf_mvx, *leaf_mvy;
    int depth_lo, depth_hi, use_ref_mv;
    FastDiv div_2wr, div_2hr;  // division by 2 Wr, 2 Hr
    long n8_r;                 // 8x8 blocks of the reference rung (bounds checks)
    int *status;
};

struct DependentItem {
    const void *cur, *ref;
    long pitch_bytes;
    char *block;             // this (slot, rung) block
    const char *ref_block;   // the frame's block of the parent rung (whose decisions this rung refines)
    int rung;
    int parent;              // the parent rung
    int qp;
    int cta_begin;           // first CTA of this item in the per-CTU kernels (one CTA per CTU)
};

// Evaluated CUs of a launch, one list per CU size class c (size 8 << c).
// A task is (item | (CTU * keys per CTU + key slot) << 8) in the low word and
// the centre (cx & 0xffff | cy << 16) in the high word.  CUs larger than the
// batch's range (16 or 32) are searched in range x range pieces whose
// candidate SADs add up in a per-CU table of (2r+1)^2 sums (classes 2 and 3
// have table room).  Such a CU whose four sub-CUs are evaluated around its
// own centre is inherited: it has no task and its SADs are the sums of its
// sub-CUs'.  If they are single pieces, its table (a slot counted down from
// the top of the class's capacity) takes the SADs their lanes add into it,
// named by up[c][task] of each sub-CU (0xffffffff: none).  If they have
// tables of their own (a 64x64 CU of 32x32 sub-CUs at pieces of 16), it has
// none: the decisions add the four tables entry by entry.
constexpr int kSizeClasses = 4;
constexpr int kFirstSummedClass = 2;
constexpr int kFirstUpClass = kFirstSummedClass - 1;  // classes whose CUs may have an inherited ancestor
constexpr uint32_t kNoUp = 0xffffffffu;
// counters of one set of task lists: tasks per class, inherited CUs per
// class, then the staged search's next tile (zero before each batch)
constexpr int kTileCounter = 2 * kSizeClasses;
constexpr int kDepCounters = 2 * kSizeClasses + 1;
constexpr int kDepBand = 17;  // candidate rows per lane task (9 for r <= 4)

struct DependentBatch {
    int n;
    int r;                  // refinement range
    int range;              // CUs larger than this (16 or 32) are searched in pieces of this side
    int band;               // candidate rows per lane task: 9 or 17
    int ctas_per_sm;        // search grid: CTAs per SM (0: as many as fit)
    int staged;             // 1: each tile's windows staged in shared memory first (10-bit, r >= 4); 0: read from L1
    int inherit;            // 1: CUs whose sub-CUs share their centre take their SADs as sums (kRuleInherited)
    int satd_mode;
    int depth_lo, depth_hi, use_ref_mv;
    int total_ctas;         // CTUs of the batch
    int *status;
    unsigned long long *tasks[kSizeClasses];  // per size class, capacity cap[c]
    unsigned int *pos[kSizeClasses];          // per task: the CU's origin, x | y << 16
    unsigned int *sums[kSizeClasses];         // classes >= kFirstSummedClass: cap[c] x (2r+1)^2
    unsigned int *up[kSizeClasses];           // classes kFirstUpClass .. kSizeClasses - 2: per task, the table
                                              // slot of the CU's inherited parent (kNoUp: none)
    unsigned int cap[kSizeClasses];
    unsigned int *counts;   // kDepCounters counters, zero before the rules kernel: tasks per class, inherited
                            // CUs per class (their table slots count down from cap[c] - 1), the next tile
    unsigned long long *evals;  // running count of the SAD-candidate evaluations searched (8x8 block x candidate)
    uint32_t one;           // 1, as an operand the compiler cannot fold
    RungInfo rung[kMaxRungs];
    DependentItem item[kMaxDepItems];
};
// Rules, reachability, centres and task lists (one CTA per CTU); the search
// over the task lists (persistent grid); SATD, cost, split and leaf maps (one
// CTA per CTU).  Launched in this order on one stream.
cudaError_t launch_dependent_rules(int ctu, const DependentBatch &b, cudaStream_t s);
cudaError_t launch_dependent_search(int bit_depth, const DependentBatch &b, cudaStream_t s);
cudaError_t launch_dependent_decide(int bit_depth, int ctu, const DependentBatch &b, cudaStream_t s);

// Decisions of one analysed rung at further QPs: one CTA per (CTU, QP),
// the resident vectors and SATDs, cost / split / leaf maps per QP.
constexpr int kMaxQps = 8;
struct QpBatch {
    int n_qps;
    int qp[kMaxQps];
    RungGeom g;
    DecOffsets off;
    const char *block;       // the (slot, rung) decision block
    int dependent;           // 1: rule flags of the dependent analysis; 0: flags of the geometry
    DevDecisions out[kMaxQps];  // cost, best, split and leaf maps set
};
cudaError_t launch_decide_qps(int ctu, const QpBatch &b, cudaStream_t s);

// Quarter-pel refinement of one analysed rung: one CTA per CTU.
// One (frame, rung) job of a quarter-pel refinement launch.
struct SubpelItem {
    int rung;
    int cta_begin;           // first refinement CTA (one per CTU)
    int icta_begin, icols;   // first interpolation CTA; interpolation tiles per row
    RungGeom g;
    DecOffsets off;
    const char *block;       // the (slot, rung) decision block
    int dependent;           // 1: rule flags of the dependent analysis; 0: flags of the geometry
    int qp;
    const void *cur, *ref;
    long pitch_bytes;
    // the 16 interpolated planes of ref (phase fy * 4 + fx), each covering
    // the positions -4 .. W+3 by -4 .. H+3 (subpel_workspace_layout)
    char *planes;
    long plane_pitch, plane_bytes;
    // spatial predictor: the SATD of every position the two rounds can
    // visit, kSubpelTab per evaluated CU (after the planes in the workspace)
    int32_t *table;
    DevDecisions out;        // mvx, mvy (quarter-pel), satd, cost, best, split and leaf maps set
};
constexpr int kMaxSubpelItems = 16;
struct SubpelBatch {
    int n;
    int satd_mode;
    SubpelItem item[kMaxSubpelItems];
};
// Quarter-pel positions within +-3 of 4 mv in each axis, 4 mv itself left
// out: every position the half-pel round (+-2) and the quarter-pel round
// (+-1 around any half-pel best) can visit.  Index: raster order over
// (oy, ox) in [-3, 3]^2, skipping (0, 0).
constexpr int kSubpelTab = 48;
__host__ __device__ constexpr int subpel_tab_index(int ox, int oy)
{
    return (oy + 3) * 7 + (ox + 3) < 24 ? (oy + 3) * 7 + (ox + 3) : (oy + 3) * 7 + (ox + 3) - 1;
}
// Bytes of the SATD table of a rung (per CTU, keys_per_ctu x kSubpelTab int32).
inline long subpel_table_bytes(int ctu_cols, int ctu_rows, int dmax)
{
    return (static_cast<long>(ctu_cols) * ctu_rows * keys_per_ctu(dmax) * kSubpelTab * 4 + 255) / 256 * 256;
}
// The refinement with the spatial predictor, decided CTU by CTU in wavefront
// order from the tables (one CTA per CTU row, rows wait on the row above).
struct SubpelMvpItem {
    char *block;            // the (slot, rung) decision block: flags, integer vectors and SATDs, hand-off words
    int rung, qp, dependent;
    int cta_begin;          // CTA of the item's first CTU row
    const int32_t *table;   // per CTU and key, kSubpelTab SATDs
    DevDecisions out;
};
struct SubpelMvpBatch {
    int n;
    int *status;
    int spin;          // polls of one wait before it gives up
    int lost_handoff;  // test control: 1 = rows wait for a hand-off generation no row publishes
    RungInfo rung[kMaxRungs];
    SubpelMvpItem item[kMaxSubpelItems];
};
// The table launch (after the interpolation) and the cooperative wavefront
// launch of ctas CTAs.
cudaError_t launch_subpel_table(int bit_depth, int ctu, const SubpelBatch &b, int ctas, int interp_ctas,
                                cudaStream_t s);
cudaError_t launch_subpel_mvp(int ctu, const SubpelMvpBatch &b, int ctas, cudaStream_t s);
// CTAs of the refinement wavefront kernel that fit on the device at once.
int subpel_mvp_capacity(int ctu, int sm_count);

// ---- spatial MV predictor (wavefront re-decision) -------------------------
// One item = one analysed (frame slot, rung), decided again with the
// spatial predictor: one CTA per CTU row, rows in wavefront lockstep.
struct MvpItem {
    char *block;
    int rung, qp, dependent;
    int cta_begin;  // CTA of the item's first CTU row
};
constexpr int kMaxMvpItems = kMaxDepItems;
constexpr int kMvpSpinDefault = 1 << 22;  // polls (an L2 round trip each, under a microsecond) before a wait gives up
struct MvpBatch {
    int n;
    int *status;
    int spin;          // polls of one wait before it gives up (kMvpSpinDefault unless a test lowers it)
    int lost_handoff;  // test control: 1 = rows wait for a hand-off generation no row publishes

    // use_out: decisions at item 0's QP into `out` (cost, best, split, leaf
    // maps; n must be 1) instead of in place (further-QP decisions)
    int use_out;
    DevDecisions out;
    RungInfo rung[kMaxRungs];
    MvpItem item[kMaxMvpItems];
};
// Cooperative launch of ctas CTAs (every CTA resident: rows wait on rows).
cudaError_t launch_decide_mvp(int ctu, const MvpBatch &b, int ctas, cudaStream_t s);
// CTAs of the wavefront kernel that fit on the device at once.
int decide_mvp_capacity(int ctu, int sm_count);

// Bytes of the interpolation workspace of a W x H plane (16 planes), with the
// row pitch and the bytes of one plane.
long subpel_workspace_layout(int bit_depth, int W, int H, long *plane_pitch, long *plane_bytes);
// Interpolation tiles of a W x H plane: (columns, rows).
void subpel_interp_tiles(int W, int H, int *cols, int *rows);
// Two launches: the interpolated planes of every job, then the refinements
// (the items' CTA ranges set by the caller, in item order).
cudaError_t launch_subpel(int bit_depth, int ctu, const SubpelBatch &b, int ctas, int interp_ctas, cudaStream_t s);

// Fills the keys of every block of a batch with ~0 (key initialisation).
struct FillItem {
    unsigned long long *keys;
    long n;
};
struct FillBatch {
    int n;
    FillItem item[kMaxItems];
};
cudaError_t launch_fill_keys(const FillBatch &b, cudaStream_t s);

// Sets the kernels' shared-memory attributes for a geometry (before any
// stream capture).
cudaError_t prepare_full_search(int bit_depth, int ctu, int R);
cudaError_t prepare_kernels(int bit_depth, int ctu, int R, int r);

}  // namespace ladder_impl
