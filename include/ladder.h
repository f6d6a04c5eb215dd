/*
 * ladder.h -- C ABI of libladder.so: GB300 (sm_103a) inter analysis for
 * multi-resolution (ABR ladder) encoding.
 *
 * The library analyses frame pairs (current, reference) of 8- or 10-bit luma:
 * integer full-search block-matching motion estimation by SAD (Sec. 5.4.1,
 * SAD equation), then, per CU of the quadtree (Sec. 2.1: a CTU of 64x64,
 * 32x32 or 16x16 split down to 8x8), an 8x8-Hadamard SATD at the chosen
 * vector (Sec. 5.4.1, SATD equation) plus lambda(QP) times an MV-bit estimate,
 * and the bottom-up rate-distortion split decision (Sec. 2.1).  One rung of
 * the ladder (the reference rung) is analysed independently; the other rungs
 * are analysed as dependents that reuse the reference rung's co-located CU
 * depth and its motion vector scaled by the resolution ratio, refined in a
 * small window (inter-resolution analysis sharing with refinement, Sec. 4.3
 * and Sec. 6.3; the reuse and refinement controls of App. A.1 / A.2).
 *
 * All analysis is integer; results are bit-exact against a plain CPU oracle.
 *
 * Threading and streams: a ladder_t is not thread-safe; serialise calls on
 * one handle.  Every call that takes a stream enqueues work on it and returns
 * without waiting, except fetch_decisions (waits for its copies) and
 * ladder_sync.  The analyses of one frame must be enqueued on one stream, or
 * the caller orders the streams itself (the dependent reads device state that
 * the reference analysis writes).  Different frames may go to different
 * streams and then run side by side: the library orders what their analyses
 * share (the dependent task lists come in three sets: a batch takes its
 * stream's last set, else an unused one, else the least recently used one
 * after that set's last batch).  Captured graphs of one handle
 * take no such waits: replay them one at a time, and not while other
 * analyses of the handle are in flight on another stream.
 *
 * Memory: the caller owns the input planes (device pointers, typically from
 * PyTorch tensors) and must keep them alive and unmodified until the stream
 * has passed the call.  The library owns its decision buffers and the
 * resident reference decisions of each frame slot until ladder_release_frame
 * or ladder_destroy.  fetch_decisions copies into caller-owned host arrays.
 */
#ifndef LADDER_H
#define LADDER_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LADDER_API __attribute__((visibility("default")))
#else
#define LADDER_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ladder ladder_t; /* opaque, library-owned */

typedef enum {
    LADDER_OK = 0,
    LADDER_E_INVAL = -1,   /* bad argument (geometry, QP, pitch, rung, pointer) */
    LADDER_E_NOMEM = -2,   /* device or host allocation failed */
    LADDER_E_NOREF = -3,   /* dependent analysis before its frame's reference */
    LADDER_E_BUSY = -4,    /* no free frame slot */
    LADDER_E_CUDA = -5,    /* a CUDA runtime call failed; see ladder_last_error */
    LADDER_E_TIMEOUT = -6, /* a bounded device wait ran out (device status word) */
    LADDER_E_STATE = -7,   /* call out of order (e.g. fetch before analysis) */
    LADDER_E_BOUNDS = -8   /* debug builds only: a device-side bounds check failed (the access was skipped) */
} ladder_status;

#define LADDER_MAX_DEPTHS 4 /* CU depths 0..3 for a 64x64 CTU: 64, 32, 16, 8 */

typedef struct {
    int width, height; /* luma size in samples; both must be even */
} ladder_rung;

typedef struct {
    int n_rungs;               /* 1..16 */
    const ladder_rung *rungs;  /* copied at init */
    int ref_rung;              /* index of the independently analysed rung */
    int bit_depth;             /* 8 => uint8 samples, 10 => uint16 samples in [0, 1023] */
    int ctu_size;              /* 16, 32 or 64; smallest CU is 8x8, so depths 0..log2(ctu/8) */
    int ref_search_range;      /* R: full search +-R around (0,0), 4..64 */
    int dep_refine_range;      /* r: dependents search +-r around the scaled vector, 0..32 */
    int dep_depth_lo;          /* allowed dependent leaf depths [Deq+lo, Deq+hi]; */
    int dep_depth_hi;          /*   defaults 0, +1 (evaluate depth n and n+1) */
    int dep_use_ref_mv;        /* 1: search centre = scaled reference MV; 0: (0,0) */
    int satd_mode;             /* 0: 8x8 Hadamard, (sum|T|)>>2; 1: two 4x4 per 8x4 half, >>1 */
    int max_frames;            /* resident frame slots (1..256) */
} ladder_geometry;

/* Decisions of one rung for one frame, all in CU raster order of the frame's
 * depth-d CU grid: cols_d = ceil(W8 / S_d), rows_d = ceil(H8 / S_d) with
 * W8, H8 the size rounded up to a multiple of 8 and S_d = ctu_size >> d.
 * Arrays for depths beyond log2(ctu/8) are ignored and may be NULL.
 * Not-evaluated CUs carry mv = INT16_MIN and sad/satd/cost = INT32_MAX. */
typedef struct {
    int16_t *mvx[LADDER_MAX_DEPTHS], *mvy[LADDER_MAX_DEPTHS];
    int32_t *sad[LADDER_MAX_DEPTHS];   /* SAD at the chosen vector */
    int32_t *satd[LADDER_MAX_DEPTHS];  /* SATD at the chosen vector */
    int32_t *cost[LADDER_MAX_DEPTHS];  /* J = SATD + ((lambdaQ16[qp]*bits + 2^15) >> 16) */
    int32_t *best[LADDER_MAX_DEPTHS];  /* min over the subtree; INT32_MAX if unreachable */
    uint8_t *split[LADDER_MAX_DEPTHS]; /* 1 = split into four children */
    uint8_t *evaluated[LADDER_MAX_DEPTHS];
    uint8_t *leaf_depth;               /* per 8x8, (W8/8) x (H8/8) raster */
    int16_t *leaf_mvx, *leaf_mvy;      /* per 8x8: vector of its leaf CU */
} ladder_decisions;

/* Creates a ladder handle: validates the geometry (LADDER_E_INVAL), sizes and
 * allocates every device buffer up front (LADDER_E_NOMEM), and uploads the
 * constant tables on `cuda_stream` (a cudaStream_t, NULL for the legacy
 * default stream).  On success *out owns everything; free with ladder_destroy. */
LADDER_API ladder_status ladder_init(const ladder_geometry *geometry, void *cuda_stream, ladder_t **out);

/* Independent analysis of the reference rung of frame `frame_id` (any int):
 * full search +-R for every CU at every depth, SATD, cost and split (the
 * analysis that the x265 "analysis-save" master encode performs, App. A.1).
 * `cur` and `ref` are device pointers to W x H planes of the reference rung,
 * rows `pitch_bytes` apart (a multiple of 16, >= W * sample size).  Claims a
 * frame slot for `frame_id` (LADDER_E_BUSY if none is free; re-analysing a
 * frame that holds a slot reuses it).  QP outside 0..51 -> LADDER_E_INVAL. */
LADDER_API ladder_status analyze_reference(ladder_t *ladder, int frame_id, const void *cur, const void *ref,
                                long pitch_bytes, int qp, void *cuda_stream);

/* Dependent analysis of rung `rung` (!= ref_rung) of frame `frame_id`: each
 * CU maps its centre to the reference rung, takes the co-located reference
 * leaf's depth and MV, searches +-r around the MV scaled by the rung ratio
 * (round half away from zero) and only at the depths the reference leaf
 * allows (Sec. 4.3 / 6.3 reuse with refinement).  LADDER_E_NOREF if the
 * frame's reference rung has not been analysed. */
LADDER_API ladder_status analyze_dependent(ladder_t *ladder, int rung, int frame_id, const void *cur,
                                const void *ref, long pitch_bytes, int qp, void *cuda_stream);

/* Several dependent rungs of frame `frame_id` in one launch (all CTUs of
 * all listed rungs run concurrently; results are identical to one
 * analyze_dependent call per rung).  n in 1..16, rungs distinct and not the
 * reference rung; cur[k], ref[k], pitch_bytes[k] describe rung rungs[k]. */
LADDER_API ladder_status analyze_dependents(ladder_t *ladder, int frame_id, int n, const int *rungs,
                                            const void *const *cur, const void *const *ref,
                                            const long *pitch_bytes, int qp, void *cuda_stream);

/* One frame of one ladder in a batch: its planes for every rung, in rung
 * order (device pointers), and its QP.  `frame_id` names its frame slot. */
typedef struct {
    int frame_id;
    int qp;
    const void *const *cur;     /* n_rungs current planes */
    const void *const *ref;     /* n_rungs reference planes */
    const long *pitch_bytes;    /* n_rungs row pitches */
} ladder_request;

/* Analyses many ladder frames together: the reference rung of every request
 * independently, then every other rung as a dependent of its own frame's
 * reference (results identical to analyze_reference + analyze_dependents per
 * request).  Four launches for the whole batch: key reset, full search,
 * decisions, dependents.  n in 1..64 and n x (n_rungs - 1) <= 192; frame ids
 * distinct.  LADDER_E_BUSY when the batch needs more free frame slots than
 * there are (nothing is launched then). */
LADDER_API ladder_status ladder_analyze_batch(ladder_t *ladder, const ladder_request *requests, int n,
                                              void *cuda_stream);

/* One rung of one frame: kind 0 = independent full search (the reference
 * rung's makes the frame's reference resident), kind 1 = dependent of the
 * frame's reference. */
typedef struct {
    int frame_id;
    int rung;
    int kind;
    int qp;
    const void *cur, *ref;
    long pitch_bytes;
} ladder_job;

/* Any mix of jobs of any frames in one call: all independent jobs in
 * batched launches first, then all dependent jobs in batched launches, on
 * `cuda_stream` (a dependent may use a reference job of the same call).
 * (frame, rung) pairs distinct.  Results are identical to one call per job.
 * LADDER_E_NOREF if a dependent's frame has no reference (resident or in
 * the call); LADDER_E_BUSY if the new frames need more free slots than
 * there are; nothing is launched on an error. */
LADDER_API ladder_status ladder_analyze_jobs(ladder_t *ladder, const ladder_job *jobs, int n, void *cuda_stream);

/* Every rung of every request analysed independently (full search +-R on
 * each rung), batched like ladder_analyze_batch: the per-rung baseline of the
 * multi-resolution speedup.  n in 1..64. */
LADDER_API ladder_status ladder_analyze_batch_independent(ladder_t *ladder, const ladder_request *requests, int n,
                                                          void *cuda_stream);

/* A batch captured once into a CUDA graph, replayed by ladder_graph_launch
 * (the planes named in the requests are read at every replay, so the caller
 * refills those buffers between replays).  Capture runs on `cuda_stream`,
 * which must not be the legacy default stream; kernel timing is off inside
 * the graph. */
typedef struct ladder_graph ladder_graph_t;
LADDER_API ladder_status ladder_capture_batch(ladder_t *ladder, const ladder_request *requests, int n,
                                              void *cuda_stream, ladder_graph_t **out);
LADDER_API ladder_status ladder_graph_launch(ladder_graph_t *graph, void *cuda_stream);
LADDER_API void ladder_graph_destroy(ladder_graph_t *graph);

/* Kernel-shape knobs (no counterpart in the paper: they choose how the
 * search is laid out on the GPU, never what it computes; every setting
 * gives bit-identical decisions).  A change applies to later launches;
 * captured graphs keep the shapes they were captured with.  Values:
 *   LADDER_TUNE_FS_BAND          full search: candidate rows per lane task,
 *                                13 (default) or 9 (64x64 CTUs only)
 *   LADDER_TUNE_DEP_BAND         dependent search: candidate rows per lane
 *                                task, 0 (automatic), 9 or 17
 *   LADDER_TUNE_DEP_RANGE        dependent search: CUs larger than this
 *                                side (16, default, or 32) are searched in
 *                                pieces of this side
 *   LADDER_TUNE_DEP_CTAS_PER_SM  dependent search grid: CTAs per SM, 0 (as
 *                                many as fit, default) to 8
 *   LADDER_TUNE_FS_GROUP         full search: consecutive warp tiles of one
 *                                CTU per CTA, sharing one staged window:
 *                                0 (automatic, default) to 4
 *   LADDER_TUNE_FS_FUSE          1 (default): the last full-search CTA of
 *                                each CTU also takes the CTU's decisions;
 *                                0: separate key-fill and decision kernels
 *   LADDER_TUNE_DEP_STAGED       dependent search, refinement ranges of 4
 *                                and more (8- and 10-bit): 1 (default)
 *                                stages each tile's reference windows in
 *                                shared memory, 2 does so into two buffers
 *                                (the next tile's copies in flight during
 *                                the current one), 0 reads the windows
 *                                through L1
 *   LADDER_TUNE_DEP_INHERIT      1 (default): a dependent CU searched in
 *                                pieces whose four sub-CUs are evaluated
 *                                around its own centre is not searched; its
 *                                candidate SADs are the sums of theirs (the
 *                                same candidates over four disjoint quarters
 *                                of its samples), added by the lanes that
 *                                search the sub-CUs or, where these have
 *                                sum tables, from those tables; 0: every
 *                                evaluated CU is searched
 * LADDER_E_INVAL for an unknown knob or value. */
typedef enum {
    LADDER_TUNE_FS_BAND = 0,
    LADDER_TUNE_DEP_BAND = 1,
    LADDER_TUNE_DEP_RANGE = 2,
    LADDER_TUNE_DEP_CTAS_PER_SM = 3,
    LADDER_TUNE_FS_GROUP = 4,
    LADDER_TUNE_FS_FUSE = 5,
    LADDER_TUNE_DEP_STAGED = 6,
    LADDER_TUNE_DEP_INHERIT = 7
} ladder_tune_knob;
LADDER_API ladder_status ladder_set_tuning(ladder_t *ladder, int knob, int value);
LADDER_API ladder_status ladder_get_tuning(const ladder_t *ladder, int knob, int *value);

/* Work the dependent searches did (no counterpart in the paper; for
 * measurement): the SAD-candidate evaluations (one 8x8 block at one
 * candidate, 64 absolute differences) of the CUs they searched since the
 * previous call, over every dependent launch of the handle on any stream.
 * CUs whose SADs were summed from their sub-CUs' (LADDER_TUNE_DEP_INHERIT)
 * are not counted, as the SAD tree's larger CUs are not counted for the
 * reference rung.  Waits for `cuda_stream` (launches on other streams are
 * counted once they have run), writes the count to *evals and resets it.
 * LADDER_E_INVAL for a null handle or pointer; LADDER_E_CUDA if the copy
 * fails. */
LADDER_API ladder_status ladder_dependent_evals(ladder_t *ladder, void *cuda_stream, unsigned long long *evals);

/* Test controls for the failure paths (no counterpart in the paper): they
 * exist so that a test can make a bounded device wait run out on purpose and
 * see it reported, with nothing faulting or hanging.
 *   LADDER_DEBUG_WAIT_POLLS    polls of each wavefront wait (spatial MV
 *                              predictor) before it gives up: 0 (default,
 *                              2^22 polls, about a second) or 64 .. 2^22
 *   LADDER_DEBUG_LOST_HANDOFF  1: the wavefront rows wait for a hand-off that
 *                              no row publishes, so every wait of a row
 *                              below the first runs out, sets the device
 *                              status to LADDER_E_TIMEOUT and stops its row
 *                              (the decisions of that launch are not to be
 *                              trusted); 0 (default): normal operation
 * Apply to later launches.  LADDER_E_INVAL for an unknown control or value. */
typedef enum {
    LADDER_DEBUG_WAIT_POLLS = 0,
    LADDER_DEBUG_LOST_HANDOFF = 1
} ladder_debug_control;
LADDER_API ladder_status ladder_set_debug(ladder_t *ladder, int control, int value);

/* Device bytes the handle holds (decision buffers of every frame slot). */
LADDER_API long ladder_device_bytes(const ladder_t *ladder);

/* Independent full search (+-R) of any rung, the per-rung baseline against
 * which the multi-resolution speedup is measured.  Needs no reference; claims
 * a frame slot like analyze_reference, and does not change the frame's
 * reference decisions unless `rung` is the reference rung. */
LADDER_API ladder_status analyze_independent(ladder_t *ladder, int rung, int frame_id, const void *cur,
                                  const void *ref, long pitch_bytes, int qp, void *cuda_stream);

/* Analysis save (the x265 analysis-save side of App. A.1: the decisions a
 * master encode hands to the encodes that reuse them): copies the decisions
 * of (rung, frame_id) into caller-owned host arrays
 * (sizes per ladder_grid); NULL members are skipped.  Waits for the copies on
 * `cuda_stream`, then checks the device status word: LADDER_E_TIMEOUT if a
 * bounded device wait ran out, LADDER_E_STATE if the rung was not analysed. */
LADDER_API ladder_status fetch_decisions(ladder_t *ladder, int rung, int frame_id, ladder_decisions *out,
                              void *cuda_stream);

/* Analysis load (the x265 analysis-load side of App. A.1: encodes that
 * reuse a master encode's analysis read it back instead of analysing
 * again): makes a reference analysis saved by fetch_decisions -- caller-owned
 * HOST arrays of the reference rung, laid out as fetch_decisions writes them,
 * every member up to depth log2(ctu_size/8) set -- the resident reference of
 * frame `frame_id`, as if analyze_reference had produced it: dependents of
 * the frame can then be analysed (resuming a ladder without its reference
 * analysis, e.g. after a restart).  Claims a frame slot like
 * analyze_reference (LADDER_E_BUSY if none is free).  Copies on
 * `cuda_stream` and waits for the copy.  LADDER_E_INVAL for a missing array.
 * The arrays are taken as given: decisions that no analysis of this geometry
 * could give make the dependents' rules read them as they are. */
LADDER_API ladder_status ladder_load_reference(ladder_t *ladder, int frame_id, const ladder_decisions *in,
                                               void *cuda_stream);

/* Cascaded reference chain (Sec. 6.5, the proposed multi-encoding scheme:
 * the refined decisions of one resolution tier are the reference of the
 * next, e.g. 540p -> 1080p -> 2160p).  parent[r] is the rung whose decisions
 * the dependent analysis of rung r refines (its co-located leaf depths and
 * vectors); parent[ref_rung] = -1, and following the parents must lead every
 * rung to the reference rung (no cycles): LADDER_E_INVAL otherwise.  Default
 * at init: the reference rung is every rung's parent.  A dependent analysis
 * needs its parent's analysis of the same frame, resident or in the same
 * call (the library then analyses the rungs tier by tier, parents first):
 * LADDER_E_NOREF otherwise.  Applies to later calls. */
LADDER_API ladder_status ladder_set_parents(ladder_t *ladder, const int *parent);

/* MV predictor of the rate term of later analyses.  mode 0 (default): the
 * predictor (0, 0), every CTU decided independently.  mode 1: a spatial
 * predictor with the wavefront CTU order of WPP (Sec. 2.2: a CTU starts once
 * the CTU above and to its right is done).  The predictor of a CU of size S
 * at (x, y) is the component-wise median of the final leaf vectors at
 * A1 = (x-1, y+S-1), B1 = (x+S-1, y-1) and B0 = (x+S, y-1); a position counts
 * as (0, 0) unless it lies inside the 8-aligned frame, outside the CU's own
 * CTU (one motion estimation region, analysed in parallel) and in the CTU to
 * the left or in the row above at most one column to the right.  bits =
 * se(4 (mvx - pmx)) + se(4 (mvy - pmy)).  The search (SAD) and the SATD do
 * not use the rate, so only cost, best, split and the leaf maps change: after
 * the parallel search and SATD of a batch, one more launch decides them row
 * by row, each row waiting for the row above (a cooperative launch; a wait
 * that runs out sets the device status to LADDER_E_TIMEOUT, read by
 * ladder_sync).  Independent and dependent analyses both take it (a tier's
 * decisions are final before the next tier derives its rules from them);
 * ladder_decide_qps decides every further QP with it too (one wavefront
 * launch per QP, in order); ladder_refine_subpel takes it over the refined
 * quarter-pel vectors (see there); analyze_reference_noalloc keeps the
 * predictor (0, 0).  LADDER_E_INVAL for another mode. */
LADDER_API ladder_status ladder_set_mv_predictor(ladder_t *ladder, int mode);

/* Decisions of one analysed rung at further QPs (intra-resolution analysis
 * sharing, Sec. 4.2: the encodes of one resolution at several QPs share one
 * analysis, with the median QP as the master encode).  The rung's resident
 * motion search and its SATDs at the chosen vectors do not depend on the QP
 * and are shared; for each qps[k] the cost J = SATD + ((lambdaQ16[qps[k]] *
 * bits + 2^15) >> 16), the bottom-up split and the leaf maps are recomputed
 * into out[k].  A dependent rung keeps its rules (derived from the reference
 * decisions of the frame's own analysis).  So out[k] equals what analysing
 * the rung at qps[k] gives for cost, best, split and the leaf maps, given
 * the reference analysed at the master QP.
 *   out[k]: caller-owned DEVICE arrays laid out as the same fields of
 *   ladder_decisions (sizes per ladder_grid); every member for depths
 *   0..dmax must be set.
 * n in 1..LADDER_MAX_QPS, QPs in 0..51 (LADDER_E_INVAL); LADDER_E_STATE if
 * the rung of frame_id has not been analysed.  Asynchronous on
 * `cuda_stream` (one launch); the frame's analysis must be ordered before it
 * on that stream. */
#define LADDER_MAX_QPS 8
typedef struct {
    int32_t *cost[LADDER_MAX_DEPTHS];
    int32_t *best[LADDER_MAX_DEPTHS];
    uint8_t *split[LADDER_MAX_DEPTHS];
    uint8_t *leaf_depth;
    int16_t *leaf_mvx, *leaf_mvy;
} ladder_qp_decisions;
LADDER_API ladder_status ladder_decide_qps(ladder_t *ladder, int rung, int frame_id, int n, const int *qps,
                                           const ladder_qp_decisions *out, void *cuda_stream);

/* Quarter-pel refinement with SATD of one analysed rung (SATD finds the
 * quarter-pel vectors, Sec. 5.4.1).  Every evaluated CU starts at its
 * integer vector (4 mv in quarter-pel units) with its cost; a half-pel round
 * tries the 8 neighbours at +-2 quarter units and a quarter-pel round the 8
 * at +-1 around the best so far, each candidate replacing the best only with
 * a strictly lower cost J = SATD + ((lambdaQ16[qp] * (se(qx) + se(qy)) +
 * 2^15) >> 16) (candidates in raster order).  The prediction at a
 * fractional position is the two-dimensional 8-tap luma filter of HEVC
 * (phases 0, 1/4, 1/2, 3/4) summed exactly and rounded once, clip(floor((sum
 * + 2^11) / 2^12)), the reference clamped to the frame.  The split is then
 * decided again over the refined costs, with the rung's own flags (and a
 * dependent rung's rules).  cur / ref / pitch_bytes: the rung's planes (as
 * analysed); qp: the QP of the analysis.  out: caller-owned DEVICE arrays
 * laid out as the same fields of ladder_decisions, qmvx / qmvy in
 * quarter-pel units (INT16_MIN where not evaluated), satd / cost at the
 * refined vector; every member for depths 0..dmax must be set.
 * With the spatial MV predictor on (ladder_set_mv_predictor mode 1) every
 * candidate's rate, the integer start included, is taken against the
 * predictor of the integer decisions formed from the REFINED quarter-pel
 * leaf vectors: bits = se(qx - pqx) + se(qy - pqy), the CTUs refined in the
 * wavefront order of WPP (Sec. 2.2).  The SATDs of the 48 quarter-pel
 * positions within +-3 of 4 mv are computed first for every evaluated CU,
 * then one more (cooperative) launch decides the CTUs row by row; a wait
 * that runs out sets the device status to LADDER_E_TIMEOUT.  Refinements of
 * one rung of one frame must be ordered (they share its hand-off words).
 * workspace: caller-owned DEVICE scratch of at least
 * ladder_subpel_workspace_bytes(ladder, rung) bytes, 256-byte aligned
 * (LADDER_E_INVAL otherwise), that receives the 16 interpolated phase planes
 * of ref (and the SATD table of the spatial-predictor refinement); calls
 * that share a workspace must be ordered (one stream).  Asynchronous on
 * cuda_stream (two launches: interpolation, refinement; three with the
 * spatial predictor); LADDER_E_STATE if the rung of frame_id has not been
 * analysed. */
typedef struct {
    int16_t *qmvx[LADDER_MAX_DEPTHS], *qmvy[LADDER_MAX_DEPTHS];
    int32_t *satd[LADDER_MAX_DEPTHS], *cost[LADDER_MAX_DEPTHS], *best[LADDER_MAX_DEPTHS];
    uint8_t *split[LADDER_MAX_DEPTHS];
    uint8_t *leaf_depth;
    int16_t *leaf_qmvx, *leaf_qmvy;
} ladder_subpel_decisions;
/* Bytes of the workspace ladder_refine_subpel needs for `rung`: 16 planes
 * of (W + 8) x (H + 8) samples, the positions -4 .. W+3 by -4 .. H+3 of each
 * quarter-pel phase, then 48 int32 SATDs per CU key of every CTU (the
 * spatial-predictor refinement's table; counted in either mode) (0 for a bad
 * handle or rung). */
LADDER_API long ladder_subpel_workspace_bytes(const ladder_t *ladder, int rung);
LADDER_API ladder_status ladder_refine_subpel(ladder_t *ladder, int rung, int frame_id, const void *cur,
                                              const void *ref, long pitch_bytes, int qp,
                                              const ladder_subpel_decisions *out, void *workspace,
                                              long workspace_bytes, void *cuda_stream);

/* Several quarter-pel refinements in one pair of launches (e.g. every rung
 * of a frame): job k is ladder_refine_subpel(ladder, jobs[k].rung,
 * jobs[k].frame_id, jobs[k].cur, jobs[k].ref, jobs[k].pitch_bytes,
 * jobs[k].qp, jobs[k].out, jobs[k].workspace, jobs[k].workspace_bytes),
 * with the same checks; the jobs' workspaces and outputs must not overlap.
 * Small rungs leave most of the GPU idle on their own; batched, their CTAs
 * run beside the large rungs'.  1 <= n <= LADDER_MAX_SUBPEL_JOBS
 * (LADDER_E_INVAL otherwise); nothing is launched if any job fails its
 * checks. */
#define LADDER_MAX_SUBPEL_JOBS 16
typedef struct {
    int frame_id, rung, qp;
    const void *cur, *ref;
    long pitch_bytes;
    const ladder_subpel_decisions *out;
    void *workspace;
    long workspace_bytes;
} ladder_subpel_job;
LADDER_API ladder_status ladder_refine_subpel_batch(ladder_t *ladder, int n, const ladder_subpel_job *jobs,
                                                    void *cuda_stream);

/* Asynchronous fetch of a whole frame (every rung's decisions), for callers
 * that overlap copies with later analyses.  The frame is packed rung after
 * rung, ladder_frame_bytes() bytes in all; ladder_decision_offsets() gives
 * the byte offset, within the packed frame, of each array of a rung:
 * offsets[8*d + k] for depth d = 0..3 and field k = mvx, mvy, sad, satd,
 * cost, best, split, evaluated (-1 past the rung's deepest depth), then
 * offsets[32..34] = leaf_depth, leaf_mvx, leaf_mvy (35 entries, element
 * types and sizes as in ladder_decisions).  ladder_fetch_frame_async
 * enqueues one device-to-host copy per rung on `cuda_stream` into host_dst
 * (caller-owned, `bytes` >= ladder_frame_bytes; pinned memory keeps the
 * copies asynchronous) and returns without waiting: the caller synchronises
 * the stream (or an event) before reading, and orders the frame's next
 * analysis after the copies.  Rungs of the frame that were not analysed are
 * copied as they stand.  LADDER_E_STATE if the frame holds no slot. */
LADDER_API long ladder_frame_bytes(const ladder_t *ladder);
LADDER_API ladder_status ladder_decision_offsets(const ladder_t *ladder, int rung, long *offsets);
LADDER_API ladder_status ladder_fetch_frame_async(ladder_t *ladder, int frame_id, void *host_dst, long bytes,
                                                  void *cuda_stream);

/* Frame pipeline (no counterpart in the paper: the runtime around the
 * analyses that a serving or encoding loop needs, in the spirit of x265's
 * frame threads).  `depth` frame slots (1..8), frame ids base_frame_id ..
 * base_frame_id + depth - 1, each with a device input buffer of in_bytes and
 * its own analysis stream (owned by the pipeline); one upload stream and one
 * read-back stream.  A frame's input is one packed host buffer holding every
 * rung's cur and ref planes: rung r's planes start at cur_off[r] / ref_off[r]
 * with row pitch pitch[r] bytes (offsets 16-byte aligned, pitch a multiple
 * of 16 and >= width * sample bytes, planes inside in_bytes).
 * ladder_pipeline_submit copies host_in (pinned, in_bytes) to the next
 * slot's buffer, analyses the reference rung and then the dependent rungs at
 * qp on the slot's stream, and copies the frame's packed decisions
 * (ladder_frame_bytes, laid out per ladder_decision_offsets) to host_out
 * (pinned).  Uploads, the analyses of neighbouring frames and read-backs
 * overlap.  submit blocks the host only until the slot's previous frame is
 * done (its host_out complete) and returns a ticket; ladder_pipeline_wait
 * returns once the ticket's decisions are in its host_out; host_in may be
 * reused then.  The device status word is read back with every frame's
 * decisions: a bounded device wait that ran out (the decisions of the frames
 * then in flight are not to be trusted) is reported once, as
 * LADDER_E_TIMEOUT, by the wait for a frame that read it back, or else by
 * the next submit that finds it (which then enqueues nothing); the word is
 * cleared when it is reported.  Errors: LADDER_E_INVAL (sizes, layout,
 * depth), LADDER_E_CUDA; the analyses' own errors (LADDER_E_BUSY without
 * free frame slots) pass through. */
typedef struct ladder_pipeline ladder_pipeline_t;
LADDER_API ladder_status ladder_pipeline_create(ladder_t *ladder, int depth, int base_frame_id, long in_bytes,
                                                const long *cur_off, const long *ref_off, const long *pitch,
                                                ladder_pipeline_t **out);
LADDER_API ladder_status ladder_pipeline_submit(ladder_pipeline_t *pipe, const void *host_in, int qp,
                                                void *host_out, long *ticket);
LADDER_API ladder_status ladder_pipeline_wait(ladder_pipeline_t *pipe, long ticket);
/* Waits for the pipeline's work and frees it (not the ladder; destroy every
 * pipeline of a ladder before the ladder itself).  NULL is ignored. */
LADDER_API void ladder_pipeline_destroy(ladder_pipeline_t *pipe);

/* Grid of a rung: dims[2d], dims[2d+1] = cols_d, rows_d for d = 0..dmax, then
 * dims[2(dmax+1)], dims[2(dmax+1)+1] = 8x8 cols, rows; returns dmax in *n_depths - 1.
 * `dims` must hold 2 * LADDER_MAX_DEPTHS + 2 ints. */
LADDER_API ladder_status ladder_grid(const ladder_t *ladder, int rung, int *dims, int *n_depths);

/* Frees the frame slot of `frame_id`: the frame's resident decisions, which
 * stand in for the analysis file the master encode writes for the encodes
 * that reuse it (App. A.1), are no longer needed.
 * Enqueued work that still reads the slot must have completed (ladder_sync). */
LADDER_API ladder_status ladder_release_frame(ladder_t *ladder, int frame_id);

/* Waits for `cuda_stream` and returns the device status word (LADDER_OK or
 * LADDER_E_TIMEOUT), clearing it. */
LADDER_API ladder_status ladder_sync(ladder_t *ladder, void *cuda_stream);

/* Waits for the work the handle's calls enqueued (on the streams they were
 * given, and its graphs' replays), then frees every buffer.  Other work on
 * the device is not waited for.  NULL is ignored. */
LADDER_API void ladder_destroy(ladder_t *ladder);

/* Text of the last error on this handle ("" if none).  Valid until the next call. */
LADDER_API const char *ladder_last_error(const ladder_t *ladder);

/* Tracing.  Every call that enqueues or waits for device work opens an
 * NVTX range named after the call (NVTX 3; free unless a profiler that reads
 * NVTX is attached), so a timeline shows each call beside its kernels.
 * Kernel timing: launches are always counted per kernel kind;
 * when timing is enabled every launch is also bracketed by CUDA events on
 * its own stream (a few microseconds per launch, off by default).  Kinds:
 * 0 full search, 1 SATD/cost/split of an independent rung, 2 refinement
 * search of dependent rungs, 3 key initialisation, 4 dependent constraint
 * derivation (rules, centres, task lists), 5 SATD/cost/split of dependent
 * rungs, 6 cost/split at further QPs (ladder_decide_qps), 7 quarter-pel
 * refinement (ladder_refine_subpel), 8 decisions with the spatial MV
 * predictor (ladder_set_mv_predictor). */
LADDER_API ladder_status ladder_profile_enable(ladder_t *ladder, int enable);

/* Reads the launch count and the summed event time (ms; 0 when timing was
 * off) of kernel kind `kind`, waiting for pending events; clears the kind's
 * counters when `reset` != 0.  LADDER_E_INVAL for an unknown kind. */
LADDER_API ladder_status ladder_profile_read(ladder_t *ladder, int kind, long *launches, double *total_ms,
                                             int reset);

/* Independent analysis of one frame pair that allocates no memory (the
 * paper has no counterpart: this is for callers that cannot call cudaMalloc,
 * such as a plugin inside an application that owns all device memory through
 * its own pool, or a real-time pipeline that forbids allocation after
 * start-up).  Same analysis as analyze_reference on a one-rung ladder of the
 * given geometry, without a ladder handle: `cur` / `ref` are device planes as
 * for analyze_reference, and `out` holds DEVICE pointers to caller-owned
 * decision arrays (every member up to depth log2(ctu_size/8) must be set),
 * which are written asynchronously on `cuda_stream`.
 * Scratch lives in a fixed 2 MiB device array inside the library (every GPU
 * that loads the library holds it until exit): frames of at most 3083 CTUs
 * of 64x64 (a 3840x2160 frame has 2040; about 4x that count at CTU 32) fit; larger ones
 * return LADDER_E_INVAL, like any argument the other entry points refuse.
 * Every call looks up the array's device address in the current device's
 * context; the first lookup in a context loads the module there, so make the
 * first call on a device before any stream capture.  All calls share the
 * array and it keeps the last call's contents (each call resets what must
 * start empty); calls whose work overlaps on the GPU race on it, so order
 * them.  A bounded device wait that runs out (its decisions are then not to
 * be trusted) sets the array's status word, which stays set until
 * analyze_reference_noalloc_status reads it. */
LADDER_API ladder_status analyze_reference_noalloc(const void *cur, const void *ref, int width, int height,
                                                   long pitch_bytes, int bit_depth, int ctu_size, int search_range,
                                                   int qp, int satd_mode, const ladder_decisions *out,
                                                   void *cuda_stream);

/* Status of the allocation-free analyses on the current device since the
 * last query: waits for `cuda_stream` (order it after the calls to check),
 * then returns LADDER_OK, or LADDER_E_TIMEOUT if a bounded device wait of one
 * of them ran out (their decisions are not to be trusted), clearing the
 * status word.  Allocates nothing.  LADDER_E_CUDA if a CUDA call fails. */
LADDER_API ladder_status analyze_reference_noalloc_status(void *cuda_stream);

/* Measures, on the current device, the throughput of the packed
 * absolute-difference accumulate in the form the motion searches issue it
 * (no counterpart in the paper: the denominator of the integer-ALU
 * roofline, confirmed in the same run as the kernels it bounds).
 * bit_depth 8: vabsdiff4 .add, 4 absolute differences per instruction;
 * 10: min.u16x2 + mad.lo, the sum(min(a, b)) term of the 10-bit SAD
 * (sum(a) + sum(b) - 2 sum(min(a, b))), 2 per pair.  Sixteen independent
 * chains per thread, eight 256-thread CTAs per SM, one warm-up and one timed
 * launch with CUDA events on `cuda_stream`; waits for them.  Writes absolute
 * differences per second to *absdiffs_per_s.  LADDER_E_INVAL for another
 * bit depth or a NULL output, LADDER_E_CUDA if a CUDA call fails. */
LADDER_API ladder_status ladder_measure_sad_rate(int bit_depth, void *cuda_stream, double *absdiffs_per_s);

/* Library version string. */
LADDER_API const char *ladder_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LADDER_H */
