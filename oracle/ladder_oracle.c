/*
 * ladder_oracle.c -- plain, slow CPU oracle for the per-CTU inter analysis of
 * multi-resolution encoding: integer full-search block-matching motion
 * estimation (SAD), 8x8 SATD at the chosen vector, the lambda * MV-bits cost
 * and the bottom-up CU quadtree split decision, for an independently analysed
 * representation and for a dependent representation that reuses a reference
 * representation's co-located depth and scaled motion vector.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the bench's
 * CPU-baseline / reference legs load this library.  It shares no code, header,
 * table or constant with the CUDA library; the lambda table below is computed
 * from its formula here, not copied.
 *
 * Every function computes the plain definition: per-CU exhaustive search at
 * every depth (no SAD tree, no sharing of partial sums), explicit Hadamard
 * matrix products, explicit quadtree recursion.  Passages followed:
 *   SAD      -- Sec. 5.4.1, SAD equation; Sec. 5.4.2, plain SAD listing.
 *   SATD     -- Sec. 5.4.1, SATD equation (sum |H| / 2); Sec. 5.4.2, satd8 /
 *               satd_8x4 / HADAMARD4 listings (the PAPER4x4 mode).
 *   quadtree -- Sec. 2.1 (CTU of 64x64 split into CUs of 64..8).
 *   RDO      -- Sec. 2.1 (rate-distortion decision over the quadtree).
 *   reuse    -- Sec. 4.3 and Sec. 6.3 (inter-resolution sharing with
 *               refinement), App. A.1 (--scale-factor, reuse level 10:
 *               quadtree + MVs), App. A.2 (refine level 1: evaluate the
 *               reused depth n and n+1).
 * Readings where the paper is silent (tie-break, lambda, MV bits, SATD
 * normalisation for 8x8, edges, non-dyadic scaling) are the ones listed in
 * the design notes and restated at each function.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXD 4 /* depths 0..3: 64, 32, 16, 8 */

typedef struct {
    int16_t *mvx[OR_MAXD], *mvy[OR_MAXD];
    int32_t *sad[OR_MAXD], *satd[OR_MAXD], *cost[OR_MAXD], *best[OR_MAXD];
    uint8_t *split[OR_MAXD], *evaluated[OR_MAXD];
    uint8_t *leaf_depth;           /* per 8x8, (W8/8) x (H8/8) raster */
    int16_t *leaf_mvx, *leaf_mvy;  /* per 8x8 */
} oracle_decisions;

typedef struct {
    /* frame */
    const void *cur, *ref;
    int width, height;   /* luma samples */
    long pitch;          /* samples per row (both planes) */
    int bit_depth;       /* 8: uint8 samples, 10: uint16 samples */
    /* analysis */
    int ctu;             /* 16, 32 or 64 */
    int qp;              /* 0..51 */
    int satd_mode;       /* 0: HAD8, 1: PAPER4x4 */
    int range;           /* R' : candidates centre +- range */
    /* dependent mode (dep == 0: independent) */
    int dep;
    int ref_width, ref_height;          /* reference rung size */
    const uint8_t *ref_leaf_depth;      /* reference per-8x8 leaf depth */
    const int16_t *ref_leaf_mvx, *ref_leaf_mvy;
    int depth_lo, depth_hi;             /* allowed leaf window [Deq+lo, Deq+hi] */
    int use_ref_mv;                     /* 1: centre = scaled reference MV */
    /* optional CTU sample: analyse only CTUs with ctu_mask[row * cols + col] != 0 */
    const uint8_t *ctu_mask;
    /* MV predictor of the rate term: 0 = (0, 0); 1 = spatial (median of
     * neighbouring leaf vectors, CTUs decided in wavefront order) */
    int mvp;
} oracle_job;

/* ------------------------------------------------------------------ */
/* Samples (edge handling reading): the current block is padded to a   */
/* multiple of 8 by replicating its last column / row; the reference    */
/* is clamped to the frame for any integer position.                   */
/* ------------------------------------------------------------------ */
static int sample_at(const oracle_job *j, const void *plane, int x, int y)
{
    if (j->bit_depth == 8)
        return ((const uint8_t *)plane)[(long)y * j->pitch + x];
    return ((const uint16_t *)plane)[(long)y * j->pitch + x];
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int cur_sample(const oracle_job *j, int x, int y)
{
    return sample_at(j, j->cur, x < j->width ? x : j->width - 1,
                     y < j->height ? y : j->height - 1);
}

static int ref_sample(const oracle_job *j, int x, int y)
{
    return sample_at(j, j->ref, clampi(x, 0, j->width - 1), clampi(y, 0, j->height - 1));
}

/* SAD of an S x S block at (x0, y0) against the reference displaced by
 * (mvx, mvy): sum over the block of |O - P| (Sec. 5.4.1, SAD equation;
 * the plain listing of Sec. 5.4.2 accumulates it row by row in an int). */
static int32_t block_sad(const oracle_job *j, int x0, int y0, int S, int mvx, int mvy)
{
    int32_t sum = 0;
    for (int y = 0; y < S; y++)
        for (int x = 0; x < S; x++) {
            int d = cur_sample(j, x0 + x, y0 + y) - ref_sample(j, x0 + x + mvx, y0 + y + mvy);
            sum += d < 0 ? -d : d;
        }
    return sum;
}

/* ------------------------------------------------------------------ */
/* SATD                                                                 */
/* ------------------------------------------------------------------ */
/* Sylvester Hadamard entry: H_n[i][k] = (-1)^popcount(i & k). */
static int had_entry(int i, int k) { return (__builtin_popcount((unsigned)(i & k)) & 1) ? -1 : 1; }

/* 8x8 Hadamard SATD of a residual block: T = H8 * D * H8^T, result
 * (sum |T|) >> 2 (Sec. 5.4.1 SATD equation applied to an 8x8 transform; the
 * 8x8 transform has twice the gain of the 4x4 one of the listing, so the
 * normalisation is a shift by 2 instead of 1, truncating like the listing). */
int oracle_satd8_had8(const int32_t d[64])
{
    int64_t tmp[8][8], t[8][8], sum = 0;
    for (int u = 0; u < 8; u++)          /* tmp = H8 * D */
        for (int x = 0; x < 8; x++) {
            int64_t s = 0;
            for (int y = 0; y < 8; y++) s += (int64_t)had_entry(u, y) * d[y * 8 + x];
            tmp[u][x] = s;
        }
    for (int u = 0; u < 8; u++)          /* t = tmp * H8^T */
        for (int v = 0; v < 8; v++) {
            int64_t s = 0;
            for (int x = 0; x < 8; x++) s += tmp[u][x] * had_entry(v, x);
            t[u][v] = s;
        }
    for (int u = 0; u < 8; u++)
        for (int v = 0; v < 8; v++) sum += t[u][v] < 0 ? -t[u][v] : t[u][v];
    return (int)(sum >> 2);
}

/* 4x4 Hadamard coefficients' absolute sum of the 4x4 sub-block at (bx, by). */
static int64_t had4_abs_sum(const int32_t d[64], int bx, int by)
{
    int64_t tmp[4][4], sum = 0;
    for (int u = 0; u < 4; u++)
        for (int x = 0; x < 4; x++) {
            int64_t s = 0;
            for (int y = 0; y < 4; y++) s += (int64_t)had_entry(u, y) * d[(by + y) * 8 + bx + x];
            tmp[u][x] = s;
        }
    for (int u = 0; u < 4; u++)
        for (int v = 0; v < 4; v++) {
            int64_t s = 0;
            for (int x = 0; x < 4; x++) s += tmp[u][x] * had_entry(v, x);
            sum += s < 0 ? -s : s;
        }
    return sum;
}

/* PAPER4x4 mode: the satd8 listing tiles the block in 8x4 halves; each half
 * is two 4x4 Hadamards (columns 0-3 and 4-7, packed side by side in the
 * listing) whose absolute coefficient sums are added and halved (Sec. 5.4.2,
 * satd8 / satd_8x4 / HADAMARD4 listings). */
int oracle_satd8_paper4x4(const int32_t d[64])
{
    int total = 0;
    for (int half = 0; half < 2; half++) {
        int64_t s = had4_abs_sum(d, 0, 4 * half) + had4_abs_sum(d, 4, 4 * half);
        total += (int)(s >> 1);
    }
    return total;
}

static int32_t block_satd(const oracle_job *j, int x0, int y0, int S, int mvx, int mvy)
{
    int32_t total = 0, d[64];
    for (int by = 0; by < S; by += 8)
        for (int bx = 0; bx < S; bx += 8) {
            for (int y = 0; y < 8; y++)
                for (int x = 0; x < 8; x++)
                    d[y * 8 + x] = cur_sample(j, x0 + bx + x, y0 + by + y) -
                                   ref_sample(j, x0 + bx + x + mvx, y0 + by + y + mvy);
            total += j->satd_mode == 1 ? oracle_satd8_paper4x4(d) : oracle_satd8_had8(d);
        }
    return total;
}

/* ------------------------------------------------------------------ */
/* Rate term (readings; the paper does not define the estimate)         */
/* ------------------------------------------------------------------ */
/* Length of the signed Exp-Golomb code se(v). */
int oracle_se_bits(int v)
{
    long k = v > 0 ? 2L * v - 1 : -2L * v;
    int n = 0;
    while ((k + 1) >> (n + 1)) n++;   /* n = floor(log2(k + 1)) */
    return 2 * n + 1;
}

/* MV bits: se(v) of each quarter-pel component, predictor (0, 0). */
int oracle_mv_bits(int mvx, int mvy) { return oracle_se_bits(4 * mvx) + oracle_se_bits(4 * mvy); }

/* Lambda in Q16: round(65536 * sqrt(0.57 * 2^((qp - 12) / 3))) -- the
 * SAD-domain lambda of common HEVC encoders; computed from the formula. */
long long oracle_lambda_q16(int qp)
{
    double lam = sqrt(0.57 * pow(2.0, (qp - 12) / 3.0));
    return (long long)floor(65536.0 * lam + 0.5);
}

/* J = SATD + round(lambda * bits) with lambda in Q16 (int64 product). */
static int32_t rd_cost(int32_t satd, int qp, int mvx, int mvy)
{
    long long prod = oracle_lambda_q16(qp) * (long long)oracle_mv_bits(mvx, mvy);
    return satd + (int32_t)((prod + 32768) >> 16);
}

/* Spatial MV predictor (reading for the wavefront CTU order of WPP,
 * Sec. 2.2: a CTU starts once the CTU above and to its right is done).
 * The predictor of the CU of size S at (x0, y0) is the component-wise
 * median of the final leaf vectors at three neighbouring positions, as in
 * the spatial candidates of HEVC's AMVP:
 *   A1 = (x0 - 1, y0 + S - 1)   left of the CU's bottom-left sample
 *   B1 = (x0 + S - 1, y0 - 1)   above the CU's top-right sample
 *   B0 = (x0 + S, y0 - 1)       above-right
 * A position counts as vector (0, 0) unless it is available: inside the
 * 8-aligned frame, outside the CU's own CTU (the CTU is one motion
 * estimation region whose CUs are analysed in parallel), and in a CTU that
 * is decided before the CU's CTU in wavefront order -- the CTU to the left
 * in the same row, or a CTU of the row above at most one column to the
 * right.  leaf_mvx / leaf_mvy: the frame's per-8x8 leaf vectors (only the
 * available positions are read). */
static int med3(int a, int b, int c)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return c < lo ? lo : (c > hi ? hi : c);
}

static int mvp_available(int ctu, int W8, int H8, int x0, int y0, int px, int py)
{
    if (px < 0 || py < 0 || px >= W8 || py >= H8) return 0;
    int cx = x0 / ctu, cy = y0 / ctu, qx = px / ctu, qy = py / ctu;
    if (qx == cx && qy == cy) return 0;
    if (qy == cy) return qx < cx;
    if (qy == cy - 1) return qx <= cx + 1;
    return qy < cy - 1;
}

static void spatial_mvp(int ctu, int W8, int H8, const int16_t *leaf_mvx, const int16_t *leaf_mvy, int x0,
                        int y0, int S, int *pmx, int *pmy)
{
    const int px[3] = {x0 - 1, x0 + S - 1, x0 + S};
    const int py[3] = {y0 + S - 1, y0 - 1, y0 - 1};
    int vx[3], vy[3], cols8 = W8 / 8;
    for (int k = 0; k < 3; k++) {
        vx[k] = vy[k] = 0;
        if (mvp_available(ctu, W8, H8, x0, y0, px[k], py[k])) {
            long li = (long)(py[k] / 8) * cols8 + px[k] / 8;
            vx[k] = leaf_mvx[li];
            vy[k] = leaf_mvy[li];
        }
    }
    *pmx = med3(vx[0], vx[1], vx[2]);
    *pmy = med3(vy[0], vy[1], vy[2]);
}

/* J with the predictor (pmx, pmy): bits = se() lengths of the quarter-pel
 * components of the vector minus the predictor. */
static int32_t rd_cost_pred(int32_t satd, int qp, int mvx, int mvy, int pmx, int pmy)
{
    long long bits = oracle_se_bits(4 * (mvx - pmx)) + oracle_se_bits(4 * (mvy - pmy));
    return satd + (int32_t)((oracle_lambda_q16(qp) * bits + 32768) >> 16);
}

/* ------------------------------------------------------------------ */
/* Dependent-mode constraint derivation (Sec. 4.3 / 6.3, App. A.1-A.2)  */
/* ------------------------------------------------------------------ */
static int scale_mv(int v, int to, int from)
{
    /* sign(v) * floor((2|v| * to + from) / (2 from)): round half away */
    long a = v < 0 ? -(long)v : v;
    long s = (2 * a * to + from) / (2L * from);
    int r = (int)(v < 0 ? -s : s);
    return clampi(r, -256, 256);
}

typedef struct { int cx, cy, allowed_leaf, allowed_split; } cu_rule;

static int ilog2i(int v) { int n = 0; while ((1 << (n + 1)) <= v) n++; return n; }

static cu_rule derive_rule(const oracle_job *j, int d, int x0, int y0)
{
    int dmax = ilog2i(j->ctu / 8);
    int S = j->ctu >> d;
    cu_rule r;
    if (!j->dep) {
        r.cx = r.cy = 0;
        r.allowed_leaf = 1;
        r.allowed_split = d < dmax;
        return r;
    }
    int Wd = j->width, Hd = j->height, Wr = j->ref_width, Hr = j->ref_height;
    /* co-located point of the CU centre in the reference rung */
    long xm = ((long)(2 * x0 + S) * Wr) / (2L * Wd);
    long ym = ((long)(2 * y0 + S) * Hr) / (2L * Hd);
    xm = xm < 0 ? 0 : (xm > Wr - 1 ? Wr - 1 : xm);
    ym = ym < 0 ? 0 : (ym > Hr - 1 ? Hr - 1 : ym);
    int cols_r = (Wr + 7) / 8;
    long li = (ym >> 3) * cols_r + (xm >> 3);
    int depth_r = j->ref_leaf_depth[li];
    int mvx_r = j->ref_leaf_mvx[li], mvy_r = j->ref_leaf_mvy[li];
    if (j->use_ref_mv) {
        r.cx = scale_mv(mvx_r, Wd, Wr);
        r.cy = scale_mv(mvy_r, Hd, Hr);
    } else {
        r.cx = r.cy = 0;
    }
    /* Deq: the smallest CU that still covers the projected reference leaf */
    int sz_r = j->ctu >> depth_r, deq = 0;
    for (int dd = 0; dd <= dmax; dd++)
        if ((long)(j->ctu >> dd) * Wr >= (long)sz_r * Wd) deq = dd;
    r.allowed_split = d < dmax && d < deq + j->depth_hi;
    r.allowed_leaf = (deq + j->depth_lo <= d && d <= deq + j->depth_hi) || d == dmax || !r.allowed_split;
    return r;
}

/* ------------------------------------------------------------------ */
/* Per-CU motion search and quadtree decision                           */
/* ------------------------------------------------------------------ */
typedef struct {
    const oracle_job *job;
    oracle_decisions *out;
    int W8, H8, dmax, ctu_cols, ctu_rows;
    int next_row;
    pthread_mutex_t lock;
} oracle_ctx;

static int grid_cols(const oracle_ctx *c, int d) { int S = c->job->ctu >> d; return (c->W8 + S - 1) / S; }

/* Full search: argmin over candidates centre + (dx, dy), |dx|,|dy| <= range,
 * of the key (SAD, |dx|+|dy|, dy, dx) compared lexicographically (tie-break
 * reading: among equal SADs prefer the smallest offset, then raster order). */
static void motion_search(const oracle_job *j, int x0, int y0, int S, int cx, int cy,
                          int *bmx, int *bmy, int32_t *bsad)
{
    int R = j->range;
    int32_t best = INT32_MAX;
    int bl1 = 0, bdy = 0, bdx = 0, have = 0;
    for (int dy = -R; dy <= R; dy++)
        for (int dx = -R; dx <= R; dx++) {
            int32_t s = block_sad(j, x0, y0, S, cx + dx, cy + dy);
            int l1 = abs(dx) + abs(dy);
            int better = !have || s < best ||
                         (s == best && (l1 < bl1 || (l1 == bl1 && (dy < bdy || (dy == bdy && dx < bdx)))));
            if (better) { best = s; bl1 = l1; bdy = dy; bdx = dx; have = 1; }
        }
    *bmx = cx + bdx;
    *bmy = cy + bdy;
    *bsad = best;
}

/* Analyse the CU (d, x0, y0) of one CTU and, recursively, its children;
 * returns best(CU).  A CU is reachable when every ancestor may split (the
 * root always is); it is evaluated (motion search + cost) when it is
 * reachable, inside the 8-aligned frame and allowed as a leaf.  Split
 * reading: a reachable CU splits iff it is forced (partial CU), or it may
 * split and either it is not evaluated or its children's best sum is
 * strictly smaller than its own J (ties keep the larger CU). */
static int32_t analyse_cu(oracle_ctx *c, int d, int x0, int y0, int reachable)
{
    const oracle_job *j = c->job;
    oracle_decisions *o = c->out;
    int S = j->ctu >> d;
    long idx = (long)(y0 / S) * grid_cols(c, d) + x0 / S;
    int inside = x0 + S <= c->W8 && y0 + S <= c->H8;
    cu_rule rule = derive_rule(j, d, x0, y0);
    int evaluated = reachable && inside && rule.allowed_leaf;
    int32_t J = INT32_MAX;

    o->evaluated[d][idx] = (uint8_t)evaluated;
    if (evaluated) {
        int mvx, mvy;
        int32_t sad;
        motion_search(j, x0, y0, S, rule.cx, rule.cy, &mvx, &mvy, &sad);
        int32_t satd = block_satd(j, x0, y0, S, mvx, mvy);
        if (j->mvp) {
            int pmx, pmy;
            spatial_mvp(j->ctu, c->W8, c->H8, o->leaf_mvx, o->leaf_mvy, x0, y0, S, &pmx, &pmy);
            J = rd_cost_pred(satd, j->qp, mvx, mvy, pmx, pmy);
        } else {
            J = rd_cost(satd, j->qp, mvx, mvy);
        }
        o->mvx[d][idx] = (int16_t)mvx;
        o->mvy[d][idx] = (int16_t)mvy;
        o->sad[d][idx] = sad;
        o->satd[d][idx] = satd;
        o->cost[d][idx] = J;
    } else {
        o->mvx[d][idx] = INT16_MIN;
        o->mvy[d][idx] = INT16_MIN;
        o->sad[d][idx] = INT32_MAX;
        o->satd[d][idx] = INT32_MAX;
        o->cost[d][idx] = INT32_MAX;
    }
    if (d == c->dmax) {
        o->best[d][idx] = J;
        return J;
    }
    int forced = !inside;
    int can_split = reachable && (forced || rule.allowed_split);
    int32_t children = 0;
    int h = S / 2;
    for (int q = 0; q < 4; q++) {
        int cx0 = x0 + (q & 1) * h, cy0 = y0 + (q >> 1) * h;
        if (cx0 < c->W8 && cy0 < c->H8) {
            int32_t b = analyse_cu(c, d + 1, cx0, cy0, can_split);
            if (can_split) children += b;
        }
    }
    int split = can_split && (!evaluated || children < J);
    o->split[d][idx] = (uint8_t)split;
    int32_t best = !reachable ? INT32_MAX : (split ? children : J);
    o->best[d][idx] = best;
    return best;
}

/* Leaf depth / MV of every 8x8: follow the split flags down from the CTU. */
static void fill_leaves(oracle_ctx *c, int d, int x0, int y0)
{
    const oracle_job *j = c->job;
    oracle_decisions *o = c->out;
    int S = j->ctu >> d;
    long idx = (long)(y0 / S) * grid_cols(c, d) + x0 / S;
    if (d < c->dmax && o->split[d][idx]) {
        int h = S / 2;
        for (int q = 0; q < 4; q++) {
            int cx0 = x0 + (q & 1) * h, cy0 = y0 + (q >> 1) * h;
            if (cx0 < c->W8 && cy0 < c->H8) fill_leaves(c, d + 1, cx0, cy0);
        }
        return;
    }
    int cols8 = c->W8 / 8;
    for (int y = y0; y < y0 + S && y < c->H8; y += 8)
        for (int x = x0; x < x0 + S && x < c->W8; x += 8) {
            long li = (long)(y / 8) * cols8 + x / 8;
            o->leaf_depth[li] = (uint8_t)d;
            o->leaf_mvx[li] = o->mvx[d][idx];
            o->leaf_mvy[li] = o->mvy[d][idx];
        }
}

static void *worker(void *arg)
{
    oracle_ctx *c = (oracle_ctx *)arg;
    for (;;) {
        pthread_mutex_lock(&c->lock);
        int row = c->next_row++;
        pthread_mutex_unlock(&c->lock);
        if (row >= c->ctu_rows) break;
        for (int col = 0; col < c->ctu_cols; col++) {
            if (c->job->ctu_mask && !c->job->ctu_mask[row * c->ctu_cols + col]) continue;
            int x0 = col * c->job->ctu, y0 = row * c->job->ctu;
            analyse_cu(c, 0, x0, y0, 1);
            fill_leaves(c, 0, x0, y0);
        }
    }
    return NULL;
}

static int valid_job(const oracle_job *j)
{
    if (!j || !j->cur || !j->ref) return 0;
    if (j->width <= 0 || j->height <= 0 || j->pitch < j->width) return 0;
    if (j->bit_depth != 8 && j->bit_depth != 10) return 0;
    if (j->ctu != 16 && j->ctu != 32 && j->ctu != 64) return 0;
    if (j->qp < 0 || j->qp > 51 || j->range < 0 || j->range > 128) return 0;
    if (j->dep && (!j->ref_leaf_depth || !j->ref_leaf_mvx || !j->ref_leaf_mvy ||
                   j->ref_width <= 0 || j->ref_height <= 0)) return 0;
    if (j->mvp != 0 && j->mvp != 1) return 0;
    if (j->mvp && j->ctu_mask) return 0;  /* predictors need every earlier CTU */
    return 1;
}

/* Analyse one frame pair; returns 0 on success, -1 on invalid arguments.
 * threads <= 0 means one thread. */
int oracle_analyze(const oracle_job *job, oracle_decisions *out, int threads)
{
    if (!valid_job(job) || !out) return -1;
    oracle_ctx c;
    memset(&c, 0, sizeof c);
    c.job = job;
    c.out = out;
    c.W8 = (job->width + 7) / 8 * 8;
    c.H8 = (job->height + 7) / 8 * 8;
    c.dmax = ilog2i(job->ctu / 8);
    c.ctu_cols = (c.W8 + job->ctu - 1) / job->ctu;
    c.ctu_rows = (c.H8 + job->ctu - 1) / job->ctu;
    pthread_mutex_init(&c.lock, NULL);
    /* spatial predictor: CTUs one by one in raster order (every CTU a CU's
     * predictor reads is decided before it) */
    if (threads <= 1 || job->mvp) {
        worker(&c);
    } else {
        pthread_t *t = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
        if (!t) return -1;
        for (int i = 0; i < threads; i++) pthread_create(&t[i], NULL, worker, &c);
        for (int i = 0; i < threads; i++) pthread_join(t[i], NULL);
        free(t);
    }
    pthread_mutex_destroy(&c.lock);
    return 0;
}

/* Probe: the spatial predictor of the CU (S at x0, y0) of a width x height
 * frame with CTU size ctu, over caller-given per-8x8 leaf vectors. */
void oracle_spatial_mvp(int width, int height, int ctu, const int16_t *leaf_mvx, const int16_t *leaf_mvy, int x0,
                        int y0, int S, int out[2])
{
    spatial_mvp(ctu, (width + 7) / 8 * 8, (height + 7) / 8 * 8, leaf_mvx, leaf_mvy, x0, y0, S, &out[0], &out[1]);
}

/* Single-CU probes used by the pinning tests. */
int32_t oracle_block_sad(const oracle_job *job, int x0, int y0, int S, int mvx, int mvy)
{
    return block_sad(job, x0, y0, S, mvx, mvy);
}

int32_t oracle_block_satd(const oracle_job *job, int x0, int y0, int S, int mvx, int mvy)
{
    return block_satd(job, x0, y0, S, mvx, mvy);
}

/* Constraint derivation probe: fills (cx, cy, allowed_leaf, allowed_split). */
void oracle_derive_rule(const oracle_job *job, int d, int x0, int y0, int out[4])
{
    cu_rule r = derive_rule(job, d, x0, y0);
    out[0] = r.cx; out[1] = r.cy; out[2] = r.allowed_leaf; out[3] = r.allowed_split;
}

/* ------------------------------------------------------------------ */
/* Quarter-pel refinement with SATD around the integer vector           */
/* (Sec. 5.4.1: SAD finds the integer vectors, SATD the quarter-pel     */
/* ones; the interpolation filters are among the kernels the encoder    */
/* accelerates, Sec. 6.6).  Readings, the paper giving no filter or     */
/* search pattern: the 8-tap luma filters of HEVC for the phases 0,     */
/* 1/4, 1/2, 3/4, applied as the exact two-dimensional separable sum    */
/* and rounded once; a half-pel round (the 8 neighbours at +-2 quarter  */
/* units) then a quarter-pel round (+-1) around the best so far, each   */
/* keeping the current best unless a candidate's cost is strictly lower */
/* (candidates in raster order, dy then dx); cost = SATD + lambda *     */
/* se-bits of the quarter-pel components.  The split is then decided    */
/* again over the refined costs.                                        */
/* ------------------------------------------------------------------ */
static const int OR_FILT[4][8] = {
    {0, 0, 0, 64, 0, 0, 0, 0},
    {-1, 4, -10, 58, 17, -5, 1, 0},
    {-1, 4, -11, 40, 40, -11, 4, -1},
    {0, 1, -5, 17, 58, -10, 4, -1},
};

static int floor_div4(int v) { return v >= 0 ? v / 4 : -((-v + 3) / 4); }

/* Prediction of the sample at (x, y) displaced by the quarter-pel vector
 * (qx, qy): P = clip((sum_j f_fy[j] sum_i f_fx[i] Ref(X+i-3, Y+j-3) + 2^11)
 * >> 12), X = x + floor(qx / 4), fx = qx - 4 floor(qx / 4) (likewise y);
 * Ref clamped to the frame.  At an integer vector P is the sample itself. */
static int pred_sample(const oracle_job *j, int x, int y, int qx, int qy)
{
    int X = x + floor_div4(qx), Y = y + floor_div4(qy);
    int fx = qx - 4 * floor_div4(qx), fy = qy - 4 * floor_div4(qy);
    long long sum = 0;
    for (int jj = 0; jj < 8; jj++)
        for (int ii = 0; ii < 8; ii++)
            sum += (long long)OR_FILT[fy][jj] * OR_FILT[fx][ii] * ref_sample(j, X + ii - 3, Y + jj - 3);
    long long p = sum + 2048;
    p = p >= 0 ? p / 4096 : -((-p + 4095) / 4096);  /* floor */
    long long maxv = (1 << j->bit_depth) - 1;
    return (int)(p < 0 ? 0 : (p > maxv ? maxv : p));
}

/* SATD of the S x S CU at (x0, y0) against the quarter-pel prediction. */
static int32_t block_satd_q(const oracle_job *j, int x0, int y0, int S, int qx, int qy)
{
    int32_t total = 0, d[64];
    for (int by = 0; by < S; by += 8)
        for (int bx = 0; bx < S; bx += 8) {
            for (int y = 0; y < 8; y++)
                for (int x = 0; x < 8; x++)
                    d[y * 8 + x] = cur_sample(j, x0 + bx + x, y0 + by + y) -
                                   pred_sample(j, x0 + bx + x, y0 + by + y, qx, qy);
            total += j->satd_mode == 1 ? oracle_satd8_paper4x4(d) : oracle_satd8_had8(d);
        }
    return total;
}

/* J = SATD + round(lambda * (se(qx) + se(qy))), the components in quarter-pel units. */
static int32_t rd_cost_q(int32_t satd, int qp, int qx, int qy)
{
    long long prod = oracle_lambda_q16(qp) * (long long)(oracle_se_bits(qx) + oracle_se_bits(qy));
    return satd + (int32_t)((prod + 32768) >> 16);
}

typedef struct {
    int16_t *qmvx[OR_MAXD], *qmvy[OR_MAXD];
    int32_t *satd[OR_MAXD], *cost[OR_MAXD], *best[OR_MAXD];
    uint8_t *split[OR_MAXD];
    uint8_t *leaf_depth;
    int16_t *leaf_qmvx, *leaf_qmvy;
} oracle_subpel;

typedef struct {
    const oracle_job *job;
    const oracle_decisions *in;
    oracle_subpel *out;
    int W8, H8, dmax, ctu_cols, ctu_rows;
    int next_row;
    pthread_mutex_t lock;
} subpel_ctx;

static int grid_cols_s(const subpel_ctx *c, int d) { int S = c->job->ctu >> d; return (c->W8 + S - 1) / S; }

/* The two rounds of one evaluated CU, from its integer vector and SATD;
 * (pqx, pqy): the predictor of the rate term, quarter-pel units ((0, 0)
 * unless the spatial predictor is on). */
static void subpel_search(const oracle_job *j, int x0, int y0, int S, int mvx, int mvy, int32_t satd0, int pqx,
                          int pqy, int *oqx, int *oqy, int32_t *osatd, int32_t *oj)
{
    int bx = 4 * mvx, by = 4 * mvy;
    int32_t bs = satd0, bj = rd_cost_q(satd0, j->qp, bx - pqx, by - pqy);
    for (int step = 2; step >= 1; step--) {
        int cx = bx, cy = by;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                if (!dx && !dy) continue;
                int qx = cx + step * dx, qy = cy + step * dy;
                int32_t s = block_satd_q(j, x0, y0, S, qx, qy);
                int32_t J = rd_cost_q(s, j->qp, qx - pqx, qy - pqy);
                if (J < bj) { bj = J; bs = s; bx = qx; by = qy; }
            }
    }
    *oqx = bx; *oqy = by; *osatd = bs; *oj = bj;
}

/* The quadtree again (same reachability, rules and forced splits as
 * analyse_cu), with each evaluated CU's cost taken after its refinement. */
static int32_t refine_cu(subpel_ctx *c, int d, int x0, int y0, int reachable)
{
    const oracle_job *j = c->job;
    oracle_subpel *o = c->out;
    int S = j->ctu >> d;
    long idx = (long)(y0 / S) * grid_cols_s(c, d) + x0 / S;
    int inside = x0 + S <= c->W8 && y0 + S <= c->H8;
    cu_rule rule = derive_rule(j, d, x0, y0);
    int evaluated = c->in->evaluated[d][idx];
    int32_t J = INT32_MAX;
    if (evaluated) {
        int qx, qy, pqx = 0, pqy = 0;
        int32_t s;
        /* spatial predictor: the median of the refined quarter-pel leaf
         * vectors of the earlier CTUs, read as the integer analysis reads
         * its leaf vectors */
        if (j->mvp) spatial_mvp(j->ctu, c->W8, c->H8, o->leaf_qmvx, o->leaf_qmvy, x0, y0, S, &pqx, &pqy);
        subpel_search(j, x0, y0, S, c->in->mvx[d][idx], c->in->mvy[d][idx], c->in->satd[d][idx], pqx, pqy, &qx,
                      &qy, &s, &J);
        o->qmvx[d][idx] = (int16_t)qx;
        o->qmvy[d][idx] = (int16_t)qy;
        o->satd[d][idx] = s;
        o->cost[d][idx] = J;
    } else {
        o->qmvx[d][idx] = INT16_MIN;
        o->qmvy[d][idx] = INT16_MIN;
        o->satd[d][idx] = INT32_MAX;
        o->cost[d][idx] = INT32_MAX;
    }
    if (d == c->dmax) {
        o->best[d][idx] = J;
        return J;
    }
    int forced = !inside;
    int can_split = reachable && (forced || rule.allowed_split);
    int32_t children = 0;
    int h = S / 2;
    for (int q = 0; q < 4; q++) {
        int cx0 = x0 + (q & 1) * h, cy0 = y0 + (q >> 1) * h;
        if (cx0 < c->W8 && cy0 < c->H8) {
            int32_t b = refine_cu(c, d + 1, cx0, cy0, can_split);
            if (can_split) children += b;
        }
    }
    int split = can_split && (!evaluated || children < J);
    o->split[d][idx] = (uint8_t)split;
    int32_t best = !reachable ? INT32_MAX : (split ? children : J);
    o->best[d][idx] = best;
    return best;
}

static void refine_leaves(subpel_ctx *c, int d, int x0, int y0)
{
    const oracle_job *j = c->job;
    oracle_subpel *o = c->out;
    int S = j->ctu >> d;
    long idx = (long)(y0 / S) * grid_cols_s(c, d) + x0 / S;
    if (d < c->dmax && o->split[d][idx]) {
        int h = S / 2;
        for (int q = 0; q < 4; q++) {
            int cx0 = x0 + (q & 1) * h, cy0 = y0 + (q >> 1) * h;
            if (cx0 < c->W8 && cy0 < c->H8) refine_leaves(c, d + 1, cx0, cy0);
        }
        return;
    }
    int cols8 = c->W8 / 8;
    for (int y = y0; y < y0 + S && y < c->H8; y += 8)
        for (int x = x0; x < x0 + S && x < c->W8; x += 8) {
            long li = (long)(y / 8) * cols8 + x / 8;
            o->leaf_depth[li] = (uint8_t)d;
            o->leaf_qmvx[li] = o->qmvx[d][idx];
            o->leaf_qmvy[li] = o->qmvy[d][idx];
        }
}

static void *refine_worker(void *arg)
{
    subpel_ctx *c = (subpel_ctx *)arg;
    for (;;) {
        pthread_mutex_lock(&c->lock);
        int row = c->next_row++;
        pthread_mutex_unlock(&c->lock);
        if (row >= c->ctu_rows) break;
        for (int col = 0; col < c->ctu_cols; col++) {
            int x0 = col * c->job->ctu, y0 = row * c->job->ctu;
            refine_cu(c, 0, x0, y0, 1);
            refine_leaves(c, 0, x0, y0);
        }
    }
    return NULL;
}

/* Quarter-pel refinement of an analysis `in` of the same job (its integer
 * vectors, SATDs and evaluated flags); returns 0, or -1 on bad arguments.
 * With the spatial predictor (job->mvp) the rate term of every candidate
 * takes the predictor of the integer analysis, formed from the refined
 * quarter-pel leaf vectors, and the CTUs are refined one by one in raster
 * order (every CTU a predictor reads is refined before the CU's CTU). */
int oracle_refine_subpel(const oracle_job *job, const oracle_decisions *in, oracle_subpel *out, int threads)
{
    if (!valid_job(job) || !in || !out) return -1;
    subpel_ctx c;
    memset(&c, 0, sizeof c);
    c.job = job;
    c.in = in;
    c.out = out;
    c.W8 = (job->width + 7) / 8 * 8;
    c.H8 = (job->height + 7) / 8 * 8;
    c.dmax = ilog2i(job->ctu / 8);
    c.ctu_cols = (c.W8 + job->ctu - 1) / job->ctu;
    c.ctu_rows = (c.H8 + job->ctu - 1) / job->ctu;
    pthread_mutex_init(&c.lock, NULL);
    if (threads <= 1 || job->mvp) {
        refine_worker(&c);
    } else {
        pthread_t *t = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
        if (!t) return -1;
        for (int i = 0; i < threads; i++) pthread_create(&t[i], NULL, refine_worker, &c);
        for (int i = 0; i < threads; i++) pthread_join(t[i], NULL);
        free(t);
    }
    pthread_mutex_destroy(&c.lock);
    return 0;
}

/* Probes for the pinning tests. */
int oracle_pred_sample(const oracle_job *job, int x, int y, int qx, int qy)
{
    return pred_sample(job, x, y, qx, qy);
}

int32_t oracle_block_satd_q(const oracle_job *job, int x0, int y0, int S, int qx, int qy)
{
    return block_satd_q(job, x0, y0, S, qx, qy);
}
