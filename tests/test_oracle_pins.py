"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

Each check is chosen so that a plausible slip in the oracle (dropped term,
wrong sign or index, transposed operand, wrong clamp, wrong tie-break, wrong
rounding) fails at least one of them.  Nothing here calls the CUDA library.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2301_12191_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- SATD ----
def _golden_block(kind, p):
    y, x = np.mgrid[0:8, 0:8]
    if kind == "constant":
        return np.full((8, 8), p)
    if kind == "impulse":
        b = np.zeros((8, 8), dtype=np.int64)
        b[3, 5] = p
        return b
    if kind == "checkerboard":
        return p * (-1) ** (x + y)
    if kind == "rowstripes":
        return p * (-1) ** y
    raise ValueError(kind)


@pytest.mark.parametrize("row", _golden_rows("satd_blocks.txt"))
def test_satd_hand_values(row):
    kind, p, had8, p4 = row[0], int(row[1]), int(row[2]), int(row[3])
    b = _golden_block(kind, p)
    assert oracle.satd8(b, 0) == had8
    assert oracle.satd8(b, 1) == p4


def test_satd_impulse_any_position():
    # every coefficient of an impulse's 8x8 Hadamard has magnitude |v|
    for pos in range(64):
        b = np.zeros(64, dtype=np.int32)
        b[pos] = -7
        assert oracle.satd8(b, 0) == 16 * 7
        assert oracle.satd8(b, 1) == 8 * 7


def test_satd_matches_scipy_hadamard():
    rng = np.random.default_rng(1)
    H8 = scipy.linalg.hadamard(8).astype(np.int64)
    H4 = scipy.linalg.hadamard(4).astype(np.int64)
    for _ in range(300):
        lim = int(rng.choice([3, 255, 1023]))
        D = rng.integers(-lim, lim + 1, size=(8, 8)).astype(np.int64)
        T = H8 @ D @ H8.T
        assert oracle.satd8(D, 0) == int(np.abs(T).sum()) >> 2
        # Parseval for the unnormalised transform: sum T^2 = 64 sum D^2
        assert int((T * T).sum()) == 64 * int((D * D).sum())
        p4 = 0
        for r0 in (0, 4):
            s = 0
            for c0 in (0, 4):
                blk = D[r0:r0 + 4, c0:c0 + 4]
                s += int(np.abs(H4 @ blk @ H4.T).sum())
            p4 += s >> 1
        assert oracle.satd8(D, 1) == p4


def test_satd_transpose_and_sign_invariance():
    rng = np.random.default_rng(2)
    for _ in range(50):
        D = rng.integers(-255, 256, size=(8, 8))
        v = oracle.satd8(D, 0)
        assert oracle.satd8(D.T, 0) == v
        assert oracle.satd8(-D, 0) == v


# ---------------------------------------------------------- bits, lambda ----
def test_exp_golomb_textbook_lengths():
    # se(v): codeNum k = 2v-1 (v>0) or -2v; length 2*floor(log2(k+1))+1
    table = {0: 1, 1: 3, -1: 3, 2: 5, -2: 5, 3: 5, 4: 7, -4: 7, 7: 7, 8: 9, -8: 9, 16: 11}
    for v, n in table.items():
        assert oracle.se_bits(v) == n, v
    for v in range(-300, 301):
        k = 2 * v - 1 if v > 0 else -2 * v
        assert oracle.se_bits(v) == 2 * (len(bin(k + 1)) - 3) + 1
    assert oracle.mv_bits(0, 0) == 2
    assert oracle.mv_bits(1, 0) == 7 + 1      # 4 quarter-pel -> 7 bits
    assert oracle.mv_bits(-1, -1) == 14


def test_lambda_anchors_and_doubling():
    for qp, val in _golden_rows("lambda_anchors.txt"):
        assert oracle.lambda_q16(int(qp)) == int(val)
    lam = [oracle.lambda_q16(q) for q in range(52)]
    assert all(a < b for a, b in zip(lam, lam[1:]))
    for q in range(46):   # doubles every 6 QP, up to the two roundings
        assert abs(lam[q + 6] - 2 * lam[q]) <= 2


def test_library_lambda_table_equals_the_oracle():
    """The CUDA library keeps lambda as a frozen integer table (written once
    by its generator script); the oracle computes it from the formula.  The
    two copies must agree at every QP."""
    import re
    path = os.path.join(os.path.dirname(GOLDEN), os.pardir, "paper_2301_12191_gb300", "csrc", "lambda_table.inc")
    with open(path) as f:
        body = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    table = [int(v) for v in re.findall(r"-?\d+", body)]
    assert len(table) == 52
    assert table == [oracle.lambda_q16(q) for q in range(52)]


# ------------------------------------------------------------ helpers ----
def _brute_indep(cur, ref, R, ctu):
    """Exhaustive search written independently: edge-padded planes and a
    lexsort over (SAD, L1, dy, dx)."""
    H, W = cur.shape
    W8, H8 = (W + 7) // 8 * 8, (H + 7) // 8 * 8
    cp = np.pad(cur.astype(np.int64), ((0, H8 - H), (0, W8 - W)), mode="edge")
    P = R + ctu + 8
    rp = np.pad(ref.astype(np.int64), ((P, P + H8 - H), (P, P + W8 - W)), mode="edge")
    dmax = int(math.log2(ctu // 8))
    offs = [(dx, dy) for dy in range(-R, R + 1) for dx in range(-R, R + 1)]
    res = []
    for d in range(dmax + 1):
        S = ctu >> d
        cols, rows = -(-W8 // S), -(-H8 // S)
        mv = np.full((rows * cols, 2), -32768, dtype=np.int64)
        sad = np.full(rows * cols, 2**31 - 1, dtype=np.int64)
        for r in range(rows):
            for c in range(cols):
                x0, y0 = c * S, r * S
                if x0 + S > W8 or y0 + S > H8:
                    continue
                blk = cp[y0:y0 + S, x0:x0 + S]
                sads = np.array([np.abs(blk - rp[P + y0 + dy:P + y0 + dy + S,
                                                 P + x0 + dx:P + x0 + dx + S]).sum()
                                 for dx, dy in offs])
                l1 = np.array([abs(dx) + abs(dy) for dx, dy in offs])
                dys = np.array([dy for _, dy in offs])
                dxs = np.array([dx for dx, _ in offs])
                best = np.lexsort((dxs, dys, l1, sads))[0]
                mv[r * cols + c] = offs[best]
                sad[r * cols + c] = sads[best]
        res.append((mv, sad))
    return res


def _cost(satd, qp, mvx, mvy):
    """Independent restatement of J from textbook pieces (Python ints)."""
    def eg(v):
        k = 2 * v - 1 if v > 0 else -2 * v
        return 2 * (len(bin(k + 1)) - 3) + 1
    lam = int(math.floor(65536 * math.sqrt(0.57 * 2 ** ((qp - 12) / 3)) + 0.5))
    return satd + ((lam * (eg(4 * mvx) + eg(4 * mvy)) + 32768) >> 16)


# ---------------------------------------------------------------- ME ------
@pytest.mark.parametrize("W,H,ctu,R,seed,bd", [
    (40, 24, 16, 3, 1, 8), (37, 21, 16, 2, 2, 8), (64, 40, 32, 3, 3, 8),
    (48, 48, 32, 2, 4, 10), (70, 66, 64, 2, 5, 8),
])
def test_me_matches_brute_force(W, H, ctu, R, seed, bd):
    fp = synth.frame_pair(seed, W, H, bd, global_range=2, patch_range=3, patch_size=16,
                          n_patches=2)
    out = oracle.analyze(fp.cur, fp.ref, qp=30, search_range=R, ctu=ctu, threads=2)
    ref = _brute_indep(fp.cur, fp.ref, R, ctu)
    for d, (mv, sad) in enumerate(ref):
        ev = out["evaluated"][d].astype(bool)
        inside = sad < 2**31 - 1
        assert np.array_equal(ev, inside)
        assert np.array_equal(out["mvx"][d][ev], mv[ev, 0])
        assert np.array_equal(out["mvy"][d][ev], mv[ev, 1])
        assert np.array_equal(out["sad"][d][ev], sad[ev])


def test_constant_frames_zero_motion():
    cur = np.full((40, 56), 77, dtype=np.uint8)
    out = oracle.analyze(cur, cur.copy(), qp=32, search_range=4, ctu=16)
    for d in range(2):
        ev = out["evaluated"][d].astype(bool)
        assert np.all(out["sad"][d][ev] == 0)
        assert np.all(out["satd"][d][ev] == 0)
        assert np.all(out["mvx"][d][ev] == 0) and np.all(out["mvy"][d][ev] == 0)
        # J = lambda * bits(0,0) = round(lambda * 2)
        assert np.all(out["cost"][d][ev] == _cost(0, 32, 0, 0))
    # ties never split: inside 16x16 CUs stay whole; the partial ones on the
    # right (x 48..64 > 56) and bottom (y 32..48 > 40) are forced to split
    inside = out["evaluated"][0].astype(bool)
    assert list(inside) == [1, 1, 1, 0] * 2 + [0] * 4
    assert np.all(out["split"][0] == ~inside)
    ld = out["leaf_depth"].reshape(5, 7)
    assert np.all(ld[:4, :6] == 0) and np.all(ld[4, :] == 1) and np.all(ld[:, 6] == 1)


@pytest.mark.parametrize("mv", [(3, -2), (-5, 4), (0, 7)])
def test_planted_global_motion_found_exactly(mv):
    fp = synth.frame_pair(11, 96, 80, 8, global_mv=mv, n_patches=0, cur_sigma=0.0)
    R = 8
    out = oracle.analyze(fp.cur, fp.ref, qp=27, search_range=R, ctu=32)
    for d in range(3):
        S = 32 >> d
        cols, rows = out["grid"][d]
        for r in range(rows):
            for c in range(cols):
                x0, y0 = c * S, r * S
                # CU whose displaced block stays inside the frame (no clamped reads)
                if not (0 <= x0 + mv[0] and x0 + S + mv[0] <= 96 and
                        0 <= y0 + mv[1] and y0 + S + mv[1] <= 80 and
                        x0 + S <= 96 and y0 + S <= 80):
                    continue
                i = r * cols + c
                assert (out["mvx"][d][i], out["mvy"][d][i]) == mv
                assert out["sad"][d][i] == 0 and out["satd"][d][i] == 0


def test_planted_motion_with_noise_background():
    """Global motion with sigma-2 noise (config-1 recipe): CUs away from the
    patches and the frame edge return the planted global vector."""
    fp = synth.frame_pair(5, 416, 240, 8)
    out = oracle.analyze(fp.cur, fp.ref, qp=32, search_range=16, ctu=64)
    gx, gy = fp.global_mv
    hits = total = 0
    S = 16
    cols, rows = out["grid"][2]
    for r in range(rows):
        for c in range(cols):
            x0, y0 = c * S, r * S
            if x0 + S > 416 or y0 + S > 240:
                continue
            if not (0 <= x0 + gx and x0 + S + gx <= 416 and 0 <= y0 + gy and y0 + S + gy <= 240):
                continue
            near_patch = any(x0 < px + ps + 16 and px - 16 < x0 + S and y0 < py + ps + 16
                             and py - 16 < y0 + S for (px, py, ps, _) in fp.patches)
            if near_patch:
                continue
            total += 1
            i = r * cols + c
            hits += (out["mvx"][2][i], out["mvy"][2][i]) == (gx, gy)
    assert total > 50
    assert hits == total


def test_satd_and_cost_at_chosen_mv():
    fp = synth.frame_pair(7, 64, 48, 8)
    out = oracle.analyze(fp.cur, fp.ref, qp=22, search_range=4, ctu=32)
    H8 = scipy.linalg.hadamard(8).astype(np.int64)
    cur = fp.cur.astype(np.int64)
    P = 40
    rp = np.pad(fp.ref.astype(np.int64), P, mode="edge")
    for d in range(3):
        S = 32 >> d
        cols, rows = out["grid"][d]
        for i in range(cols * rows):
            if not out["evaluated"][d][i]:
                continue
            x0, y0 = (i % cols) * S, (i // cols) * S
            mx, my = int(out["mvx"][d][i]), int(out["mvy"][d][i])
            tot = 0
            for by in range(0, S, 8):
                for bx in range(0, S, 8):
                    D = cur[y0 + by:y0 + by + 8, x0 + bx:x0 + bx + 8] - rp[
                        P + y0 + by + my:P + y0 + by + my + 8, P + x0 + bx + mx:P + x0 + bx + mx + 8]
                    tot += int(np.abs(H8 @ D @ H8.T).sum()) >> 2
            assert out["satd"][d][i] == tot
            assert out["cost"][d][i] == _cost(tot, 22, mx, my)


# -------------------------------------------------------------- split -----
def _enumerate(costs, d, x, y, dmax, S):
    """All partitions of CU (d, x, y): list of (total J, frozenset of leaves)."""
    cols = costs[d]["cols"]
    J = int(costs[d]["J"][y * cols + x])
    opts = [(J, frozenset([(d, x, y)]))]
    if d < dmax:
        kids = [_enumerate(costs, d + 1, 2 * x + (q & 1), 2 * y + (q >> 1), dmax, S)
                for q in range(4)]
        for combo in itertools.product(*kids):
            opts.append((sum(c[0] for c in combo), frozenset().union(*(c[1] for c in combo))))
    return opts


@pytest.mark.parametrize("seed,ctu", [(21, 32), (22, 32), (23, 64)])
def test_split_is_optimal_over_all_partitions(seed, ctu):
    W = H = ctu
    fp = synth.frame_pair(seed, W, H, 8, global_range=2, patch_range=4, patch_size=16, n_patches=2)
    out = oracle.analyze(fp.cur, fp.ref, qp=37, search_range=2, ctu=ctu)
    dmax = int(math.log2(ctu // 8))
    costs = [{"cols": out["grid"][d][0], "J": out["cost"][d]} for d in range(dmax + 1)]
    opts = _enumerate(costs, 0, 0, 0, dmax, ctu)
    expected = {32: 17, 64: 83522}[ctu]
    assert len(opts) == expected
    best_total = min(o[0] for o in opts)
    assert out["best"][0][0] == best_total
    # the oracle's leaves form a partition with that total
    leaves = set()
    c8 = out["grid8"][0]
    for i, ld in enumerate(out["leaf_depth"]):
        S = ctu >> int(ld)
        leaves.add((int(ld), (i % c8) * 8 // S, (i // c8) * 8 // S))
    total = sum(int(out["cost"][d][y * out["grid"][d][0] + x]) for d, x, y in leaves)
    assert total == best_total
    assert frozenset(leaves) in {o[1] for o in opts if o[0] == best_total}


def test_split_tie_does_not_split():
    # constant frame: every CU has J = round(2 lambda); the 4 children sum to
    # 4x that, so nothing splits; best(root) = J(root).
    cur = np.full((32, 32), 9, dtype=np.uint8)
    out = oracle.analyze(cur, cur.copy(), qp=12, search_range=1, ctu=32)
    assert out["best"][0][0] == out["cost"][0][0]
    assert not out["split"][0][0]


def test_partial_ctu_is_forced_split():
    # 40x24 frame, 32x32 CTUs: the CTU at x=32 only has 8 columns -> forced
    fp = synth.frame_pair(3, 40, 24, 8, n_patches=0)
    out = oracle.analyze(fp.cur, fp.ref, qp=27, search_range=2, ctu=32)
    assert out["grid"][0] == (2, 1)
    assert list(out["evaluated"][0]) == [0, 0]        # neither 32x32 is inside (H8=24)
    assert list(out["split"][0]) == [1, 1]
    assert np.all(out["leaf_depth"] >= 1)
    cols, rows = out["grid"][1]
    assert (cols, rows) == (3, 2)
    # 16x16 row 1 spans y 16..32 > 24 -> not inside -> forced split to 8x8
    assert list(out["evaluated"][1][cols:]) == [0, 0, 0]
    assert list(out["evaluated"][1][:cols]) == [1, 1, 0]   # x=32 CU spans to 48 > 40


# ---------------------------------------------------------- dependent ----
def _dep_from(out, size, **kw):
    d = {"ref_size": size, "leaf_depth": out["leaf_depth"], "leaf_mvx": out["leaf_mvx"],
         "leaf_mvy": out["leaf_mvy"]}
    d.update(kw)
    return d


def test_unconstrained_dependent_equals_independent():
    fp = synth.frame_pair(31, 96, 72, 8)
    ref_out = oracle.analyze(fp.ref, fp.cur, qp=32, search_range=5, ctu=32)  # any reference rung
    indep = oracle.analyze(fp.cur, fp.ref, qp=32, search_range=5, ctu=32)
    dep = oracle.analyze(fp.cur, fp.ref, qp=32, search_range=5, ctu=32,
                         dep=_dep_from(ref_out, (96, 72), use_ref_mv=0, depth_lo=-2, depth_hi=2))
    for k in ("mvx", "mvy", "sad", "satd", "cost", "best", "split", "evaluated"):
        for d in range(3):
            assert np.array_equal(indep[k][d], dep[k][d]), (k, d)
    for k in ("leaf_depth", "leaf_mvx", "leaf_mvy"):
        assert np.array_equal(indep[k], dep[k])


def _brute_dep(cur, ref, x0, y0, S, cx, cy, r):
    """Exhaustive refinement around the centre (cx, cy), written
    independently: edge-clamped reference reads and the key (SAD, |ox|+|oy|,
    oy, ox) over the offsets (ox, oy) from the centre."""
    H, W = cur.shape
    ys = np.arange(y0, y0 + S)
    xs = np.arange(x0, x0 + S)
    blk = cur[np.ix_(np.minimum(ys, H - 1), np.minimum(xs, W - 1))].astype(np.int64)
    best = None
    for oy in range(-r, r + 1):
        for ox in range(-r, r + 1):
            ry = np.clip(ys + cy + oy, 0, H - 1)
            rx = np.clip(xs + cx + ox, 0, W - 1)
            sad = int(np.abs(blk - ref[np.ix_(ry, rx)].astype(np.int64)).sum())
            key = (sad, abs(ox) + abs(oy), oy, ox)
            if best is None or key < best:
                best = key
    return cx + best[3], cy + best[2], best[0]


@pytest.mark.parametrize("content", ["flat", "columns", "levels3"])
def test_dependent_tie_break_is_relative_to_the_centre(content):
    """Ratio-2 dependent rung whose co-located reference leaves carry
    non-zero vectors, on content where many candidates tie: every evaluated
    CU must return the brute-force argmin of (SAD, L1 offset from the
    centre, dy, dx).  On flat content every SAD is 0, so the vector is the
    centre itself (a tie-break on the absolute vector would move it)."""
    rng = np.random.default_rng(71)
    Wr, Hr, Wd, Hd, r = 40, 32, 80, 64, 3
    n8 = (Wr // 8) * (Hr // 8)
    lmx = rng.integers(-3, 4, n8).astype(np.int16)
    lmy = rng.integers(-3, 4, n8).astype(np.int16)
    lmy[lmy == 0] = 2
    dep = {"ref_size": (Wr, Hr), "leaf_depth": np.full(n8, 3, np.uint8), "leaf_mvx": lmx, "leaf_mvy": lmy}
    if content == "flat":
        ref = np.full((Hd, Wd), 100, np.uint8)
        cur = ref.copy()
    elif content == "columns":
        ref = np.tile((40 * (np.arange(Wd) % 4)).astype(np.uint8), (Hd, 1))
        cur = ref.copy()
    else:
        ref = rng.integers(0, 3, (Hd, Wd)).astype(np.uint8)
        cur = np.roll(ref, (1, -2), axis=(0, 1)) ^ (rng.random((Hd, Wd)) < 0.2).astype(np.uint8)
    out = oracle.analyze(cur, ref, qp=30, search_range=r, ctu=64, dep=dep, threads=2)
    checked = moved = 0
    for d in range(4):
        S = 64 >> d
        cols, rows = out["grid"][d]
        for i in np.flatnonzero(out["evaluated"][d]):
            x0, y0 = (i % cols) * S, (i // cols) * S
            cx, cy, _, _ = oracle.derive_rule((Wd, Hd), dep, d, x0, y0)
            want = _brute_dep(cur, ref, x0, y0, S, cx, cy, r)
            got = (int(out["mvx"][d][i]), int(out["mvy"][d][i]), int(out["sad"][d][i]))
            assert got == want, (content, d, x0, y0, (cx, cy), got, want)
            checked += 1
            moved += cy != 0
            if content == "flat":
                assert got[:2] == (cx, cy)
    assert checked >= 40 and moved >= 20


def test_deq_worked_examples():
    # ratio 3 (640 -> 1920): a reference 8x8 leaf projects to 24 -> Deq = 1,
    # leaves allowed at depths 1, 2 (32, 16); split allowed at 0, 1.
    lz = np.full(80 * 45, 3, dtype=np.uint8)
    mz = np.zeros(80 * 45, dtype=np.int16)
    dep = {"ref_size": (640, 360), "leaf_depth": lz, "leaf_mvx": mz, "leaf_mvy": mz}
    rules = [oracle.derive_rule((1920, 1080), dep, d, 64, 64) for d in range(4)]
    assert [r[2] for r in rules] == [0, 1, 1, 1]   # depth 3 = dmax is always a leaf
    assert [r[3] for r in rules] == [1, 1, 0, 0]
    # ratio 1.5 (640 -> 960): a reference 64 leaf projects to 96 -> Deq = 0,
    # leaves at depths 0, 1; split allowed at 0 only.  The per-CU rule also
    # lets depths 2, 3 be leaves (they may not split), but they are
    # unreachable because depth 1 may not split.
    lz0 = np.zeros(80 * 45, dtype=np.uint8)
    dep0 = {"ref_size": (640, 360), "leaf_depth": lz0, "leaf_mvx": mz, "leaf_mvy": mz}
    rules = [oracle.derive_rule((960, 540), dep0, d, 0, 0) for d in range(4)]
    assert [r[2] for r in rules] == [1, 1, 1, 1]
    assert [r[3] for r in rules] == [1, 0, 0, 0]


def test_unreachable_cus_are_not_evaluated():
    # Ratio 3, reference all 8x8 leaves: Deq = 1 everywhere, so 16x16 CUs may
    # not split and their 8x8 children are unreachable; 64x64 may not be a
    # leaf.  Only depths 1 and 2 are searched (the refinement's n and n+1).
    rfp = synth.frame_pair(61, 64, 48, 8)
    rout = {"leaf_depth": np.full(8 * 6, 3, np.uint8), "leaf_mvx": np.zeros(48, np.int16),
            "leaf_mvy": np.zeros(48, np.int16)}
    fp = synth.frame_pair(62, 192, 144, 8)
    dout = oracle.analyze(fp.cur, fp.ref, qp=27, search_range=1, ctu=64,
                          dep=dict(rout, ref_size=(64, 48)))
    assert not dout["evaluated"][0].any()
    assert not dout["evaluated"][3].any()
    # every inside 32x32 and 16x16 is evaluated
    for d in (1, 2):
        S = 64 >> d
        cols, rows = dout["grid"][d]
        for i in range(cols * rows):
            x0, y0 = (i % cols) * S, (i // cols) * S
            assert dout["evaluated"][d][i] == (x0 + S <= 192 and y0 + S <= 144)
    assert set(np.unique(dout["leaf_depth"])) <= {1, 2}


def test_mv_scaling_round_half_away():
    # centre = sign(v) * floor((2|v| Wd + Wr) / (2 Wr)), per component
    cases = [((640, 360), (960, 540), 1, 2), ((640, 360), (960, 540), -1, -2),
             ((640, 360), (960, 540), 3, 5), ((640, 360), (960, 540), -3, -5),
             ((640, 360), (1280, 720), 7, 14), ((640, 360), (1920, 1080), -5, -15),
             ((960, 540), (1280, 720), 3, 4), ((960, 540), (1280, 720), -3, -4),
             ((640, 360), (3840, 2160), 100, 256), ((640, 360), (3840, 2160), -50, -256)]
    for rs, ds, v, want in cases:
        n8 = ((rs[0] + 7) // 8) * ((rs[1] + 7) // 8)
        dep = {"ref_size": rs, "leaf_depth": np.full(n8, 3, np.uint8),
               "leaf_mvx": np.full(n8, v, np.int16), "leaf_mvy": np.full(n8, v, np.int16)}
        cx, cy, _, _ = oracle.derive_rule(ds, dep, 3, 8, 8)
        assert (cx, cy) == (want, want), (rs, ds, v)


def test_colocated_point_picks_the_right_leaf():
    # reference leaves carry their own index as MV; ratio 2: the dependent CU
    # at (x0, y0) of size S has centre (2x0+S)/2 -> reference point half that.
    rs, ds = (64, 48), (128, 96)
    c8, r8 = 8, 6
    idx = np.arange(c8 * r8)
    dep = {"ref_size": rs, "leaf_depth": np.full(c8 * r8, 3, np.uint8),
           "leaf_mvx": (idx % c8).astype(np.int16), "leaf_mvy": (idx // c8).astype(np.int16),
           "use_ref_mv": 1}
    for d, x0, y0 in [(3, 0, 0), (3, 120, 88), (2, 48, 32), (0, 64, 0), (1, 96, 64)]:
        S = 64 >> d
        xm, ym = (2 * x0 + S) * 64 // 256, (2 * y0 + S) * 48 // 192
        cx, cy, _, _ = oracle.derive_rule(ds, dep, d, x0, y0)
        # scaled by 2: centre = 2 * leaf coordinate index
        assert (cx, cy) == (2 * (xm >> 3), 2 * (ym >> 3))


@pytest.mark.parametrize("ratio", [2, 3])
def test_integer_ratio_planted_motion(ratio):
    """Reference rung with motion m/ratio, dependent rung with motion m (zero
    noise): the scaled centre is the true vector and every evaluated inside
    CU away from the frame edge returns it with SAD 0."""
    m = (2 * ratio, -ratio)
    Wr, Hr = 64, 48
    Wd, Hd = Wr * ratio, Hr * ratio
    rfp = synth.frame_pair(41, Wr, Hr, 8, global_mv=(m[0] // ratio, m[1] // ratio),
                           n_patches=0, cur_sigma=0.0)
    rout = oracle.analyze(rfp.cur, rfp.ref, qp=27, search_range=4, ctu=64)
    dfp = synth.frame_pair(42, Wd, Hd, 8, global_mv=m, n_patches=0, cur_sigma=0.0)
    dout = oracle.analyze(dfp.cur, dfp.ref, qp=27, search_range=1, ctu=64,
                          dep=_dep_from(rout, (Wr, Hr)))
    checked = 0
    for d in range(4):
        S = 64 >> d
        cols, rows = dout["grid"][d]
        for i in range(cols * rows):
            x0, y0 = (i % cols) * S, (i // cols) * S
            if not dout["evaluated"][d][i]:
                continue
            if not (0 <= x0 + m[0] and x0 + S + m[0] <= Wd and 0 <= y0 + m[1] and
                    y0 + S + m[1] <= Hd):
                continue
            # was the co-located reference leaf itself on the true vector?
            xm = min((2 * x0 + S) * Wr // (2 * Wd), Wr - 1)
            ym = min((2 * y0 + S) * Hr // (2 * Hd), Hr - 1)
            li = (ym >> 3) * (Wr // 8) + (xm >> 3)
            if (rout["leaf_mvx"][li], rout["leaf_mvy"][li]) != (m[0] // ratio, m[1] // ratio):
                continue
            checked += 1
            assert (dout["mvx"][d][i], dout["mvy"][d][i]) == m
            assert dout["sad"][d][i] == 0
    assert checked > 10


def _check_leaf_chain(out, ctu):
    """Every 8x8 lies in an evaluated leaf CU whose MV it carries, and every
    ancestor of that leaf is split."""
    c8, r8 = out["grid8"]
    for i in range(c8 * r8):
        x, y = (i % c8) * 8, (i // c8) * 8
        ld = int(out["leaf_depth"][i])
        S = ctu >> ld
        cols = out["grid"][ld][0]
        li = (y // S) * cols + x // S
        assert out["evaluated"][ld][li]
        assert out["mvx"][ld][li] == out["leaf_mvx"][i]
        assert out["mvy"][ld][li] == out["leaf_mvy"][i]
        if ld < len(out["grid"]) - 1:
            assert not out["split"][ld][li]
        for d in range(ld):
            Sd = ctu >> d
            assert out["split"][d][(y // Sd) * out["grid"][d][0] + x // Sd]


def test_dependent_not_evaluated_sentinels():
    fp = synth.frame_pair(51, 128, 96, 8)
    rfp = synth.frame_pair(52, 64, 48, 8)
    rout = oracle.analyze(rfp.cur, rfp.ref, qp=32, search_range=4, ctu=64)
    dout = oracle.analyze(fp.cur, fp.ref, qp=32, search_range=2, ctu=64, dep=_dep_from(rout, (64, 48)))
    for d in range(4):
        ne = ~dout["evaluated"][d].astype(bool)
        assert np.all(dout["mvx"][d][ne] == -32768)
        assert np.all(dout["sad"][d][ne] == 2**31 - 1)
        assert np.all(dout["cost"][d][ne] == 2**31 - 1)
    _check_leaf_chain(dout, 64)
    _check_leaf_chain(rout, 64)


def test_leaf_chain_independent_partial_frame():
    fp = synth.frame_pair(53, 100, 70, 8)
    out = oracle.analyze(fp.cur, fp.ref, qp=37, search_range=3, ctu=64)
    _check_leaf_chain(out, 64)
