"""Pins of the oracle's quarter-pel refinement (interpolation, search,
split over the refined costs) against closed forms, hand values and
invariants.  Nothing here calls the CUDA library."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2301_12191_gb300 import synth


# ------------------------------------------------------------ filter -----
@pytest.mark.parametrize("qx,qy", [(0, 0), (1, 0), (2, 0), (3, 0), (0, 1), (0, 2), (2, 3), (-5, 7), (13, -6)])
def test_constant_plane_interpolates_to_itself(qx, qy):
    for bd, v in ((8, 77), (10, 1000)):
        r = np.full((24, 24), v, np.uint8 if bd == 8 else np.uint16)
        assert oracle.pred_sample(r, 11, 9, qx, qy) == v


def test_integer_vectors_give_the_reference_samples():
    rng = np.random.default_rng(5)
    r = rng.integers(0, 256, (32, 32), dtype=np.uint8)
    for (x, y, mx, my) in ((10, 10, 0, 0), (3, 4, -2, 1), (0, 0, -3, -3), (31, 31, 2, 5)):
        want = r[min(max(y + my, 0), 31), min(max(x + mx, 0), 31)]
        assert oracle.pred_sample(r, x, y, 4 * mx, 4 * my) == want
    # the quarter-pel SATD at 4*mv is the integer SATD at mv
    c = rng.integers(0, 256, (32, 32), dtype=np.uint8)
    for mx, my in ((0, 0), (1, -2), (-3, 2)):
        assert oracle.block_satd_q(c, r, 8, 8, 16, 4 * mx, 4 * my) == oracle.block_satd(c, r, 8, 8, 16, mx, my)


# closed forms on a ramp 4x + 100: sum f_k[i] (i - 3) = 0, 15, 32, 49 for the
# phases 0, 1/4, 1/2, 3/4, so P = 4x + 100 + floor((4 * 64 * m + 2048) / 4096)
@pytest.mark.parametrize("phase,add", [(0, 0), (1, 1), (2, 2), (3, 3)])
def test_ramp_closed_forms(phase, add):
    ramp = (np.arange(40) * 4 + 100).astype(np.uint16)
    horiz = np.tile(ramp, (24, 1))
    vert = np.ascontiguousarray(horiz.T)
    for x in (8, 9, 15):
        assert oracle.pred_sample(horiz, x, 10, phase, 0) == 4 * x + 100 + add
        assert oracle.pred_sample(vert, 10, x, 0, phase) == 4 * x + 100 + add


def test_impulse_shows_the_half_pel_taps():
    r = np.zeros((24, 24), np.uint16)
    r[12, 12] = 1023
    # half-pel to the right: the sample at x sees tap i = 12 - x + 3
    got = [oracle.pred_sample(r, x, 12, 2, 0) for x in range(8, 17)]
    # taps -1, 4, -11, 40, 40, -11, 4, -1 at i = 7..0 (x = 8..15); negatives clip to 0
    want = [0, 64, 0, 639, 639, 0, 64, 0, 0]
    assert got == want
    # both axes at half-pel: (40 * 40 * 1023 + 2048) >> 12 = 400
    assert oracle.pred_sample(r, 12, 12, 2, 2) == 400
    # quarter phase picks the 58 tap at the sample itself: (58 * 1023 * 64 + 2048) >> 12 = 927
    assert oracle.pred_sample(r, 12, 12, 1, 0) == 927


# ------------------------------------------------------------ search -----
def _planted_quarter_pel(seed, qx, qy, W=128, H=96):
    fp = synth.frame_pair(seed, W, H, 8, global_range=0, patch_range=0, n_patches=0, cur_sigma=0)
    ref = fp.ref
    cur = np.array([[oracle.pred_sample(ref, x, y, qx, qy) for x in range(W)] for y in range(H)], np.uint8)
    return cur, ref


@pytest.mark.parametrize("qx,qy", [(5, -7), (-2, 3), (1, 1)])
def test_planted_quarter_pel_motion_found(qx, qy):
    cur, ref = _planted_quarter_pel(61, qx, qy)
    ana = oracle.analyze(cur, ref, qp=22, search_range=4, ctu=32)
    sp = oracle.refine_subpel(cur, ref, ana, qp=22, ctu=32)
    # 8x8 CUs at least 12 samples inside the frame
    cols, rows = sp["grid"][2]
    hits = total = 0
    for by in range(rows):
        for bx in range(cols):
            if not (2 <= bx < cols - 2 and 2 <= by < rows - 2):
                continue
            i = by * cols + bx
            total += 1
            hits += sp["qmvx"][2][i] == qx and sp["qmvy"][2][i] == qy and sp["satd"][2][i] == 0
    assert hits >= 0.9 * total, (hits, total)


@pytest.mark.parametrize("qx,qy", [(2, 1), (-2, 5), (6, -3), (-3, -6)])
def test_quarter_round_centres_on_the_half_pel_best(qx, qy):
    """Planted vectors with one component at a half-pel position and the
    other at a quarter-pel one: a half-pel component is at least 2 quarter
    units from every integer vector, so the quarter-pel round reaches the
    planted vector only when it is centred on the half-pel round's best (a
    quarter round around the integer vector stops one quarter unit short)."""
    assert qx % 4 == 2 or qy % 4 == 2
    cur, ref = _planted_quarter_pel(64, qx, qy)
    ana = oracle.analyze(cur, ref, qp=22, search_range=4, ctu=32)
    sp = oracle.refine_subpel(cur, ref, ana, qp=22, ctu=32)
    cols, rows = sp["grid"][2]
    hits = total = 0
    for by in range(2, rows - 2):
        for bx in range(2, cols - 2):
            i = by * cols + bx
            total += 1
            hits += sp["qmvx"][2][i] == qx and sp["qmvy"][2][i] == qy and sp["satd"][2][i] == 0
    assert hits >= 0.9 * total, (hits, total)


def test_refinement_never_raises_the_cost():
    fp = synth.frame_pair(62, 96, 64, 8)
    ana = oracle.analyze(fp.cur, fp.ref, qp=27, search_range=6, ctu=32)
    sp = oracle.refine_subpel(fp.cur, fp.ref, ana, qp=27, ctu=32)
    for d in range(len(sp["grid"])):
        ev = ana["evaluated"][d] == 1
        assert np.all(sp["cost"][d][ev] <= ana["cost"][d][ev])
        # the vector moves at most 3 quarter units from 4 * mv in each axis
        assert np.all(np.abs(sp["qmvx"][d][ev] - 4 * ana["mvx"][d][ev].astype(int)) <= 3)
        assert np.all(np.abs(sp["qmvy"][d][ev] - 4 * ana["mvy"][d][ev].astype(int)) <= 3)
        # cost = SATD + lambda * se-bits of the quarter-pel components
        lam = oracle.lambda_q16(27)
        for i in np.flatnonzero(ev)[:20]:
            bits = oracle.se_bits(int(sp["qmvx"][d][i])) + oracle.se_bits(int(sp["qmvy"][d][i]))
            assert sp["cost"][d][i] == sp["satd"][d][i] + ((lam * bits + 32768) >> 16)


def _enumerate(J, d, x, y, dmax):
    cols = J[d]["cols"]
    opts = [int(J[d]["J"][y * cols + x])]
    if d < dmax:
        kids = [_enumerate(J, d + 1, 2 * x + (q & 1), 2 * y + (q >> 1), dmax) for q in range(4)]
        opts += [sum(c) for c in itertools.product(*kids)]
    return opts


def test_refined_split_is_optimal_over_all_partitions():
    fp = synth.frame_pair(63, 32, 32, 8, global_range=2, patch_range=3, patch_size=16, n_patches=1)
    ana = oracle.analyze(fp.cur, fp.ref, qp=32, search_range=2, ctu=32)
    sp = oracle.refine_subpel(fp.cur, fp.ref, ana, qp=32, ctu=32)
    dmax = int(math.log2(32 // 8))
    J = [{"cols": sp["grid"][d][0], "J": sp["cost"][d]} for d in range(dmax + 1)]
    opts = _enumerate(J, 0, 0, 0, dmax)
    assert len(opts) == 17
    assert sp["best"][0][0] == min(opts)


# -------------------------------------------- spatial predictor -----
# The refinement with the spatial MV predictor, re-derived here from its
# definition with Python's own arithmetic: the predictor of a CU is the
# component-wise median of the refined quarter-pel leaf vectors at A1, B1,
# B0 (available: inside the 8-aligned frame, outside the CU's CTU, in an
# earlier CTU of the wavefront), every candidate's rate is taken against it,
# and the two rounds (half-pel, then quarter-pel around the best so far)
# keep the first strictly lower cost.  Only the quarter-pel SATD probe of the
# oracle is reused (it is pinned by the filter and search cases above).
def _py_se_bits(v):
    k = 2 * v - 1 if v > 0 else -2 * v
    return 2 * ((k + 1).bit_length() - 1) + 1


def _py_lambda_q16(qp):
    return math.floor(65536.0 * math.sqrt(0.57 * 2.0 ** ((qp - 12) / 3.0)) + 0.5)


def _available(ctu, W8, H8, x0, y0, px, py):
    if px < 0 or py < 0 or px >= W8 or py >= H8:
        return False
    cx, cy, qx, qy = x0 // ctu, y0 // ctu, px // ctu, py // ctu
    if (qx, qy) == (cx, cy):
        return False
    if qy == cy:
        return qx < cx
    if qy == cy - 1:
        return qx <= cx + 1
    return qy < cy - 1


def _py_predictor(sp, ctu, W8, H8, x0, y0, S):
    cols8 = W8 // 8
    vx, vy = [], []
    for px, py in ((x0 - 1, y0 + S - 1), (x0 + S - 1, y0 - 1), (x0 + S, y0 - 1)):
        if _available(ctu, W8, H8, x0, y0, px, py):
            li = (py // 8) * cols8 + px // 8
            vx.append(int(sp["leaf_qmvx"][li]))
            vy.append(int(sp["leaf_qmvy"][li]))
        else:
            vx.append(0)
            vy.append(0)
    return sorted(vx)[1], sorted(vy)[1]


def _py_two_rounds(cur, ref, x0, y0, S, mvx, mvy, satd0, qp, pqx, pqy):
    lam = _py_lambda_q16(qp)

    def cost(s, qx, qy):
        return s + ((lam * (_py_se_bits(qx - pqx) + _py_se_bits(qy - pqy)) + 32768) >> 16)

    bx, by, bs = 4 * mvx, 4 * mvy, satd0
    bj = cost(satd0, bx, by)
    for step in (2, 1):
        cx, cy = bx, by
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == 0 and dy == 0:
                    continue
                qx, qy = cx + step * dx, cy + step * dy
                s = oracle.block_satd_q(cur, ref, x0, y0, S, qx, qy)
                j = cost(s, qx, qy)
                if j < bj:
                    bx, by, bs, bj = qx, qy, s, j
    return bx, by, bs, bj


def _check_spatial_refinement(cur, ref, qp, ctu, R):
    H, W = cur.shape
    W8, H8 = (W + 7) // 8 * 8, (H + 7) // 8 * 8
    ana = oracle.analyze(cur, ref, qp=qp, search_range=R, ctu=ctu, mvp=1)
    sp = oracle.refine_subpel(cur, ref, ana, qp=qp, ctu=ctu, mvp=1)
    dmax = int(math.log2(ctu // 8))
    checked = 0
    for d in range(dmax + 1):
        S = ctu >> d
        cols, rows = sp["grid"][d]
        for i in np.flatnonzero(ana["evaluated"][d] == 1):
            x0, y0 = (i % cols) * S, (i // cols) * S
            pqx, pqy = _py_predictor(sp, ctu, W8, H8, x0, y0, S)
            want = _py_two_rounds(cur, ref, x0, y0, S, int(ana["mvx"][d][i]), int(ana["mvy"][d][i]),
                                  int(ana["satd"][d][i]), qp, pqx, pqy)
            got = (int(sp["qmvx"][d][i]), int(sp["qmvy"][d][i]), int(sp["satd"][d][i]), int(sp["cost"][d][i]))
            assert got == want, (d, i, got, want, (pqx, pqy))
            checked += 1
    # the split over the refined costs: best = min(J, children's best) where split
    for d in range(dmax):
        cols, rows = sp["grid"][d]
        ccols = sp["grid"][d + 1][0]
        for i in range(cols * rows):
            x, y = i % cols, i // cols
            kids = [(2 * y + (q >> 1)) * ccols + 2 * x + (q & 1) for q in range(4)]
            if sp["split"][d][i]:
                assert sp["best"][d][i] == sum(int(sp["best"][d + 1][k]) for k in kids)
            elif ana["evaluated"][d][i]:
                assert sp["best"][d][i] == sp["cost"][d][i]
    return ana, sp, checked


@pytest.mark.parametrize("bd,ctu,qp", [(8, 16, 37), (10, 32, 32)])
def test_spatial_predictor_refinement_rederived(bd, ctu, qp):
    fp = synth.frame_pair(71 + bd, 96, 64, bd, global_range=3, patch_range=5, patch_size=16, n_patches=2)
    ana, sp, checked = _check_spatial_refinement(fp.cur, fp.ref, qp, ctu, 4)
    assert checked >= 20
    # not vacuous: the predictor moves some CU's refined vector or cost
    sp0 = oracle.refine_subpel(fp.cur, fp.ref, ana, qp=qp, ctu=ctu, mvp=0)
    assert any(not np.array_equal(sp["cost"][d], sp0["cost"][d]) for d in range(len(sp["grid"])))


def test_spatial_refinement_of_the_first_ctu_has_no_predictor():
    """CTU (0, 0) reads no available position: its refinement is the one with
    the predictor (0, 0), whatever the later CTUs hold."""
    fp = synth.frame_pair(75, 96, 64, 8, global_range=3, patch_range=5, patch_size=16, n_patches=2)
    ana = oracle.analyze(fp.cur, fp.ref, qp=37, search_range=4, ctu=32, mvp=1)
    sp1 = oracle.refine_subpel(fp.cur, fp.ref, ana, qp=37, ctu=32, mvp=1)
    sp0 = oracle.refine_subpel(fp.cur, fp.ref, ana, qp=37, ctu=32, mvp=0)
    for d in range(len(sp1["grid"])):
        n = 1 << d
        cols = sp1["grid"][d][0]
        idx = [y * cols + x for y in range(n) for x in range(n)]
        for k in ("qmvx", "qmvy", "satd", "cost", "best", "split"):
            assert np.array_equal(sp1[k][d][idx], sp0[k][d][idx]), (k, d)
