"""Pins of the oracle's spatial MV predictor (wavefront CTU order, the WPP
dependency of Sec. 2.2) against values derived by hand from its definition:
the component-wise median of the leaf vectors at A1 = (x0-1, y0+S-1),
B1 = (x0+S-1, y0-1), B0 = (x0+S, y0-1), each (0, 0) unless inside the
8-aligned frame, outside the CU's CTU and in the CTU to the left or in the
row above at most one column to the right."""
import numpy as np
import pytest

import oracle
from paper_2301_12191_gb300 import synth

W, H, CTU = 192, 128, 64          # 3 x 2 CTUs, 24 x 16 blocks of 8x8
BX, BY = np.meshgrid(np.arange(W // 8), np.arange(H // 8))
LEAF_X = (BX + 1).astype(np.int16).reshape(-1)   # vector at (px, py) = (px // 8 + 1, py // 8 + 1)
LEAF_Y = (BY + 1).astype(np.int16).reshape(-1)

# (x0, y0, S) -> expected predictor, worked out from the positions:
HAND = [
    # CTU (1,1) whole: A1 (63,127) left CTU -> (8,16); B1 (127,63) CTU (1,0) -> (16,8);
    # B0 (128,63) CTU (2,0) = above-right -> (17,8); median x (8,16,17) = 16, y (16,8,8) = 8
    ((64, 64, 64), (16, 8)),
    # CTU (1,1) bottom-right 32: A1 (95,127), B1 (127,95) inside; B0 (128,95) CTU (2,1) not yet decided
    ((96, 96, 32), (0, 0)),
    # CTU (1,1) top-right 32: A1 (95,95) inside -> 0; B1 (127,63) -> (16,8); B0 (128,63) -> (17,8)
    ((96, 64, 32), (16, 8)),
    # CTU (1,1) bottom-left 32: A1 (63,127) -> (8,16); B1 (95,95), B0 (96,95) inside -> 0
    ((64, 96, 32), (0, 0)),
    # CTU (1,1) top-left 8: A1 (63,71) -> (8,9); B1 (71,63) -> (9,8); B0 (72,63) -> (10,8)
    ((64, 64, 8), (9, 8)),
    # CTU (2,1): A1 (127,127) -> (16,16); B1 (191,63) -> (24,8); B0 (192,63) outside the frame
    ((128, 64, 64), (16, 8)),
    # CTU (0,0): nothing decided before it
    ((0, 0, 64), (0, 0)),
    # CTU (0,1): A1 (-1,127) outside; B1 (63,63) -> (8,8); B0 (64,63) -> (9,8)
    ((0, 64, 64), (8, 8)),
    # CTU (1,0), top row: A1 (63,63) CTU (0,0) -> (8,8); B1, B0 above the frame
    ((64, 0, 64), (0, 0)),
]


@pytest.mark.parametrize("cu,want", HAND)
def test_spatial_mvp_hand_cases(cu, want):
    assert oracle.spatial_mvp(W, H, CTU, LEAF_X, LEAF_Y, *cu) == want


RAND = np.random.default_rng(12)
RX = RAND.integers(-40, 41, (H // 8) * (W // 8)).astype(np.int16)
RY = RAND.integers(-40, 41, (H // 8) * (W // 8)).astype(np.int16)


def _at(px, py):
    i = (py // 8) * (W // 8) + px // 8
    return int(RX[i]), int(RY[i])


def _med(vs):
    return tuple(int(np.median([v[k] for v in vs])) for k in range(2))


# (x0, y0, S) -> the positions that are available, listed by hand (the
# others count as (0, 0)); distinct vectors everywhere, so a wrong position
# changes the median
RAND_CASES = [
    ((64, 64, 64), [(63, 127), (127, 63), (128, 63)]),
    ((96, 64, 32), [(127, 63), (128, 63)]),
    ((64, 96, 32), [(63, 127)]),
    ((64, 80, 16), [(63, 95)]),
    ((64, 64, 16), [(63, 79), (79, 63), (80, 63)]),
    ((112, 64, 16), [(127, 63), (128, 63)]),
    ((128, 64, 32), [(127, 95), (159, 63), (160, 63)]),
    ((0, 64, 32), [(31, 63), (32, 63)]),
]


@pytest.mark.parametrize("cu,avail", RAND_CASES)
def test_spatial_mvp_random_leaves(cu, avail):
    vs = [_at(*q) for q in avail] + [(0, 0)] * (3 - len(avail))
    assert oracle.spatial_mvp(W, H, CTU, RX, RY, *cu) == _med(vs)


def test_spatial_mvp_negative_vectors():
    # the same positions as the first case with every vector negated: the
    # median of (-8, -16, -17) is -16, of (-16, -8, -8) is -8
    assert oracle.spatial_mvp(W, H, CTU, -LEAF_X, -LEAF_Y, 64, 64, 64) == (-16, -8)


def test_spatial_mvp_ragged_frame():
    # 180 x 120: the 8-aligned frame is 184 x 120; B0 of CTU (2,1)'s 32x32
    # top-left CU at (160, 63) lies inside it, in CTU (2,0) -> (21, 8)
    w, h = 180, 120
    bx, by = np.meshgrid(np.arange(23), np.arange(15))
    lx, ly = (bx + 1).reshape(-1), (by + 1).reshape(-1)
    # A1 (127, 95) -> (16, 12); B1 (159, 63) -> (20, 8); B0 (160, 63) -> (21, 8)
    assert oracle.spatial_mvp(w, h, CTU, lx, ly, 128, 64, 32) == (20, 8)
    # the depth-0 CU of CTU (2,1): B0 at (192, 63) is past the 8-aligned width
    # A1 (127, 119) -> (16, 15); B1 (191, 63) past the width too -> 0
    assert oracle.spatial_mvp(w, h, CTU, lx, ly, 128, 64, 64) == (0, 0)


@pytest.mark.parametrize("size", [(64, 64), (48, 40)])
def test_single_ctu_has_no_predictor(size):
    p = synth.frame_pair(11, *size)
    a = oracle.analyze(p.cur, p.ref, qp=27, search_range=8, ctu=64)
    b = oracle.analyze(p.cur, p.ref, qp=27, search_range=8, ctu=64, mvp=1)
    for k in ("cost", "best", "split"):
        for d in range(len(a["grid"])):
            assert np.array_equal(a[k][d], b[k][d]), (k, d)
    assert np.array_equal(a["leaf_depth"], b["leaf_depth"])


def test_uniform_motion_cost_closed_form():
    """Every CU finds the planted vector v: a CU with at least two available
    neighbours is predicted by v (bits se(0) + se(0) = 2), one with at most
    one by (0, 0) (bits se(4 vx) + se(4 vy))."""
    v = (3, -2)
    p = synth.frame_pair(5, W, H, global_mv=v, n_patches=0, cur_sigma=0.0)
    qp = 30
    a = oracle.analyze(p.cur, p.ref, qp=qp, search_range=6, ctu=CTU, mvp=1)
    assert (a["leaf_mvx"] == v[0]).all() and (a["leaf_mvy"] == v[1]).all()
    lam = oracle.lambda_q16(qp)
    rate = lambda bits: (lam * bits + 32768) >> 16
    zero_bits = oracle.se_bits(4 * v[0]) + oracle.se_bits(4 * v[1])
    cols0 = a["grid"][0][0]
    # depth 0: CTU (1,1) and (2,1) have >= 2 available neighbours, (0,0) and (1,0) none or one
    for (cx, cy), bits in (((1, 1), 2), ((2, 1), 2), ((0, 1), 2), ((0, 0), zero_bits), ((1, 0), zero_bits)):
        i = cy * cols0 + cx
        assert a["cost"][0][i] == a["satd"][0][i] + rate(bits), (cx, cy)
    # depth 3 (8x8): the bottom-right block of CTU (1,1) has no available neighbour
    cols3 = a["grid"][3][0]
    i = (64 // 8 + 7) * cols3 + 64 // 8 + 7
    assert a["cost"][3][i] == a["satd"][3][i] + rate(zero_bits)
    # its top-left block has A1, B1, B0 available
    i = (64 // 8) * cols3 + 64 // 8
    assert a["cost"][3][i] == a["satd"][3][i] + rate(2)


def _ctu_fields(a, cx, cy, ctu=CTU):
    out = []
    for d, (c, r) in enumerate(a["grid"]):
        n = 1 << d
        for k in ("cost", "best", "split"):
            g = np.asarray(a[k][d]).reshape(r, c)
            out.append(g[cy * n:(cy + 1) * n, cx * n:(cx + 1) * n].copy())
    return out


def test_wavefront_dependencies():
    """CTU (1,2) of a 4 x 3 CTU frame reads, transitively, only the CTUs to
    its left and those above it up to one more column per row: changing the
    content of CTU (3,1) or (2,2) leaves its decisions unchanged."""
    w, h = 256, 192
    p = synth.frame_pair(21, w, h, global_range=4, patch_range=6, n_patches=6, patch_size=24)
    base = oracle.analyze(p.cur, p.ref, qp=32, search_range=6, ctu=CTU, mvp=1)
    want = _ctu_fields(base, 1, 2)
    rng = np.random.default_rng(3)
    for (qx, qy) in ((3, 1), (2, 2)):
        cur = p.cur.copy()
        cur[qy * 64:(qy + 1) * 64, qx * 64:(qx + 1) * 64] = rng.integers(0, 256, (64, 64), dtype=np.uint8)
        a = oracle.analyze(cur, p.ref, qp=32, search_range=6, ctu=CTU, mvp=1)
        changed = any(not np.array_equal(x, y) for x, y in zip(_ctu_fields(a, qx, qy), _ctu_fields(base, qx, qy)))
        assert changed, "the planted change must reach the modified CTU"
        for x, y in zip(_ctu_fields(a, 1, 2), want):
            assert np.array_equal(x, y), (qx, qy)


def test_mvp_rejects_ctu_sample():
    p = synth.frame_pair(2, 128, 64)
    with pytest.raises(ValueError):
        oracle.analyze(p.cur, p.ref, qp=27, search_range=4, ctu=64, mvp=1, ctu_mask=[1, 0])
