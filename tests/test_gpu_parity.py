"""Parity of the CUDA path with the CPU oracle, bit-exact on every decision
(MVs, SAD, SATD, cost, best, split flags, evaluated flags, leaf maps).

All calls go through the C ABI (ctypes binding); inputs are seeded synthetic
planes from ``synth``; expected values come only from ``oracle``.
"""
import numpy as np
import pytest

import oracle
from paper_2301_12191_gb300 import synth
from helpers import assert_decisions_equal, dep_from

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402


def _run_independent(fp, *, ctu, R, qp, satd_mode=0, frame_id=0):
    bd = fp.bit_depth
    with L.Ladder([(fp.width, fp.height)], 0, bit_depth=bd, ctu_size=ctu, search_range=R,
                  satd_mode=satd_mode, max_frames=1) as lad:
        cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
        lad.analyze_reference(frame_id, cur, ref, qp)
        return lad.fetch(0, frame_id)


def test_config1_frame_pair_independent():
    """416x240 8-bit, 64x64 CTUs, +-16 full search, QP32 (the small case)."""
    fp = synth.frame_pair(1, 416, 240, 8)
    gpu = _run_independent(fp, ctu=64, R=16, qp=32)
    ora = oracle.analyze(fp.cur, fp.ref, qp=32, search_range=16, ctu=64)
    assert_decisions_equal(gpu, ora, 64, where="config1")


@pytest.mark.parametrize("W,H,ctu,R,bd,satd,qp,seed", [
    (64, 64, 64, 4, 8, 0, 22, 2),      # one CTU, smallest range
    (100, 70, 64, 8, 8, 0, 37, 3),     # partial CTUs both ways, ragged 8-alignment
    (130, 66, 32, 5, 8, 1, 27, 4),     # 32x32 CTUs, odd range, PAPER4x4 SATD
    (96, 48, 16, 6, 10, 0, 32, 5),     # 16x16 CTUs, 10-bit
    (200, 120, 64, 16, 10, 0, 22, 6),  # 10-bit, 64x64
    (72, 40, 64, 4, 8, 0, 51, 7),      # frame smaller than two CTUs, max QP
    (418, 238, 64, 12, 8, 0, 0, 8),    # ragged tail, QP 0
    (16, 16, 16, 4, 8, 0, 30, 9),      # minimum frame
    (34, 18, 32, 7, 10, 1, 30, 10),    # tiny 10-bit with PAPER4x4
])
def test_independent_small(W, H, ctu, R, bd, satd, qp, seed):
    fp = synth.frame_pair(seed, W, H, bd, global_range=3, patch_range=5, patch_size=24)
    gpu = _run_independent(fp, ctu=ctu, R=R, qp=qp, satd_mode=satd)
    ora = oracle.analyze(fp.cur, fp.ref, qp=qp, search_range=R, ctu=ctu, satd_mode=satd)
    assert_decisions_equal(gpu, ora, ctu, where=f"{W}x{H} ctu{ctu} R{R} bd{bd}")


def test_max_range_10bit():
    """R = 64 (largest window the TMA box and shared memory allow)."""
    fp = synth.frame_pair(12, 192, 128, 10, global_range=30, patch_range=40, patch_size=32)
    gpu = _run_independent(fp, ctu=64, R=64, qp=27)
    ora = oracle.analyze(fp.cur, fp.ref, qp=27, search_range=64, ctu=64)
    assert_decisions_equal(gpu, ora, 64, where="R64 10-bit")


def test_max_range_8bit():
    fp = synth.frame_pair(13, 256, 136, 8, global_range=30, patch_range=50, patch_size=48)
    gpu = _run_independent(fp, ctu=64, R=64, qp=32)
    ora = oracle.analyze(fp.cur, fp.ref, qp=32, search_range=64, ctu=64)
    assert_decisions_equal(gpu, ora, 64, where="R64 8-bit")


def test_constant_frames():
    cur = np.full((48, 80), 200, dtype=np.uint8)
    fp = synth.FramePair(cur=cur, ref=cur.copy(), bit_depth=8, global_mv=(0, 0), patches=[])
    gpu = _run_independent(fp, ctu=32, R=6, qp=32)
    ora = oracle.analyze(fp.cur, fp.ref, qp=32, search_range=6, ctu=32)
    assert_decisions_equal(gpu, ora, 32, where="constant")
    assert np.all(gpu["leaf_mvx"] == 0) and np.all(gpu["leaf_mvy"] == 0)


def _ladder_case(seed, src, rungs, ref_idx, bd, R, r, qp, ctu=64, lo=0, hi=1, use_ref_mv=1, satd=0,
                 independent_too=False, include_source=False):
    pairs, _ = synth.ladder_pairs(seed, source=src, rungs=rungs, bit_depth=bd, include_source=include_source)
    sizes = [(w, h) for (w, h, _, _) in pairs]
    with L.Ladder(sizes, ref_idx, bit_depth=bd, ctu_size=ctu, search_range=R, refine_range=r,
                  depth_lo=lo, depth_hi=hi, use_ref_mv=use_ref_mv, satd_mode=satd, max_frames=2) as lad:
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_reference(5, *planes[ref_idx], qp)
        for i in range(len(pairs)):
            if i != ref_idx:
                lad.analyze_dependent(i, 5, *planes[i], qp)
        gpu = [lad.fetch(i, 5) for i in range(len(pairs))]
        gpu_ind = None
        if independent_too:
            for i in range(len(pairs)):
                lad.analyze_independent(i, 6, *planes[i], qp)
            gpu_ind = [lad.fetch(i, 6) for i in range(len(pairs))]
    w, h, c, f = pairs[ref_idx]
    ora_ref = oracle.analyze(c, f, qp=qp, search_range=R, ctu=ctu, satd_mode=satd)
    oras = []
    for i, (w, h, c, f) in enumerate(pairs):
        if i == ref_idx:
            oras.append(ora_ref)
        else:
            oras.append(oracle.analyze(c, f, qp=qp, search_range=r, ctu=ctu, satd_mode=satd,
                                       dep=dep_from(ora_ref, sizes[ref_idx], depth_lo=lo, depth_hi=hi,
                                                    use_ref_mv=use_ref_mv)))
    return pairs, gpu, oras, gpu_ind


@pytest.mark.parametrize("bd,R,r,lo,hi,use_mv,satd", [
    (8, 8, 2, 0, 1, 1, 0),
    (8, 8, 4, 0, 1, 0, 0),
    (8, 6, 3, -1, 1, 1, 1),
    (10, 8, 2, 0, 2, 1, 0),
    (8, 8, 9, 0, 0, 1, 0),     # r > 8 exercises the 17-wide column chunks
    (8, 8, 0, 0, 1, 1, 0),     # r = 0: reuse the scaled vector as is
    (10, 16, 8, 0, 1, 1, 0),   # 10-bit r = 8: the 17-row band of 16-bit samples the UHD ladder uses
    (10, 16, 8, -1, 2, 1, 1),  # the same with a wider depth window and PAPER4x4
])
def test_dependent_small_ladder(bd, R, r, lo, hi, use_mv, satd):
    pairs, gpu, oras, _ = _ladder_case(21, (640, 360), [(480, 270), (320, 180), (160, 90)], 2, bd, R, r, 27,
                                       lo=lo, hi=hi, use_ref_mv=use_mv, satd=satd)
    for i in range(len(pairs)):
        assert_decisions_equal(gpu[i], oras[i], 64, where=f"rung {i}")


def test_batched_dependents_equal_single_calls():
    pairs, _ = synth.ladder_pairs(25, source=(960, 540), rungs=[(640, 360), (480, 270), (320, 180)])
    sizes = [(w, h) for (w, h, _, _) in pairs]
    with L.Ladder(sizes, 3, search_range=8, refine_range=3, max_frames=2) as lad:
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        for fid in (0, 1):
            lad.analyze_reference(fid, *planes[3], 32)
        for i in range(3):
            lad.analyze_dependent(i, 0, *planes[i], 32)
        lad.analyze_dependents(1, [(i, planes[i][0], planes[i][1]) for i in (2, 0, 1)], 32)
        single = [lad.fetch(i, 0) for i in range(3)]
        batched = [lad.fetch(i, 1) for i in range(3)]
    ref = oracle.analyze(pairs[3][2], pairs[3][3], qp=32, search_range=8)
    for i in range(3):
        assert_decisions_equal(batched[i], single[i], 64, where=f"batched rung {i}")
        ora = oracle.analyze(pairs[i][2], pairs[i][3], qp=32, search_range=3,
                             dep=dep_from(ref, sizes[3]))
        assert_decisions_equal(batched[i], ora, 64, where=f"batched vs oracle rung {i}")


def _batch_frames(n, seed0, sizes_src=(640, 360), rungs=((480, 270), (320, 180))):
    out = []
    for k in range(n):
        pairs, _ = synth.ladder_pairs(seed0 + k, source=sizes_src, rungs=list(rungs), include_source=True)
        out.append(pairs)
    return out


def test_analyze_batch_equals_per_call_and_oracle():
    frames = _batch_frames(5, 300)
    sizes = [(w, h) for (w, h, _, _) in frames[0]]
    ref_i, qps = 2, [22, 27, 32, 37, 30]
    with L.Ladder(sizes, ref_i, search_range=12, refine_range=3, max_frames=10) as lad:
        planes = [[(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in fr] for fr in frames]
        lad.analyze_batch([(100 + k, qps[k], planes[k]) for k in range(5)])
        got = [[lad.fetch(r, 100 + k) for r in range(3)] for k in range(5)]
        for k in range(5):   # the same frames one call at a time
            lad.analyze_reference(200 + k, *planes[k][ref_i], qps[k])
            lad.analyze_dependents(200 + k, [(r, *planes[k][r]) for r in range(3) if r != ref_i], qps[k])
        single = [[lad.fetch(r, 200 + k) for r in range(3)] for k in range(5)]
    for k in range(5):
        for r in range(3):
            assert_decisions_equal(got[k][r], single[k][r], 64, where=f"batch frame {k} rung {r}")
    for k in (0, 3):
        fr = frames[k]
        ora_ref = oracle.analyze(fr[ref_i][2], fr[ref_i][3], qp=qps[k], search_range=12)
        assert_decisions_equal(got[k][ref_i], ora_ref, 64, where=f"batch vs oracle ref {k}")
        for r in (0, 1):
            ora = oracle.analyze(fr[r][2], fr[r][3], qp=qps[k], search_range=3, dep=dep_from(ora_ref, sizes[ref_i]))
            assert_decisions_equal(got[k][r], ora, 64, where=f"batch vs oracle frame {k} rung {r}")


def test_captured_batch_graph_replays():
    frames = _batch_frames(3, 400)
    sizes = [(w, h) for (w, h, _, _) in frames[0]]
    with L.Ladder(sizes, 2, search_range=8, refine_range=2, max_frames=6) as lad:
        planes = [[(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in fr] for fr in frames]
        items = [(k, 32, planes[k]) for k in range(3)]
        lad.analyze_batch(items)
        eager = [[lad.fetch(r, k) for r in range(3)] for k in range(3)]
        stream = torch.cuda.Stream()
        graph = lad.capture_batch(items, stream)
        for _ in range(2):
            graph.launch(stream)
        stream.synchronize()
        replayed = [[lad.fetch(r, k) for r in range(3)] for k in range(3)]
        # new content in the same buffers: the replay reads it
        other = _batch_frames(1, 500)[0]
        for r, (_, _, c, f) in enumerate(other):
            planes[1][r][0].copy_(L.device_plane(c))
            planes[1][r][1].copy_(L.device_plane(f))
        graph.launch(stream)
        stream.synchronize()
        fresh = [lad.fetch(r, 1) for r in range(3)]
        graph.close()
    for k in range(3):
        for r in range(3):
            assert_decisions_equal(replayed[k][r], eager[k][r], 64, where=f"graph frame {k} rung {r}")
    ora_ref = oracle.analyze(other[2][2], other[2][3], qp=32, search_range=8)
    assert_decisions_equal(fresh[2], ora_ref, 64, where="graph new content")


def test_batch_status_codes():
    frames = _batch_frames(2, 600)
    sizes = [(w, h) for (w, h, _, _) in frames[0]]
    with L.Ladder(sizes, 2, search_range=8, refine_range=2, max_frames=1) as lad:
        planes = [[(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in fr] for fr in frames]
        with pytest.raises(L.LadderError) as e:
            lad.analyze_batch([(0, 30, planes[0]), (1, 30, planes[1])])
        assert e.value.status == -4          # two frames, one slot
        with pytest.raises(L.LadderError) as e:
            lad.analyze_batch([(0, 30, planes[0]), (0, 30, planes[1])])
        assert e.value.status == -1          # same frame twice
        lad.analyze_batch([(7, 30, planes[0])])
        lad.sync()


def test_dependent_ctu32():
    pairs, gpu, oras, _ = _ladder_case(22, (384, 216), [(288, 162), (192, 108)], 1, 8, 6, 3, 32, ctu=32)
    for i in range(len(pairs)):
        assert_decisions_equal(gpu[i], oras[i], 32, where=f"rung {i}")


def test_unconstrained_dependent_equals_independent_gpu():
    fp = synth.frame_pair(23, 160, 96, 8)
    with L.Ladder([(160, 96), (160, 96)], 0, search_range=8, refine_range=8, depth_lo=-3, depth_hi=3,
                  use_ref_mv=0, max_frames=1) as lad:
        cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
        # the reference rung gets other content: the dependent must not care
        other = synth.frame_pair(24, 160, 96, 8)
        lad.analyze_reference(0, L.device_plane(other.cur), L.device_plane(other.ref), 30)
        lad.analyze_dependent(1, 0, cur, ref, 30)
        dep = lad.fetch(1, 0)
    ind = _run_independent(fp, ctu=64, R=8, qp=30)
    assert_decisions_equal(dep, ind, 64, where="unconstrained")


def test_config2_ladder_full_size():
    """1080p source -> 720p / 540p / 360p, 360p reference at +-32, dependents
    +-4 with depth n, n+1, QP27; plus independent +-32 on every rung (the
    launch configuration the bench times)."""
    pairs, gpu, oras, gpu_ind = _ladder_case(2, (1920, 1080), [(1280, 720), (960, 540), (640, 360)], 3,
                                             8, 32, 4, 27, independent_too=True, include_source=True)
    for i in range(4):
        assert_decisions_equal(gpu[i], oras[i], 64, where=f"config2 rung {i}")
    # independent +-32 of every rung: sampled CTUs, computed one by one
    rng = np.random.default_rng(7)
    for i, (w, h, c, f) in enumerate(pairs):
        dims, _ = oracle.grid(w, h, 64)
        n = dims[0][0] * dims[0][1]
        mask = np.zeros(n, dtype=np.uint8)
        mask[rng.choice(n, size=min(n, 12), replace=False)] = 1
        mask[-1] = 1   # always include the ragged bottom-right CTU
        ora = oracle.analyze(c, f, qp=27, search_range=32, ctu=64, ctu_mask=mask)
        assert_decisions_equal(gpu_ind[i], ora, 64, ctu_mask=mask, where=f"indep rung {i}")


def test_repeat_calls_are_identical():
    fp = synth.frame_pair(31, 320, 192, 8)
    with L.Ladder([(320, 192)], 0, search_range=16, max_frames=3) as lad:
        cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
        outs = []
        for fid in (1, 2, 1):
            lad.analyze_reference(fid, cur, ref, 32)
            outs.append(lad.fetch(0, fid))
    for o in outs[1:]:
        assert_decisions_equal(o, outs[0], 64, where="repeat")


def test_status_codes():
    fp = synth.frame_pair(41, 128, 64, 8)
    with L.Ladder([(128, 64), (64, 32)], 0, search_range=8, max_frames=1) as lad:
        cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
        small = synth.frame_pair(42, 64, 32, 8)
        sc, sr = L.device_plane(small.cur), L.device_plane(small.ref)
        with pytest.raises(L.LadderError) as e:
            lad.analyze_dependent(1, 9, sc, sr, 30)
        assert e.value.status == -3          # no reference yet
        with pytest.raises(L.LadderError) as e:
            lad.fetch(0, 9)
        assert e.value.status == -7          # nothing analysed
        with pytest.raises(L.LadderError) as e:
            lad.analyze_reference(9, cur, ref, 52)
        assert e.value.status == -1          # QP out of range
        with pytest.raises(L.LadderError) as e:
            L.analyze_reference(lad.handle, 9, cur.data_ptr(), ref.data_ptr(), 130, 30)
        assert e.value.status == -1          # pitch not a multiple of 16
        with pytest.raises(L.LadderError) as e:
            L.analyze_reference(lad.handle, 9, cur.data_ptr() + 1, ref.data_ptr(), 128, 30)
        assert e.value.status == -1          # misaligned plane
        lad.analyze_reference(9, cur, ref, 30)
        with pytest.raises(L.LadderError) as e:
            lad.analyze_reference(10, cur, ref, 30)
        assert e.value.status == -4          # one slot only
        lad.release_frame(9)
        lad.analyze_reference(10, cur, ref, 30)
        lad.analyze_dependent(1, 10, sc, sr, 30)
        lad.sync()
