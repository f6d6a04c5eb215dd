"""Spatial MV predictor with the wavefront CTU order (WPP, Sec. 2.2): the
CUDA path -- parallel search and SATD, then one launch that decides cost,
split and leaf maps row by row -- equals the oracle's analysis with mvp=1
(CTUs decided one by one in raster order), field for field, for
independent rungs, dependent rungs of a cascaded chain (per call and
batched), after switching back to the predictor (0, 0), and for a replayed
CUDA graph."""
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


@pytest.mark.parametrize("W,H,ctu,R,bd,satd,qp,seed", [
    (400, 224, 64, 12, 8, 0, 30, 1),   # 7 x 4 CTUs, ragged both ways
    (320, 180, 32, 8, 10, 0, 27, 2),   # 10 x 6 CTUs, 10-bit
    (200, 136, 16, 6, 8, 1, 32, 3),    # 13 x 9 CTUs of 16x16, PAPER4x4 SATD
    (130, 66, 32, 5, 8, 0, 22, 4),     # ragged 8-alignment
    (64, 64, 64, 4, 8, 0, 27, 5),      # one CTU: no neighbour available
    (1280, 64, 64, 8, 8, 0, 37, 6),    # one row of 20 CTUs
    (64, 1280, 64, 8, 8, 0, 37, 7),    # one column of 20 CTUs (every row waits)
])
def test_mvp_independent(W, H, ctu, R, bd, satd, qp, seed):
    fp = synth.frame_pair(seed, W, H, bd, global_range=4, patch_range=6, patch_size=24)
    with L.Ladder([(W, H)], 0, bit_depth=bd, ctu_size=ctu, search_range=R, satd_mode=satd,
                  max_frames=1) as lad:
        lad.set_mv_predictor(1)
        cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
        lad.analyze_reference(0, cur, ref, qp)
        gpu = lad.fetch(0, 0)
        assert lad.kernel_stats()["decide_mvp"][0] == 1  # one wavefront launch after the search
    ora = oracle.analyze(fp.cur, fp.ref, qp=qp, search_range=R, ctu=ctu, satd_mode=satd, mvp=1)
    assert_decisions_equal(gpu, ora, ctu, where=f"{W}x{H} ctu{ctu} bd{bd}")


PARENT = [2, 3, 3, -1]


def _oracle_chain(pairs, sizes, R, r, qp, mvp):
    out = [None] * 4
    out[3] = oracle.analyze(pairs[3][2], pairs[3][3], qp=qp, search_range=R, mvp=mvp)
    for i in (2, 1, 0):  # parents before children
        p = PARENT[i]
        out[i] = oracle.analyze(pairs[i][2], pairs[i][3], qp=qp, search_range=r, dep=dep_from(out[p], sizes[p]),
                                mvp=mvp)
    return out


def test_mvp_chain_per_call_batched_and_back_to_zero():
    pairs, _ = synth.ladder_pairs(43, source=(1280, 720), rungs=[(960, 540), (640, 360), (320, 180)])
    sizes = [(w, h) for (w, h, _, _) in pairs]
    R, r, qp = 8, 3, 30
    with L.Ladder(sizes, 3, search_range=R, refine_range=r, max_frames=3) as lad:
        lad.set_parents(PARENT)
        lad.set_mv_predictor(1)
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_reference(0, *planes[3], qp)
        lad.analyze_dependents(0, [(i, planes[i][0], planes[i][1]) for i in (0, 1, 2)], qp)  # tiers inside
        lad.analyze_batch([(1, qp, planes)])
        per_call = [lad.fetch(i, 0) for i in range(4)]
        batched = [lad.fetch(i, 1) for i in range(4)]
        lad.set_mv_predictor(0)
        lad.analyze_batch([(2, qp, planes)])
        zero = [lad.fetch(i, 2) for i in range(4)]
        with pytest.raises(L.LadderError):
            lad.set_mv_predictor(2)
    ora = _oracle_chain(pairs, sizes, R, r, qp, 1)
    ora0 = _oracle_chain(pairs, sizes, R, r, qp, 0)
    for i in range(4):
        assert_decisions_equal(per_call[i], ora[i], 64, where=f"per call rung {i}")
        assert_decisions_equal(batched[i], ora[i], 64, where=f"batched rung {i}")
        assert_decisions_equal(zero[i], ora0[i], 64, where=f"predictor (0,0) rung {i}")


def test_mvp_graph_replay_new_content():
    """A captured graph bakes its launch parameters: each replay must still
    wait for its own rows (a generation per launch, kept on the device)."""
    pairs, _ = synth.ladder_pairs(44, source=(640, 360), rungs=[(480, 270), (320, 180)])
    sizes = [(w, h) for (w, h, _, _) in pairs]
    R, r, qp = 8, 3, 32
    with L.Ladder(sizes, 2, search_range=R, refine_range=r, max_frames=1) as lad:
        lad.set_mv_predictor(1)
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        stream = torch.cuda.Stream()
        graph = lad.capture_batch([(0, qp, planes)], stream)
        graph.launch(stream)
        stream.synchronize()
        first = [lad.fetch(i, 0) for i in range(3)]
        other, _ = synth.ladder_pairs(45, source=(640, 360), rungs=[(480, 270), (320, 180)])
        for i, (_, _, c, f) in enumerate(other):
            planes[i][0].copy_(L.device_plane(c))
            planes[i][1].copy_(L.device_plane(f))
        graph.launch(stream)
        graph.launch(stream)
        stream.synchronize()
        second = [lad.fetch(i, 0) for i in range(3)]
        graph.close()
        lad.sync(stream)  # raises if a wavefront wait ran out
    for got, src in ((first, pairs), (second, other)):
        ref = oracle.analyze(src[2][2], src[2][3], qp=qp, search_range=R, mvp=1)
        assert_decisions_equal(got[2], ref, 64, where="graph reference rung")
        for i in (0, 1):
            ora = oracle.analyze(src[i][2], src[i][3], qp=qp, search_range=r, dep=dep_from(ref, sizes[2]), mvp=1)
            assert_decisions_equal(got[i], ora, 64, where=f"graph rung {i}")


def test_mvp_batch_wider_than_the_device():
    """64 frames of 1920x2496 in one batch: 64 x 39 = 2496 CTU rows, more than
    the wavefront CTAs that can ever be resident (16 per SM: 2048 threads of
    128), so the decisions run as several cooperative launches.  Every frame
    equals the same frame analysed alone."""
    W, H, R, qp = 1920, 2496, 4, 30
    srcs = [synth.frame_pair(80 + k, W, H, global_range=3, patch_range=4) for k in range(4)]
    planes = [(L.device_plane(p.cur), L.device_plane(p.ref)) for p in srcs]
    with L.Ladder([(W, H)], 0, search_range=R, max_frames=64) as lad:
        lad.set_mv_predictor(1)
        lad.kernel_stats(reset=True)
        lad.analyze_batch_independent([(f, qp, [planes[f % 4]]) for f in range(64)])
        launches = lad.kernel_stats(reset=True)["decide_mvp"][0]
        got = {f: lad.fetch(0, f) for f in (0, 1, 2, 3, 33, 62, 63)}
        for f in range(64):
            lad.release_frame(f)
        alone = []
        for k in range(4):
            lad.analyze_reference(k, *planes[k], qp)
            alone.append(lad.fetch(0, k))
    assert launches >= 2, "the batch should need more than one wavefront launch"
    for f, dec in got.items():
        assert_decisions_equal(dec, alone[f % 4], 64, where=f"batched frame {f}")


@pytest.mark.parametrize("bd", [8, 10])
def test_mvp_further_qps(bd):
    """With the spatial predictor on, the decisions at further QPs equal the
    oracle's analysis at each QP with the predictor (a dependent rung keeps
    the rules of the reference decided at the master QP)."""
    pairs, _ = synth.ladder_pairs(46, source=(640, 360), rungs=[(480, 270), (320, 180)], bit_depth=bd)
    sizes = [(w, h) for (w, h, _, _) in pairs]
    R, r, master, others = 10, 3, 27, [22, 37]
    with L.Ladder(sizes, 2, bit_depth=bd, search_range=R, refine_range=r, max_frames=1) as lad:
        lad.set_mv_predictor(1)
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_reference(0, *planes[2], master)
        lad.analyze_dependents(0, [(i, planes[i][0], planes[i][1]) for i in (0, 1)], master)
        lad.kernel_stats(reset=True)
        got = {i: lad.decide_qps(i, 0, others + [master]) for i in range(3)}
        assert lad.kernel_stats()["decide_mvp"][0] == 3 * 3  # one launch per QP and rung
        master_fetch = [lad.fetch(i, 0) for i in range(3)]
    ref_master = oracle.analyze(pairs[2][2], pairs[2][3], qp=master, search_range=R, mvp=1)
    for q in others + [master]:
        for i in range(3):
            c, f = pairs[i][2], pairs[i][3]
            if i == 2:
                ora = oracle.analyze(c, f, qp=q, search_range=R, mvp=1)
            else:
                ora = oracle.analyze(c, f, qp=q, search_range=r, dep=dep_from(ref_master, sizes[2]), mvp=1)
            for k in ("cost", "best", "split"):
                for d in range(len(ora["grid"])):
                    assert np.array_equal(np.asarray(got[i][q][k][d]), np.asarray(ora[k][d])), (i, q, k, d)
            for k in ("leaf_depth", "leaf_mvx", "leaf_mvy"):
                assert np.array_equal(np.asarray(got[i][q][k]), np.asarray(ora[k])), (i, q, k)
    for i in range(3):  # the master QP again: the analysis's own decisions
        for k in ("cost", "best", "split"):
            for d in range(len(master_fetch[i]["grid"])):
                assert np.array_equal(np.asarray(got[i][master][k][d]), np.asarray(master_fetch[i][k][d]))
