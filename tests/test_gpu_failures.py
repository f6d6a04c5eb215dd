"""Failure detection without a GPU fault: a bounded device wait is made to
run out on purpose (the wavefront rows of the spatial-predictor decisions
wait for a hand-off that no row publishes, with a short poll limit), and
every way results leave the library reports it: ladder_sync, a fetch of the
decisions, and the frame pipeline's wait / next submit.  The handle stays
usable: the next analysis with normal hand-offs matches the oracle.
Nothing here traps, faults or waits without a bound."""
import numpy as np
import pytest

import oracle
from paper_2301_12191_gb300 import synth
from helpers import assert_decisions_equal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402

TIMEOUT = -6
POLLS = 4096   # each poll is one L2 round trip: a few milliseconds per wait


def test_wavefront_wait_runs_out_and_is_reported():
    fp = synth.frame_pair(81, 256, 200, 8)     # 4 CTU rows: rows 1..3 wait on the row above
    with L.Ladder([(256, 200)], 0, search_range=8, max_frames=1) as lad:
        cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
        lad.set_mv_predictor(1)
        lad.set_debug(wait_polls=POLLS, lost_handoff=1)
        lad.analyze_reference(0, cur, ref, 30)
        with pytest.raises(L.LadderError) as e:
            lad.sync()
        assert e.value.status == TIMEOUT
        lad.sync()                              # reported once: the word is clear again
        # a fetch of a timed-out analysis reports it too
        lad.analyze_reference(0, cur, ref, 30)
        with pytest.raises(L.LadderError) as e:
            lad.fetch(0, 0)
        assert e.value.status == TIMEOUT
        # normal hand-offs again: the same handle gives the oracle's decisions
        lad.set_debug(wait_polls=0, lost_handoff=0)
        lad.analyze_reference(0, cur, ref, 30)
        got = lad.fetch(0, 0)
    ora = oracle.analyze(fp.cur, fp.ref, qp=30, search_range=8, mvp=1)
    assert_decisions_equal(got, ora, 64, where="after recovery")


def test_pipeline_reports_a_device_timeout():
    pairs, _ = synth.ladder_pairs(82, source=(512, 320), rungs=[(256, 160)])
    sizes = [(w, h) for (w, h, _, _) in pairs]
    pitch = [(w + 127) // 128 * 128 for (w, _) in sizes]
    cur_off, ref_off, off = [], [], 0
    for (w, h), p in zip(sizes, pitch):
        cur_off.append(off)
        ref_off.append(off + h * p)
        off += 2 * h * p
    host_in = torch.zeros(off, dtype=torch.uint8).pin_memory()
    nb = host_in.numpy()
    for r, (w, h, c, f) in enumerate(pairs):
        for o, pl in ((cur_off[r], c), (ref_off[r], f)):
            nb[o:o + h * pitch[r]].reshape(h, pitch[r])[:, :w] = pl
    with L.Ladder(sizes, 1, search_range=8, refine_range=3, max_frames=3) as lad:
        outs = [torch.empty(lad.frame_bytes(), dtype=torch.uint8).pin_memory() for _ in range(4)]
        lad.set_mv_predictor(1)
        lad.set_debug(wait_polls=POLLS, lost_handoff=1)
        with lad.pipeline(2, 0, off, cur_off, ref_off, pitch) as pipe:
            t0 = pipe.submit(host_in, 30, outs[0])
            with pytest.raises(L.LadderError) as e:
                pipe.wait(t0)
            assert e.value.status == TIMEOUT
            # a frame nobody waited for: the next submit on its slot reports it
            pipe.submit(host_in, 30, outs[1])
            t2 = pipe.submit(host_in, 30, outs[2])
            with pytest.raises(L.LadderError) as e:
                pipe.submit(host_in, 30, outs[3])
            assert e.value.status == TIMEOUT
            with pytest.raises(L.LadderError) as e:   # the frame still in flight then timed out too
                pipe.wait(t2)
            assert e.value.status == TIMEOUT
            lad.set_debug(wait_polls=0, lost_handoff=0)
            lad.sync()
            # recovered: frames decide normally again
            t = pipe.submit(host_in, 30, outs[3])
            pipe.wait(t)
            got = lad.frame_views(outs[3].numpy())
    ref = oracle.analyze(pairs[1][2], pairs[1][3], qp=30, search_range=8, mvp=1)
    assert_decisions_equal(got[1], ref, 64, where="pipeline after recovery")


def test_debug_controls_are_validated():
    with L.Ladder([(64, 64)], 0, search_range=4, max_frames=1) as lad:
        for kw in ({"wait_polls": 10}, {"wait_polls": 1 << 23}, {"lost_handoff": 2}):
            with pytest.raises(L.LadderError):
                lad.set_debug(**kw)
        with pytest.raises(L.LadderError):
            L._call(lad.handle, "ladder_set_debug", lad.handle, 7, 0)
        lad.set_debug(wait_polls=64, lost_handoff=0)
        lad.set_debug(wait_polls=0)
    assert np.int32(TIMEOUT) == -6


def test_refinement_wavefront_wait_runs_out_and_is_reported():
    """The quarter-pel refinement with the spatial predictor has a wavefront
    of its own: its rows' waits run out the same way, ladder_sync reports
    it, and the next refinement with normal hand-offs matches the oracle."""
    fp = synth.frame_pair(83, 256, 200, 8)
    with L.Ladder([(256, 200)], 0, search_range=8, max_frames=1) as lad:
        cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
        lad.set_mv_predictor(1)
        lad.analyze_reference(0, cur, ref, 30)
        lad.sync()
        lad.set_debug(wait_polls=POLLS, lost_handoff=1)
        lad.refine_subpel(0, 0, cur, ref, 30)
        with pytest.raises(L.LadderError) as e:
            lad.sync()
        assert e.value.status == TIMEOUT
        lad.set_debug(wait_polls=0, lost_handoff=0)
        got = lad.refine_subpel(0, 0, cur, ref, 30)
        lad.sync()
    ana = oracle.analyze(fp.cur, fp.ref, qp=30, search_range=8, mvp=1)
    want = oracle.refine_subpel(fp.cur, fp.ref, ana, qp=30, mvp=1)
    for k in ("qmvx", "qmvy", "satd", "cost", "best", "split"):
        for d in range(len(want["grid"])):
            assert np.array_equal(np.asarray(got[k][d]), want[k][d]), (k, d)
    for k in ("leaf_depth", "leaf_qmvx", "leaf_qmvy"):
        assert np.array_equal(np.asarray(got[k]), want[k]), k
