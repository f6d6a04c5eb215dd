"""Quarter-pel refinement with SATD: the CUDA path equals the oracle's
refinement of the oracle's own analysis, field for field (refined vectors,
SATD, cost, best, split, leaf maps), for an independent and two dependent
rungs, 8- and 10-bit, both SATD modes."""
import numpy as np
import pytest

import oracle
from paper_2301_12191_gb300 import synth
from helpers import dep_from

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402

FIELDS = ("qmvx", "qmvy", "satd", "cost", "best", "split")


def _check(got, want, where):
    for k in FIELDS:
        for d in range(len(want["grid"])):
            g, o = np.asarray(got[k][d]), np.asarray(want[k][d])
            assert np.array_equal(g, o), f"{where}: {k} depth {d}: {np.count_nonzero(g != o)} mismatches"
    for k in ("leaf_depth", "leaf_qmvx", "leaf_qmvy"):
        assert np.array_equal(np.asarray(got[k]), np.asarray(want[k])), f"{where}: {k}"


@pytest.mark.parametrize("bd,satd,ctu", [(8, 0, 64), (10, 1, 32)])
def test_subpel_matches_oracle(bd, satd, ctu):
    pairs, _ = synth.ladder_pairs(71, source=(480, 270), rungs=[(400, 224), (320, 180)], bit_depth=bd)
    sizes = [(w, h) for (w, h, _, _) in pairs]
    R, r, qp = 8, 3, 30
    with L.Ladder(sizes, 2, bit_depth=bd, ctu_size=ctu, search_range=R, refine_range=r, satd_mode=satd,
                  max_frames=1) as lad:
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_reference(0, *planes[2], qp)
        lad.analyze_dependents(0, [(i, planes[i][0], planes[i][1]) for i in (0, 1)], qp)
        got = [lad.refine_subpel(i, 0, planes[i][0], planes[i][1], qp) for i in range(3)]
        # the same three refinements as one batched call (independent rung first inside)
        got_batch = lad.refine_subpel_batch([(0, i, planes[i][0], planes[i][1], qp) for i in (0, 2, 1)])
    ref_ana = oracle.analyze(pairs[2][2], pairs[2][3], qp=qp, search_range=R, ctu=ctu, satd_mode=satd)
    want = {2: oracle.refine_subpel(pairs[2][2], pairs[2][3], ref_ana, qp=qp, ctu=ctu, satd_mode=satd)}
    for i in (0, 1):
        dep = dep_from(ref_ana, sizes[2])
        ana = oracle.analyze(pairs[i][2], pairs[i][3], qp=qp, search_range=r, ctu=ctu, satd_mode=satd, dep=dep)
        want[i] = oracle.refine_subpel(pairs[i][2], pairs[i][3], ana, qp=qp, ctu=ctu, satd_mode=satd, dep=dep)
    for i in range(3):
        _check(got[i], want[i], f"rung {i} bd{bd} satd{satd}")
    for k, i in enumerate((0, 2, 1)):
        _check(got_batch[k], want[i], f"batched rung {i} bd{bd} satd{satd}")


def test_subpel_needs_an_analysis():
    with L.Ladder([(64, 64)], 0, ctu_size=32, search_range=4, max_frames=1) as lad:
        p = synth.frame_pair(3, 64, 64)
        c, f = L.device_plane(p.cur), L.device_plane(p.ref)
        with pytest.raises(L.LadderError):
            lad.refine_subpel(0, 0, c, f, 27)


@pytest.mark.parametrize("bd,W,H,gmv,ctu", [(8, 72, 40, (14, -11), 32), (10, 40, 24, (-13, 9), 16),
                                             (8, 18, 16, (3, -2), 16)])
def test_subpel_edges(bd, W, H, gmv, ctu):
    """Vectors that reach past the frame (prediction from clamped samples),
    ragged CTUs and a frame of the smallest size a ladder accepts."""
    p = synth.frame_pair(29, W, H, bit_depth=bd, global_mv=gmv, patch_size=8)
    R, qp = 16, 25
    with L.Ladder([(W, H)], 0, bit_depth=bd, ctu_size=ctu, search_range=R, max_frames=1) as lad:
        c, f = L.device_plane(p.cur), L.device_plane(p.ref)
        lad.analyze_reference(0, c, f, qp)
        got = lad.refine_subpel(0, 0, c, f, qp)
    ana = oracle.analyze(p.cur, p.ref, qp=qp, search_range=R, ctu=ctu)
    want = oracle.refine_subpel(p.cur, p.ref, ana, qp=qp, ctu=ctu)
    _check(got, want, f"{W}x{H} bd{bd}")


def test_subpel_workspace_checked():
    import ctypes
    with L.Ladder([(64, 48)], 0, ctu_size=32, search_range=4, max_frames=1) as lad:
        p = synth.frame_pair(4, 64, 48)
        c, f = L.device_plane(p.cur), L.device_plane(p.ref)
        lad.analyze_reference(0, c, f, 27)
        need = int(L.load().ladder_subpel_workspace_bytes(lad.handle, 0))
        assert need >= 16 * 56 * 72 and int(L.load().ladder_subpel_workspace_bytes(lad.handle, 1)) == 0
        t, o, ws = lad.subpel_buffers(0)
        with pytest.raises(L.LadderError):
            L._call(lad.handle, "ladder_refine_subpel", lad.handle, 0, 0, c.data_ptr(), f.data_ptr(),
                    L._pitch_bytes(c), 27, ctypes.byref(o), ws.data_ptr(), need - 1, None)
        with pytest.raises(L.LadderError):
            L._call(lad.handle, "ladder_refine_subpel", lad.handle, 0, 0, c.data_ptr(), f.data_ptr(),
                    L._pitch_bytes(c), 27, ctypes.byref(o), ws.data_ptr() + 16, need, None)


def test_subpel_workspace_reused_across_frames():
    """One workspace, two frames with different references, back to back on
    one stream: each refinement sees its own interpolated planes."""
    W, H, R, qp = 136, 72, 8, 27
    ps = [synth.frame_pair(40 + k, W, H, global_mv=(3 - 5 * k, 2 * k - 1)) for k in range(2)]
    with L.Ladder([(W, H)], 0, ctu_size=32, search_range=R, max_frames=2) as lad:
        dev = [(L.device_plane(p.cur), L.device_plane(p.ref)) for p in ps]
        bufs = [lad.subpel_buffers(0) for _ in range(2)]
        ws = bufs[0][2]
        for k in range(2):
            lad.analyze_reference(k, *dev[k], qp)
        import ctypes
        s = torch.cuda.current_stream()
        for k in range(2):
            L._call(lad.handle, "ladder_refine_subpel", lad.handle, 0, k, dev[k][0].data_ptr(), dev[k][1].data_ptr(),
                    L._pitch_bytes(dev[k][0]), qp, ctypes.byref(bufs[k][1]), ws.data_ptr(), ws.numel(),
                    ctypes.c_void_p(s.cuda_stream))
        s.synchronize()
        got = [{k: ([a.cpu().numpy() for a in v] if isinstance(v, list) else v.cpu().numpy())
                for k, v in bufs[i][0].items()} for i in range(2)]
    for k, p in enumerate(ps):
        ana = oracle.analyze(p.cur, p.ref, qp=qp, search_range=R, ctu=32)
        want = oracle.refine_subpel(p.cur, p.ref, ana, qp=qp, ctu=32)
        _check(got[k], want, f"frame {k}")


def test_subpel_batch_checked():
    """Job counts outside 1..16 and a job that fails its checks launch nothing."""
    import ctypes
    with L.Ladder([(64, 48), (32, 24)], 1, ctu_size=32, search_range=4, refine_range=2, max_frames=1) as lad:
        p = synth.frame_pair(4, 64, 48)
        q = synth.frame_pair(5, 32, 24)
        c, f = L.device_plane(p.cur), L.device_plane(p.ref)
        c2, f2 = L.device_plane(q.cur), L.device_plane(q.ref)
        lad.analyze_reference(0, c2, f2, 27)
        bufs = [lad.subpel_buffers(0), lad.subpel_buffers(1)]
        jobs = lad.subpel_jobs([(0, 1, c2, f2, 27), (0, 0, c, f, 27)], bufs)
        for n in (0, L.MAX_SUBPEL_JOBS + 1):
            with pytest.raises(L.LadderError):
                L._call(lad.handle, "ladder_refine_subpel_batch", lad.handle, n, jobs, None)
        with pytest.raises(L.LadderError):  # rung 0 of frame 0 has not been analysed
            L._call(lad.handle, "ladder_refine_subpel_batch", lad.handle, 2, jobs, None)
        # the analysed job alone goes through
        L._call(lad.handle, "ladder_refine_subpel_batch", lad.handle, 1, jobs, None)
        torch.cuda.synchronize()


# ------------------------------------------- spatial MV predictor -----
@pytest.mark.parametrize("bd,satd,ctu", [(8, 0, 64), (10, 1, 32), (8, 0, 16)])
def test_subpel_spatial_predictor_matches_oracle(bd, satd, ctu):
    """With the spatial predictor on, the refinement (SATD tables, then the
    wavefront over the refined quarter-pel vectors) equals the oracle's
    refinement with mvp=1 of its own mvp=1 analysis: an independent and two
    dependent rungs, per call and batched."""
    pairs, _ = synth.ladder_pairs(73, source=(480, 270), rungs=[(400, 224), (320, 180)], bit_depth=bd)
    sizes = [(w, h) for (w, h, _, _) in pairs]
    R, r, qp = 8, 3, 36
    with L.Ladder(sizes, 2, bit_depth=bd, ctu_size=ctu, search_range=R, refine_range=r, satd_mode=satd,
                  max_frames=1) as lad:
        lad.set_mv_predictor(1)
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_reference(0, *planes[2], qp)
        lad.analyze_dependents(0, [(i, planes[i][0], planes[i][1]) for i in (0, 1)], qp)
        got = [lad.refine_subpel(i, 0, planes[i][0], planes[i][1], qp) for i in range(3)]
        got_batch = lad.refine_subpel_batch([(0, i, planes[i][0], planes[i][1], qp) for i in (0, 2, 1)])
        lad.sync()
        # back to the predictor (0, 0): the two-round kernel again
        lad.set_mv_predictor(0)
        zero = lad.refine_subpel(2, 0, planes[2][0], planes[2][1], qp)
    ref_ana = oracle.analyze(pairs[2][2], pairs[2][3], qp=qp, search_range=R, ctu=ctu, satd_mode=satd, mvp=1)
    want = {2: oracle.refine_subpel(pairs[2][2], pairs[2][3], ref_ana, qp=qp, ctu=ctu, satd_mode=satd, mvp=1)}
    for i in (0, 1):
        dep = dep_from(ref_ana, sizes[2])
        ana = oracle.analyze(pairs[i][2], pairs[i][3], qp=qp, search_range=r, ctu=ctu, satd_mode=satd, dep=dep,
                             mvp=1)
        want[i] = oracle.refine_subpel(pairs[i][2], pairs[i][3], ana, qp=qp, ctu=ctu, satd_mode=satd, dep=dep,
                                       mvp=1)
    for i in range(3):
        _check(got[i], want[i], f"mvp rung {i} bd{bd} satd{satd} ctu{ctu}")
    for k, i in enumerate((0, 2, 1)):
        _check(got_batch[k], want[i], f"mvp batched rung {i} bd{bd} satd{satd} ctu{ctu}")
    want0 = oracle.refine_subpel(pairs[2][2], pairs[2][3], ref_ana, qp=qp, ctu=ctu, satd_mode=satd, mvp=0)
    _check(zero, want0, f"predictor (0, 0) after mode 1, bd{bd}")
    # the predictor changes some refined cost (the case is not vacuous)
    assert any(not np.array_equal(np.asarray(want[2]["cost"][d]), np.asarray(want0["cost"][d]))
               for d in range(len(want0["grid"])))


@pytest.mark.parametrize("bd,W,H,gmv,ctu", [(8, 72, 40, (14, -11), 32), (10, 40, 24, (-13, 9), 16),
                                             (8, 200, 136, (-6, 5), 16)])
def test_subpel_spatial_predictor_edges(bd, W, H, gmv, ctu):
    """Ragged CTUs and vectors past the frame with the spatial predictor;
    the last case has more CTU rows than columns (deep wavefront)."""
    p = synth.frame_pair(31, W, H, bit_depth=bd, global_mv=gmv, patch_size=8)
    R, qp = 16, 33
    with L.Ladder([(W, H)], 0, bit_depth=bd, ctu_size=ctu, search_range=R, max_frames=1) as lad:
        lad.set_mv_predictor(1)
        c, f = L.device_plane(p.cur), L.device_plane(p.ref)
        lad.analyze_reference(0, c, f, qp)
        got = lad.refine_subpel(0, 0, c, f, qp)
        again = lad.refine_subpel(0, 0, c, f, qp)  # a second launch on the same hand-off words
        lad.sync()
    ana = oracle.analyze(p.cur, p.ref, qp=qp, search_range=R, ctu=ctu, mvp=1)
    want = oracle.refine_subpel(p.cur, p.ref, ana, qp=qp, ctu=ctu, mvp=1)
    _check(got, want, f"mvp {W}x{H} bd{bd}")
    _check(again, want, f"mvp again {W}x{H} bd{bd}")
