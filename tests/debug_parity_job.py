"""Small parity cases on the bounds-checked debug library (run by
tests/test_gpu_debug_build.py in a process of its own with
LADDER_DEBUG_BUILD=1).  Every fetch and sync also reads the device status
word, so a failed device-side bounds check fails the case with
LADDER_E_BOUNDS; the decisions must still equal the oracle's."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from helpers import assert_decisions_equal, dep_from  # noqa: E402
from paper_2301_12191_gb300 import ladder as L, synth  # noqa: E402


def main():
    assert L.debug_build_requested()
    version = L.load().ladder_version().decode()
    assert "bounds-checked" in version, version
    cases = 0
    # independent analyses: fused and separate decisions, 8/10-bit, CTU 16/32/64, ragged frames
    for (W, H, ctu, R, bd, fuse) in ((100, 70, 64, 8, 8, 1), (130, 66, 32, 5, 8, 0), (96, 48, 16, 6, 10, 1),
                                     (200, 120, 64, 16, 10, 0), (192, 128, 64, 64, 10, 1)):
        fp = synth.frame_pair(W + H, W, H, bd, global_range=3, patch_range=5, patch_size=24)
        with L.Ladder([(W, H)], 0, bit_depth=bd, ctu_size=ctu, search_range=R, max_frames=1) as lad:
            lad.set_tuning(fs_fuse=fuse)
            lad.analyze_reference(0, L.device_plane(fp.cur), L.device_plane(fp.ref), 30)
            got = lad.fetch(0, 0)
        assert_decisions_equal(got, oracle.analyze(fp.cur, fp.ref, qp=30, search_range=R, ctu=ctu), ctu,
                               where=f"debug independent {W}x{H}")
        cases += 1
    # dependent ladders: L1 and staged searches (one and two buffers), both bands, pieces of 16 and 32
    for bd, r, knobs in ((8, 4, {}), (10, 8, {"dep_staged": 1}), (10, 8, {"dep_staged": 2, "dep_band": 17}),
                         (10, 8, {"dep_staged": 0}), (10, 8, {"dep_staged": 1, "dep_range": 32}),
                         (10, 5, {"dep_staged": 1})):
        pairs, _ = synth.ladder_pairs(40 + r, source=(640, 360), rungs=[(480, 270), (320, 180)], bit_depth=bd)
        sizes = [(w, h) for (w, h, _, _) in pairs]
        with L.Ladder(sizes, 2, bit_depth=bd, search_range=12, refine_range=r, max_frames=1) as lad:
            lad.set_tuning(**knobs)
            planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
            lad.analyze_batch([(0, 27, planes)])
            got = [lad.fetch(i, 0) for i in range(3)]
        ref = oracle.analyze(pairs[2][2], pairs[2][3], qp=27, search_range=12)
        assert_decisions_equal(got[2], ref, 64, where="debug reference")
        for i in (0, 1):
            ora = oracle.analyze(pairs[i][2], pairs[i][3], qp=27, search_range=r, dep=dep_from(ref, sizes[2]))
            assert_decisions_equal(got[i], ora, 64, where=f"debug dependent bd{bd} r{r} {knobs} rung {i}")
        cases += 1
    # spatial predictor (wavefront decisions) and further QPs
    fp = synth.frame_pair(77, 256, 200, 8)
    with L.Ladder([(256, 200)], 0, search_range=8, max_frames=1) as lad:
        lad.set_mv_predictor(1)
        lad.analyze_reference(0, L.device_plane(fp.cur), L.device_plane(fp.ref), 30)
        got = lad.fetch(0, 0)
        qps = lad.decide_qps(0, 0, [22, 37])
        lad.sync()
    assert_decisions_equal(got, oracle.analyze(fp.cur, fp.ref, qp=30, search_range=8, mvp=1), 64,
                           where="debug spatial predictor")
    for q in (22, 37):
        o = oracle.analyze(fp.cur, fp.ref, qp=q, search_range=8, mvp=1)
        for d in range(4):
            assert (qps[q]["cost"][d] == o["cost"][d]).all()
    cases += 1
    print(f"debug build ok: {cases} cases, {version}")


if __name__ == "__main__":
    main()
