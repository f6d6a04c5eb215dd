"""Further-QP decisions (intra-resolution multi-QP sharing, Sec. 4.2).

One analysis per rung at the master QP (the median of the QP set, here 27);
the cost, split and leaf maps at the other QPs come from ladder_decide_qps.
Because the motion search (pure SAD) and the SATDs at the chosen vectors do
not depend on the QP, each result must equal the oracle's analysis of that
rung at that QP; a dependent rung keeps the rules derived from the reference
analysed at the master QP."""
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

FIELDS = ("cost", "best", "split")
MASTER, OTHERS = 27, [22, 32, 37]


def _check(got, ora, where):
    for k in FIELDS:
        for d in range(len(ora["grid"])):
            g, o = np.asarray(got[k][d]), np.asarray(ora[k][d])
            assert np.array_equal(g, o), f"{where}: {k} depth {d}: {np.count_nonzero(g != o)} mismatches"
    for k in ("leaf_depth", "leaf_mvx", "leaf_mvy"):
        assert np.array_equal(np.asarray(got[k]), np.asarray(ora[k])), f"{where}: {k}"


@pytest.mark.parametrize("bd,R,r,satd", [(8, 12, 3, 0), (10, 8, 2, 1)])
def test_further_qps_equal_analysis_at_each_qp(bd, R, r, satd):
    pairs, _ = synth.ladder_pairs(31, source=(640, 360), rungs=[(480, 270), (320, 180)], bit_depth=bd)
    sizes = [(w, h) for (w, h, _, _) in pairs]
    ref_i = 2
    with L.Ladder(sizes, ref_i, bit_depth=bd, search_range=R, refine_range=r, satd_mode=satd,
                  max_frames=1) as lad:
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_reference(0, *planes[ref_i], MASTER)
        lad.analyze_dependents(0, [(i, planes[i][0], planes[i][1]) for i in (0, 1)], MASTER)
        got = {i: lad.decide_qps(i, 0, OTHERS + [MASTER]) for i in range(3)}
        master_fetch = [lad.fetch(i, 0) for i in range(3)]
    ref_master = oracle.analyze(pairs[ref_i][2], pairs[ref_i][3], qp=MASTER, search_range=R, satd_mode=satd)
    for q in OTHERS + [MASTER]:
        for i in range(3):
            c, f = pairs[i][2], pairs[i][3]
            if i == ref_i:
                ora = oracle.analyze(c, f, qp=q, search_range=R, satd_mode=satd)
            else:
                ora = oracle.analyze(c, f, qp=q, search_range=r, satd_mode=satd, dep=dep_from(ref_master, sizes[ref_i]))
            _check(got[i][q], ora, f"rung {i} qp {q}")
    # the master QP recomputed equals the analysis's own decisions
    for i in range(3):
        _check(got[i][MASTER], master_fetch[i], f"rung {i} master")


def test_bad_arguments():
    with L.Ladder([(64, 64)], 0, ctu_size=32, search_range=4, max_frames=1) as lad:
        with pytest.raises(L.LadderError):
            lad.decide_qps(0, 0, [22])  # frame not analysed
        p = synth.frame_pair(3, 64, 64)
        lad.analyze_reference(0, L.device_plane(p.cur), L.device_plane(p.ref), 27)
        for qps in ([52], [-1], list(range(20, 29))):
            with pytest.raises(L.LadderError):
                lad.decide_qps(0, 0, qps)
        assert set(lad.decide_qps(0, 0, [30])) == {30}
