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
    ref_ana = oracle.analyze(pairs[2][2], pairs[2][3], qp=qp, search_range=R, ctu=ctu, satd_mode=satd)
    want = {2: oracle.refine_subpel(pairs[2][2], pairs[2][3], ref_ana, qp=qp, ctu=ctu, satd_mode=satd)}
    for i in (0, 1):
        dep = dep_from(ref_ana, sizes[2])
        ana = oracle.analyze(pairs[i][2], pairs[i][3], qp=qp, search_range=r, ctu=ctu, satd_mode=satd, dep=dep)
        want[i] = oracle.refine_subpel(pairs[i][2], pairs[i][3], ana, qp=qp, ctu=ctu, satd_mode=satd, dep=dep)
    for i in range(3):
        _check(got[i], want[i], f"rung {i} bd{bd} satd{satd}")


def test_subpel_needs_an_analysis():
    with L.Ladder([(64, 64)], 0, ctu_size=32, search_range=4, max_frames=1) as lad:
        p = synth.frame_pair(3, 64, 64)
        c, f = L.device_plane(p.cur), L.device_plane(p.ref)
        with pytest.raises(L.LadderError):
            lad.refine_subpel(0, 0, c, f, 27)
