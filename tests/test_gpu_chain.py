"""Cascaded reference chain (Sec. 6.5, the proposed multi-encoding scheme):
a dependent rung's refined decisions are the reference of the next tier.

Rungs 1280x720 (0), 960x540 (1), 640x360 (2), 320x180 (3, the reference):
3 -> 2 -> 0 is a chain, 3 -> 1 a direct child.  Each rung must equal the
oracle's dependent analysis against its own parent's oracle decisions."""
import pytest

import oracle
from paper_2301_12191_gb300 import synth
from helpers import assert_decisions_equal, dep_from

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402

PARENT = [2, 3, 3, -1]


def _oracle_chain(pairs, sizes, R, r, qp):
    out = [None] * 4
    out[3] = oracle.analyze(pairs[3][2], pairs[3][3], qp=qp, search_range=R)
    for i in (2, 1, 0):  # parents before children
        p = PARENT[i]
        out[i] = oracle.analyze(pairs[i][2], pairs[i][3], qp=qp, search_range=r, dep=dep_from(out[p], sizes[p]))
    return out


@pytest.mark.parametrize("bd,R,r,qp", [(8, 8, 3, 30), (10, 16, 8, 22)])
def test_chain_equals_oracle_per_call_and_batched(bd, R, r, qp):
    pairs, _ = synth.ladder_pairs(41, source=(1280, 720), rungs=[(960, 540), (640, 360), (320, 180)],
                                  bit_depth=bd)
    sizes = [(w, h) for (w, h, _, _) in pairs]
    with L.Ladder(sizes, 3, bit_depth=bd, search_range=R, refine_range=r, max_frames=2) as lad:
        lad.set_parents(PARENT)
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_reference(0, *planes[3], qp)
        lad.analyze_dependents(0, [(i, planes[i][0], planes[i][1]) for i in (0, 1, 2)], qp)  # tiers inside
        lad.analyze_batch([(1, qp, planes)])
        per_call = [lad.fetch(i, 0) for i in range(4)]
        batched = [lad.fetch(i, 1) for i in range(4)]
    ora = _oracle_chain(pairs, sizes, R, r, qp)
    for i in range(4):
        assert_decisions_equal(per_call[i], ora[i], 64, where=f"per call rung {i}")
        assert_decisions_equal(batched[i], ora[i], 64, where=f"batched rung {i}")


def test_chain_needs_the_parent_analysis():
    pairs, _ = synth.ladder_pairs(42, source=(640, 360), rungs=[(480, 270), (320, 180), (160, 90)])
    sizes = [(w, h) for (w, h, _, _) in pairs]
    with L.Ladder(sizes, 3, search_range=4, refine_range=2, max_frames=1) as lad:
        lad.set_parents(PARENT)
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_reference(0, *planes[3], 27)
        with pytest.raises(L.LadderError):
            lad.analyze_dependent(0, 0, *planes[0], 27)  # parent rung 2 not analysed yet
        lad.analyze_dependent(2, 0, *planes[2], 27)
        lad.analyze_dependent(0, 0, *planes[0], 27)
        got = lad.fetch(0, 0)
    ref = oracle.analyze(pairs[3][2], pairs[3][3], qp=27, search_range=4)
    mid = oracle.analyze(pairs[2][2], pairs[2][3], qp=27, search_range=2, dep=dep_from(ref, sizes[3]))
    top = oracle.analyze(pairs[0][2], pairs[0][3], qp=27, search_range=2, dep=dep_from(mid, sizes[2]))
    assert_decisions_equal(got, top, 64, where="rung 0 after its parent")


def test_bad_parents_are_refused():
    with L.Ladder([(128, 128), (64, 64), (32, 32)], 2, ctu_size=32, search_range=4, max_frames=1) as lad:
        for parent in ([1, 0, -1], [1, 2, 0], [0, 2, -1], [5, 2, -1], [-1, 2, -1]):
            with pytest.raises(L.LadderError):
                lad.set_parents(parent)
        lad.set_parents([1, 2, -1])
