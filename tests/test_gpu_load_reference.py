"""Analysis save and load (App. A.1: encodes that reuse a master encode's
analysis read it back instead of analysing again): a reference analysis
fetched from one handle and loaded into another lets the second handle
analyse the dependents exactly as if it had analysed the reference itself,
and exactly as the oracle does."""
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


@pytest.mark.parametrize("bd", [8, 10])
def test_loaded_reference_resumes_the_dependents(bd):
    pairs, _ = synth.ladder_pairs(91, source=(960, 544), rungs=[(640, 360), (320, 180)], bit_depth=bd)
    sizes = [(w, h) for (w, h, _, _) in pairs]
    kw = dict(bit_depth=bd, search_range=12, refine_range=4, max_frames=2)
    planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
    with L.Ladder(sizes, 2, **kw) as a:
        a.analyze_reference(3, *planes[2], 27)
        a.analyze_dependents(3, [(i, *planes[i]) for i in (0, 1)], 27)
        saved = a.fetch(2, 3)
        want = [a.fetch(i, 3) for i in (0, 1)]
    with L.Ladder(sizes, 2, **kw) as b:        # a fresh handle: only the saved analysis
        with pytest.raises(L.LadderError) as e:
            b.analyze_dependent(0, 8, *planes[0], 27)
        assert e.value.status == -3              # no reference yet
        b.load_reference(8, saved)
        b.analyze_dependents(8, [(i, *planes[i]) for i in (0, 1)], 27)
        got = [b.fetch(i, 8) for i in (0, 1)]
        back = b.fetch(2, 8)
    assert_decisions_equal(back, saved, 64, where="loaded reference read back")
    for i in (0, 1):
        assert_decisions_equal(got[i], want[i], 64, where=f"rung {i} after load vs after analysis")
        ora = oracle.analyze(pairs[i][2], pairs[i][3], qp=27, search_range=4, dep=dep_from(saved, sizes[2]))
        assert_decisions_equal(got[i], ora, 64, where=f"rung {i} after load vs oracle")


def test_load_reference_refuses_bad_input():
    with L.Ladder([(128, 64), (64, 32)], 1, search_range=8, max_frames=1) as lad:
        with pytest.raises(L.LadderError):
            L._call(lad.handle, "ladder_load_reference", lad.handle, 0, L.Decisions(), 0)  # no arrays
        fp = synth.frame_pair(92, 64, 32, 8)
        lad.analyze_reference(1, L.device_plane(fp.cur), L.device_plane(fp.ref), 30)
        saved = lad.fetch(1, 1)
        with pytest.raises(L.LadderError) as e:
            lad.load_reference(2, saved)        # the only slot holds frame 1
        assert e.value.status == -4
        bad = dict(saved, leaf_mvx=np.zeros(3, np.int16))
        with pytest.raises(ValueError):
            lad.load_reference(1, bad)
        lad.load_reference(1, saved)            # re-loading a frame that holds the slot reuses it
        lad.sync()
