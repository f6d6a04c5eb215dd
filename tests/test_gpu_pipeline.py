"""The frame pipeline (ladder_pipeline_*): packed frames submitted back to
back, each uploaded, analysed (reference rung, then the dependents) and read
back while its neighbours overlap, give every frame exactly the oracle's
decisions; bad layouts and depths are refused."""
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


def _layout(sizes, es):
    cur_off, ref_off, pitch, off = [], [], [], 0
    for (w, h) in sizes:
        p = (w * es + 127) // 128 * 128
        cur_off.append(off)
        ref_off.append(off + h * p)
        pitch.append(p)
        off += 2 * h * p
    return cur_off, ref_off, pitch, off


def _pack(pairs, layout, es):
    cur_off, ref_off, pitch, total = layout
    buf = torch.zeros(total, dtype=torch.uint8).pin_memory()
    nb = buf.numpy()
    for r, (w, h, c, f) in enumerate(pairs):
        for o, pl in ((cur_off[r], c), (ref_off[r], f)):
            rows = nb[o:o + h * pitch[r]].reshape(h, pitch[r])
            rows[:, :w * es] = np.ascontiguousarray(pl).view(np.uint8).reshape(h, w * es)
    return buf


# depths 4 and 5 run more analysis streams than the handle has dependent
# task-list sets (3): batches then take the least recently used set
@pytest.mark.parametrize("bd,depth", [(8, 2), (10, 3), (8, 4), (8, 5)])
def test_pipeline_frames_equal_oracle(bd, depth):
    es = 1 if bd == 8 else 2
    frames = [synth.ladder_pairs(60 + k, source=(480, 272), rungs=[(320, 180), (240, 136)], bit_depth=bd)[0]
              for k in range(5)]
    sizes = [(w, h) for (w, h, _, _) in frames[0]]
    R, r, qp = 8, 3, 30
    layout = _layout(sizes, es)
    host_in = [_pack(fr, layout, es) for fr in frames]
    with L.Ladder(sizes, 2, bit_depth=bd, search_range=R, refine_range=r, max_frames=depth + 1) as lad:
        outs = [torch.empty(lad.frame_bytes(), dtype=torch.uint8).pin_memory() for _ in range(9)]
        with lad.pipeline(depth, 10, layout[3], *layout[:3]) as pipe:
            tickets = [pipe.submit(host_in[k % 5], qp, outs[k]) for k in range(9)]
            for t in tickets:
                pipe.wait(t)
        lad.sync()
        got = [lad.frame_views(o.numpy()) for o in outs]
    for k in range(9):
        fr = frames[k % 5]
        ref = oracle.analyze(fr[2][2], fr[2][3], qp=qp, search_range=R)
        assert_decisions_equal(got[k][2], ref, 64, where=f"frame {k} reference")
        for i in (0, 1):
            ora = oracle.analyze(fr[i][2], fr[i][3], qp=qp, search_range=r, dep=dep_from(ref, sizes[2]))
            assert_decisions_equal(got[k][i], ora, 64, where=f"frame {k} rung {i}")


def test_pipeline_refuses_bad_layouts():
    sizes = [(320, 180), (160, 90)]
    cur_off, ref_off, pitch, total = _layout(sizes, 1)
    with L.Ladder(sizes, 1, search_range=8, refine_range=2, max_frames=2) as lad:
        for depth in (0, 9):
            with pytest.raises(L.LadderError):
                lad.pipeline(depth, 0, total, cur_off, ref_off, pitch)
        with pytest.raises(L.LadderError):  # unaligned plane
            lad.pipeline(2, 0, total, [cur_off[0] + 8, cur_off[1]], ref_off, pitch)
        with pytest.raises(L.LadderError):  # pitch below the width
            lad.pipeline(2, 0, total, cur_off, ref_off, [160, pitch[1]])
        with pytest.raises(L.LadderError):  # planes past the input
            lad.pipeline(2, 0, total - 16, cur_off, ref_off, pitch)
        with lad.pipeline(2, 0, total, cur_off, ref_off, pitch) as pipe:
            with pytest.raises(L.LadderError):
                pipe.wait(0)  # nothing submitted
