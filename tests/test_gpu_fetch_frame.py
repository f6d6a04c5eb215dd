"""The asynchronous whole-frame fetch returns, per rung, exactly what the
synchronous per-rung fetch returns."""
import numpy as np
import pytest

from paper_2301_12191_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402

FIELDS = ("mvx", "mvy", "sad", "satd", "cost", "best", "split", "evaluated")


def test_fetch_frame_async_equals_per_rung_fetch():
    pairs, _ = synth.ladder_pairs(51, source=(640, 360), rungs=[(480, 270), (320, 180)])
    sizes = [(w, h) for (w, h, _, _) in pairs]
    with L.Ladder(sizes, 2, search_range=8, refine_range=2, max_frames=2) as lad:
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.analyze_batch([(7, 27, planes)])
        host = torch.empty(lad.frame_bytes(), dtype=torch.uint8).pin_memory()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        lad.fetch_frame_async(7, host, s)
        s.synchronize()
        views = lad.frame_views(host.numpy())
        for r in range(len(sizes)):
            ref = lad.fetch(r, 7)
            for k in FIELDS:
                for d in range(len(ref["grid"])):
                    assert np.array_equal(views[r][k][d], ref[k][d]), (r, k, d)
            for k in ("leaf_depth", "leaf_mvx", "leaf_mvy"):
                assert np.array_equal(views[r][k], ref[k]), (r, k)
        with pytest.raises(L.LadderError):
            lad.fetch_frame_async(8, host, s)  # no such frame
