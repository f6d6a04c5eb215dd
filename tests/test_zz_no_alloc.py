"""The allocation-free entry point (analyze_reference_noalloc) against the
regular one (analyze_reference on a one-rung ladder).

Some callers cannot call cudaMalloc (an encoder plugin whose host
application owns all device memory, a real-time pipeline that forbids
allocation after start-up); this entry point serves them from a fixed
scratch array inside the library.  The check: two calls in a row, on
different frames of the same geometry, each equal (bit-exact, as every
result of this library) to the regular entry point's decisions, so the
shared scratch carries nothing from one call into the next.  The file is
collected last so that a stop at the first failure has already run every
other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402
from paper_2301_12191_gb300 import synth  # noqa: E402
from helpers import assert_decisions_equal  # noqa: E402

FIELDS = (("mvx", torch.int16), ("mvy", torch.int16), ("sad", torch.int32), ("satd", torch.int32),
          ("cost", torch.int32), ("best", torch.int32), ("split", torch.uint8), ("evaluated", torch.uint8))


def _noalloc_run(fp, ctu, R, qp, satd_mode, dims, grid8, check_status=True):
    """Caller-owned device outputs, filled by the allocation-free call."""
    dev = {k: [torch.full((c * r,), -7, dtype=dt, device="cuda") for (c, r) in dims] for k, dt in FIELDS}
    n8 = grid8[0] * grid8[1]
    leaf = {"leaf_depth": torch.full((n8,), 9, dtype=torch.uint8, device="cuda"),
            "leaf_mvx": torch.full((n8,), -7, dtype=torch.int16, device="cuda"),
            "leaf_mvy": torch.full((n8,), -7, dtype=torch.int16, device="cuda")}
    dec = L.Decisions()
    for k, _ in FIELDS:
        for d, t in enumerate(dev[k]):
            getattr(dec, k)[d] = t.data_ptr()
    for k, t in leaf.items():
        setattr(dec, k, t.data_ptr())
    cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
    stream = torch.cuda.current_stream()
    L.analyze_reference_noalloc(cur.data_ptr(), ref.data_ptr(), fp.width, fp.height,
                                int(cur.stride(0) * cur.element_size()), fp.bit_depth, ctu, R, qp, satd_mode, dec,
                                int(stream.cuda_stream))
    torch.cuda.synchronize()
    if check_status:   # no bounded wait ran out (the status query allocates nothing either)
        assert L.analyze_reference_noalloc_status(int(stream.cuda_stream)) == 0
    out = {k: [t.cpu().numpy() for t in dev[k]] for k, _ in FIELDS}
    out.update({k: t.cpu().numpy() for k, t in leaf.items()})
    out["grid"] = dims
    out["grid8"] = grid8
    return out


def _regular_run(fp, ctu, R, qp, satd_mode):
    with L.Ladder([(fp.width, fp.height)], 0, bit_depth=fp.bit_depth, ctu_size=ctu, search_range=R,
                  satd_mode=satd_mode, max_frames=1) as lad:
        cur, ref = L.device_plane(fp.cur), L.device_plane(fp.ref)
        lad.analyze_reference(0, cur, ref, qp)
        return lad.fetch(0, 0)


@pytest.mark.parametrize("W,H,bd,ctu,R,qp,satd", [
    (416, 240, 8, 64, 16, 32, 0),
    (200, 120, 10, 32, 12, 27, 1),
])
def test_noalloc_equals_regular_entry_point_on_two_calls(W, H, bd, ctu, R, qp, satd):
    frames = [synth.frame_pair(seed, W, H, bd) for seed in (101, 202)]
    for fp in frames:   # two calls in a row through the shared scratch
        reg = _regular_run(fp, ctu, R, qp, satd)
        got = _noalloc_run(fp, ctu, R, qp, satd, reg["grid"], reg["grid8"])
        assert_decisions_equal(got, reg, ctu, where=f"noalloc {W}x{H} bd{bd}")


def test_noalloc_near_its_limit_2160p_10bit():
    """3840x2160 10-bit at CTU 64 (2040 of the 3083 CTUs the scratch holds),
    every CTU against the regular entry point."""
    fp = synth.frame_pair(303, 3840, 2160, 10, global_range=8, patch_range=12, patch_size=64)
    reg = _regular_run(fp, 64, 8, 27, 0)
    got = _noalloc_run(fp, 64, 8, 27, 0, reg["grid"], reg["grid8"])
    assert_decisions_equal(got, reg, 64, where="noalloc 2160p 10-bit")


def test_noalloc_refuses_frames_beyond_its_scratch():
    # 4096x3200 needs 3200 CTUs of 64x64, more than the 3083 the scratch holds
    dummy = torch.zeros((16, 4096), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LadderError) as e:
        L.analyze_reference_noalloc(dummy.data_ptr(), dummy.data_ptr(), 4096, 3200, 4096, 8, 64, 16, 32, 0,
                                    L.Decisions(), 0)
    assert e.value.status == -1
