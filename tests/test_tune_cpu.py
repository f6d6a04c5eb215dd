"""The autotuner's search and cache on the host (fake ladder, fake timer)."""
import types

import pytest

from paper_2301_12191_gb300 import tune
from paper_2301_12191_gb300.ladder import LadderError


class FakeLadder:
    def __init__(self, ctu=64):
        self.rungs = [(1280, 720), (640, 360)]
        self.geometry = types.SimpleNamespace(bit_depth=8, ctu_size=ctu, ref_search_range=32, dep_refine_range=4,
                                              ref_rung=1)
        self.knobs = dict(tune.DEFAULTS)
        self.ctu = ctu

    def set_tuning(self, **kw):
        if kw.get("fs_band") == 9 and self.ctu != 64:
            raise LadderError(-1, "band 9 needs 64x64 CTUs")
        self.knobs.update(kw)


def cost(knobs):
    # a made-up landscape: fs_band 9 and dep_range 32 help, dep_ctas 1 hurts
    ms = 10.0
    ms -= 2.0 if knobs["fs_band"] == 9 else 0.0
    ms -= 1.0 if knobs["dep_range"] == 32 else 0.0
    ms += 3.0 if knobs["dep_ctas_per_sm"] == 1 else 0.0
    ms -= 0.05 if knobs["dep_band"] == 17 else 0.0   # inside the noise margin
    return ms


def test_coordinate_descent_and_cache(tmp_path):
    lad = FakeLadder()
    timer = lambda fn: cost(lad.knobs)  # noqa: E731
    path = str(tmp_path / "cache.json")
    res = tune.tune(lad, None, tag="t1", timer=timer, device="fake", cache_path=path)
    assert res["knobs"] == {"fs_band": 9, "fs_group": 0, "fs_fuse": 1, "dep_range": 32, "dep_band": 0,
                            "dep_ctas_per_sm": 0, "dep_staged": 1, "dep_inherit": 1}
    assert res["ms"] == pytest.approx(7.0)
    assert lad.knobs == res["knobs"] and not res["cached"]
    # baseline, fs_band, fs_group, fs_fuse, the 17 other (piece size, band,
    # form) settings, grid size
    assert len(res["trials"]) == 1 + 1 + 3 + 1 + 17 + 2
    # the cache answers the same workload key without timing anything
    lad2 = FakeLadder()
    res2 = tune.tune(lad2, None, tag="t1", timer=lambda fn: pytest.fail("timed"), device="fake", cache_path=path)
    assert res2["cached"] and lad2.knobs == res["knobs"]
    # another key is tuned afresh
    res3 = tune.tune(FakeLadder(), None, tag="t2", timer=timer, device="fake", cache_path=path)
    assert not res3["cached"]


def test_invalid_shapes_are_skipped(tmp_path):
    lad = FakeLadder(ctu=32)
    res = tune.tune(lad, None, tag="x", timer=lambda fn: cost(lad.knobs), device="fake",
                    cache_path=str(tmp_path / "c.json"))
    assert res["knobs"]["fs_band"] == 13
    assert all(k["fs_band"] == 13 for k, _ in res["trials"])


def test_workload_key_names_the_geometry():
    key = tune.workload_key(FakeLadder(), "frames32")
    assert "bd8" in key and "R32" in key and "1280x720" in key and key.endswith("frames32")


def test_piece_size_and_band_are_tried_jointly(tmp_path):
    # pieces of 32 help at the default band, but the best pair is pieces of
    # 16 with bands of 17 (pieces of 32 with bands of 17 do not fit): one
    # knob at a time would keep (32, 0)
    def pair_cost(knobs):
        return {(16, 0): 10.0, (32, 0): 9.0, (16, 17): 8.0, (32, 17): 12.0,
                (16, 9): 10.0, (32, 9): 9.0}[(knobs["dep_range"], knobs["dep_band"])]

    lad = FakeLadder()
    res = tune.tune(lad, None, tag="pairs", timer=lambda fn: pair_cost(lad.knobs), device="fake",
                    cache_path=str(tmp_path / "cache.json"), use_cache=False)
    assert (res["knobs"]["dep_range"], res["knobs"]["dep_band"]) == (16, 17)
    assert res["ms"] == pytest.approx(8.0)
