"""Kernel-shape knobs never change a decision; the autotuner picks valid shapes."""
import numpy as np
import pytest

from paper_2301_12191_gb300 import synth
from helpers import assert_decisions_equal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402
from paper_2301_12191_gb300 import tune  # noqa: E402

SETTINGS = [
    {"fs_band": 9},
    {"dep_range": 32},
    {"dep_band": 17},
    {"dep_band": 9},
    {"dep_ctas_per_sm": 1},
    {"fs_group": 2},
    {"fs_group": 4},
    {"fs_group": 3, "fs_band": 9},
    {"fs_fuse": 0},
    {"fs_fuse": 0, "fs_group": 2},
    {"fs_band": 9, "dep_range": 32, "dep_band": 17, "dep_ctas_per_sm": 2},
    {"dep_staged": 0},
    {"dep_staged": 2},
    {"dep_staged": 2, "dep_band": 17},
    {"dep_staged": 0, "dep_band": 17},
    {"dep_range": 32, "dep_band": 17},
    {"dep_inherit": 0},
    {"dep_inherit": 0, "dep_range": 32, "dep_staged": 0},
]

CASES = [
    # (source, rungs below the source, bit depth, R, r)
    ((640, 360), [(480, 270), (320, 180)], 8, 16, 4),
    ((1280, 720), [(640, 360), (320, 180)], 8, 32, 6),
    ((512, 288), [(384, 216), (256, 144)], 10, 24, 8),
]


def _run(lad, frames, qp=27):
    ref = len(lad.rungs) - 1
    items = [(f, qp, planes) for f, planes in enumerate(frames)]
    lad.analyze_batch(items)
    out = {(f, r): lad.fetch(r, f) for f in range(len(frames)) for r in range(len(lad.rungs))}
    for f in range(len(frames)):
        lad.release_frame(f)
    return out


@pytest.mark.parametrize("src,rungs,bd,R,r", CASES)
def test_knobs_do_not_change_decisions(src, rungs, bd, R, r):
    frames = []
    for seed in (5, 6):
        pairs, _ = synth.ladder_pairs(seed, source=src, rungs=rungs, bit_depth=bd)
        frames.append([(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs])
    sizes = [src] + list(rungs)
    with L.Ladder(sizes, len(sizes) - 1, bit_depth=bd, search_range=R, refine_range=r, max_frames=2) as lad:
        base = _run(lad, frames)
        for knobs in SETTINGS:
            lad.set_tuning(**tune.DEFAULTS)
            lad.set_tuning(**knobs)
            got = _run(lad, frames)
            for key in base:
                assert_decisions_equal(got[key], base[key], 64, where=f"{knobs} frame/rung {key}")


def test_bad_knobs_are_refused():
    with L.Ladder([(64, 64)], 0, ctu_size=32, max_frames=1) as lad:
        for knobs in ({"fs_band": 9}, {"fs_band": 11}, {"dep_range": 8}, {"dep_band": 5}, {"dep_ctas_per_sm": 9}, {"fs_group": 5},
                      {"dep_inherit": 2}):
            with pytest.raises(L.LadderError):
                lad.set_tuning(**knobs)
        assert lad.tuning() == tune.DEFAULTS


def test_autotuner_on_a_batch(tmp_path):
    frames = []
    for seed in (11, 12, 13):
        pairs, _ = synth.ladder_pairs(seed, source=(640, 360), rungs=[(320, 180)])
        frames.append([(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs])
    with L.Ladder([(640, 360), (320, 180)], 1, search_range=16, refine_range=4, max_frames=3) as lad:
        items = [(f, 27, planes) for f, planes in enumerate(frames)]

        def step():
            lad.analyze_batch(items)
            for f in range(3):
                lad.release_frame(f)

        res = tune.tune(lad, step, tag="frames3", reps=3, warmup=1, cache_path=str(tmp_path / "c.json"))
        assert set(res["knobs"]) == set(tune.DEFAULTS)
        for k, v in res["knobs"].items():
            assert v in tune.knob_values(k)
        assert lad.tuning() == res["knobs"]
        assert res["ms"] > 0 and len(res["trials"]) >= 4
        again = tune.tune(lad, step, tag="frames3", cache_path=str(tmp_path / "c.json"))
        assert again["cached"] and again["knobs"] == res["knobs"]
