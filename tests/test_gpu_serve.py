"""The serving loop on the GPU: every served result is bit-identical to the
same request analysed alone, and to the oracle.

A seeded Poisson stream of 8- and 10-bit requests of several rungs is served
with continuous batching (several batches in flight on separate streams,
dependents joining while their reference's batch still runs).  Each result
is then recomputed with the request alone on a fresh library handle: the
reference rung by itself, a dependent rung after its own frame's reference.
"""
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
from paper_2301_12191_gb300 import serve  # noqa: E402

CLASSES = {
    "l8": serve.LadderClass(rungs=[(640, 360), (480, 270), (320, 180)], ref_rung=2, bit_depth=8,
                            search_range=16, refine_range=4, max_frames=6),
    "l10": serve.LadderClass(rungs=[(512, 288), (256, 144)], ref_rung=1, bit_depth=10,
                             search_range=12, refine_range=3, max_frames=6),
}


def _content(seed, klass, n):
    c = CLASSES[klass]
    src = c.rungs[0]
    out = []
    for k in range(n):
        pairs, _ = synth.ladder_pairs(seed + k, source=src, rungs=c.rungs[1:], bit_depth=c.bit_depth)
        out.append([(cur, ref) for (_, _, cur, ref) in pairs])
    return out


def _alone(req, content):
    """The request analysed by itself on a fresh handle."""
    c = CLASSES[req.klass]
    frames = content[req.klass]
    planes = frames[req.frame % len(frames)]
    with L.Ladder(c.rungs, c.ref_rung, bit_depth=c.bit_depth, search_range=c.search_range,
                  refine_range=c.refine_range, max_frames=1) as lad:
        rc, rf = planes[c.ref_rung]
        lad.analyze_reference(req.frame, L.device_plane(rc), L.device_plane(rf), req.qp)
        if req.dependent:
            cur, ref = planes[req.rung]
            lad.analyze_dependent(req.rung, req.frame, L.device_plane(cur), L.device_plane(ref), req.qp)
        return lad.fetch(req.rung, req.frame)


def test_served_results_equal_alone_and_oracle():
    content = {k: _content(100 + 10 * i, k, 2) for i, k in enumerate(sorted(CLASSES))}
    pinned = {k: [[(serve.pin_plane(cu), serve.pin_plane(re)) for cu, re in fr] for fr in v]
              for k, v in content.items()}
    reqs = serve.request_stream(7, 48, 3000.0, CLASSES, pinned, n_open=5, ttl=60.0)
    ex = serve.GpuExecutor(CLASSES, n_streams=3)
    try:
        srv = serve.Server(CLASSES, ex, hbm_budget=1 << 30, max_batch=6, max_inflight=3)
        rep = srv.run(reqs, poll=0)
        torch.cuda.synchronize()
    finally:
        ex.close()
    assert rep["completed"] == len(reqs) and rep["failed"] == 0
    assert not srv.frame_state and sum(srv.slots_used.values()) == 0
    # the mix really was concurrent: batched, and some dependents joined
    # while their reference's batch was still in flight
    assert rep["batches"] < len(reqs)

    for r in reqs:
        got = srv.results[r.rid].decisions
        assert_decisions_equal(got, _alone(r, content), 64, where=f"request {r.rid} ({r.klass} rung {r.rung})")

    # close the chain to the oracle on one ladder frame of each class
    for klass, c in CLASSES.items():
        frame = next(r.frame for r in reqs if r.klass == klass and not r.dependent)
        planes = content[klass][frame % 2]
        mine = [r for r in reqs if r.klass == klass and r.frame == frame]
        ref_req = next(r for r in mine if not r.dependent)
        rc, rf = planes[c.ref_rung]
        ora_ref = oracle.analyze(rc, rf, qp=ref_req.qp, search_range=c.search_range)
        assert_decisions_equal(srv.results[ref_req.rid].decisions, ora_ref, 64, where=f"{klass} reference")
        for r in mine:
            if r.dependent:
                cu, re = planes[r.rung]
                ora = oracle.analyze(cu, re, qp=r.qp, search_range=c.refine_range,
                                     dep=dep_from(ora_ref, c.rungs[c.ref_rung]))
                assert_decisions_equal(srv.results[r.rid].decisions, ora, 64, where=f"{klass} rung {r.rung}")


def test_jobs_call_equals_per_call():
    """ladder_analyze_jobs with references and dependents of several frames
    mixed in one call equals the per-call entry points."""
    c = CLASSES["l8"]
    content = _content(300, "l8", 3)
    dev = [[(L.device_plane(cu), L.device_plane(re)) for cu, re in fr] for fr in content]
    qps = [22, 32, 37]
    with L.Ladder(c.rungs, c.ref_rung, search_range=c.search_range, refine_range=c.refine_range,
                  max_frames=4) as lad:
        # frame 0's reference first in a call of its own; then one call with
        # frame 0's dependents, frames 1 and 2 (references + dependents, in
        # shuffled order)
        lad.analyze_jobs([(0, c.ref_rung, 0, qps[0], *dev[0][c.ref_rung])])
        jobs = [(0, 0, 1, qps[0], *dev[0][0]), (2, 1, 1, qps[2], *dev[2][1]), (1, c.ref_rung, 0, qps[1],
                *dev[1][c.ref_rung]), (0, 1, 1, qps[0], *dev[0][1]), (1, 0, 1, qps[1], *dev[1][0]),
                (2, c.ref_rung, 0, qps[2], *dev[2][c.ref_rung]), (2, 0, 1, qps[2], *dev[2][0]),
                (1, 1, 1, qps[1], *dev[1][1])]
        lad.analyze_jobs(jobs)
        got = {(f, r): lad.fetch(r, f) for f in range(3) for r in range(3)}
    for f in range(3):
        with L.Ladder(c.rungs, c.ref_rung, search_range=c.search_range, refine_range=c.refine_range,
                      max_frames=1) as lad:
            lad.analyze_reference(f, *dev[f][c.ref_rung], qps[f])
            for r in (0, 1):
                lad.analyze_dependent(r, f, *dev[f][r], qps[f])
            for r in range(3):
                assert_decisions_equal(got[(f, r)], lad.fetch(r, f), 64, where=f"frame {f} rung {r}")


def test_jobs_status_codes():
    c = CLASSES["l8"]
    content = _content(400, "l8", 1)
    dev = [(L.device_plane(cu), L.device_plane(re)) for cu, re in content[0]]
    with L.Ladder(c.rungs, c.ref_rung, search_range=c.search_range, max_frames=1) as lad:
        with pytest.raises(L.LadderError) as e:
            lad.analyze_jobs([(5, 0, 1, 27, *dev[0])])              # no reference for frame 5
        assert e.value.status == -3
        with pytest.raises(L.LadderError) as e:
            lad.analyze_jobs([(5, c.ref_rung, 1, 27, *dev[2])])     # reference rung as dependent
        assert e.value.status == -1
        with pytest.raises(L.LadderError) as e:
            lad.analyze_jobs([(5, c.ref_rung, 0, 27, *dev[2]), (6, c.ref_rung, 0, 27, *dev[2])])
        assert e.value.status == -4                                  # two new frames, one slot
        lad.analyze_jobs([(5, c.ref_rung, 0, 27, *dev[2]), (5, 0, 1, 27, *dev[0])])
        lad.sync()
