"""Host-side rules of the serving loop, with a fake executor (no GPU)."""
import collections

import numpy as np

from paper_2301_12191_gb300 import serve

TINY = np.zeros((8, 8), np.uint8)


def classes(max_frames=4):
    return {
        "a8": serve.LadderClass(rungs=[(640, 360), (320, 180), (160, 90)], ref_rung=2, bit_depth=8,
                                max_frames=max_frames),
        "b10": serve.LadderClass(rungs=[(640, 360), (160, 90)], ref_rung=1, bit_depth=10, max_frames=max_frames),
    }


def content(cl):
    return {k: [[(TINY, TINY) for _ in c.rungs]] for k, c in cl.items()}


def run(reqs, cl, latency=0.005, **kw):
    ex = serve.FakeExecutor(cl, latency=latency, slot_bytes=1 << 16)
    srv = serve.Server(cl, ex, **kw)
    rep = srv.run(reqs, poll=1e-4)
    return srv, ex, rep


def test_stream_shape():
    cl = classes()
    reqs = serve.request_stream(1, 400, 2000.0, cl, content(cl), n_open=3)
    assert len(reqs) == 400
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert abs(np.mean(np.diff(arr)) - 1 / 2000.0) < 0.3 / 2000.0
    seen_ref = set()
    per_frame = collections.Counter()
    for r in reqs:
        key = (r.klass, r.frame)
        if r.dependent:
            assert key in seen_ref, "a dependent arrived before its reference"
            per_frame[key] += 1
        else:
            assert key not in seen_ref
            seen_ref.add(key)
    for r in reqs:
        if not r.dependent:
            assert r.expect_dependents == per_frame[(r.klass, r.frame)]
            assert r.expect_dependents <= len(cl[r.klass].rungs) - 1
    # seeded: the same stream twice
    again = serve.request_stream(1, 400, 2000.0, cl, content(cl), n_open=3)
    assert [(r.klass, r.frame, r.rung, r.qp, r.arrival) for r in reqs] == \
           [(r.klass, r.frame, r.rung, r.qp, r.arrival) for r in again]


def test_all_complete_and_frames_released():
    cl = classes()
    reqs = serve.request_stream(2, 300, 3000.0, cl, content(cl), n_open=4)
    srv, ex, rep = run(reqs, cl)
    assert rep["completed"] == 300 and rep["failed"] == 0
    assert not srv.frame_state and sum(srv.slots_used.values()) == 0
    frames = {(r.klass, r.frame) for r in reqs}
    assert sorted(ex.released) == sorted(frames)
    assert rep["latency_p99_ms"] >= rep["latency_p50_ms"] > 0


def test_reference_launched_before_its_dependents():
    cl = classes()
    reqs = serve.request_stream(3, 200, 5000.0, cl, content(cl), n_open=4)
    srv, ex, _ = run(reqs, cl, latency=0.01)
    by_rid = {r.rid: r for r in reqs}
    batch_of = {}
    for b, (_, rids, _, _) in enumerate(ex.launched):
        for rid in rids:
            batch_of[rid] = b
    ref_batch = {(r.klass, r.frame): batch_of[r.rid] for r in reqs if not r.dependent}
    for r in reqs:
        if r.dependent:
            assert batch_of[r.rid] >= ref_batch[(r.klass, r.frame)]
    # a dependent launched in a later batch while its reference's batch was
    # still in flight waits on that batch
    for b, (_, rids, t, waits) in enumerate(ex.launched):
        for rid in rids:
            r = by_rid[rid]
            if r.dependent and batch_of[rid] > ref_batch[(r.klass, r.frame)]:
                ref_b = ref_batch[(r.klass, r.frame)]
                ref_t = ex.launched[ref_b][2]
                if t - ref_t < 0.009:  # reference surely not finished yet
                    assert any(w["reqs"][0].rid in ex.launched[ref_b][1] for w in waits)


def test_dependent_waits_for_late_reference_and_orphans_expire():
    cl = classes()
    c = cl["a8"]
    reqs = [
        serve.Request(0, "a8", 7, 0, True, 27, TINY, TINY, arrival=0.000),            # before its reference
        serve.Request(1, "a8", 7, 2, False, 27, TINY, TINY, arrival=0.010, expect_dependents=1),
        serve.Request(2, "a8", 9, 1, True, 27, TINY, TINY, arrival=0.000, ttl=0.03),  # reference never comes
    ]
    srv, ex, rep = run(reqs, cl)
    assert srv.results[0].ok and srv.results[1].ok
    assert not srv.results[2].ok and "expired" in srv.results[2].error
    launched_order = [rid for _, rids, _, _ in ex.launched for rid in rids]
    assert launched_order.index(1) <= launched_order.index(0)
    assert ("a8", 7) in ex.released and not srv.frame_state
    assert c.plane_bytes(0) == 2 * 640 * 360


def test_memory_budget_and_slots_bound():
    cl = classes(max_frames=2)
    reqs = serve.request_stream(4, 240, 20000.0, cl, content(cl), n_open=6)
    # budget for about three 640x360 requests plus a few slots
    budget = 3 * cl["a8"].plane_bytes(0) + 4 * (1 << 16)
    srv, ex, rep = run(reqs, cl, latency=0.002, hbm_budget=budget)
    assert rep["completed"] == 240
    assert rep["held_bytes_max"] <= budget
    assert srv.slots_max <= 2
    assert len(ex.released) == len({(r.klass, r.frame) for r in reqs})


def test_continuous_batching_overlaps_batches():
    cl = classes(max_frames=16)
    reqs = serve.request_stream(5, 120, 4000.0, cl, content(cl), n_open=6)
    srv, ex, rep = run(reqs, cl, latency=0.02, max_inflight=3)
    starts = [t for _, _, t, _ in ex.launched]
    # some batch started while an earlier one (20 ms long) was still running
    assert any(b - a < 0.02 for a, b in zip(starts, starts[1:]))
    assert rep["batches"] < len(reqs)          # requests were batched together
    assert rep["completed"] == 120


def test_max_batch_respected():
    cl = classes(max_frames=32)
    reqs = serve.request_stream(6, 100, 1e6, cl, content(cl), n_open=8)
    srv, ex, rep = run(reqs, cl, latency=0.003, max_batch=5)
    assert max(len(r) for _, r, _, _ in ex.launched) <= 5
    assert rep["completed"] == 100
