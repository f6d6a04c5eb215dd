"""Continuous-batching serving loop for frame-pair analysis requests.

A request is one frame pair at one rung of one ladder frame: the reference
rung (analysed independently, its decisions then stay resident on the device)
or a dependent rung (analysed from its frame's resident reference
decisions).  Requests of mixed resolutions and bit depths arrive over time.
The loop:

* admits waiting requests in arrival order while the device-memory budget
  (planes of in-flight requests + decision slots of resident frames) and the
  frame slots allow; a dependent is admitted once its frame's reference has
  been launched: in the same batch (same stream, so launch order orders
  them), or in an earlier batch, in which case its batch's stream waits on
  that batch's completion event before the dependent kernels run;
* launches every admitted request of a ladder class in one
  ``ladder_analyze_jobs`` call on the next of several streams, so batches
  overlap on the device and requests that arrive meanwhile join the next
  batch instead of waiting for the running ones to drain;
* polls the in-flight batches, reads back the finished requests' decisions,
  releases their plane buffers and, once a frame's announced dependents are
  done, its frame slot (the resident reference state);
* expires requests that wait longer than their time-to-live (e.g. a
  dependent whose reference never arrives) with an error result.

Scheduling is host logic in this module; every analysis runs in the CUDA
library.  ``FakeExecutor`` replaces the GPU so the scheduling rules can be
tested on the CPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class LadderClass:
    """Geometry shared by the ladders of one class (one library handle)."""
    rungs: list                 # [(W, H), ...]
    ref_rung: int
    bit_depth: int = 8
    search_range: int = 32
    refine_range: int = 4
    ctu: int = 64
    max_frames: int = 32        # frame slots (resident reference state)

    def plane_bytes(self, rung: int) -> int:
        W, H = self.rungs[rung]
        es = 1 if self.bit_depth == 8 else 2
        pitch = (W * es + 127) // 128 * 128
        return 2 * pitch * H


@dataclasses.dataclass
class Request:
    rid: int
    klass: str                  # ladder class name
    frame: int                  # frame id inside the class (ladder instance x frame index)
    rung: int
    dependent: bool
    qp: int
    cur: np.ndarray
    ref: np.ndarray
    arrival: float = 0.0        # seconds from the start of the run
    expect_dependents: int = 0  # reference requests: dependents that will follow
    ttl: float = 5.0            # seconds a request may wait before it expires


@dataclasses.dataclass
class Result:
    rid: int
    ok: bool
    decisions: dict | None
    arrival: float
    done: float
    error: str = ""

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class GpuExecutor:
    """Runs batches with the CUDA library on several streams."""

    def __init__(self, classes: dict, n_streams: int = 3, device: str = "cuda"):
        import torch

        from . import ladder as L
        self.torch, self.L, self.device = torch, L, device
        self.ladders = {name: L.Ladder(c.rungs, c.ref_rung, bit_depth=c.bit_depth, ctu_size=c.ctu,
                                       search_range=c.search_range, refine_range=c.refine_range,
                                       max_frames=c.max_frames)
                        for name, c in classes.items()}
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        # read-back runs on a stream of its own: a fetch synchronises its
        # stream, and a launch stream may already hold a later batch
        self.fetch_stream = torch.cuda.Stream()
        self.next_stream = 0

    def slot_bytes(self, klass: str) -> int:
        lad = self.ladders[klass]
        return lad.device_bytes() // max(1, lad.geometry.max_frames)

    def _upload(self, plane, stream):
        """Device copy of a plane with a 128-byte row pitch.  Pinned torch
        planes (see ``pin_plane``) are copied asynchronously on `stream`."""
        torch = self.torch
        if isinstance(plane, np.ndarray):
            return self.L.device_plane(plane, self.device)
        H, W = plane.shape
        es = plane.element_size()
        pitch = (W * es + 127) // 128 * 128
        buf = torch.empty((H, pitch // es), dtype=plane.dtype, device=self.device)
        view = buf[:, :W]
        view.copy_(plane, non_blocking=True)
        return view

    def launch(self, klass: str, reqs: list, waits=()):
        """Copies the planes in and analyses the requests on the next stream;
        `waits` are handles of earlier batches whose completion the
        dependents of this batch need.  Returns a handle."""
        torch = self.torch
        stream = self.streams[self.next_stream]
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        jobs, keep = [], []
        with torch.cuda.stream(stream):
            for h in waits:
                stream.wait_event(h["event"])
            for r in reqs:
                cur = self._upload(r.cur, stream)
                ref = self._upload(r.ref, stream)
                keep += [cur, ref]
                jobs.append((r.frame, r.rung, 1 if r.dependent else 0, r.qp, cur, ref))
            self.ladders[klass].analyze_jobs(jobs, stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return {"event": ev, "stream": stream, "keep": keep, "klass": klass, "reqs": reqs}

    def done(self, handle) -> bool:
        return handle["event"].query()

    def collect(self, handle) -> list:
        lad = self.ladders[handle["klass"]]
        self.fetch_stream.wait_event(handle["event"])
        out = [lad.fetch(r.rung, r.frame, self.fetch_stream) for r in handle["reqs"]]
        handle["keep"].clear()
        return out

    def release_frame(self, klass: str, frame: int):
        self.ladders[klass].release_frame(frame)

    def close(self):
        for lad in self.ladders.values():
            lad.close()


class Server:
    """Admission, continuous batching and completion of analysis requests.

    `classes` maps a class name to its ``LadderClass``; `executor` runs the
    batches (``GpuExecutor``, or ``FakeExecutor`` for host-only tests).
    `hbm_budget` bounds the device bytes held by in-flight planes plus the
    decision slots of resident frames; `max_batch` bounds the requests of one
    launch and `max_inflight` the batches on the device at once.
    """

    def __init__(self, classes: dict, executor, hbm_budget: int = 8 << 30, max_batch: int = 64,
                 max_inflight: int = 3):
        self.classes = classes
        self.ex = executor
        self.budget = hbm_budget
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.waiting = collections.deque()
        self.inflight = []                    # [handle, plane bytes]
        # (klass, frame) -> {"ref": "launched" | "done", "left": dependents
        #                    still to finish, "handle": batch of the reference}
        self.frame_state = {}
        self.slots_used = collections.Counter()
        self.bytes_inflight = 0
        self.results = {}
        self.resident_samples = []
        self.held_max = 0
        self.slots_max = 0
        self.batches = []                     # (klass, [rid]) per launch
        self._t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self._t0

    # -- device memory -----------------------------------------------------
    def resident_bytes(self) -> int:
        """Decision slots held for resident frames."""
        return sum(n * self.ex.slot_bytes(k) for k, n in self.slots_used.items())

    def held_bytes(self) -> int:
        return self.bytes_inflight + self.resident_bytes()

    def _fits(self, extra: int) -> bool:
        return self.held_bytes() + extra <= self.budget

    # -- frame bookkeeping -------------------------------------------------
    def _dependent_finished(self, key):
        st = self.frame_state.get(key)
        if st is None:
            return
        st["left"] -= 1
        self._maybe_release(key)

    def _maybe_release(self, key):
        st = self.frame_state[key]
        if st["ref"] == "done" and st["left"] <= 0:
            self.ex.release_frame(key[0], key[1])
            self.slots_used[key[0]] -= 1
            del self.frame_state[key]

    # -- admission ---------------------------------------------------------
    def _admit(self, now: float):
        """Moves admissible waiting requests into per-class batches.

        Requests are taken in arrival order; one that cannot be admitted yet
        stays queued without blocking later ones (a later reference may fit
        where an earlier dependent must wait for its reference)."""
        batch = collections.defaultdict(list)
        waits = collections.defaultdict(list)
        kept = collections.deque()
        extra = 0
        n_admitted = 0
        room = len(self.inflight) < self.max_inflight
        while self.waiting:
            r = self.waiting.popleft()
            key = (r.klass, r.frame)
            if now - r.arrival > r.ttl:
                self.results[r.rid] = Result(r.rid, False, None, r.arrival, now, "expired while waiting")
                if r.dependent:
                    self._dependent_finished(key)
                continue
            if not room or n_admitted >= self.max_batch:
                kept.append(r)
                continue
            c = self.classes[r.klass]
            cost = c.plane_bytes(r.rung)
            st = self.frame_state.get(key)
            if r.dependent:
                if st is None or not self._fits(extra + cost):
                    kept.append(r)
                    continue
                h = st.get("handle")
                if st["ref"] == "launched" and h is not None and all(w is not h for w in waits[r.klass]):
                    waits[r.klass].append(h)   # the reference ran in an earlier, unfinished batch
            else:
                if st is not None:
                    self.results[r.rid] = Result(r.rid, False, None, r.arrival, now,
                                                 "frame already has a reference")
                    continue
                slot = self.ex.slot_bytes(r.klass)
                if self.slots_used[r.klass] >= c.max_frames or not self._fits(extra + cost + slot):
                    kept.append(r)
                    continue
                self.slots_used[r.klass] += 1
                self.frame_state[key] = {"ref": "launched", "left": r.expect_dependents, "handle": None}
            extra += cost
            n_admitted += 1
            batch[r.klass].append(r)
        self.waiting = kept
        return batch, waits

    def _launch(self, batch, waits):
        for klass, reqs in batch.items():
            bytes_ = sum(self.classes[klass].plane_bytes(r.rung) for r in reqs)
            h = self.ex.launch(klass, reqs, waits.get(klass, ()))
            for r in reqs:
                if not r.dependent:
                    self.frame_state[(r.klass, r.frame)]["handle"] = h
            self.inflight.append([h, bytes_])
            self.bytes_inflight += bytes_
            self.batches.append((klass, [r.rid for r in reqs]))

    # -- completion --------------------------------------------------------
    def _retire(self):
        still = []
        for h, bytes_ in self.inflight:
            if not self.ex.done(h):
                still.append([h, bytes_])
                continue
            decs = self.ex.collect(h)
            t = self.now()
            refs_first = sorted(zip(h["reqs"], decs), key=lambda rd: rd[0].dependent)
            for r, d in refs_first:
                self.results[r.rid] = Result(r.rid, True, d, r.arrival, t)
                key = (r.klass, r.frame)
                if r.dependent:
                    self._dependent_finished(key)
                elif key in self.frame_state:
                    st = self.frame_state[key]
                    st["ref"], st["handle"] = "done", None
                    self._maybe_release(key)
            self.bytes_inflight -= bytes_
        self.inflight = still

    def step(self):
        """One scheduling pass: retire finished batches, then admit and
        launch what fits."""
        self._retire()
        now = self.now()
        batch, waits = self._admit(now)
        if batch:
            self._launch(batch, waits)
        self.resident_samples.append(self.resident_bytes())
        self.held_max = max(self.held_max, self.held_bytes())
        self.slots_max = max(self.slots_max, max(self.slots_used.values(), default=0))

    def submit(self, req: Request):
        self.waiting.append(req)

    def idle(self) -> bool:
        return not self.waiting and not self.inflight

    def run(self, requests: list, poll: float = 2e-4) -> dict:
        """Feeds requests at their arrival times (seconds after the start)
        and serves until every request has a result."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self._t0 = time.perf_counter()
        i = 0
        while i < len(pending) or not self.idle():
            now = self.now()
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i])
                i += 1
            self.step()
            if poll:
                time.sleep(poll)
        return self.report(self.now())

    def report(self, elapsed: float) -> dict:
        ok = [r for r in self.results.values() if r.ok]
        lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
        return {
            "requests": len(self.results),
            "completed": len(ok),
            "failed": len(self.results) - len(ok),
            "elapsed_s": elapsed,
            "throughput_req_s": len(ok) / elapsed if elapsed > 0 else 0.0,
            "latency_p50_ms": float(np.percentile(lat, 50) * 1e3),
            "latency_p99_ms": float(np.percentile(lat, 99) * 1e3),
            "resident_bytes_max": int(max(self.resident_samples, default=0)),
            "resident_bytes_mean": float(np.mean(self.resident_samples)) if self.resident_samples else 0.0,
            "held_bytes_max": int(self.held_max),
            "batches": len(self.batches),
            "mean_batch": float(np.mean([len(b) for _, b in self.batches])) if self.batches else 0.0,
        }


def request_stream(seed: int, n_requests: int, rate: float, classes: dict, content: dict, *,
                   qps=(22, 27, 32, 37), n_open: int = 4, ttl: float = 5.0, first_frame: int = 0):
    """A Poisson stream of per-rung frame-pair requests over open ladder frames.

    Each ladder frame (of a class drawn uniformly from `classes`) asks for
    every rung of its class: the reference rung first, then the dependent
    rungs in random order, so over a long stream the rungs are drawn
    uniformly.  Up to `n_open` ladder frames are open at once and each
    arrival continues one of them, chosen uniformly, which interleaves the
    ladders.  Inter-arrival times are exponential with mean 1/`rate` s.
    `content[klass]` is a list of ladder frames, each a list over rungs of
    (cur, ref) planes; ladder frame f of a class uses content f mod len.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    names = sorted(classes)
    frame_no = collections.Counter()
    opened = []                       # [klass, frame, qp, [rungs left]]

    def open_one():
        k = names[int(rng.integers(len(names)))]
        c = classes[k]
        f = first_frame + frame_no[k]
        frame_no[k] += 1
        deps = [r for r in range(len(c.rungs)) if r != c.ref_rung]
        rng.shuffle(deps)
        opened.append([k, f, int(qps[int(rng.integers(len(qps)))]), [c.ref_rung] + deps])

    out = []
    t = 0.0
    for rid in range(n_requests):
        while len(opened) < n_open:
            open_one()
        t += float(rng.exponential(1.0 / rate))
        j = int(rng.integers(len(opened)))
        k, f, qp, left = opened[j]
        rung = left.pop(0)
        c = classes[k]
        frames = content[k]
        cur, ref = frames[f % len(frames)][rung]
        dep = rung != c.ref_rung
        out.append(Request(rid=rid, klass=k, frame=f, rung=rung, dependent=dep, qp=qp, cur=cur, ref=ref,
                           arrival=t, expect_dependents=0 if dep else len(c.rungs) - 1, ttl=ttl))
        if not left:
            opened.pop(j)
    # ladder frames cut off by the end of the stream expect fewer dependents
    sent = collections.Counter((r.klass, r.frame) for r in out if r.dependent)
    for r in out:
        if not r.dependent:
            r.expect_dependents = sent[(r.klass, r.frame)]
    return out


def pin_plane(plane: np.ndarray):
    """A page-locked torch copy of a plane (10-bit planes as int16 bits) so
    that the executor's upload runs asynchronously."""
    import torch
    a = np.ascontiguousarray(plane)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).pin_memory()


class FakeExecutor:
    """CPU stand-in for GpuExecutor: a batch completes `latency` seconds
    after its launch; decisions are placeholders.  For scheduling tests."""

    def __init__(self, classes: dict, latency: float = 0.01, slot_bytes: int = 1 << 20):
        self.classes = classes
        self.latency = latency
        self._slot = slot_bytes
        self.released = []
        self.launched = []

    def slot_bytes(self, klass: str) -> int:
        return self._slot

    def launch(self, klass, reqs, waits=()):
        t = time.perf_counter()
        self.launched.append((klass, [r.rid for r in reqs], t, list(waits)))
        return {"t": t, "klass": klass, "reqs": reqs, "waits": list(waits)}

    def done(self, h) -> bool:
        # a batch that waits on earlier batches finishes after them
        return time.perf_counter() - h["t"] >= self.latency and all(self.done(w) for w in h["waits"])

    def collect(self, h):
        return [{"rid": r.rid} for r in h["reqs"]]

    def release_frame(self, klass, frame):
        self.released.append((klass, frame))
