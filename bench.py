#!/usr/bin/env python3
"""Throughput of multi-resolution inter analysis on GB300.

A step analyses ladder frames: the reference rung of each frame
independently (full search +-R), then every other rung as a dependent
(scaled reference MVs, +-r refinement, depth n..n+1).  ``value`` is ladder
frames per second with the planes already resident in HBM; ``e2e`` is the
same through the C ABI's frame pipeline with every frame's planes copied
from pinned host memory and every rung's decisions read back inside the
timed region.  The same ladders analysed independently (+-R on every rung)
give the multi-resolution speedup.

The default workload is the 2160p -> 360p 10-bit ladder (eight frame pairs
per step, six rungs, 360p reference at +-64, dependents at +-8); the
1080p -> 360p 8-bit ladder is measured beside it as an extra key.

``--impl reference`` times the CPU oracle (the only reference this method
has) on the host cores for the same workload and ``config``.
``--gpus N`` without a launcher's environment starts N ranks itself (one
process per GPU, replicas with no collective on the data path).
"""
from __future__ import annotations

import argparse
import concurrent.futures
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2301_12191_gb300 import replicas, synth  # noqa: E402

UHD_RUNGS = [(3840, 2160), (2560, 1440), (1920, 1080), (1280, 720), (960, 540), (640, 360)]
WORKLOADS = {
    # 1080p source pair -> 1080p / 720p / 540p / 360p rungs; 360p reference
    "ladder1080": dict(source=(1920, 1080), rungs=[(1920, 1080), (1280, 720), (960, 540), (640, 360)], ref=3,
                       bit_depth=8, R=32, r=4, qp=27, ctu=64, multi_qps=[22, 32, 37], subpel=True, mvp=True,
                       pipelined_frames=24),
    # 8 ladders x 5 consecutive frames (4 pairs each) of 1080p, one batched graph per step
    "batch8x5": dict(mode="batch", ladders=8, frames=5, source=(1920, 1080),
                     rungs=[(1920, 1080), (1280, 720), (960, 540), (640, 360)], ref=3, bit_depth=8, R=32, r=4,
                     qps=[22, 27, 32, 37], sigmas=[1, 4, 8], global_range=16, patch_range=24, ctu=64, mvp=True,
                     oracle_every=8),
    # 8 frame pairs of 2160p 10-bit -> six rungs; 360p reference at +-64, dependents +-8
    "uhd8": dict(mode="batch", ladders=8, frames=2, source=(3840, 2160), rungs=UHD_RUNGS, ref=5,
                 bit_depth=10, R=64, r=8, qps=[22, 27, 32, 37], sigmas=[8], global_range=8 * 3840 // 416,
                 patch_range=12 * 3840 // 416, ctu=64, oracle_every=4),
    # uhd8 with the cascaded reference chain of the proposed multi-encoding
    # scheme: 360p -> 720p -> 1440p and 360p -> 540p -> 1080p -> 2160p
    "uhd8chain": dict(mode="batch", ladders=8, frames=2, source=(3840, 2160), rungs=UHD_RUNGS, ref=5,
                      parents=[2, 3, 4, 5, 5, -1],
                      bit_depth=10, R=64, r=8, qps=[22, 27, 32, 37], sigmas=[8], global_range=8 * 3840 // 416,
                      patch_range=12 * 3840 // 416, ctu=64, oracle_every=4),
    # serving: Poisson requests (200/s) for single rungs of 2160p->360p ladders,
    # 8- and 10-bit mixed, continuous batching on several streams
    "serve": dict(mode="serve", rate=200.0, seconds=10.0, source=(3840, 2160), rungs=UHD_RUNGS, ref=5,
                  bit_depths=[8, 10], R=64, r=8, qps=[22, 27, 32, 37], ctu=64, max_frames=24,
                  hbm_budget=16 << 30, n_open=6, streams=3, max_batch=32),
    # single 416x240 pair, independent only
    "frame416": dict(source=(416, 240), rungs=[(416, 240)], ref=0, bit_depth=8, R=16, r=4, qp=32, ctu=64),
}
DEFAULT_CONFIG = "uhd8"
# workloads measured beside a workload's line, each nested under its name
EXTRA = {"uhd8": ["ladder1080"]}
METRIC = "ladder frames/sec (multi-resolution inter analysis)"
# The paper's own measurements, quoted with the hardware it states: context
# beside the numbers, not a target (it times whole x265 / XVC encodes on a
# laptop CPU, never this analysis path alone).
PAPER_CONTEXT = {
    "hardware": "Intel Core i7-7500U (2 cores / 4 threads, about 2.9 GHz), 16 GB DDR4, x265 medium preset",
    "inter_res_encode_time_reduction": "540p -> 1080p with refinement: 28.99% (CQP); 1080p / 2160p with "
                                       "refinement: 50.45% / 52.82% (cVBR)",
    "multi_encoding_scheme": "up to 2.5x faster than single-instance encoding",
    "simd_kernels": "SAD 2.40x-6.46x and SATD 3.45x-10.22x faster than C++ (Arowana XVC, SSE4/AVX2)",
}
UNIT = "ladder_frames/s"
E2E_DEPTH = 5  # frame slots of the end-to-end pipeline
PIPE_STREAMS = 3  # streams (and frame slots) of the pipelined device measurement
L2_FLUSH_BYTES = 256 << 20
DATA = ("synthetic (seeded sinusoid texture + planted global/patch motion + noise; rungs by Q16 bilinear "
        "downscaling)")

# DRAM bytes (read + write) of one launch from an ncu capture (the summaries
# under profiles/), keyed by kernel, workload and the hash of the kernel
# sources it was taken on, with the kernel shapes of the capture: reported
# only when the run's shapes are those and the sources unchanged.  The uhd8
# figures come from the 3-ladder case (--ladders 3) scaled by 8/3: the work
# of a launch grows with its ladders.
KERNEL_SOURCES = {"full_search": ["me_full.cu", "common.cuh"], "dependent": ["me_dependent.cu", "common.cuh"]}
TRAFFIC_NCU = {
    ("dependent", "uhd8", "076570b74ddb"): {"bytes": (259427328 + 36680960) * 8 // 3,
                                            "knobs": {"dep_band": 17, "dep_range": 16, "dep_staged": 1,
                                                      "dep_inherit": 1}},
    ("full_search", "uhd8", "fb7e3970fc46"): {"bytes": 2999296 * 8 // 3, "knobs": {"fs_band": 13}},
}


def traffic_of(kname, name, knobs):
    """The captured DRAM bytes of one launch of kernel kname in workload
    name, or None (no capture of these sources with these shapes)."""
    ent = TRAFFIC_NCU.get((kname, name, kernel_source_hash(kname)))
    if not ent or any(knobs.get(k) != v for k, v in ent["knobs"].items()):
        return None
    return ent["bytes"]


def kernel_source_hash(kernel):
    m = hashlib.sha1()
    for name in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_2301_12191_gb300", "csrc", name), "rb") as f:
            m.update(f.read())
    return m.hexdigest()[:12]


def parents_of(wl):
    ref_i = wl["ref"]
    return wl.get("parents") or [-1 if i == ref_i else ref_i for i in range(len(wl["rungs"]))]


def workload_config(name, wl):
    """The `config` of a workload's line: identical for the GPU arm and the
    oracle arm."""
    c = {"workload": name, "rungs": [f"{w}x{h}" for (w, h) in wl["rungs"]],
         "reference_rung": "{}x{}".format(*wl["rungs"][wl["ref"]]), "search_range": wl["R"],
         "refine_range": wl["r"], "ctu": wl["ctu"], "depth_window": [0, 1]}
    if wl.get("mode") == "batch":
        c.update(bit_depth=wl["bit_depth"], qps=wl["qps"], ladders=wl["ladders"],
                 ladder_frames_per_step=wl["ladders"] * (wl["frames"] - 1))
    else:
        c.update(bit_depth=wl["bit_depth"], qp=wl["qp"], ladder_frames_per_step=1)
    if wl.get("parents"):
        c["parents"] = wl["parents"]
    return c


def make_frames(wl, n_frames, seed0):
    """n_frames independent ladder frames [(w, h, cur, ref) per rung]."""
    def one(f):
        pairs, _ = synth.ladder_pairs(seed0 + f, source=wl["source"], rungs=wl["rungs"][1:],
                                      bit_depth=wl["bit_depth"], include_source=True)
        return pairs
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, range(n_frames)))


def batch_requests(wl, seed0, ladders=None):
    """Per ladder a seeded sequence; consecutive frames form the pairs.
    Returns (frames[l][t][rung] planes, [(ladder, t, qp)] per request)."""
    W = wl["source"][0]
    n_lad = wl["ladders"] if ladders is None else ladders

    def one(l):
        return synth.ladder_sequence(seed0 + l, wl["frames"], source=wl["source"], rungs=wl["rungs"],
                                     bit_depth=wl["bit_depth"], global_range=wl["global_range"],
                                     patch_range=wl["patch_range"], patch_size=int(round(64 * W / 416 / 8)) * 8,
                                     noise_sigma=wl["sigmas"][l % len(wl["sigmas"])])
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        frames = list(ex.map(one, range(n_lad)))
    reqs = [(l, t, wl["qps"][l % len(wl["qps"])]) for l in range(n_lad) for t in range(wl["frames"] - 1)]
    return frames, reqs


def request_pairs(wl, frames, req):
    """[(w, h, cur, ref)] of every rung of one batch request."""
    l, t, _ = req
    return [(w, h, frames[l][t + 1][r], frames[l][t][r]) for r, (w, h) in enumerate(wl["rungs"])]


def packed_layout(planes):
    """Packed host layout of one ladder frame: per rung (cur offset, ref
    offset, pitch, rows, width, sample bytes), rows padded to 128 bytes;
    planes = [(cur, ref)] per rung."""
    offs, off = [], 0
    for c, _ in planes:
        h, w = c.shape
        es = c.dtype.itemsize
        pitch = (w * es + 127) // 128 * 128
        offs.append((off, off + h * pitch, pitch, h, w, es))
        off += 2 * h * pitch
    return offs, off


def pack_host(planes, lay, in_bytes):
    import torch
    buf = torch.zeros(in_bytes, dtype=torch.uint8).pin_memory()
    nb = buf.numpy()
    for (oc, orf, pitch, h, w, es), (c, f) in zip(lay, planes):
        for o, pl in ((oc, c), (orf, f)):
            rows = nb[o:o + h * pitch].reshape(h, pitch)
            rows[:, :w * es] = np.ascontiguousarray(pl).view(np.uint8).reshape(h, w * es)
    return buf


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ oracle leg --
def ctu_count(w, h, ctu):
    return ((w + 7) // 8 * 8 + ctu - 1) // ctu * (((h + 7) // 8 * 8 + ctu - 1) // ctu)


def dep_args(pairs, out, p):
    return {"ref_size": (pairs[p][0], pairs[p][1]), "leaf_depth": out[p]["leaf_depth"],
            "leaf_mvx": out[p]["leaf_mvx"], "leaf_mvy": out[p]["leaf_mvy"]}


def oracle_ladder_frame(wl, pairs, threads, qp):
    """One ladder frame by the oracle: the reference rung, then every other
    rung as a dependent of its parent (the reference rung, or the parents of
    a cascaded chain), parents first.  Returns every rung's decisions."""
    import oracle
    ref_i = wl["ref"]
    parents = parents_of(wl)
    out = {}
    w, h, c, f = pairs[ref_i]
    out[ref_i] = oracle.analyze(c, f, qp=qp, search_range=wl["R"], ctu=wl["ctu"], threads=threads)
    while len(out) < len(pairs):
        for i, (w2, h2, c2, f2) in enumerate(pairs):
            p = parents[i]
            if i in out or p not in out:
                continue
            out[i] = oracle.analyze(c2, f2, qp=qp, search_range=wl["r"], ctu=wl["ctu"], threads=threads,
                                    dep=dep_args(pairs, out, p))
    return out


def oracle_parent_decisions(wl, pairs, qp, threads):
    """Full oracle decisions of every rung that is some rung's parent (the
    reference rung and the inner rungs of a chain), for sampled analyses."""
    import oracle
    ref_i, parents = wl["ref"], parents_of(wl)
    need = {p for p in parents if p >= 0} | {ref_i}
    out = {}
    w, h, c, f = pairs[ref_i]
    out[ref_i] = oracle.analyze(c, f, qp=qp, search_range=wl["R"], ctu=wl["ctu"], threads=threads)
    while not need <= set(out):
        for i in sorted(need - set(out)):
            p = parents[i]
            if p in out:
                out[i] = oracle.analyze(pairs[i][2], pairs[i][3], qp=qp, search_range=wl["r"], ctu=wl["ctu"],
                                        threads=threads, dep=dep_args(pairs, out, p))
    return out


def oracle_frame_sampled(wl, pairs, qp, pre, threads, every, phase=0):
    """Seconds of one ladder frame by the oracle, estimated from a sample:
    every `every`-th CTU of each rung (starting at `phase`), the dependents'
    rules reading their parents' decisions made beforehand (`pre`), each
    rung's time scaled by its CTUs over the CTUs sampled.  Returns
    (seconds per frame, CTUs sampled)."""
    import oracle
    ref_i, parents = wl["ref"], parents_of(wl)
    total, sampled = 0.0, 0
    for i, (w, h, c, f) in enumerate(pairs):
        n = ctu_count(w, h, wl["ctu"])
        mask = np.zeros(n, np.uint8)
        mask[phase % every::every] = 1
        if not mask.any():
            mask[0] = 1
        dep = None if i == ref_i else dep_args(pairs, pre, parents[i])
        t0 = time.perf_counter()
        oracle.analyze(c, f, qp=qp, search_range=wl["R"] if i == ref_i else wl["r"], ctu=wl["ctu"],
                       threads=threads, ctu_mask=mask, dep=dep)
        total += (time.perf_counter() - t0) * n / int(mask.sum())
        sampled += int(mask.sum())
    return total, sampled


def cpu_baseline(wl, samples, budget_s=10.0):
    """The oracle as it stands, all host cores, whole ladder frames until the
    budget is used (at least one); samples = [(pairs, qp)] cycled.  Beside
    it a one-core estimate from a CTU sample of the first frame."""
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    n = 0
    while True:
        pairs, qp = samples[n % len(samples)]
        oracle_ladder_frame(wl, pairs, threads, qp)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    pairs, qp = samples[0]
    pre = oracle_parent_decisions(wl, pairs, qp, threads)
    every = 16
    secs, sampled = oracle_frame_sampled(wl, pairs, qp, pre, 1, every)
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} whole ladder frame(s) of the bench workload ({dt:.1f} s)",
            "one_core": {"value": 1.0 / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"every {every}th CTU of each rung ({sampled} CTUs) single-threaded, the "
                                   "dependents' rules from parent decisions made beforehand, time scaled to "
                                   "the whole frame"}}


# --------------------------------------------------------- device helpers --
def evals_of(out, ctu, rng):
    """SAD-candidate evaluations (8x8 block x candidate) the analysis made."""
    total = 0
    for d, ev in enumerate(out["evaluated"]):
        S = ctu >> d
        total += int(np.count_nonzero(ev)) * (S // 8) ** 2 * (2 * rng + 1) ** 2
    return total


def full_evals(w, h, R):
    return ((w + 7) // 8) * ((h + 7) // 8) * (2 * R + 1) ** 2


def sad_peak(bit_depth, props, clocks, stream):
    """The integer-ALU peak of the SAD kernels: derived from the pipes'
    unit counts and the SM clock (the packed absdiff-accumulate issues at
    64 lanes per clock per SM, 4 absolute differences per 8-bit
    instruction, 2 per 10-bit instruction pair), and the same rate measured
    in this run by the library's probe kernel."""
    from paper_2301_12191_gb300 import ladder as L
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    per_instr = 4 if bit_depth == 8 else 2
    derived = props.multi_processor_count * 64 * per_instr * sm_max * 1e6 / 1e12
    measured = L.ladder_measure_sad_rate(bit_depth, int(stream.cuda_stream)) / 1e12
    note = (f"{props.multi_processor_count} SMs x 64 lanes/clk x {per_instr} absdiff per "
            + ("vabsdiff4.add" if bit_depth == 8 else "min.u16x2 + mad pair") + f" x {sm_max:.0f} MHz")
    return derived, measured, note


def autotune(args, lad, step, tag, stream):
    """Kernel shapes for this workload from the project's autotuner (untimed;
    every shape gives identical decisions)."""
    if args.knobs:
        # fixed shapes (profiler captures that must match a given setting)
        lad.set_tuning(**{k: int(v) for k, v in (kv.split("=") for kv in args.knobs.split(","))})
        return {"knobs": lad.tuning(), "tuned": False, "fixed": args.knobs}
    if args.no_tune:
        return {"knobs": lad.tuning(), "tuned": False}
    from paper_2301_12191_gb300 import tune
    import tempfile
    cache = os.path.join(tempfile.gettempdir(), "ladder_tuning_bench.json")
    res = tune.tune(lad, step, tag=tag, stream=stream, reps=3, warmup=1, cache_path=cache, use_cache=False)
    return {"knobs": res["knobs"], "tuned": True, "trials": len(res["trials"]), "seconds": round(res["seconds"], 2),
            "best_ms": res["ms"]}


def kernel_table(stats):
    tot = max(1e-9, sum(v[1] for v in stats.values()))
    return {k: {"launches": n, "ms_total": ms, "share": ms / tot} for k, (n, ms) in stats.items()}


def decisions_match(a, b, keys=("mvx", "sad", "best")):
    return all(np.array_equal(a[k][d], b[k][d]) for k in keys for d in range(len(b[k])))


# ---------------------------------------------------- one ladder frame / step --
def run_ours(args, wl, name, ctx, extra=False):
    """One ladder frame per step (ladder1080, frame416).  `extra`: the core
    figures only (measured beside another workload's line)."""
    import torch
    from paper_2301_12191_gb300 import ladder as L

    rank, world, local = ctx
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    n_frames = 4
    frames = make_frames(wl, n_frames, seed0=replicas.seed_base(rank))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not extra:
        cpu = cpu_baseline(wl, [(fr, wl["qp"]) for fr in frames])

    sizes = [(w, h) for (w, h, _, _) in frames[0]]
    lad = L.Ladder(sizes, wl["ref"], bit_depth=wl["bit_depth"], ctu_size=wl["ctu"], search_range=wl["R"],
                   refine_range=wl["r"], max_frames=max(E2E_DEPTH, PIPE_STREAMS + 1))
    # the pipelined measurement cycles through more distinct frames than fit
    # in L2 (no flush inside its timed region)
    n_dev = max(n_frames, wl.get("pipelined_frames", n_frames))
    dev_frames = frames + (make_frames(wl, n_dev - n_frames, seed0=replicas.seed_base(rank) + n_frames)
                           if n_dev > n_frames else [])
    dplanes = [[(L.device_plane(c, dev), L.device_plane(f, dev)) for (_, _, c, f) in fr] for fr in dev_frames]
    dev_in_bytes = sum(2 * p[0].numel() * p[0].element_size() for fr in dplanes for p in fr)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ref_i, qp = wl["ref"], wl["qp"]
    n_rungs = len(sizes)

    def step_multi(fi, frame_id=0):
        pl = dplanes[fi % n_dev]
        lad.analyze_reference(frame_id, pl[ref_i][0], pl[ref_i][1], qp)
        if n_rungs > 1:
            lad.analyze_dependents(frame_id, [(i, pl[i][0], pl[i][1]) for i in range(n_rungs) if i != ref_i], qp)

    def step_indep(fi, frame_id=PIPE_STREAMS):
        pl = dplanes[fi % n_frames]
        for i in range(n_rungs):
            lad.analyze_independent(i, frame_id, pl[i][0], pl[i][1], qp)

    def timed(step, K, W):
        for i in range(W):
            step(i)
        torch.cuda.synchronize()
        replicas.barrier()
        torch.cuda.synchronize()
        evs = []
        for i in range(K):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(i)
            b.record(stream)
            flush.fill_(i & 0xff)          # L2 flush between timed steps (not timed)
            evs.append((a, b))
        torch.cuda.synchronize()
        replicas.barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        lad.sync()
        return ms

    def max_over_ranks(v):
        return replicas.max_over_ranks(v, dev)

    # Frame-level parallelism (as x265 encodes several frames at once):
    # consecutive ladder frames take turns on PIPE_STREAMS streams and frame
    # slots, so one frame's full search overlaps the previous frames'
    # dependent kernels.  Timed as one region from the first launch to the
    # last completion; the inputs cycle through n_dev distinct frames.
    pipe_streams = [stream] + [torch.cuda.Stream(dev) for _ in range(PIPE_STREAMS - 1)]

    def step_pipe(i):
        j = i % PIPE_STREAMS
        with torch.cuda.stream(pipe_streams[j]):
            pl = dplanes[i % n_dev]
            lad.analyze_reference(j, pl[ref_i][0], pl[ref_i][1], qp)
            if n_rungs > 1:
                lad.analyze_dependents(j, [(r, pl[r][0], pl[r][1]) for r in range(n_rungs) if r != ref_i], qp)

    def timed_pipe(K, W, step=None):
        step = step or step_pipe
        for i in range(W):
            step(i)
        torch.cuda.synchronize()
        replicas.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(pipe_streams[0])
        for ps in pipe_streams[1:]:
            ps.wait_event(t0)
        for i in range(W, W + K):
            step(i)
        for ps in pipe_streams[1:]:
            joined = torch.cuda.Event()
            joined.record(ps)
            pipe_streams[0].wait_event(joined)
        t1.record(pipe_streams[0])
        torch.cuda.synchronize()
        replicas.barrier()
        lad.sync()
        return t0.elapsed_time(t1)

    # Work per step from one untimed pass.  One SAD-candidate evaluation = one
    # 8x8 block x one candidate (64 absdiffs).  A full search counts its 8x8
    # level only (the SAD tree gets 16/32/64 for free); a dependent rung
    # searches every evaluated CU separately.
    step_multi(0)
    tuning = autotune(args, lad, lambda: step_multi(0), "frames1", stream)
    evals_ref = full_evals(*sizes[ref_i], wl["R"])
    evals_dep = 0
    for i in range(n_rungs):
        if i != ref_i:
            evals_dep += evals_of(lad.fetch(i, 0), wl["ctu"], wl["r"])
    # the evaluations the dependent searches make: the CUs assembled from
    # their sub-CUs' sums are not searched (as the SAD tree's 16/32/64 sums
    # of the full search are not counted)
    torch.cuda.synchronize()
    lad.dependent_evals(stream)
    step_multi(0)
    torch.cuda.synchronize()
    evals_dep_done = lad.dependent_evals(stream)
    evals_multi = evals_ref + evals_dep_done
    evals_every = evals_ref + evals_dep
    evals_indep = sum(full_evals(w, h, wl["R"]) for (w, h) in sizes)

    K, W = args.steps, args.warmup
    indep_steps = max(3, K // 2)
    if args.only_multires:
        ms = max_over_ranks(timed(step_multi, K, W))
        lad.close()
        return {"metric": METRIC, "value": world * K / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": ms / K, "only": "multires"}
    with ClockSampler(local) as clk:
        # untimed soak so that the clock samples (every 200 ms) see the load
        t_end = time.perf_counter() + args.soak
        i = 0
        while time.perf_counter() < t_end:
            step_multi(i)
            i += 1
            if i % 64 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        launches0 = sum(n for n, _ in lad.kernel_stats().values())
        ms_pipe = timed_pipe(K, W)
        launches1 = sum(n for n, _ in lad.kernel_stats().values())
        # the last pipelined frame's decisions equal a serial analysis of the same frame
        last = [lad.fetch(r, (W + K - 1) % PIPE_STREAMS) for r in range(n_rungs)]
        step_multi(W + K - 1, frame_id=PIPE_STREAMS)
        torch.cuda.synchronize()
        again = [lad.fetch(r, PIPE_STREAMS) for r in range(n_rungs)]
        if not all(decisions_match(a, b, ("mvx", "cost", "split")) for a, b in zip(last, again)):
            raise RuntimeError("pipelined decisions differ from a serial analysis of the same frame")
        ms_multi = timed(step_multi, K, W)
        ms_indep = timed(step_indep, indep_steps, W)
    gpu_launches = (launches1 - launches0) * K // (K + W)
    ms_pipe = max_over_ranks(ms_pipe)
    ms_multi = max_over_ranks(ms_multi)
    ms_indep = max_over_ranks(ms_indep)

    # per-kernel device time (events on the launching stream), separate pass
    lad.kernel_stats(reset=True)
    lad.profile(True)
    timed(step_multi, K, 0)
    stats = lad.kernel_stats(reset=True)
    lad.profile(False)

    # end to end through the public API: every step uploads its frame's
    # planes (one copy of a packed pinned buffer holding every rung's cur/ref
    # planes in device-plane layout), analyses it, and reads back every
    # rung's decisions into pinned memory, all inside the timed region.
    host_planes = [[(c, f) for (_, _, c, f) in fr] for fr in frames]
    lay, in_bytes = packed_layout(host_planes[0])
    host_in = [pack_host(hp, lay, in_bytes) for hp in host_planes]
    fbytes = lad.frame_bytes()
    host_out = [torch.empty(fbytes, dtype=torch.uint8).pin_memory() for _ in range(E2E_DEPTH)]
    # the library's frame pipeline (ladder_pipeline_*): each submit uploads
    # one packed frame, analyses it on its slot's stream and reads every
    # rung's decisions back, overlapped with the neighbouring frames; the
    # slots (frame ids 0 .. E2E_DEPTH - 1) take turns, enough of them to hide
    # the copies (about 40 + 10 us per frame at 200 GB/s)
    pipe = lad.pipeline(E2E_DEPTH, 0, in_bytes, [o[0] for o in lay], [o[1] for o in lay], [o[2] for o in lay])
    ticket = 0
    last = -1
    for i in range(W):
        last = pipe.submit(host_in[i % n_frames], qp, host_out[ticket % E2E_DEPTH])
        ticket += 1
    pipe.wait(last)
    torch.cuda.synchronize()
    replicas.barrier()
    t0 = time.perf_counter()
    for i in range(K):
        last = pipe.submit(host_in[i % n_frames], qp, host_out[ticket % E2E_DEPTH])
        ticket += 1
    pipe.wait(last)
    torch.cuda.synchronize()
    replicas.barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    pipe.close()
    lad.sync()
    # the read-back of the last step is that frame's analysis: check one rung
    # of it against a synchronous fetch of the same slot
    jl = last % E2E_DEPTH
    got = lad.frame_views(host_out[jl].numpy())[ref_i]
    if not decisions_match(got, lad.fetch(ref_i, jl)):
        raise RuntimeError("end-to-end read-back differs from the frame's decisions")

    multi_qp = subpel = mvp = None
    if not extra:
        multi_qp = measure_multi_qp(wl, lad, dplanes, step_multi, timed, max_over_ranks, ms_multi, K, W, world, dev)
        subpel = measure_subpel(wl, lad, dplanes, n_dev, step_multi, step_pipe, pipe_streams, timed, timed_pipe,
                                max_over_ranks, ms_multi, K, W, world)
        if wl.get("mvp"):
            lad.set_mv_predictor(1)
            ms_mvp = max_over_ranks(timed(step_multi, K, W))
            ms_mvp_pipe = max_over_ranks(timed_pipe(K, W))
            lad.kernel_stats(reset=True)
            lad.profile(True)
            timed(step_multi, 3, 0)
            st_mvp = lad.kernel_stats(reset=True)
            lad.profile(False)
            # the quarter-pel refinement with the spatial predictor over the
            # refined vectors (SATD tables, then a wavefront launch per frame)
            subpel_mvp = measure_subpel(wl, lad, dplanes, n_dev, step_multi, step_pipe, pipe_streams, timed,
                                        timed_pipe, max_over_ranks, ms_mvp, K, W, world)
            lad.set_mv_predictor(0)
            n_w, t_w = st_mvp.get("decide_mvp", (0, 0.0))
            mvp = {"launches_per_step": n_w // 3, "ms_per_step": ms_mvp / K,
                   "extra_ms_per_step": (ms_mvp - ms_multi) / K,
                   "wavefront_kernel_ms_per_step": t_w / 3 if n_w else None,
                   "ladder_frames_per_s": world * K / (ms_mvp * 1e-3),
                   "pipelined_ladder_frames_per_s": world * K / (ms_mvp_pipe * 1e-3)}
            if subpel_mvp:
                subpel_mvp["launches_per_step"] = 3  # interpolation, SATD tables, wavefront
                mvp["subpel"] = subpel_mvp

    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    peak, peak_probe, peak_note = sad_peak(wl["bit_depth"], props, clocks, stream)

    # dominant kernel of the step
    dom = max(stats.items(), key=lambda kv: kv[1][1])
    kname, (klaunch, kms) = dom
    if kname == "full_search":
        algo = 64 * evals_ref
    elif kname == "dependent":
        algo = 64 * evals_dep_done   # one launch covers every dependent rung
    else:
        algo = None
    achieved = (algo / (kms / klaunch * 1e-3) / 1e12) if (algo and klaunch) else None
    traffic = traffic_of(kname, name, tuning["knobs"])

    frames_per_s = world * K / (ms_pipe * 1e-3)
    result = {
        "metric": METRIC,
        "value": frames_per_s,
        "unit": UNIT,
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms_pipe / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8" if wl["bit_depth"] == 8 else "u16",
        "data": DATA,
        "config": workload_config(name, wl),
        "setup": {
            "distinct_frames": n_dev,
            "l2": (f"inputs larger than L2 ({n_dev} distinct ladder frames, {dev_in_bytes / 2**20:.0f} MiB of "
                   "planes) for the pipelined value; the serial steps flush L2 between steps (256 MiB write, "
                   "outside the step events)"),
            "pipelining": f"consecutive ladder frames take turns on {PIPE_STREAMS} streams and frame slots",
            "parallelism": f"replicas x{world} (independent ladders per GPU)",
            "tuning": tuning,
        },
        "sad_candidate_evals_per_s": evals_multi * world * K / (ms_pipe * 1e-3),
        "sad_candidate_evals_per_step": {"searched": evals_multi, "every_evaluated_cu": evals_every},
        "serial": {"frames_per_s": world * K / (ms_multi * 1e-3), "ms_per_step": ms_multi / K,
                   "note": "one frame at a time on one stream, L2 flushed between steps"},
        "independent": {
            "frames_per_s": world * indep_steps / (ms_indep * 1e-3),
            "ms_per_step": ms_indep / indep_steps,
            "sad_candidate_evals_per_s": evals_indep * world * indep_steps / (ms_indep * 1e-3),
        },
        "multires_speedup_vs_independent": (ms_indep / indep_steps) / (ms_multi / K),  # serial vs serial
        "e2e": {"value": world * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": fbytes},
        "gpu_launches": int(gpu_launches),
        "kernels": kernel_table(stats),
        "roofline": {
            "kernel": kname,
            "bound": "alu",
            "achieved": achieved,
            "peak": peak,
            "unit": "Tabsdiff/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic,
            "peak_note": peak_note,
            "peak_probe_in_run": peak_probe,
            "algorithmic_absdiffs_per_launch": algo,
            "avg_launch_ms": (kms / klaunch) if klaunch else None,
        },
        # the whole path's SAD work (full search + dependent searches) over the
        # pipelined step time, against the same peak
        "path_roofline": {"achieved": evals_multi * 64 * world * K / (ms_pipe * 1e-3) / 1e12, "peak": peak,
                          "unit": "Tabsdiff/s",
                          "frac": evals_multi * 64 * world * K / (ms_pipe * 1e-3) / 1e12 / peak},
        "clocks": dict(clocks, window="untimed soak + timed multi-res and independent loops"),
    }
    if not extra:
        result.update(paper_context=PAPER_CONTEXT, multi_qp=multi_qp, subpel=subpel, spatial_mvp=mvp)
    if cpu is not None:
        result["cpu_baseline"] = cpu
    lad.close()
    return result


def measure_multi_qp(wl, lad, dplanes, step_multi, timed, max_over_ranks, ms_multi, K, W, world, dev):
    """Intra-resolution multi-QP sharing: the decisions of every rung at
    three more QPs from the resident analysis (one launch per rung), per
    frame."""
    import torch
    from paper_2301_12191_gb300 import ladder as L
    if not wl.get("multi_qps"):
        return None
    qps, qp, n_rungs = wl["multi_qps"], wl["qp"], len(lad.rungs)
    outs, keep = {}, []
    for i in range(n_rungs):
        dims, (c8, r8) = lad.grid(i)
        row = []
        for _ in qps:
            o = L.QpDecisions()
            for d, (c, r) in enumerate(dims):
                for k, dt in (("cost", torch.int32), ("best", torch.int32), ("split", torch.uint8)):
                    a = torch.empty(c * r, dtype=dt, device=dev)
                    keep.append(a)
                    getattr(o, k)[d] = a.data_ptr()
            for k, dt in (("leaf_depth", torch.uint8), ("leaf_mvx", torch.int16), ("leaf_mvy", torch.int16)):
                a = torch.empty(c8 * r8, dtype=dt, device=dev)
                keep.append(a)
                setattr(o, k, a.data_ptr())
            row.append(o)
        outs[i] = row
    sh = torch.cuda.current_stream().cuda_stream

    def step_qps(i):
        step_multi(i)
        for r in range(n_rungs):
            L.ladder_decide_qps(lad.handle, r, 0, qps, outs[r], sh)

    ms_qps = max_over_ranks(timed(step_qps, K, W))
    return {"qps": [qp] + list(qps), "master_qp": qp, "launches_per_step": n_rungs,
            "ms_per_step": ms_qps / K, "extra_ms_per_step": (ms_qps - ms_multi) / K,
            "ladder_frames_qps_per_s": world * K * (1 + len(qps)) / (ms_qps * 1e-3)}


def measure_subpel(wl, lad, dplanes, n_dev, step_multi, step_pipe, pipe_streams, timed, timed_pipe,
                   max_over_ranks, ms_multi, K, W, world):
    """Quarter-pel refinement with SATD of every rung of the frame, one
    batched call per frame (two launches: interpolated planes of every rung,
    refinements of every rung)."""
    import torch
    from paper_2301_12191_gb300 import ladder as L
    if not wl.get("subpel"):
        return None
    qp, n_rungs = wl["qp"], len(lad.rungs)
    bufs = [lad.subpel_buffers(r) for r in range(n_rungs)]
    sh2 = torch.cuda.current_stream().cuda_stream
    sp_jobs = [lad.subpel_jobs([(0, r, pl[r][0], pl[r][1], qp) for r in range(n_rungs)], bufs) for pl in dplanes]

    def step_subpel(i):
        step_multi(i)
        L._call(lad.handle, "ladder_refine_subpel_batch", lad.handle, n_rungs, sp_jobs[i % n_dev], sh2)

    ms_sp = max_over_ranks(timed(step_subpel, K, W))
    lad.kernel_stats(reset=True)
    lad.profile(True)
    timed(step_subpel, 3, 0)
    st_sp = lad.kernel_stats(reset=True)
    lad.profile(False)
    n_sp, t_sp = st_sp.get("subpel", (0, 0.0))
    # the same with consecutive frames pipelined: each slot refines on its
    # own stream into its own outputs and workspaces
    slot_bufs = [[lad.subpel_buffers(r) for r in range(n_rungs)] for _ in range(PIPE_STREAMS)]
    slot_jobs = [[lad.subpel_jobs([(j, r, pl[r][0], pl[r][1], qp) for r in range(n_rungs)], slot_bufs[j])
                  for pl in dplanes] for j in range(PIPE_STREAMS)]

    def step_pipe_sp(i):
        step_pipe(i)
        j = i % PIPE_STREAMS
        L._call(lad.handle, "ladder_refine_subpel_batch", lad.handle, n_rungs, slot_jobs[j][i % n_dev],
                pipe_streams[j].cuda_stream)

    ms_sp_pipe = max_over_ranks(timed_pipe(K, W, step_pipe_sp))
    return {"launches_per_step": 2, "ms_per_step": ms_sp / K, "extra_ms_per_step": (ms_sp - ms_multi) / K,
            "kernel_ms_per_step": t_sp / 3 if n_sp else None,
            "ladder_frames_per_s": world * K / (ms_sp * 1e-3),
            "pipelined_ladder_frames_per_s": world * K / (ms_sp_pipe * 1e-3)}


# ------------------------------------------------ batched ladder frames --
def run_batch(args, wl, name, ctx):
    """Many ladder frames per step: one captured graph replays
    ladder_analyze_batch over every (ladder, consecutive pair)."""
    import torch
    from paper_2301_12191_gb300 import ladder as L

    rank, world, local = ctx
    dev = torch.device("cuda", local)
    if args.ladders:
        wl = dict(wl, ladders=args.ladders)  # smaller batches for profiler captures
    frames, reqs = batch_requests(wl, seed0=3000 + 1000 * rank)
    n = len(reqs)
    sizes = list(wl["rungs"])
    ref_i = wl["ref"]
    qps = [q for (_, _, q) in reqs]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, [(request_pairs(wl, frames, reqs[k]), qps[k]) for k in range(min(2, n))])
    dplanes = [[[L.device_plane(p, dev) for p in fr] for fr in seq] for seq in frames]
    dev_in_bytes = sum(p.numel() * p.element_size() for seq in dplanes for fr in seq for p in fr)
    items = [(k, qp, [(dplanes[l][t + 1][r], dplanes[l][t][r]) for r in range(len(sizes))])
             for k, (l, t, qp) in enumerate(reqs)]
    lad = L.Ladder(sizes, ref_i, bit_depth=wl["bit_depth"], ctu_size=wl["ctu"], search_range=wl["R"],
                   refine_range=wl["r"], max_frames=2 * n)
    if wl.get("parents"):
        lad.set_parents(wl["parents"])  # cascaded reference chain
    items_ind = [(n + k, qp, pl) for (k, qp, pl) in items]
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        lad.analyze_batch(items, stream)                 # eager once (sets up slots)
        if not args.only_multires:
            lad.analyze_batch_independent(items_ind, stream)
    stream.synchronize()
    lad.sync(stream)
    tuning = autotune(args, lad, lambda: lad.analyze_batch(items, stream), f"frames{n}", stream)
    g_multi = lad.capture_batch(items, stream)

    def timed(fn, K, W):
        for _ in range(W):
            fn()
        stream.synchronize()
        replicas.barrier()
        stream.synchronize()
        evs = []
        for _ in range(K):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        stream.synchronize()
        replicas.barrier()
        return sum(a.elapsed_time(b) for a, b in evs)

    def max_over_ranks(v):
        return replicas.max_over_ranks(v, dev)

    K, W = args.steps, args.warmup
    if args.only_multires:
        # warm-up and timed graph replays only: one eager batch, then W + K
        # replays of 4 launches each (the profiler's launch list)
        ms = max_over_ranks(timed(lambda: g_multi.launch(stream), K, W))
        lad.sync(stream)
        g_multi.close()
        lad.close()
        return {"metric": METRIC, "value": world * n * K / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": ms / K, "only": "multires", "ladder_frames_per_step": n}
    # algorithmic work: the full search at its 8x8 level, the dependents'
    # evaluated CUs of every request of the batch (per request, averaged)
    evals_ref = full_evals(*sizes[ref_i], wl["R"])
    evals_dep = sum(evals_of(lad.fetch(r, k), wl["ctu"], wl["r"]) for k in range(n)
                    for r in range(len(sizes)) if r != ref_i) / n
    evals_multi = n * (evals_ref + evals_dep)
    evals_indep = n * sum(full_evals(w, h, wl["R"]) for (w, h) in sizes)
    indep_steps = max(3, K // 2)
    with ClockSampler(local) as clk:
        t_end = time.perf_counter() + args.soak
        while time.perf_counter() < t_end:
            g_multi.launch(stream)
            stream.synchronize()
        ms_multi = max_over_ranks(timed(lambda: g_multi.launch(stream), K, W))
        ms_indep = max_over_ranks(timed(lambda: lad.analyze_batch_independent(items_ind, stream), indep_steps, W))
    lad.sync(stream)
    lad.kernel_stats(reset=True)
    lad.dependent_evals(stream)  # reset the count of evaluations the dependent searches make
    lad.profile(True)
    for _ in range(3):
        lad.analyze_batch(items, stream)
    stats = lad.kernel_stats(reset=True)
    lad.profile(False)
    # evaluations the dependent searches made per ladder frame: the CUs
    # assembled from their sub-CUs' sums are not searched (as the SAD tree's
    # 16/32/64 sums of the full search are not counted)
    evals_dep_done = lad.dependent_evals(stream) / (3 * n)
    launches_per_step = sum(nl for nl, _ in stats.values()) // 3
    dom = max(stats.items(), key=lambda kv: kv[1][1])
    kname, (klaunch, kms) = dom

    # end to end through the library's frame pipeline (ladder_pipeline_*):
    # each submit uploads one ladder frame's packed planes from pinned host
    # memory, analyses it (reference rung, then the dependents) on its slot's
    # stream and reads every rung's decisions back into pinned memory; the
    # frames of a step are the batch's n ladder frames
    lad_e2e = L.Ladder(sizes, ref_i, bit_depth=wl["bit_depth"], ctu_size=wl["ctu"], search_range=wl["R"],
                       refine_range=wl["r"], max_frames=E2E_DEPTH)
    if wl.get("parents"):
        lad_e2e.set_parents(wl["parents"])
    lad_e2e.set_tuning(**lad.tuning())
    host_planes = [[(frames[l][t + 1][r], frames[l][t][r]) for r in range(len(sizes))] for (l, t, _) in reqs]
    lay, in_bytes = packed_layout(host_planes[0])
    host_in = [pack_host(hp, lay, in_bytes) for hp in host_planes]
    fbytes = lad_e2e.frame_bytes()
    host_out = [torch.empty(fbytes, dtype=torch.uint8).pin_memory() for _ in range(E2E_DEPTH)]
    pipe = lad_e2e.pipeline(E2E_DEPTH, 0, in_bytes, [o[0] for o in lay], [o[1] for o in lay], [o[2] for o in lay])
    ticket, last = 0, -1
    for i in range(W * n):
        last = pipe.submit(host_in[i % n], qps[i % n], host_out[ticket % E2E_DEPTH])
        ticket += 1
    pipe.wait(last)
    torch.cuda.synchronize()
    replicas.barrier()
    t0 = time.perf_counter()
    for i in range(K * n):
        last = pipe.submit(host_in[i % n], qps[i % n], host_out[ticket % E2E_DEPTH])
        ticket += 1
    pipe.wait(last)
    torch.cuda.synchronize()
    replicas.barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    pipe.close()
    lad_e2e.sync()
    # the last frame read back equals the batch's analysis of the same request
    got = lad_e2e.frame_views(host_out[last % E2E_DEPTH].numpy())
    k_last = (K * n - 1) % n
    for r in (ref_i, 0):
        if not decisions_match(got[r], lad.fetch(r, k_last)):
            raise RuntimeError(f"end-to-end read-back of rung {r} differs from the batch's analysis")
    lad_e2e.close()

    props = torch.cuda.get_device_properties(dev)
    clocks = clk.summary()
    peak, peak_probe, peak_note = sad_peak(wl["bit_depth"], props, clocks, stream)
    # algorithmic absdiffs of one step (all the kind's launches of the step:
    # a cascaded chain runs one dependent search per tier) over its summed
    # kernel time per step (the profile pass ran 3 steps)
    algo = {"full_search": 64 * evals_ref * n, "dependent": 64 * evals_dep_done * n}.get(kname)
    achieved = (algo / (kms / 3 * 1e-3) / 1e12) if (algo and klaunch) else None
    other = "dependent" if kname == "full_search" else "full_search"
    o_n, o_ms = stats.get(other, (0, 0.0))
    o_algo = 64 * (evals_dep_done if other == "dependent" else evals_ref) * n
    evals_done = n * (evals_ref + evals_dep_done)
    result = {
        "metric": METRIC, "value": world * n * K / (ms_multi * 1e-3), "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms_multi / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8" if wl["bit_depth"] == 8 else "u16", "data": DATA,
        "config": workload_config(name, wl),
        "setup": {"ladder_frames_per_step": n, "l2": f"inputs larger than L2 ({dev_in_bytes / 2**20:.0f} MiB of "
                  "planes, no flush)", "launch": f"one CUDA graph per step ({launches_per_step} kernels)",
                  "parallelism": f"replicas x{world} (independent ladders per GPU)", "tuning": tuning},
        "sad_candidate_evals_per_s": world * evals_done * K / (ms_multi * 1e-3),
        "sad_candidate_evals_per_step": {"searched": evals_done, "every_evaluated_cu": evals_multi,
                                         "note": "searched: the reference rung's 8x8 level and the dependent "
                                                 "CUs searched; every_evaluated_cu also counts the dependent CUs "
                                                 "whose SADs are sums of their sub-CUs'"},
        "independent": {"frames_per_s": world * n * indep_steps / (ms_indep * 1e-3),
                        "ms_per_step": ms_indep / indep_steps,
                        "sad_candidate_evals_per_s": world * evals_indep * indep_steps / (ms_indep * 1e-3)},
        "multires_speedup_vs_independent": (ms_indep / indep_steps) / (ms_multi / K),
        "e2e": {"value": world * n * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": in_bytes * n,
                "d2h_bytes_per_step": fbytes * n,
                "path": f"ladder_pipeline_submit per ladder frame, {E2E_DEPTH} frame slots"},
        "kernels": kernel_table(stats),
        "gpu_launches": launches_per_step * K,
        "roofline": {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tabsdiff/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic_of(kname, name, tuning["knobs"]),
                     "peak_note": peak_note, "peak_probe_in_run": peak_probe,
                     "algorithmic_absdiffs_per_step": algo, "kernel_ms_per_step": kms / 3,
                     "launches_per_step": klaunch // 3,
                     other: {"achieved": (o_algo / (o_ms / 3 * 1e-3) / 1e12) if o_n else None,
                             "frac": (o_algo / (o_ms / 3 * 1e-3) / 1e12 / peak) if o_n else None,
                             "kernel_ms_per_step": o_ms / 3}},
        # the whole path's SAD work over the step time, against the same peak
        "path_roofline": {"achieved": evals_done * 64 * K / (ms_multi * 1e-3) / 1e12, "peak": peak,
                          "unit": "Tabsdiff/s", "frac": evals_done * 64 * K / (ms_multi * 1e-3) / 1e12 / peak},
        "clocks": dict(clocks, window="untimed soak + timed loops"),
        "paper_context": PAPER_CONTEXT,
    }
    # spatial MV predictor with the wavefront CTU order: the same step with
    # every rung's cost / split decided row by row (one more launch per tier)
    if wl.get("mvp"):
        lad.set_mv_predictor(1)
        g_mvp = lad.capture_batch(items, stream)
        ms_mvp = max_over_ranks(timed(lambda: g_mvp.launch(stream), K, W))
        lad.kernel_stats(reset=True)
        lad.profile(True)
        for _ in range(3):
            lad.analyze_batch(items, stream)
        st_mvp = lad.kernel_stats(reset=True)
        lad.profile(False)
        lad.set_mv_predictor(0)
        g_mvp.close()
        n_w, t_w = st_mvp.get("decide_mvp", (0, 0.0))
        result["spatial_mvp"] = {"launches_per_step": n_w // 3, "ms_per_step": ms_mvp / K,
                                 "extra_ms_per_step": (ms_mvp - ms_multi) / K,
                                 "wavefront_kernel_ms_per_step": t_w / 3 if n_w else None,
                                 "ladder_frames_per_s": world * n * K / (ms_mvp * 1e-3)}
    if cpu:
        result["cpu_baseline"] = cpu
    lad.sync(stream)
    g_multi.close()
    lad.close()
    return result


# ------------------------------------------------------------- serving --
def serve_setup(wl, seed0=500):
    """Ladder classes (one per bit depth) and their pre-made content: two
    ladder frames each, as lists over rungs of (cur, ref) planes."""
    from paper_2301_12191_gb300 import serve
    classes, content = {}, {}
    for bd in wl["bit_depths"]:
        k = f"ladder{bd}"
        classes[k] = serve.LadderClass(rungs=wl["rungs"], ref_rung=wl["ref"], bit_depth=bd,
                                       search_range=wl["R"], refine_range=wl["r"], ctu=wl["ctu"],
                                       max_frames=wl["max_frames"])
        frames = []
        for f in range(2):
            pairs, _ = synth.ladder_pairs(seed0 + 10 * bd + f, source=wl["source"], rungs=wl["rungs"][1:],
                                          bit_depth=bd, include_source=True)
            frames.append([(c, r) for (_, _, c, r) in pairs])
        content[k] = frames
    return classes, content


def run_serve(args, wl, name, ctx):
    """Continuous-batching serving loop, one per GPU (each rank serves its
    own seeded request stream): latency percentiles, throughput and device
    memory held by resident reference state."""
    import torch
    from paper_2301_12191_gb300 import serve

    rank, world, local = ctx
    dev = torch.device("cuda", local)
    classes, content = serve_setup(wl)
    pinned = {k: [[(serve.pin_plane(c), serve.pin_plane(r)) for c, r in fr] for fr in v]
              for k, v in content.items()}
    ex = serve.GpuExecutor(classes, n_streams=wl["streams"])
    kw = dict(hbm_budget=wl["hbm_budget"], max_batch=wl["max_batch"], max_inflight=wl["streams"])
    # warm-up: a short burst through every class (module load, first launches)
    warm = serve.request_stream(99, 12 * max(1, args.warmup), 2000.0, classes, pinned, qps=wl["qps"],
                                n_open=wl["n_open"], first_frame=1 << 20)
    serve.Server(classes, ex, **kw).run(warm)
    torch.cuda.synchronize()
    n_req = int(wl["rate"] * wl["seconds"])
    reqs = serve.request_stream(7 + rank, n_req, wl["rate"], classes, pinned, qps=wl["qps"], n_open=wl["n_open"])
    launches0 = sum(n for lad in ex.ladders.values() for n, _ in lad.kernel_stats().values())
    srv = serve.Server(classes, ex, **kw)
    replicas.barrier()
    with ClockSampler(local) as clk:
        rep = srv.run(reqs)
        torch.cuda.synchronize()
    replicas.barrier()
    launches = sum(n for lad in ex.ladders.values() for n, _ in lad.kernel_stats().values()) - launches0
    h2d = sum(2 * classes[r.klass].plane_bytes(r.rung) for r in reqs) // max(1, len(reqs))
    rung_mix = {f"{w}x{h}": sum(1 for r in reqs if classes[r.klass].rungs[r.rung] == (w, h)) for (w, h) in wl["rungs"]}
    ex.close()
    # whole job: every rank's completed requests over the slowest rank's time;
    # latency percentiles: the worst rank's
    elapsed = replicas.max_over_ranks(rep["elapsed_s"], dev)
    completed = replicas.sum_over_ranks(rep["completed"], dev)
    p50 = replicas.max_over_ranks(rep["latency_p50_ms"], dev)
    p99 = replicas.max_over_ranks(rep["latency_p99_ms"], dev)
    return {
        "metric": "served frame-pair analysis requests/sec (continuous batching)",
        "value": completed / elapsed, "unit": "requests/s", "n_gpus": world,
        "higher_is_better": True, "dtype": "u8+u16", "data": "synthetic", "scaling": "weak",
        "offered_rate": wl["rate"] * world, "latency_p50_ms": p50, "latency_p99_ms": p99,
        "completed": rep["completed"], "failed": rep["failed"], "elapsed_s": elapsed,
        "resident_bytes_max": rep["resident_bytes_max"], "resident_bytes_mean": rep["resident_bytes_mean"],
        "held_bytes_max": rep["held_bytes_max"], "batches": rep["batches"], "mean_batch": rep["mean_batch"],
        "gpu_launches": launches, "h2d_bytes_per_request": h2d, "clocks": clk.summary(),
        "config": {"workload": name, "rungs": [f"{w}x{h}" for (w, h) in wl["rungs"]], "bit_depths": wl["bit_depths"],
                   "R": wl["R"], "r": wl["r"], "rung_mix": rung_mix, "streams": wl["streams"],
                   "hbm_budget": wl["hbm_budget"], "max_frames": wl["max_frames"]},
    }


# ---------------------------------------------------------- oracle arm --
def run_reference(args, wl, name):
    """The oracle on the host cores, same metric, workload and config.  A
    step is one ladder frame: whole frames for the 1080p ladder and the
    single pair; for the batched workloads a CTU sample of every rung of one
    ladder frame (every oracle_every-th CTU, a different phase each step),
    its time scaled to the whole frame, so that K + W steps end within a few
    minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    threads = os.cpu_count() or 1
    if wl.get("mode") == "batch":
        frames, reqs = batch_requests(wl, seed0=3000, ladders=2)
        samples = [(request_pairs(wl, frames, q), q[2]) for q in reqs]
        pre = [oracle_parent_decisions(wl, pairs, qp, threads) for pairs, qp in samples]
        every = wl.get("oracle_every", 4)

        def step(i):
            pairs, qp = samples[i % len(samples)]
            return oracle_frame_sampled(wl, pairs, qp, pre[i % len(samples)], threads, every, phase=i)[0]

        for i in range(args.warmup):
            step(i)
        secs = sum(step(args.warmup + i) for i in range(args.steps))
        sample = (f"{args.steps} ladder frames, each estimated from every {every}th CTU of each rung (a new "
                  "phase per step), the dependents' rules from parent decisions made beforehand (untimed)")
    else:
        frames = make_frames(wl, 2, seed0=1000)
        for i in range(args.warmup):
            oracle_ladder_frame(wl, frames[i % 2], threads, wl["qp"])
        t0 = time.perf_counter()
        for i in range(args.steps):
            oracle_ladder_frame(wl, frames[i % 2], threads, wl["qp"])
        secs = time.perf_counter() - t0
        sample = f"{args.steps} whole ladder frames"
    v = args.steps / secs
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8" if wl["bit_depth"] == 8 else "u16",
        "data": DATA, "config": workload_config(name, wl),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def summary_of(res):
    """The core figures of a workload measured beside the main line."""
    keep = ("value", "unit", "ms_per_step", "dtype", "config", "serial", "independent",
            "multires_speedup_vs_independent", "e2e", "roofline", "path_roofline", "gpu_launches", "kernels",
            "clocks", "setup")
    return {k: res[k] for k in keep if k in res}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(WORKLOADS), default=DEFAULT_CONFIG)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the workloads measured beside the main line")
    ap.add_argument("--no-tune", action="store_true", help="keep the default kernel shapes (skip the autotuner)")
    ap.add_argument("--knobs", default="", help="fixed kernel shapes, e.g. dep_band=17,dep_range=16 (no autotuner)")
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--soak", type=float, default=1.5, help="untimed seconds of load before timing (clock sampling)")
    ap.add_argument("--only-multires", action="store_true",
                    help="run only warm-up + the timed multi-resolution steps (for profiler launch lists)")
    ap.add_argument("--ladders", type=int, default=0,
                    help="batched workloads: ladders per step instead of the workload's (smaller profiler cases)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start the ranks here (torchrun-style launch)
        sys.exit(replicas.spawn(os.path.abspath(__file__), sys.argv[1:], args.gpus).returncode)
    name = args.config
    wl = WORKLOADS[name]
    if args.impl == "reference":
        if wl.get("mode") == "serve":
            res = {"impl": "reference", "unavailable": "the serving loop has no CPU counterpart; the oracle is "
                   "timed on the ladder workloads"}
        else:
            res = run_reference(args, wl, name)
        if res is not None:
            print(json.dumps(res))
        return
    import torch
    rank, world, local = replicas.env()
    torch.cuda.set_device(local)
    replicas.init("nccl")
    ctx = (rank, world, local)
    runner = {"serve": run_serve, "batch": run_batch}.get(wl.get("mode"), run_ours)
    res = runner(args, wl, name, ctx)
    if not args.no_extra and not args.only_multires:
        for ex_name in EXTRA.get(name, []):
            res[ex_name] = summary_of(run_ours(args, WORKLOADS[ex_name], ex_name, ctx, extra=True))
    replicas.barrier()
    if rank == 0:
        print(json.dumps(res))
        if args.json_out:
            with open(args.json_out, "w") as fh:
                json.dump(res, fh, indent=1)
    replicas.finish()


if __name__ == "__main__":
    main()
