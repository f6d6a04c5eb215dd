"""ctypes binding of libladder.so (C ABI in include/ladder.h).

Argument marshalling only: every step of the analysis runs in the CUDA
library.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library cannot be loaded this module raises.

Functions with the C names (``ladder_init``, ``analyze_reference``,
``analyze_dependent``, ``analyze_independent``, ``fetch_decisions``,
``ladder_grid``, ``ladder_sync``, ``ladder_release_frame``,
``ladder_destroy``) take raw pointers; :class:`Ladder` wraps them for torch
tensors and numpy outputs.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAX_DEPTHS = 4
STATUS = {0: "LADDER_OK", -1: "LADDER_E_INVAL", -2: "LADDER_E_NOMEM", -3: "LADDER_E_NOREF",
          -4: "LADDER_E_BUSY", -5: "LADDER_E_CUDA", -6: "LADDER_E_TIMEOUT", -7: "LADDER_E_STATE",
          -8: "LADDER_E_BOUNDS"}


class LadderError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Rung(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int)]


class Geometry(ctypes.Structure):
    _fields_ = [("n_rungs", ctypes.c_int), ("rungs", ctypes.POINTER(Rung)), ("ref_rung", ctypes.c_int),
                ("bit_depth", ctypes.c_int), ("ctu_size", ctypes.c_int), ("ref_search_range", ctypes.c_int),
                ("dep_refine_range", ctypes.c_int), ("dep_depth_lo", ctypes.c_int),
                ("dep_depth_hi", ctypes.c_int), ("dep_use_ref_mv", ctypes.c_int), ("satd_mode", ctypes.c_int),
                ("max_frames", ctypes.c_int)]


class Decisions(ctypes.Structure):
    _fields_ = [("mvx", ctypes.c_void_p * MAX_DEPTHS), ("mvy", ctypes.c_void_p * MAX_DEPTHS),
                ("sad", ctypes.c_void_p * MAX_DEPTHS), ("satd", ctypes.c_void_p * MAX_DEPTHS),
                ("cost", ctypes.c_void_p * MAX_DEPTHS), ("best", ctypes.c_void_p * MAX_DEPTHS),
                ("split", ctypes.c_void_p * MAX_DEPTHS), ("evaluated", ctypes.c_void_p * MAX_DEPTHS),
                ("leaf_depth", ctypes.c_void_p), ("leaf_mvx", ctypes.c_void_p), ("leaf_mvy", ctypes.c_void_p)]


class QpDecisions(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_void_p * MAX_DEPTHS), ("best", ctypes.c_void_p * MAX_DEPTHS),
                ("split", ctypes.c_void_p * MAX_DEPTHS),
                ("leaf_depth", ctypes.c_void_p), ("leaf_mvx", ctypes.c_void_p), ("leaf_mvy", ctypes.c_void_p)]


class SubpelDecisions(ctypes.Structure):
    _fields_ = [("qmvx", ctypes.c_void_p * MAX_DEPTHS), ("qmvy", ctypes.c_void_p * MAX_DEPTHS),
                ("satd", ctypes.c_void_p * MAX_DEPTHS), ("cost", ctypes.c_void_p * MAX_DEPTHS),
                ("best", ctypes.c_void_p * MAX_DEPTHS), ("split", ctypes.c_void_p * MAX_DEPTHS),
                ("leaf_depth", ctypes.c_void_p), ("leaf_qmvx", ctypes.c_void_p), ("leaf_qmvy", ctypes.c_void_p)]


class SubpelJob(ctypes.Structure):
    _fields_ = [("frame_id", ctypes.c_int), ("rung", ctypes.c_int), ("qp", ctypes.c_int),
                ("cur", ctypes.c_void_p), ("ref", ctypes.c_void_p), ("pitch_bytes", ctypes.c_long),
                ("out", ctypes.POINTER(SubpelDecisions)), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_long)]


MAX_SUBPEL_JOBS = 16


class Job(ctypes.Structure):
    _fields_ = [("frame_id", ctypes.c_int), ("rung", ctypes.c_int), ("kind", ctypes.c_int), ("qp", ctypes.c_int),
                ("cur", ctypes.c_void_p), ("ref", ctypes.c_void_p), ("pitch_bytes", ctypes.c_long)]


class Request(ctypes.Structure):
    _fields_ = [("frame_id", ctypes.c_int), ("qp", ctypes.c_int), ("cur", ctypes.POINTER(ctypes.c_void_p)),
                ("ref", ctypes.POINTER(ctypes.c_void_p)), ("pitch_bytes", ctypes.POINTER(ctypes.c_long))]


# (name, restype, argtypes) of every symbol declared in include/ladder.h
SIGNATURES = [
    ("ladder_init", ctypes.c_int, [ctypes.POINTER(Geometry), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("analyze_reference", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_long, ctypes.c_int, ctypes.c_void_p]),
    ("analyze_dependent", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_void_p]),
    ("analyze_dependents", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.POINTER(ctypes.c_long), ctypes.c_int, ctypes.c_void_p]),
    ("ladder_analyze_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.c_int, ctypes.c_void_p]),
    ("ladder_analyze_jobs", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Job), ctypes.c_int, ctypes.c_void_p]),
    ("ladder_analyze_batch_independent", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.c_int,
                                                        ctypes.c_void_p]),
    ("ladder_capture_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.c_int, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    ("ladder_graph_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ladder_graph_destroy", None, [ctypes.c_void_p]),
    ("ladder_device_bytes", ctypes.c_long, [ctypes.c_void_p]),
    ("analyze_independent", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_void_p]),
    ("fetch_decisions", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Decisions),
                                       ctypes.c_void_p]),
    ("ladder_set_parents", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("ladder_load_reference", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Decisions),
                                             ctypes.c_void_p]),
    ("ladder_set_mv_predictor", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("ladder_refine_subpel", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_long, ctypes.c_int,
                                            ctypes.POINTER(SubpelDecisions), ctypes.c_void_p, ctypes.c_long,
                                            ctypes.c_void_p]),
    ("ladder_subpel_workspace_bytes", ctypes.c_long, [ctypes.c_void_p, ctypes.c_int]),
    ("ladder_pipeline_create", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_long,
                                              ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                                              ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_void_p)]),
    ("ladder_pipeline_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.POINTER(ctypes.c_long)]),
    ("ladder_pipeline_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_long]),
    ("ladder_pipeline_destroy", None, [ctypes.c_void_p]),
    ("ladder_refine_subpel_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(SubpelJob),
                                                  ctypes.c_void_p]),
    ("ladder_frame_bytes", ctypes.c_long, [ctypes.c_void_p]),
    ("ladder_decision_offsets", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_long)]),
    ("ladder_fetch_frame_async", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_long,
                                                ctypes.c_void_p]),
    ("ladder_decide_qps", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(QpDecisions), ctypes.c_void_p]),
    ("ladder_grid", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]),
    ("ladder_release_frame", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("ladder_sync", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ladder_destroy", None, [ctypes.c_void_p]),
    ("ladder_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("ladder_profile_enable", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("ladder_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_long),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("analyze_reference_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, ctypes.POINTER(Decisions),
                                                 ctypes.c_void_p]),
    ("analyze_reference_noalloc_status", ctypes.c_int, [ctypes.c_void_p]),
    ("ladder_measure_sad_rate", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("ladder_version", ctypes.c_char_p, []),
    ("ladder_set_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("ladder_get_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("ladder_set_debug", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("ladder_dependent_evals", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.POINTER(ctypes.c_ulonglong)]),
]

KERNEL_KINDS = ("full_search", "decide", "dependent", "fill_keys", "dep_rules", "dep_decide", "decide_qps",
                "subpel", "decide_mvp")
TUNE_KNOBS = {"fs_band": 0, "dep_band": 1, "dep_range": 2, "dep_ctas_per_sm": 3, "fs_group": 4, "fs_fuse": 5,
              "dep_staged": 6, "dep_inherit": 7}
DEBUG_CONTROLS = {"wait_polls": 0, "lost_handoff": 1}

_lib = None


def debug_build_requested() -> bool:
    """LADDER_DEBUG_BUILD=1 in the environment selects the bounds-checked
    debug build of the library (libladder_debug.so) for this process."""
    return os.environ.get("LADDER_DEBUG_BUILD", "0") not in ("", "0")


def library_path() -> str:
    return _build.LIB_DEBUG if debug_build_requested() else _build.LIB


def load(build_if_missing: bool = True):
    """Loads libladder.so, or libladder_debug.so when LADDER_DEBUG_BUILD=1
    (building it first when it is missing or stale and nvcc is available);
    raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    debug = debug_build_requested()
    path = library_path()
    if build_if_missing and _build.stale(debug=debug):
        _build.build(debug=debug)
    if not os.path.exists(path):
        raise OSError(f"{os.path.basename(path)} not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _call(handle, name, *args):
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        msg = lib.ladder_last_error(handle).decode() if handle else ""
        raise LadderError(st, f"{name}: {msg}")
    return st


# ---- C names, raw pointers ------------------------------------------------
def ladder_init(geometry: Geometry, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    st = load().ladder_init(ctypes.byref(geometry), ctypes.c_void_p(stream), ctypes.byref(h))
    if st != 0:
        raise LadderError(st, "ladder_init")
    return h.value


def analyze_reference(h, frame_id, cur_ptr, ref_ptr, pitch_bytes, qp, stream=0):
    return _call(h, "analyze_reference", h, frame_id, cur_ptr, ref_ptr, pitch_bytes, qp, stream)


def analyze_dependent(h, rung, frame_id, cur_ptr, ref_ptr, pitch_bytes, qp, stream=0):
    return _call(h, "analyze_dependent", h, rung, frame_id, cur_ptr, ref_ptr, pitch_bytes, qp, stream)


def analyze_dependents(h, frame_id, rungs, cur_ptrs, ref_ptrs, pitches, qp, stream=0):
    n = len(rungs)
    return _call(h, "analyze_dependents", h, frame_id, n, (ctypes.c_int * n)(*rungs),
                 (ctypes.c_void_p * n)(*cur_ptrs), (ctypes.c_void_p * n)(*ref_ptrs), (ctypes.c_long * n)(*pitches),
                 qp, stream)


def analyze_independent(h, rung, frame_id, cur_ptr, ref_ptr, pitch_bytes, qp, stream=0):
    return _call(h, "analyze_independent", h, rung, frame_id, cur_ptr, ref_ptr, pitch_bytes, qp, stream)


def fetch_decisions(h, rung, frame_id, decisions: Decisions, stream=0):
    return _call(h, "fetch_decisions", h, rung, frame_id, ctypes.byref(decisions), stream)


def ladder_decide_qps(h, rung, frame_id, qps, outs, stream=0):
    n = len(qps)
    arr = (ctypes.c_int * n)(*qps)
    out = (QpDecisions * n)(*outs)
    _call(h, "ladder_decide_qps", h, rung, frame_id, n, arr, out, stream)


def ladder_grid(h, rung):
    dims = (ctypes.c_int * (2 * MAX_DEPTHS + 2))()
    nd = ctypes.c_int()
    _call(h, "ladder_grid", h, rung, dims, ctypes.byref(nd))
    n = nd.value
    return [(dims[2 * d], dims[2 * d + 1]) for d in range(n)], (dims[2 * n], dims[2 * n + 1])


def ladder_sync(h, stream=0):
    return _call(h, "ladder_sync", h, stream)


def ladder_release_frame(h, frame_id):
    return _call(h, "ladder_release_frame", h, frame_id)


def ladder_destroy(h):
    load().ladder_destroy(h)


def ladder_profile_enable(h, enable: bool):
    return _call(h, "ladder_profile_enable", h, 1 if enable else 0)


def ladder_profile_read(h, kind: int, reset: bool = False):
    n = ctypes.c_long()
    ms = ctypes.c_double()
    _call(h, "ladder_profile_read", h, kind, ctypes.byref(n), ctypes.byref(ms), 1 if reset else 0)
    return n.value, ms.value


def analyze_reference_noalloc(cur_ptr, ref_ptr, width, height, pitch_bytes, bit_depth, ctu_size, search_range, qp,
                              satd_mode, device_decisions: Decisions, stream=0):
    """One-frame independent analysis into caller-owned device arrays; the
    library allocates nothing (see include/ladder.h)."""
    st = load().analyze_reference_noalloc(cur_ptr, ref_ptr, width, height, pitch_bytes, bit_depth, ctu_size,
                                          search_range, qp, satd_mode, ctypes.byref(device_decisions), stream)
    if st != 0:
        raise LadderError(st, "analyze_reference_noalloc")
    return st


def ladder_measure_sad_rate(bit_depth: int, stream=0) -> float:
    """Absolute differences per second of the searches' packed SAD
    instruction form on the current device (see include/ladder.h)."""
    v = ctypes.c_double()
    st = load().ladder_measure_sad_rate(int(bit_depth), stream, ctypes.byref(v))
    if st != 0:
        raise LadderError(st, "ladder_measure_sad_rate")
    return v.value


def analyze_reference_noalloc_status(stream=0) -> int:
    """Status of the allocation-free analyses since the last query (0, or
    -6 if a bounded device wait ran out); waits for `stream`, clears it."""
    return int(load().analyze_reference_noalloc_status(stream))


# ---- torch convenience ----------------------------------------------------
def device_plane(array, device="cuda"):
    """Copies an (H, W) uint8 / uint16 numpy plane into a CUDA tensor whose
    row pitch is a multiple of 128 bytes; returns the (H, W) view."""
    import torch
    a = np.ascontiguousarray(array)
    H, W = a.shape
    if a.dtype == np.uint8:
        tdt, es = torch.uint8, 1
        src = torch.from_numpy(a)
    elif a.dtype == np.uint16:
        tdt, es = torch.int16, 2          # same bits for samples in [0, 1023]
        src = torch.from_numpy(a.view(np.int16))
    else:
        raise ValueError("planes must be uint8 or uint16")
    pitch = (W * es + 127) // 128 * 128
    buf = torch.zeros((H, pitch // es), dtype=tdt, device=device)
    view = buf[:, :W]
    view.copy_(src.to(device))
    return view


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _pitch_bytes(t) -> int:
    return int(t.stride(0) * t.element_size())


class Pipeline:
    """A frame pipeline (ladder_pipeline_create): submit(host_in, qp,
    host_out) uploads one packed frame, analyses every rung and reads the
    frame's packed decisions back, overlapped with its neighbours; wait(ticket)
    blocks until that frame's decisions are in its host_out."""

    def __init__(self, ladder, handle):
        self.ladder = ladder
        self.handle = handle
        self._ticket = ctypes.c_long()

    def submit(self, host_in, qp: int, host_out) -> int:
        """host_in / host_out: pinned CPU tensors (or raw addresses)."""
        src = host_in.data_ptr() if hasattr(host_in, "data_ptr") else int(host_in)
        dst = host_out.data_ptr() if hasattr(host_out, "data_ptr") else int(host_out)
        _call(self.ladder.handle, "ladder_pipeline_submit", self.handle, src, int(qp), dst,
              ctypes.byref(self._ticket))
        return self._ticket.value

    def wait(self, ticket: int):
        _call(self.ladder.handle, "ladder_pipeline_wait", self.handle, int(ticket))

    def close(self):
        if self.handle:
            load().ladder_pipeline_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A captured batch (ladder_capture_batch); launch() replays it."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def launch(self, stream=None):
        st = load().ladder_graph_launch(self.handle, _stream_handle(stream))
        if st != 0:
            raise LadderError(st, "ladder_graph_launch")

    def close(self):
        if self.handle:
            load().ladder_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ladder:
    """One ladder geometry (rungs, reference rung, search ranges) and its
    resident per-frame decision state on the device."""

    def __init__(self, rungs, ref_rung, *, bit_depth=8, ctu_size=64, search_range=32, refine_range=4,
                 depth_lo=0, depth_hi=1, use_ref_mv=1, satd_mode=0, max_frames=4, stream=None):
        self.rungs = [tuple(r) for r in rungs]
        self._rung_arr = (Rung * len(self.rungs))(*[Rung(w, h) for w, h in self.rungs])
        g = Geometry(len(self.rungs), self._rung_arr, ref_rung, bit_depth, ctu_size, search_range,
                     refine_range, depth_lo, depth_hi, use_ref_mv, satd_mode, max_frames)
        self.geometry = g
        self.ref_rung = ref_rung
        self.bit_depth = bit_depth
        self.ctu_size = ctu_size
        self.handle = ladder_init(g, _stream_handle(stream))

    def close(self):
        if self.handle:
            ladder_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def analyze_reference(self, frame_id, cur, ref, qp, stream=None):
        analyze_reference(self.handle, frame_id, cur.data_ptr(), ref.data_ptr(), _pitch_bytes(cur), qp,
                          _stream_handle(stream))

    def analyze_dependent(self, rung, frame_id, cur, ref, qp, stream=None):
        analyze_dependent(self.handle, rung, frame_id, cur.data_ptr(), ref.data_ptr(), _pitch_bytes(cur), qp,
                          _stream_handle(stream))

    def analyze_dependents(self, frame_id, items, qp, stream=None):
        """items: [(rung, cur, ref), ...] analysed by one launch."""
        analyze_dependents(self.handle, frame_id, [r for r, _, _ in items], [c.data_ptr() for _, c, _ in items],
                           [f.data_ptr() for _, _, f in items], [_pitch_bytes(c) for _, c, _ in items], qp,
                           _stream_handle(stream))

    def analyze_independent(self, rung, frame_id, cur, ref, qp, stream=None):
        analyze_independent(self.handle, rung, frame_id, cur.data_ptr(), ref.data_ptr(), _pitch_bytes(cur), qp,
                            _stream_handle(stream))

    def _requests(self, items):
        """items: [(frame_id, qp, [(cur, ref), ...] per rung)] -> ctypes array (kept alive on self)."""
        reqs = (Request * len(items))()
        keep = []
        for k, (fid, qp, planes) in enumerate(items):
            n = len(planes)
            cur = (ctypes.c_void_p * n)(*[c.data_ptr() for c, _ in planes])
            ref = (ctypes.c_void_p * n)(*[f.data_ptr() for _, f in planes])
            pit = (ctypes.c_long * n)(*[_pitch_bytes(c) for c, _ in planes])
            keep += [cur, ref, pit]
            reqs[k] = Request(fid, qp, cur, ref, pit)
        self._keep_requests = (reqs, keep)
        return reqs

    def analyze_batch(self, items, stream=None):
        """Many ladder frames in one batch: items = [(frame_id, qp, planes)],
        planes = [(cur, ref)] for every rung in rung order."""
        reqs = self._requests(items)
        _call(self.handle, "ladder_analyze_batch", self.handle, reqs, len(items), _stream_handle(stream))

    def analyze_jobs(self, jobs, stream=None):
        """jobs: [(frame_id, rung, kind, qp, cur, ref)], kind 0 = independent,
        1 = dependent; one call, batched launches."""
        arr = (Job * len(jobs))(*[Job(f, r, k, q, c.data_ptr(), x.data_ptr(), _pitch_bytes(c))
                                  for (f, r, k, q, c, x) in jobs])
        _call(self.handle, "ladder_analyze_jobs", self.handle, arr, len(jobs), _stream_handle(stream))

    def analyze_batch_independent(self, items, stream=None):
        """Every rung of every item analysed independently (full search)."""
        reqs = self._requests(items)
        _call(self.handle, "ladder_analyze_batch_independent", self.handle, reqs, len(items), _stream_handle(stream))

    def capture_batch(self, items, stream):
        """Captures analyze_batch(items) into a CUDA graph on `stream`."""
        reqs = self._requests(items)
        g = ctypes.c_void_p()
        _call(self.handle, "ladder_capture_batch", self.handle, reqs, len(items), _stream_handle(stream),
              ctypes.byref(g))
        return Graph(g.value, (reqs, self._keep_requests))

    def set_tuning(self, **knobs):
        """Kernel shapes, e.g. set_tuning(fs_band=9, dep_range=32); results
        are identical for every setting."""
        for name, value in knobs.items():
            _call(self.handle, "ladder_set_tuning", self.handle, TUNE_KNOBS[name], int(value))

    def set_debug(self, **controls):
        """Test controls of the failure paths, e.g. set_debug(wait_polls=4096,
        lost_handoff=1) makes the wavefront waits run out (include/ladder.h)."""
        for name, value in controls.items():
            _call(self.handle, "ladder_set_debug", self.handle, DEBUG_CONTROLS[name], int(value))

    def tuning(self) -> dict:
        out = {}
        for name, k in TUNE_KNOBS.items():
            v = ctypes.c_int()
            _call(self.handle, "ladder_get_tuning", self.handle, k, ctypes.byref(v))
            out[name] = v.value
        return out

    def dependent_evals(self, stream=None) -> int:
        """SAD-candidate evaluations the dependent searches made since the
        previous call (CUs summed from their sub-CUs not counted); resets
        the count."""
        v = ctypes.c_ulonglong()
        _call(self.handle, "ladder_dependent_evals", self.handle, _stream_handle(stream), ctypes.byref(v))
        return int(v.value)

    def device_bytes(self) -> int:
        return int(load().ladder_device_bytes(self.handle))

    def grid(self, rung):
        return ladder_grid(self.handle, rung)

    def sync(self, stream=None):
        ladder_sync(self.handle, _stream_handle(stream))

    def release_frame(self, frame_id):
        ladder_release_frame(self.handle, frame_id)

    def profile(self, enable: bool = True):
        ladder_profile_enable(self.handle, enable)

    def kernel_stats(self, reset: bool = False) -> dict:
        """{kind: (launches, summed event ms)} since the last reset."""
        return {name: ladder_profile_read(self.handle, k, reset) for k, name in enumerate(KERNEL_KINDS)}

    def set_parents(self, parent):
        """parent[r]: the rung whose decisions rung r refines (-1 for the
        reference rung); a cascaded chain analyses tier by tier."""
        arr = (ctypes.c_int * len(self.rungs))(*parent)
        _call(self.handle, "ladder_set_parents", self.handle, arr)
        self.parent = list(parent)

    def pipeline(self, depth: int, base_frame_id: int, in_bytes: int, cur_off, ref_off, pitch) -> "Pipeline":
        """Frame pipeline over frame ids base_frame_id .. + depth - 1; the
        packed input holds rung r's planes at cur_off[r] / ref_off[r] with
        row pitch pitch[r] bytes."""
        n = len(self.rungs)
        arr = lambda v: (ctypes.c_long * n)(*[int(x) for x in v])
        h = ctypes.c_void_p()
        _call(self.handle, "ladder_pipeline_create", self.handle, int(depth), int(base_frame_id), int(in_bytes),
              arr(cur_off), arr(ref_off), arr(pitch), ctypes.byref(h))
        return Pipeline(self, h.value)

    def set_mv_predictor(self, mode: int):
        """0: predictor (0, 0); 1: spatial predictor, CTUs decided in
        wavefront order (later analyses)."""
        _call(self.handle, "ladder_set_mv_predictor", self.handle, int(mode))
        self.mv_predictor = int(mode)

    def decide_qps(self, rung, frame_id, qps, stream=None) -> dict:
        """Cost, best, split and leaf maps of (rung, frame) at each QP of
        `qps` from the resident analysis (intra-resolution multi-QP sharing),
        as {qp: {field: numpy arrays laid out like fetch()}}."""
        import torch

        dims, (c8, r8) = self.grid(rung)
        dev = torch.device("cuda", torch.cuda.current_device())
        tensors, outs = [], []
        for _ in qps:
            t = {"cost": [], "best": [], "split": []}
            o = QpDecisions()
            for d, (c, r) in enumerate(dims):
                for k, dt in (("cost", torch.int32), ("best", torch.int32), ("split", torch.uint8)):
                    a = torch.empty(c * r, dtype=dt, device=dev)
                    t[k].append(a)
                    getattr(o, k)[d] = a.data_ptr()
            for k, dt in (("leaf_depth", torch.uint8), ("leaf_mvx", torch.int16), ("leaf_mvy", torch.int16)):
                a = torch.empty(c8 * r8, dtype=dt, device=dev)
                t[k] = a
                setattr(o, k, a.data_ptr())
            tensors.append(t)
            outs.append(o)
        s = _stream_handle(stream)
        ladder_decide_qps(self.handle, rung, frame_id, list(qps), outs, s)
        if stream is None:
            torch.cuda.current_stream().synchronize()
        else:
            stream.synchronize()
        res = {}
        for q, t in zip(qps, tensors):
            res[q] = {k: ([a.cpu().numpy() for a in v] if isinstance(v, list) else v.cpu().numpy()) for k, v in t.items()}
        return res

    def subpel_buffers(self, rung):
        """Device arrays for ladder_refine_subpel of `rung`: (tensors dict,
        SubpelDecisions struct pointing at them, interpolation workspace)."""
        import torch

        dims, (c8, r8) = self.grid(rung)
        dev = torch.device("cuda", torch.cuda.current_device())
        t = {k: [] for k in ("qmvx", "qmvy", "satd", "cost", "best", "split")}
        o = SubpelDecisions()
        for d, (c, r) in enumerate(dims):
            for k, dt in (("qmvx", torch.int16), ("qmvy", torch.int16), ("satd", torch.int32),
                          ("cost", torch.int32), ("best", torch.int32), ("split", torch.uint8)):
                a = torch.empty(c * r, dtype=dt, device=dev)
                t[k].append(a)
                getattr(o, k)[d] = a.data_ptr()
        for k, dt in (("leaf_depth", torch.uint8), ("leaf_qmvx", torch.int16), ("leaf_qmvy", torch.int16)):
            a = torch.empty(c8 * r8, dtype=dt, device=dev)
            t[k] = a
            setattr(o, k, a.data_ptr())
        ws = torch.empty(int(load().ladder_subpel_workspace_bytes(self.handle, rung)), dtype=torch.uint8, device=dev)
        return t, o, ws

    def refine_subpel(self, rung, frame_id, cur, ref, qp, stream=None, buffers=None) -> dict:
        """Quarter-pel refinement of an analysed (rung, frame): returns the
        refined arrays as numpy (qmvx / qmvy in quarter-pel units) after
        waiting for the stream; `buffers` = subpel_buffers(rung) to reuse."""
        import torch

        t, o, ws = buffers if buffers is not None else self.subpel_buffers(rung)
        s = _stream_handle(stream)
        _call(self.handle, "ladder_refine_subpel", self.handle, rung, frame_id, cur.data_ptr(), ref.data_ptr(),
              _pitch_bytes(cur), qp, ctypes.byref(o), ws.data_ptr(), ws.numel(), s)
        (stream or torch.cuda.current_stream()).synchronize()
        out = {k: ([a.cpu().numpy() for a in v] if isinstance(v, list) else v.cpu().numpy()) for k, v in t.items()}
        out["grid"], out["grid8"] = self.grid(rung)
        return out

    def subpel_jobs(self, specs, buffers):
        """ctypes array of SubpelJob for ladder_refine_subpel_batch: specs =
        [(frame_id, rung, cur, ref, qp)], buffers[k] = subpel_buffers(rung)."""
        jobs = (SubpelJob * len(specs))()
        for k, ((frame_id, rung, cur, ref, qp), (_, o, ws)) in enumerate(zip(specs, buffers)):
            jobs[k] = SubpelJob(frame_id, rung, qp, cur.data_ptr(), ref.data_ptr(), _pitch_bytes(cur),
                                ctypes.pointer(o), ws.data_ptr(), ws.numel())
        return jobs

    def refine_subpel_batch(self, specs, stream=None, buffers=None) -> list:
        """Several refinements in one pair of launches: specs = [(frame_id,
        rung, cur, ref, qp)]; returns one dict per job as refine_subpel."""
        import torch

        buffers = buffers if buffers is not None else [self.subpel_buffers(sp[1]) for sp in specs]
        jobs = self.subpel_jobs(specs, buffers)
        _call(self.handle, "ladder_refine_subpel_batch", self.handle, len(specs), jobs, _stream_handle(stream))
        (stream or torch.cuda.current_stream()).synchronize()
        res = []
        for (frame_id, rung, *_), (t, _, _) in zip(specs, buffers):
            out = {k: ([a.cpu().numpy() for a in v] if isinstance(v, list) else v.cpu().numpy()) for k, v in t.items()}
            out["grid"], out["grid8"] = self.grid(rung)
            res.append(out)
        return res

    def frame_bytes(self) -> int:
        """Bytes of one frame's packed decisions (every rung)."""
        return int(load().ladder_frame_bytes(self.handle))

    def frame_views(self, buf) -> list:
        """numpy views, per rung, into a packed frame `buf` (a uint8 numpy
        array of frame_bytes() bytes), laid out like fetch()."""
        out = []
        for r in range(len(self.rungs)):
            offs = (ctypes.c_long * 35)()
            _call(self.handle, "ladder_decision_offsets", self.handle, r, offs)
            dims, (c8, r8) = self.grid(r)
            v = {k: [] for k in ("mvx", "mvy", "sad", "satd", "cost", "best", "split", "evaluated")}
            for d, (c, rr) in enumerate(dims):
                n = c * rr
                for k, (name, dt) in enumerate((("mvx", np.int16), ("mvy", np.int16), ("sad", np.int32),
                                                 ("satd", np.int32), ("cost", np.int32), ("best", np.int32),
                                                 ("split", np.uint8), ("evaluated", np.uint8))):
                    o = offs[8 * d + k]
                    v[name].append(buf[o:o + n * np.dtype(dt).itemsize].view(dt))
            for k, (name, dt) in enumerate((("leaf_depth", np.uint8), ("leaf_mvx", np.int16), ("leaf_mvy", np.int16))):
                o = offs[32 + k]
                v[name] = buf[o:o + c8 * r8 * np.dtype(dt).itemsize].view(dt)
            v["grid"] = dims
            v["grid8"] = (c8, r8)
            v["size"] = self.rungs[r]
            out.append(v)
        return out

    def fetch_frame_async(self, frame_id, host, stream=None):
        """Enqueues the copy of every rung's decisions of `frame_id` into
        `host` (a pinned uint8 tensor of frame_bytes() bytes) on `stream`;
        does not wait."""
        _call(self.handle, "ladder_fetch_frame_async", self.handle, frame_id, host.data_ptr(), host.numel(),
              _stream_handle(stream))

    def load_reference(self, frame_id, saved: dict, stream=None):
        """Makes a reference analysis saved by fetch() (the reference rung's
        arrays) the resident reference of frame_id (ladder_load_reference)."""
        dims, (c8, r8) = self.grid(self.ref_rung)
        dec = Decisions()
        keep = []
        for d in range(len(dims)):
            for k, dt in (("mvx", np.int16), ("mvy", np.int16), ("sad", np.int32), ("satd", np.int32),
                          ("cost", np.int32), ("best", np.int32), ("split", np.uint8), ("evaluated", np.uint8)):
                a = np.ascontiguousarray(saved[k][d], dtype=dt)
                if a.size != dims[d][0] * dims[d][1]:
                    raise ValueError(f"{k}[{d}] has {a.size} entries, the grid {dims[d]}")
                keep.append(a)
                getattr(dec, k)[d] = a.ctypes.data
        for k, dt in (("leaf_depth", np.uint8), ("leaf_mvx", np.int16), ("leaf_mvy", np.int16)):
            a = np.ascontiguousarray(saved[k], dtype=dt)
            if a.size != c8 * r8:
                raise ValueError(f"{k} has {a.size} entries, the 8x8 grid {c8}x{r8}")
            keep.append(a)
            setattr(dec, k, a.ctypes.data)
        _call(self.handle, "ladder_load_reference", self.handle, int(frame_id), ctypes.byref(dec),
              _stream_handle(stream))

    def fetch(self, rung, frame_id, stream=None) -> dict:
        """Decisions of (rung, frame) as numpy arrays, laid out like the
        oracle's output (per-depth lists in CU raster order + per-8x8 maps)."""
        dims, (c8, r8) = self.grid(rung)
        out = {k: [] for k in ("mvx", "mvy", "sad", "satd", "cost", "best", "split", "evaluated")}
        dec = Decisions()
        for d, (c, r) in enumerate(dims):
            n = c * r
            for k, dt in (("mvx", np.int16), ("mvy", np.int16), ("sad", np.int32), ("satd", np.int32),
                          ("cost", np.int32), ("best", np.int32), ("split", np.uint8), ("evaluated", np.uint8)):
                a = np.zeros(n, dtype=dt)
                out[k].append(a)
                getattr(dec, k)[d] = a.ctypes.data
        for k, dt in (("leaf_depth", np.uint8), ("leaf_mvx", np.int16), ("leaf_mvy", np.int16)):
            a = np.zeros(c8 * r8, dtype=dt)
            out[k] = a
            setattr(dec, k, a.ctypes.data)
        fetch_decisions(self.handle, rung, frame_id, dec, _stream_handle(stream))
        out["grid"] = dims
        out["grid8"] = (c8, r8)
        out["size"] = self.rungs[rung]
        return out
