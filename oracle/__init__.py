"""CPU oracle for the per-CTU inter analysis (ctypes over ``ladder_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline / reference legs may import this package.  It shares no
code with the CUDA library and never imports it.

The C source computes the plain definitions (per-CU exhaustive search at every
depth, explicit Hadamard products, explicit quadtree recursion); this module
only marshals numpy arrays.  Parity of every function here is pinned by the
``-m "not gpu"`` tests (brute force, closed forms, invariants, planted motion,
exhaustive quadtree enumeration).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ladder_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXD = 4


class _Decisions(ctypes.Structure):
    _fields_ = [
        ("mvx", ctypes.c_void_p * MAXD), ("mvy", ctypes.c_void_p * MAXD),
        ("sad", ctypes.c_void_p * MAXD), ("satd", ctypes.c_void_p * MAXD),
        ("cost", ctypes.c_void_p * MAXD), ("best", ctypes.c_void_p * MAXD),
        ("split", ctypes.c_void_p * MAXD), ("evaluated", ctypes.c_void_p * MAXD),
        ("leaf_depth", ctypes.c_void_p), ("leaf_mvx", ctypes.c_void_p),
        ("leaf_mvy", ctypes.c_void_p),
    ]


class _Subpel(ctypes.Structure):
    _fields_ = [
        ("qmvx", ctypes.c_void_p * MAXD), ("qmvy", ctypes.c_void_p * MAXD),
        ("satd", ctypes.c_void_p * MAXD), ("cost", ctypes.c_void_p * MAXD),
        ("best", ctypes.c_void_p * MAXD), ("split", ctypes.c_void_p * MAXD),
        ("leaf_depth", ctypes.c_void_p), ("leaf_qmvx", ctypes.c_void_p),
        ("leaf_qmvy", ctypes.c_void_p),
    ]


class _Job(ctypes.Structure):
    _fields_ = [
        ("cur", ctypes.c_void_p), ("ref", ctypes.c_void_p),
        ("width", ctypes.c_int), ("height", ctypes.c_int), ("pitch", ctypes.c_long),
        ("bit_depth", ctypes.c_int), ("ctu", ctypes.c_int), ("qp", ctypes.c_int),
        ("satd_mode", ctypes.c_int), ("range", ctypes.c_int), ("dep", ctypes.c_int),
        ("ref_width", ctypes.c_int), ("ref_height", ctypes.c_int),
        ("ref_leaf_depth", ctypes.c_void_p), ("ref_leaf_mvx", ctypes.c_void_p),
        ("ref_leaf_mvy", ctypes.c_void_p),
        ("depth_lo", ctypes.c_int), ("depth_hi", ctypes.c_int), ("use_ref_mv", ctypes.c_int),
        ("ctu_mask", ctypes.c_void_p), ("mvp", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with the host C compiler (plain -O2, no SIMD flags)."""
    with _lock:
        fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
        if force or not fresh:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                                   "-lpthread", "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_analyze.argtypes = [ctypes.POINTER(_Job), ctypes.POINTER(_Decisions), ctypes.c_int]
        lib.oracle_analyze.restype = ctypes.c_int
        lib.oracle_satd8_had8.argtypes = [ctypes.c_void_p]
        lib.oracle_satd8_had8.restype = ctypes.c_int
        lib.oracle_satd8_paper4x4.argtypes = [ctypes.c_void_p]
        lib.oracle_satd8_paper4x4.restype = ctypes.c_int
        lib.oracle_se_bits.argtypes = [ctypes.c_int]
        lib.oracle_se_bits.restype = ctypes.c_int
        lib.oracle_mv_bits.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.oracle_mv_bits.restype = ctypes.c_int
        lib.oracle_lambda_q16.argtypes = [ctypes.c_int]
        lib.oracle_lambda_q16.restype = ctypes.c_longlong
        for name in ("oracle_block_sad", "oracle_block_satd"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.POINTER(_Job)] + [ctypes.c_int] * 5
            fn.restype = ctypes.c_int32
        lib.oracle_derive_rule.argtypes = [ctypes.POINTER(_Job)] + [ctypes.c_int] * 3 + [ctypes.c_void_p]
        lib.oracle_derive_rule.restype = None
        lib.oracle_refine_subpel.argtypes = [ctypes.POINTER(_Job), ctypes.POINTER(_Decisions),
                                             ctypes.POINTER(_Subpel), ctypes.c_int]
        lib.oracle_refine_subpel.restype = ctypes.c_int
        lib.oracle_pred_sample.argtypes = [ctypes.POINTER(_Job)] + [ctypes.c_int] * 4
        lib.oracle_pred_sample.restype = ctypes.c_int
        lib.oracle_block_satd_q.argtypes = [ctypes.POINTER(_Job)] + [ctypes.c_int] * 5
        lib.oracle_block_satd_q.restype = ctypes.c_int32
        lib.oracle_spatial_mvp.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 2 + [ctypes.c_int] * 3 + [
            ctypes.POINTER(ctypes.c_int)]
        lib.oracle_spatial_mvp.restype = None
        _lib = lib
    return _lib


def grid(width: int, height: int, ctu: int = 64):
    """Per-depth CU grid (cols, rows) and the 8x8 grid of a frame."""
    W8, H8 = (width + 7) // 8 * 8, (height + 7) // 8 * 8
    dmax = int(np.log2(ctu // 8))
    dims = []
    for d in range(dmax + 1):
        S = ctu >> d
        dims.append(((W8 + S - 1) // S, (H8 + S - 1) // S))
    return dims, (W8 // 8, H8 // 8)


def _make_job(cur, ref, qp, ctu, search_range, satd_mode, dep):
    cur = np.ascontiguousarray(cur)
    ref = np.ascontiguousarray(ref)
    if cur.shape != ref.shape or cur.dtype != ref.dtype:
        raise ValueError("cur and ref must have the same shape and dtype")
    bit_depth = 8 if cur.dtype == np.uint8 else 10
    if cur.dtype not in (np.uint8, np.uint16):
        raise ValueError("planes must be uint8 (8-bit) or uint16 (10-bit)")
    H, W = cur.shape
    job = _Job()
    job.cur, job.ref = cur.ctypes.data, ref.ctypes.data
    job.width, job.height, job.pitch = W, H, W
    job.bit_depth, job.ctu, job.qp = bit_depth, ctu, qp
    job.satd_mode, job.range = satd_mode, search_range
    keep = [cur, ref]
    if dep is not None:
        job.dep = 1
        job.ref_width, job.ref_height = dep["ref_size"]
        ld = np.ascontiguousarray(dep["leaf_depth"], dtype=np.uint8)
        lx = np.ascontiguousarray(dep["leaf_mvx"], dtype=np.int16)
        ly = np.ascontiguousarray(dep["leaf_mvy"], dtype=np.int16)
        keep += [ld, lx, ly]
        job.ref_leaf_depth, job.ref_leaf_mvx, job.ref_leaf_mvy = (
            ld.ctypes.data, lx.ctypes.data, ly.ctypes.data)
        job.depth_lo = dep.get("depth_lo", 0)
        job.depth_hi = dep.get("depth_hi", 1)
        job.use_ref_mv = dep.get("use_ref_mv", 1)
    return job, keep


def analyze(cur, ref, *, qp: int, search_range: int, ctu: int = 64, satd_mode: int = 0,
            dep: dict | None = None, threads: int | None = None, ctu_mask=None, mvp: int = 0) -> dict:
    """Analyse one frame pair.

    ``dep`` (dependent mode) holds ``ref_size=(Wr, Hr)`` and the reference
    rung's per-8x8 ``leaf_depth``, ``leaf_mvx``, ``leaf_mvy`` plus optional
    ``depth_lo``, ``depth_hi``, ``use_ref_mv``; ``search_range`` is then the
    refinement range r around the centre.  ``mvp=1`` takes the rate term's
    predictor from the spatial neighbours (CTUs decided in raster order).
    Returns per-depth lists ``mvx, mvy, sad, satd, cost, best, split,
    evaluated`` (CU raster order) and per-8x8 ``leaf_depth, leaf_mvx, leaf_mvy``.
    """
    lib = _load()
    job, keep = _make_job(cur, ref, qp, ctu, search_range, satd_mode, dep)
    dims, (c8, r8) = grid(job.width, job.height, ctu)
    job.mvp = int(mvp)
    if ctu_mask is not None:
        m = np.ascontiguousarray(np.asarray(ctu_mask, dtype=np.uint8).reshape(-1))
        if m.size != dims[0][0] * dims[0][1]:
            raise ValueError("ctu_mask must have one entry per CTU")
        keep.append(m)
        job.ctu_mask = m.ctypes.data
    out = {k: [] for k in ("mvx", "mvy", "sad", "satd", "cost", "best", "split", "evaluated")}
    dec = _Decisions()
    for d, (c, r) in enumerate(dims):
        n = c * r
        for k, dt in (("mvx", np.int16), ("mvy", np.int16), ("sad", np.int32), ("satd", np.int32),
                      ("cost", np.int32), ("best", np.int32), ("split", np.uint8),
                      ("evaluated", np.uint8)):
            a = np.zeros(n, dtype=dt)
            out[k].append(a)
            getattr(dec, k)[d] = a.ctypes.data
    out["leaf_depth"] = np.zeros(c8 * r8, dtype=np.uint8)
    out["leaf_mvx"] = np.zeros(c8 * r8, dtype=np.int16)
    out["leaf_mvy"] = np.zeros(c8 * r8, dtype=np.int16)
    dec.leaf_depth = out["leaf_depth"].ctypes.data
    dec.leaf_mvx = out["leaf_mvx"].ctypes.data
    dec.leaf_mvy = out["leaf_mvy"].ctypes.data
    if threads is None:
        threads = os.cpu_count() or 1
    rc = lib.oracle_analyze(ctypes.byref(job), ctypes.byref(dec), int(threads))
    del keep
    if rc != 0:
        raise ValueError("oracle_analyze rejected its arguments")
    out["grid"] = dims
    out["grid8"] = (c8, r8)
    out["size"] = (job.width, job.height)
    return out


def satd8(block, mode: int = 0) -> int:
    """SATD of one 8x8 residual block (mode 0: HAD8, 1: PAPER4x4)."""
    d = np.ascontiguousarray(np.asarray(block, dtype=np.int32).reshape(64))
    lib = _load()
    fn = lib.oracle_satd8_paper4x4 if mode == 1 else lib.oracle_satd8_had8
    return int(fn(d.ctypes.data))


def se_bits(v: int) -> int:
    return int(_load().oracle_se_bits(int(v)))


def mv_bits(mvx: int, mvy: int) -> int:
    return int(_load().oracle_mv_bits(int(mvx), int(mvy)))


def lambda_q16(qp: int) -> int:
    return int(_load().oracle_lambda_q16(int(qp)))


def block_sad(cur, ref, x0, y0, size, mvx, mvy) -> int:
    job, keep = _make_job(cur, ref, 0, 64, 0, 0, None)
    r = int(_load().oracle_block_sad(ctypes.byref(job), x0, y0, size, mvx, mvy))
    del keep
    return r


def block_satd(cur, ref, x0, y0, size, mvx, mvy, satd_mode: int = 0) -> int:
    job, keep = _make_job(cur, ref, 0, 64, 0, satd_mode, None)
    r = int(_load().oracle_block_satd(ctypes.byref(job), x0, y0, size, mvx, mvy))
    del keep
    return r


_dummies: dict = {}


def derive_rule(dep_size, dep: dict, d: int, x0: int, y0: int, ctu: int = 64):
    """Dependent-mode rule of CU (d, x0, y0): (cx, cy, allowed_leaf, allowed_split)."""
    W, H = dep_size
    dummy = _dummies.get((W, H))
    if dummy is None:  # a placeholder frame of the rung's size (the rule reads no samples)
        dummy = _dummies.setdefault((W, H), np.zeros((H, W), dtype=np.uint8))
    job, keep = _make_job(dummy, dummy, 0, ctu, 0, 0, dep)
    out = np.zeros(4, dtype=np.int32)
    _load().oracle_derive_rule(ctypes.byref(job), d, x0, y0, out.ctypes.data)
    del keep
    return tuple(int(v) for v in out)


def refine_subpel(cur, ref, analysis: dict, *, qp: int, ctu: int = 64, satd_mode: int = 0,
                  dep: dict | None = None, threads: int | None = None, mvp: int = 0) -> dict:
    """Quarter-pel refinement of an analysis of the same frame pair (as
    returned by analyze() with the same qp / ctu / satd_mode / dep / mvp):
    per depth ``qmvx, qmvy`` (quarter-pel units), ``satd``, ``cost``,
    ``best``, ``split``, and per 8x8 ``leaf_depth, leaf_qmvx, leaf_qmvy``.
    ``mvp=1``: the rate term of every candidate takes the spatial predictor
    formed from the refined quarter-pel leaf vectors of the earlier CTUs."""
    lib = _load()
    job, keep = _make_job(cur, ref, qp, ctu, 0, satd_mode, dep)
    job.mvp = int(mvp)
    dims, (c8, r8) = grid(job.width, job.height, ctu)
    dec = _Decisions()
    for d in range(len(dims)):
        for k in ("mvx", "mvy", "sad", "satd", "cost", "best", "split", "evaluated"):
            a = np.ascontiguousarray(analysis[k][d])
            keep.append(a)
            getattr(dec, k)[d] = a.ctypes.data
    for k in ("leaf_depth", "leaf_mvx", "leaf_mvy"):
        a = np.ascontiguousarray(analysis[k])
        keep.append(a)
        setattr(dec, k, a.ctypes.data)
    out = {k: [] for k in ("qmvx", "qmvy", "satd", "cost", "best", "split")}
    sp = _Subpel()
    for d, (c, r) in enumerate(dims):
        for k, dt in (("qmvx", np.int16), ("qmvy", np.int16), ("satd", np.int32), ("cost", np.int32),
                      ("best", np.int32), ("split", np.uint8)):
            a = np.zeros(c * r, dtype=dt)
            out[k].append(a)
            getattr(sp, k)[d] = a.ctypes.data
    for k, dt in (("leaf_depth", np.uint8), ("leaf_qmvx", np.int16), ("leaf_qmvy", np.int16)):
        a = np.zeros(c8 * r8, dtype=dt)
        out[k] = a
        setattr(sp, k, a.ctypes.data)
    if threads is None:
        threads = os.cpu_count() or 1
    rc = lib.oracle_refine_subpel(ctypes.byref(job), ctypes.byref(dec), ctypes.byref(sp), int(threads))
    del keep
    if rc != 0:
        raise ValueError("oracle_refine_subpel rejected its arguments")
    out["grid"] = dims
    out["grid8"] = (c8, r8)
    return out


def spatial_mvp(width: int, height: int, ctu: int, leaf_mvx, leaf_mvy, x0: int, y0: int, size: int):
    """Spatial predictor (pmx, pmy) of the CU (size at x0, y0) over the given
    per-8x8 leaf vectors of a width x height frame."""
    c8 = (width + 7) // 8
    r8 = (height + 7) // 8
    mx = np.ascontiguousarray(np.asarray(leaf_mvx, dtype=np.int16).reshape(-1))
    my = np.ascontiguousarray(np.asarray(leaf_mvy, dtype=np.int16).reshape(-1))
    if mx.size != c8 * r8 or my.size != c8 * r8:
        raise ValueError("leaf maps must have one entry per 8x8 block")
    out = (ctypes.c_int * 2)()
    _load().oracle_spatial_mvp(width, height, ctu, mx.ctypes.data, my.ctypes.data, x0, y0, size, out)
    return int(out[0]), int(out[1])


def pred_sample(ref, x: int, y: int, qx: int, qy: int) -> int:
    """Quarter-pel prediction of sample (x, y) displaced by (qx, qy) quarter units."""
    job, keep = _make_job(ref, ref, 0, 64, 0, 0, None)
    r = int(_load().oracle_pred_sample(ctypes.byref(job), x, y, qx, qy))
    del keep
    return r


def block_satd_q(cur, ref, x0, y0, size, qx, qy, satd_mode: int = 0) -> int:
    """SATD of a size x size block against the quarter-pel prediction."""
    job, keep = _make_job(cur, ref, 0, 64, 0, satd_mode, None)
    r = int(_load().oracle_block_satd_q(ctypes.byref(job), x0, y0, size, qx, qy))
    del keep
    return r
