"""Seeded synthetic luma planes shaped like the paper's test content.

The paper measures on three natural 50 fps sequences (Sec. 4.1) that are not
available here; these generators stand in for them.  This module only makes
inputs: it holds none of the analysis arithmetic (no SAD, SATD, cost or
split), so both the CUDA path and the CPU oracle can consume its planes.

Recipe (every draw from ``numpy.random.Generator(PCG64(seed))``):

* texture: ``offset + sum_k A_k sin(2 pi (fx_k x + fy_k y) + phi_k)`` over six
  sinusoids, ``A_k ~ U[8, 24]`` (x4 for 10-bit), periods ``~ U[8, 64]`` px
  times ``motion_scale``, random orientation and phase; plus Gaussian noise
  (sigma 4 for 8-bit, 8 for 10-bit); rounded and clipped to the sample range;
* current frame: the reference displaced by a global integer motion, then
  ``n_patches`` square patches each displaced by its own integer motion
  (``cur(p) = ref(p + mv)`` with clamped reads), plus Gaussian noise;
* ladder rungs: every rung is made from the source pair directly with a
  fixed separable 2-tap bilinear filter in Q16 fixed point, rounded half up.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = ["FramePair", "frame_pair", "sequence", "downscale", "ladder_pairs", "ladder_sequence", "RUNGS"]

RUNGS = {
    "2160p": (3840, 2160),
    "1440p": (2560, 1440),
    "1080p": (1920, 1080),
    "720p": (1280, 720),
    "540p": (960, 540),
    "360p": (640, 360),
    "240p": (416, 240),
}


@dataclasses.dataclass
class FramePair:
    cur: np.ndarray          # (H, W) uint8 or uint16
    ref: np.ndarray
    bit_depth: int
    global_mv: tuple[int, int]
    patches: list            # [(x, y, size, (mvx, mvy)), ...]

    @property
    def width(self) -> int:
        return int(self.cur.shape[1])

    @property
    def height(self) -> int:
        return int(self.cur.shape[0])


def _dtype(bit_depth: int):
    if bit_depth == 8:
        return np.uint8
    if bit_depth == 10:
        return np.uint16
    raise ValueError("bit_depth must be 8 or 10")


def _texture(rng, W, H, bit_depth, period_scale, noise_sigma):
    amp_scale = 1 if bit_depth == 8 else 4
    offset = 128 if bit_depth == 8 else 512
    hi = (1 << bit_depth) - 1
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    base = np.full((H, W), float(offset))
    for _ in range(6):
        amp = rng.uniform(8.0, 24.0) * amp_scale
        period = rng.uniform(8.0, 64.0) * period_scale
        theta = rng.uniform(0.0, np.pi)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        fx, fy = np.cos(theta) / period, np.sin(theta) / period
        base += amp * np.sin(2.0 * np.pi * (fx * x + fy * y) + phi)
    base += rng.normal(0.0, noise_sigma, size=(H, W))
    return np.clip(np.rint(base), 0, hi)


def _displace(src, dst, x0, y0, w, h, mvx, mvy):
    """dst[y, x] = src[clamp(y + mvy), clamp(x + mvx)] over the given rectangle."""
    H, W = src.shape
    ys = np.clip(np.arange(y0, y0 + h) + mvy, 0, H - 1)
    xs = np.clip(np.arange(x0, x0 + w) + mvx, 0, W - 1)
    dst[y0:y0 + h, x0:x0 + w] = src[np.ix_(ys, xs)]


def frame_pair(seed: int, width: int, height: int, bit_depth: int = 8, *,
               global_range: int = 8, patch_range: int = 12, n_patches: int = 4,
               patch_size: int = 64, motion_scale: float = 1.0,
               texture_sigma: float | None = None, cur_sigma: float | None = None,
               global_mv: tuple[int, int] | None = None) -> FramePair:
    """One (current, reference) pair with planted motion.

    ``motion_scale`` multiplies the motion ranges, the patch size (rounded to a
    multiple of 8) and the texture periods, so content keeps its look when the
    frame grows.  ``global_mv`` pins the global motion instead of drawing it.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if texture_sigma is None:
        texture_sigma = 4.0 if bit_depth == 8 else 8.0
    if cur_sigma is None:
        cur_sigma = 2.0 if bit_depth == 8 else 8.0
    hi = (1 << bit_depth) - 1
    ref = _texture(rng, width, height, bit_depth, motion_scale, texture_sigma)
    g = int(round(global_range * motion_scale))
    p = int(round(patch_range * motion_scale))
    size = max(8, int(round(patch_size * motion_scale / 8.0)) * 8)
    if global_mv is None:
        gmv = (int(rng.integers(-g, g + 1)), int(rng.integers(-g, g + 1)))
    else:
        gmv = (int(global_mv[0]), int(global_mv[1]))
    cur = np.empty_like(ref)
    _displace(ref, cur, 0, 0, width, height, gmv[0], gmv[1])
    patches = []
    for _ in range(n_patches):
        pw, ph = min(size, width), min(size, height)
        px = int(rng.integers(0, width - pw + 1))
        py = int(rng.integers(0, height - ph + 1))
        mv = (int(rng.integers(-p, p + 1)), int(rng.integers(-p, p + 1)))
        _displace(ref, cur, px, py, pw, ph, mv[0], mv[1])
        patches.append((px, py, pw, mv))
    if cur_sigma > 0:
        cur = cur + rng.normal(0.0, cur_sigma, size=cur.shape)
    cur = np.clip(np.rint(cur), 0, hi)
    dt = _dtype(bit_depth)
    return FramePair(cur=cur.astype(dt), ref=ref.astype(dt), bit_depth=bit_depth,
                     global_mv=gmv, patches=patches)


def sequence(seed: int, width: int, height: int, n_frames: int, bit_depth: int = 8, *, global_range: int = 16,
             patch_range: int = 24, n_patches: int = 4, patch_size: int = 64, period_scale: float = 1.0,
             noise_sigma: float = 4.0):
    """Consecutive frames: frame t+1 is frame t moved by a fresh global integer
    motion (uniform in +-global_range) with ``n_patches`` patches moved by
    their own motion (+-patch_range), plus Gaussian noise of ``noise_sigma``.
    Returns the list of frames and the per-step motions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hi = (1 << bit_depth) - 1
    frame = _texture(rng, width, height, bit_depth, period_scale, noise_sigma)
    frames, motions = [frame], []
    for _ in range(n_frames - 1):
        g = (int(rng.integers(-global_range, global_range + 1)), int(rng.integers(-global_range, global_range + 1)))
        nxt = np.empty_like(frame)
        _displace(frame, nxt, 0, 0, width, height, g[0], g[1])
        patches = []
        for _ in range(n_patches):
            pw, ph = min(patch_size, width), min(patch_size, height)
            px = int(rng.integers(0, width - pw + 1))
            py = int(rng.integers(0, height - ph + 1))
            mv = (int(rng.integers(-patch_range, patch_range + 1)), int(rng.integers(-patch_range, patch_range + 1)))
            _displace(frame, nxt, px, py, pw, ph, mv[0], mv[1])
            patches.append((px, py, pw, mv))
        if noise_sigma > 0:
            nxt = nxt + rng.normal(0.0, noise_sigma, size=nxt.shape)
        frame = np.clip(np.rint(nxt), 0, hi)
        frames.append(frame)
        motions.append((g, patches))
    dt = _dtype(bit_depth)
    return [f.astype(dt) for f in frames], motions


def ladder_sequence(seed: int, n_frames: int, source=(1920, 1080), rungs=((1920, 1080), (1280, 720), (960, 540),
                                                                         (640, 360)), bit_depth: int = 8, **kw):
    """A sequence at the source size and every rung made from each frame
    directly: returns ``[[plane of rung r for frame t] for r] ...`` as
    ``out[t][r]``."""
    W, H = source
    kw.setdefault("period_scale", W / 416.0)
    frames, _ = sequence(seed, W, H, n_frames, bit_depth, **kw)
    out = []
    for f in frames:
        out.append([f if (w, h) == (W, H) else downscale(f, w, h) for (w, h) in rungs])
    return out


def _taps(n_in: int, n_out: int):
    """Source taps and Q16 fraction of each output position.

    Position of output x in the source is (x + 0.5) * n_in / n_out - 0.5, in
    Q16: ((2x + 1) n_in - n_out) * 2^15 / n_out, clamped at 0.
    """
    x = np.arange(n_out, dtype=np.int64)
    pos = ((2 * x + 1) * n_in - n_out) * 32768 // n_out
    pos = np.maximum(pos, 0)
    p0 = pos >> 16
    frac = pos & 0xFFFF
    p1 = np.minimum(p0 + 1, n_in - 1)
    return p0, p1, frac


def downscale(plane: np.ndarray, width: int, height: int) -> np.ndarray:
    """Separable 2-tap bilinear resize in Q16, rounded half up at the end.

    The horizontal pass keeps its Q16 sums unrounded; the vertical pass takes
    them to Q32 and the result is ``(acc + 2^31) >> 32``.
    """
    src = plane.astype(np.int64)
    H, W = src.shape
    x0, x1, fx = _taps(W, width)
    y0, y1, fy = _taps(H, height)
    horiz = src[:, x0] * (65536 - fx) + src[:, x1] * fx               # Q16
    acc = horiz[y0, :] * (65536 - fy)[:, None] + horiz[y1, :] * fy[:, None]  # Q32
    out = (acc + (1 << 31)) >> 32
    return out.astype(plane.dtype)


def ladder_pairs(seed: int, source=(1920, 1080), rungs=((1280, 720), (960, 540), (640, 360)),
                 bit_depth: int = 8, include_source: bool = True, **kw):
    """Source pair plus every rung made from it directly (never cascaded).

    Motion, patch size and texture periods are scaled by source_width / 416.
    Returns ``[(width, height, cur, ref), ...]`` from the largest rung down.
    """
    W, H = source
    kw.setdefault("motion_scale", W / 416.0)
    src = frame_pair(seed, W, H, bit_depth, **kw)
    out = []
    if include_source:
        out.append((W, H, src.cur, src.ref))
    for (w, h) in rungs:
        out.append((w, h, downscale(src.cur, w, h), downscale(src.ref, w, h)))
    return out, src
