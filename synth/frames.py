"""Seeded synthetic video for the analyzer's tests and benchmark.

The paper measures on UHD 8-bit videos and the VCD dataset (Section 3); neither is
available here, so these frames stand in for them with the same shapes: planar
YUV 4:2:0, 8-bit samples in uint8 or 10-bit samples in 16-bit words.

Content model (one "scene" = one parameter draw; a scene cut draws a new one):

* luma = linear gradient + 3-6 windowed 2-D sinusoid patches (random period,
  orientation, phase, amplitude) + Gaussian noise redrawn every frame, rounded
  half-to-even and clipped to [16, 235];
* chroma = the same model drawn independently at half resolution, clipped to
  [16, 240];
* motion: every frame the scene is re-evaluated at integer offsets that follow a
  random walk (dx, dy uniform in [-m, m]) or a constant global pan;
* optional flat regions: block-aligned rectangles fixed on screen, filled with
  a constant and no noise (whole analyzer blocks in all three planes are flat);
* 10-bit / 12-bit: the 8-bit model scaled by 4 / 16 (noise sigma too), clipped to
  [64, 940] / [256, 3760];
* chroma format 4:2:0 (default: chroma planes of half width and height) or 4:4:4
  (full-size chroma planes, rendered at full resolution).

Everything is a pure function of the seed; the same call gives the same frames on
the same machine.  This module holds none of the analyzer's arithmetic.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LUMA_RANGE_8 = (16, 235)
CHROMA_RANGE_8 = (16, 240)


@dataclass(frozen=True)
class Patch:
    cx: float
    cy: float
    rx: float
    ry: float
    amp: float
    period: float
    theta: float
    phase: float


@dataclass(frozen=True)
class PlaneScene:
    base: float
    gx: float
    gy: float
    patches: tuple


@dataclass
class SequenceSpec:
    """Recipe of one synthetic sequence."""

    width: int
    height: int
    n_frames: int
    seed: int
    bit_depth: int = 8
    sigma: float | tuple = 4.0          # per-scene noise sigma (a tuple cycles per scene)
    cuts: tuple = ()                     # frame indices that start a new scene
    cut_every: int = 0                   # alternatively a cut every n frames (0 = none)
    motion: int = 4                      # random-walk step range [-motion, motion]
    pan: tuple | None = None             # (min, max) px/frame of a constant global pan instead
    periods: tuple = (2.0, 64.0)         # sinusoid period range (px, log-uniform)
    n_patches: tuple = (3, 6)
    flat_fraction: float = 0.0           # share of the area made of flat, noise-free blocks
    flat_align: int = 32                 # luma alignment of the flat rectangles
    chroma_format: str = "420"           # "420", "422" or "444"
    extra: dict = field(default_factory=dict)


def _draw_scene(rng: np.random.Generator, w: int, h: int, spec: SequenceSpec, chroma: bool) -> PlaneScene:
    lo_p, hi_p = spec.periods
    n = int(rng.integers(spec.n_patches[0], spec.n_patches[1] + 1))
    patches = []
    for _ in range(n):
        patches.append(Patch(
            cx=float(rng.uniform(0, w)), cy=float(rng.uniform(0, h)),
            rx=float(rng.uniform(w / 10, w / 4)), ry=float(rng.uniform(h / 10, h / 4)),
            amp=float(rng.uniform(15, 60)),
            period=float(math.exp(rng.uniform(math.log(lo_p), math.log(hi_p)))),
            theta=float(rng.uniform(0, math.pi)), phase=float(rng.uniform(0, 2 * math.pi))))
    base = float(rng.uniform(100, 156) if chroma else rng.uniform(60, 140))
    return PlaneScene(base=base, gx=float(rng.uniform(-40, 40)), gy=float(rng.uniform(-40, 40)),
                      patches=tuple(patches))


def _render(scene: PlaneScene, w: int, h: int, ox: float, oy: float) -> np.ndarray:
    """Noise-free scene evaluated at screen pixel (x, y) -> scene point (x + ox, y + oy)."""
    xs = (np.arange(w, dtype=np.float64) + ox)
    ys = (np.arange(h, dtype=np.float64) + oy)
    img = (scene.base + scene.gx * xs / w)[None, :] + (scene.gy * ys / h)[:, None]
    img = img.astype(np.float32)
    for p in scene.patches:
        x0 = max(0, int(math.floor(p.cx - p.rx - ox)))
        x1 = min(w, int(math.ceil(p.cx + p.rx - ox)) + 1)
        y0 = max(0, int(math.floor(p.cy - p.ry - oy)))
        y1 = min(h, int(math.ceil(p.cy + p.ry - oy)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        px = xs[x0:x1]
        py = ys[y0:y1]
        wx = 0.5 * (1 + np.cos(np.pi * np.clip(np.abs(px - p.cx) / p.rx, 0, 1)))
        wy = 0.5 * (1 + np.cos(np.pi * np.clip(np.abs(py - p.cy) / p.ry, 0, 1)))
        k = 2 * math.pi / p.period
        arg = (k * math.cos(p.theta)) * px[None, :] + (k * math.sin(p.theta)) * py[:, None] + p.phase
        img[y0:y1, x0:x1] += (p.amp * wy[:, None] * wx[None, :] * np.sin(arg)).astype(np.float32)
    return img


def _flat_mask(rng: np.random.Generator, width: int, height: int, spec: SequenceSpec):
    """Block-aligned flat rectangles on the luma grid: list of (x0, y0, x1, y1, level)."""
    a = spec.flat_align
    nbx, nby = width // a, height // a
    target = spec.flat_fraction * nbx * nby
    covered = np.zeros((nby, nbx), dtype=bool)
    rects = []
    tries = 0
    while covered.sum() < target and tries < 10000:
        tries += 1
        bw = int(rng.integers(2, max(3, nbx // 4)))
        bh = int(rng.integers(2, max(3, nby // 4)))
        bx = int(rng.integers(0, max(1, nbx - bw)))
        by = int(rng.integers(0, max(1, nby - bh)))
        need = target - covered.sum()
        if bw * bh > need:  # shrink the last rectangle towards the exact target
            bh = max(1, min(bh, int(need // max(bw, 1)) or 1))
        covered[by:by + bh, bx:bx + bw] = True
        rects.append((bx * a, by * a, (bx + bw) * a, (by + bh) * a, float(rng.uniform(40, 200))))
    return rects


def _quantize(img: np.ndarray, lo: int, hi: int, scale: int, dtype) -> np.ndarray:
    return np.clip(np.rint(img * scale), lo * scale, hi * scale).astype(dtype)


def _sigma_for_scene(spec: SequenceSpec, scene_idx: int) -> float:
    if isinstance(spec.sigma, (tuple, list)):
        return float(spec.sigma[scene_idx % len(spec.sigma)])
    return float(spec.sigma)


def generate(spec: SequenceSpec, start: int = 0, stop: int | None = None):
    """Yield (y, u, v) numpy planes for frames [start, stop) of the sequence.

    8-bit planes are uint8; 10-bit planes are uint16.  Frames before ``start`` are
    not rendered, but their random draws are replayed so any window of the
    sequence is the same as in a full pass.
    """
    stop = spec.n_frames if stop is None else min(stop, spec.n_frames)
    W, H = spec.width, spec.height
    if spec.chroma_format == "444":
        cw, ch = W, H
    elif spec.chroma_format == "422":
        cw, ch = (W + 1) // 2, H
    else:
        cw, ch = (W + 1) // 2, (H + 1) // 2
    scale = 1 << (spec.bit_depth - 8)
    dtype = np.uint16 if spec.bit_depth > 8 else np.uint8
    cuts = set(spec.cuts)
    if spec.cut_every:
        cuts |= set(range(spec.cut_every, spec.n_frames, spec.cut_every))
    master = np.random.Generator(np.random.PCG64(spec.seed))
    motion_rng = np.random.Generator(np.random.PCG64(spec.seed + 7919))
    scene_idx = -1
    ox = oy = 0.0
    pan = (0.0, 0.0)
    rects = []
    scenes = None
    for t in range(stop):
        if t == 0 or t in cuts:
            scene_idx += 1
            srng = np.random.Generator(np.random.PCG64([spec.seed, scene_idx]))
            scenes = (_draw_scene(srng, W, H, spec, False),
                      _draw_scene(srng, cw, ch, spec, True),
                      _draw_scene(srng, cw, ch, spec, True))
            rects = _flat_mask(srng, W, H, spec) if spec.flat_fraction > 0 else []
            if spec.pan is not None:
                speed = srng.uniform(spec.pan[0], spec.pan[1])
                ang = srng.uniform(0, 2 * math.pi)
                pan = (round(speed * math.cos(ang)), round(speed * math.sin(ang)))
                if pan == (0, 0):
                    pan = (int(spec.pan[0]), 0)
            ox = oy = 0.0
        else:
            if spec.pan is not None:
                ox += pan[0]
                oy += pan[1]
            else:
                d = motion_rng.integers(-spec.motion, spec.motion + 1, size=2)
                ox += float(d[0])
                oy += float(d[1])
        sigma = _sigma_for_scene(spec, scene_idx)
        noise_seed = int(master.integers(0, 2**63 - 1))
        if t < start:
            continue
        nrng = np.random.Generator(np.random.PCG64(noise_seed))
        planes = []
        for i, (scene, w, h) in enumerate(((scenes[0], W, H), (scenes[1], cw, ch), (scenes[2], cw, ch))):
            dx = 1 if i == 0 or cw == W else 2
            dy = 1 if i == 0 or ch == H else 2
            img = _render(scene, w, h, ox / dx, oy / dy)
            img += (sigma * nrng.standard_normal((h, w), dtype=np.float32))
            for (x0, y0, x1, y1, level) in rects:
                img[y0 // dy:y1 // dy, x0 // dx:x1 // dx] = level
            lo, hi = LUMA_RANGE_8 if i == 0 else CHROMA_RANGE_8
            planes.append(_quantize(img, lo, hi, scale, dtype))
        yield tuple(planes)


def frames_list(spec: SequenceSpec, start: int = 0, stop: int | None = None) -> list:
    return list(generate(spec, start, stop))


def pack_planes(frames: list, pitch_align: int = 64):
    """Stack frames into three contiguous arrays (F, rows, pitch) with padded pitch.

    Returns dict with arrays ``y``, ``u``, ``v`` and the byte pitches.  The padding
    columns are filled with a recognisable value (0xA5 bytes) that no analyzer
    should ever read.
    """
    y0, u0, _ = frames[0]
    es = y0.dtype.itemsize

    def stack(planes):
        h, w = planes[0].shape
        pitch = -(-(w * es) // pitch_align) * pitch_align
        arr = np.empty((len(planes), h, pitch // es), dtype=planes[0].dtype)
        arr.view(np.uint8)[...] = 0xA5
        for i, p in enumerate(planes):
            arr[i, :, :w] = p
        return arr, pitch

    y, py = stack([f[0] for f in frames])
    u, pu = stack([f[1] for f in frames])
    v, pv = stack([f[2] for f in frames])
    assert pu == pv
    return {"y": y, "u": u, "v": v, "pitch_y": py, "pitch_uv": pu}


# ---------------------------------------------------------------------------
# The workloads: shapes and content of the paper's measurement conditions
# ---------------------------------------------------------------------------

def tiny_spec(seed: int = 1) -> SequenceSpec:
    """16 frames 640x352 8-bit, sigma 4, random-walk motion in [-4, 4], scene cut at frame 8."""
    return SequenceSpec(640, 352, 16, seed, sigma=4.0, cuts=(8,), motion=4)


def hd_spec(seed: int = 2, n_frames: int = 120) -> SequenceSpec:
    """1920x1080 8-bit, sigma alternating 2 / 8 per scene, a scene cut every 40 frames."""
    return SequenceSpec(1920, 1080, n_frames, seed, sigma=(2.0, 8.0), cut_every=40, motion=4)


def uhd_spec(seed: int = 3, n_frames: int = 600, bit_depth: int = 8) -> SequenceSpec:
    """3840x2160: 30% flat block-aligned area, sinusoid periods 2-8 px, global pan 1-8 px/frame."""
    return SequenceSpec(3840, 2160, n_frames, seed, bit_depth=bit_depth, sigma=4.0, cut_every=150,
                        pan=(1, 8), periods=(2.0, 8.0), n_patches=(4, 6), flat_fraction=0.30)


LADDER_RESOLUTIONS = ((640, 360), (960, 540), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))


def ladder_specs(seed: int = 4, n_frames: int = 300) -> list:
    """24 streams: 4 per resolution, 2 at 8-bit and 2 at 10-bit each."""
    specs = []
    i = 0
    for (w, h) in LADDER_RESOLUTIONS:
        for bd in (8, 8, 10, 10):
            specs.append(SequenceSpec(w, h, n_frames, seed * 1000 + i, bit_depth=bd, sigma=4.0, cuts=(n_frames // 2,)))
            i += 1
    return specs
