"""Seeded synthetic infrared frames.

This module only draws inputs. It contains none of the filter's arithmetic
(no window, no extreme test, no median), so both the CUDA path and the CPU
oracle can consume the same bytes without sharing any of the method.

The paper's only test image (a 364x244 8-bit street scene, Sec. 4.2) is not
available, so every workload is a synthetic frame built the way the paper
argues IR frames look (Sec. 3, Eq. 1 and Eq. 2):

* a smooth temperature field T(x, y) in [250, 320] K, made of 8 Gaussian
  blobs (heat conduction keeps the surface temperature smooth and monotone,
  Eq. 2);
* gray level proportional to radiant emittance, i.e. to T^4 (Eq. 1),
  rescaled to the sensor range [0, MAXV];
* additive Gaussian sensor noise (sigma DN), rounded and clamped;
* impulse noise: each pixel independently replaced with probability p,
  either salt-and-pepper (0 or MAXV, half each) or random-valued
  (uniform integer in [0, MAXV]);
* optionally thin structures (1-pixel hot lines, 2x2 hot targets) inserted
  before the sensor noise, at +0.1*MAXV over the local field.

Seeds follow ``seed_for(config_index, frame_index)`` so every frame of every
workload is reproducible from two small integers.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 12013972
T_LO, T_HI = 250.0, 320.0

U8, U16, U14 = 0, 1, 2          # same codes as the C ABI's ir_dtype
MAXV = {U8: 255, U16: 65535, U14: 16383}
NP_DTYPE = {U8: np.uint8, U16: np.uint16, U14: np.uint16}


def seed_for(config_index: int, frame_index: int) -> int:
    """Seed = 12013972 + 1000 * config index + frame index."""
    return SEED_BASE + 1000 * int(config_index) + int(frame_index)


def thermal_field(rng: np.random.Generator, H: int, W: int, blobs: int = 8) -> np.ndarray:
    """Temperature field in kelvin, float64, shape (H, W), range [250, 320]."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    acc = np.zeros((H, W), dtype=np.float64)
    smin = float(min(H, W))
    for _ in range(blobs):
        cy = rng.uniform(0.0, H)
        cx = rng.uniform(0.0, W)
        s = rng.uniform(0.05, 0.25) * smin
        a = rng.uniform(0.3, 1.0)
        s = max(s, 0.5)
        acc += a * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * s * s))
    lo, hi = acc.min(), acc.max()
    if hi - lo < 1e-12:
        return np.full((H, W), 0.5 * (T_LO + T_HI))
    return T_LO + (acc - lo) * ((T_HI - T_LO) / (hi - lo))


def emittance_to_gray(T: np.ndarray, maxv: int) -> np.ndarray:
    """Gray level proportional to T^4 (Eq. 1), affine to [0, maxv], float64."""
    return maxv * (T ** 4 - T_LO ** 4) / (T_HI ** 4 - T_LO ** 4)


def add_thin_structures(rng: np.random.Generator, g: np.ndarray, maxv: int,
                        lines: int = 4, targets: int = 16, return_mask: bool = False):
    """Insert 1-pixel hot lines (2 horizontal, 1 vertical, 1 diagonal) and 2x2
    hot targets at +0.1*maxv over the local field (float, before noise).
    With return_mask, also the boolean mask of the pixels they cover."""
    H, W = g.shape
    g = g.copy()
    g0 = g.copy()
    bump = 0.1 * maxv
    kinds = ["h", "h", "v", "d"][:lines]
    for kind in kinds:
        if kind == "h":
            y = int(rng.integers(0, H))
            g[y, :] += bump
        elif kind == "v":
            x = int(rng.integers(0, W))
            g[:, x] += bump
        else:
            n = min(H, W)
            y0 = int(rng.integers(0, H - n + 1))
            x0 = int(rng.integers(0, W - n + 1))
            idx = np.arange(n)
            g[y0 + idx, x0 + idx] += bump
    for _ in range(targets):
        y = int(rng.integers(0, max(H - 1, 1)))
        x = int(rng.integers(0, max(W - 1, 1)))
        g[y:y + 2, x:x + 2] += bump
    if return_mask:
        return g, g != g0
    return g


def add_impulses(rng: np.random.Generator, img: np.ndarray, p: float, maxv: int,
                 kind: str = "sp") -> np.ndarray:
    """Corrupt each pixel independently with probability p.

    kind='sp': salt-and-pepper, 0 or maxv with probability 1/2 each.
    kind='rv': random-valued, uniform integer in [0, maxv].
    """
    out = img.copy()
    hit = rng.random(img.shape) < p
    if kind == "sp":
        salt = rng.random(img.shape) < 0.5
        vals = np.where(salt, maxv, 0)
    elif kind == "rv":
        vals = rng.integers(0, maxv + 1, size=img.shape)
    else:
        raise ValueError(f"unknown impulse kind {kind!r}")
    out[hit] = vals[hit].astype(out.dtype)
    return out


def make_frame_parts(H: int, W: int, dtype: int, seed: int, sigma: float, p: float,
                     impulse: str = "sp", thin: bool = False):
    """The seeded synthetic IR frame with its parts: (frame, the frame before
    impulses, mask of the thin-structure pixels (all False without them))."""
    if dtype not in MAXV:
        raise ValueError("dtype must be U8, U16 or U14")
    maxv = MAXV[dtype]
    rng = np.random.Generator(np.random.PCG64(seed))
    g = emittance_to_gray(thermal_field(rng, H, W), maxv)
    mask = np.zeros((H, W), dtype=bool)
    if thin:
        g, mask = add_thin_structures(rng, g, maxv, return_mask=True)
    g = g + rng.normal(0.0, sigma, size=(H, W))
    g = np.clip(np.rint(g), 0, maxv).astype(NP_DTYPE[dtype])
    pre = np.ascontiguousarray(g)
    if p > 0:
        g = add_impulses(rng, g, p, maxv, impulse)
    return np.ascontiguousarray(g), pre, mask


def make_frame(H: int, W: int, dtype: int, seed: int, sigma: float, p: float,
               impulse: str = "sp", thin: bool = False) -> np.ndarray:
    """One seeded synthetic IR frame as a contiguous (H, W) uint8/uint16 array."""
    return make_frame_parts(H, W, dtype, seed, sigma, p, impulse, thin)[0]


# ---------------------------------------------------------------------------
# The five workloads (frames of 1-5 below). Each is a list of FrameSpec; a
# spec is cheap, frames are materialised with .make().
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class FrameSpec:
    H: int
    W: int
    dtype: int
    k: int
    seed: int
    sigma: float
    p: float
    impulse: str = "sp"
    thin: bool = False
    tag: str = ""

    def make(self) -> np.ndarray:
        return make_frame(self.H, self.W, self.dtype, self.seed, self.sigma,
                          self.p, self.impulse, self.thin)

    @property
    def pixels(self) -> int:
        return self.H * self.W

    @property
    def esize(self) -> int:
        return 1 if self.dtype == U8 else 2


def sigma_for(dtype: int) -> float:
    return 2.0 if dtype == U8 else 8.0


def workload_single_u8() -> List[FrameSpec]:
    """320x240 u8, sigma 2 DN, 10% salt-and-pepper, 3x3 window, one frame."""
    return [FrameSpec(240, 320, U8, 3, seed_for(0, 0), 2.0, 0.10, "sp", False,
                      "320x240 u8 sp10 k3")]


def workload_sweep_u14() -> List[FrameSpec]:
    """640x512 14-bit, sigma 8 DN, hot lines + 2x2 targets, salt-and-pepper
    5/10/20/40%, windows 3/5/7 (12 runs)."""
    out = []
    i = 0
    for p in (0.05, 0.10, 0.20, 0.40):
        for k in (3, 5, 7):
            out.append(FrameSpec(512, 640, U14, k, seed_for(1, i), 8.0, p, "sp", True,
                                 f"640x512 u14 sp{int(p * 100)} k{k}"))
            i += 1
    return out


def workload_large_k() -> List[FrameSpec]:
    """1280x1024 14-bit, 20% random-valued impulses, windows 9/13/17/21."""
    return [FrameSpec(1024, 1280, U14, k, seed_for(2, i), 8.0, 0.20, "rv", False,
                      f"1280x1024 u14 rv20 k{k}")
            for i, k in enumerate((9, 13, 17, 21))]


BATCH_SIZES = ((120, 160), (240, 320), (512, 640), (1024, 1280), (1080, 1920))
BATCH_KS = (3, 5, 7, 9, 15)


def workload_batch(n: int = 256, ks: Sequence[int] = BATCH_KS, seed_cfg: int = 3) -> List[FrameSpec]:
    """Mixed batch: sizes uniform over 5 shapes, dtype u8/u14 50/50, k uniform
    over ``ks``, salt-and-pepper density uniform in [5%, 30%]."""
    rng = np.random.Generator(np.random.PCG64(seed_for(seed_cfg, 999)))
    out = []
    for i in range(n):
        H, W = BATCH_SIZES[int(rng.integers(0, len(BATCH_SIZES)))]
        dt = U8 if rng.random() < 0.5 else U14
        k = int(ks[int(rng.integers(0, len(ks)))])
        p = float(rng.uniform(0.05, 0.30))
        out.append(FrameSpec(H, W, dt, k, seed_for(seed_cfg, i), sigma_for(dt), p, "sp", False,
                             f"batch#{i} {W}x{H} {'u8' if dt == U8 else 'u14'} k{k}"))
    return out


SERVE_SIZES = ((240, 320), (512, 640), (1024, 1280))
SERVE_KS = (3, 5, 7)


@dataclass(frozen=True)
class StreamSpec:
    """One simulated video stream: fixed resolution and window, Poisson
    arrivals at ``fps``; its j-th frame is frame (offset + j) % pool of the
    shared pool of its resolution (see ``serve_pool``)."""
    stream_id: int
    H: int
    W: int
    k: int
    fps: float
    pool: int
    offset: int
    size_index: int

    def pool_index(self, j: int) -> int:
        return (self.offset + j) % self.pool


def serve_pool(size_index: int, pool: int = 30) -> List[FrameSpec]:
    """The pool of pre-generated 14-bit frames (10% salt-and-pepper) that all
    streams of one resolution loop over."""
    H, W = SERVE_SIZES[size_index]
    return [FrameSpec(H, W, U14, 3, seed_for(4, 100 * size_index + j), 8.0, 0.10, "sp", False,
                      f"serve {W}x{H} #{j}") for j in range(pool)]


def workload_serve(streams: int = 64, fps: float = 30.0, pool: int = 30) -> List[StreamSpec]:
    """64 streams at 30 fps: resolution round-robin over 320x240 / 640x512 /
    1280x1024, window round-robin over 3 / 5 / 7, 14-bit, 10% impulses."""
    out = []
    for s in range(streams):
        si = s % len(SERVE_SIZES)
        H, W = SERVE_SIZES[si]
        k = SERVE_KS[(s // len(SERVE_SIZES)) % len(SERVE_KS)]
        out.append(StreamSpec(s, H, W, k, fps, pool, (7 * s) % pool, si))
    return out


def poisson_arrivals(rng: np.random.Generator, rate: float, duration: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of ``rate`` per second on [0, duration)."""
    if rate <= 0 or duration <= 0:
        return np.zeros(0)
    n_guess = int(rate * duration * 1.5 + 20)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_guess))
    while t[-1] < duration:
        more = t[-1] + np.cumsum(rng.exponential(1.0 / rate, size=n_guess))
        t = np.concatenate([t, more])
    return t[t < duration]


def pitched_copy(frame: np.ndarray, pitch_elems: int, offset_elems: int = 0,
                 fill: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Lay ``frame`` into a larger row-pitched buffer (for odd-pitch and
    misaligned-base cases). Returns (buffer, view of the frame in it)."""
    H, W = frame.shape
    if pitch_elems < W:
        raise ValueError("pitch smaller than width")
    buf = np.full(offset_elems + H * pitch_elems, fill, dtype=frame.dtype)
    view = np.lib.stride_tricks.as_strided(
        buf[offset_elems:], shape=(H, W),
        strides=(pitch_elems * frame.itemsize, frame.itemsize))
    view[...] = frame
    return buf, view
