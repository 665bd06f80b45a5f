"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds random-number generation and input recipes only: no
binning, no prefix sums, none of the method's arithmetic.  Both the CUDA path
and the CPU oracle consume the bytes it produces.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: output i of a stream
with seed s is mix(s + (i + 1) * GAMMA).  Gaussians come from the Box-Muller
transform in double precision, rounded half-to-even and clipped to [0, 255].

The paper measures on unnamed "HD images" and image sequences (Sec. 4.4-4.7);
the recipes below stand in for them with the sizes and bin counts of its
experiments.  Recipes:

* ``uniform_frame``   i.i.d. uniform pixels (top byte of each draw).
* ``gradient_frame``  255 * (x/(W-1) + y/(H-1)) / 2 plus N(0, sigma^2) noise.
* ``sinusoid_frame``  128 + 50 sin(2 pi x/997) + 40 sin(2 pi y/1231)
                      + 25 sin(2 pi (x+y)/313) + U[-12, 12].
* ``rects``           inclusive rectangles, x0 <= x1 and y0 <= y1 each a
                      sorted pair of uniform integers.
* ``uneven_batch``    frames with resolution drawn from {320x240, 640x480,
                      1280x720, 1920x1080} and bin count from {16, 32, 64}.
* ``poisson_arrivals`` exponential inter-arrival gaps.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
SEED_XOR = 0x171101919
_ROWS_PER_BLOCK = 512

BATCH_RESOLUTIONS = ((320, 240), (640, 480), (1280, 720), (1920, 1080))  # (W, H)
BATCH_BINS = (16, 32, 64)


def workload_seed(index: int) -> int:
    """Seed of the numbered workload (1..5): index XOR 0x171101919."""
    return int(index) ^ SEED_XOR


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 stream with this seed."""
    i = np.arange(offset + 1, offset + 1 + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * np.uint64(GAMMA)
        return _mix(z)


def substream_seed(seed: int, index: int) -> int:
    """Seed of sub-stream `index`: output `index` of the parent stream."""
    return int(splitmix64(seed, 1, index)[0])


def _unit(z: np.ndarray) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits."""
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_frame(seed: int, h: int, w: int) -> np.ndarray:
    """h x w uint8, i.i.d. uniform on {0..255}: the top byte of each draw."""
    out = np.empty((h, w), dtype=np.uint8)
    for r0 in range(0, h, _ROWS_PER_BLOCK):
        r1 = min(h, r0 + _ROWS_PER_BLOCK)
        z = splitmix64(seed, (r1 - r0) * w, r0 * w)
        out[r0:r1] = (z >> np.uint64(56)).astype(np.uint8).reshape(r1 - r0, w)
    return out


def _gauss(seed: int, n: int, offset: int) -> np.ndarray:
    """n standard normals (Box-Muller); value j uses draws 2*(j//2), 2*(j//2)+1."""
    p0 = offset // 2
    p1 = (offset + n + 1) // 2
    z = splitmix64(seed, 2 * (p1 - p0), 2 * p0)
    u1 = 1.0 - _unit(z[0::2])  # (0, 1]
    u2 = _unit(z[1::2])
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    pair = np.empty(2 * (p1 - p0), dtype=np.float64)
    pair[0::2] = r * np.cos(t)
    pair[1::2] = r * np.sin(t)
    s = offset - 2 * p0
    return pair[s:s + n]


def gradient_frame(seed: int, h: int, w: int, sigma: float = 20.0) -> np.ndarray:
    """Smooth diagonal ramp 255*(x/(W-1) + y/(H-1))/2 plus Gaussian noise."""
    out = np.empty((h, w), dtype=np.uint8)
    gx = np.arange(w, dtype=np.float64) / max(w - 1, 1)
    for r0 in range(0, h, _ROWS_PER_BLOCK):
        r1 = min(h, r0 + _ROWS_PER_BLOCK)
        gy = np.arange(r0, r1, dtype=np.float64)[:, None] / max(h - 1, 1)
        g = 255.0 * (gx[None, :] + gy) / 2.0
        n = _gauss(seed, (r1 - r0) * w, r0 * w).reshape(r1 - r0, w)
        out[r0:r1] = np.clip(np.rint(g + sigma * n), 0, 255).astype(np.uint8)
    return out


def sinusoid_frame(seed: int, h: int, w: int) -> np.ndarray:
    """Seeded 2-D sum of sinusoids plus U[-12, 12] noise, clipped to [0, 255]."""
    out = np.empty((h, w), dtype=np.uint8)
    x = np.arange(w, dtype=np.float64)
    sx = 50.0 * np.sin(2.0 * math.pi * x / 997.0)
    for r0 in range(0, h, _ROWS_PER_BLOCK):
        r1 = min(h, r0 + _ROWS_PER_BLOCK)
        y = np.arange(r0, r1, dtype=np.float64)[:, None]
        v = 128.0 + sx[None, :] + 40.0 * np.sin(2.0 * math.pi * y / 1231.0)
        v = v + 25.0 * np.sin(2.0 * math.pi * (x[None, :] + y) / 313.0)
        u = _unit(splitmix64(seed, (r1 - r0) * w, r0 * w)).reshape(r1 - r0, w)
        out[r0:r1] = np.clip(np.rint(v + (-12.0 + 24.0 * u)), 0, 255).astype(np.uint8)
    return out


def _below(z: np.ndarray, n: int) -> np.ndarray:
    """Integers in [0, n) from the top 32 bits (multiply-shift)."""
    return (((z >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def rects(seed: int, n: int, h: int, w: int) -> np.ndarray:
    """n inclusive rectangles (x0, y0, x1, y1) as int32 [n][4]."""
    z = splitmix64(seed, 4 * n).reshape(n, 4)
    xa, xb = _below(z[:, 0], w), _below(z[:, 1], w)
    ya, yb = _below(z[:, 2], h), _below(z[:, 3], h)
    out = np.empty((n, 4), dtype=np.int32)
    out[:, 0] = np.minimum(xa, xb)
    out[:, 1] = np.minimum(ya, yb)
    out[:, 2] = np.maximum(xa, xb)
    out[:, 3] = np.maximum(ya, yb)
    return out


def uneven_batch_specs(seed: int, n: int):
    """[(h, w, nbins, frame_seed)] for an uneven batch of n frames."""
    meta = splitmix64(seed, 2 * n, 0).reshape(n, 2)
    specs = []
    for f in range(n):
        wv, hv = BATCH_RESOLUTIONS[int(_below(meta[f:f + 1, 0], len(BATCH_RESOLUTIONS))[0])]
        b = BATCH_BINS[int(_below(meta[f:f + 1, 1], len(BATCH_BINS))[0])]
        specs.append((hv, wv, b, substream_seed(seed, 1000 + f)))
    return specs


def uneven_batch(seed: int, n: int):
    """[(frame uint8 [h][w], nbins)] for an uneven batch of n uniform frames."""
    return [(uniform_frame(s, h, w), b) for (h, w, b, s) in uneven_batch_specs(seed, n)]


def poisson_arrivals(seed: int, rate_hz: float, duration_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process on [0, duration_s)."""
    n = max(16, int(rate_hz * duration_s * 1.5) + 64)
    while True:
        gaps = -np.log(1.0 - _unit(splitmix64(seed, n))) / rate_hz
        t = np.cumsum(gaps)
        if t[-1] >= duration_s:
            return t[t < duration_s]
        n *= 2


def fnv1a64_rows(img: np.ndarray) -> int:
    """FNV-1a 64 of each row, then FNV-1a 64 over the little-endian row hashes."""
    a = np.ascontiguousarray(img, dtype=np.uint8)
    prime = np.uint64(0x100000001B3)
    hrow = np.full(a.shape[0], 0xCBF29CE484222325, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for c in range(a.shape[1]):
            hrow = (hrow ^ a[:, c].astype(np.uint64)) * prime
    h = 0xCBF29CE484222325
    for byte in hrow.astype("<u8").tobytes():
        h = ((h ^ byte) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h
