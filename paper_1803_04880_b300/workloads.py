"""Seeded synthetic inputs for the five workloads (shared by the oracle tests,
the GPU tests and the benchmark).

This module generates bytes only: it holds none of the transform's or the
cipher's arithmetic.  The thesis measured on a bitmap image, English text and
video files that are not available here; these generators stand in for them
with the shapes the workloads name (Sec. 5.3 uses images, text and video
chunks; Table 5.x times chunks of 1024^2 .. 4800^2 bytes):

* ``c1``: one 256 x 256 matrix of uniform random bytes (seed 0), width 256,
  1 level, key 00 01 .. 0f, nonce 0.
* ``c2``: a 3-plane 4096 x 4096 "bitmap" (seed 1): per plane a smooth 2-D
  sinusoid plus gradient background, Gaussian noise (sigma 8), 200 solid
  axis-aligned rectangles painted in order, rounded and clipped to 0..255;
  width 4096, 3 levels, one item per plane with nonce = plane index.
* ``c3``: a 256 MiB format-agnostic buffer (seed 2) in three parts: uniform
  bytes; ASCII text from a seeded order-1 Markov chain over the 95 printable
  characters and newline (Zipf-skewed transition rows, order-0 entropy near
  the 4.6 bits of the thesis's text chunks); a little-endian int32 random walk
  with N(0, 1000^2) steps.  Width 8192, run at 2 and 4 levels.
* ``c4``: 10,000 buffers with log-uniform sizes in [4 KiB, 64 MiB] (seed 3),
  width = 2^round(log2(n)/2), levels uniform in 1..4, nonce = index, contents
  uniform random bytes drawn on the device.
* ``c5``: a Poisson stream of protect/recover requests (seed 4), sizes
  log-uniform in [1 KiB, 256 MiB], width 4096, 3 levels.

Generators take a size argument so tests can draw the same recipe at sizes
the oracle finishes in seconds.
"""
from __future__ import annotations

import math

import numpy as np

KEY = bytes(range(16))  # 000102..0f


# -- C1 --------------------------------------------------------------------------

def c1(side: int = 256) -> np.ndarray:
    rng = np.random.default_rng(0)
    return rng.integers(0, 256, (side, side), dtype=np.uint8)


# -- C2 --------------------------------------------------------------------------

def c2_plane(rng: np.random.Generator, side: int, n_rects: int = 200) -> np.ndarray:
    y, x = np.meshgrid(np.arange(side, dtype=np.float32), np.arange(side, dtype=np.float32),
                       indexing="ij")
    fx, fy = rng.uniform(0.5, 4.0, 2) / side
    phi = rng.uniform(0, 2 * np.pi)
    gx, gy = rng.uniform(-40.0, 40.0, 2) / side
    img = 128.0 + 60.0 * np.sin(2 * np.pi * (fx * x + fy * y) + phi) + gx * x + gy * y
    img += rng.normal(0.0, 8.0, (side, side)).astype(np.float32)
    lo = max(1, (8 * side) // 4096)
    hi = max(lo + 1, (1024 * side) // 4096)
    for _ in range(n_rects):
        h, w = rng.integers(lo, hi + 1, 2)
        r0 = rng.integers(0, side)
        c0 = rng.integers(0, side)
        img[r0:r0 + h, c0:c0 + w] = rng.integers(0, 256)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def c2(side: int = 4096, planes: int = 3) -> np.ndarray:
    """(planes, side, side) uint8."""
    rng = np.random.default_rng(1)
    return np.stack([c2_plane(rng, side) for _ in range(planes)])


# -- C3 --------------------------------------------------------------------------

C3_BYTES = 256 * 1024 * 1024
C3_WIDTH = 8192


def _markov_text(rng: np.random.Generator, n: int, chains: int = 4096) -> np.ndarray:
    """Order-1 Markov text, stepped as ``chains`` independent chains (each
    started in state 0) that are concatenated; rows are Dirichlet draws around
    a Zipf(1.1) base so that the order-0 entropy is about 4.5 bits."""
    symbols = np.array([10] + list(range(32, 127)), dtype=np.uint8)  # '\n' + printables
    symbols = symbols[rng.permutation(96)]
    base = 1.0 / np.arange(1, 97) ** 1.10
    base /= base.sum()
    P = rng.dirichlet(20.0 * base + 1e-3, size=96)
    C = np.cumsum(P, axis=1)
    C[:, -1] = 1.0
    flat = (C + np.arange(96)[:, None]).ravel()
    chains = max(1, min(chains, n))
    steps = -(-n // chains)
    st = np.zeros(chains, dtype=np.int64)
    out = np.empty((chains, steps), dtype=np.uint8)
    for t in range(steps):
        u = rng.random(chains)
        st = np.searchsorted(flat, st + u, side="left") - st * 96
        np.clip(st, 0, 95, out=st)
        out[:, t] = st
    return symbols[out.ravel()[:n]]


def c3(total: int = C3_BYTES) -> np.ndarray:
    """Flat uint8 buffer: uniform | Markov text | int32 random walk."""
    rng = np.random.default_rng(2)
    third = (total // 3) // 4 * 4
    p1 = third
    p2 = third
    p3 = total - p1 - p2
    p3 -= p3 % 4
    p1 = total - p2 - p3
    a = rng.integers(0, 256, p1, dtype=np.uint8)
    b = _markov_text(rng, p2)
    steps = np.rint(rng.normal(0.0, 1000.0, p3 // 4)).astype(np.int64)
    walk = np.cumsum(steps).astype(np.int64)
    walk = ((walk + 2**31) % 2**32 - 2**31).astype("<i4")
    return np.concatenate([a, b, walk.view(np.uint8)])


# -- C4 --------------------------------------------------------------------------

def c4_items(count: int = 10000, lo: int = 4096, hi: int = 1 << 26, seed: int = 3):
    """List of (n, width, levels, nonce) tuples."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)
    levels = rng.integers(1, 5, count)
    items = []
    for i, (n, L) in enumerate(zip(sizes, levels)):
        w = 1 << int(round(math.log2(int(n)) / 2))
        w = max(w, 1 << int(L))
        items.append((int(n), int(w), int(L), i))
    return items


def c4_content(index: int, n: int, device="cpu", seed: int = 3):
    """Uniform random bytes of item ``index`` (torch tensor on ``device``; the
    CPU and CUDA generators give different streams, so compare like with like)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed * 1_000_003 + index)
    return torch.randint(0, 256, (n,), dtype=torch.uint8, device=device, generator=g)


# -- C5 --------------------------------------------------------------------------

def c5_requests(count: int, rate_per_s: float, lo: int = 1024, hi: int = 1 << 28,
                seed: int = 4):
    """List of (arrival_s, kind, n) with kind in {'protect', 'recover'}."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, count)
    t = np.cumsum(gaps)
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)
    kinds = np.where(rng.random(count) < 0.5, "protect", "recover")
    return [(float(a), str(k), int(n)) for a, k, n in zip(t, kinds, sizes)]


def random_bytes(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).integers(0, 256, n, dtype=np.uint8)
