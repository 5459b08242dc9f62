"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the transform itself: it only draws
random numbers (residual blocks, angle indices, permutations, set indices,
correlated patches) with numpy.  Both the CUDA path (through the tests and
the benchmark) and the CPU oracle take their inputs from here.

The paper evaluates on HEVC common-test-condition sequences and on JEM-2.0
training data (Sec. VI); neither is available, so these generators stand in
for them with the block sizes (4x4, 8x8, 16x16), the 35 x 3 = 105 transform
sets per block size and the int16 residual range the paper implies.
"""
from __future__ import annotations

import math
import os

import numpy as np

SKIP = 0xFFFF
CHUNK = 1 << 16  # blocks per independently seeded chunk


def _chunk_rng(seed: int, chunk: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream), int(chunk)])


def laplacian_blocks(nblocks: int, n: int, scale: float, lo: int, hi: int, seed: int,
                     first_block: int = 0, count: int | None = None) -> np.ndarray:
    """int16 residual blocks [count][n] drawn i.i.d. from Laplace(0, scale).

    Values are rounded half away from zero and clipped to [lo, hi].  Blocks
    are drawn in chunks of ``CHUNK`` blocks, each from its own generator
    seeded by (seed, chunk index), so any block range can be regenerated on
    its own: rows [first_block, first_block + count) of the full array.
    """
    if count is None:
        count = nblocks - first_block
    out = np.empty((count, n), np.int16)
    end = first_block + count
    spans = []  # (chunk, first row in the chunk, rows)
    b = first_block
    while b < end:
        ch = b // CHUNK
        c0 = ch * CHUNK
        s0, s1 = b - c0, min(end, min(c0 + CHUNK, nblocks)) - c0
        spans.append((ch, s0, s1 - s0))
        b = c0 + s1

    def draw(span):
        ch, s0, rows = span
        c0 = ch * CHUNK
        rng = _chunk_rng(seed, ch, 1)
        v = rng.laplace(0.0, scale, size=(min(c0 + CHUNK, nblocks) - c0, n))
        v = np.sign(v) * np.floor(np.abs(v) + 0.5)
        np.clip(v, lo, hi, out=v)
        o = c0 + s0 - first_block
        out[o:o + rows] = v[s0:s0 + rows].astype(np.int16)

    # chunks are independent (own generator each): draw them on threads
    # (numpy releases the GIL while it fills arrays); the result does not
    # depend on the thread count
    if len(spans) > 4:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(draw, spans))
    else:
        for sp in spans:
            draw(sp)
    return out


def angle_indices(num_sets: int, rounds: int, log2n: int, seed: int) -> np.ndarray:
    """8-bit angle indices [S][R][log2 n][n/2], uniform over 0..255."""
    rng = np.random.default_rng([int(seed), 2])
    return rng.integers(0, 256, size=(num_sets, rounds, log2n, (1 << log2n) // 2),
                        dtype=np.uint8)


def permutations(num_sets: int, rounds: int, n: int, seed: int,
                 between_rounds_only: bool = True) -> np.ndarray:
    """Gather permutations [S][R][n] (uint16), one slot after each round.

    With ``between_rounds_only`` the slots between rounds (0..R-2) are random
    and the last slot (the optional final sort) is the identity.
    """
    rng = np.random.default_rng([int(seed), 3])
    out = np.empty((num_sets, rounds, n), np.uint16)
    for s in range(num_sets):
        for r in range(rounds):
            if between_rounds_only and r == rounds - 1:
                out[s, r] = np.arange(n, dtype=np.uint16)
            else:
                out[s, r] = rng.permutation(n).astype(np.uint16)
    return out


def set_indices(nblocks: int, num_sets: int, seed: int, skip_frac: float = 0.0) -> np.ndarray:
    """Per-block transform-set index, uniform over 0..num_sets-1 (uint16).

    A fraction ``skip_frac`` of the blocks (Bernoulli) gets the sentinel
    0xFFFF: no secondary transform for that block.
    """
    rng = np.random.default_rng([int(seed), 4])
    s = rng.integers(0, num_sets, size=nblocks, dtype=np.uint16)
    if skip_frac > 0:
        s[rng.random(nblocks) < skip_frac] = SKIP
    return s


def theta_uniform(shape, seed: int) -> np.ndarray:
    """Free angles drawn uniformly from [-pi, pi) (float64)."""
    rng = np.random.default_rng([int(seed), 5])
    return rng.uniform(-math.pi, math.pi, size=shape)


def theta_from_indices(angle_idx: np.ndarray, angle_bits: int = 8) -> np.ndarray:
    """The angle an index stands for, 2*pi*q / 2^angle_bits, as float64."""
    return (2.0 * math.pi / float(1 << angle_bits)) * angle_idx.astype(np.float64)


def _chol_kron_ar1(rho_h: float, rho_v: float, side: int) -> np.ndarray:
    i = np.arange(side)
    ch = rho_h ** np.abs(i[:, None] - i[None, :])
    cv = rho_v ** np.abs(i[:, None] - i[None, :])
    return np.linalg.cholesky(np.kron(cv, ch))


def _chol_rotated_ar1(rho_along: float, rho_across: float, side: int) -> np.ndarray:
    yy, xx = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    x = xx.ravel().astype(np.float64)
    y = yy.ravel().astype(np.float64)
    du = ((x[:, None] - x[None, :]) + (y[:, None] - y[None, :])) / math.sqrt(2.0)
    dv = ((x[:, None] - x[None, :]) - (y[:, None] - y[None, :])) / math.sqrt(2.0)
    C = rho_along ** np.abs(du) * rho_across ** np.abs(dv)
    return np.linalg.cholesky(C + 1e-12 * np.eye(C.shape[0]))


def ar1_patches(nvec: int, side: int, seed: int, rho_h: float = 0.95, rho_v: float = 0.9,
                rho_along: float = 0.97, rho_across: float = 0.6) -> np.ndarray:
    """float32 patches [nvec][side*side], raster order, unit marginal variance.

    Half are drawn from a separable 2-D AR(1) Gaussian (rho_h, rho_v), half
    from an AR(1) field rotated by 45 degrees (rho_along along the diagonal,
    rho_across across it); the two halves are interleaved by a seeded shuffle.
    """
    rng = np.random.default_rng([int(seed), 6])
    n = side * side
    half = nvec // 2
    L1 = _chol_kron_ar1(rho_h, rho_v, side)
    L2 = _chol_rotated_ar1(rho_along, rho_across, side)
    z = rng.standard_normal((nvec, n))
    out = np.empty((nvec, n), np.float64)
    out[:half] = z[:half] @ L1.T
    out[half:] = z[half:] @ L2.T
    order = rng.permutation(nvec)
    return out[order].astype(np.float32)


def mixed_frame_tiling(frames: int, width: int, height: int, seed: int,
                       area_mix=(0.50, 0.35, 0.15)):
    """Split 16x16 units of a frame sequence into 4x4 / 8x8 / 16x16 blocks.

    Returns the number of blocks of each size (N = 16, 64, 256).  Exactly
    round(area_mix[i] * units) of the 16x16 units are tiled with blocks of
    size class i (16 4x4 blocks, 4 8x8 blocks or one 16x16 block per unit);
    the assignment of units to classes is a seeded shuffle.
    """
    units = frames * (width // 16) * (height // 16)
    n16 = int(round(area_mix[0] * units))
    n64 = int(round(area_mix[1] * units))
    n256 = units - n16 - n64
    rng = np.random.default_rng([int(seed), 7])
    labels = np.concatenate([np.zeros(n16, np.int8), np.ones(n64, np.int8),
                             np.full(n256, 2, np.int8)])
    rng.shuffle(labels)
    return {"units": units, "labels": labels,
            "blocks": (16 * n16, 4 * n64, n256)}
