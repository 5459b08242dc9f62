"""Pins of the oracle's secondary-transform pipeline (Sec. VI), CPU only.

The pipeline: an integer 2-D DCT-II primary of an M x M residual block
(C = round(256 D), rows then columns, each output rounded half up), then the
integer HyGT on the top-left s x s coefficients (s = 4 for 4 x 4 blocks,
8 for larger ones, raster order); the inverse undoes them in reverse order.
Pinned by: the DCT-II matrix against scipy's orthonormal DCT-II and the
hand-worked 4-point integer matrix (tests/golden/dct4_int.txt); the
constant block's closed form; the integer primary within its derived
rounding bound of scipy's FP64 2-D DCT; the secondary acting only on the
top-left sub-block, as the (brute-force pinned) HyGT oracle of that
sub-block; quarter-turn angles giving an exact signed permutation of the
sub-block; skip and bad set indices.
"""
import math
import os

import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
scipy_fft = pytest.importorskip("scipy.fft")


@pytest.mark.parametrize("log2m", [1, 2, 3, 4, 5])
def test_dct_matrix_definition(orc, log2m):
    M = 1 << log2m
    C, D = orc.dct_matrix(log2m)
    ref = scipy_fft.dct(np.eye(M), type=2, norm="ortho", axis=0)
    assert np.max(np.abs(D - ref)) < 1e-14
    assert np.max(np.abs(D @ D.T - np.eye(M))) < 1e-14
    frac = np.abs(256 * D - np.floor(256 * D) - 0.5)
    assert frac.min() > 1e-6          # no entry near a rounding tie
    assert np.max(np.abs(C - 256 * D)) <= 0.5


def test_dct4_integer_matrix_hand_worked(orc):
    want = np.loadtxt(os.path.join(GOLDEN, "dct4_int.txt"), dtype=np.int64)
    C, _ = orc.dct_matrix(2)
    assert np.array_equal(C, want)


def _blocks(B, M, seed, scale=40.0, lo=-512, hi=511):
    return inputs.laplacian_blocks(B, M * M, scale, lo, hi, seed=seed)


def test_constant_block_closed_form(orc):
    """A constant block c has only a DC coefficient: 4c for M = 4 (row stage
    2c, column stage 4c, hand-worked from C above) and 16c for M = 16
    (C[0][i] = 64 exactly)."""
    q = np.zeros((1, 2, 4, 8), np.uint8)
    for c in (-300, -1, 0, 1, 77, 511):
        x = np.full((1, 16), c, np.int16)
        y, st = orc.secondary_fwd(x, 2, q, 4, 2, None, np.array([0xFFFF], np.uint16))
        assert st == 0
        assert y[0, 0] == 4 * c and np.all(y[0, 1:] == 0)
        x16 = np.full((1, 256), c, np.int16)
        q8 = np.zeros((1, 2, 6, 32), np.uint8)
        y16, st = orc.secondary_fwd(x16, 4, q8, 6, 2, None, np.array([0xFFFF], np.uint16))
        assert st == 0 and y16[0, 0] == 16 * c


@pytest.mark.parametrize("log2m,log2n", [(2, 4), (3, 6), (4, 6), (5, 6)])
def test_integer_primary_near_fp64_dct(orc, log2m, log2n):
    """Primary only (skip sentinel): within the bound that C's quantisation
    (<= 1/2 per entry, of 256) and the two roundings give against scipy's
    FP64 2-D DCT-II; a transposed or mis-ordered stage would be off by
    O(max |x|)."""
    M = 1 << log2m
    B = 200
    x = _blocks(B, M, seed=log2m)
    sets = np.full(B, 0xFFFF, np.uint16)
    q = np.zeros((1, 2, log2n, (1 << log2n) // 2), np.uint8)
    y, st = orc.secondary_fwd(x, log2m, q, log2n, 2, None, sets)
    assert st == 0
    X = x.reshape(B, M, M).astype(np.float64)
    ref = scipy_fft.dctn(X, type=2, norm="ortho", axes=(1, 2)).reshape(B, M * M)
    for b in range(B):
        xm = np.abs(X[b])
        e1 = 0.5 + xm.sum(axis=1).max() / 512.0          # row stage, per output
        t_abs = np.abs(scipy_fft.dct(X[b], type=2, norm="ortho", axis=1)) + e1
        bound = 0.5 + t_abs.sum(axis=0).max() / 512.0 + math.sqrt(M) * e1
        assert np.max(np.abs(y[b] - ref[b])) <= bound


@pytest.mark.parametrize("log2m,log2n", [(2, 4), (3, 6), (5, 6)])
def test_secondary_acts_on_top_left_only(orc, log2m, log2n):
    M, N = 1 << log2m, 1 << log2n
    s = 1 << (log2n // 2)
    S, B, R = 3, 300, 2
    q = inputs.angle_indices(S, R, log2n, seed=log2m)
    perms = inputs.permutations(S, R, N, seed=log2m)
    x = _blocks(B, M, seed=10 + log2m)
    sets = inputs.set_indices(B, S, seed=log2m)
    y, st = orc.secondary_fwd(x, log2m, q, log2n, R, perms, sets)
    assert st == 0
    prim, st = orc.secondary_fwd(x, log2m, q, log2n, R, perms, np.full(B, 0xFFFF, np.uint16))
    assert st == 0
    Y, P = y.reshape(B, M, M), prim.reshape(B, M, M)
    outside = np.ones((M, M), bool)
    outside[:s, :s] = False
    assert np.array_equal(Y[:, outside], P[:, outside])
    sub = np.ascontiguousarray(P[:, :s, :s]).reshape(B, N)
    assert np.abs(sub).max() < 32768  # the oracle's HyGT takes int16 input
    ys, st = orc.fwd_int(sub.astype(np.int16), q, log2n, R, perms, sets)
    assert st == 0
    assert np.array_equal(Y[:, :s, :s].reshape(B, N), ys)
    # inverse: back to the primary coefficients, then near x
    xr, st = orc.secondary_inv(y, log2m, q, log2n, R, perms, sets)
    assert st == 0
    assert np.max(np.abs(xr.astype(np.int64) - x)) <= 4 + 0.02 * np.abs(x).max()


def test_quarter_turn_secondary_is_signed_permutation(orc):
    """Quarter-turn angles make the secondary an exact signed permutation of
    the top-left sub-block, built here from explicit Givens matrices."""
    log2m, log2n, R = 3, 6, 2
    M, N = 8, 64
    rng = np.random.default_rng(4)
    q = rng.choice(np.array([0, 64, 128, 192], np.uint8), size=(1, R, log2n, N // 2))
    T = np.eye(N, dtype=np.int64)
    for r in range(R):
        for p in range(log2n):
            F = np.eye(N, dtype=np.int64)
            j = 0
            for m in range(N):
                if (m >> p) & 1:
                    continue
                n = m + (1 << p)
                c = int(round(math.cos(2 * math.pi * q[0, r, p, j] / 256)))
                sn = int(round(math.sin(2 * math.pi * q[0, r, p, j] / 256)))
                F[m, m], F[m, n], F[n, m], F[n, n] = c, sn, -sn, c
                j += 1
            T = F @ T
    x = _blocks(50, M, seed=5)
    y, st = orc.secondary_fwd(x, log2m, q, log2n, R)
    prim, _ = orc.secondary_fwd(x, log2m, q, log2n, R, None, np.full(50, 0xFFFF, np.uint16))
    assert st == 0
    sub = prim.reshape(50, M, M)[:, :8, :8].reshape(50, N).astype(np.int64)
    assert np.array_equal(y.reshape(50, M, M)[:, :8, :8].reshape(50, N), sub @ T.T)


def test_skip_bad_set_and_shapes(orc):
    log2m, log2n, R = 2, 4, 2
    q = inputs.angle_indices(2, R, log2n, seed=1)
    x = _blocks(4, 4, seed=2)
    sets = np.array([0, 5, 0xFFFF, 1], np.uint16)
    y, st = orc.secondary_fwd(x, log2m, q, log2n, R, None, sets)
    assert st == orc.ERR_SET and np.all(y[1] == 0)
    prim, _ = orc.secondary_fwd(x[2:3], log2m, q, log2n, R, None, np.array([0xFFFF], np.uint16))
    assert np.array_equal(y[2], prim[0])
    # an 8x8 secondary needs a block of at least 8x8; a 4x4 block takes a 4x4 one
    assert orc.secondary_fwd(x, 2, inputs.angle_indices(1, R, 6, seed=1), 6, R)[1] == orc.ERR_ARG
    x8 = _blocks(2, 8, seed=3)
    assert orc.secondary_fwd(x8, 3, q, 4, R)[1] == orc.ERR_ARG
