"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: trig
identities and hand-worked values of the multiplier table, brute-force
enumeration of the hypercube pairs, special angles whose rotations are exact
signed permutations, a dense product of explicit Givens matrices built from
the paper's element-wise definition, orthogonality, and hand-worked integer
examples (tests/golden/hand_worked_int.txt).
"""
import math
import os

import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Multiplier table (Sec. IV, Fig. 5: on-the-fly conversion)
# --------------------------------------------------------------------------
def test_cs_table_special_values(orc):
    c, s = orc.cs_table(8, 8)
    # theta = 0, pi/2, pi, 3pi/2 give exact axis values
    assert (c[0], s[0]) == (256, 0)
    assert (c[64], s[64]) == (0, 256)
    assert (c[128], s[128]) == (-256, 0)
    assert (c[192], s[192]) == (0, -256)
    # theta = pi/4: 256/sqrt(2) = 181.019...; theta = pi/8: 236.516..., 97.96...
    assert (c[32], s[32]) == (181, 181)
    assert (c[16], s[16]) == (237, 98)


def test_cs_table_symmetries(orc):
    c, s = orc.cs_table(8, 8)
    q = np.arange(256)
    # cos(-t) = cos t, sin(-t) = -sin t  (q -> 256 - q)
    assert np.array_equal(c[(256 - q) % 256], c)
    assert np.array_equal(s[(256 - q) % 256], -s)
    # sin(t + pi/2) = cos t, cos(t + pi/2) = -sin t  (q -> q + 64)
    assert np.array_equal(s[(q + 64) % 256], c)
    assert np.array_equal(c[(q + 64) % 256], -s)
    # rotation gain stays within the bound of a rounded unit vector
    g = np.sqrt(c.astype(float) ** 2 + s.astype(float) ** 2) / 256.0
    assert g.min() > 0.995 and g.max() < 1.005
    assert np.all(np.abs(c) <= 256) and np.all(np.abs(s) <= 256)


def test_cs_table_other_precisions(orc):
    c, s = orc.cs_table(4, 6)  # 16 angles, 6 fractional bits
    assert (c[0], s[0]) == (64, 0)
    assert (c[4], s[4]) == (0, 64)
    assert (c[2], s[2]) == (45, 45)  # 64/sqrt(2) = 45.25


# --------------------------------------------------------------------------
# Hypercube pairing (Sec. IV, Fig. 3, Fig. 4; pair cover equation)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("log2n", [1, 2, 3, 4, 6, 8])
def test_pairs_cover_hypercube_edges(orc, log2n):
    N = 1 << log2n
    for p in range(log2n):
        # brute force: all edges along dimension p, in increasing order of m
        expect = [(m, m ^ (1 << p)) for m in range(N) if not (m >> p) & 1]
        got = [orc.pair(p, j) for j in range(N // 2)]
        assert got == expect
        flat = sorted(i for mn in got for i in mn)
        assert flat == list(range(N))  # the pairs cover 0..N-1 exactly once


# --------------------------------------------------------------------------
# Brute force: product of explicit Givens matrices (Sec. IV element-wise
# definition; PMPT product order of Eq. 5; gather permutation slots)
# --------------------------------------------------------------------------
def givens_matrix(N, m, n, theta):
    G = np.eye(N)
    G[m, m] = math.cos(theta)
    G[n, n] = math.cos(theta)
    G[m, n] = math.sin(theta)
    G[n, m] = -math.sin(theta)
    return G


def brute_force_T(theta, perms, log2n, rounds):
    """Dense T = P_R F_{R,k} ... F_{R,1} ... P_1 F_{1,k} ... F_{1,1}."""
    N = 1 << log2n
    T = np.eye(N)
    for r in range(rounds):
        for p in range(log2n):
            # pairs found by scanning i < j with j = i XOR 2^p, in increasing i
            pairs = [(i, i ^ (1 << p)) for i in range(N) if i < (i ^ (1 << p))]
            F = np.eye(N)
            for jj, (m, n) in enumerate(pairs):
                F = givens_matrix(N, m, n, theta[r, p, jj]) @ F
            T = F @ T
        if perms is not None:
            P = np.zeros((N, N))
            P[np.arange(N), perms[r]] = 1.0  # v'[i] = v[perm[i]]
            T = P @ T
    return T


@pytest.mark.parametrize("log2n,rounds", [(2, 1), (2, 3), (3, 2), (4, 1), (4, 2), (4, 3)])
@pytest.mark.parametrize("with_perm", [False, True])
def test_brute_force_dense_product(orc, log2n, rounds, with_perm):
    N = 1 << log2n
    theta = inputs.theta_uniform((1, rounds, log2n, N // 2), seed=11 + log2n + rounds)
    perms = inputs.permutations(1, rounds, N, seed=3, between_rounds_only=False) if with_perm else None
    Tb = brute_force_T(theta[0], None if perms is None else perms[0], log2n, rounds)
    To = orc.dense_f64(theta[0], log2n, rounds, None if perms is None else perms[0])
    assert np.max(np.abs(To - Tb)) < 1e-12
    x = np.random.default_rng(5).standard_normal((7, N))
    y, st = orc.fwd_f64(x, theta, log2n, rounds, perms)
    assert st == 0
    assert np.max(np.abs(y - x @ Tb.T)) < 1e-12


def test_dense_product_nonsymmetric_order(orc):
    """Swapping pass order or angle order changes T: the pins above would
    catch a reversed product (F_1 ... F_P instead of F_P ... F_1)."""
    log2n, rounds = 3, 2
    N = 8
    theta = inputs.theta_uniform((1, rounds, log2n, N // 2), seed=2)
    T = orc.dense_f64(theta[0], log2n, rounds)
    rev = theta[0][:, ::-1, :].copy()
    T2 = orc.dense_f64(rev, log2n, rounds)
    assert np.max(np.abs(T - T2)) > 1e-3


# --------------------------------------------------------------------------
# Orthogonality, energy and the inverse (Sec. III: orthogonal group,
# inverse product; Sec. IV: inverse of the parallel-Givens matrix)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("log2n,rounds", [(4, 2), (6, 2), (6, 4), (8, 3)])
def test_orthogonal_energy_inverse(orc, log2n, rounds):
    N = 1 << log2n
    S = 3
    theta = inputs.theta_uniform((S, rounds, log2n, N // 2), seed=log2n)
    perms = inputs.permutations(S, rounds, N, seed=9)
    T = orc.dense_f64(theta[1], log2n, rounds, perms[1])
    assert np.max(np.abs(T @ T.T - np.eye(N))) < 1e-12
    x = np.random.default_rng(1).standard_normal((50, N)) * 100
    sets = np.random.default_rng(2).integers(0, S, 50).astype(np.uint16)
    y, st = orc.fwd_f64(x, theta, log2n, rounds, perms, sets)
    assert st == 0
    rel = np.abs(np.linalg.norm(y, axis=1) / np.linalg.norm(x, axis=1) - 1.0)
    assert rel.max() < 1e-12
    xr, st = orc.inv_f64(y, theta, log2n, rounds, perms, sets)
    assert st == 0
    assert np.max(np.abs(xr - x)) < 1e-12 * np.max(np.abs(x))


# --------------------------------------------------------------------------
# Special angles: zero angles give the pure permutation; q = 64 and q = 128
# give exact signed swaps, so the integer path is an exact signed permutation
# --------------------------------------------------------------------------
@pytest.mark.parametrize("log2n,rounds", [(4, 2), (6, 2), (8, 3)])
def test_zero_angles_pure_permutation(orc, log2n, rounds):
    N = 1 << log2n
    S = 2
    q = np.zeros((S, rounds, log2n, N // 2), np.uint8)
    perms = inputs.permutations(S, rounds, N, seed=4, between_rounds_only=False)
    x = inputs.laplacian_blocks(40, N, 300.0, -32768, 32767, seed=1)
    sets = (np.arange(40) % S).astype(np.uint16)
    y, st = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    assert st == 0
    expect = x.astype(np.int64)
    for b in range(40):
        v = expect[b]
        for r in range(rounds):
            v = v[perms[sets[b], r]]
        assert np.array_equal(y[b], v)
    yf, _ = orc.fwd_f64(x.astype(float), np.zeros(q.shape), log2n, rounds, perms, sets)
    assert np.array_equal(yf, y.astype(float))
    xr, st = orc.inv_int(y, q, log2n, rounds, perms, sets)
    assert st == 0 and np.array_equal(xr, x)


@pytest.mark.parametrize("log2n,rounds", [(2, 2), (4, 2), (6, 2)])
def test_quarter_turn_angles_signed_permutation(orc, log2n, rounds):
    """Angles from {0, 64, 128, 192} give integer matrices with entries in
    {-1, 0, 1}; the integer HyGT must equal the exact product of the
    explicit integer Givens matrices (no rounding happens)."""
    N = 1 << log2n
    rng = np.random.default_rng(7)
    q = rng.choice(np.array([0, 64, 128, 192], np.uint8), size=(1, rounds, log2n, N // 2))
    perms = inputs.permutations(1, rounds, N, seed=8, between_rounds_only=False)
    T = np.rint(brute_force_T(2 * math.pi * q[0].astype(float) / 256, perms[0], log2n, rounds))
    T = T.astype(np.int64)
    x = inputs.laplacian_blocks(30, N, 1000.0, -32768, 32767, seed=2)
    y, st = orc.fwd_int(x, q, log2n, rounds, perms)
    assert st == 0
    assert np.array_equal(y, x.astype(np.int64) @ T.T)
    xr, st = orc.inv_int(y, q, log2n, rounds, perms)
    assert st == 0 and np.array_equal(xr, x)


# --------------------------------------------------------------------------
# Hand-worked integer examples (rounding, pair/angle order, perm slot)
# --------------------------------------------------------------------------
def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "hand_worked_int.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            name, log2n, rounds = tok[0], int(tok[1]), int(tok[2])
            angles = [int(a) for a in tok[3].split(",")]
            perm = None if tok[4] == "-" else [int(a) for a in tok[4].split(",")]
            N = 1 << log2n
            vals = [int(v) for v in tok[5:]]
            rows.append((name, log2n, rounds, angles, perm, vals[:N], vals[N:]))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_hand_worked_integer(orc, row):
    name, log2n, rounds, angles, perm, xin, expect = row
    N = 1 << log2n
    q = np.array(angles, np.uint8).reshape(1, rounds, log2n, N // 2)
    perms = None if perm is None else np.array(perm, np.uint16).reshape(1, rounds, N)
    if name.startswith("I"):
        out, st = orc.inv_int(np.array([xin], np.int32), q, log2n, rounds, perms)
    else:
        out, st = orc.fwd_int(np.array([xin], np.int16), q, log2n, rounds, perms)
    assert st == 0
    assert out[0].tolist() == expect


# --------------------------------------------------------------------------
# Integer vs FP64 on the same angles: the rounding error per pass is at most
# 1/2 per coefficient plus the table quantisation (|c - 256 cos| <= 1/2), so
# the deviation grows at most linearly in the number of passes.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("log2n,rounds", [(4, 2), (6, 2), (8, 3)])
def test_integer_close_to_float(orc, log2n, rounds):
    N = 1 << log2n
    S = 4
    q = inputs.angle_indices(S, rounds, log2n, seed=1)
    perms = inputs.permutations(S, rounds, N, seed=2)
    x = inputs.laplacian_blocks(200, N, 12.0, -512, 511, seed=3)
    sets = inputs.set_indices(200, S, seed=4)
    y, st = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    assert st == 0
    theta = inputs.theta_from_indices(q)
    yf, _ = orc.fwd_f64(x.astype(float), theta, log2n, rounds, perms, sets)
    P = rounds * log2n
    # per pass: rounding <= 1/2 per element (norm <= sqrt(N)/2); table error
    # <= |x| * sqrt(2) * 0.5/256 relative; bound on the vector norm
    nx = np.linalg.norm(x.astype(float), axis=1)
    bound = P * (math.sqrt(N) / 2 + nx * math.sqrt(2) * 0.5 / 256) * 1.01 ** P
    err = np.linalg.norm(y - yf, axis=1)
    assert np.all(err <= bound)


# --------------------------------------------------------------------------
# Set indices: skip sentinel is identity, out-of-range sets are errors
# --------------------------------------------------------------------------
def test_skip_and_bad_set(orc):
    log2n, rounds, N = 4, 2, 16
    q = inputs.angle_indices(2, rounds, log2n, seed=1)
    x = inputs.laplacian_blocks(4, N, 12.0, -512, 511, seed=3)
    sets = np.array([0, 0xFFFF, 1, 0], np.uint16)
    y, st = orc.fwd_int(x, q, log2n, rounds, None, sets)
    assert st == 0
    assert np.array_equal(y[1], x[1].astype(np.int32))
    big = np.array([[70000] * N, [-70000] * N], np.int32)
    xr, st = orc.inv_int(big, q, log2n, rounds, None, np.array([0xFFFF, 0xFFFF], np.uint16))
    assert st == 0 and np.all(xr[0] == 32767) and np.all(xr[1] == -32768)
    sets_bad = np.array([0, 2, 1, 0], np.uint16)
    y2, st = orc.fwd_int(x, q, log2n, rounds, None, sets_bad)
    assert st == orc.ERR_SET
    assert np.all(y2[1] == 0)
    assert np.array_equal(y2[[0, 2, 3]], y[[0, 2, 3]])


def test_overflow_is_reported(orc):
    log2n, rounds, N = 2, 1, 4
    q = np.full((1, rounds, log2n, N // 2), 32, np.uint8)
    y = np.full((1, N), 1 << 24, np.int32)  # products exceed int32
    _, st = orc.inv_int(y, q, log2n, rounds)
    assert st == orc.ERR_OVERFLOW


# --------------------------------------------------------------------------
# Dense matrix transform (Eq. 3).  Pinned by what the mathematics fixes, not
# by restating y = K x: with K the dense form of a HyGT set (Eq. 5), the
# matrix transform must reproduce the pass-by-pass FP64 HyGT, which the
# brute-force Givens product pins above; with K = 2^f times an exact signed
# permutation (quarter-turn angles, entries in {-1, 0, 1}), the integer
# transform is exact, since floor((2^f t + 2^(f-1)) / 2^f) = t for every
# integer t; K = 2^f I returns x; the skip sentinel and bad set indices
# behave as in the integer HyGT.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("log2n,rounds", [(4, 2), (6, 2), (8, 3)])
def test_dense_apply_f64_equals_hygt(orc, log2n, rounds):
    """Eq. 3 with the Eq. 5 product as K: equal to the FP64 HyGT to 1e-12."""
    N = 1 << log2n
    S, B = 3, 60
    theta = inputs.theta_uniform((S, rounds, log2n, N // 2), seed=20 + log2n)
    perms = inputs.permutations(S, rounds, N, seed=21)
    K = np.stack([orc.dense_f64(theta[s], log2n, rounds, perms[s]) for s in range(S)])
    x = np.random.default_rng(22).standard_normal((B, N)) * 50
    sets = inputs.set_indices(B, S, seed=23, skip_frac=0.1)
    y_dense, st = orc.dense_apply_f64(x, K, sets)
    assert st == 0
    y_hygt, st = orc.fwd_f64(x, theta, log2n, rounds, perms, sets)
    assert st == 0
    assert np.max(np.abs(y_dense - y_hygt)) < 1e-12 * max(1.0, np.max(np.abs(x)))
    # a different set's matrix would not match: the set lookup matters
    wrong, _ = orc.dense_apply_f64(x, K[[1, 2, 0]], sets)
    live = sets != 0xFFFF
    assert np.max(np.abs(wrong[live] - y_hygt[live])) > 1e-3


@pytest.mark.parametrize("log2n,rounds", [(2, 2), (4, 2), (6, 2)])
def test_dense_apply_int_signed_permutation_exact(orc, log2n, rounds):
    """K = 256 T with T the exact signed permutation of quarter-turn angles
    (built from explicit Givens matrices): the integer matrix transform
    returns x T^T exactly, and so does the integer HyGT of the same angles."""
    N = 1 << log2n
    rng = np.random.default_rng(31)
    q = rng.choice(np.array([0, 64, 128, 192], np.uint8), size=(2, rounds, log2n, N // 2))
    perms = inputs.permutations(2, rounds, N, seed=32, between_rounds_only=False)
    T = np.stack([np.rint(brute_force_T(2 * math.pi * q[s].astype(float) / 256, perms[s],
                                        log2n, rounds)).astype(np.int64) for s in range(2)])
    assert set(np.unique(T).tolist()) <= {-1, 0, 1}
    assert np.all(np.abs(T).sum(axis=2) == 1)  # one nonzero per row: a signed permutation
    x = inputs.laplacian_blocks(40, N, 1000.0, -32768, 32767, seed=33)
    sets = (np.arange(40) % 2).astype(np.uint16)
    y, st = orc.dense_apply_int(x, (256 * T).astype(np.int32), 8, sets)
    assert st == 0
    expect = np.einsum("bij,bj->bi", T[sets], x.astype(np.int64))  # signed permutation of x
    assert np.array_equal(y, expect)
    yh, st = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    assert st == 0 and np.array_equal(yh, y)


@pytest.mark.parametrize("frac_bits", [1, 8, 14])
def test_dense_apply_int_identity(orc, frac_bits):
    """K = 2^f I returns x for every f (the rounding offset never carries)."""
    N, B = 64, 25
    K = np.broadcast_to(np.eye(N, dtype=np.int32) << frac_bits, (2, N, N)).copy()
    x = inputs.laplacian_blocks(B, N, 5000.0, -32768, 32767, seed=41)
    sets = (np.arange(B) % 2).astype(np.uint16)
    y, st = orc.dense_apply_int(x, K, frac_bits, sets)
    assert st == 0 and np.array_equal(y, x.astype(np.int32))
    yf, st = orc.dense_apply_f64(x.astype(float), np.eye(N)[None].repeat(2, 0), sets)
    assert st == 0 and np.array_equal(yf, x.astype(float))


def test_dense_apply_rounding_half_up(orc):
    """One hand-worked row: K = [[128, 128]] (1/2, 1/2 at f = 8) on
    (1, 0), (-1, 0), (3, 0), (1, 1): sums 128, -128, 384, 256 plus 128,
    floored over 256 -> 1, 0, 2, 1 (round half up, like the HyGT butterfly)."""
    K = np.array([[[128, 128], [0, 256]]], np.int32)
    x = np.array([[1, 0], [-1, 0], [3, 0], [1, 1]], np.int16)
    y, st = orc.dense_apply_int(x, K, 8)
    assert st == 0
    assert y[:, 0].tolist() == [1, 0, 2, 1]
    assert y[:, 1].tolist() == [0, 0, 0, 1]


def test_dense_apply_skip_and_bad_set_like_hygt(orc):
    """0xFFFF is the identity (widened) and a set index >= S zeroes the block
    and reports ERR_SET, exactly as in the integer HyGT."""
    log2n, rounds, N, S = 4, 2, 16, 2
    q = inputs.angle_indices(S, rounds, log2n, seed=51)
    x = inputs.laplacian_blocks(6, N, 100.0, -1024, 1023, seed=52)
    sets = np.array([0, 0xFFFF, 5, 1, 0xFFFF, 2], np.uint16)
    yh, sth = orc.fwd_int(x, q, log2n, rounds, None, sets)
    K = np.stack([np.eye(N, dtype=np.int32) * 256] * S)
    yd, std = orc.dense_apply_int(x, K, 8, sets)
    assert sth == std == orc.ERR_SET
    for b in (1, 2, 4, 5):
        assert np.array_equal(yd[b], yh[b])
    assert np.all(yd[2] == 0) and np.all(yd[5] == 0)
    assert np.array_equal(yd[1], x[1].astype(np.int32))
    yf, stf = orc.dense_apply_f64(x.astype(float), K.astype(float) / 256, sets)
    assert stf == orc.ERR_SET and np.all(yf[2] == 0) and np.array_equal(yf[1], x[1].astype(float))


# --------------------------------------------------------------------------
# Parameter count (Sec. IV: R N log2(N) / 2 angles) and Table II memory ratios
# --------------------------------------------------------------------------
def _table2():
    rows = {}
    with open(os.path.join(GOLDEN, "table2_memory_ratios.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                tok = line.split()
                rows[tok[0]] = tuple(float(v) for v in tok[1:])
    return rows


def test_table2_memory_ratios_reproduce():
    """The printed ratios follow from 1 byte per KLT entry (N^2 per transform)
    and 1 byte per HyGT angle (R N log2 N / 2 per transform)."""
    def mem(kind, log2n):
        N = 1 << log2n
        return N * N if kind == "K" else int(kind[2:-1]) * N * log2n // 2

    for scheme, (r4, r8, ravg) in _table2().items():
        a, b = scheme.split("/")
        k4, k8 = 16 * 16, 64 * 64
        h4, h8 = mem(a, 4), mem(b, 6)  # 4x4 blocks: N = 16; 8x8 blocks: N = 64
        assert abs(k4 / h4 - r4) <= 0.05 + 1e-9
        assert abs(k8 / h8 - r8) <= 0.05 + 1e-9
        assert abs((k4 + k8) / (h4 + h8) - ravg) <= 0.05 + 1e-9
