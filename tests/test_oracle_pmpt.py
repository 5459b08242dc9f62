"""Pins of the oracle's general PMPT (explicit pair covers), CPU only.

A PMPT pass is a parallel-Givens matrix over an arbitrary cover of 0..N-1 by
N/2 disjoint pairs (Sec. IV, Eq. 7-8); the transform is the product of its
passes, the first applied first (Sec. III, Eq. 5), and the inverse runs the
passes in reverse with negated angles (Eq. 9).  Pinned by: the product of
explicit Givens matrices built from the element-wise definition of Sec. IV;
the hypercube covers reproducing the HyGT oracle (itself pinned by brute
force); the commutativity of the rotations inside a pass (shuffled pair
order gives the same integers); orthogonality and the inverse; quarter-turn
angles giving exact signed permutations; zero angles giving the identity;
and the rejection of index vectors that do not cover 0..N-1 exactly once.
"""
import math

import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs


def random_covers(S, P, N, seed):
    """Random perfect matchings of 0..N-1: m, n arrays [S][P][N/2]."""
    rng = np.random.default_rng(seed)
    m = np.empty((S, P, N // 2), np.uint16)
    n = np.empty((S, P, N // 2), np.uint16)
    for s in range(S):
        for p in range(P):
            perm = rng.permutation(N)
            m[s, p], n[s, p] = perm[0::2], perm[1::2]
    return m, n


def hypercube_covers(log2n, rounds):
    """The hypercube edges of every pass, found by scanning i < j with
    j = i XOR 2^p (not by a closed formula), in increasing order of i."""
    N = 1 << log2n
    ms, ns = [], []
    for _ in range(rounds):
        for p in range(log2n):
            pairs = [(i, j) for i in range(N) for j in range(i + 1, N) if j == i ^ (1 << p)]
            ms.append([a for a, _ in pairs])
            ns.append([b for _, b in pairs])
    return np.array(ms, np.uint16)[None], np.array(ns, np.uint16)[None]


def givens(N, m, n, t):
    """G(m, n, theta) from the element-wise definition of Sec. IV."""
    G = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i == j and i in (m, n):
                G[i, j] = math.cos(t)
            elif i == m and j == n:
                G[i, j] = math.sin(t)
            elif i == n and j == m:
                G[i, j] = -math.sin(t)
            elif i == j:
                G[i, j] = 1.0
    return G


def brute_T(theta, m, n, N):
    """Product of every explicit Givens matrix, pass 0 first."""
    T = np.eye(N)
    for p in range(theta.shape[0]):
        F = np.eye(N)
        for j in range(N // 2):
            F = givens(N, int(m[p, j]), int(n[p, j]), theta[p, j]) @ F
        T = F @ T
    return T


@pytest.mark.parametrize("N,P", [(2, 1), (6, 3), (10, 4), (16, 5)])
def test_explicit_givens_product(orc, N, P):
    S = 2
    m, n = random_covers(S, P, N, seed=N)
    theta = inputs.theta_uniform((S, P, N // 2), seed=N + 1)
    x = np.random.default_rng(N).standard_normal((9, N)) * 10
    sets = (np.arange(9) % S).astype(np.uint16)
    y, st = orc.pmpt_fwd_f64(x, theta, m, n, N, P, sets)
    assert st == 0
    for s in range(S):
        T = brute_T(theta[s], m[s], n[s], N)
        assert np.max(np.abs(y[sets == s] - x[sets == s] @ T.T)) < 1e-12
        assert np.max(np.abs(T @ T.T - np.eye(N))) < 1e-12
    xr, st = orc.pmpt_inv_f64(y, theta, m, n, N, P, sets)
    assert st == 0 and np.max(np.abs(xr - x)) < 1e-12 * np.max(np.abs(x))


@pytest.mark.parametrize("log2n,rounds", [(2, 2), (4, 2), (6, 2), (8, 3)])
def test_hypercube_covers_reproduce_hygt(orc, log2n, rounds):
    N = 1 << log2n
    m, n = hypercube_covers(log2n, rounds)
    P = rounds * log2n
    S, B = 1, 300
    q = inputs.angle_indices(S, rounds, log2n, seed=log2n)
    x = inputs.laplacian_blocks(B, N, 200.0, -32768, 32767, seed=3)
    yh, st = orc.fwd_int(x, q, log2n, rounds)
    assert st == 0
    yp, st = orc.pmpt_fwd_int(x, q.reshape(S, P, N // 2), m, n, N, P)
    assert st == 0 and np.array_equal(yp, yh)
    xh, _ = orc.inv_int(yh, q, log2n, rounds)
    xp, st = orc.pmpt_inv_int(yh, q.reshape(S, P, N // 2), m, n, N, P)
    assert st == 0 and np.array_equal(xp, xh)
    th = inputs.theta_from_indices(q)
    yf, _ = orc.fwd_f64(x.astype(float), th, log2n, rounds)
    ypf, st = orc.pmpt_fwd_f64(x.astype(float), th.reshape(S, P, N // 2), m, n, N, P)
    assert st == 0 and np.max(np.abs(ypf - yf)) < 1e-9


def test_pairs_within_a_pass_commute(orc):
    """Eq. 8: with a pair cover the rotations of a pass commute, so the
    order of the pairs (with their angles) cannot change the integers."""
    N, P, S = 12, 6, 3
    m, n = random_covers(S, P, N, seed=5)
    q = np.random.default_rng(6).integers(0, 256, (S, P, N // 2)).astype(np.uint8)
    x = inputs.laplacian_blocks(200, N, 500.0, -32768, 32767, seed=7)
    sets = (np.arange(200) % S).astype(np.uint16)
    y, st = orc.pmpt_fwd_int(x, q, m, n, N, P, sets)
    assert st == 0
    rng = np.random.default_rng(8)
    order = np.stack([[rng.permutation(N // 2) for _ in range(P)] for _ in range(S)])
    pick = lambda a: np.take_along_axis(a, order, axis=2)  # noqa: E731
    y2, st = orc.pmpt_fwd_int(x, pick(q), pick(m), pick(n), N, P, sets)
    assert st == 0 and np.array_equal(y2, y)


@pytest.mark.parametrize("N", [4, 8, 14])
def test_quarter_turns_exact_signed_permutation(orc, N):
    P, S = 5, 1
    m, n = random_covers(S, P, N, seed=N + 30)
    q = np.random.default_rng(N).choice(np.array([0, 64, 128, 192], np.uint8), (S, P, N // 2))
    T = np.rint(brute_T(2 * math.pi * q[0].astype(float) / 256, m[0], n[0], N)).astype(np.int64)
    assert np.all(np.abs(T).sum(axis=1) == 1)
    x = inputs.laplacian_blocks(50, N, 1000.0, -32768, 32767, seed=N)
    y, st = orc.pmpt_fwd_int(x, q, m, n, N, P)
    assert st == 0 and np.array_equal(y, x.astype(np.int64) @ T.T)
    xr, st = orc.pmpt_inv_int(y, q, m, n, N, P)
    assert st == 0 and np.array_equal(xr, x)


def test_zero_angles_identity_and_set_handling(orc):
    N, P, S = 8, 3, 2
    m, n = random_covers(S, P, N, seed=1)
    q = np.zeros((S, P, N // 2), np.uint8)
    x = inputs.laplacian_blocks(6, N, 100.0, -1024, 1023, seed=2)
    sets = np.array([0, 1, 0xFFFF, 7, 1, 0], np.uint16)
    y, st = orc.pmpt_fwd_int(x, q, m, n, N, P, sets)
    assert st == orc.ERR_SET
    assert np.all(y[3] == 0)
    keep = [0, 1, 2, 4, 5]
    assert np.array_equal(y[keep], x[keep].astype(np.int32))
    big = np.full((2, N), 70000, np.int32)
    xr, st = orc.pmpt_inv_int(big, q, m, n, N, P, np.array([0xFFFF, 0], np.uint16))
    assert st == 0 and np.all(xr == 32767)


def test_rejects_index_vectors_that_are_not_a_cover(orc):
    N, P = 8, 2
    m, n = random_covers(1, P, N, seed=3)
    q = np.zeros((1, P, N // 2), np.uint8)
    x = np.zeros((1, N), np.int16)
    bad = m.copy()
    bad[0, 1, 0] = bad[0, 1, 1]          # an index used twice
    assert orc.pmpt_fwd_int(x, q, bad, n, N, P)[1] == orc.ERR_ARG
    bad = n.copy()
    bad[0, 0, 2] = N                     # out of range
    assert orc.pmpt_fwd_int(x, q, m, bad, N, P)[1] == orc.ERR_ARG
    bad = n.copy()
    bad[0, 0, 0] = m[0, 0, 0]            # a pair (i, i)
    assert orc.pmpt_fwd_int(x, q, m, bad, N, P)[1] == orc.ERR_ARG
    assert orc.pmpt_fwd_int(np.zeros((1, 7), np.int16), np.zeros((1, P, 3), np.uint8),
                            np.zeros((1, P, 3), np.uint16), np.ones((1, P, 3), np.uint16),
                            7, P)[1] == orc.ERR_ARG  # odd N
