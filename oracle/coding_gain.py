"""Coding-gain objective of the HyGT parameters, in FP64 (test infrastructure only).

Sec. V of Said et al. rates a transform by the variances of its outputs:
for residuals with covariance Phi, the transform T gives the variance vector
v = diag(T Phi T^T) (the variance-vector definition of Sec. V), and under the
high-rate approximation R(D) = 1/2 log2(eps^2 sigma^2 / D) each coefficient
costs 1/2 log2(v_i) bits plus terms that do not depend on T.  The average
rate per coefficient the transform controls is therefore

    J(theta) = 1 / (2N) * sum_i log2 v_i,

and, since an orthogonal T keeps sum_i v_i = trace(Phi), minimising J is
maximising the transform coding gain mean(v) / geomean(v).  (The paper fits
its angles with a Laplacian variation of the same model whose details it
leaves out; the constants eps and D drop out of J.)

The transform is built here as an explicit product of its layers -- one
parallel-Givens matrix per pass (Sec. IV) and one permutation matrix after
each round whose slot is given -- with the pairs of a pass found by
scanning the indices in increasing order (pair j of pass p is the j-th
index m with bit p clear, partner m + 2^p).  The gradient of J with respect
to every angle comes from the same product: with G = dJ/dT, the derivative
with respect to layer t is A_t^T G B_t^T (A_t the layers after t, B_t those
before), contracted with the derivative of that layer's 2x2 rotation block.
Nothing here is shared with the CUDA library or the C oracle.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["pass_pairs", "layers", "transform", "variances", "objective", "objective_grad",
           "coding_gain", "klt_bound"]


def pass_pairs(log2n: int, p: int) -> list[tuple[int, int]]:
    """Pairs (m, m + 2^p) of pass p, in increasing order of m."""
    N = 1 << log2n
    return [(m, m + (1 << p)) for m in range(N) if not (m >> p) & 1]


def _givens_layer(log2n, p, angles):
    """The parallel-Givens matrix of pass p: y_m = c x_m + s x_n,
    y_n = -s x_m + c x_n for each pair (m, n) with its own angle."""
    N = 1 << log2n
    F = np.eye(N)
    for j, (m, n) in enumerate(pass_pairs(log2n, p)):
        c, s = math.cos(angles[j]), math.sin(angles[j])
        F[m, m], F[m, n], F[n, m], F[n, n] = c, s, -s, c
    return F


def _perm_layer(perm):
    """Gather v'[i] = v[perm[i]] as a matrix."""
    N = len(perm)
    P = np.zeros((N, N))
    P[np.arange(N), np.asarray(perm, dtype=np.int64)] = 1.0
    return P


def layers(theta, log2n, rounds, perms=None):
    """The layers of one set's transform in the order they are applied:
    a list of (matrix, (r, p) or None for a permutation)."""
    theta = np.asarray(theta, np.float64).reshape(rounds, log2n, (1 << log2n) // 2)
    out = []
    for r in range(rounds):
        for p in range(log2n):
            out.append((_givens_layer(log2n, p, theta[r, p]), (r, p)))
        if perms is not None:
            out.append((_perm_layer(np.asarray(perms).reshape(rounds, -1)[r]), None))
    return out


def transform(theta, log2n, rounds, perms=None):
    """T = L_M ... L_1 (the first layer applied first, Eq. 5)."""
    T = np.eye(1 << log2n)
    for L, _ in layers(theta, log2n, rounds, perms):
        T = L @ T
    return T


def variances(T, phi):
    """v = diag(T Phi T^T)."""
    return np.einsum("ia,ab,ib->i", T, phi, T)


def objective(theta, log2n, rounds, phi, perms=None):
    """J = 1/(2N) sum_i log2 v_i."""
    v = variances(transform(theta, log2n, rounds, perms), phi)
    return float(np.sum(np.log2(v)) / (2 * len(v)))


def objective_grad(theta, log2n, rounds, phi, perms=None):
    """(J, dJ/dtheta [R][k][N/2]) by the chain rule through the layers."""
    N = 1 << log2n
    Ls = layers(theta, log2n, rounds, perms)
    M = len(Ls)
    before = [np.eye(N)]                  # before[t] = L_t-1 ... L_0
    for L, _ in Ls:
        before.append(L @ before[-1])
    T = before[-1]
    v = variances(T, phi)
    J = float(np.sum(np.log2(v)) / (2 * N))
    G = (T @ phi) / (v[:, None] * N * math.log(2.0))   # dJ/dT
    grad = np.zeros((rounds, log2n, N // 2))
    after = np.eye(N)                      # after = L_M-1 ... L_t+1
    th = np.asarray(theta, np.float64).reshape(rounds, log2n, N // 2)
    for t in range(M - 1, -1, -1):
        L, tag = Ls[t]
        if tag is not None:
            r, p = tag
            D = after.T @ G @ before[t].T    # dJ/dL_t
            for j, (m, n) in enumerate(pass_pairs(log2n, p)):
                c, s = math.cos(th[r, p, j]), math.sin(th[r, p, j])
                # d/dtheta of [[c, s], [-s, c]] at rows/cols (m, n)
                grad[r, p, j] = (D[m, m] * -s + D[m, n] * c + D[n, m] * -c + D[n, n] * -s)
        after = after @ L
    return J, grad


def coding_gain(v):
    """Transform coding gain mean(v) / geomean(v)."""
    v = np.asarray(v, np.float64)
    return float(np.mean(v) / np.exp(np.mean(np.log(v))))


def klt_bound(phi):
    """The smallest J any orthogonal transform reaches: 1/(2N) sum log2 of
    Phi's eigenvalues (Hadamard's inequality; the KLT of Eq. 2 attains it)."""
    lam = np.linalg.eigvalsh(phi)
    return float(np.sum(np.log2(lam)) / (2 * len(lam)))
