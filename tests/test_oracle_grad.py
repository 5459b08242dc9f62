"""Pins of the oracle's energy-compaction loss and analytic gradient.

The loss L = (1/B) sum_b sum_{i >= K} y_{b,i}^2 is a coding-gain proxy (the
paper optimises coding gain from the transformed variances, Sec. V).  Its
gradient is pinned by FP64 central finite differences, by invariants
(energy is preserved, so K = 0 and K = N give a constant loss) and by the
closed form dL/dx = (2/B) T^T M T x with M the mask of the kept entries.
"""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs


@pytest.mark.parametrize("log2n,rounds,with_perm", [(3, 2, False), (4, 2, True), (6, 1, True)])
def test_gradient_matches_finite_differences(orc, log2n, rounds, with_perm):
    N = 1 << log2n
    theta = inputs.theta_uniform((rounds, log2n, N // 2), seed=3)
    perms = inputs.permutations(1, rounds, N, seed=5)[0] if with_perm else None
    x = inputs.ar1_patches(64, int(np.sqrt(N)) if log2n % 2 == 0 else 1, seed=1) \
        if log2n % 2 == 0 else np.random.default_rng(0).standard_normal((64, N))
    x = np.asarray(x, np.float64).reshape(64, N)
    K = N // 4
    loss, g, _ = orc.loss_grad_f64(x, theta, log2n, rounds, K, perms)
    assert abs(loss - orc.loss_f64(x, theta, log2n, rounds, K, perms)) < 1e-12 * max(1.0, loss)
    h = 1e-6
    fd = np.zeros_like(theta)
    it = np.nditer(theta, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        tp = theta.copy()
        tp[idx] += h
        tm = theta.copy()
        tm[idx] -= h
        fd[idx] = (orc.loss_f64(x, tp, log2n, rounds, K, perms)
                   - orc.loss_f64(x, tm, log2n, rounds, K, perms)) / (2 * h)
    err = np.max(np.abs(g - fd)) / np.max(np.abs(fd))
    assert err < 1e-6


@pytest.mark.parametrize("K", [0, 16])
def test_gradient_zero_when_loss_is_energy(orc, K):
    log2n, rounds, N = 4, 2, 16
    theta = inputs.theta_uniform((rounds, log2n, N // 2), seed=1)
    x = np.random.default_rng(1).standard_normal((32, N))
    loss, g, _ = orc.loss_grad_f64(x, theta, log2n, rounds, K)
    assert np.max(np.abs(g)) < 1e-12
    energy = np.mean(np.sum(x * x, axis=1))
    assert abs(loss - (energy if K == 0 else 0.0)) < 1e-12 * energy


def test_input_gradient_closed_form(orc):
    log2n, rounds, N, K = 4, 3, 16, 5
    theta = inputs.theta_uniform((rounds, log2n, N // 2), seed=2)
    perms = inputs.permutations(1, rounds, N, seed=2)[0]
    x = np.random.default_rng(3).standard_normal((10, N))
    _, _, gx = orc.loss_grad_f64(x, theta, log2n, rounds, K, perms, want_gx=True)
    T = orc.dense_f64(theta, log2n, rounds, perms)
    M = np.diag([0.0] * K + [1.0] * (N - K))
    expect = (2.0 / 10) * (x @ T.T @ M @ T)
    assert np.max(np.abs(gx - expect)) < 1e-12


@pytest.mark.parametrize("log2n,rounds,K", [(4, 2, 4), (6, 2, 8)])
def test_loss_respects_the_ky_fan_bound(orc, log2n, rounds, K):
    """Energy outside the first K outputs is at least the sum of the N - K
    smallest eigenvalues of the data's covariance (Ky Fan; the KLT of Eq. 2
    attains it), for any angles."""
    N, B = 1 << log2n, 512
    x = np.random.default_rng(5).standard_normal((B, N)) @ np.linalg.cholesky(
        0.9 ** np.abs(np.subtract.outer(np.arange(N), np.arange(N)))).T
    lam = np.sort(np.linalg.eigvalsh(x.T @ x / B))
    bound = np.sum(lam[:N - K])
    for seed in range(4):
        theta = inputs.theta_uniform((rounds, log2n, N // 2), seed=seed)
        perms = inputs.permutations(1, rounds, N, seed=seed)[0]
        assert orc.loss_f64(x, theta, log2n, rounds, K, perms) >= bound - 1e-9


def test_loss_meets_the_ky_fan_bound_at_its_klt(orc):
    """Data whose covariance has the rows of a HyGT T0 as eigenvectors, with
    decreasing eigenvalues: at T0's angles the loss equals the bound and the
    gradient vanishes."""
    log2n, rounds, N, K = 4, 2, 16, 5
    theta = inputs.theta_uniform((rounds, log2n, N // 2), seed=8)
    perms = inputs.permutations(1, rounds, N, seed=8)[0]
    T0 = orc.dense_f64(theta, log2n, rounds, perms)
    d = np.linspace(3.0, 0.2, N)
    q, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((4 * N, N)))
    z = q * np.sqrt(4 * N)                       # z^T z / B = I exactly
    x = (z * d) @ T0                             # x_b = T0^T diag(d) z_b
    loss, g, _ = orc.loss_grad_f64(x, theta, log2n, rounds, K, perms)
    assert abs(loss - np.sum(d[K:] ** 2)) < 1e-10
    assert np.max(np.abs(g)) < 1e-10
