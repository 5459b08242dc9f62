"""Pins of the coding-gain objective oracle (oracle/coding_gain.py), CPU only.

J(theta) = 1/(2N) sum_i log2 v_i with v = diag(T Phi T^T) (Sec. V variance
vector and high-rate model).  Pinned by: the closed form for N = 2; the
identity covariance; trace invariance; Hadamard's inequality (the KLT bound
of Eq. 2) and its equality case, where the gradient must vanish; central
finite differences of the gradient; and the C oracle's pass-by-pass
transform, which builds T independently."""
import math

import numpy as np
import pytest

from oracle import coding_gain as cg


def _ar1(N, rho_h, rho_v):
    """Separable AR(1) covariance of a sqrt(N) x sqrt(N) raster block."""
    n = int(round(math.sqrt(N)))
    idx = np.arange(N)
    r, c = idx // n, idx % n
    return rho_v ** np.abs(r[:, None] - r[None, :]) * rho_h ** np.abs(c[:, None] - c[None, :])


def _theta(S, R, log2n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-math.pi, math.pi, size=(R, log2n, (1 << log2n) // 2))


def _perms(R, N, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.permutation(N) for _ in range(R)]).astype(np.uint16)


@pytest.mark.parametrize("rho,theta", [(0.9, 0.3), (0.5, -1.1), (0.95, math.pi / 4)])
def test_two_point_closed_form(rho, theta):
    phi = np.array([[1.0, rho], [rho, 1.0]])
    a = rho * math.sin(2 * theta)
    J, g = cg.objective_grad(np.array([theta]), 1, 1, phi)
    assert J == pytest.approx(0.25 * math.log2(1 - a * a), abs=1e-14)
    want = -rho * rho * math.sin(4 * theta) / (2 * math.log(2) * (1 - a * a))
    assert g.ravel()[0] == pytest.approx(want, abs=1e-13)
    if theta == math.pi / 4:  # the KLT of this covariance: the bound, a stationary point
        assert J == pytest.approx(cg.klt_bound(phi), abs=1e-14)


def test_identity_covariance_is_flat():
    th = _theta(1, 2, 4, 0)
    J, g = cg.objective_grad(th, 4, 2, np.eye(16), _perms(2, 16, 0))
    assert abs(J) < 1e-14 and np.max(np.abs(g)) < 1e-13


@pytest.mark.parametrize("log2n,rounds", [(4, 2), (6, 2)])
def test_trace_and_klt_bound(log2n, rounds):
    N = 1 << log2n
    phi = _ar1(N, 0.95, 0.9)
    for seed in range(3):
        T = cg.transform(_theta(1, rounds, log2n, seed), log2n, rounds, _perms(rounds, N, seed))
        v = cg.variances(T, phi)
        assert np.sum(v) == pytest.approx(np.trace(phi), rel=1e-12)
        J = np.sum(np.log2(v)) / (2 * N)
        assert J >= cg.klt_bound(phi) - 1e-12
        lam = np.linalg.eigvalsh(phi)
        assert cg.coding_gain(v) <= cg.coding_gain(lam) * (1 + 1e-12)


def test_optimum_when_the_klt_is_a_hygt():
    """Phi = T0^T diag(lam) T0 with T0 a HyGT: at theta0 the variances are lam,
    J meets the KLT bound and the gradient vanishes."""
    log2n, R, N = 4, 2, 16
    th0 = _theta(1, R, log2n, 7)
    perms = _perms(R, N, 7)
    T0 = cg.transform(th0, log2n, R, perms)
    lam = np.linspace(4.0, 0.05, N)
    phi = T0.T @ np.diag(lam) @ T0
    J, g = cg.objective_grad(th0, log2n, R, phi, perms)
    assert np.allclose(cg.variances(T0, phi), lam, atol=1e-12)
    assert J == pytest.approx(cg.klt_bound(phi), abs=1e-12)
    assert np.max(np.abs(g)) < 1e-11
    # away from theta0 the objective is larger
    J1 = cg.objective(th0 + 0.05, log2n, R, phi, perms)
    assert J1 > J + 1e-6


@pytest.mark.parametrize("log2n,rounds,with_perms", [(3, 2, True), (4, 2, True), (6, 1, False)])
def test_gradient_matches_central_differences(log2n, rounds, with_perms):
    N = 1 << log2n
    phi = _ar1(N, 0.95, 0.9) if log2n % 2 == 0 else _ar1_1d(N, 0.9)
    th = _theta(1, rounds, log2n, 3)
    perms = _perms(rounds, N, 3) if with_perms else None
    J, g = cg.objective_grad(th, log2n, rounds, phi, perms)
    h = 1e-6
    flat = th.ravel()
    idx = range(flat.size) if flat.size <= 64 else np.random.default_rng(0).choice(
        flat.size, 48, replace=False)
    for i in idx:
        tp, tm = flat.copy(), flat.copy()
        tp[i] += h
        tm[i] -= h
        fd = (cg.objective(tp, log2n, rounds, phi, perms) -
              cg.objective(tm, log2n, rounds, phi, perms)) / (2 * h)
        assert g.ravel()[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def _ar1_1d(N, rho):
    i = np.arange(N)
    return rho ** np.abs(i[:, None] - i[None, :])


@pytest.mark.parametrize("log2n,rounds", [(3, 3), (4, 2), (6, 2)])
def test_layer_product_equals_the_c_oracle(orc, log2n, rounds):
    """The explicit layer product equals the C oracle's pass-by-pass transform
    (Fig. 4 index formula there, index scanning here), and the variances equal
    those of the oracle's forward of a Cholesky factor's columns."""
    N = 1 << log2n
    th = _theta(1, rounds, log2n, 11)
    perms = _perms(rounds, N, 11)
    T = cg.transform(th, log2n, rounds, perms)
    Tc = orc.dense_f64(th, log2n, rounds, perms)
    assert np.max(np.abs(T - Tc)) < 1e-12
    phi = _ar1_1d(N, 0.8)
    C = np.linalg.cholesky(phi)
    y, st = orc.fwd_f64(C.T.copy(), th.reshape(1, rounds, log2n, N // 2), log2n, rounds,
                        perms.reshape(1, rounds, N))
    assert st == 0
    assert np.allclose(np.sum(y * y, axis=0), cg.variances(T, phi), rtol=1e-12, atol=1e-12)
