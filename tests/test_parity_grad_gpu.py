"""Parity of the FP32 backward (dL/dx, dL/dtheta) with the CPU oracle.

dL/dtheta of the energy-compaction loss is compared with the oracle's
analytic FP64 gradient (itself pinned to finite differences) and, for a
general dL/dy, with FP64 central finite differences of <dL/dy, T(theta) x>
evaluated by the oracle.  Tolerance: 1e-4 relative (max-abs over angles)."""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-4


def _t(a):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("log2n,rounds,with_perm", [(4, 2, True), (6, 4, False), (6, 2, True), (8, 2, True)])
def test_energy_loss_gradient(gpu, orc, log2n, rounds, with_perm):
    import torch
    N = 1 << log2n
    K = 8 if N >= 16 else 1
    B = 20000
    theta = inputs.theta_uniform((1, rounds, log2n, N // 2), seed=4)
    perms = inputs.permutations(1, rounds, N, seed=4) if with_perm else None
    side = int(round(N ** 0.5))
    x = inputs.ar1_patches(B, side, seed=2) if side * side == N else \
        np.random.default_rng(2).standard_normal((B, N)).astype(np.float32)
    plan = gpu.Plan.from_theta(log2n, rounds, theta.astype(np.float32), perms)
    dx = _t(x)
    y = plan.forward_f32(dx)
    mask = torch.zeros(N, device="cuda")
    mask[K:] = 1.0
    gy = (2.0 / B) * y * mask
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gx, gth = plan.backward_f32(y, gy, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    loss, g_o, gx_o = orc.loss_grad_f64(x.astype(np.float64), theta[0], log2n, rounds, K,
                                        None if perms is None else perms[0], want_gx=True)
    assert _rel(gth.cpu().numpy(), g_o.ravel()) <= GRAD_TOL
    assert _rel(gx.cpu().numpy().astype(np.float64), gx_o) <= GRAD_TOL


def test_general_dy_multi_set_against_finite_differences(gpu, orc):
    """Several sets, skip and bad blocks, an arbitrary dL/dy."""
    import torch
    log2n, rounds, S, B = 6, 2, 3, 3000
    N = 64
    theta = inputs.theta_uniform((S, rounds, log2n, N // 2), seed=6)
    perms = inputs.permutations(S, rounds, N, seed=6)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((B, N))
    gy = rng.standard_normal((B, N))
    sets = inputs.set_indices(B, S, seed=6, skip_frac=0.05)
    sets[7] = 99  # bad set index
    plan = gpu.Plan.from_theta(log2n, rounds, theta.astype(np.float32), perms)
    y = plan.forward_f32(_t(x.astype(np.float32)), _t(sets))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gx, gth = plan.backward_f32(y, _t(gy.astype(np.float32)), _t(sets), status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 4
    gth = gth.cpu().numpy().reshape(theta.shape)
    gx = gx.cpu().numpy().astype(np.float64)
    # dL/dx = T^T gy (= inverse transform for an orthogonal T); skip: gy; bad: 0
    gx_o, _ = orc.inv_f64(gy, theta, log2n, rounds, perms, sets)
    gx_o[sets == 0xFFFF] = gy[sets == 0xFFFF]
    assert _rel(gx, gx_o) <= GRAD_TOL
    assert np.all(gx[7] == 0)

    def f(th):
        yy, _ = orc.fwd_f64(x, th, log2n, rounds, perms, sets)
        ok = (sets != 0xFFFF) & (sets < S)
        return float(np.sum(gy[ok] * yy[ok]))

    h = 1e-6
    picks = [(s, r, p, j) for s in range(S) for (r, p, j) in [(0, 0, 3), (1, 5, 31), (0, 4, 17)]]
    fd, an = [], []
    for idx in picks:
        tp = theta.copy()
        tp[idx] += h
        tm = theta.copy()
        tm[idx] -= h
        fd.append((f(tp) - f(tm)) / (2 * h))
        an.append(gth[idx])
    fd, an = np.array(fd), np.array(an)
    assert np.max(np.abs(an - fd)) / np.max(np.abs(fd)) <= GRAD_TOL


def test_autograd_layer_and_fit(gpu, orc):
    """torch.autograd through the CUDA forward/backward; a few Adam steps on
    correlated patches reduce the energy outside the first K coefficients,
    which stays above the Ky Fan bound of the covariance (KLT optimality)."""
    import torch
    log2n, rounds, K, B = 6, 4, 8, 65536
    x = torch.from_numpy(inputs.ar1_patches(B, 8, seed=1)).cuda()
    layer = gpu.HyGTLayer(log2n, rounds, seed=3)
    y = layer(x)
    loss = (y[:, K:] ** 2).sum(dim=1).mean()
    loss.backward()
    _, g_o, _ = orc.loss_grad_f64(x.cpu().numpy().astype(np.float64),
                                  layer.theta.detach().cpu().numpy()[0].astype(np.float64),
                                  log2n, rounds, K)
    assert _rel(layer.theta.grad.cpu().numpy()[0].astype(np.float64), g_o) <= GRAD_TOL
    opt = torch.optim.Adam(layer.parameters(), lr=0.02)
    first = float(loss.item())
    for _ in range(30):
        opt.zero_grad()
        loss = (layer(x)[:, K:] ** 2).sum(dim=1).mean()
        loss.backward()
        opt.step()
    final = float((layer(x)[:, K:] ** 2).sum(dim=1).mean().item())
    assert final < 0.8 * first
    xc = x.double().cpu().numpy()
    ev = np.sort(np.linalg.eigvalsh(xc.T @ xc / B))[::-1]
    total = float(np.trace(xc.T @ xc / B))
    assert final >= total - ev[:K].sum() - 1e-6 * total


def test_fit_workload_full_batch(gpu, orc):
    """1,048,576 patches, N=64, 4 rounds: dL/dtheta vs the oracle gradient
    and vs FP64 central differences on sampled angles."""
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get_fit("hygt8x8_r4_fit")
    x = w.patches()
    theta = w.theta0()
    plan = gpu.Plan.from_theta(w.log2n, w.rounds, theta.astype(np.float32))
    y = plan.forward_f32(_t(x))
    mask = torch.zeros(w.N, device="cuda")
    mask[w.keep:] = 1.0
    gy = (2.0 / w.nvec) * y * mask
    _, gth = plan.backward_f32(y, gy)
    gth = gth.cpu().numpy().reshape(theta.shape[1:])
    x64 = x.astype(np.float64)
    _, g_o, _ = orc.loss_grad_f64(x64, theta[0], w.log2n, w.rounds, w.keep)
    assert _rel(gth, g_o) <= GRAD_TOL
    h = 1e-6
    rng = np.random.default_rng(0)
    idxs = [tuple(int(rng.integers(0, d)) for d in theta.shape[1:]) for _ in range(6)]
    for idx in idxs:
        tp = theta[0].copy()
        tp[idx] += h
        tm = theta[0].copy()
        tm[idx] -= h
        fd = (orc.loss_f64(x64, tp, w.log2n, w.rounds, w.keep)
              - orc.loss_f64(x64, tm, w.log2n, w.rounds, w.keep)) / (2 * h)
        assert abs(gth[idx] - fd) <= GRAD_TOL * np.max(np.abs(g_o))
