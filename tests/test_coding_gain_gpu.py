"""The coding-gain objective of Sec. V on the GPU, against the FP64 oracle.

J(theta) = 1/(2N) sum_i log2 v_i with v = diag(T Phi T^T): on a batch x the
GPU estimates v from the transformed blocks, so with Phi the batch's own
correlation (x^T x / B, FP64 on the host) the oracle (oracle/coding_gain.py,
pinned on CPU) gives the same J and dJ/dtheta.  Also checked: the diagonal
backward equals the general backward fed w * y; the energy-compaction loss
through the diagonal backward equals the C oracle's gradient; and a seeded
multi-restart fit on the correlated-patch workload (separable and
45-degree AR(1) 8x8 patches) ends between the KLT bound (Eq. 2) and the
separable DCT's value.
"""
import math

import numpy as np
import pytest

from oracle import coding_gain as cg
from paper_2505_21728_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu


def _patches(nvec):
    w = workloads.get_fit("hygt8x8_r4_fit")
    return w.patches(nvec)


def _phi(x):
    x64 = x.astype(np.float64)
    return x64.T @ x64 / x64.shape[0]


def _dct2_sep(n):
    """Orthonormal 2-D DCT-II of n x n raster blocks, from its cosine definition."""
    k = np.arange(n)
    D = np.sqrt(2.0 / n) * np.cos(np.pi * (2 * k[None, :] + 1) * k[:, None] / (2 * n))
    D[0] /= np.sqrt(2.0)
    return np.kron(D, D)


@pytest.fixture(scope="module")
def data(gpu):
    import torch
    x = _patches(1 << 18)
    return x, torch.from_numpy(x).cuda(), _phi(x)


@pytest.mark.parametrize("rounds,with_perm", [(4, False), (2, True)])
def test_objective_and_gradient_match_oracle(gpu, data, rounds, with_perm):
    from paper_2505_21728_gb300 import fit
    x, dx, phi = data
    log2n, N = 6, 64
    perms = inputs.permutations(1, rounds, N, seed=5) if with_perm else None
    f = fit.CodingGainFit(dx, log2n, rounds, perms)
    th = inputs.theta_uniform((rounds, log2n, N // 2), seed=3).astype(np.float32)
    J, g = f.objective_grad(th)
    p0 = None if perms is None else perms[0]
    Je, ge = cg.objective_grad(th.astype(np.float64), log2n, rounds, phi, p0)
    assert abs(J - Je) <= 1e-5 * max(1.0, abs(Je))
    err = np.max(np.abs(g - ge)) / np.max(np.abs(ge))
    assert err <= 1e-4, "dJ/dtheta relative error %.3g" % err
    _, v = f.objective(th)
    ve = cg.variances(cg.transform(th.astype(np.float64), log2n, rounds, p0), phi)
    assert np.max(np.abs(v - ve) / ve) <= 1e-5
    f.close()


def test_diag_backward_equals_general_backward(gpu, data):
    import torch
    from paper_2505_21728_gb300 import hygt
    _, dx, _ = data
    log2n, rounds, N = 6, 3, 64
    th = inputs.theta_uniform((1, rounds, log2n, N // 2), seed=8).astype(np.float32)
    plan = hygt.Plan.from_theta(log2n, rounds, th)
    y = plan.forward_f32(dx)
    wv = torch.linspace(0.5, 2.0, N, device="cuda", dtype=torch.float32) / y.shape[0]
    gx_ref, gth_ref = plan.backward_f32(y, (y * wv).contiguous())
    B = y.shape[0]
    wb = hygt.hygt_backward_workspace_bytes(plan.handle, B)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    gx = torch.full_like(y, 7.0)
    gth = torch.empty_like(gth_ref)
    stream = torch.cuda.current_stream().cuda_stream
    code = hygt.hygt_backward_diag_f32(plan.handle, y.data_ptr(), wv.data_ptr(), gx.data_ptr(),
                                       gth.data_ptr(), None, B, work.data_ptr(), wb, stream, None)
    assert code == hygt.HYGT_OK
    torch.cuda.synchronize()
    assert torch.equal(gx, gx_ref)
    assert torch.equal(gth, gth_ref)
    # without dL/dx: the same dL/dtheta, and the output buffer is untouched
    gx2 = torch.full_like(y, 7.0)
    gth2 = torch.empty_like(gth_ref)
    code = hygt.hygt_backward_diag_f32(plan.handle, y.data_ptr(), wv.data_ptr(), None,
                                       gth2.data_ptr(), None, B, work.data_ptr(), wb, stream, None)
    assert code == hygt.HYGT_OK
    torch.cuda.synchronize()
    assert torch.equal(gth2, gth_ref) and bool((gx2 == 7.0).all())
    plan.close()


def test_energy_compaction_through_diag_backward(gpu, data, orc):
    import torch
    from paper_2505_21728_gb300 import hygt
    x, dx, _ = data
    log2n, rounds, N, K = 6, 4, 64, 8
    B = 1 << 15
    th = inputs.theta_uniform((1, rounds, log2n, N // 2), seed=9).astype(np.float32)
    plan = hygt.Plan.from_theta(log2n, rounds, th)
    xb = dx[:B].contiguous()
    y = plan.forward_f32(xb)
    wv = torch.zeros(N, dtype=torch.float32, device="cuda")
    wv[K:] = 2.0 / B
    wb = hygt.hygt_backward_workspace_bytes(plan.handle, B)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    gth = torch.empty(rounds * log2n * N // 2, dtype=torch.float64, device="cuda")
    code = hygt.hygt_backward_diag_f32(plan.handle, y.data_ptr(), wv.data_ptr(), None,
                                       gth.data_ptr(), None, B, work.data_ptr(), wb,
                                       torch.cuda.current_stream().cuda_stream, None)
    assert code == hygt.HYGT_OK
    _, ge, _ = orc.loss_grad_f64(x[:B].astype(np.float64), th[0].astype(np.float64), log2n,
                                 rounds, K)
    g = gth.cpu().numpy().reshape(ge.shape)
    assert np.max(np.abs(g - ge)) / np.max(np.abs(ge)) <= 1e-4
    plan.close()


def test_fit_with_restarts_between_klt_bound_and_dct(gpu, data):
    from paper_2505_21728_gb300 import fit
    x, dx, phi = data
    log2n, rounds, N = 6, 4, 64
    f = fit.CodingGainFit(dx, log2n, rounds)
    th, J, finals = f.fit(restarts=3, iters=300, lr=0.02, seed=0)
    bound = cg.klt_bound(phi)
    T = _dct2_sep(8)
    J_dct = float(np.sum(np.log2(cg.variances(T, phi))) / (2 * N))
    # the fitted value is what the oracle gives at the fitted angles
    Je = cg.objective(th.astype(np.float64), log2n, rounds, phi)
    assert abs(J - Je) <= 1e-5 * max(1.0, abs(Je))
    assert J == min(finals)
    assert J >= bound - 1e-9           # no orthogonal transform beats the KLT (Eq. 2)
    assert J < J_dct - 0.1             # clearly better than the separable DCT
    assert J - bound < 0.3             # within 0.3 bit per coefficient of the KLT
    # one restart's history: the objective went down
    _, hist, Jend = f.run(inputs.theta_uniform((rounds, log2n, N // 2), seed=1), 100)
    assert Jend < hist[0] - 0.5
    f.close()


def test_coding_gain_rejects_bad_arguments(gpu):
    import torch
    from paper_2505_21728_gb300 import hygt
    plan = hygt.Plan.from_theta(1, 1, np.zeros(1, np.float32))
    assert hygt.hygt_coding_gain_workspace_bytes(plan.handle, 100) == 0  # N = 2
    plan.close()
    plan = hygt.Plan.from_theta(4, 1, np.zeros(32, np.float32))
    y = torch.zeros((10, 16), dtype=torch.float32, device="cuda")
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    w = torch.zeros(16, dtype=torch.float32, device="cuda")
    ws = hygt.hygt_coding_gain_workspace_bytes(plan.handle, 10)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert hygt.hygt_coding_gain_f32(plan.handle, y.data_ptr(), 10, d.data_ptr(), w.data_ptr(),
                                     d.data_ptr(), work.data_ptr(), ws - 8, s) == hygt.HYGT_ERR_ARG
    assert hygt.hygt_coding_gain_f32(plan.handle, y.data_ptr(), 0, d.data_ptr(), w.data_ptr(),
                                     d.data_ptr(), work.data_ptr(), ws, s) == hygt.HYGT_ERR_ARG
    th = torch.zeros(4, dtype=torch.float32, device="cuda")
    g = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert hygt.hygt_adam_step(th.data_ptr(), g.data_ptr(), th.data_ptr(), th.data_ptr(), 4,
                               0.01, 0.9, 0.999, 1e-8, 0, s) == hygt.HYGT_ERR_ARG
    plan.close()
