"""Parity of the general PMPT kernels (explicit pair covers) with the oracle:
integer forward and inverse bit-exact, FP32 within 1e-5 of the FP64
oracle, for even N from 2 to 256 (powers of two and not), several sets,
skip and bad set indices, ragged batch sizes; and the hypercube covers
reproducing the HyGT kernels' integers."""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def covers(S, P, N, seed):
    rng = np.random.default_rng(seed)
    m = np.empty((S, P, N // 2), np.uint16)
    n = np.empty((S, P, N // 2), np.uint16)
    for s in range(S):
        for p in range(P):
            perm = rng.permutation(N)
            m[s, p], n[s, p] = perm[0::2], perm[1::2]
    return m, n


@pytest.mark.parametrize("N,P,B", [(2, 3, 1001), (6, 5, 777), (16, 8, 5003), (30, 7, 333),
                                   (64, 12, 4099), (100, 9, 257), (256, 24, 300)])
def test_pmpt_int_bit_exact(gpu, orc, N, P, B):
    import torch
    S = 5
    m, n = covers(S, P, N, seed=N)
    q = np.random.default_rng(N + 1).integers(0, 256, (S, P, N // 2)).astype(np.uint8)
    x = inputs.laplacian_blocks(B, N, 40.0, -32768, 32767, seed=N)
    sets = inputs.set_indices(B, S, seed=N, skip_frac=0.1)
    pm = gpu.PMPT(N, P, m, n, angle_idx=q)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = pm.forward(_t(x), _t(sets), status=st)
    xr = pm.inverse(y, _t(sets), status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ye, s1 = orc.pmpt_fwd_int(x, q, m, n, N, P, sets)
    xe, s2 = orc.pmpt_inv_int(ye, q, m, n, N, P, sets)
    assert s1 == s2 == 0
    assert np.array_equal(y.cpu().numpy(), ye)
    assert np.array_equal(xr.cpu().numpy(), xe)
    pm.close()


@pytest.mark.parametrize("N,P", [(8, 4), (64, 12), (144, 10)])
def test_pmpt_f32_within_tolerance(gpu, orc, N, P):
    S, B = 3, 2000
    m, n = covers(S, P, N, seed=N + 7)
    theta = inputs.theta_uniform((S, P, N // 2), seed=N).astype(np.float32)
    x = np.random.default_rng(N).standard_normal((B, N)).astype(np.float32) * 100
    sets = inputs.set_indices(B, S, seed=N + 1, skip_frac=0.1)
    pm = gpu.PMPT(N, P, m, n, theta=theta)
    y = pm.forward_f32(_t(x), _t(sets))
    xr = pm.inverse_f32(y, _t(sets))
    ye, _ = orc.pmpt_fwd_f64(x.astype(np.float64), theta.astype(np.float64), m, n, N, P, sets)
    yg = y.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(yg - ye)) <= 1e-5 * np.max(np.abs(ye))
    xe, _ = orc.pmpt_inv_f64(yg, theta.astype(np.float64), m, n, N, P, sets)
    assert np.max(np.abs(xr.cpu().numpy() - xe)) <= 1e-5 * np.max(np.abs(xe))
    pm.close()


@pytest.mark.parametrize("log2n,rounds", [(4, 2), (6, 2), (8, 3)])
def test_hypercube_covers_equal_hygt_kernels(gpu, log2n, rounds):
    """With the hypercube's pairs (pair j of pass p: j with a zero bit
    inserted at p, and that index + 2^p) the PMPT kernels give the HyGT
    kernels' integers."""
    N = 1 << log2n
    P, S, B = rounds * log2n, 4, 3000
    m = np.empty((S, P, N // 2), np.uint16)
    n = np.empty((S, P, N // 2), np.uint16)
    for k in range(P):
        p = k % log2n
        j = np.arange(N // 2)
        mm = ((j >> p) << (p + 1)) | (j & ((1 << p) - 1))
        m[:, k], n[:, k] = mm, mm + (1 << p)
    q = inputs.angle_indices(S, rounds, log2n, seed=log2n)
    x = inputs.laplacian_blocks(B, N, 60.0, -32768, 32767, seed=log2n)
    sets = inputs.set_indices(B, S, seed=log2n, skip_frac=0.05)
    plan = gpu.Plan(log2n, rounds, q)
    pm = gpu.PMPT(N, P, m, n, angle_idx=q.reshape(S, P, N // 2))
    dx, ds = _t(x), _t(sets)
    yh = plan.forward(dx, ds)
    yp = pm.forward(dx, ds)
    assert bool((yh == yp).all())
    assert bool((plan.inverse(yh, ds) == pm.inverse(yp, ds)).all())
    pm.close()
    plan.close()


def test_pmpt_bad_sets_and_arguments(gpu, orc):
    import torch
    N, P, S = 10, 3, 2
    m, n = covers(S, P, N, seed=1)
    q = np.random.default_rng(2).integers(0, 256, (S, P, N // 2)).astype(np.uint8)
    x = inputs.laplacian_blocks(7, N, 100.0, -1024, 1023, seed=3)
    sets = np.array([0, 1, 9, 0xFFFF, 1, 2, 0], np.uint16)
    pm = gpu.PMPT(N, P, m, n, angle_idx=q)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = pm.forward(_t(x), _t(sets), status=st).cpu().numpy()
    ye, ste = orc.pmpt_fwd_int(x, q, m, n, N, P, sets)
    assert int(st.item()) == gpu.HYGT_ERR_SET_INDEX and ste == orc.ERR_SET
    assert np.array_equal(y, ye)
    assert np.all(y[2] == 0) and np.array_equal(y[3], x[3].astype(np.int32))
    # empty batch
    e = pm.forward(torch.zeros((0, N), dtype=torch.int16, device="cuda"))
    assert e.shape == (0, N)
    # not a cover, odd N, both or neither angle arrays
    bad = m.copy()
    bad[1, 2, 0] = bad[1, 2, 1]
    assert gpu.hygt_pmpt_create(N, P, S, q, None, bad, n)[0] == gpu.HYGT_ERR_ARG
    assert gpu.hygt_pmpt_create(9, P, S, np.zeros((S, P, 4), np.uint8), None,
                                np.zeros((S, P, 4), np.uint16),
                                np.ones((S, P, 4), np.uint16))[0] == gpu.HYGT_ERR_ARG
    assert gpu.hygt_pmpt_create(N, P, S, None, None, m, n)[0] == gpu.HYGT_ERR_ARG
    # an FP32-only plan refuses the integer calls
    pf = gpu.PMPT(N, P, m, n, theta=np.zeros((S, P, N // 2), np.float32))
    with pytest.raises(gpu.HygtError):
        pf.forward(_t(x))
    assert gpu.hygt_pmpt_param_bytes(64, 12, 105) == 105 * 12 * 32 * 3
    pf.close()
    pm.close()
