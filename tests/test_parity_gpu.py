"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results must be bit-exact; FP32 results must satisfy
max |y_gpu - y_f64| <= 1e-5 * max |y_f64| over the batch.  Sizes span
several CTAs and warps with ragged tails; the full 8x8 workload (4,194,304
blocks, 105 sets) is compared on every block.
"""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu

FP_TOL = 1e-5


def _t(a):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _status():
    import torch
    return torch.zeros(1, dtype=torch.int32, device="cuda")


def run_int(gpu, log2n, rounds, q, perms, x, sets):
    plan = gpu.Plan(log2n, rounds, q, perms)
    st = _status()
    y = plan.forward(_t(x), None if sets is None else _t(sets), status=st)
    xr = plan.inverse(y, None if sets is None else _t(sets), status=st)
    out = y.cpu().numpy(), xr.cpu().numpy(), int(st.item())
    plan.close()
    return out


CASES = [(log2n, rounds) for log2n in range(1, 9) for rounds in (1, 3)]


@pytest.mark.parametrize("log2n,rounds", CASES)
@pytest.mark.parametrize("perm_kind", ["none", "between", "all"])
def test_int_parity_small(gpu, orc, log2n, rounds, perm_kind):
    N = 1 << log2n
    S = 7
    B = 3001
    q = inputs.angle_indices(S, rounds, log2n, seed=log2n * 10 + rounds)
    perms = None
    if perm_kind != "none":
        perms = inputs.permutations(S, rounds, N, seed=5, between_rounds_only=(perm_kind == "between"))
    x = inputs.laplacian_blocks(B, N, 40.0, -32768, 32767, seed=rounds)
    sets = inputs.set_indices(B, S, seed=2, skip_frac=0.1)
    y, xr, st = run_int(gpu, log2n, rounds, q, perms, x, sets)
    ye, ste = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    assert ste == 0 and st == 0
    assert np.array_equal(y, ye)
    xe, ste = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert ste == 0
    assert np.array_equal(xr, xe)


@pytest.mark.parametrize("B", [1, 31, 32, 33, 129])
def test_int_parity_ragged_counts(gpu, orc, B):
    log2n, rounds, S = 6, 2, 3
    q = inputs.angle_indices(S, rounds, log2n, seed=1)
    perms = inputs.permutations(S, rounds, 64, seed=1)
    x = inputs.laplacian_blocks(B, 64, 8.0, -1024, 1023, seed=B)
    sets = inputs.set_indices(B, S, seed=B)
    y, xr, st = run_int(gpu, log2n, rounds, q, perms, x, sets)
    ye, _ = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert st == 0 and np.array_equal(y, ye) and np.array_equal(xr, xe)


def test_int_extremes_max_rounds(gpu, orc):
    """Full int16 range at the largest block size and round count: the oracle
    checks every int64 intermediate fits int32, the GPU must agree bit for bit."""
    log2n, rounds, S = 8, 8, 2
    N = 256
    q = inputs.angle_indices(S, rounds, log2n, seed=3)
    perms = inputs.permutations(S, rounds, N, seed=3, between_rounds_only=False)
    B = 64
    rng = np.random.default_rng(0)
    x = rng.choice(np.array([-32768, 32767], np.int16), size=(B, N))
    x[:8] = 32767
    x[8:16] = -32768
    sets = (np.arange(B) % S).astype(np.uint16)
    y, xr, st = run_int(gpu, log2n, rounds, q, perms, x, sets)
    ye, ste = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    assert ste == 0 and st == 0 and np.array_equal(y, ye)
    xe, ste = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert ste == 0 and np.array_equal(xr, xe)


def test_int_no_sets_and_empty(gpu, orc):
    import torch
    log2n, rounds = 4, 2
    q = inputs.angle_indices(1, rounds, log2n, seed=0)
    x = inputs.laplacian_blocks(500, 16, 12.0, -512, 511, seed=0)
    y, xr, st = run_int(gpu, log2n, rounds, q, None, x, None)
    ye, _ = orc.fwd_int(x, q, log2n, rounds)
    assert st == 0 and np.array_equal(y, ye)
    plan = gpu.Plan(log2n, rounds, q)
    e = torch.empty((0, 16), dtype=torch.int16, device="cuda")
    assert plan.forward(e).shape == (0, 16)


def test_bad_set_index_reports_and_zeroes(gpu, orc):
    log2n, rounds, S = 6, 2, 4
    q = inputs.angle_indices(S, rounds, log2n, seed=4)
    x = inputs.laplacian_blocks(300, 64, 8.0, -1024, 1023, seed=4)
    sets = inputs.set_indices(300, S, seed=4)
    sets[17] = S      # out of range
    sets[200] = 1000  # out of range
    sets[5] = 0xFFFF  # skip
    y, xr, st = run_int(gpu, log2n, rounds, q, None, x, sets)
    assert st == 4
    ye, ste = orc.fwd_int(x, q, log2n, rounds, None, sets)
    assert ste == orc.ERR_SET
    assert np.array_equal(y, ye)
    assert np.all(y[17] == 0) and np.all(y[200] == 0)
    assert np.array_equal(y[5], x[5].astype(np.int32))


def test_inverse_saturates(gpu, orc):
    log2n, rounds = 4, 1
    q = np.zeros((1, rounds, log2n, 8), np.uint8)  # identity angles
    y = np.array([[40000] * 8 + [-40000] * 8, list(range(-8, 8))], np.int32)
    plan = gpu.Plan(log2n, rounds, q)
    xr = plan.inverse(_t(y)).cpu().numpy()
    xe, _ = orc.inv_int(y, q, log2n, rounds)
    assert np.array_equal(xr, xe)
    assert xr[0, 0] == 32767 and xr[0, 15] == -32768


def test_misaligned_pointer_rejected(gpu):
    import torch
    q = inputs.angle_indices(1, 2, 4, seed=0)
    plan = gpu.Plan(4, 2, q)
    buf = torch.zeros(16 * 10 + 8, dtype=torch.int16, device="cuda")
    x = buf[8:].view(10, 16)  # 16-byte offset -> aligned; shift by 1 element:
    bad = buf[1:161].view(10, 16)
    y = torch.empty((10, 16), dtype=torch.int32, device="cuda")
    plan.forward(x, out=y)
    with pytest.raises(gpu.HygtError) as e:
        plan.forward(bad, out=y)
    assert e.value.code == gpu.HYGT_ERR_ARG


# ---------------------------------------------------------------- FP32
def _rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30)


@pytest.mark.parametrize("log2n,rounds", [(1, 1), (2, 2), (3, 1), (4, 2), (5, 2), (6, 2), (6, 4), (7, 2), (8, 3)])
def test_f32_parity_from_indices(gpu, orc, log2n, rounds):
    import torch
    N = 1 << log2n
    S, B = 5, 2049
    q = inputs.angle_indices(S, rounds, log2n, seed=7)
    perms = inputs.permutations(S, rounds, N, seed=7)
    x = inputs.laplacian_blocks(B, N, 12.0, -512, 511, seed=7).astype(np.float32)
    sets = inputs.set_indices(B, S, seed=7, skip_frac=0.05)
    plan = gpu.Plan(log2n, rounds, q, perms)
    st = _status()
    y = plan.forward_f32(_t(x), _t(sets), status=st)
    xr = plan.inverse_f32(y, _t(sets), status=st)
    torch.cuda.synchronize()
    theta = inputs.theta_from_indices(q)
    ye, _ = orc.fwd_f64(x.astype(np.float64), theta, log2n, rounds, perms, sets)
    assert int(st.item()) == 0
    assert _rel_err(y.cpu().numpy().astype(np.float64), ye) <= FP_TOL
    xe, _ = orc.inv_f64(y.cpu().numpy().astype(np.float64), theta, log2n, rounds, perms, sets)
    assert _rel_err(xr.cpu().numpy().astype(np.float64), xe) <= FP_TOL


@pytest.mark.parametrize("log2n,rounds", [(4, 2), (6, 4), (8, 3)])
def test_f32_parity_free_theta(gpu, orc, log2n, rounds):
    N = 1 << log2n
    S, B = 3, 1500
    theta = inputs.theta_uniform((S, rounds, log2n, N // 2), seed=3).astype(np.float32)
    perms = inputs.permutations(S, rounds, N, seed=3)
    x = np.random.default_rng(3).standard_normal((B, N)).astype(np.float32)
    sets = inputs.set_indices(B, S, seed=3)
    plan = gpu.Plan.from_theta(log2n, rounds, theta, perms)
    y = plan.forward_f32(_t(x), _t(sets))
    ye, _ = orc.fwd_f64(x.astype(np.float64), theta.astype(np.float64), log2n, rounds, perms, sets)
    assert _rel_err(y.cpu().numpy().astype(np.float64), ye) <= FP_TOL
    with pytest.raises(gpu.HygtError) as e:
        import torch
        plan.forward(_t(x.astype(np.int16)), out=torch.empty((B, N), dtype=torch.int32, device="cuda"))
    assert e.value.code == gpu.HYGT_ERR_UNSUPPORTED


@pytest.mark.parametrize("log2n,rounds,with_perm", [(1, 2, True), (2, 1, False), (3, 2, True),
                                                  (4, 2, True), (5, 3, True), (6, 4, False),
                                                  (6, 2, True), (7, 2, True), (8, 3, True)])
def test_f32_one_set_parity(gpu, orc, log2n, rounds, with_perm):
    """FP32 forward and inverse without set indices (every block uses set 0;
    the one-set kernels): against the FP64 oracle, ragged block count."""
    import torch
    N = 1 << log2n
    S, B = 2, 5003
    theta = inputs.theta_uniform((S, rounds, log2n, N // 2), seed=11).astype(np.float32)
    perms = inputs.permutations(S, rounds, N, seed=11) if with_perm else None
    x = np.random.default_rng(11).standard_normal((B, N)).astype(np.float32)
    plan = gpu.Plan.from_theta(log2n, rounds, theta, perms)
    y = plan.forward_f32(_t(x))
    xr = plan.inverse_f32(y)
    torch.cuda.synchronize()
    ye, _ = orc.fwd_f64(x.astype(np.float64), theta.astype(np.float64), log2n, rounds, perms, None)
    assert _rel_err(y.cpu().numpy().astype(np.float64), ye) <= FP_TOL
    xe, _ = orc.inv_f64(y.cpu().numpy().astype(np.float64), theta.astype(np.float64), log2n,
                        rounds, perms, None)
    assert _rel_err(xr.cpu().numpy().astype(np.float64), xe) <= FP_TOL
    assert _rel_err(xr.cpu().numpy().astype(np.float64), x.astype(np.float64)) <= 1e-4


# ---------------------------------------------------------------- workloads
def test_workload_4x4_full(gpu, orc):
    """4x4 blocks (N=16), 2 rounds, one set, 65,536 blocks: every block."""
    from paper_2505_21728_gb300 import workloads
    w = workloads.get("hygt4x4_r2")
    d = w.generate()
    y, xr, st = run_int(gpu, w.log2n, w.rounds, d["angle_idx"], d["perms"], d["x"], d["sets"])
    ye, _ = orc.fwd_int(d["x"], d["angle_idx"], w.log2n, w.rounds, d["perms"], d["sets"])
    xe, _ = orc.inv_int(ye, d["angle_idx"], w.log2n, w.rounds, d["perms"], d["sets"])
    assert st == 0 and np.array_equal(y, ye) and np.array_equal(xr, xe)


def test_workload_8x8_105_sets_full(gpu, orc):
    """8x8 blocks (N=64), 2 rounds, 105 sets, 4,194,304 blocks, the launch
    configuration the benchmark times: every block, bit-exact."""
    from paper_2505_21728_gb300 import workloads
    w = workloads.get("hygt8x8_r2_s105")
    d = w.generate()
    y, xr, st = run_int(gpu, w.log2n, w.rounds, d["angle_idx"], d["perms"], d["x"], d["sets"])
    ye, ste = orc.fwd_int(d["x"], d["angle_idx"], w.log2n, w.rounds, d["perms"], d["sets"])
    assert ste == 0 and st == 0
    assert np.array_equal(y, ye)
    del ye
    xe, ste = orc.inv_int(y, d["angle_idx"], w.log2n, w.rounds, d["perms"], d["sets"])
    assert ste == 0
    assert np.array_equal(xr, xe)


def test_f32_workload_16x16_full(gpu, orc):
    """FP32 path of the 16x16 / 3-round / 16-set workload on all 16,777,216
    blocks (set indices given): forward and inverse within the FP32 bound
    (max abs error <= 1e-5 x max abs value over the whole batch), compared in
    chunks of 1,048,576 blocks."""
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get("hygt16x16_r3_s16")
    d = w.generate()
    n = w.nblocks
    plan = gpu.Plan(w.log2n, w.rounds, d["angle_idx"], d["perms"])
    ds = _t(d["sets"])
    st = _status()
    xf = _t(d["x"]).float()
    y = plan.forward_f32(xf, ds, status=st)
    xr = plan.inverse_f32(y, ds, status=st)
    # the same through the set-bucketed FP32 kernels
    b = gpu.Batch(plan, n).build(ds)
    yb = b.forward_f32(xf, status=st)
    xrb = b.inverse_f32(yb, status=st)
    del xf
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    theta = inputs.theta_from_indices(d["angle_idx"])
    CH = 1 << 20
    err = {"y": 0.0, "x": 0.0, "yb": 0.0, "xb": 0.0}
    max_y = max_x = 0.0
    for off in range(0, n, CH):
        sl = slice(off, min(n, off + CH))
        ye, _ = orc.fwd_f64(d["x"][sl].astype(np.float64), theta, w.log2n, w.rounds, d["perms"],
                            d["sets"][sl])
        max_y = max(max_y, float(np.max(np.abs(ye))))
        xe, _ = orc.inv_f64(ye, theta, w.log2n, w.rounds, d["perms"], d["sets"][sl])
        max_x = max(max_x, float(np.max(np.abs(xe))))
        for key, out, ref in (("y", y, ye), ("yb", yb, ye), ("x", xr, xe), ("xb", xrb, xe)):
            e = float(np.max(np.abs(out[sl].cpu().numpy().astype(np.float64) - ref)))
            err[key] = max(err[key], e)
    # the inverse input is each path's own forward output; its error includes the forward's
    assert err["y"] <= FP_TOL * max_y and err["yb"] <= FP_TOL * max_y, err
    assert err["x"] <= 2 * FP_TOL * max_x and err["xb"] <= 2 * FP_TOL * max_x, err
