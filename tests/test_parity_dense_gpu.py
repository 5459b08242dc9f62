"""Parity of the dense matrix-transform baseline with the CPU oracle.

Integer kernel: bit-exact against the oracle's int64 matrix product.
BF16 tensor-core kernel: against the FP64 product of the BF16-rounded
matrices and inputs (the kernel's FP32 accumulation error is <= N 2^-24 of
the sum of |terms|), and within BF16 accuracy of the exact FP64 product."""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bf16_round(a):
    """Round-to-nearest-even to BF16, returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def e4m3_round(a):
    """Round-to-nearest-even to FP8 E4M3 (4 exponent bits, bias 7, 3 mantissa
    bits, subnormals below 2^-6), saturating at +-448; returned as float64."""
    a = np.asarray(a, np.float64)
    m = np.abs(a)
    e = np.maximum(np.floor(np.log2(np.where(m > 0, m, 1.0))), -6.0)
    q = 2.0 ** (e - 3)  # spacing of the binade
    r = np.minimum(np.round(m / q) * q, 448.0)  # np.round: half to even
    return np.sign(a) * r


def hygt_matrices(orc, log2n, rounds, S, seed):
    N = 1 << log2n
    theta = inputs.theta_uniform((S, rounds, log2n, N // 2), seed=seed)
    perms = inputs.permutations(S, rounds, N, seed=seed)
    return np.stack([orc.dense_f64(theta[s], log2n, rounds, perms[s]) for s in range(S)])


@pytest.mark.parametrize("log2n,S,B", [(4, 3, 1000), (6, 7, 3001), (6, 105, 20000)])
def test_dense_int_bit_exact(gpu, orc, log2n, S, B):
    import torch
    N = 1 << log2n
    K = hygt_matrices(orc, log2n, 2, S, seed=log2n)
    K_int = np.sign(256 * K) * np.floor(np.abs(256 * K) + 0.5)  # round half away from zero
    x = inputs.laplacian_blocks(B, N, 30.0, -1024, 1023, seed=1)
    sets = inputs.set_indices(B, S, seed=1, skip_frac=0.05)
    d = gpu.DenseKLT(log2n, K.astype(np.float32)).build(_t(sets), B)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = d.apply(_t(x), kind=gpu.DENSE_KLT_INT, status=st).cpu().numpy()
    K_int_f32 = np.sign(256 * K.astype(np.float32).astype(np.float64)) * \
        np.floor(np.abs(256 * K.astype(np.float32).astype(np.float64)) + 0.5)
    ye, ste = orc.dense_apply_int(x, K_int_f32.astype(np.int32), 8, sets)
    assert ste == 0 and int(st.item()) == 0
    assert np.array_equal(y, ye)


# the larger cases give every CTA of the persistent launch many tiles (deep
# pipelining) and, with 105 sets, several changes of the set matrix
@pytest.mark.parametrize("log2n,S,B", [(6, 5, 2000), (6, 105, 30000), (8, 4, 1500),
                                       (6, 2, 200000), (6, 105, 400000), (8, 3, 40000)])
def test_dense_bf16_tensor_cores(gpu, orc, log2n, S, B):
    import torch
    N = 1 << log2n
    K = hygt_matrices(orc, log2n, 2, S, seed=2 * log2n)
    x = inputs.laplacian_blocks(B, N, 60.0, -2048, 2047, seed=3)
    sets = inputs.set_indices(B, S, seed=3, skip_frac=0.05)
    d = gpu.DenseKLT(log2n, K.astype(np.float32)).build(_t(sets), B)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = d.apply(_t(x), kind=gpu.DENSE_KLT_BF16, status=st).cpu().numpy().astype(np.float64)
    assert int(st.item()) == 0
    Kb = bf16_round(K.astype(np.float32))
    xb = bf16_round(x.astype(np.float32))
    yb, _ = orc.dense_apply_f64(xb, Kb, sets)
    skip = sets == 0xFFFF
    yb[skip] = x[skip]
    scale = np.einsum("bij,bj->bi", np.abs(Kb[np.where(skip, 0, sets)]), np.abs(xb))
    assert np.all(np.abs(y - yb) <= N * 2.0 ** -23 * scale + 1e-9)
    ye, _ = orc.dense_apply_f64(x.astype(np.float64), K, sets)
    ye[skip] = x[skip]
    rel = np.max(np.abs(y - ye)) / np.max(np.abs(ye))
    assert rel < 2 ** -7  # BF16 has 8 significant bits


def test_e4m3_rounding_reference():
    """The test's E4M3 rounding against values fixed by the format."""
    v = np.array([0.0, 1.0, 1.0625, 1.1875, 448.0, 460.0, 470.0, 1e6, -3.3, 2.0 ** -9,
                  2.0 ** -10, 3 * 2.0 ** -11, 0.013671875])
    want = np.array([0.0, 1.0, 1.0, 1.25, 448.0, 448.0, 448.0, 448.0, -3.25, 2.0 ** -9,
                     0.0, 2.0 ** -9, 0.013671875])
    assert np.array_equal(e4m3_round(v), want)


@pytest.mark.parametrize("log2n,S,B", [(6, 5, 3000), (6, 105, 200000), (8, 3, 20000)])
def test_dense_fp8_tensor_cores(gpu, orc, log2n, S, B):
    """E4M3 x E4M3 with FP32 accumulation: equal to the FP64 product of the
    same E4M3-rounded, scaled operands within FP32 accumulation error, and
    within the E4M3 precision of the exact transform."""
    import torch
    N = 1 << log2n
    K = hygt_matrices(orc, log2n, 2, S, seed=3 * log2n).astype(np.float32)
    x = inputs.laplacian_blocks(B, N, 60.0, -2048, 2047, seed=5)
    sets = inputs.set_indices(B, S, seed=5, skip_frac=0.05)
    d = gpu.DenseKLT(log2n, K).build(_t(sets), B)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = d.apply(_t(x), kind=gpu.DENSE_KLT_FP8, status=st).cpu().numpy().astype(np.float64)
    assert int(st.item()) == 0
    # operands as the library forms them (FP32 scale factors, E4M3 rounding)
    kamax = np.abs(K).reshape(S, -1).max(axis=1).astype(np.float32)
    kinv = np.float32(448.0) / kamax
    kscale = kamax / np.float32(448.0)
    K8 = e4m3_round((K * kinv[:, None, None]).astype(np.float32))
    xamax = np.abs(x.astype(np.int32)).max(axis=1).astype(np.float32)
    xinv = np.where(xamax > 0, np.float32(448.0) / np.maximum(xamax, 1), np.float32(1.0))
    xscale = np.where(xamax > 0, xamax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    x8 = e4m3_round((x.astype(np.float32) * xinv[:, None].astype(np.float32)).astype(np.float32))
    osc = (xscale * kscale[np.where(sets == 0xFFFF, 0, np.minimum(sets, S - 1))]).astype(np.float32)
    skip = sets == 0xFFFF
    kk = K8[np.where(skip, 0, sets)]
    yq = np.einsum("bij,bj->bi", kk, x8) * osc[:, None].astype(np.float64)
    scale = np.einsum("bij,bj->bi", np.abs(kk), np.abs(x8)) * osc[:, None].astype(np.float64)
    yq[skip] = x[skip]
    scale[skip] = 0.0
    assert np.all(np.abs(y - yq) <= (N * 2.0 ** -23 + 2.0 ** -22) * scale + 1e-9)
    ye, _ = orc.dense_apply_f64(x.astype(np.float64), K.astype(np.float64), sets)
    ye[skip] = x[skip]
    rel = np.max(np.abs(y - ye)) / np.max(np.abs(ye))
    assert rel < 2 ** -3  # E4M3 has 4 significant bits


def test_dense_bad_set_and_empty(gpu, orc):
    import torch
    K = hygt_matrices(orc, 6, 2, 3, seed=9)
    x = inputs.laplacian_blocks(300, 64, 20.0, -512, 511, seed=9)
    sets = inputs.set_indices(300, 3, seed=9)
    sets[10] = 77
    d = gpu.DenseKLT(6, K.astype(np.float32)).build(_t(sets), 300)
    for kind in (gpu.DENSE_KLT_BF16, gpu.DENSE_KLT_INT, gpu.DENSE_KLT_FP8):
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        y = d.apply(_t(x), kind=kind, status=st).cpu().numpy()
        assert int(st.item()) == 4 and np.all(y[10] == 0)


def test_stress_workload_paths_error_vs_fp64(gpu, orc, capsys):
    """The large-transform workload (16x16 blocks, N = 256, 3 rounds, 16 sets):
    every path's error against the FP64 oracle on its first 65,536 blocks --
    the exact integer HyGT (rounding per pass, within the integer-vs-float
    bound), the FP32 HyGT (<= 1e-5 of max |y|), and the dense 256 x 256
    matrix transform with BF16 and FP8 E4M3 tensor cores (within the
    precision of their operands).  The errors are printed."""
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.truncated(workloads.get("hygt16x16_r3_s16"), 65536)
    d = w.generate()
    N, n = w.N, w.nblocks
    theta = inputs.theta_from_indices(d["angle_idx"])
    ye, st = orc.fwd_f64(d["x"].astype(np.float64), theta, w.log2n, w.rounds, d["perms"],
                         d["sets"])
    assert st == 0
    scale = np.max(np.abs(ye))
    plan = gpu.Plan(w.log2n, w.rounds, d["angle_idx"], d["perms"])
    x, s = _t(d["x"]), _t(d["sets"])
    y_int = gpu.Batch(plan, n).build(s).forward(x).cpu().numpy().astype(np.float64)
    y_f32 = plan.forward_f32(x.float(), s).cpu().numpy().astype(np.float64)
    dk = gpu.DenseKLT(w.log2n, plan.dense_matrices()).build(s, n)
    y_bf16 = dk.apply(x, kind=gpu.DENSE_KLT_BF16).cpu().numpy().astype(np.float64)
    y_fp8 = dk.apply(x, kind=gpu.DENSE_KLT_FP8).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    errs = {k: float(np.max(np.abs(v - ye))) for k, v in
            (("int32", y_int), ("fp32", y_f32), ("bf16", y_bf16), ("fp8_e4m3", y_fp8))}
    with capsys.disabled():
        print("\nstress 16x16 max|y|=%.1f; max abs error vs FP64: %s" % (
            scale, ", ".join("%s %.4g (%.2e rel)" % (k, e, e / scale) for k, e in errs.items())))
    # integer: table quantisation (|c - 256 cos| <= 1/2) and 1/2 per pass, 24 passes
    assert errs["int32"] <= 24 * 0.5 + 24 * scale / 256.0
    assert errs["fp32"] <= 1e-5 * scale
    assert errs["bf16"] <= 2.0 ** -7 * 4 * scale      # BF16 operands (8-bit mantissa)
    assert errs["fp8_e4m3"] <= 2.0 ** -3 * 4 * scale  # E4M3 operands (3-bit mantissa)
    assert errs["fp8_e4m3"] > errs["bf16"] > errs["fp32"]
    dk.close()
    plan.close()
