"""Parity of the fused secondary-transform kernel (Sec. VI: integer DCT-II
primary, HyGT on the top-left 4x4 / 8x8 coefficients) with the oracle: bit
for bit, forward and inverse, for 4x4, 8x8, 16x16 and 32x32 blocks, 105
sets, permutation slots, the skip sentinel (primary only) and bad set
indices, ragged batch sizes."""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("log2m,B", [(2, 20011), (3, 9001), (4, 3001), (5, 777)])
@pytest.mark.parametrize("rounds,perm_kind", [(2, "between"), (3, "all")])
def test_secondary_bit_exact(gpu, orc, log2m, B, rounds, perm_kind):
    import torch
    log2n = 4 if log2m == 2 else 6
    N, S, M = 1 << log2n, 105, 1 << log2m
    q = inputs.angle_indices(S, rounds, log2n, seed=log2m + rounds)
    perms = inputs.permutations(S, rounds, N, seed=log2m,
                                between_rounds_only=(perm_kind == "between"))
    x = inputs.laplacian_blocks(B, M * M, 30.0, -32768, 32767, seed=log2m)
    sets = inputs.set_indices(B, S, seed=log2m, skip_frac=0.1)
    plan = gpu.Plan(log2n, rounds, q, perms)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ds = _t(sets)
    y = plan.secondary_forward(_t(x), log2m, ds, status=st)
    xr = plan.secondary_inverse(y, log2m, ds, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ye, s1 = orc.secondary_fwd(x, log2m, q, log2n, rounds, perms, sets)
    xe, s2 = orc.secondary_inv(ye, log2m, q, log2n, rounds, perms, sets)
    assert s1 == s2 == 0
    assert np.array_equal(y.cpu().numpy(), ye)
    assert np.array_equal(xr.cpu().numpy(), xe)
    plan.close()


def test_secondary_frame_of_8x8_blocks(gpu, orc):
    """A 3840x2160 frame tiled into 8x8 blocks (129,600 blocks), Laplacian
    residuals clipped to [-1024, 1023], set index uniform over 105 sets with
    10% of the blocks transformed by the primary alone."""
    import torch
    log2m, log2n, R, S, B = 3, 6, 2, 105, 129600
    q = inputs.angle_indices(S, R, log2n, seed=11)
    perms = inputs.permutations(S, R, 64, seed=11)
    x = inputs.laplacian_blocks(B, 64, 8.0, -1024, 1023, seed=11)
    sets = inputs.set_indices(B, S, seed=11, skip_frac=0.1)
    plan = gpu.Plan(log2n, R, q, perms)
    y = plan.secondary_forward(_t(x), log2m, _t(sets))
    xr = plan.secondary_inverse(y, log2m, _t(sets))
    ye, _ = orc.secondary_fwd(x, log2m, q, log2n, R, perms, sets)
    xe, _ = orc.secondary_inv(ye, log2m, q, log2n, R, perms, sets)
    assert np.array_equal(y.cpu().numpy(), ye)
    assert np.array_equal(xr.cpu().numpy(), xe)
    torch.cuda.synchronize()
    plan.close()


def test_secondary_bad_sets_and_arguments(gpu, orc):
    import torch
    log2m, log2n, R, S = 3, 6, 2, 4
    q = inputs.angle_indices(S, R, log2n, seed=1)
    x = inputs.laplacian_blocks(9, 64, 50.0, -1024, 1023, seed=2)
    sets = np.array([0, 1, 2, 3, 4, 0xFFFF, 100, 1, 0], np.uint16)
    plan = gpu.Plan(log2n, R, q)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = plan.secondary_forward(_t(x), log2m, _t(sets), status=st)
    ye, ste = orc.secondary_fwd(x, log2m, q, log2n, R, None, sets)
    assert ste == orc.ERR_SET and int(st.item()) == gpu.HYGT_ERR_SET_INDEX
    assert np.array_equal(y.cpu().numpy(), ye)
    # a 4x4 block needs the 4x4 secondary; FP32 plans are refused
    with pytest.raises(gpu.HygtError):
        plan.secondary_forward(_t(np.zeros((3, 16), np.int16)), 2)
    fp = gpu.Plan.from_theta(log2n, R, np.zeros(R * log2n * 32, np.float32))
    with pytest.raises(gpu.HygtError):
        fp.secondary_forward(_t(x), log2m)
    e = plan.secondary_forward(torch.zeros((0, 64), dtype=torch.int16, device="cuda"), log2m)
    assert e.shape == (0, 64)
    fp.close()
    plan.close()


@pytest.mark.parametrize("log2m,B", [(2, 30011), (3, 12007)])
@pytest.mark.parametrize("rounds,perm_kind", [(2, "between"), (3, "all")])
def test_secondary_fused_bucketed_bit_exact(gpu, orc, log2m, B, rounds, perm_kind):
    """4x4 and 8x8 blocks through the bucketed kernels with the primary
    fused: bit for bit the oracle (skip and bad set indices included), for
    the default launch and every staging choice."""
    import torch
    log2n = 2 * log2m
    N, S, M = 1 << log2n, 105, 1 << log2m
    q = inputs.angle_indices(S, rounds, log2n, seed=log2m + 9 * rounds)
    perms = inputs.permutations(S, rounds, N, seed=log2m + 1,
                                between_rounds_only=(perm_kind == "between"))
    x = inputs.laplacian_blocks(B, M * M, 30.0, -32768, 32767, seed=log2m + 5)
    sets = inputs.set_indices(B, S, seed=log2m + 6, skip_frac=0.1)
    sets[11] = 999
    ye, s1 = orc.secondary_fwd(x, log2m, q, log2n, rounds, perms, sets)
    xe, s2 = orc.secondary_inv(ye, log2m, q, log2n, rounds, perms, sets)
    assert s1 == s2 == orc.ERR_SET
    plan = gpu.Plan(log2n, rounds, q, perms)
    b = gpu.Batch(plan, B).build(_t(sets))
    for stage in (-1, 0, 1, 2, 3):
        for inv in (0, 1):
            assert gpu.hygt_batch_set_tuning(plan.handle, inv, 0, 0, stage) == gpu.HYGT_OK
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        y = b.secondary_forward(_t(x), log2m, status=st)
        xr = b.secondary_inverse(_t(ye), log2m, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == gpu.HYGT_ERR_SET_INDEX
        assert np.array_equal(y.cpu().numpy(), ye), stage
        assert np.array_equal(xr.cpu().numpy(), xe), stage
    plan.close()
