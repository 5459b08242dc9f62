"""hygt_forward_static: the integer forward for callers that cannot allocate
device memory when they transform (it keeps its schedule in a fixed array
the library holds on every GPU, instead of a caller workspace).

Its output must equal the workspace path (hygt_batch_build +
hygt_forward_batch) bit for bit, on two calls in a row (the array keeps the
previous call's schedule), and a batch larger than the array must be
refused before anything runs.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("log2n", [4, 6])
def test_static_scratch_forward_matches_workspace_path(gpu, log2n):
    import torch
    rounds, S, N = 2, 105, 1 << log2n
    q = inputs.angle_indices(S, rounds, log2n, seed=21)
    perms = inputs.permutations(S, rounds, N, seed=21)
    plan = gpu.Plan(log2n, rounds, q, perms)
    stream = torch.cuda.current_stream().cuda_stream
    for call, B in enumerate([200003, 77777]):  # two calls in a row, different sizes
        x = inputs.laplacian_blocks(B, N, 8.0, -1024, 1023, seed=30 + call)
        sets = inputs.set_indices(B, S, seed=30 + call, skip_frac=0.1)
        dx, ds = _t(x), _t(sets)
        ref = gpu.Batch(plan, B).build(ds).forward(dx)
        y = torch.full((B, N), -7, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        code = gpu.hygt_forward_static(plan.handle, dx.data_ptr(), y.data_ptr(), ds.data_ptr(),
                                       B, stream, st.data_ptr())
        assert code == gpu.HYGT_OK
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert torch.equal(y, ref)


def test_static_scratch_rejects_oversized_batch(gpu):
    """The smallest batch whose schedule no longer fits is refused.  Its
    buffers are allocated in full, so a regression of the size check would
    give a wrong return code, not an access past the end of a buffer."""
    import torch
    q = inputs.angle_indices(4, 2, 6, seed=1)
    plan = gpu.Plan(6, 2, q)
    lo, hi = 1, 4_000_000  # the 8 MiB limit lies between these block counts
    assert gpu.hygt_batch_workspace_bytes(plan.handle, hi) > 8 << 20
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if gpu.hygt_batch_workspace_bytes(plan.handle, mid) > 8 << 20:
            hi = mid
        else:
            lo = mid
    B = hi
    x = torch.zeros((B, 64), dtype=torch.int16, device="cuda")
    y = torch.zeros((B, 64), dtype=torch.int32, device="cuda")
    s = torch.zeros(B, dtype=torch.int16, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = gpu.hygt_forward_static(plan.handle, x.data_ptr(), y.data_ptr(), s.data_ptr(), B,
                                   stream, st.data_ptr())
    assert code == gpu.HYGT_ERR_TOO_LARGE
    assert "static scratch" in gpu.hygt_status_string(code)
    # one block fewer fits, and runs
    code = gpu.hygt_forward_static(plan.handle, x.data_ptr(), y.data_ptr(), s.data_ptr(), lo,
                                   stream, st.data_ptr())
    assert code == gpu.HYGT_OK
    torch.cuda.synchronize()
    assert int(st.item()) == 0
