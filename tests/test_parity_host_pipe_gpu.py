"""The host-buffer round trip (hygt_host_roundtrip): chunked forward +
inverse of a batch in host memory, bit-exact against the oracle, including
a ragged last chunk, no set indices, and an out-of-range set index."""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu


def _host(a, pinned=True):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("log2n,rounds,S,B,chunk,pinned", [
    (6, 2, 105, 300001, 65536, True),   # five chunks, ragged last one
    (4, 2, 3, 70000, 1 << 19, True),    # one chunk
    (8, 3, 4, 20000, 4096, False),      # pageable host memory
])
def test_host_roundtrip_parity(gpu, orc, log2n, rounds, S, B, chunk, pinned):
    N = 1 << log2n
    q = inputs.angle_indices(S, rounds, log2n, seed=21)
    perms = inputs.permutations(S, rounds, N, seed=21)
    x = inputs.laplacian_blocks(B, N, 30.0, -32768, 32767, seed=21)
    sets = inputs.set_indices(B, S, seed=21, skip_frac=0.05)
    plan = gpu.Plan(log2n, rounds, q, perms)
    pipe = gpu.HostPipe(plan, chunk)
    y, xr, status = pipe.roundtrip(_host(x, pinned), _host(sets, pinned))
    assert status == 0
    ye, _ = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert np.array_equal(y.numpy(), ye)
    assert np.array_equal(xr.numpy(), xe)
    pipe.close()


def test_host_roundtrip_no_sets_and_bad_set(gpu, orc):
    N, rounds, S, B = 64, 2, 5, 50000
    q = inputs.angle_indices(S, rounds, 6, seed=22)
    x = inputs.laplacian_blocks(B, N, 10.0, -1024, 1023, seed=22)
    plan = gpu.Plan(6, rounds, q, None)
    pipe = gpu.HostPipe(plan, 16384)
    y, xr, status = pipe.roundtrip(_host(x))
    assert status == 0
    ye, _ = orc.fwd_int(x, q, 6, rounds, None, None)
    assert np.array_equal(y.numpy(), ye)
    sets = inputs.set_indices(B, S, seed=22)
    sets[40000] = 77
    y, xr, status = pipe.roundtrip(_host(x), _host(sets))
    assert status == gpu.HYGT_ERR_SET_INDEX
    assert np.all(y.numpy()[40000] == 0)
    ye, _ = orc.fwd_int(x, q, 6, rounds, None, sets)
    assert np.array_equal(y.numpy(), ye)
    pipe.close()


def test_host_roundtrip_reconstruction_only(gpu, orc):
    """With no coefficient buffer only the reconstruction comes back; it
    equals the oracle's inverse of its forward."""
    import torch
    log2n, rounds, S, B = 6, 2, 105, 300007
    N = 1 << log2n
    q = inputs.angle_indices(S, rounds, log2n, seed=12)
    perms = inputs.permutations(S, rounds, N, seed=12)
    x = inputs.laplacian_blocks(B, N, 8.0, -1024, 1023, seed=12)
    sets = inputs.set_indices(B, S, seed=12, skip_frac=0.1)
    plan = gpu.Plan(log2n, rounds, q, perms)
    pipe = gpu.HostPipe(plan, 65536)
    y, xr, status = pipe.roundtrip(torch.from_numpy(x).pin_memory(),
                                   torch.from_numpy(sets.view(np.int16)).pin_memory(),
                                   coefficients=False)
    assert y is None and status == 0
    ye, _ = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert np.array_equal(xr.numpy(), xe)
    pipe.close()
    plan.close()
