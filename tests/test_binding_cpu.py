"""Argument checks of the Python binding that run before any library call
(no GPU): buffers whose size or type does not match the batch are refused
instead of being handed to the C ABI as raw pointers."""
import types

import pytest

from paper_2505_21728_gb300 import build as hb


@pytest.fixture(scope="module")
def hygt():
    hb.build()
    from paper_2505_21728_gb300 import hygt as h
    return h


def _pipe(hygt, N=64):
    p = hygt.HostPipe.__new__(hygt.HostPipe)
    p.plan = types.SimpleNamespace(N=N)
    p.handle = None
    return p


def test_host_pipe_rejects_mismatched_outputs(hygt):
    import torch
    p = _pipe(hygt)
    x = torch.zeros((4, 64), dtype=torch.int16)
    with pytest.raises(ValueError, match="y must be"):
        p.roundtrip(x, y=torch.empty((3, 64), dtype=torch.int32))
    with pytest.raises(ValueError, match="y must be"):
        p.roundtrip(x, y=torch.empty((4, 64), dtype=torch.int16))
    with pytest.raises(ValueError, match="xr must be"):
        p.roundtrip(x, xr=torch.empty((4, 32), dtype=torch.int16))
    with pytest.raises(ValueError, match="xr must be"):
        p.roundtrip(x, xr=torch.empty((64, 4), dtype=torch.int16).t())
    with pytest.raises(ValueError, match="x must be"):
        p.roundtrip(torch.zeros((4, 32), dtype=torch.int16))
    with pytest.raises(ValueError, match="sets must be"):
        p.roundtrip(x, sets=torch.zeros(3, dtype=torch.int16))


def _dense(hygt, nblocks=None, work=None):
    d = hygt.DenseKLT.__new__(hygt.DenseKLT)
    d.log2n, d.N, d.num_sets, d.handle = 6, 64, 3, None
    d.work, d.nblocks = work, nblocks
    return d


def test_dense_apply_needs_a_matching_schedule(hygt):
    import torch
    x = torch.zeros((10, 64), dtype=torch.int16)
    with pytest.raises(RuntimeError, match="before build"):
        _dense(hygt).apply(x)
    d = _dense(hygt, nblocks=12, work=torch.zeros(1, dtype=torch.uint8))
    with pytest.raises(ValueError, match="built for 12 blocks"):
        d.apply(x)
    d = _dense(hygt, nblocks=10, work=torch.zeros(1, dtype=torch.uint8))
    with pytest.raises(ValueError, match="out must have shape"):
        d.apply(x, out=torch.empty((9, 64), dtype=torch.float32))


def test_dense_build_needs_one_set_per_block(hygt):
    import torch
    with pytest.raises(ValueError, match="one entry per block"):
        _dense(hygt).build(torch.zeros(5, dtype=torch.int16), 6)
