"""Parameter files (checkpoint / resume of the transform angles), CPU only:
round trips of integer and FP32 parameters, and refusal of files whose
header and arrays disagree."""
import json

import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs, params


def test_round_trip_integer(tmp_path):
    S, R, log2n = 105, 2, 6
    q = inputs.angle_indices(S, R, log2n, seed=4)
    perms = inputs.permutations(S, R, 64, seed=4)
    f = tmp_path / "p.npz"
    params.save_params(f, log2n, R, angle_idx=q, perms=perms)
    p = params.load_params(f)
    assert (p["kind"], p["log2n"], p["rounds"], p["num_sets"]) == ("int", 6, 2, 105)
    assert (p["angle_bits"], p["frac_bits"]) == (8, 8)
    assert np.array_equal(p["angle_idx"], np.asarray(q).reshape(S, R, log2n, 32))
    assert np.array_equal(p["perms"], np.asarray(perms).reshape(S, R, 64))


def test_round_trip_float_without_perms(tmp_path):
    rng = np.random.default_rng(0)
    th = rng.uniform(-np.pi, np.pi, size=(1, 4, 6, 32)).astype(np.float32)
    f = tmp_path / "t.npz"
    params.save_params(f, 6, 4, theta=th)
    p = params.load_params(f)
    assert p["kind"] == "float" and p["perms"] is None
    assert np.array_equal(p["theta"], th)


def test_save_refuses_bad_parameters(tmp_path):
    f = tmp_path / "x.npz"
    q = np.zeros((2, 2, 4, 8), np.uint8)
    with pytest.raises(ValueError, match="exactly one"):
        params.save_params(f, 4, 2)
    with pytest.raises(ValueError, match="exactly one"):
        params.save_params(f, 4, 2, angle_idx=q, theta=q.astype(np.float32))
    with pytest.raises(ValueError, match="multiple"):
        params.save_params(f, 4, 2, angle_idx=np.zeros(7, np.uint8))
    with pytest.raises(ValueError, match="below 2"):
        params.save_params(f, 4, 2, angle_idx=q + 16, angle_bits=4)
    bad = np.tile(np.arange(16, dtype=np.uint16), (2, 2, 1))
    bad[1, 0, 3] = 2  # a repeated index
    with pytest.raises(ValueError, match="permutation"):
        params.save_params(f, 4, 2, angle_idx=q, perms=bad)
    with pytest.raises(ValueError, match="finite"):
        params.save_params(f, 4, 2, theta=np.full((1, 2, 4, 8), np.nan, np.float32))
    with pytest.raises(ValueError, match="log2n"):
        params.save_params(f, 9, 1, angle_idx=np.zeros(9 * 256, np.uint8))


def _write_raw(path, header, **arrays):
    with open(path, "wb") as fh:
        np.savez(fh, header=np.frombuffer(json.dumps(header).encode(), dtype=np.uint8), **arrays)


def test_load_refuses_inconsistent_files(tmp_path):
    good = {"format": "hygt-params", "version": 1, "log2n": 4, "rounds": 2, "num_sets": 3,
            "kind": "int", "angle_bits": 8, "frac_bits": 8}
    q = np.zeros((3, 2, 4, 8), np.uint8)
    f = tmp_path / "r.npz"
    _write_raw(f, good, angle_idx=q)
    assert params.load_params(f)["num_sets"] == 3
    _write_raw(f, dict(good, num_sets=4), angle_idx=q)
    with pytest.raises(ValueError, match="shape"):
        params.load_params(f)
    _write_raw(f, dict(good, version=2), angle_idx=q)
    with pytest.raises(ValueError, match="unsupported"):
        params.load_params(f)
    _write_raw(f, dict(good, kind="float"), angle_idx=q)
    with pytest.raises(ValueError, match="no theta"):
        params.load_params(f)
    _write_raw(f, good, angle_idx=q, perms=np.zeros((3, 2, 16), np.uint16))
    with pytest.raises(ValueError, match="permutation"):
        params.load_params(f)
    with open(f, "wb") as fh:
        np.savez(fh, angle_idx=q)
    with pytest.raises(ValueError, match="no header"):
        params.load_params(f)
