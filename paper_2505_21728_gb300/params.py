"""Saving and loading HyGT transform parameters (checkpoint / resume).

A parameter file is one ``.npz`` archive (read without pickle) holding a JSON
header and the arrays of every set:

    header     JSON: {"format": "hygt-params", "version": 1, "log2n", "rounds",
               "num_sets", "kind": "int" | "float", "angle_bits", "frac_bits"}
    angle_idx  uint8   [S][R][log2 N][N/2]  kind "int": angle indices q, theta = 2 pi q / 2^angle_bits
    theta      float32 [S][R][log2 N][N/2]  kind "float": free angles in radians
    perms      uint16  [S][R][N]            optional: the gather permutation of each round's slot

The angle layout is the one every entry point uses: set, round, pass, pair
(pair j of pass p joins the j-th index m with bit p clear to m + 2^p, Sec. IV).
``load_params`` checks the header against the arrays before anything is built
from them.
"""
from __future__ import annotations

import json

import numpy as np

FORMAT = "hygt-params"
VERSION = 1
MAX_LOG2N = 8
MAX_ROUNDS = 8

__all__ = ["save_params", "load_params", "plan_from_params", "FORMAT", "VERSION"]


def _shape(log2n, rounds, num_sets):
    return (num_sets, rounds, log2n, (1 << log2n) // 2)


def _check(log2n, rounds, num_sets, kind, angles, perms, angle_bits):
    if not (1 <= log2n <= MAX_LOG2N) or not (1 <= rounds <= MAX_ROUNDS) or num_sets < 1:
        raise ValueError("log2n must be 1..%d, rounds 1..%d, num_sets >= 1" % (MAX_LOG2N, MAX_ROUNDS))
    if tuple(angles.shape) != _shape(log2n, rounds, num_sets):
        raise ValueError("angles have shape %s, expected %s"
                         % (tuple(angles.shape), _shape(log2n, rounds, num_sets)))
    if kind == "int":
        if angles.dtype != np.uint8:
            raise ValueError("angle indices must be uint8")
        if not (1 <= angle_bits <= 8) or int(angles.max(initial=0)) >> angle_bits:
            raise ValueError("angle indices must be below 2^angle_bits")
    elif kind == "float":
        if angles.dtype != np.float32 or not np.all(np.isfinite(angles)):
            raise ValueError("angles must be finite float32")
    else:
        raise ValueError("kind must be 'int' or 'float'")
    if perms is not None:
        N = 1 << log2n
        if perms.dtype != np.uint16 or tuple(perms.shape) != (num_sets, rounds, N):
            raise ValueError("perms must be uint16 [%d][%d][%d]" % (num_sets, rounds, N))
        if not np.array_equal(np.sort(perms, axis=-1),
                              np.broadcast_to(np.arange(N, dtype=np.uint16), perms.shape)):
            raise ValueError("every permutation slot must be a permutation of 0..N-1")


def save_params(path, log2n, rounds, angle_idx=None, theta=None, perms=None, angle_bits=8,
                frac_bits=8):
    """Write one parameter file: integer angle indices or free FP32 angles
    (exactly one of the two), and optional permutation slots."""
    if (angle_idx is None) == (theta is None):
        raise ValueError("give exactly one of angle_idx and theta")
    kind = "int" if angle_idx is not None else "float"
    angles = np.ascontiguousarray(angle_idx if kind == "int" else theta)
    if kind == "int":
        angles = angles.astype(np.uint8) if angles.dtype != np.uint8 else angles
    else:
        angles = angles.astype(np.float32)
    per_set = rounds * log2n * ((1 << log2n) // 2)
    if angles.size % per_set:
        raise ValueError("angle count is not a multiple of R log2(N) N / 2")
    num_sets = angles.size // per_set
    angles = angles.reshape(_shape(log2n, rounds, num_sets))
    p = None
    if perms is not None:
        p = np.ascontiguousarray(perms).astype(np.uint16).reshape(num_sets, rounds, 1 << log2n)
    _check(log2n, rounds, num_sets, kind, angles, p, angle_bits)
    header = {"format": FORMAT, "version": VERSION, "log2n": int(log2n), "rounds": int(rounds),
              "num_sets": int(num_sets), "kind": kind, "angle_bits": int(angle_bits),
              "frac_bits": int(frac_bits)}
    arrays = {"header": np.frombuffer(json.dumps(header).encode(), dtype=np.uint8),
              ("angle_idx" if kind == "int" else "theta"): angles}
    if p is not None:
        arrays["perms"] = p
    with open(path, "wb") as f:
        np.savez(f, **arrays)


def load_params(path):
    """Read and check a parameter file; returns a dict with the header fields
    and the arrays (``angle_idx`` or ``theta``, and ``perms`` or None)."""
    with np.load(path, allow_pickle=False) as z:
        if "header" not in z.files:
            raise ValueError("not a HyGT parameter file (no header)")
        h = json.loads(bytes(z["header"]).decode())
        if h.get("format") != FORMAT or h.get("version") != VERSION:
            raise ValueError("unsupported parameter file: %r" % {k: h.get(k) for k in
                                                                  ("format", "version")})
        kind = h.get("kind")
        name = "angle_idx" if kind == "int" else "theta"
        if name not in z.files:
            raise ValueError("header says kind %r but the file has no %s" % (kind, name))
        angles = z[name]
        perms = z["perms"] if "perms" in z.files else None
    _check(h["log2n"], h["rounds"], h["num_sets"], kind, angles, perms, h["angle_bits"])
    out = dict(h)
    out[name] = angles
    out["perms"] = perms
    return out


def plan_from_params(params):
    """A ``hygt.Plan`` on the current CUDA device from ``load_params``' result."""
    from . import hygt
    if params["kind"] == "int":
        return hygt.Plan(params["log2n"], params["rounds"], params["angle_idx"], params["perms"],
                         angle_bits=params["angle_bits"], frac_bits=params["frac_bits"])
    return hygt.Plan.from_theta(params["log2n"], params["rounds"], params["theta"],
                                params["perms"])
