"""ctypes binding of the C oracle in ``hygt_oracle.c`` (test infrastructure only).

The oracle is a plain, slow, single-file C implementation of the
Hypercube-Givens Transform (Said et al., Sec. III-IV), in int64 and FP64.
``build()`` compiles it with gcc; the wrappers below only marshal numpy
arrays.  Nothing here is used by the CUDA library; see the header of
``hygt_oracle.c`` for the definitions it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

__all__ = [
    "build", "lib", "OK", "ERR_ARG", "ERR_SET", "ERR_OVERFLOW", "SKIP",
    "pair", "cs_table", "fwd_int", "inv_int", "fwd_f64", "inv_f64", "dense_f64",
    "loss_grad_f64", "loss_f64", "dense_apply_f64", "dense_apply_int",
    "num_threads", "set_num_threads", "pmpt_fwd_int", "pmpt_inv_int", "pmpt_fwd_f64",
    "pmpt_inv_f64", "dct_matrix", "secondary_fwd", "secondary_inv",
]

OK, ERR_ARG, ERR_SET, ERR_OVERFLOW = 0, 1, 4, 5
SKIP = 0xFFFF

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hygt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) and return the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int, ctypes.c_int64
        L.oracle_num_threads.restype = i32
        L.oracle_set_num_threads.argtypes = [i32]
        L.oracle_pair.argtypes = [i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.oracle_cs_table.argtypes = [i32, i32, P, P]
        L.oracle_cs_table.restype = i32
        for name in ("oracle_fwd_int", "oracle_inv_int"):
            f = getattr(L, name)
            f.argtypes = [i32, i32, i32, P, P, i32, i32, P, P, i64, P]
            f.restype = i32
        for name in ("oracle_fwd_f64", "oracle_inv_f64"):
            f = getattr(L, name)
            f.argtypes = [i32, i32, i32, P, P, P, P, i64, P]
            f.restype = i32
        L.oracle_dense_f64.argtypes = [i32, i32, P, P, P]
        L.oracle_dense_f64.restype = i32
        L.oracle_loss_grad_f64.argtypes = [i32, i32, P, P, P, i64, i32, P, P, P]
        L.oracle_loss_grad_f64.restype = i32
        L.oracle_loss_f64.argtypes = [i32, i32, P, P, P, i64, i32, P]
        L.oracle_loss_f64.restype = i32
        L.oracle_dense_apply_f64.argtypes = [i32, i32, P, P, P, i64, P]
        L.oracle_dense_apply_f64.restype = i32
        L.oracle_dense_apply_int.argtypes = [i32, i32, P, i32, P, P, i64, P]
        L.oracle_dense_apply_int.restype = i32
        for name in ("oracle_pmpt_fwd_int", "oracle_pmpt_inv_int"):
            f = getattr(L, name)
            f.argtypes = [i32, i32, i32, P, P, P, i32, i32, P, P, i64, P]
            f.restype = i32
        for name in ("oracle_pmpt_fwd_f64", "oracle_pmpt_inv_f64"):
            f = getattr(L, name)
            f.argtypes = [i32, i32, i32, P, P, P, P, P, i64, P]
            f.restype = i32
        L.oracle_dct_matrix.argtypes = [i32, P, P]
        L.oracle_dct_matrix.restype = i32
        for name in ("oracle_secondary_fwd", "oracle_secondary_inv"):
            f = getattr(L, name)
            f.argtypes = [i32, i32, i32, i32, P, P, i32, i32, P, P, i64, P]
            f.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def pair(p: int, j: int) -> tuple[int, int]:
    """(m, n) of pair j in pass p (Sec. IV, Fig. 4)."""
    m, n = ctypes.c_int(), ctypes.c_int()
    lib().oracle_pair(p, j, ctypes.byref(m), ctypes.byref(n))
    return m.value, n.value


def cs_table(angle_bits: int = 8, frac_bits: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """Integer multipliers (c[q], s[q]) of every angle index q (Sec. IV, Fig. 5)."""
    c = np.zeros(1 << angle_bits, np.int32)
    s = np.zeros(1 << angle_bits, np.int32)
    st = lib().oracle_cs_table(angle_bits, frac_bits, _ptr(c), _ptr(s))
    if st:
        raise ValueError("oracle_cs_table: bad arguments")
    return c, s


def _shape(angle, log2n, rounds):
    half = 1 << (log2n - 1)
    assert angle.size % (rounds * log2n * half) == 0
    return angle.size // (rounds * log2n * half)


def fwd_int(x, angle_idx, log2n, rounds, perms=None, set_idx=None,
            angle_bits=8, frac_bits=8):
    """Integer forward HyGT of int16 blocks x[B][N] -> (int32 y[B][N], status)."""
    x = _c(x, np.int16)
    a = _c(angle_idx, np.uint8)
    p = _c(perms, np.uint16)
    s = _c(set_idx, np.uint16)
    S = _shape(a, log2n, rounds)
    N = 1 << log2n
    B = x.size // N
    y = np.zeros((B, N), np.int32)
    st = lib().oracle_fwd_int(log2n, rounds, S, _ptr(a), _ptr(p), angle_bits, frac_bits,
                              _ptr(x), _ptr(s), B, _ptr(y))
    return y, int(st)


def inv_int(y, angle_idx, log2n, rounds, perms=None, set_idx=None,
            angle_bits=8, frac_bits=8):
    """Integer inverse HyGT of int32 blocks y[B][N] -> (int16 x[B][N], status)."""
    y = _c(y, np.int32)
    a = _c(angle_idx, np.uint8)
    p = _c(perms, np.uint16)
    s = _c(set_idx, np.uint16)
    S = _shape(a, log2n, rounds)
    N = 1 << log2n
    B = y.size // N
    x = np.zeros((B, N), np.int16)
    st = lib().oracle_inv_int(log2n, rounds, S, _ptr(a), _ptr(p), angle_bits, frac_bits,
                              _ptr(y), _ptr(s), B, _ptr(x))
    return x, int(st)


def fwd_f64(x, theta, log2n, rounds, perms=None, set_idx=None):
    """FP64 forward HyGT with free angles theta[S][R][k][N/2] -> (y, status)."""
    x = _c(x, np.float64)
    t = _c(theta, np.float64)
    p = _c(perms, np.uint16)
    s = _c(set_idx, np.uint16)
    S = _shape(t, log2n, rounds)
    N = 1 << log2n
    B = x.size // N
    y = np.zeros((B, N), np.float64)
    st = lib().oracle_fwd_f64(log2n, rounds, S, _ptr(t), _ptr(p), _ptr(x), _ptr(s), B, _ptr(y))
    return y, int(st)


def inv_f64(y, theta, log2n, rounds, perms=None, set_idx=None):
    """FP64 inverse HyGT -> (x, status)."""
    y = _c(y, np.float64)
    t = _c(theta, np.float64)
    p = _c(perms, np.uint16)
    s = _c(set_idx, np.uint16)
    S = _shape(t, log2n, rounds)
    N = 1 << log2n
    B = y.size // N
    x = np.zeros((B, N), np.float64)
    st = lib().oracle_inv_f64(log2n, rounds, S, _ptr(t), _ptr(p), _ptr(y), _ptr(s), B, _ptr(x))
    return x, int(st)


def dense_f64(theta_set, log2n, rounds, perms_set=None):
    """Dense N x N matrix of one set: column k = forward(e_k) (Eq. 5)."""
    t = _c(theta_set, np.float64)
    p = _c(perms_set, np.uint16)
    N = 1 << log2n
    T = np.zeros((N, N), np.float64)
    st = lib().oracle_dense_f64(log2n, rounds, _ptr(t), _ptr(p), _ptr(T))
    if st:
        raise ValueError("oracle_dense_f64: bad arguments")
    return T


def loss_grad_f64(x, theta, log2n, rounds, K, perms=None, want_gx=False):
    """Energy outside the first K coefficients and its analytic gradient.

    Returns (loss, gtheta[R][k][N/2], gx or None) for one set.
    """
    x = _c(x, np.float64)
    t = _c(theta, np.float64)
    p = _c(perms, np.uint16)
    N = 1 << log2n
    B = x.size // N
    g = np.zeros(t.shape, np.float64)
    gx = np.zeros((B, N), np.float64) if want_gx else None
    loss = ctypes.c_double()
    st = lib().oracle_loss_grad_f64(log2n, rounds, _ptr(t), _ptr(p), _ptr(x), B, K,
                                    ctypes.byref(loss), _ptr(g), _ptr(gx))
    if st:
        raise ValueError("oracle_loss_grad_f64: bad arguments")
    return loss.value, g, gx


def loss_f64(x, theta, log2n, rounds, K, perms=None):
    x = _c(x, np.float64)
    t = _c(theta, np.float64)
    p = _c(perms, np.uint16)
    N = 1 << log2n
    B = x.size // N
    loss = ctypes.c_double()
    st = lib().oracle_loss_f64(log2n, rounds, _ptr(t), _ptr(p), _ptr(x), B, K, ctypes.byref(loss))
    if st:
        raise ValueError("oracle_loss_f64: bad arguments")
    return loss.value


def dense_apply_f64(x, K, set_idx=None):
    """y_b = K[set(b)] x_b in FP64 (the matrix transform, Eq. 3)."""
    K = _c(K, np.float64)
    S, n, _ = K.shape
    x = _c(x, np.float64)
    s = _c(set_idx, np.uint16)
    B = x.size // n
    y = np.zeros((B, n), np.float64)
    st = lib().oracle_dense_apply_f64(n, S, _ptr(K), _ptr(x), _ptr(s), B, _ptr(y))
    return y, int(st)


def dense_apply_int(x, K_int, frac_bits=8, set_idx=None):
    """y_b = floor((K_int[set(b)] x_b + 2^(f-1)) / 2^f), int64 accumulation."""
    K = _c(K_int, np.int32)
    S, n, _ = K.shape
    x = _c(x, np.int16)
    s = _c(set_idx, np.uint16)
    B = x.size // n
    y = np.zeros((B, n), np.int32)
    st = lib().oracle_dense_apply_int(n, S, _ptr(K), frac_bits, _ptr(x), _ptr(s), B, _ptr(y))
    return y, int(st)


def _pmpt_shape(angles, m_idx, n, passes):
    assert m_idx.size == angles.size and angles.size % (passes * (n // 2)) == 0
    return angles.size // (passes * (n // 2))


def _pmpt_int(fn, inp, in_dtype, out_dtype, angle_idx, m_idx, n_idx, n, passes, set_idx,
              angle_bits, frac_bits):
    v = _c(inp, in_dtype)
    a = _c(angle_idx, np.uint8)
    mi, ni = _c(m_idx, np.uint16), _c(n_idx, np.uint16)
    s = _c(set_idx, np.uint16)
    S = _pmpt_shape(a, mi, n, passes)
    B = v.size // n
    out = np.zeros((B, n), out_dtype)
    st = fn(n, passes, S, _ptr(a), _ptr(mi), _ptr(ni), angle_bits, frac_bits, _ptr(v), _ptr(s),
            B, _ptr(out))
    return out, int(st)


def pmpt_fwd_int(x, angle_idx, m_idx, n_idx, n, passes, set_idx=None, angle_bits=8,
                 frac_bits=8):
    """Integer PMPT with explicit pair covers (Sec. III-IV): int16 x[B][n] ->
    (int32 y, status); angle_idx, m_idx, n_idx of shape [S][passes][n/2]."""
    return _pmpt_int(lib().oracle_pmpt_fwd_int, x, np.int16, np.int32, angle_idx, m_idx, n_idx,
                     n, passes, set_idx, angle_bits, frac_bits)


def pmpt_inv_int(y, angle_idx, m_idx, n_idx, n, passes, set_idx=None, angle_bits=8,
                 frac_bits=8):
    """Inverse integer PMPT: int32 y -> (int16 x saturated, status)."""
    return _pmpt_int(lib().oracle_pmpt_inv_int, y, np.int32, np.int16, angle_idx, m_idx, n_idx,
                     n, passes, set_idx, angle_bits, frac_bits)


def _pmpt_f64(fn, inp, theta, m_idx, n_idx, n, passes, set_idx):
    v = _c(inp, np.float64)
    t = _c(theta, np.float64)
    mi, ni = _c(m_idx, np.uint16), _c(n_idx, np.uint16)
    s = _c(set_idx, np.uint16)
    S = _pmpt_shape(t, mi, n, passes)
    B = v.size // n
    out = np.zeros((B, n), np.float64)
    st = fn(n, passes, S, _ptr(t), _ptr(mi), _ptr(ni), _ptr(v), _ptr(s), B, _ptr(out))
    return out, int(st)


def pmpt_fwd_f64(x, theta, m_idx, n_idx, n, passes, set_idx=None):
    """FP64 PMPT with free angles theta[S][passes][n/2] -> (y, status)."""
    return _pmpt_f64(lib().oracle_pmpt_fwd_f64, x, theta, m_idx, n_idx, n, passes, set_idx)


def pmpt_inv_f64(y, theta, m_idx, n_idx, n, passes, set_idx=None):
    return _pmpt_f64(lib().oracle_pmpt_inv_f64, y, theta, m_idx, n_idx, n, passes, set_idx)


def dct_matrix(log2m):
    """(integer C = round(256 D), FP64 D) of the M x M orthonormal DCT-II
    (row k = basis function k), the primary transform of the Sec. VI
    pipeline."""
    M = 1 << log2m
    C = np.zeros((M, M), np.int32)
    D = np.zeros((M, M), np.float64)
    if lib().oracle_dct_matrix(log2m, _ptr(C), _ptr(D)):
        raise ValueError("oracle_dct_matrix: bad arguments")
    return C, D


def _secondary(fn, inp, in_dtype, out_dtype, log2m, angle_idx, log2n, rounds, perms, set_idx,
               angle_bits, frac_bits):
    v = _c(inp, in_dtype)
    a = _c(angle_idx, np.uint8)
    p = _c(perms, np.uint16)
    s = _c(set_idx, np.uint16)
    S = _shape(a, log2n, rounds)
    MM = 1 << (2 * log2m)
    B = v.size // MM
    out = np.zeros((B, MM), out_dtype)
    st = fn(log2m, log2n, rounds, S, _ptr(a), _ptr(p), angle_bits, frac_bits, _ptr(v), _ptr(s), B,
            _ptr(out))
    return out, int(st)


def secondary_fwd(x, log2m, angle_idx, log2n, rounds, perms=None, set_idx=None, angle_bits=8,
                  frac_bits=8):
    """Integer DCT-II primary of M x M int16 blocks x[B][M*M] (raster), then
    the integer HyGT on the top-left s x s coefficients -> (int32 y, status)."""
    return _secondary(lib().oracle_secondary_fwd, x, np.int16, np.int32, log2m, angle_idx, log2n,
                      rounds, perms, set_idx, angle_bits, frac_bits)


def secondary_inv(y, log2m, angle_idx, log2n, rounds, perms=None, set_idx=None, angle_bits=8,
                  frac_bits=8):
    """Inverse HyGT on the top-left sub-block, then the inverse DCT-II ->
    (int16 x saturated, status)."""
    return _secondary(lib().oracle_secondary_inv, y, np.int32, np.int16, log2m, angle_idx, log2n,
                      rounds, perms, set_idx, angle_bits, frac_bits)
