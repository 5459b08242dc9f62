"""Thin Python binding of libhygt.so (argument marshalling only).

The functions named ``hygt_*`` mirror the C ABI in ``include/hygt.h`` one to
one and take raw device pointers (ints) and a CUDA stream handle.  ``Plan``
wraps a plan handle and accepts torch CUDA tensors: it checks dtypes,
shapes and devices, then passes ``data_ptr()`` and the current stream to the
C entry point.  Every step of the transform runs in the CUDA kernels of the
library; there is no other implementation behind this module.  Importing it
raises if the library has not been built for this machine.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import SO

HYGT_OK = 0
HYGT_ERR_ARG = 1
HYGT_ERR_CUDA = 2
HYGT_ERR_OOM = 3
HYGT_ERR_SET_INDEX = 4
HYGT_ERR_UNSUPPORTED = 6
HYGT_ERR_TOO_LARGE = 7
HYGT_SKIP_SET = 0xFFFF
DENSE_KLT_BF16 = 0
DENSE_KLT_INT = 1
DENSE_KLT_FP8 = 2


class HygtError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (status %d)" % (where, hygt_status_string(code), code))


class MixedClass(ctypes.Structure):
    """hygt_mixed_class of include/hygt.h."""
    _fields_ = [("plan", ctypes.c_void_p), ("d_set", ctypes.c_void_p),
                ("nblocks", ctypes.c_int64), ("d_work", ctypes.c_void_p),
                ("work_bytes", ctypes.c_size_t), ("d_x", ctypes.c_void_p),
                ("d_y", ctypes.c_void_p), ("d_xr", ctypes.c_void_p), ("ctas", ctypes.c_int)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(SO):
        raise ImportError("libhygt.so is not built (%s); run "
                          "paper_2505_21728_gb300.build.build() first" % SO)
    L = ctypes.CDLL(SO)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    L.hygt_create.argtypes = [ctypes.POINTER(P), i32, i32, i32, P, P, i32, i32]
    L.hygt_create.restype = i32
    L.hygt_create_float.argtypes = [ctypes.POINTER(P), i32, i32, i32, P, P]
    L.hygt_create_float.restype = i32
    L.hygt_destroy.argtypes = [P]
    L.hygt_destroy.restype = None
    for name in ("hygt_forward", "hygt_inverse", "hygt_forward_f32", "hygt_inverse_f32"):
        f = getattr(L, name)
        f.argtypes = [P, P, P, P, i64, P, P]
        f.restype = i32
    L.hygt_batch_workspace_bytes.argtypes = [P, i64]
    L.hygt_batch_workspace_bytes.restype = ctypes.c_size_t
    L.hygt_batch_build.argtypes = [P, P, i64, P, ctypes.c_size_t, P]
    L.hygt_batch_build.restype = i32
    for name in ("hygt_forward_batch", "hygt_inverse_batch", "hygt_forward_batch_f32",
                 "hygt_inverse_batch_f32"):
        f = getattr(L, name)
        f.argtypes = [P, P, P, P, i64, P, P]
        f.restype = i32
    L.hygt_forward_static.argtypes = [P, P, P, P, i64, P, P]
    L.hygt_forward_static.restype = i32
    L.hygt_host_pipe_create.argtypes = [ctypes.POINTER(P), P, i64]
    L.hygt_host_pipe_create.restype = i32
    L.hygt_host_roundtrip.argtypes = [P, P, P, P, P, i64, ctypes.POINTER(i32)]
    L.hygt_host_roundtrip.restype = i32
    L.hygt_host_pipe_destroy.argtypes = [P]
    L.hygt_host_pipe_destroy.restype = None
    L.hygt_update_theta.argtypes = [P, P, P]
    L.hygt_update_theta.restype = i32
    L.hygt_backward_workspace_bytes.argtypes = [P, i64]
    L.hygt_backward_workspace_bytes.restype = ctypes.c_size_t
    L.hygt_backward_f32.argtypes = [P, P, P, P, P, P, i64, P, ctypes.c_size_t, P, P]
    L.hygt_backward_f32.restype = i32
    L.hygt_backward_diag_f32.argtypes = [P, P, P, P, P, P, i64, P, ctypes.c_size_t, P, P]
    L.hygt_backward_diag_f32.restype = i32
    L.hygt_coding_gain_workspace_bytes.argtypes = [P, i64]
    L.hygt_coding_gain_workspace_bytes.restype = ctypes.c_size_t
    L.hygt_coding_gain_f32.argtypes = [P, P, i64, P, P, P, P, ctypes.c_size_t, P]
    L.hygt_coding_gain_f32.restype = i32
    f32 = ctypes.c_float
    L.hygt_adam_step.argtypes = [P, P, P, P, i64, f32, f32, f32, f32, i32, P]
    L.hygt_adam_step.restype = i32
    for name in ("hygt_secondary_forward_batch", "hygt_secondary_inverse_batch"):
        f = getattr(L, name)
        f.argtypes = [P, P, i32, P, P, i64, P, P]
        f.restype = i32
    for name in ("hygt_secondary_forward", "hygt_secondary_inverse"):
        f = getattr(L, name)
        f.argtypes = [P, i32, P, P, P, i64, P, P]
        f.restype = i32
    L.hygt_pmpt_create.argtypes = [ctypes.POINTER(P), i32, i32, i32, P, P, P, P, i32, i32]
    L.hygt_pmpt_create.restype = i32
    L.hygt_pmpt_destroy.argtypes = [P]
    L.hygt_pmpt_destroy.restype = None
    L.hygt_pmpt_param_bytes.argtypes = [i32, i32, i32]
    L.hygt_pmpt_param_bytes.restype = ctypes.c_size_t
    for name in ("hygt_pmpt_forward", "hygt_pmpt_inverse", "hygt_pmpt_forward_f32",
                 "hygt_pmpt_inverse_f32"):
        f = getattr(L, name)
        f.argtypes = [P, P, P, P, i64, P, P]
        f.restype = i32
    L.dense_klt_create.argtypes = [ctypes.POINTER(P), i32, i32, P, i32]
    L.dense_klt_create.restype = i32
    L.dense_klt_destroy.argtypes = [P]
    L.dense_klt_destroy.restype = None
    L.dense_klt_workspace_bytes.argtypes = [P, i64]
    L.dense_klt_workspace_bytes.restype = ctypes.c_size_t
    L.dense_klt_build.argtypes = [P, P, i64, P, ctypes.c_size_t, P]
    L.dense_klt_build.restype = i32
    L.dense_klt_apply.argtypes = [P, P, P, P, i64, i32, P, P]
    L.dense_klt_apply.restype = i32
    L.hygt_batch_set_tuning.argtypes = [P, i32, i32, i32, i32, i32]
    L.hygt_batch_set_tuning.restype = i32
    L.hygt_batch_get_tuning.argtypes = [P, i32] + [ctypes.POINTER(i32)] * 5
    L.hygt_batch_get_tuning.restype = i32
    L.hygt_batch_set_tail.argtypes = [P, i32, i32]
    L.hygt_batch_set_tail.restype = i32
    L.hygt_batch_get_tail.argtypes = [P, i32, ctypes.POINTER(i32)]
    L.hygt_batch_get_tail.restype = i32
    L.hygt_mixed_ctas.argtypes = []
    L.hygt_mixed_ctas.restype = i32
    L.hygt_mixed_class_variant.argtypes = [P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.hygt_mixed_class_variant.restype = i32
    for name in ("hygt_forward_mixed", "hygt_inverse_mixed"):
        f = getattr(L, name)
        f.argtypes = [ctypes.POINTER(MixedClass), i32, P, P]
        f.restype = i32
    L.hygt_mixed_graph_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(MixedClass), i32, P]
    L.hygt_mixed_graph_create.restype = i32
    L.hygt_graph_launch.argtypes = [P, P]
    L.hygt_graph_launch.restype = i32
    L.hygt_graph_destroy.argtypes = [P]
    L.hygt_graph_destroy.restype = None
    L.hygt_plan_info.argtypes = [P] + [ctypes.POINTER(i32)] * 4
    L.hygt_plan_info.restype = i32
    L.hygt_param_bytes.argtypes = [i32, i32, i32]
    L.hygt_param_bytes.restype = ctypes.c_size_t
    L.hygt_status_string.argtypes = [i32]
    L.hygt_status_string.restype = ctypes.c_char_p
    return L


_lib = _load()


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(code: int, where: str) -> None:
    if code != HYGT_OK:
        raise HygtError(code, where)


# ---------------------------------------------------------------- C ABI, 1:1
def hygt_status_string(code: int) -> str:
    return _lib.hygt_status_string(int(code)).decode()


def hygt_param_bytes(log2n: int, rounds: int, num_sets: int) -> int:
    return int(_lib.hygt_param_bytes(log2n, rounds, num_sets))


def hygt_create(log2n, rounds, num_sets, angle_idx, perms=None, angle_bits=8, frac_bits=8):
    """Returns (status, plan handle); angle_idx uint8, perms uint16 or None."""
    a = np.ascontiguousarray(angle_idx, dtype=np.uint8)
    p = None if perms is None else np.ascontiguousarray(perms, dtype=np.uint16)
    h = ctypes.c_void_p()
    st = _lib.hygt_create(ctypes.byref(h), log2n, rounds, num_sets, _np_ptr(a), _np_ptr(p),
                          angle_bits, frac_bits)
    return int(st), h.value


def hygt_create_float(log2n, rounds, num_sets, theta, perms=None):
    t = np.ascontiguousarray(theta, dtype=np.float32)
    p = None if perms is None else np.ascontiguousarray(perms, dtype=np.uint16)
    h = ctypes.c_void_p()
    st = _lib.hygt_create_float(ctypes.byref(h), log2n, rounds, num_sets, _np_ptr(t), _np_ptr(p))
    return int(st), h.value


def hygt_destroy(plan) -> None:
    _lib.hygt_destroy(plan)


def hygt_forward(plan, d_x, d_y, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_forward(plan, d_x, d_y, d_set, nblocks, stream, d_status))


def hygt_inverse(plan, d_y, d_x, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_inverse(plan, d_y, d_x, d_set, nblocks, stream, d_status))


def hygt_forward_f32(plan, d_x, d_y, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_forward_f32(plan, d_x, d_y, d_set, nblocks, stream, d_status))


def hygt_inverse_f32(plan, d_y, d_x, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_inverse_f32(plan, d_y, d_x, d_set, nblocks, stream, d_status))


def hygt_batch_workspace_bytes(plan, nblocks):
    return int(_lib.hygt_batch_workspace_bytes(plan, nblocks))


def hygt_batch_build(plan, d_set, nblocks, d_work, work_bytes, stream):
    return int(_lib.hygt_batch_build(plan, d_set, nblocks, d_work, work_bytes, stream))


def hygt_forward_batch(plan, d_work, d_x, d_y, nblocks, stream, d_status):
    return int(_lib.hygt_forward_batch(plan, d_work, d_x, d_y, nblocks, stream, d_status))


def hygt_inverse_batch(plan, d_work, d_y, d_x, nblocks, stream, d_status):
    return int(_lib.hygt_inverse_batch(plan, d_work, d_y, d_x, nblocks, stream, d_status))


def hygt_forward_batch_f32(plan, d_work, d_x, d_y, nblocks, stream, d_status):
    return int(_lib.hygt_forward_batch_f32(plan, d_work, d_x, d_y, nblocks, stream, d_status))


def hygt_inverse_batch_f32(plan, d_work, d_y, d_x, nblocks, stream, d_status):
    return int(_lib.hygt_inverse_batch_f32(plan, d_work, d_y, d_x, nblocks, stream, d_status))


def hygt_forward_static(plan, d_x, d_y, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_forward_static(plan, d_x, d_y, d_set, nblocks, stream, d_status))


def hygt_host_pipe_create(plan, chunk_blocks):
    h = ctypes.c_void_p()
    st = int(_lib.hygt_host_pipe_create(ctypes.byref(h), plan, chunk_blocks))
    return st, h.value


def hygt_host_roundtrip(pipe, h_x, h_set, h_y, h_xr, nblocks):
    status = ctypes.c_int(0)
    st = int(_lib.hygt_host_roundtrip(pipe, h_x, h_set, h_y, h_xr, nblocks, ctypes.byref(status)))
    return st, int(status.value)


def hygt_host_pipe_destroy(pipe):
    _lib.hygt_host_pipe_destroy(pipe)


def hygt_update_theta(plan, d_theta, stream):
    return int(_lib.hygt_update_theta(plan, d_theta, stream))


def hygt_backward_workspace_bytes(plan, nblocks):
    return int(_lib.hygt_backward_workspace_bytes(plan, nblocks))


def hygt_backward_f32(plan, d_y, d_gy, d_gx, d_gtheta, d_set, nblocks, d_work, work_bytes,
                      stream, d_status):
    return int(_lib.hygt_backward_f32(plan, d_y, d_gy, d_gx, d_gtheta, d_set, nblocks, d_work,
                                      work_bytes, stream, d_status))


def hygt_backward_diag_f32(plan, d_y, d_w, d_gx, d_gtheta, d_set, nblocks, d_work, work_bytes,
                           stream, d_status):
    return int(_lib.hygt_backward_diag_f32(plan, d_y, d_w, d_gx, d_gtheta, d_set, nblocks,
                                           d_work, work_bytes, stream, d_status))


def hygt_coding_gain_workspace_bytes(plan, nblocks):
    return int(_lib.hygt_coding_gain_workspace_bytes(plan, nblocks))


def hygt_coding_gain_f32(plan, d_y, nblocks, d_v, d_w, d_J, d_work, work_bytes, stream):
    return int(_lib.hygt_coding_gain_f32(plan, d_y, nblocks, d_v, d_w, d_J, d_work, work_bytes,
                                         stream))


def hygt_adam_step(d_theta, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, step, stream):
    return int(_lib.hygt_adam_step(d_theta, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, step,
                                   stream))


def hygt_secondary_forward(plan, log2m, d_x, d_y, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_secondary_forward(plan, log2m, d_x, d_y, d_set, nblocks, stream,
                                           d_status))


def hygt_secondary_inverse(plan, log2m, d_y, d_x, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_secondary_inverse(plan, log2m, d_y, d_x, d_set, nblocks, stream,
                                           d_status))


def hygt_secondary_forward_batch(plan, d_work, log2m, d_x, d_y, nblocks, stream, d_status):
    return int(_lib.hygt_secondary_forward_batch(plan, d_work, log2m, d_x, d_y, nblocks, stream,
                                                 d_status))


def hygt_secondary_inverse_batch(plan, d_work, log2m, d_y, d_x, nblocks, stream, d_status):
    return int(_lib.hygt_secondary_inverse_batch(plan, d_work, log2m, d_y, d_x, nblocks, stream,
                                                 d_status))


def hygt_pmpt_create(n, passes, num_sets, angle_idx, theta, m_idx, n_idx, angle_bits=8,
                     frac_bits=8):
    a = None if angle_idx is None else np.ascontiguousarray(angle_idx, dtype=np.uint8)
    t = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
    mi = np.ascontiguousarray(m_idx, dtype=np.uint16)
    ni = np.ascontiguousarray(n_idx, dtype=np.uint16)
    h = ctypes.c_void_p()
    st = _lib.hygt_pmpt_create(ctypes.byref(h), n, passes, num_sets, _np_ptr(a), _np_ptr(t),
                               _np_ptr(mi), _np_ptr(ni), angle_bits, frac_bits)
    return int(st), h.value


def hygt_pmpt_destroy(pm):
    _lib.hygt_pmpt_destroy(pm)


def hygt_pmpt_param_bytes(n, passes, num_sets):
    return int(_lib.hygt_pmpt_param_bytes(n, passes, num_sets))


def hygt_pmpt_forward(pm, d_x, d_y, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_pmpt_forward(pm, d_x, d_y, d_set, nblocks, stream, d_status))


def hygt_pmpt_inverse(pm, d_y, d_x, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_pmpt_inverse(pm, d_y, d_x, d_set, nblocks, stream, d_status))


def hygt_pmpt_forward_f32(pm, d_x, d_y, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_pmpt_forward_f32(pm, d_x, d_y, d_set, nblocks, stream, d_status))


def hygt_pmpt_inverse_f32(pm, d_y, d_x, d_set, nblocks, stream, d_status):
    return int(_lib.hygt_pmpt_inverse_f32(pm, d_y, d_x, d_set, nblocks, stream, d_status))


def dense_klt_create(log2n, num_sets, K, frac_bits=8):
    k = np.ascontiguousarray(K, dtype=np.float32)
    h = ctypes.c_void_p()
    st = _lib.dense_klt_create(ctypes.byref(h), log2n, num_sets, _np_ptr(k), frac_bits)
    return int(st), h.value


def dense_klt_destroy(d):
    _lib.dense_klt_destroy(d)


def dense_klt_workspace_bytes(d, nblocks):
    return int(_lib.dense_klt_workspace_bytes(d, nblocks))


def dense_klt_build(d, d_set, nblocks, d_work, work_bytes, stream):
    return int(_lib.dense_klt_build(d, d_set, nblocks, d_work, work_bytes, stream))


def dense_klt_apply(d, d_work, d_x, d_y, nblocks, kind, stream, d_status):
    return int(_lib.dense_klt_apply(d, d_work, d_x, d_y, nblocks, kind, stream, d_status))


def hygt_batch_set_tuning(plan, inverse, warps_per_cta, ctas_per_sm, stage, layout=0):
    return int(_lib.hygt_batch_set_tuning(plan, int(inverse), int(warps_per_cta),
                                          int(ctas_per_sm), int(stage), int(layout)))


def hygt_batch_get_tuning(plan, inverse):
    """(warps_per_cta, ctas_per_sm, stage, layout, max_warps) of one
    direction; max_warps is that of the layout set."""
    vals = [ctypes.c_int() for _ in range(5)]
    _check(_lib.hygt_batch_get_tuning(plan, int(inverse), *[ctypes.byref(v) for v in vals]),
           "hygt_batch_get_tuning")
    return tuple(v.value for v in vals)


def hygt_batch_set_tail(plan, inverse, tail_64ths):
    return int(_lib.hygt_batch_set_tail(plan, int(inverse), int(tail_64ths)))


def hygt_batch_get_tail(plan, inverse):
    v = ctypes.c_int()
    _check(_lib.hygt_batch_get_tail(plan, int(inverse), ctypes.byref(v)), "hygt_batch_get_tail")
    return v.value


def hygt_mixed_ctas():
    return int(_lib.hygt_mixed_ctas())


def hygt_mixed_class_variant(plan, inverse):
    """(stage, layout) in which a single mixed launch runs a class of
    ``plan`` in one direction under the plan's current tuning."""
    st, lay = ctypes.c_int(), ctypes.c_int()
    _check(_lib.hygt_mixed_class_variant(plan, int(inverse), ctypes.byref(st), ctypes.byref(lay)),
           "hygt_mixed_class_variant")
    return st.value, lay.value


def hygt_forward_mixed(classes, nclasses, stream, d_status):
    return int(_lib.hygt_forward_mixed(classes, nclasses, stream, d_status))


def hygt_inverse_mixed(classes, nclasses, stream, d_status):
    return int(_lib.hygt_inverse_mixed(classes, nclasses, stream, d_status))


def hygt_mixed_graph_create(classes, nclasses, d_status):
    h = ctypes.c_void_p()
    st = _lib.hygt_mixed_graph_create(ctypes.byref(h), classes, nclasses, d_status)
    return int(st), h.value


def hygt_graph_launch(graph, stream):
    return int(_lib.hygt_graph_launch(graph, stream))


def hygt_graph_destroy(graph):
    _lib.hygt_graph_destroy(graph)


def hygt_plan_info(plan):
    vals = [ctypes.c_int() for _ in range(4)]
    _check(_lib.hygt_plan_info(plan, *[ctypes.byref(v) for v in vals]), "hygt_plan_info")
    return tuple(v.value for v in vals)


# ---------------------------------------------------------------- torch wrapper
def _stream_handle(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _dptr(t, dtype, shape_last=None, name="tensor"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError("%s must have shape [nblocks, %d]" % (name, shape_last))
    return t.data_ptr()


class Plan:
    """A transform plan on the current CUDA device.

    ``Plan(log2n, rounds, angle_idx, perms)`` builds an integer plan (its
    FP32 calls use the same angles); ``Plan.from_theta(...)`` builds an FP32
    plan with free angles.
    """

    def __init__(self, log2n, rounds, angle_idx=None, perms=None, angle_bits=8, frac_bits=8,
                 _handle=None, _num_sets=None):
        self.log2n = int(log2n)
        self.rounds = int(rounds)
        self.N = 1 << self.log2n
        if _handle is not None:
            self.handle = _handle
            self.num_sets = _num_sets
            return
        a = np.ascontiguousarray(angle_idx, dtype=np.uint8)
        self.num_sets = a.size // (self.rounds * self.log2n * (self.N // 2))
        st, h = hygt_create(self.log2n, self.rounds, self.num_sets, a, perms, angle_bits, frac_bits)
        _check(st, "hygt_create")
        self.handle = h

    @classmethod
    def from_theta(cls, log2n, rounds, theta, perms=None):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        N = 1 << log2n
        S = t.size // (rounds * log2n * (N // 2))
        st, h = hygt_create_float(log2n, rounds, S, t, perms)
        _check(st, "hygt_create_float")
        return cls(log2n, rounds, _handle=h, _num_sets=S)

    def close(self):
        if getattr(self, "handle", None):
            hygt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, fn, name, x, out, sets, in_dtype, out_dtype, status, stream):
        import torch
        nb = x.shape[0] if x.dim() == 2 else 0
        px = _dptr(x, in_dtype, self.N, "input")
        po = _dptr(out, out_dtype, self.N, "output")
        if out.shape[0] != nb:
            raise ValueError("output has %d blocks, input %d" % (out.shape[0], nb))
        ps = None
        if sets is not None:
            ps = _dptr(sets, torch.int16 if sets.dtype == torch.int16 else torch.uint16, None, "sets")
            if sets.numel() != nb:
                raise ValueError("sets must have one entry per block")
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        _check(fn(self.handle, px, po, ps, nb, _stream_handle(stream), pst), name)
        return out

    def forward(self, x, sets=None, out=None, status=None, stream=None):
        """int16 [B, N] -> int32 [B, N] (integer HyGT)."""
        import torch
        if out is None:
            out = torch.empty(x.shape, dtype=torch.int32, device=x.device)
        return self._call(hygt_forward, "hygt_forward", x, out, sets, torch.int16, torch.int32,
                          status, stream)

    def inverse(self, y, sets=None, out=None, status=None, stream=None):
        """int32 [B, N] -> int16 [B, N] (integer inverse HyGT, saturated)."""
        import torch
        if out is None:
            out = torch.empty(y.shape, dtype=torch.int16, device=y.device)
        return self._call(hygt_inverse, "hygt_inverse", y, out, sets, torch.int32, torch.int16,
                          status, stream)

    def update_theta(self, theta, stream=None):
        """Recompute the FP32 table from device angles (float32, layout of
        the angles); FP32 plans only."""
        import torch
        pt = _dptr(theta.contiguous() if theta.is_cuda else theta, torch.float32, None, "theta")
        _check(hygt_update_theta(self.handle, pt, _stream_handle(stream)), "hygt_update_theta")

    def backward_f32(self, y, gy, sets=None, status=None, stream=None):
        """dL/dx (float32 [B, N]) and dL/dtheta (float64, flat) from the
        forward output y and dL/dy."""
        import torch
        py = _dptr(y, torch.float32, self.N, "y")
        pgy = _dptr(gy, torch.float32, self.N, "gy")
        nb = y.shape[0]
        if gy.shape[0] != nb:
            raise ValueError("gy must have the shape of y")
        if sets is not None and sets.numel() != nb:
            raise ValueError("sets must have one entry per block")
        gx = torch.empty_like(y)
        angles = self.num_sets * self.rounds * self.log2n * (self.N // 2)
        gth = torch.empty(angles, dtype=torch.float64, device=y.device)
        wb = hygt_backward_workspace_bytes(self.handle, nb)
        if wb == 0:
            raise HygtError(HYGT_ERR_UNSUPPORTED, "hygt_backward_workspace_bytes")
        work = torch.empty(wb, dtype=torch.uint8, device=y.device)
        ps = None
        if sets is not None:
            ps = _dptr(sets, torch.int16 if sets.dtype == torch.int16 else torch.uint16, None, "sets")
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        _check(hygt_backward_f32(self.handle, py, pgy, gx.data_ptr(),
                                 gth.data_ptr(), ps, nb, work.data_ptr(), wb,
                                 _stream_handle(stream), pst), "hygt_backward_f32")
        return gx, gth

    def secondary_forward(self, x, log2m, sets=None, out=None, status=None, stream=None):
        """Integer DCT-II primary of int16 M x M blocks x [B, M*M] (raster),
        then this plan's HyGT on the top-left coefficients -> int32 [B, M*M]."""
        import torch
        M2 = 1 << (2 * int(log2m))
        if out is None:
            out = torch.empty((x.shape[0], M2), dtype=torch.int32, device=x.device)
        return self._call_sec(hygt_secondary_forward, "hygt_secondary_forward", log2m, x, out,
                              sets, torch.int16, torch.int32, status, stream)

    def secondary_inverse(self, y, log2m, sets=None, out=None, status=None, stream=None):
        import torch
        M2 = 1 << (2 * int(log2m))
        if out is None:
            out = torch.empty((y.shape[0], M2), dtype=torch.int16, device=y.device)
        return self._call_sec(hygt_secondary_inverse, "hygt_secondary_inverse", log2m, y, out,
                              sets, torch.int32, torch.int16, status, stream)

    def _call_sec(self, fn, name, log2m, x, out, sets, in_dtype, out_dtype, status, stream):
        import torch
        M2 = 1 << (2 * int(log2m))
        nb = x.shape[0]
        px = _dptr(x, in_dtype, M2, "input")
        po = _dptr(out, out_dtype, M2, "output")
        if out.shape[0] != nb:
            raise ValueError("output has %d blocks, input %d" % (out.shape[0], nb))
        ps = None
        if sets is not None:
            if sets.numel() != nb:
                raise ValueError("sets must have one entry per block")
            ps = _dptr(sets, torch.int16 if sets.dtype == torch.int16 else torch.uint16, None,
                       "sets")
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        _check(fn(self.handle, int(log2m), px, po, ps, nb, _stream_handle(stream), pst), name)
        return out

    def dense_matrices(self):
        """The N x N matrix of every set (float32 [S, N, N], y = T x), from
        the FP32 transform of the unit vectors: column i = T e_i."""
        import torch
        N, S = self.N, self.num_sets
        eye = torch.eye(N, dtype=torch.float32, device="cuda").repeat(S, 1).contiguous()
        sets = torch.arange(S, device="cuda").repeat_interleave(N).to(torch.int16)
        y = self.forward_f32(eye, sets)
        return y.view(S, N, N).transpose(1, 2).contiguous().cpu().numpy()

    def forward_f32(self, x, sets=None, out=None, status=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
        return self._call(hygt_forward_f32, "hygt_forward_f32", x, out, sets, torch.float32,
                          torch.float32, status, stream)

    def inverse_f32(self, y, sets=None, out=None, status=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(y.shape, dtype=torch.float32, device=y.device)
        return self._call(hygt_inverse_f32, "hygt_inverse_f32", y, out, sets, torch.float32,
                          torch.float32, status, stream)


class PMPT:
    """A general PMPT plan (explicit pair covers; hygt_pmpt_create).

    ``PMPT(n, passes, m_idx, n_idx, angle_idx=...)`` builds an integer plan
    (its FP32 calls use the same angles); ``theta=...`` an FP32-only plan.
    """

    def __init__(self, n, passes, m_idx, n_idx, angle_idx=None, theta=None, angle_bits=8,
                 frac_bits=8):
        self.N, self.passes = int(n), int(passes)
        ref = angle_idx if angle_idx is not None else theta
        self.num_sets = int(np.asarray(ref).size // (self.passes * (self.N // 2)))
        st, h = hygt_pmpt_create(self.N, self.passes, self.num_sets, angle_idx, theta, m_idx,
                                 n_idx, angle_bits, frac_bits)
        _check(st, "hygt_pmpt_create")
        self.handle = h

    def _call(self, fn, name, x, out_dtype, sets, status, stream):
        import torch
        nb = x.shape[0]
        px = _dptr(x, x.dtype, self.N, "input")
        out = torch.empty((nb, self.N), dtype=out_dtype, device=x.device)
        ps = None
        if sets is not None:
            if sets.numel() != nb:
                raise ValueError("sets must have one entry per block")
            ps = _dptr(sets, torch.int16 if sets.dtype == torch.int16 else torch.uint16, None,
                       "sets")
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        _check(fn(self.handle, px, out.data_ptr(), ps, nb, _stream_handle(stream), pst), name)
        return out

    def forward(self, x, sets=None, status=None, stream=None):
        import torch
        if x.dtype != torch.int16:
            raise TypeError("x must be int16")
        return self._call(hygt_pmpt_forward, "hygt_pmpt_forward", x, torch.int32, sets, status,
                          stream)

    def inverse(self, y, sets=None, status=None, stream=None):
        import torch
        if y.dtype != torch.int32:
            raise TypeError("y must be int32")
        return self._call(hygt_pmpt_inverse, "hygt_pmpt_inverse", y, torch.int16, sets, status,
                          stream)

    def forward_f32(self, x, sets=None, status=None, stream=None):
        import torch
        if x.dtype != torch.float32:
            raise TypeError("x must be float32")
        return self._call(hygt_pmpt_forward_f32, "hygt_pmpt_forward_f32", x, torch.float32,
                          sets, status, stream)

    def inverse_f32(self, y, sets=None, status=None, stream=None):
        import torch
        if y.dtype != torch.float32:
            raise TypeError("y must be float32")
        return self._call(hygt_pmpt_inverse_f32, "hygt_pmpt_inverse_f32", y, torch.float32,
                          sets, status, stream)

    def close(self):
        if getattr(self, "handle", None):
            hygt_pmpt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipe:
    """Round trips of integer batches held in host memory (hygt_host_roundtrip):
    forward coefficients and inverse reconstruction come back to host
    tensors.  Host tensors should be pinned (``tensor.pin_memory()``) for the
    copies to overlap the kernels."""

    def __init__(self, plan, chunk_blocks=1 << 17):
        st, h = hygt_host_pipe_create(plan.handle, int(chunk_blocks))
        _check(st, "hygt_host_pipe_create")
        self.handle = h
        self.plan = plan

    def roundtrip(self, x, sets=None, y=None, xr=None, coefficients=True):
        """x: int16 CPU tensor [B, N]; sets: int16/uint16 CPU tensor [B] or
        None.  Returns (y int32 [B, N] or None, xr int16 [B, N], status);
        with coefficients=False only the reconstruction comes back."""
        import torch
        N = self.plan.N
        if x.is_cuda or x.dtype != torch.int16 or x.dim() != 2 or x.shape[1] != N or \
                not x.is_contiguous():
            raise ValueError("x must be a contiguous int16 CPU tensor [nblocks, %d]" % N)
        B = x.shape[0]
        if y is None and coefficients:
            y = torch.empty((B, N), dtype=torch.int32, pin_memory=x.is_pinned())
        if not coefficients:
            y = None
        if xr is None:
            xr = torch.empty((B, N), dtype=torch.int16, pin_memory=x.is_pinned())
        for t, dt, name in ((y, torch.int32, "y"), (xr, torch.int16, "xr")):
            if t is None:
                continue
            if t.is_cuda or t.dtype != dt or tuple(t.shape) != (B, N) or not t.is_contiguous():
                raise ValueError("%s must be a contiguous %s CPU tensor [%d, %d]" % (name, dt, B, N))
        ps = None
        if sets is not None:
            if sets.is_cuda or sets.numel() != B or not sets.is_contiguous() or \
                    sets.dtype not in (torch.int16, torch.uint16):
                raise ValueError("sets must be a contiguous 16-bit CPU tensor [nblocks]")
            ps = sets.data_ptr()
        st, status = hygt_host_roundtrip(self.handle, x.data_ptr(), ps,
                                         None if y is None else y.data_ptr(), xr.data_ptr(), B)
        _check(st, "hygt_host_roundtrip")
        return y, xr, status

    def close(self):
        if getattr(self, "handle", None):
            hygt_host_pipe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A set-bucketed schedule of ``nblocks`` blocks for one plan.

    ``build(sets)`` buckets the per-block set indices on the device (into a
    workspace tensor this object owns); ``forward`` / ``inverse`` then run the
    bucketed kernels.  Rebuild whenever the set indices change.
    """

    def __init__(self, plan: Plan, nblocks: int, device=None):
        import torch
        self.plan = plan
        self.nblocks = int(nblocks)
        nbytes = hygt_batch_workspace_bytes(plan.handle, self.nblocks)
        if nbytes == 0:
            raise HygtError(HYGT_ERR_ARG, "hygt_batch_workspace_bytes")
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")

    @classmethod
    def on_workspace(cls, plan: Plan, nblocks: int, work):
        """A Batch over an existing schedule workspace (a uint8 CUDA tensor
        holding a schedule built for this plan and block count), e.g. one
        class of a MixedBatch."""
        b = cls.__new__(cls)
        b.plan, b.nblocks, b.work = plan, int(nblocks), work
        return b

    def build(self, sets=None, stream=None):
        import torch
        ps = None
        if sets is not None:
            ps = _dptr(sets, torch.int16 if sets.dtype == torch.int16 else torch.uint16, None, "sets")
            if sets.numel() != self.nblocks:
                raise ValueError("sets must have one entry per block")
        _check(hygt_batch_build(self.plan.handle, ps, self.nblocks, self.work.data_ptr(),
                                self.work.numel(), _stream_handle(stream)), "hygt_batch_build")
        return self

    def _run(self, fn, name, x, out, in_dtype, out_dtype, status, stream):
        import torch
        if x.shape[0] != self.nblocks or out.shape[0] != self.nblocks:
            raise ValueError("batch built for %d blocks" % self.nblocks)
        px = _dptr(x, in_dtype, self.plan.N, "input")
        po = _dptr(out, out_dtype, self.plan.N, "output")
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        _check(fn(self.plan.handle, self.work.data_ptr(), px, po, self.nblocks,
                  _stream_handle(stream), pst), name)
        return out

    def forward(self, x, out=None, status=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(x.shape, dtype=torch.int32, device=x.device)
        return self._run(hygt_forward_batch, "hygt_forward_batch", x, out, torch.int16,
                         torch.int32, status, stream)

    def inverse(self, y, out=None, status=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(y.shape, dtype=torch.int16, device=y.device)
        return self._run(hygt_inverse_batch, "hygt_inverse_batch", y, out, torch.int32,
                         torch.int16, status, stream)

    def secondary_forward(self, x, log2m, out=None, status=None, stream=None):
        """The secondary pipeline (DCT-II primary fused, 4x4 / 8x8 blocks)
        through this schedule: int16 [B, N] -> int32 [B, N]."""
        import torch
        if out is None:
            out = torch.empty(x.shape, dtype=torch.int32, device=x.device)
        fn = lambda h, w, px, po, nb, st, ps: hygt_secondary_forward_batch(  # noqa: E731
            h, w, int(log2m), px, po, nb, st, ps)
        return self._run(fn, "hygt_secondary_forward_batch", x, out, torch.int16, torch.int32,
                         status, stream)

    def secondary_inverse(self, y, log2m, out=None, status=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(y.shape, dtype=torch.int16, device=y.device)
        fn = lambda h, w, py, po, nb, st, ps: hygt_secondary_inverse_batch(  # noqa: E731
            h, w, int(log2m), py, po, nb, st, ps)
        return self._run(fn, "hygt_secondary_inverse_batch", y, out, torch.int32, torch.int16,
                         status, stream)

    def forward_f32(self, x, out=None, status=None, stream=None):
        """FP32 forward through the bucketed schedule (N >= 16)."""
        import torch
        if out is None:
            out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
        return self._run(hygt_forward_batch_f32, "hygt_forward_batch_f32", x, out,
                         torch.float32, torch.float32, status, stream)

    def inverse_f32(self, y, out=None, status=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(y.shape, dtype=torch.float32, device=y.device)
        return self._run(hygt_inverse_batch_f32, "hygt_inverse_batch_f32", y, out,
                         torch.float32, torch.float32, status, stream)


class MixedBatch:
    """Blocks of several sizes (N = 16, 64, 256) transformed in one launch.

    ``classes`` is a list of (plan, x, sets) with x an int16 CUDA tensor
    [nblocks, N] and sets an int16/uint16 CUDA tensor [nblocks] (or None).
    The object owns the coefficient and reconstruction tensors and one
    schedule workspace per class.
    """

    def __init__(self, classes, device=None):
        import torch
        self.entries = []
        arr = (MixedClass * len(classes))()
        for i, (plan, x, sets) in enumerate(classes):
            nb = int(x.shape[0])
            dev = device or x.device
            work = torch.empty(max(1, hygt_batch_workspace_bytes(plan.handle, nb)),
                               dtype=torch.uint8, device=dev)
            y = torch.empty((nb, plan.N), dtype=torch.int32, device=dev)
            xr = torch.empty((nb, plan.N), dtype=torch.int16, device=dev)
            _dptr(x, torch.int16, plan.N, "x")
            ps = None
            if sets is not None:
                ps = _dptr(sets, torch.int16 if sets.dtype == torch.int16 else torch.uint16,
                           None, "sets")
                if sets.numel() != nb:
                    raise ValueError("class %d: sets must have one entry per block" % i)
            arr[i] = MixedClass(plan.handle, ps, nb, work.data_ptr(), work.numel(),
                                x.data_ptr(), y.data_ptr(), xr.data_ptr(), 0)
            self.entries.append({"plan": plan, "x": x, "sets": sets, "y": y, "xr": xr,
                                 "work": work})
        self.classes = arr
        self.n = len(classes)

    def set_split(self, ctas):
        """CTAs of the mixed launch per class: all > 0, the classes run
        concurrently on these CTAs; all -1, one batch launch per class; None
        or zeros, every CTA runs every class in turn."""
        for i in range(self.n):
            self.classes[i].ctas = 0 if ctas is None else int(ctas[i])

    def variants(self):
        """Per class, ((stage, layout) forward, (stage, layout) inverse):
        what a single mixed launch runs it in under the plans' tuning."""
        return [(hygt_mixed_class_variant(e["plan"].handle, 0),
                 hygt_mixed_class_variant(e["plan"].handle, 1)) for e in self.entries]

    def build(self, stream=None):
        for i, e in enumerate(self.entries):
            c = self.classes[i]
            _check(hygt_batch_build(c.plan, c.d_set, c.nblocks, c.d_work, c.work_bytes,
                                    _stream_handle(stream)), "hygt_batch_build")
        return self

    def forward(self, status=None, stream=None):
        import torch
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        _check(hygt_forward_mixed(self.classes, self.n, _stream_handle(stream), pst),
               "hygt_forward_mixed")

    def inverse(self, status=None, stream=None):
        import torch
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        _check(hygt_inverse_mixed(self.classes, self.n, _stream_handle(stream), pst),
               "hygt_inverse_mixed")

    def graph(self, status=None):
        """A CUDA graph of one step: schedules, mixed forward, mixed inverse."""
        import torch
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        st, h = hygt_mixed_graph_create(self.classes, self.n, pst)
        _check(st, "hygt_mixed_graph_create")
        return Graph(h)


class Graph:
    def __init__(self, handle):
        self.handle = handle

    def launch(self, stream=None):
        _check(hygt_graph_launch(self.handle, _stream_handle(stream)), "hygt_graph_launch")

    def close(self):
        if getattr(self, "handle", None):
            hygt_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class HyGTFunction(torch.autograd.Function):
        """y = HyGT(theta) x on FP32 blocks; backward recomputes the passes
        from y (nothing is stored between forward and backward)."""

        @staticmethod
        def forward(ctx, x, theta, plan, sets):
            plan.update_theta(theta.detach())
            y = plan.forward_f32(x.contiguous(), sets)
            ctx.save_for_backward(y)
            ctx.plan = plan
            ctx.sets = sets
            ctx.theta_shape = theta.shape
            return y

        @staticmethod
        def backward(ctx, gy):
            (y,) = ctx.saved_tensors
            gx, gth = ctx.plan.backward_f32(y, gy.contiguous(), ctx.sets)
            return gx, gth.to(torch.float32).view(ctx.theta_shape), None, None

    return HyGTFunction


_HYGT_FN = None


def hygt_function(x, theta, plan, sets=None):
    """Differentiable HyGT: x float32 [B, N] (CUDA), theta float32 CUDA tensor
    of the angles [S, R, log2 N, N/2]; ``plan`` an FP32 plan of that shape."""
    global _HYGT_FN
    if _HYGT_FN is None:
        _HYGT_FN = _autograd_function()
    return _HYGT_FN.apply(x, theta, plan, sets)


def HyGTLayer(log2n, rounds, num_sets=1, perms=None, theta=None, seed=0):
    """A torch.nn.Module holding the angles as a parameter."""
    import torch

    class _Layer(torch.nn.Module):
        def __init__(self):
            super().__init__()
            N = 1 << log2n
            shape = (num_sets, rounds, log2n, N // 2)
            if theta is None:
                g = torch.Generator().manual_seed(seed)
                t0 = (torch.rand(shape, generator=g, dtype=torch.float64) * 2 - 1) * np.pi
            else:
                t0 = torch.as_tensor(np.asarray(theta, np.float64)).reshape(shape)
            self.theta = torch.nn.Parameter(t0.to(torch.float32).cuda())
            self.plan = Plan.from_theta(log2n, rounds, t0.numpy().astype(np.float32), perms)

        def forward(self, x, sets=None):
            return hygt_function(x, self.theta, self.plan, sets)

    return _Layer()


class DenseKLT:
    """Dense per-set matrix transform (the matrix baseline), y = K[set] x."""

    def __init__(self, log2n, K, frac_bits=8):
        K = np.ascontiguousarray(K, dtype=np.float32)
        self.log2n = int(log2n)
        self.N = 1 << self.log2n
        self.num_sets = K.shape[0]
        st, h = dense_klt_create(self.log2n, self.num_sets, K, frac_bits)
        _check(st, "dense_klt_create")
        self.handle = h
        self.work = None
        self.nblocks = None

    def build(self, sets, nblocks, stream=None):
        import torch
        nblocks = int(nblocks)
        if sets is not None and sets.numel() != nblocks:
            raise ValueError("sets must have one entry per block")
        nbytes = dense_klt_workspace_bytes(self.handle, nblocks)
        if nbytes == 0 and nblocks > 0:
            raise HygtError(HYGT_ERR_ARG, "dense_klt_workspace_bytes")
        ps = None
        if sets is not None:
            ps = _dptr(sets, torch.int16 if sets.dtype == torch.int16 else torch.uint16, None, "sets")
        if self.work is None or self.work.numel() < nbytes:
            self.work = torch.empty(max(1, nbytes), dtype=torch.uint8, device="cuda")
        self.nblocks = nblocks
        _check(dense_klt_build(self.handle, ps, self.nblocks, self.work.data_ptr(),
                               self.work.numel(), _stream_handle(stream)), "dense_klt_build")
        return self

    def apply(self, x, kind=DENSE_KLT_BF16, out=None, status=None, stream=None):
        """int16 x [nblocks, N] -> out [nblocks, N]: int32 for DENSE_KLT_INT,
        float32 otherwise; ``build`` must have been called for nblocks."""
        import torch
        if self.work is None or self.nblocks is None:
            raise RuntimeError("DenseKLT.apply before build")
        if x.dim() != 2 or x.shape[0] != self.nblocks:
            raise ValueError("schedule built for %d blocks, x has shape %s"
                             % (self.nblocks, tuple(x.shape)))
        dt = torch.int32 if kind == DENSE_KLT_INT else torch.float32
        if out is None:
            out = torch.empty((x.shape[0], self.N), dtype=dt, device=x.device)
        elif out.dim() != 2 or out.shape[0] != self.nblocks:
            raise ValueError("out must have shape [%d, %d]" % (self.nblocks, self.N))
        px = _dptr(x, torch.int16, self.N, "x")
        po = _dptr(out, dt, self.N, "out")
        pst = None if status is None else _dptr(status, torch.int32, None, "status")
        _check(dense_klt_apply(self.handle, self.work.data_ptr(), px, po, self.nblocks, kind,
                               _stream_handle(stream), pst), "dense_klt_apply")
        return out

    def close(self):
        if getattr(self, "handle", None):
            dense_klt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
