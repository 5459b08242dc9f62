"""Host-side checks of the C ABI (no GPU needed, no compute call).

The library is compiled here (nvcc cross-compiles for sm_103a), loaded, and
checked to export every function declared in include/*.h.  Argument
validation that happens before any CUDA call, the closed-form parameter
count and the status strings are checked too.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_21728_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_]\w*)\s*\(", text):
            name = m.group(1)
            # a declaration: the identifier follows a type, not a keyword or macro
            prefix = text[:m.start()].rstrip()
            if name in ("if", "sizeof", "defined") or prefix.endswith("#define"):
                continue
            if re.search(r"(hygt_status|void|size_t|char\s*\*|int|const char \*)\s*\**\s*$", prefix):
                names.add(name)
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hygt_create", "hygt_create_float", "hygt_destroy", "hygt_forward",
                 "hygt_inverse", "hygt_forward_f32", "hygt_inverse_f32",
                 "hygt_param_bytes", "hygt_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, "not exported: %s" % missing


def test_param_bytes_closed_form(lib):
    from paper_2505_21728_gb300 import hygt
    # R N log2(N) / 2 angles at one byte each (Sec. IV)
    assert hygt.hygt_param_bytes(4, 2, 1) == 2 * 16 * 4 // 2
    assert hygt.hygt_param_bytes(6, 3, 105) == 105 * 3 * 64 * 6 // 2
    assert hygt.hygt_param_bytes(8, 3, 16) == 16 * 3 * 256 * 8 // 2
    assert hygt.hygt_param_bytes(0, 2, 1) == 0
    # Table II: KLT 8x8 (4096 bytes) over HyGT H(3) on 8x8 = 7.1
    assert round(64 * 64 / hygt.hygt_param_bytes(6, 3, 1), 1) == 7.1
    assert round(16 * 16 / hygt.hygt_param_bytes(4, 2, 1), 1) == 4.0


def test_status_strings(lib):
    from paper_2505_21728_gb300 import hygt
    assert hygt.hygt_status_string(0) == "ok"
    assert "argument" in hygt.hygt_status_string(1)
    assert "set index" in hygt.hygt_status_string(4)
    assert hygt.hygt_status_string(99) == "unknown status"


def test_create_rejects_bad_arguments_before_any_cuda_call(lib):
    from paper_2505_21728_gb300 import hygt
    q = np.zeros((1, 2, 4, 8), np.uint8)
    assert hygt.hygt_create(0, 2, 1, q)[0] == hygt.HYGT_ERR_ARG          # log2n
    assert hygt.hygt_create(9, 2, 1, q)[0] == hygt.HYGT_ERR_ARG
    assert hygt.hygt_create(4, 0, 1, q)[0] == hygt.HYGT_ERR_ARG          # rounds
    assert hygt.hygt_create(4, 2, 0, q)[0] == hygt.HYGT_ERR_ARG          # sets
    assert hygt.hygt_create(4, 2, 1, q, None, 9, 8)[0] == hygt.HYGT_ERR_ARG   # angle bits
    assert hygt.hygt_create(4, 2, 1, q, None, 8, 11)[0] == hygt.HYGT_ERR_ARG  # frac bits
    q6 = np.full((1, 2, 4, 8), 200, np.uint8)  # index >= 2^6
    assert hygt.hygt_create(4, 2, 1, q6, None, 6, 8)[0] == hygt.HYGT_ERR_ARG
    bad_perm = np.tile(np.arange(16, dtype=np.uint16), (1, 2, 1))
    bad_perm[0, 0, 3] = 4  # duplicate entry
    assert hygt.hygt_create(4, 2, 1, q, bad_perm)[0] == hygt.HYGT_ERR_ARG
    bad_perm[0, 0, 3] = 16  # out of range
    assert hygt.hygt_create(4, 2, 1, q, bad_perm)[0] == hygt.HYGT_ERR_ARG
    theta = np.full((1, 2, 4, 8), np.nan, np.float32)
    assert hygt.hygt_create_float(4, 2, 1, theta)[0] == hygt.HYGT_ERR_ARG


def test_calls_reject_null_plan(lib):
    from paper_2505_21728_gb300 import hygt
    assert hygt.hygt_forward(None, None, None, None, 1, None, None) == hygt.HYGT_ERR_ARG
    assert hygt.hygt_inverse(None, None, None, None, 0, None, None) == hygt.HYGT_ERR_ARG
    assert lib.hygt_mixed_class_variant(None, 0, None, None) == hygt.HYGT_ERR_ARG
