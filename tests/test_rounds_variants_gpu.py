"""Rounds variants H(R) (Table II columns H(2) .. H(5)) fitted on the GPU
with the coding-gain objective of Sec. V and quantised to one byte per
angle (Sec. IV), on correlated 4x4 and 8x8 patches.

Checked against the FP64 oracle (oracle/coding_gain.py, with the batch's
own correlation): J at the fitted angles and at the 8-bit angles; the KLT
bound (Eq. 2) is never crossed; a larger R, started from the smaller
variant, ends at least as low; 8-bit angles cost little; the integer
transform of the 8-bit angles is bit-exact with the oracle on the scaled
patches; and the parameter memory reproduces Table II's memory ratios.
"""
import math
import os

import numpy as np
import pytest

from oracle import coding_gain as cg
from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table2_ratios():
    rows = {}
    with open(os.path.join(GOLDEN, "table2_memory_ratios.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                tok = line.split()
                rows[tok[0]] = tuple(float(v) for v in tok[1:])
    return {4: {2: rows["H(2)/K"][0], 3: rows["H(3)/K"][0]},
            6: {3: rows["K/H(3)"][1], 4: rows["K/H(4)"][1], 5: rows["K/H(5)"][1]}}


@pytest.mark.parametrize("log2n,rounds_list", [(4, (2, 3)), (6, (3, 4, 5))])
def test_rounds_ladder(gpu, orc, log2n, rounds_list):
    import torch
    from paper_2505_21728_gb300 import fit
    N = 1 << log2n
    side = int(round(math.sqrt(N)))
    x = inputs.ar1_patches(1 << 17, side, seed=3)
    x64 = x.astype(np.float64)
    phi = x64.T @ x64 / x64.shape[0]
    bound = cg.klt_bound(phi)
    res = fit.rounds_ladder(torch.from_numpy(x).cuda(), log2n, rounds_list, iters=150,
                            restarts=2, seed=1)
    ratios = _table2_ratios()[log2n]
    prev_J = None
    for r in res:
        R = r["rounds"]
        Je = cg.objective(r["theta"].astype(np.float64), log2n, R, phi)
        assert abs(r["J"] - Je) <= 1e-5 * max(1.0, abs(Je))
        th_q = r["q"].astype(np.float64) * (2 * math.pi / 256)
        Jqe = cg.objective(th_q, log2n, R, phi)
        assert abs(r["J_q"] - Jqe) <= 1e-5 * max(1.0, abs(Jqe))
        assert r["J"] >= bound - 1e-9 and r["J_q"] >= bound - 1e-9
        # one byte per angle is enough (Sec. IV), read as: rounding the angles
        # to 8 bits costs at most 0.02 bit per coefficient of the objective
        assert r["J_q"] - r["J"] <= 0.02
        if prev_J is not None:
            assert r["J"] <= prev_J + 1e-3        # started from the smaller variant
        prev_J = r["J"]
        # memory: KLT N^2 bytes against R N log2(N) / 2 bytes (Table II)
        assert r["param_bytes"] == R * N * log2n // 2
        assert abs(N * N / r["param_bytes"] - ratios[R]) <= 0.05 + 1e-9
        # the integer transform of the 8-bit angles on patches scaled to int16
        xi = np.clip(np.rint(x[:50000] * 64.0), -32768, 32767).astype(np.int16)
        plan = gpu.Plan(log2n, R, r["q"][None])
        yi = plan.forward(torch.from_numpy(xi).cuda()).cpu().numpy()
        ye, st = orc.fwd_int(xi, r["q"][None], log2n, R)
        assert st == 0 and np.array_equal(yi, ye)
        plan.close()
    assert res[-1]["J"] < res[0]["J"]
