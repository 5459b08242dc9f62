"""Angle fitting with the coding-gain objective of Sec. V (GPU).

The paper optimises the HyGT angles of each class for the highest transform
coding gain, using the variance vector v = diag(T Phi T^T) of the outputs and
a high-rate rate-distortion model, and repeats the non-convex search from
several initialisations, keeping the best local optimum (Sec. V; the
optimiser itself is left out of the paper).  ``CodingGainFit`` does this on
a batch of FP32 blocks: every iteration runs the library's kernels only --

    hygt_update_theta      angles -> (cos, sin) table
    hygt_forward_f32       y = T x
    hygt_coding_gain_f32   v, J = 1/(2N) sum log2 v_i, weights w (dJ/dy = w y)
    hygt_backward_diag_f32 dJ/dtheta (recomputing backward, dL/dy formed in
                           registers, dL/dx not written)
    hygt_adam_step         theta <- Adam(theta, dJ/dtheta)

-- and ``fit`` keeps the best of several seeded restarts.  This module only
allocates device buffers and sequences the calls.
"""
from __future__ import annotations

import math

import numpy as np

from . import hygt


class CodingGainFit:
    """Minimises J(theta) = 1/(2N) sum_i log2 v_i over the angles of an FP32
    HyGT (one class, no set indices) on the blocks ``x`` (float32 CUDA
    tensor [B, N])."""

    def __init__(self, x, log2n, rounds, perms=None):
        import torch
        self.log2n, self.rounds = int(log2n), int(rounds)
        self.N = 1 << self.log2n
        if x.dim() != 2 or x.shape[1] != self.N or x.dtype != torch.float32 or not x.is_cuda:
            raise ValueError("x must be a float32 CUDA tensor [B, %d]" % self.N)
        self.x = x.contiguous()
        self.B = int(x.shape[0])
        self.angles = self.rounds * self.log2n * (self.N // 2)
        self.plan = hygt.Plan.from_theta(self.log2n, self.rounds,
                                         np.zeros(self.angles, np.float32), perms)
        dev = x.device
        self.y = torch.empty_like(self.x)
        self.v = torch.empty(self.N, dtype=torch.float64, device=dev)
        self.w = torch.empty(self.N, dtype=torch.float32, device=dev)
        self.gtheta = torch.empty(self.angles, dtype=torch.float64, device=dev)
        self.theta = torch.empty(self.angles, dtype=torch.float32, device=dev)
        self.m = torch.zeros(self.angles, dtype=torch.float32, device=dev)
        self.s = torch.zeros(self.angles, dtype=torch.float32, device=dev)
        wb = hygt.hygt_backward_workspace_bytes(self.plan.handle, self.B)
        wc = hygt.hygt_coding_gain_workspace_bytes(self.plan.handle, self.B)
        if wb == 0 or wc == 0:
            raise hygt.HygtError(hygt.HYGT_ERR_UNSUPPORTED, "workspace size")
        self.work_b = torch.empty(wb, dtype=torch.uint8, device=dev)
        self.work_c = torch.empty(wc, dtype=torch.uint8, device=dev)

    # -- the calls of one iteration ------------------------------------------
    def _objective(self, J_ptr, stream):
        h = self.plan.handle
        hygt._check(hygt.hygt_update_theta(h, self.theta.data_ptr(), stream), "hygt_update_theta")
        hygt._check(hygt.hygt_forward_f32(h, self.x.data_ptr(), self.y.data_ptr(), None, self.B,
                                          stream, None), "hygt_forward_f32")
        hygt._check(hygt.hygt_coding_gain_f32(h, self.y.data_ptr(), self.B, self.v.data_ptr(),
                                              self.w.data_ptr(), J_ptr, self.work_c.data_ptr(),
                                              self.work_c.numel(), stream),
                    "hygt_coding_gain_f32")

    def _gradient(self, stream):
        hygt._check(hygt.hygt_backward_diag_f32(self.plan.handle, self.y.data_ptr(),
                                                self.w.data_ptr(), None, self.gtheta.data_ptr(),
                                                None, self.B, self.work_b.data_ptr(),
                                                self.work_b.numel(), stream, None),
                    "hygt_backward_diag_f32")

    def objective(self, theta):
        """(J, v) at the angles ``theta`` (array-like, R * log2 N * N/2)."""
        import torch
        self.theta.copy_(torch.as_tensor(np.asarray(theta, np.float32).ravel()))
        J = torch.empty(1, dtype=torch.float64, device=self.x.device)
        self._objective(J.data_ptr(), hygt._stream_handle())
        return float(J.item()), self.v.cpu().numpy().copy()

    def objective_grad(self, theta):
        """(J, dJ/dtheta as float64 [R, log2 N, N/2]) at ``theta``."""
        import torch
        self.theta.copy_(torch.as_tensor(np.asarray(theta, np.float32).ravel()))
        J = torch.empty(1, dtype=torch.float64, device=self.x.device)
        stream = hygt._stream_handle()
        self._objective(J.data_ptr(), stream)
        self._gradient(stream)
        return (float(J.item()),
                self.gtheta.cpu().numpy().reshape(self.rounds, self.log2n, self.N // 2))

    def run(self, theta0, iters, lr=0.02, beta1=0.9, beta2=0.999, eps=1e-12):
        """Adam from ``theta0`` for ``iters`` steps.  Returns (theta, J of
        every iteration before its step, J at the final angles)."""
        import torch
        self.theta.copy_(torch.as_tensor(np.asarray(theta0, np.float32).ravel()))
        self.m.zero_()
        self.s.zero_()
        hist = torch.empty(iters + 1, dtype=torch.float64, device=self.x.device)
        stream = hygt._stream_handle()
        for it in range(iters):
            self._objective(hist[it:].data_ptr(), stream)
            self._gradient(stream)
            hygt._check(hygt.hygt_adam_step(self.theta.data_ptr(), self.gtheta.data_ptr(),
                                            self.m.data_ptr(), self.s.data_ptr(), self.angles,
                                            lr, beta1, beta2, eps, it + 1, stream),
                        "hygt_adam_step")
        self._objective(hist[iters:].data_ptr(), stream)
        h = hist.cpu().numpy()
        return self.theta.cpu().numpy().reshape(self.rounds, self.log2n, self.N // 2), h[:-1], \
            float(h[-1])

    def fit(self, restarts, iters, lr=0.02, seed=0):
        """Seeded restarts (angles uniform in [-pi, pi)); the best final J
        wins.  Returns (theta, J, final J of every restart)."""
        best, best_J, finals = None, math.inf, []
        for r in range(restarts):
            rng = np.random.default_rng([int(seed), r])
            th0 = rng.uniform(-math.pi, math.pi, self.angles)
            th, _, J = self.run(th0, iters, lr)
            finals.append(J)
            if J < best_J:
                best, best_J = th, J
        return best, best_J, finals

    def close(self):
        self.plan.close()


def quantise_angles(theta, angle_bits=8):
    """The nearest angle index q = round(theta 2^bits / 2 pi) mod 2^bits of
    each angle (one byte per parameter at 8 bits, Sec. IV)."""
    t = np.asarray(theta, np.float64)
    q = np.rint(t * (1 << angle_bits) / (2.0 * math.pi)).astype(np.int64) % (1 << angle_bits)
    return q.astype(np.uint8)


def rounds_ladder(x, log2n, rounds_list, iters, lr=0.02, restarts=3, seed=0, angle_bits=8):
    """HyGT variants H(R) for increasing R fitted to one class (Table II's
    columns H(2) .. H(5); Sec. V objective), each quantised to one byte per
    angle (Sec. IV).

    The smallest R is fitted with seeded restarts; every larger R starts
    from the previous variant's angles with the added rounds at zero angle
    (the identity), so it starts from the previous variant's transform and
    objective.  Returns one dict per R: the FP32 angles, J, the 8-bit
    angle indices q, J at the angles q stands for, and the parameter bytes
    at one byte per angle.
    """
    out = []
    prev = None
    N = 1 << int(log2n)
    for R in sorted(rounds_list):
        f = CodingGainFit(x, log2n, R)
        if prev is None:
            th, J, _ = f.fit(restarts, iters, lr=lr, seed=seed)
        else:
            th0 = np.zeros((R, log2n, N // 2), np.float64)
            th0[:prev.shape[0]] = prev
            th, _, J = f.run(th0, iters, lr=lr)
        q = quantise_angles(th, angle_bits)
        Jq, _ = f.objective(q.astype(np.float64) * (2.0 * math.pi / (1 << angle_bits)))
        out.append({"rounds": R, "theta": th, "J": J, "q": q, "J_q": Jq,
                    "param_bytes": hygt.hygt_param_bytes(int(log2n), R, 1)})
        prev = th
        f.close()
    return out
