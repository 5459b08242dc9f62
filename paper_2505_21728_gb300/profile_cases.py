"""One kernel case at a time, for profiling (ncu) and quick timing.

    python -m paper_2505_21728_gb300.profile_cases CASE [--nblocks N] [--reps R]

Each case builds its synthetic inputs, runs its kernels twice untimed
(warm-up), then R more times, and prints the mean CUDA-event time of one
repetition.  Under ncu, skip the warm-up launches with -s and capture with -c.

Cases:
  batch      bucket + integer forward + integer inverse, 8x8 blocks, 105 sets
  direct     direct integer forward + inverse (no bucketing), same workload
  mixed      mixed 4x4/8x8/16x16 frame batch, mixed forward + inverse
  dense      dense matrix transform, tcgen05 BF16 and int32, same 8x8 blocks
  grad       FP32 forward + backward on the 8x8 / 4-round fitting workload
  stress     bucket + integer forward + inverse, 16x16 blocks, 3 rounds, 16 sets
"""
from __future__ import annotations

import argparse
import sys

import numpy as np


def _dev():
    import torch
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def _int_workload(name, nblocks):
    import torch
    from . import hygt, workloads
    w = workloads.get(name)
    if nblocks:
        w = workloads.truncated(w, nblocks)
    d = w.generate()
    plan = hygt.Plan(w.log2n, w.rounds, d["angle_idx"], d["perms"])
    x = torch.from_numpy(d["x"]).cuda()
    s = torch.from_numpy(d["sets"].view(np.int16)).cuda()
    return w, d, plan, x, s


def case_batch(args, name="hygt8x8_r2_s105"):
    import torch
    from . import hygt
    w, d, plan, x, s = _int_workload(name, args.nblocks)
    b = hygt.Batch(plan, x.shape[0])
    y = torch.empty((x.shape[0], w.N), dtype=torch.int32, device="cuda")
    xr = torch.empty_like(x)

    def run():
        b.build(s)
        b.forward(x, out=y)
        b.inverse(y, out=xr)
    return run


def case_direct(args):
    import torch
    w, d, plan, x, s = _int_workload("hygt8x8_r2_s105", args.nblocks)
    y = torch.empty((x.shape[0], w.N), dtype=torch.int32, device="cuda")
    xr = torch.empty_like(x)

    def run():
        plan.forward(x, s, out=y)
        plan.inverse(y, s, out=xr)
    return run


def case_mixed(args):
    import torch
    from . import autotune, hygt, workloads
    w = workloads.get_mixed("mixed_frame_2160p16", scale_down=args.scale_down)
    classes = []
    for cw in w.classes():
        d = cw.generate()
        plan = hygt.Plan(cw.log2n, cw.rounds, d["angle_idx"], d["perms"])
        classes.append((plan, torch.from_numpy(d["x"]).cuda(),
                        torch.from_numpy(d["sets"].view(np.int16)).cuda()))
    mb = hygt.MixedBatch(classes)
    mb.build()
    if not args.no_tune:
        autotune.tune_split(mb, reps=3, use_cache=False)

    def run():
        mb.forward()
        mb.inverse()
    return run


def case_dense(args):
    import torch
    from . import hygt
    w, d, plan, x, s = _int_workload("hygt8x8_r2_s105", args.nblocks)
    dk = hygt.DenseKLT(w.log2n, plan.dense_matrices()).build(s, x.shape[0])
    y = torch.empty((x.shape[0], w.N), dtype=torch.float32, device="cuda")
    yi = torch.empty((x.shape[0], w.N), dtype=torch.int32, device="cuda")

    def run():
        dk.apply(x, kind=hygt.DENSE_KLT_BF16, out=y)
        dk.apply(x, kind=hygt.DENSE_KLT_INT, out=yi)
    return run


def case_grad(args):
    import torch
    from . import hygt, workloads
    w = workloads.get_fit("hygt8x8_r4_fit")
    n = args.nblocks or w.nvec
    x = torch.from_numpy(w.patches(n)).cuda()
    plan = hygt.Plan.from_theta(w.log2n, w.rounds, w.theta0().astype(np.float32))
    mask = torch.zeros(w.N, device="cuda")
    mask[w.keep:] = 2.0 / n
    y = torch.empty_like(x)

    def run():
        plan.forward_f32(x, out=y)
        plan.backward_f32(y, y * mask)
    return run


def case_stress(args):
    return case_batch(args, name="hygt16x16_r3_s16")


CASES = {"batch": case_batch, "direct": case_direct, "mixed": case_mixed, "dense": case_dense,
         "grad": case_grad, "stress": case_stress}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--nblocks", type=int, default=0, help="first N blocks of the workload")
    ap.add_argument("--scale-down", type=int, default=1, help="mixed: divide the block counts")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--no-tune", action="store_true", help="mixed: default CTA split")
    args = ap.parse_args(argv)
    import torch
    from . import build
    build.build()
    _dev()
    run = CASES[args.case](args)
    run()
    run()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.reps):
        run()
    b.record()
    torch.cuda.synchronize()
    print("%s: %.4f ms per repetition" % (args.case, a.elapsed_time(b) / max(1, args.reps)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
