#!/usr/bin/env python
"""Throughput of the integer HyGT forward + inverse on GB300.

One step = integer forward HyGT then integer inverse HyGT over every block
of the workload (default: 8x8 blocks, N = 64, 2 rounds, 105 sets,
4,194,304 Laplacian int16 blocks), inputs resident in HBM.  Prints one JSON
line (rank 0).  ``--impl reference`` times the CPU oracle on a bounded
sample of the same workload instead.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
``torch.distributed.run`` (one process per GPU, NCCL).  Blocks are
independent, so every rank transforms its own full batch (weak scaling) and
there is no collective on the data path; the barrier and the max-over-ranks
reduction of the timed region are the only communication.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HyGT blocks/s (fwd+inv, int32 bit-exact) & % HBM roofline vs dense-KLT on same GB300"
DEFAULT_WORKLOAD = "hygt8x8_r2_s105"
L2_BYTES = 129 * 1024 * 1024


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the timed oracle sample (for profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary workloads (mixed block sizes)")
    ap.add_argument("--nblocks", type=int, default=0,
                    help="use only the first N blocks of the workload (profiling cases)")
    ap.add_argument("--case", choices=sorted(CASES), default=None,
                    help="run one kernel case instead of the benchmark (for ncu): its "
                         "kernels twice untimed, then --reps times, and print the mean "
                         "CUDA-event time of one repetition")
    ap.add_argument("--reps", type=int, default=1, help="--case: timed repetitions")
    ap.add_argument("--scale-down", type=int, default=1,
                    help="--case mixed: divide the frame batch's block counts")
    ap.add_argument("--no-tune", action="store_true",
                    help="--case mixed: default CTA split instead of the autotuner's")
    ap.add_argument("--autotune-cache", action="store_true",
                    help="reuse the launch tuning cached by an earlier run (profiling runs "
                         "then launch no tuning kernels)")
    ap.add_argument("--fwd-tuning", default=None,
                    help="--case batch/stress: launch tuning of the forward, "
                         "'warps,ctas_per_sm,stage[,layout[,tail_64ths]]' "
                         "(hygt_batch_set_tuning, hygt_batch_set_tail)")
    ap.add_argument("--inv-tuning", default=None, help="the same for the inverse")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_blocks(nblocks: int, rank: int, world: int, weak: bool = True):
    """Blocks a rank transforms: the full batch under weak scaling, else a
    contiguous 1/world share (remainder to the lowest ranks)."""
    if weak:
        return 0, nblocks
    base, rem = divmod(nblocks, world)
    start = rank * base + min(rank, rem)
    return start, base + (1 if rank < rem else 0)


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except OSError:
            return None
        if not rows:
            return None

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        top = max(sm) if sm else 0
        loaded = [s for s in sm if s >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- helpers
def gpu_smi_id(dev, local):
    """nvidia-smi selector of this CUDA device: its UUID when torch exposes
    it (nvidia-smi indices ignore CUDA_VISIBLE_DEVICES), else the index."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(local)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# the sources of the set-bucketed integer kernels (the benchmark's dominant kernels)
BATCH_SOURCES = ("hygt_batch.cuh", "hygt_batch_launch.cuh", "hygt_device.cuh", "hygt_primary.cuh",
                 "hygt_launch.cuh", "batch_int.cu", "batch_fwd.cu", "batch_inv.cu",
                 "batch_n_small.cu", "batch_n_4_fwd.cu", "batch_n_4_inv.cu", "batch_n_5.cu",
                 "batch_n_6_fwd.cu", "batch_n_6_inv.cu", "batch_n_7.cu", "batch_n_8_fwd.cu",
                 "batch_n_8_inv.cu")


def kernel_source_sha(files=BATCH_SOURCES) -> str:
    h = hashlib.sha256()
    for name in sorted(files):
        p = os.path.join(ROOT, "paper_2505_21728_gb300", "csrc", name)
        with open(p, "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str, tuning=None):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources and (when given) the same kernel variant: a
    line 'bench-traffic: kernel=... workload=... sha=... variant=s,l
    bytes_per_launch=...' in profiles/*.md, with s the staging choice and l
    the register layout of the launch tuning (warps per CTA and CTAs per SM
    change the launch, not the bytes a launch moves); else None.
    ``tuning``: (warps, ctas_per_sm, stage[, layout, ...])."""
    sha = kernel_source_sha()
    want = None
    if tuning is not None:
        lay = int(tuning[3]) if len(tuning) > 4 else 0
        want = "%d,%d" % (int(tuning[2]), lay)
        if len(tuning) > 5 and int(tuning[5]) > 0:  # the kernel with a dynamic tail
            want += ",tail%d" % int(tuning[5])
    for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(p) as f:
            for line in f:
                if not line.startswith("bench-traffic:"):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                if kv.get("kernel") == kernel and kv.get("workload") == workload \
                        and kv.get("sha") == sha and (want is None or kv.get("variant") == want):
                    return int(float(kv["bytes_per_launch"]))
    return None


# ---------------------------------------------------------------- CPU oracle leg
def oracle_sample(w, data, nblk):
    """Times the oracle's integer forward + inverse on the first nblk blocks."""
    import oracle
    oracle.build()
    x = data["x"][:nblk]
    s = None if data["sets"] is None else data["sets"][:nblk]
    t0 = time.perf_counter()
    y, st1 = oracle.fwd_int(x, data["angle_idx"], w.log2n, w.rounds, data["perms"], s)
    _, st2 = oracle.inv_int(y, data["angle_idx"], w.log2n, w.rounds, data["perms"], s)
    dt = time.perf_counter() - t0
    if st1 or st2:
        raise RuntimeError("oracle reported status %d/%d" % (st1, st2))
    return dt, oracle.num_threads()


def cpu_baseline(w, data, target_s=10.0):
    """The oracle, as it stands, on a bounded sample: the first blocks of the
    workload (all of it if it is small enough), repeated to about target_s."""
    nblk = min(w.nblocks, 16384)
    dt, cores = oracle_sample(w, data, nblk)
    per_block = dt / nblk
    nblk = int(min(w.nblocks, max(nblk, target_s / max(per_block, 1e-12))))
    reps = max(1, int(round(target_s / max(per_block * nblk, 1e-9))))
    total = 0.0
    for _ in range(reps):
        dt, cores = oracle_sample(w, data, nblk)
        total += dt
    return {"value": nblk * reps / total, "unit": "blocks/s", "cores": cores, "kind": "oracle",
            "sample": "integer forward + inverse of the first %d blocks of %s, %d time(s) "
                      "(C oracle, int64 arithmetic, OpenMP over blocks), %.1f s"
                      % (nblk, w.name, reps, total)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2505_21728_gb300 import workloads
    w = workloads.get(args.workload)
    nblk = min(w.nblocks, 65536)
    data = {"x": w.blocks(0, nblk), "sets": w.set_indices()[:nblk]}
    data["angle_idx"], data["perms"] = w.params()
    for _ in range(args.warmup):
        oracle_sample(w, data, nblk)
    times = []
    cores = 1
    for _ in range(args.steps):
        dt, cores = oracle_sample(w, data, nblk)
        times.append(dt)
    total = sum(times)
    value = nblk * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "blocks/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": w.name, "nblocks_per_step": nblk, "N": w.N, "rounds": w.rounds,
                   "sets": w.num_sets},
        "cpu_baseline": {"value": value, "unit": "blocks/s", "cores": cores, "kind": "oracle",
                         "sample": "first %d blocks of %s per step" % (nblk, w.name)},
        "e2e": {"value": value, "unit": "blocks/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg
def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2505_21728_gb300 import build
    build.build()
    from paper_2505_21728_gb300 import hygt, workloads

    w = workloads.get(args.workload)
    if args.nblocks:
        w = workloads.truncated(w, args.nblocks)
    data = w.generate()
    start, count = shard_blocks(w.nblocks, rank, world, weak=True)
    x_np = data["x"][start:start + count]
    s_np = data["sets"][start:start + count]
    plan = hygt.Plan(w.log2n, w.rounds, data["angle_idx"], data["perms"])
    N = w.N
    d_x = torch.from_numpy(x_np).to(dev)
    d_s = torch.from_numpy(s_np.view(np.int16)).to(dev)
    d_y = torch.empty((count, N), dtype=torch.int32, device=dev)
    d_xr = torch.empty((count, N), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)
    batch = hygt.Batch(plan, count, device=dev)
    # launch tuning (warps per CTA, CTAs per SM, staging) by the autotuner,
    # outside the timed region
    from paper_2505_21728_gb300 import autotune
    batch.build(d_s)
    tuning = autotune.tune_batch(batch, d_x, d_y, d_xr, reps=3, use_cache=args.autotune_cache)

    # One step: bucket the batch by set, forward, inverse (5 kernels).
    K = args.steps
    W = max(3, args.warmup)
    for _ in range(W):
        batch.build(d_s)
        batch.forward(d_x, out=d_y)
        batch.inverse(d_y, out=d_xr)
    torch.cuda.synchronize(dev)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * K + 1)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_smi_id(dev, local))
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    t_start.record(stream)
    ev[0].record(stream)
    for k in range(K):
        batch.build(d_s)
        ev[3 * k + 1].record(stream)
        batch.forward(d_x, out=d_y)
        ev[3 * k + 2].record(stream)
        batch.inverse(d_y, out=d_xr)
        ev[3 * k + 3].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clock_info = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    build_ms = [ev[3 * k].elapsed_time(ev[3 * k + 1]) for k in range(K)]
    fwd_ms = [ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(K)]
    inv_ms = [ev[3 * k + 2].elapsed_time(ev[3 * k + 3]) for k in range(K)]
    total_ms = max_over_ranks(total_ms, world, dev)

    blocks_total = count * world * K
    value = blocks_total / (total_ms / 1000.0)

    # roofline of the dominant kernel (algorithmic bytes / average duration)
    bytes_per_launch = count * (2 * N + 4 * N + 2)  # same for forward and inverse
    f_avg, i_avg = statistics.mean(fwd_ms), statistics.mean(inv_ms)
    dom_name, dom_ms = (("hygt_batch_forward", f_avg) if f_avg >= i_avg
                        else ("hygt_batch_inverse", i_avg))
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / (dom_ms / 1000.0) / 1e9
    step_bytes = 2 * bytes_per_launch
    dom_tuning = tuning["forward" if dom_name == "hygt_batch_forward" else "inverse"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(dom_name, w.name, dom_tuning),
                "kernel": dom_name, "peak_source": peak_kind,
                "bytes_per_launch": bytes_per_launch,
                "fwd_ms": f_avg, "inv_ms": i_avg, "schedule_ms": statistics.mean(build_ms),
                "step_frac": (step_bytes / (total_ms / K / 1000.0) / 1e9) / peak}

    # the same step repeated for about two seconds after the timed region, with
    # its own clock record (the timed region itself is short)
    sustained = sustained_leg(batch, d_s, d_x, d_y, d_xr, dev, stream, local, total_ms / K)

    # context: the direct (unbucketed) kernels on the same data
    direct = direct_path_ms(plan, d_x, d_s, d_y, d_xr, stream)
    del d_y, d_xr

    line = {
        "metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": total_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": w.name, "nblocks": count, "N": N, "rounds": w.rounds,
                   "sets": w.num_sets, "parallelism": "dp%d" % world,
                   "step": "bucket blocks by set, integer forward, integer inverse",
                   "launch_tuning": {d: {"warps_per_cta": v[0], "ctas_per_sm": v[1],
                                         "stage": v[2], "layout": v[3], "tuner_ms": v[4],
                                         "tail_64ths": v[5] if len(v) > 5 else 0}
                                     for d, v in tuning.items()},
                   "l2": "inputs larger than L2 (%.0f MB read + %.0f MB written per step "
                         "vs %d MB L2), no flush" % (count * 6 * N / 1e6, count * 6 * N / 1e6,
                                                     L2_BYTES >> 20),
                   "description": w.description},
        "roofline": roofline,
        "gpu_launches": 5 * K,
        "clocks": clock_info,
        "sustained": sustained,
        "direct_path": direct,
    }

    if not args.no_e2e:
        line["e2e"] = e2e_leg(plan, x_np, s_np, N, dev, stream, world)

    if not args.no_extras and rank == 0:
        line["dense_klt"] = dense_leg(w, data, d_x, d_s, dev, stream, steps=max(5, K // 4),
                                      hygt_step_ms=total_ms / K)
        line["mixed"] = mixed_leg(dev, stream, steps=max(10, K // 2))
        line["backward"] = backward_leg(dev, stream, steps=max(5, K // 4))
        line["small_4x4"] = small_leg(dev, stream, steps=max(20, K))
        line["coding_gain"] = coding_gain_leg(dev, stream)
        line["rounds_variants"] = rounds_leg(dev)
        line["secondary_8x8"] = secondary_leg(dev, stream)
        line["pmpt_64"] = pmpt_leg(dev, stream)
        del d_x, d_s
        torch.cuda.empty_cache()
        line["stress_16x16"] = stress_leg(dev, stream)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, data)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def sustained_leg(batch, d_s, d_x, d_y, d_xr, dev, stream, local, step_ms, seconds=2.0):
    import torch
    steps = max(20, int(seconds * 1000.0 / max(step_ms, 1e-3)))
    clocks = ClockSampler(gpu_smi_id(dev, local))
    clocks.start()
    time.sleep(0.3)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        batch.build(d_s)
        batch.forward(d_x, out=d_y)
        batch.inverse(d_y, out=d_xr)
    b.record(stream)
    torch.cuda.synchronize(dev)
    info = clocks.stop()
    ms = a.elapsed_time(b) / steps
    return {"steps": steps, "ms_per_step": ms, "seconds": ms * steps / 1000.0,
            "value": d_x.shape[0] / (ms / 1000.0), "unit": "blocks/s", "clocks": info}


def stress_leg(dev, stream, steps=4, name="hygt16x16_r3_s16", sample=65536):
    """The large-transform workload (16x16 blocks, N = 256, 3 rounds, 16 sets,
    16,777,216 blocks): integer forward + inverse through the bucketed path,
    the FP32 path, and the dense 256 x 256 matrix transform (tcgen05 BF16 and
    FP8 E4M3), each timed.  Deviations are reported on the first `sample`
    blocks against the FP32 HyGT output (the parity tests hold that path
    within 1e-5 of the FP64 oracle and measure every path against it)."""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, workloads
    w = workloads.get(name)
    d = w.generate()
    n, N = w.nblocks, w.N
    plan = hygt.Plan(w.log2n, w.rounds, d["angle_idx"], d["perms"])
    x = torch.from_numpy(d["x"]).to(dev)
    s = torch.from_numpy(d["sets"].view(np.int16)).to(dev)
    del d
    b = hygt.Batch(plan, n, device=dev)
    y = torch.empty((n, N), dtype=torch.int32, device=dev)
    xr = torch.empty_like(x)
    from paper_2505_21728_gb300 import autotune
    b.build(s)
    tuning = autotune.tune_batch(b, x, y, xr, reps=2, use_cache=False)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def int_step():
        ev[0].record(stream)
        b.build(s)
        ev[1].record(stream)
        b.forward(x, out=y)
        ev[2].record(stream)
        b.inverse(y, out=xr)
        ev[3].record(stream)

    int_step()
    torch.cuda.synchronize(dev)
    tb, tf, ti = [], [], []
    for _ in range(steps):
        int_step()
        torch.cuda.synchronize(dev)
        tb.append(ev[0].elapsed_time(ev[1]))
        tf.append(ev[1].elapsed_time(ev[2]))
        ti.append(ev[2].elapsed_time(ev[3]))
    f_ms, i_ms, b_ms = statistics.mean(tf), statistics.mean(ti), statistics.mean(tb)
    peak, kind = measured_peaks()
    bpl = n * (6 * N + 2)
    dom_ms = max(f_ms, i_ms)
    out = {"workload": w.name, "description": w.description, "nblocks": n,
           "int32": {"fwd_ms": f_ms, "inv_ms": i_ms, "schedule_ms": b_ms,
                     "launch_tuning": {d: list(v) for d, v in tuning.items()},
                     "value": n / ((f_ms + i_ms + b_ms) / 1000.0), "unit": "blocks/s",
                     "roofline": {"bound": "hbm", "achieved": bpl / (dom_ms / 1000.0) / 1e9,
                                  "peak": peak, "unit": "GB/s",
                                  "frac": bpl / (dom_ms / 1000.0) / 1e9 / peak,
                                  "peak_source": kind, "bytes_per_launch": bpl,
                                  "kernel": "hygt_batch_kernel<8,*>"}}}
    yi_sample = y[:sample].to(torch.float64)
    del y, xr
    torch.cuda.empty_cache()

    # FP32 path (float32 in and out) through the same set-bucketed schedule
    xf = x.to(torch.float32)
    yf = torch.empty_like(xf)
    xrf = torch.empty_like(xf)
    b.forward_f32(xf, out=yf)
    b.inverse_f32(yf, out=xrf)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    b.forward_f32(xf, out=yf)
    ev[1].record(stream)
    b.inverse_f32(yf, out=xrf)
    ev[2].record(stream)
    torch.cuda.synchronize(dev)
    ff, fi = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    ref = yf[:sample].to(torch.float64)
    scale = float(ref.abs().max())
    out["fp32"] = {"fwd_ms": ff, "inv_ms": fi, "value": n / ((ff + fi) / 1000.0),
                   "unit": "blocks/s",
                   "roofline": {"bound": "hbm", "achieved": 8 * N * n / (ff / 1000.0) / 1e9,
                                "peak": peak, "unit": "GB/s",
                                "frac": 8 * N * n / (ff / 1000.0) / 1e9 / peak,
                                "peak_source": kind, "kernel": "hygt_f32b_kernel<8,*>"}}
    out["int32"]["max_abs_dev_vs_fp32_hygt"] = float((yi_sample - ref).abs().max())
    del xf, yf, xrf
    torch.cuda.empty_cache()

    # dense 256 x 256 matrix transform of the same blocks (the HyGT's own matrices)
    dk = hygt.DenseKLT(w.log2n, plan.dense_matrices()).build(s, n)
    yd = torch.empty((n, N), dtype=torch.float32, device=dev)
    for nm, kd in (("dense_bf16_tcgen05", hygt.DENSE_KLT_BF16),
                   ("dense_fp8_e4m3_tcgen05", hygt.DENSE_KLT_FP8)):
        dk.apply(x, kind=kd, out=yd)
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for _ in range(2):
            dk.apply(x, kind=kd, out=yd)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        ms = ev[0].elapsed_time(ev[1]) / 2
        gbs = n * (6 * N + 4) / (ms / 1000.0) / 1e9
        dev_max = float((yd[:sample].to(torch.float64) - ref).abs().max())
        out[nm] = {"ms_per_apply": ms, "blocks_per_s_one_direction": n / (ms / 1000.0),
                   "tflops": 2.0 * N * N * n / (ms / 1000.0) / 1e12,
                   "max_abs_dev_vs_fp32_hygt": dev_max, "rel_dev": dev_max / scale,
                   "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                "frac": gbs / peak, "peak_source": kind}}
    out["deviation_sample"] = ("first %d blocks, against the FP32 HyGT output (max |y| = %.1f)"
                               % (sample, scale))
    dk.close()
    plan.close()
    return out


def coding_gain_leg(dev, stream, restarts=3, iters=200):
    """The coding-gain angle fit of Sec. V on the correlated-patch workload:
    seeded restarts of Adam on J = 1/(2N) sum log2 v_i, every iteration in the
    library's kernels (forward, objective, diagonal backward, Adam)."""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import fit, workloads
    w = workloads.get_fit("hygt8x8_r4_fit")
    x_np = w.patches()
    f = fit.CodingGainFit(torch.from_numpy(x_np).to(dev), w.log2n, w.rounds)
    f.run(w.theta0(), 3)  # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    th, J, finals = f.fit(restarts, iters, lr=0.02, seed=0)
    secs = time.perf_counter() - t0
    # context: the KLT bound and the separable DCT-II of the same correlation
    x64 = x_np.astype(np.float64)
    phi = x64.T @ x64 / x64.shape[0]
    bound = float(np.sum(np.log2(np.linalg.eigvalsh(phi))) / (2 * w.N))
    k = np.arange(8)
    D = np.sqrt(2.0 / 8) * np.cos(np.pi * (2 * k[None, :] + 1) * k[:, None] / 16)
    D[0] /= np.sqrt(2.0)
    T = np.kron(D, D)
    J_dct = float(np.sum(np.log2(np.einsum("ia,ab,ib->i", T, phi, T))) / (2 * w.N))
    f.close()
    return {"workload": w.name, "nvec": w.nvec, "rounds": w.rounds,
            "restarts": restarts, "iterations": iters,
            "objective": "J = 1/(2N) sum log2 v_i (bits per coefficient, up to constants)",
            "J_best": J, "J_restarts": finals, "J_klt_bound": bound, "J_dct2": J_dct,
            "gap_to_klt_bits": J - bound, "gain_over_dct_bits": J_dct - J,
            "iterations_per_s": restarts * iters / secs,
            "ms_per_iteration": 1000.0 * secs / (restarts * iters)}


def _timed(fn, dev, stream, reps):
    import torch
    fn()
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / reps


def secondary_leg(dev, stream, reps=5):
    """The secondary-transform pipeline (Sec. VI) on 16 frames of 3840x2160
    tiled into 8x8 blocks: the fused kernel runs the integer DCT-II primary
    and the 8x8 HyGT (2 rounds, 105 sets, 10% of the blocks without a
    secondary transform) on the top-left coefficients, then the inverse."""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, inputs
    B, R, S = 16 * (3840 // 8) * (2160 // 8), 2, 105
    q = inputs.angle_indices(S, R, 6, seed=7)
    perms = inputs.permutations(S, R, 64, seed=7)
    plan = hygt.Plan(6, R, q, perms)
    x = torch.from_numpy(inputs.laplacian_blocks(B, 64, 8.0, -1024, 1023, seed=7)).to(dev)
    s = torch.from_numpy(inputs.set_indices(B, S, seed=7, skip_frac=0.1).view(np.int16)).to(dev)
    y = torch.empty((B, 64), dtype=torch.int32, device=dev)
    xr = torch.empty_like(x)
    # the bucketed kernels with the primary fused (one step: schedule,
    # forward, inverse), the launch tuning's staging choice timed
    b = hygt.Batch(plan, B, device=dev)
    b_ms = _timed(lambda: b.build(s), dev, stream, reps)
    best = None
    for stage in (0, 1):
        for inv in (0, 1):
            hygt._check(hygt.hygt_batch_set_tuning(plan.handle, inv, 0, 0, stage), "tuning")
        f = _timed(lambda: b.secondary_forward(x, 3, out=y), dev, stream, reps)
        i = _timed(lambda: b.secondary_inverse(y, 3, out=xr), dev, stream, reps)
        if best is None or f + i < best[0] + best[1]:
            best = (f, i, stage)
    f_ms, i_ms, stage = best
    # context: the generic kernel (any block size, no schedule)
    gf_ms = _timed(lambda: plan.secondary_forward(x, 3, s, out=y), dev, stream, reps)
    gi_ms = _timed(lambda: plan.secondary_inverse(y, 3, s, out=xr), dev, stream, reps)
    peak, kind = measured_peaks()
    bpl = B * (6 * 64 + 2)
    dom = max(f_ms, i_ms)
    plan.close()
    return {"workload": "16 frames of 3840x2160 in 8x8 blocks (%d blocks), 8x8 HyGT secondary, "
                        "2 rounds, 105 sets, 10%% primary only" % B,
            "fwd_ms": f_ms, "inv_ms": i_ms, "schedule_ms": b_ms, "stage": stage,
            "value": B / ((f_ms + i_ms + b_ms) / 1000.0), "unit": "blocks/s",
            "generic_kernel": {"fwd_ms": gf_ms, "inv_ms": gi_ms},
            "roofline": {"bound": "hbm", "achieved": bpl / (dom / 1000.0) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bpl / (dom / 1000.0) / 1e9 / peak,
                         "peak_source": kind,
                         "kernel": "hygt_batch_kernel<6, *, *, true> (DCT-II primary fused)"}}


def pmpt_leg(dev, stream, reps=5, B=1 << 22):
    """The general PMPT with explicit pair covers (random perfect matchings,
    12 passes of N = 64: as many rotations as a 2-round 8x8 HyGT) on the
    benchmark's block count, 105 sets: its time, and its parameter memory
    against the HyGT's (indices stored: 3 bytes per rotation, not 1)."""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, inputs
    N, P, S = 64, 12, 105
    rng = np.random.default_rng(9)
    m = np.empty((S, P, N // 2), np.uint16)
    n = np.empty((S, P, N // 2), np.uint16)
    for a in range(S):
        for k in range(P):
            perm = rng.permutation(N)
            m[a, k], n[a, k] = perm[0::2], perm[1::2]
    q = rng.integers(0, 256, (S, P, N // 2)).astype(np.uint8)
    pm = hygt.PMPT(N, P, m, n, angle_idx=q)
    x = torch.from_numpy(inputs.laplacian_blocks(B, N, 8.0, -1024, 1023, seed=9)).to(dev)
    s = torch.from_numpy(inputs.set_indices(B, S, seed=9).view(np.int16)).to(dev)
    y = pm.forward(x, s)
    f_ms = _timed(lambda: pm.forward(x, s), dev, stream, reps)
    i_ms = _timed(lambda: pm.inverse(y, s), dev, stream, reps)
    peak, kind = measured_peaks()
    bpl = B * (6 * N + 2)
    dom = max(f_ms, i_ms)
    pm.close()
    return {"workload": "%d blocks, N = 64, 12 passes, 105 sets, random pair covers" % B,
            "fwd_ms": f_ms, "inv_ms": i_ms, "value": B / ((f_ms + i_ms) / 1000.0),
            "unit": "blocks/s",
            "param_bytes_per_set": hygt.hygt_pmpt_param_bytes(N, P, 1),
            "hygt_param_bytes_per_set": hygt.hygt_param_bytes(6, 2, 1),
            "roofline": {"bound": "hbm", "achieved": bpl / (dom / 1000.0) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bpl / (dom / 1000.0) / 1e9 / peak,
                         "peak_source": kind, "kernel": "hygt_pmpt_kernel"}}


def rounds_leg(dev, nvec=1 << 18):
    """HyGT variants H(R) fitted with the Sec. V objective on correlated 4x4
    and 8x8 patches (Table II's H(2), H(3) for 4x4 and H(3), H(4), H(5) for
    8x8), each quantised to one byte per angle: J at the FP32 and at the
    8-bit angles against the KLT bound, and the KLT/HyGT memory ratio."""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import fit, inputs
    out = []
    t0 = time.perf_counter()
    for log2n, rl in ((4, (2, 3)), (6, (3, 4, 5))):
        N = 1 << log2n
        x = inputs.ar1_patches(nvec, int(round(N ** 0.5)), seed=3)
        x64 = x.astype(np.float64)
        phi = x64.T @ x64 / nvec
        bound = float(np.sum(np.log2(np.linalg.eigvalsh(phi))) / (2 * N))
        for r in fit.rounds_ladder(torch.from_numpy(x).to(dev), log2n, rl, iters=200,
                                   restarts=2, seed=1):
            out.append({"block": "%dx%d" % (int(N ** 0.5), int(N ** 0.5)), "rounds": r["rounds"],
                        "J": r["J"], "J_8bit": r["J_q"], "J_klt": bound,
                        "gap_bits": r["J"] - bound, "gap_bits_8bit": r["J_q"] - bound,
                        "param_bytes": r["param_bytes"], "klt_bytes": N * N,
                        "memory_ratio": N * N / r["param_bytes"]})
    return {"patches_per_class": nvec, "variants": out,
            "seconds": time.perf_counter() - t0,
            "objective": "J = 1/(2N) sum log2 v_i (bits per coefficient, up to constants)"}


def mixed_leg(dev, stream, steps=20, name="mixed_frame_2160p16"):
    """The mixed-size frame batch (4x4 / 8x8 / 16x16 blocks, one persistent
    launch per direction) as a CUDA graph of one step: schedules of the three
    classes, mixed forward, mixed inverse.  The mode (one launch with every
    CTA through the classes in turn, one launch with the classes concurrent
    on a split of the CTAs, or one launch per class) is autotuned."""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import autotune, hygt, workloads
    w = workloads.get_mixed(name)
    classes = []
    for cw in w.classes():
        d = cw.generate()
        plan = hygt.Plan(cw.log2n, cw.rounds, d["angle_idx"], d["perms"])
        classes.append((plan, torch.from_numpy(d["x"]).to(dev),
                        torch.from_numpy(d["sets"].view(np.int16)).to(dev)))
    mb = hygt.MixedBatch(classes, device=dev)
    mb.build()
    tunings = autotune.tune_mixed_classes(mb, reps=3, use_cache=False)
    modes = {}
    split = autotune.tune_split(mb, reps=3, use_cache=False, report=modes)
    variants = mb.variants()
    graph = mb.graph()
    for _ in range(3):
        graph.launch()
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        graph.launch()
    b.record(stream)
    torch.cuda.synchronize(dev)
    step_ms = a.elapsed_time(b) / steps
    # the two mixed kernels alone (schedules already built)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    f_ms, i_ms = [], []
    for _ in range(steps):
        ev[0].record(stream)
        mb.forward()
        ev[1].record(stream)
        mb.inverse()
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        f_ms.append(ev[0].elapsed_time(ev[1]))
        i_ms.append(ev[1].elapsed_time(ev[2]))
    nblocks = w.nblocks
    bytes_per_launch = w.bytes_fwd_inv() // 2
    f_avg, i_avg = statistics.mean(f_ms), statistics.mean(i_ms)
    dom_name, dom_ms = (("hygt_mixed_forward", f_avg) if f_avg >= i_avg
                        else ("hygt_mixed_inverse", i_avg))
    peak, kind = measured_peaks()
    achieved = bytes_per_launch / (dom_ms / 1000.0) / 1e9
    graph.close()
    return {"workload": w.name, "description": w.description, "nblocks": nblocks,
            "blocks_per_class": list(w.counts()), "value": nblocks / (step_ms / 1000.0),
            "unit": "blocks/s", "ms_per_step": step_ms,
            "step": "CUDA graph: schedules of 3 classes, mixed forward, mixed inverse",
            "mode": ("separate launches" if all(c == -1 for c in split) else
                     "concurrent" if all(c > 0 for c in split) else "sequential"),
            "cta_split": split,
            "modes_ms_fwd_inv": modes,
            "single_launch_variants": {str(e["plan"].N): {"forward": {"stage": v[0][0],
                                                                      "layout": v[0][1]},
                                                          "inverse": {"stage": v[1][0],
                                                                      "layout": v[1][1]}}
                                       for e, v in zip(mb.entries, variants)},
            "class_launch_tuning": {str(n): {d: {"warps_per_cta": v[0], "ctas_per_sm": v[1],
                                                 "stage": v[2], "layout": v[3],
                                                 "tuner_ms": v[4],
                                                 "tail_64ths": v[5] if len(v) > 5 else 0}
                                             for d, v in t.items()}
                                    for n, t in tunings.items()},
            "gpu_launches_per_step": 3 * 3 + (6 if all(c == -1 for c in split) else 2),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "kernel": dom_name, "peak_source": kind,
                         "bytes_per_launch": bytes_per_launch, "fwd_ms": f_avg, "inv_ms": i_avg,
                         "traffic": ncu_traffic(dom_name, w.name),
                         "step_frac": (2 * bytes_per_launch / (step_ms / 1000.0) / 1e9) / peak}}


def dense_leg(w, data, d_x, d_s, dev, stream, steps, hygt_step_ms):
    """The dense matrix transform of the same blocks and sets (one N x N
    matrix per set, the HyGT's own matrices): tcgen05 BF16 and FP8 (E4M3,
    per-block scales) and int32 CUDA-core kernels, one direction; the HyGT
    step is forward + inverse."""
    import torch
    from paper_2505_21728_gb300 import hygt
    K = hygt.Plan(w.log2n, w.rounds, data["angle_idx"], data["perms"]).dense_matrices()
    d = hygt.DenseKLT(w.log2n, K)
    nb = d_x.shape[0]
    N = w.N
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for _ in range(steps):
            fn()
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        return ev[0].elapsed_time(ev[1]) / steps

    build_ms = timed(lambda: d.build(d_s, nb))
    y = torch.empty((nb, N), dtype=torch.float32, device=dev)
    yi = torch.empty((nb, N), dtype=torch.int32, device=dev)
    out = {"matrices": "the HyGT's own %dx%d matrices, %d sets" % (N, N, w.num_sets),
           "schedule_ms": build_ms}
    peak, kind = measured_peaks()
    bytes_per_block = 2 * N + 4 * N + 4  # int16 in, 32-bit out, slot id
    for name, kd, buf in (("bf16_tcgen05", hygt.DENSE_KLT_BF16, y),
                          ("fp8_e4m3_tcgen05", hygt.DENSE_KLT_FP8, y),
                          ("int32_cuda_core", hygt.DENSE_KLT_INT, yi)):
        if (kd != hygt.DENSE_KLT_INT and N < 64) or (kd == hygt.DENSE_KLT_INT and N > 64):
            continue
        ms = timed(lambda: d.apply(d_x, kind=kd, out=buf))
        gbs = nb * bytes_per_block / (ms / 1000.0) / 1e9
        out[name] = {"ms_per_apply": ms, "blocks_per_s_one_direction": nb / (ms / 1000.0),
                     "blocks_per_s_fwd_inv": nb / ((2 * (ms + build_ms / 2)) / 1000.0),
                     "tflops": 2.0 * N * N * nb / (ms / 1000.0) / 1e12,
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                  "frac": gbs / peak, "peak_source": kind}}
    out["hygt_fwd_inv_step_ms"] = hygt_step_ms
    d.close()
    return out


def small_leg(dev, stream, steps, name="hygt4x4_r2"):
    """The 4x4 / one-set / 65,536-block case: 6.4 MB per direction, so it
    runs from L2 and is reported as such (launch- and L2-bound, not HBM)."""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, workloads
    w = workloads.get(name)
    d = w.generate()
    plan = hygt.Plan(w.log2n, w.rounds, d["angle_idx"], d["perms"])
    x = torch.from_numpy(d["x"]).to(dev)
    s = torch.from_numpy(d["sets"].view(np.int16)).to(dev)
    b = hygt.Batch(plan, w.nblocks, device=dev)
    y = torch.empty((w.nblocks, w.N), dtype=torch.int32, device=dev)
    xr = torch.empty_like(x)

    def step():
        b.build(s)
        b.forward(x, out=y)
        b.inverse(y, out=xr)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(steps):
        step()
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    ms = ev[0].elapsed_time(ev[1]) / steps
    return {"workload": w.name, "description": w.description, "nblocks": w.nblocks,
            "ms_per_step": ms, "value": w.nblocks / (ms / 1000.0), "unit": "blocks/s",
            "step": "bucket + forward + inverse (5 launches)",
            "note": "inputs and outputs (12.8 MB per step) stay in the 129 MB L2: L2/launch-bound, "
                    "not an HBM roofline case"}


def backward_leg(dev, stream, steps, name="hygt8x8_r4_fit"):
    """The differentiable FP32 path on the fitting workload: forward, the
    energy-compaction loss gradient, and the recomputing backward."""
    import torch
    from paper_2505_21728_gb300 import hygt, workloads
    w = workloads.get_fit(name)
    x = torch.from_numpy(w.patches()).to(dev)
    theta = w.theta0().astype("float32")
    plan = hygt.Plan.from_theta(w.log2n, w.rounds, theta)
    mask = torch.zeros(w.N, device=dev)
    mask[w.keep:] = 2.0 / w.nvec
    y = plan.forward_f32(x)
    gy = y * mask
    plan.backward_f32(y, gy)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    f_ms, b_ms = [], []
    for _ in range(steps):
        ev[0].record(stream)
        y = plan.forward_f32(x, out=y)
        ev[1].record(stream)
        gy = y * mask
        e2 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        plan.backward_f32(y, gy)
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        f_ms.append(ev[0].elapsed_time(ev[1]))
        b_ms.append(e2.elapsed_time(ev[2]))
    fm, bm = statistics.mean(f_ms), statistics.mean(b_ms)
    pairs = w.rounds * w.log2n * (w.N // 2)
    flops = 15.0 * pairs * w.nvec  # inverse rotation 6, gradient rotation 6, angle term 3
    sm_mhz = 2070.0
    try:
        sm_mhz = float(torch.cuda.get_device_properties(dev).clock_rate) / 1000.0 or sm_mhz
    except Exception:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12  # FFMA lanes x 2 FLOP x clock
    peak, kind = measured_peaks()
    gbs = 3 * 4 * w.N * w.nvec / (bm / 1000.0) / 1e9
    plan.close()
    return {"workload": w.name, "description": w.description, "nvec": w.nvec,
            "forward_ms": fm, "backward_ms": bm,
            "vectors_per_s_fwd_bwd": w.nvec / ((fm + bm) / 1000.0),
            "roofline": {"bound": "alu", "achieved": flops / (bm / 1000.0) / 1e12,
                         "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": flops / (bm / 1000.0) / 1e12 / fp32_peak,
                         "peak_source": "FP32 FMA lanes x clock (%d SMs x 128 x 2 x %.0f MHz)"
                                        % (sms, sm_mhz),
                         "kernel": "hygt_grad_kernel", "hbm_gbs": gbs, "hbm_frac": gbs / peak}}


def direct_path_ms(plan, d_x, d_s, d_y, d_xr, stream, steps=5):
    """Forward and inverse through the unbucketed kernels (hygt_forward /
    hygt_inverse), for context."""
    import torch
    plan.forward(d_x, d_s, out=d_y)
    plan.inverse(d_y, d_s, out=d_xr)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fw, iv = [], []
    for _ in range(steps):
        ev[0].record(stream)
        plan.forward(d_x, d_s, out=d_y)
        ev[1].record(stream)
        plan.inverse(d_y, d_s, out=d_xr)
        ev[2].record(stream)
        torch.cuda.synchronize()
        fw.append(ev[0].elapsed_time(ev[1]))
        iv.append(ev[1].elapsed_time(ev[2]))
    return {"fwd_ms": statistics.mean(fw), "inv_ms": statistics.mean(iv)}


def e2e_leg(plan, x_np, s_np, N, dev, stream, world, steps=10):
    """Same metric through the public API with host buffers: every step is
    one hygt_host_roundtrip call (HostPipe.roundtrip) on pinned host tensors
    -- the blocks and set indices go host->device, are bucketed, transformed
    forward and back, and the step's result (the reconstructed blocks) comes
    back to host memory, in chunks whose copies overlap the kernels.  The
    same with the coefficients returned as well is reported beside it."""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt
    count = x_np.shape[0]
    h_x = torch.from_numpy(x_np).pin_memory()
    h_s = torch.from_numpy(s_np.view(np.int16)).pin_memory()
    h_y = torch.empty((count, N), dtype=torch.int32).pin_memory()
    h_xr = torch.empty((count, N), dtype=torch.int16).pin_memory()
    pipe = hygt.HostPipe(plan, 1 << 17)

    def run(coefficients):
        def step():
            _, _, status = pipe.roundtrip(h_x, h_s, h_y if coefficients else None, h_xr,
                                          coefficients=coefficients)
            if status:
                raise RuntimeError("device status %d" % status)
        step()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        ms = (time.perf_counter() - t0) * 1000.0
        return max_over_ranks(ms, world, dev)

    ms = run(False)
    ms_coef = run(True)
    pipe.close()
    return {"value": count * world * steps / (ms / 1000.0), "unit": "blocks/s",
            "h2d_bytes_per_step": count * (2 * N + 2), "d2h_bytes_per_step": count * 2 * N,
            "steps": steps, "api": "hygt_host_roundtrip (HostPipe), pinned host buffers, "
                                  "chunks of 131,072 blocks on three streams; the step's "
                                  "result (the reconstruction) read back",
            "with_coefficients": {"value": count * world * steps / (ms_coef / 1000.0),
                                  "unit": "blocks/s", "d2h_bytes_per_step": count * 6 * N,
                                  "note": "int32 coefficients read back as well"},
            "host_link": "measured on this box: 193 GB/s device to host, 211 GB/s host to "
                         "device, 171 GB/s each way when both run (copy engines or SM "
                         "stores alike)"}


# ---------------------------------------------------------------- kernel cases (ncu)
def _int_case_data(name, nblocks):
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, workloads
    w = workloads.get(name)
    if nblocks:
        w = workloads.truncated(w, nblocks)
    d = w.generate()
    plan = hygt.Plan(w.log2n, w.rounds, d["angle_idx"], d["perms"])
    x = torch.from_numpy(d["x"]).cuda()
    s = torch.from_numpy(d["sets"].view(np.int16)).cuda()
    return w, d, plan, x, s


def case_batch(args, name=None):
    """bucket + integer forward + integer inverse (8x8 blocks, 105 sets, or
    --workload: a named workload or a class of a mixed batch)"""
    import torch
    name = name or args.workload
    from paper_2505_21728_gb300 import hygt
    w, d, plan, x, s = _int_case_data(name, args.nblocks)
    for inv, t in ((0, args.fwd_tuning), (1, args.inv_tuning)):
        if t:
            vals = [int(v) for v in t.split(",")]
            hygt._check(hygt.hygt_batch_set_tuning(plan.handle, inv, *vals[:4]),
                        "hygt_batch_set_tuning")
            if len(vals) > 4:
                hygt._check(hygt.hygt_batch_set_tail(plan.handle, inv, vals[4]),
                            "hygt_batch_set_tail")
    b = hygt.Batch(plan, x.shape[0])
    y = torch.empty((x.shape[0], w.N), dtype=torch.int32, device="cuda")
    xr = torch.empty_like(x)

    def run():
        b.build(s)
        b.forward(x, out=y)
        b.inverse(y, out=xr)
    return run


def case_stress(args):
    """the same on the 16x16 / 3-round / 16-set workload"""
    return case_batch(args, name="hygt16x16_r3_s16")


def case_direct(args):
    """direct integer forward + inverse (no bucketing), 8x8 workload"""
    import torch
    w, d, plan, x, s = _int_case_data(DEFAULT_WORKLOAD, args.nblocks)
    y = torch.empty((x.shape[0], w.N), dtype=torch.int32, device="cuda")
    xr = torch.empty_like(x)

    def run():
        plan.forward(x, s, out=y)
        plan.inverse(y, s, out=xr)
    return run


def case_mixed(args):
    """mixed 4x4 / 8x8 / 16x16 frame batch, mixed forward + inverse"""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import autotune, hygt, workloads
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
    """dense matrix transform (tcgen05 BF16, FP8, int32) of the 8x8 blocks"""
    import torch
    from paper_2505_21728_gb300 import hygt
    w, d, plan, x, s = _int_case_data(DEFAULT_WORKLOAD, args.nblocks)
    dk = hygt.DenseKLT(w.log2n, plan.dense_matrices()).build(s, x.shape[0])
    y = torch.empty((x.shape[0], w.N), dtype=torch.float32, device="cuda")
    yi = torch.empty((x.shape[0], w.N), dtype=torch.int32, device="cuda")

    def run():
        dk.apply(x, kind=hygt.DENSE_KLT_BF16, out=y)
        dk.apply(x, kind=hygt.DENSE_KLT_FP8, out=y)
        dk.apply(x, kind=hygt.DENSE_KLT_INT, out=yi)
    return run


def case_grad(args):
    """FP32 forward + backward, 8x8 patches, 4 rounds (fitting workload)"""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, workloads
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


def case_coding_gain(args):
    """one iteration of the coding-gain angle fit (forward, objective, diagonal
    backward, Adam), 8x8 patches, 4 rounds"""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import fit, workloads
    w = workloads.get_fit("hygt8x8_r4_fit")
    n = args.nblocks or w.nvec
    f = fit.CodingGainFit(torch.from_numpy(w.patches(n)).cuda(), w.log2n, w.rounds)
    th0 = w.theta0().astype(np.float32)

    def run():
        f.run(th0, 1)
    return run


def case_stress_f32(args):
    """bucket + FP32 forward + FP32 inverse (set-bucketed kernels), 16x16 workload"""
    import torch
    from paper_2505_21728_gb300 import hygt
    w, d, plan, x, s = _int_case_data("hygt16x16_r3_s16", args.nblocks)
    xf = x.float()
    b = hygt.Batch(plan, x.shape[0])
    y = torch.empty_like(xf)
    xr = torch.empty_like(xf)

    def run():
        b.build(s)
        b.forward_f32(xf, out=y)
        b.inverse_f32(y, out=xr)
    return run


def case_secondary_batch(args):
    """secondary pipeline of 8x8 blocks through the bucketed kernels with the
    primary fused: schedule, forward, inverse"""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, inputs
    B = args.nblocks or 2073600
    q = inputs.angle_indices(105, 2, 6, seed=7)
    plan = hygt.Plan(6, 2, q, inputs.permutations(105, 2, 64, seed=7))
    x = torch.from_numpy(inputs.laplacian_blocks(B, 64, 8.0, -1024, 1023, seed=7)).cuda()
    s = torch.from_numpy(inputs.set_indices(B, 105, seed=7, skip_frac=0.1).view(np.int16)).cuda()
    b = hygt.Batch(plan, B)
    y = torch.empty((B, 64), dtype=torch.int32, device="cuda")
    xr = torch.empty_like(x)

    def run():
        b.build(s)
        b.secondary_forward(x, 3, out=y)
        b.secondary_inverse(y, 3, out=xr)
    return run


def case_secondary(args):
    """fused DCT-II primary + 8x8 HyGT secondary, forward + inverse, 8x8 blocks"""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, inputs
    B = args.nblocks or 2073600
    q = inputs.angle_indices(105, 2, 6, seed=7)
    plan = hygt.Plan(6, 2, q, inputs.permutations(105, 2, 64, seed=7))
    x = torch.from_numpy(inputs.laplacian_blocks(B, 64, 8.0, -1024, 1023, seed=7)).cuda()
    s = torch.from_numpy(inputs.set_indices(B, 105, seed=7, skip_frac=0.1).view(np.int16)).cuda()
    y = torch.empty((B, 64), dtype=torch.int32, device="cuda")
    xr = torch.empty_like(x)

    def run():
        plan.secondary_forward(x, 3, s, out=y)
        plan.secondary_inverse(y, 3, s, out=xr)
    return run


def case_pmpt(args):
    """general PMPT (random pair covers), N = 64, 12 passes, forward + inverse"""
    import numpy as np
    import torch
    from paper_2505_21728_gb300 import hygt, inputs
    B, N, P, S = args.nblocks or (1 << 22), 64, 12, 105
    rng = np.random.default_rng(9)
    perm = np.stack([[rng.permutation(N) for _ in range(P)] for _ in range(S)])
    q = rng.integers(0, 256, (S, P, N // 2)).astype(np.uint8)
    pm = hygt.PMPT(N, P, perm[:, :, 0::2], perm[:, :, 1::2], angle_idx=q)
    x = torch.from_numpy(inputs.laplacian_blocks(B, N, 8.0, -1024, 1023, seed=9)).cuda()
    s = torch.from_numpy(inputs.set_indices(B, S, seed=9).view(np.int16)).cuda()

    def run():
        pm.inverse(pm.forward(x, s), s)
    return run


CASES = {"batch": case_batch, "stress": case_stress, "direct": case_direct,
         "mixed": case_mixed, "dense": case_dense, "grad": case_grad,
         "coding_gain": case_coding_gain, "stress_f32": case_stress_f32,
         "secondary": case_secondary, "secondary_batch": case_secondary_batch,
         "pmpt": case_pmpt}


def run_case(args):
    import torch
    from paper_2505_21728_gb300 import build
    build.build()
    torch.cuda.set_device(0)
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


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
