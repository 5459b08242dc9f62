"""Autotuners: the launch tuning of the bucketed kernels (blocks per CTA,
CTAs per SM, staging depth, register layout; ``tune_batch``) and the mode
of the mixed-size launch (``tune_split``).

Mixed launch.

A mixed batch runs in one of three modes: one launch in which every CTA
works through all classes in turn (split of all zeros); one launch in which
each class runs concurrently on its own share of the CTAs (so the launch
ends when the slowest class ends); or one batch launch per class (split of
all -1).  The tuner times them:

0. the sequential launch and the separate launches;
1. each class alone on all CTAs (t_c);
2. the concurrent split proportional to t_c (equal finishing times if each
   class scales linearly with its CTAs);
3. local search: move k CTAs between any two classes (k halving down to 1)
   while the measured forward + inverse time improves;

and keeps the fastest.

Results are cached in a JSON file keyed by the GPU name and the classes'
shapes (block size, rounds, sets, block count).
"""
from __future__ import annotations

import ctypes
import json
import os
import statistics

from . import hygt


def _cache_path():
    return os.environ.get("HYGT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hygt_autotune.json"))


def _key(mb):
    import torch
    dev = torch.cuda.get_device_name()
    shapes = []
    for e in mb.entries:
        p = e["plan"]
        shapes.append("N%d_R%d_S%d_B%d" % (p.N, p.rounds, p.num_sets, int(e["x"].shape[0])))
    return dev + "|" + ",".join(shapes)


def _time_pair(classes, n, reps):
    """Median time (ms) of one mixed forward + one mixed inverse launch."""
    import torch
    stream = torch.cuda.current_stream()
    h = stream.cuda_stream
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    hygt._check(hygt.hygt_forward_mixed(classes, n, h, None), "hygt_forward_mixed")
    hygt._check(hygt.hygt_inverse_mixed(classes, n, h, None), "hygt_inverse_mixed")
    times = []
    for _ in range(reps):
        a.record(stream)
        hygt._check(hygt.hygt_forward_mixed(classes, n, h, None), "hygt_forward_mixed")
        hygt._check(hygt.hygt_inverse_mixed(classes, n, h, None), "hygt_inverse_mixed")
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def _with_split(mb, split):
    arr = (hygt.MixedClass * mb.n)()
    for i in range(mb.n):
        arr[i] = mb.classes[i]
        arr[i].ctas = int(split[i])
    return arr


def tune_split(mb, reps=5, use_cache=True, verbose=False, report=None):
    """Returns the tuned CTA split (list, one entry per class) and applies it
    to ``mb``.  ``mb`` must have its schedules built.  A dict given as
    ``report`` receives the timings of the modes (ms per forward + inverse)
    when they were measured in this call."""
    key = _key(mb)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        split = cache[key]["split"]
        mb.set_split(split)
        return split

    G = hygt.hygt_mixed_ctas()
    active = [i for i in range(mb.n) if mb.classes[i].nblocks > 0]
    if len(active) <= 1 or G < len(active):
        split = [G if i in active else 0 for i in range(mb.n)]
        mb.set_split(split)
        return split

    # 0. sequential launch, separate launches
    seq = [0] * mb.n
    seq_ms = _time_pair(_with_split(mb, seq), mb.n, reps)
    sep = [-1] * mb.n
    sep_ms = _time_pair(_with_split(mb, sep), mb.n, reps)
    # 1. each class alone on all CTAs
    alone = {}
    for i in active:
        one = (hygt.MixedClass * 1)()
        one[0] = mb.classes[i]
        one[0].ctas = G
        alone[i] = _time_pair(one, 1, reps)
    # 2. proportional split
    tot = sum(alone.values())
    split = [0] * mb.n
    for i in active:
        split[i] = max(1, int(round(G * alone[i] / tot)))
    big = max(active, key=lambda i: alone[i])
    split[big] += G - sum(split)
    best = _time_pair(_with_split(mb, split), mb.n, reps)
    trials = [(list(split), best)]
    # 3. local search
    step = max(1, G // 16)
    while step >= 1:
        improved = True
        while improved:
            improved = False
            for a in active:
                for b in active:
                    if a == b or split[a] - step < 1:
                        continue
                    cand = list(split)
                    cand[a] -= step
                    cand[b] += step
                    t = _time_pair(_with_split(mb, cand), mb.n, reps)
                    trials.append((cand, t))
                    if t < best * 0.995:
                        best, split, improved = t, cand, True
        step //= 2
    if seq_ms <= best:
        split, best = seq, seq_ms
    if sep_ms <= best:
        split, best = sep, sep_ms
    if verbose:
        print("autotune: sequential %.4f ms, separate %.4f ms, alone" % (seq_ms, sep_ms), alone,
              "best", split, "%.4f ms" % best)
    if report is not None:
        report.update({"sequential_ms": seq_ms, "separate_ms": sep_ms,
                       "best_concurrent_ms": min(t for _, t in trials), "chosen_ms": best})
    mb.set_split(split)
    if use_cache:
        cache[key] = {"split": split, "ms": best, "sequential_ms": seq_ms, "separate_ms": sep_ms,
                      "alone_ms": {str(k): v for k, v in alone.items()},
                      "trials": len(trials)}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return split


# ---------------------------------------------------------------- launch tuning
def batch_candidates(max_warps, log2n, layout=0):
    """(warps_per_cta, ctas_per_sm, stage, layout) points the batch tuner
    times for one register layout: blocks per CTA through the warps of a
    CTA, CTAs per SM, and the staging depth (0: none, 1: the next task's
    blocks copied into shared memory ahead, 2: prefetched into L2 ahead, 3:
    as 1 by one bulk copy per block; N >= 16 only; layouts other than 0
    without 3; 4: no staging, tasks interleaved across the sets so that the
    blocks of a 128-byte line are read together, for 4x4 blocks in layouts 0
    and 2, one CTA per SM when the set tables fill its shared memory)."""
    warps = sorted({w for w in (max_warps, (3 * max_warps) // 4, max_warps // 2,
                                max_warps // 3, 4) if w >= 2})
    if log2n < 4:
        stages = (-1,)
    else:
        stages = (0, 1, 2, 3) if layout == 0 else (0, 1, 2)
    if log2n == 4 and layout in (0, 2):
        stages += (4,)
    out = []
    for w in warps:
        for c in (0, 1, 2):
            for s in stages:
                out.append((w, c, s, layout))
    return out


BATCH_LAYOUTS = 6


def batch_layouts(plan, inverse):
    """Register layouts the plan supports for one direction (0 always; 1,
    one lane per block, for 4x4 and 8x8 blocks; 2, other values per lane and
    blocks per lane group, for 4x4, 8x8 and 16x16 blocks; 3, eight blocks per
    lane group in both directions, for 4x4 and 8x8 blocks; 4, the cross-lane
    passes replaced by register passes on the transposed block, for 4x4,
    8x8 and 16x16 blocks; 5, layout 4 with two blocks per lane group, for
    16x16 blocks)."""
    out = [0]
    for lay in range(1, BATCH_LAYOUTS):
        if hygt.hygt_batch_set_tuning(plan.handle, inverse, 0, 0, -1, lay) == hygt.HYGT_OK:
            out.append(lay)
    hygt._check(hygt.hygt_batch_set_tuning(plan.handle, inverse, 0, 0, -1, 0),
                "hygt_batch_set_tuning")
    return out


def all_batch_candidates(plan, inverse):
    """batch_candidates over every layout the plan supports."""
    out = []
    for lay in batch_layouts(plan, inverse):
        hygt._check(hygt.hygt_batch_set_tuning(plan.handle, inverse, 0, 0, -1, lay),
                    "hygt_batch_set_tuning")
        max_warps = hygt.hygt_batch_get_tuning(plan.handle, inverse)[4]
        out += batch_candidates(max_warps, plan.log2n, lay)
    hygt._check(hygt.hygt_batch_set_tuning(plan.handle, inverse, 0, 0, -1, 0),
                "hygt_batch_set_tuning")
    return out


def _time_dir(fn, reps):
    import torch
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


# Dynamic tails the batch tuner tries on its best point, in 64ths of the
# tasks (hygt_batch_set_tail); one is kept only if it is 1% faster.
BATCH_TAILS = (4, 8, 16)


def tune_batch(batch, x, y, xr, reps=5, use_cache=True, verbose=False, time_fn=None):
    """Times every launch tuning of ``all_batch_candidates`` for the
    bucketed forward and inverse of ``batch`` (a hygt.Batch with its schedule
    built), sets the fastest on the plan (hygt_batch_set_tuning), then tries
    the dynamic tails of BATCH_TAILS on it (hygt_batch_set_tail).  Returns
    {"forward": (warps, ctas_per_sm, stage, layout, ms, tail_64ths),
    "inverse": (...)}.  Results are cached by GPU name, block size, rounds,
    sets and block count.  ``time_fn(direction, point)`` replaces the GPU
    timing (tests); ``point`` is a tuning, with the tail as a fifth entry
    when one is timed."""
    plan = batch.plan
    key = None
    cache, path = {}, _cache_path()
    if use_cache:
        import torch
        key = "batch3|%s|N%d_R%d_S%d_B%d" % (torch.cuda.get_device_name(), plan.N, plan.rounds,
                                              plan.num_sets, batch.nblocks)
        if os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if key in cache:
            res = {d: tuple(v) for d, v in cache[key].items()}
            for inv, d in ((0, "forward"), (1, "inverse")):
                hygt._check(hygt.hygt_batch_set_tail(plan.handle, inv, 0), "hygt_batch_set_tail")
                hygt._check(hygt.hygt_batch_set_tuning(plan.handle, inv, *res[d][:4]),
                            "hygt_batch_set_tuning")
                hygt._check(hygt.hygt_batch_set_tail(plan.handle, inv, res[d][5]),
                            "hygt_batch_set_tail")
            return res
    res = {}
    for inv, d in ((0, "forward"), (1, "inverse")):
        fn = (lambda: batch.forward(x, out=y)) if inv == 0 else (lambda: batch.inverse(y, out=xr))

        def timed(point):
            if time_fn is not None:
                return time_fn(d, point)
            try:
                return _time_dir(fn, reps)
            except hygt.HygtError:
                return None  # this point does not fit (shared memory)

        hygt._check(hygt.hygt_batch_set_tail(plan.handle, inv, 0), "hygt_batch_set_tail")
        best = None
        for cand in all_batch_candidates(plan, inv):
            if hygt.hygt_batch_set_tuning(plan.handle, inv, *cand) != hygt.HYGT_OK:
                continue
            ms = timed(tuple(cand))
            if ms is None:
                continue
            if verbose:
                print("tune %s %s: %.4f ms" % (d, cand, ms))
            if best is None or ms < best[4]:
                best = tuple(cand[:4]) + (ms,)
        if best is None:
            best = (0, 0, -1, 0, float("nan"))
        hygt._check(hygt.hygt_batch_set_tuning(plan.handle, inv, *best[:4]),
                    "hygt_batch_set_tuning")
        tail, tail_ms = 0, best[4]
        for t in BATCH_TAILS:
            if hygt.hygt_batch_set_tail(plan.handle, inv, t) != hygt.HYGT_OK:
                break  # no dynamic tail for this point
            ms = timed(tuple(best[:4]) + (t,))
            if verbose and ms is not None:
                print("tune %s %s tail %d/64: %.4f ms" % (d, best[:4], t, ms))
            if ms is not None and ms < tail_ms and ms < best[4] * 0.99:
                tail, tail_ms = t, ms
        hygt._check(hygt.hygt_batch_set_tail(plan.handle, inv, tail), "hygt_batch_set_tail")
        res[d] = tuple(best[:4]) + (tail_ms, tail)
    if use_cache and key is not None:
        cache[key] = {d: list(v) for d, v in res.items()}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return res


def tune_mixed_classes(mb, reps=3, use_cache=True):
    """tune_batch for every class of a MixedBatch (schedules built): the
    per-class launches of its separate mode use these tunings.  Returns
    {N: result of tune_batch}."""
    out = {}
    for e in mb.entries:
        plan = e["plan"]
        b = hygt.Batch.on_workspace(plan, int(e["x"].shape[0]), e["work"])
        out[plan.N] = tune_batch(b, e["x"], e["y"], e["xr"], reps=reps, use_cache=use_cache)
    return out
