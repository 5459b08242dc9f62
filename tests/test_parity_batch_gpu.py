"""Parity of the set-bucketed batch path (hygt_batch_build + hygt_forward_batch /
hygt_inverse_batch) with the CPU oracle: bit-exact, including skip and
out-of-range set indices, ragged batch sizes and a stale schedule."""
import numpy as np
import pytest

from paper_2505_21728_gb300 import inputs

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_batch(gpu, log2n, rounds, q, perms, x, sets):
    import torch
    plan = gpu.Plan(log2n, rounds, q, perms)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    b = gpu.Batch(plan, x.shape[0]).build(None if sets is None else _t(sets))
    y = b.forward(_t(x), status=st)
    xr = b.inverse(y, status=st)
    return y.cpu().numpy(), xr.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("log2n", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("rounds,perm_kind", [(1, "none"), (2, "between"), (3, "all")])
def test_batch_parity(gpu, orc, log2n, rounds, perm_kind):
    N = 1 << log2n
    S, B = 9, 5003
    q = inputs.angle_indices(S, rounds, log2n, seed=log2n + 7 * rounds)
    perms = None if perm_kind == "none" else inputs.permutations(
        S, rounds, N, seed=3, between_rounds_only=(perm_kind == "between"))
    x = inputs.laplacian_blocks(B, N, 50.0, -32768, 32767, seed=log2n)
    sets = inputs.set_indices(B, S, seed=log2n, skip_frac=0.1)
    y, xr, st = run_batch(gpu, log2n, rounds, q, perms, x, sets)
    ye, _ = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert st == 0
    assert np.array_equal(y, ye)
    assert np.array_equal(xr, xe)


@pytest.mark.parametrize("log2n", [4, 6])
@pytest.mark.parametrize("B", [1, 31, 32, 33, 1000, 3 * 4096 + 77])
def test_batch_ragged_and_bad_sets(gpu, orc, log2n, B):
    rounds, S, N = 2, 105, 1 << log2n
    q = inputs.angle_indices(S, rounds, log2n, seed=2)
    perms = inputs.permutations(S, rounds, N, seed=2)
    x = inputs.laplacian_blocks(B, N, 8.0, -1024, 1023, seed=B)
    sets = inputs.set_indices(B, S, seed=B, skip_frac=0.1)
    if B > 20:
        sets[3] = 200
        sets[B - 1] = S
    y, xr, st = run_batch(gpu, log2n, rounds, q, perms, x, sets)
    ye, ste = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert st == (4 if B > 20 else 0) and ste == (orc.ERR_SET if B > 20 else 0)
    assert np.array_equal(y, ye) and np.array_equal(xr, xe)


def test_batch_no_sets_one_set(gpu, orc):
    log2n, rounds = 4, 2
    q = inputs.angle_indices(1, rounds, log2n, seed=0)
    perms = inputs.permutations(1, rounds, 16, seed=0)
    x = inputs.laplacian_blocks(4097, 16, 12.0, -512, 511, seed=0)
    y, xr, st = run_batch(gpu, log2n, rounds, q, perms, x, None)
    ye, _ = orc.fwd_int(x, q, log2n, rounds, perms)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms)
    assert st == 0 and np.array_equal(y, ye) and np.array_equal(xr, xe)


@pytest.mark.parametrize("S,rounds", [(200, 2), (105, 8), (128, 2)])
def test_batch_4x4_runs_of_sets(gpu, orc, S, rounds):
    """4x4 blocks with long runs: 4096 skip blocks, then 4096 blocks of one
    set, then uniform sets with one bad index; many sets (200) and large
    tables (8 rounds)."""
    log2n, N, B = 4, 16, 2 * 4096 + 4096 + 999
    q = inputs.angle_indices(S, rounds, log2n, seed=S + rounds)
    perms = inputs.permutations(S, rounds, N, seed=S)
    x = inputs.laplacian_blocks(B, N, 12.0, -512, 511, seed=S)
    sets = inputs.set_indices(B, S, seed=S, skip_frac=0.1)
    sets[:4096] = 0xFFFF                 # a run of skip blocks
    sets[4096:8192] = S - 1              # a run of one set
    sets[9000] = S + 5                   # a bad index
    y, xr, st = run_batch(gpu, log2n, rounds, q, perms, x, sets)
    ye, ste = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert st == 4 and ste == orc.ERR_SET
    assert np.array_equal(y, ye) and np.array_equal(xr, xe)


def test_batch_many_sets_uncached(gpu, orc):
    """Few blocks per set: a CTA's tasks span more sets than fit in shared
    memory, so the kernel reads the multipliers from global memory."""
    log2n, rounds, S = 8, 3, 600
    q = inputs.angle_indices(S, rounds, log2n, seed=9)
    perms = inputs.permutations(S, rounds, 256, seed=9)
    B = 3000
    x = inputs.laplacian_blocks(B, 256, 30.0, -2048, 2047, seed=9)
    sets = inputs.set_indices(B, S, seed=9)
    y, xr, st = run_batch(gpu, log2n, rounds, q, perms, x, sets)
    ye, _ = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert st == 0 and np.array_equal(y, ye) and np.array_equal(xr, xe)


def test_batch_max_rounds_extremes(gpu, orc):
    log2n, rounds, S = 8, 8, 3
    q = inputs.angle_indices(S, rounds, log2n, seed=5)
    perms = inputs.permutations(S, rounds, 256, seed=5, between_rounds_only=False)
    rng = np.random.default_rng(1)
    x = rng.choice(np.array([-32768, 32767], np.int16), size=(100, 256))
    sets = (np.arange(100) % S).astype(np.uint16)
    y, xr, st = run_batch(gpu, log2n, rounds, q, perms, x, sets)
    ye, ste = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    assert st == 0 and ste == 0 and np.array_equal(y, ye) and np.array_equal(xr, xe)


def test_batch_schedule_size_mismatch_reports(gpu):
    import torch
    q = inputs.angle_indices(3, 2, 6, seed=0)
    plan = gpu.Plan(6, 2, q)
    x = _t(inputs.laplacian_blocks(100, 64, 8.0, -1024, 1023, seed=0))
    sets = _t(inputs.set_indices(100, 3, seed=0))
    b = gpu.Batch(plan, 100).build(sets)
    # a schedule for 100 blocks used for 64 blocks: status ERR_ARG, output untouched
    b64 = gpu.Batch(plan, 64)
    b64.work.copy_(b.work[:b64.work.numel()])
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.full((64, 64), 7, dtype=torch.int32, device="cuda")
    b64.forward(x[:64], out=out, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == gpu.HYGT_ERR_ARG
    assert bool((out == 7).all())


def test_batch_workload_8x8_full(gpu, orc):
    """The benchmark's launch configuration on all 4,194,304 blocks."""
    from paper_2505_21728_gb300 import workloads
    w = workloads.get("hygt8x8_r2_s105")
    d = w.generate()
    y, xr, st = run_batch(gpu, w.log2n, w.rounds, d["angle_idx"], d["perms"], d["x"], d["sets"])
    ye, ste = orc.fwd_int(d["x"], d["angle_idx"], w.log2n, w.rounds, d["perms"], d["sets"])
    assert st == 0 and ste == 0
    assert np.array_equal(y, ye)
    del ye
    xe, _ = orc.inv_int(y, d["angle_idx"], w.log2n, w.rounds, d["perms"], d["sets"])
    assert np.array_equal(xr, xe)


def test_batch_workload_16x16_full(gpu, orc):
    """16x16 blocks (N=256), 3 rounds, 16 sets, all 16,777,216 blocks through
    the bucketed path, every block compared with the oracle bit for bit
    (forward and inverse), in chunks of 1,048,576 blocks."""
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get("hygt16x16_r3_s16")
    d = w.generate()
    n = w.nblocks
    plan = gpu.Plan(w.log2n, w.rounds, d["angle_idx"], d["perms"])
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    b = gpu.Batch(plan, n).build(_t(d["sets"]))
    y = b.forward(_t(d["x"]), status=st)
    xr = b.inverse(y, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    CH = 1 << 20
    for off in range(0, n, CH):
        sl = slice(off, min(n, off + CH))
        ye, ste = orc.fwd_int(d["x"][sl], d["angle_idx"], w.log2n, w.rounds, d["perms"],
                              d["sets"][sl])
        assert ste == 0
        assert np.array_equal(y[sl].cpu().numpy(), ye), off
        xe, _ = orc.inv_int(ye, d["angle_idx"], w.log2n, w.rounds, d["perms"], d["sets"][sl])
        assert np.array_equal(xr[sl].cpu().numpy(), xe), off


@pytest.mark.parametrize("log2n", [4, 5, 6, 7, 8])
@pytest.mark.parametrize("rounds,perm_kind", [(1, "none"), (2, "between"), (3, "all")])
def test_batch_f32_parity(gpu, orc, log2n, rounds, perm_kind):
    """The set-bucketed FP32 kernels against the FP64 oracle (max abs error
    <= 1e-5 of max |y|), with skip and bad set indices."""
    import torch
    N = 1 << log2n
    S, B = 9, 4003
    q = inputs.angle_indices(S, rounds, log2n, seed=log2n + 3 * rounds)
    perms = None if perm_kind == "none" else inputs.permutations(
        S, rounds, N, seed=5, between_rounds_only=(perm_kind == "between"))
    x = inputs.laplacian_blocks(B, N, 50.0, -32768, 32767, seed=log2n + 1).astype(np.float32)
    sets = inputs.set_indices(B, S, seed=log2n + 2, skip_frac=0.1)
    sets[7] = 50  # a bad set index
    plan = gpu.Plan(log2n, rounds, q, perms)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    b = gpu.Batch(plan, B).build(_t(sets))
    y = b.forward_f32(_t(x), status=st)
    xr = b.inverse_f32(y, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == gpu.HYGT_ERR_SET_INDEX
    theta = inputs.theta_from_indices(q)
    ye, ste = orc.fwd_f64(x.astype(np.float64), theta, log2n, rounds, perms, sets)
    assert ste == orc.ERR_SET
    yg = y.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(yg - ye)) <= 1e-5 * np.max(np.abs(ye))
    xe, _ = orc.inv_f64(yg, theta, log2n, rounds, perms, sets)
    assert np.max(np.abs(xr.cpu().numpy() - xe)) <= 1e-5 * np.max(np.abs(xe))
    assert np.all(yg[7] == 0)
    plan.close()


@pytest.mark.parametrize("log2n,rounds", [(4, 2), (5, 2), (6, 2), (7, 2), (8, 3)])
def test_batch_every_launch_tuning_bit_exact(gpu, orc, log2n, rounds):
    """Every point the launch tuner can pick (warps per CTA, CTAs per SM,
    staging depth, register layout) gives the oracle's integers, forward and
    inverse."""
    import torch
    from paper_2505_21728_gb300 import autotune
    N, S = 1 << log2n, 105
    B = 20011 if log2n <= 6 else 3001
    q = inputs.angle_indices(S, rounds, log2n, seed=log2n + 40)
    perms = inputs.permutations(S, rounds, N, seed=41)
    x = inputs.laplacian_blocks(B, N, 20.0, -32768, 32767, seed=log2n + 42)
    sets = inputs.set_indices(B, S, seed=43, skip_frac=0.1)
    ye, _ = orc.fwd_int(x, q, log2n, rounds, perms, sets)
    xe, _ = orc.inv_int(ye, q, log2n, rounds, perms, sets)
    plan = gpu.Plan(log2n, rounds, q, perms)
    b = gpu.Batch(plan, B).build(_t(sets))
    dx, dy = _t(x), _t(ye)
    ran = 0
    layouts = set()
    for inv in (0, 1):
        for cand in autotune.all_batch_candidates(plan, inv):
            assert gpu.hygt_batch_set_tuning(plan.handle, inv, *cand) == gpu.HYGT_OK
            layouts.add(cand[3])
            st = torch.zeros(1, dtype=torch.int32, device="cuda")
            try:
                out = b.forward(dx, status=st) if inv == 0 else b.inverse(dy, status=st)
            except gpu.HygtError as e:
                assert e.code == gpu.HYGT_ERR_UNSUPPORTED  # does not fit: refused
                continue
            torch.cuda.synchronize()
            assert int(st.item()) == 0, cand
            assert np.array_equal(out.cpu().numpy(), xe if inv else ye), (inv, cand)
            ran += 1
        gpu.hygt_batch_set_tuning(plan.handle, inv, 0, 0, -1, 0)
    assert ran >= 8
    assert layouts == {4: {0, 1, 2, 3, 4}, 6: {0, 1, 2, 3, 4}, 8: {0, 2, 4, 5}}.get(log2n, {0})
    plan.close()


def test_tune_batch_sets_a_fitting_point(gpu, tmp_path, monkeypatch):
    """The tuner times the candidates on the GPU and leaves the fastest set."""
    import torch
    from paper_2505_21728_gb300 import autotune
    monkeypatch.setenv("HYGT_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    log2n, R, S, B = 6, 2, 105, 1 << 18
    q = inputs.angle_indices(S, R, log2n, seed=1)
    plan = gpu.Plan(log2n, R, q)
    x = _t(inputs.laplacian_blocks(B, 64, 8.0, -1024, 1023, seed=1))
    b = gpu.Batch(plan, B).build(_t(inputs.set_indices(B, S, seed=1)))
    y = torch.empty((B, 64), dtype=torch.int32, device="cuda")
    xr = torch.empty_like(x)
    res = autotune.tune_batch(b, x, y, xr, reps=2)
    for inv, d in ((0, "forward"), (1, "inverse")):
        w, c, s, lay, ms, tail = res[d]
        assert gpu.hygt_batch_get_tuning(plan.handle, inv)[:4] == (w, c, s, lay)
        assert gpu.hygt_batch_get_tail(plan.handle, inv) == tail
        assert ms > 0
    again = autotune.tune_batch(b, x, y, xr, reps=2)  # from the cache
    assert again == {k: tuple(v) for k, v in res.items()}
    plan.close()


@pytest.mark.parametrize("perm_kind", ["none", "between", "all"])
@pytest.mark.parametrize("stage", [0, 1, 2])
@pytest.mark.parametrize("log2n,R,S,B", [(4, 2, 105, 20011), (6, 2, 105, 9001), (8, 3, 16, 3001)])
def test_batch_transposed_layout_bit_exact(gpu, orc, log2n, R, S, B, perm_kind, stage):
    """Layout 4 (cross-lane passes done as register passes on the block
    transposed through shared memory, the transpose back folded into the
    permutation slot where one follows): the oracle's integers, forward and
    inverse, with no permutation, with slots between rounds only (the last
    round transposes back explicitly) and with a slot after every round."""
    import torch
    N = 1 << log2n
    q = inputs.angle_indices(S, R, log2n, seed=71)
    perms = None if perm_kind == "none" else inputs.permutations(
        S, R, N, seed=72, between_rounds_only=(perm_kind == "between"))
    x = inputs.laplacian_blocks(B, N, 30.0, -32768, 32767, seed=73)
    sets = inputs.set_indices(B, S, seed=74, skip_frac=0.1)
    sets[5] = 999
    ye, s1 = orc.fwd_int(x, q, log2n, R, perms, sets)
    xe, s2 = orc.inv_int(ye, q, log2n, R, perms, sets)
    assert s1 == s2 == orc.ERR_SET
    plan = gpu.Plan(log2n, R, q, perms)
    b = gpu.Batch(plan, B).build(_t(sets))
    for lay in ((4, 5) if log2n == 8 else (4,)):  # 5: the same with two blocks per lane group
        for inv in (0, 1):
            assert gpu.hygt_batch_set_tuning(plan.handle, inv, 0, 0, stage, lay) == gpu.HYGT_OK
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        y = b.forward(_t(x), status=st)
        xr = b.inverse(_t(ye), status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == gpu.HYGT_ERR_SET_INDEX
        assert np.array_equal(y.cpu().numpy(), ye), lay
        assert np.array_equal(xr.cpu().numpy(), xe), lay
    plan.close()


@pytest.mark.parametrize("perm_kind", ["none", "all"])
@pytest.mark.parametrize("layout", [0, 2])
def test_batch_interleaved_order_bit_exact(gpu, orc, perm_kind, layout):
    """Stage 4 (4x4 blocks: tasks taken one set after the other, all warps
    sweeping the sets together): the oracle's integers, forward and inverse,
    with the set tables in shared memory (one CTA per SM) and read from
    global memory (two CTAs per SM: the tables no longer fit), a bad set
    index, a batch whose blocks use only three sets, and a batch smaller
    than one task."""
    import torch
    log2n, R, S, N = 4, 2, 105, 16
    q = inputs.angle_indices(S, R, log2n, seed=81)
    perms = None if perm_kind == "none" else inputs.permutations(S, R, N, seed=82)
    plan = gpu.Plan(log2n, R, q, perms)
    cases = []
    x = inputs.laplacian_blocks(40009, N, 30.0, -32768, 32767, seed=83)
    sets = inputs.set_indices(40009, S, seed=84, skip_frac=0.1)
    sets[11] = 700
    cases.append((x, sets, orc.ERR_SET))
    few = inputs.set_indices(9000, 3, seed=85, skip_frac=0.05)  # sets 0..2 and skips
    cases.append((inputs.laplacian_blocks(9000, N, 30.0, -32768, 32767, seed=86), few, 0))
    cases.append((inputs.laplacian_blocks(5, N, 30.0, -32768, 32767, seed=87),
                  inputs.set_indices(5, S, seed=88), 0))
    for x, sets, want in cases:
        B = x.shape[0]
        ye, s1 = orc.fwd_int(x, q, log2n, R, perms, sets)
        xe, s2 = orc.inv_int(ye, q, log2n, R, perms, sets)
        assert s1 == s2 == want
        b = gpu.Batch(plan, B).build(_t(sets))
        for ctas in (1, 2):
            for w in (0, 4):
                for inv in (0, 1):
                    assert gpu.hygt_batch_set_tuning(plan.handle, inv, w, ctas, 4, layout) == 0
                st = torch.zeros(1, dtype=torch.int32, device="cuda")
                y = b.forward(_t(x), status=st)
                xr = b.inverse(_t(ye), status=st)
                torch.cuda.synchronize()
                assert int(st.item()) == (gpu.HYGT_ERR_SET_INDEX if want else 0)
                assert np.array_equal(y.cpu().numpy(), ye), (B, ctas, w)
                assert np.array_equal(xr.cpu().numpy(), xe), (B, ctas, w)
    # other block sizes and layouts have no interleaved order
    assert gpu.hygt_batch_set_tuning(plan.handle, 0, 0, 0, 4, 1) == gpu.HYGT_ERR_UNSUPPORTED
    plan.close()
    p6 = gpu.Plan(6, 2, inputs.angle_indices(3, 2, 6, seed=1))
    assert gpu.hygt_batch_set_tuning(p6.handle, 0, 0, 0, 4, 0) == gpu.HYGT_ERR_UNSUPPORTED
    p6.close()


DYN_POINTS = {6: [(lay, st) for lay in (0, 3) for st in ((0, 1, 2, 3) if lay == 0 else (0, 1, 2))],
              8: [(lay, st) for lay in (0, 4, 5) for st in ((0, 1, 2, 3) if lay == 0 else (0, 1, 2))]}


@pytest.mark.parametrize("log2n,R,S,B", [(6, 2, 105, 20011), (8, 3, 16, 3001)])
def test_batch_dynamic_tail_bit_exact(gpu, orc, log2n, R, S, B):
    """The kernels with a dynamic tail (the last t/64 of the sorted order
    handed out through an atomic counter): the oracle's integers, forward and
    inverse, at every layout and stage they take, with a quarter-size and a
    half-size tail, a bad set index, calls repeated without a rebuild (the
    counter must come back to zero), and a batch of five blocks."""
    import torch
    N = 1 << log2n
    q = inputs.angle_indices(S, R, log2n, seed=91)
    perms = inputs.permutations(S, R, N, seed=92)
    plan = gpu.Plan(log2n, R, q, perms)
    for nb in (B, 5):
        x = inputs.laplacian_blocks(nb, N, 30.0, -32768, 32767, seed=93 + nb)
        sets = inputs.set_indices(nb, S, seed=94, skip_frac=0.1)
        if nb > 100:
            sets[17] = 999
        ye, s1 = orc.fwd_int(x, q, log2n, R, perms, sets)
        xe, _ = orc.inv_int(ye, q, log2n, R, perms, sets)
        want = gpu.HYGT_ERR_SET_INDEX if s1 else 0
        b = gpu.Batch(plan, nb).build(_t(sets))
        dx, dy = _t(x), _t(ye)
        for lay, st in DYN_POINTS[log2n]:
            for tail in (16, 32):
                for inv in (0, 1):
                    assert gpu.hygt_batch_set_tail(plan.handle, inv, 0) == 0
                    assert gpu.hygt_batch_set_tuning(plan.handle, inv, 0, 0, st, lay) == 0
                    assert gpu.hygt_batch_set_tail(plan.handle, inv, tail) == 0
                    assert gpu.hygt_batch_get_tail(plan.handle, inv) == tail
                for rep in range(2):  # the second pass runs on the counters the first reset
                    st_ = torch.zeros(1, dtype=torch.int32, device="cuda")
                    y = b.forward(dx, status=st_)
                    xr = b.inverse(dy, status=st_)
                    torch.cuda.synchronize()
                    assert int(st_.item()) == want, (nb, lay, st, tail)
                    assert np.array_equal(y.cpu().numpy(), ye), (nb, lay, st, tail, rep)
                    assert np.array_equal(xr.cpu().numpy(), xe), (nb, lay, st, tail, rep)
    for inv in (0, 1):
        assert gpu.hygt_batch_set_tail(plan.handle, inv, 0) == 0
    # a tail is refused where no such kernel exists, and so is a tuning that
    # would leave a set tail without one
    assert gpu.hygt_batch_set_tail(plan.handle, 0, 33) == gpu.HYGT_ERR_ARG
    assert gpu.hygt_batch_set_tuning(plan.handle, 0, 0, 0, 0, 2) == 0
    assert gpu.hygt_batch_set_tail(plan.handle, 0, 8) == gpu.HYGT_ERR_UNSUPPORTED
    assert gpu.hygt_batch_set_tuning(plan.handle, 0, 0, 0, 0, 0) == 0
    assert gpu.hygt_batch_set_tail(plan.handle, 0, 8) == 0
    assert gpu.hygt_batch_set_tuning(plan.handle, 0, 0, 0, 0, 2) == gpu.HYGT_ERR_UNSUPPORTED
    plan.close()
    p4 = gpu.Plan(4, 2, inputs.angle_indices(3, 2, 4, seed=1))
    assert gpu.hygt_batch_set_tail(p4.handle, 0, 8) == gpu.HYGT_ERR_UNSUPPORTED
    p4.close()
