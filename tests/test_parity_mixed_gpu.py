"""Parity of the mixed-size persistent launch (4x4 / 8x8 / 16x16 blocks in
one kernel), its CUDA-graph replay and the autotuned CTA split, with the
CPU oracle: bit-exact on every block of every class."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_mixed(gpu, w, bad_set=False):
    classes, datas = [], []
    for cw in w.classes():
        d = cw.generate()
        if bad_set and cw.log2n == 6:
            d["sets"][5] = cw.num_sets + 3
        plan = gpu.Plan(cw.log2n, cw.rounds, d["angle_idx"], d["perms"])
        classes.append((plan, _t(d["x"]), _t(d["sets"])))
        datas.append((cw, d))
    return gpu.MixedBatch(classes), datas


def check_against_oracle(orc, mb, datas):
    for e, (cw, d) in zip(mb.entries, datas):
        ye, st1 = orc.fwd_int(d["x"], d["angle_idx"], cw.log2n, cw.rounds, d["perms"], d["sets"])
        xe, st2 = orc.inv_int(ye, d["angle_idx"], cw.log2n, cw.rounds, d["perms"], d["sets"])
        assert np.array_equal(e["y"].cpu().numpy(), ye), cw.name
        assert np.array_equal(e["xr"].cpu().numpy(), xe), cw.name


@pytest.mark.parametrize("scale_down", [400, 40])
def test_mixed_launch(gpu, orc, scale_down):
    """Default launch: every CTA works through the three classes in turn."""
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get_mixed("mixed_frame_2160p16", scale_down=scale_down)
    mb, datas = make_mixed(gpu, w)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.build()
    mb.forward(status=st)
    mb.inverse(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_against_oracle(orc, mb, datas)


def test_mixed_graph_and_split(gpu, orc):
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get_mixed("mixed_frame_2160p16", scale_down=100)
    mb, datas = make_mixed(gpu, w)
    mb.set_split([7, 5, 3])  # an explicit, deliberately uneven split
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = mb.graph(status=st)
    for e in mb.entries:
        e["y"].zero_()
        e["xr"].zero_()
    g.launch()
    g.launch()  # replaying the step twice gives the same result
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_against_oracle(orc, mb, datas)
    g.close()


def test_mixed_autotune_keeps_results(gpu, orc, tmp_path, monkeypatch):
    import torch
    from paper_2505_21728_gb300 import autotune, workloads
    monkeypatch.setenv("HYGT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    w = workloads.get_mixed("mixed_frame_2160p16", scale_down=50)
    mb, datas = make_mixed(gpu, w)
    mb.build()
    split = autotune.tune_split(mb, reps=2)
    assert len(split) == 3
    # the sequential launch (all zeros), separate launches (all -1), or a
    # concurrent split of all CTAs
    assert (all(c == 0 for c in split) or all(c == -1 for c in split) or
            (all(c >= 1 for c in split) and sum(split) == gpu.hygt_mixed_ctas()))
    assert (tmp_path / "tune.json").exists()
    assert autotune.tune_split(mb, reps=2) == split  # cached
    mb.forward()
    mb.inverse()
    torch.cuda.synchronize()
    check_against_oracle(orc, mb, datas)


def test_mixed_bad_set_reports(gpu, orc):
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get_mixed("mixed_frame_2160p16", scale_down=400)
    mb, datas = make_mixed(gpu, w, bad_set=True)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.build()
    mb.forward(status=st)
    mb.inverse(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 4
    check_against_oracle(orc, mb, datas)


def test_mixed_frame_full(gpu, orc):
    """The full 16-frame 2160p mixed batch (4,950,720 blocks), graph-replayed
    with the autotuned split: every block of every class bit-exact."""
    import torch
    from paper_2505_21728_gb300 import autotune, workloads
    w = workloads.get_mixed("mixed_frame_2160p16")
    mb, datas = make_mixed(gpu, w)
    mb.build()
    autotune.tune_split(mb, reps=3, use_cache=False)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = mb.graph(status=st)
    g.launch()
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_against_oracle(orc, mb, datas)


def test_mixed_class_order_empty_and_duplicate(gpu, orc):
    """Classes given in any order (they are stored by block size), a class
    without blocks, and two classes of one size (rejected)."""
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get_mixed("mixed_frame_2160p16", scale_down=400)
    cws = list(w.classes())
    classes, datas = [], []
    for cw in reversed(cws):  # N = 256, 64, 16
        d = cw.generate()
        plan = gpu.Plan(cw.log2n, cw.rounds, d["angle_idx"], d["perms"])
        classes.append((plan, _t(d["x"]), _t(d["sets"])))
        datas.append((cw, d))
    mb = gpu.MixedBatch(classes).build()
    for split in (None, [3, 11, 5], [-1, -1, -1]):
        mb.set_split(split)
        for e in mb.entries:
            e["y"].zero_()
            e["xr"].zero_()
        mb.forward()
        mb.inverse()
        torch.cuda.synchronize()
        check_against_oracle(orc, mb, datas)

    # the 8x8 class without blocks: the others are unaffected
    cw, d = datas[1]
    plan = classes[1][0]
    empty = (plan, torch.empty((0, cw.N), dtype=torch.int16, device="cuda"),
             torch.empty((0,), dtype=torch.int16, device="cuda"))
    mb2 = gpu.MixedBatch([classes[0], empty, classes[2]]).build()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb2.forward(status=st)
    mb2.inverse(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_against_oracle(orc, type("M", (), {"entries": [mb2.entries[0], mb2.entries[2]]}),
                         [datas[0], datas[2]])

    mb3 = gpu.MixedBatch([classes[1], classes[1]]).build()
    with pytest.raises(gpu.HygtError) as ei:
        mb3.forward()
    assert ei.value.code == gpu.HYGT_ERR_ARG


# (stage, layout) pairs of the layout-aware single launch, per log2 N; entry
# 0 is layout 0 with its default staging.
MIXED_MENU = {4: [(0, 0), (0, 2), (1, 2)],
              6: [(1, 0), (0, 3), (2, 3)],
              8: [(0, 0), (0, 5), (1, 5), (0, 4)]}


@pytest.mark.parametrize("entry", [0, 1, 2, 3])
def test_mixed_layout_variants_bit_exact(gpu, orc, entry):
    """Every menu entry of the single launch (each class tuned to the
    entry, the last one where its menu is shorter), sequential, with an
    uneven CTA split and graph-replayed: every block bit-exact."""
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get_mixed("mixed_frame_2160p16", scale_down=60)
    mb, datas = make_mixed(gpu, w)
    want = []
    for e in mb.entries:
        plan = e["plan"]
        menu = MIXED_MENU[plan.log2n]
        stage, layout = menu[min(entry, len(menu) - 1)]
        for inv in (0, 1):
            assert gpu.hygt_batch_set_tuning(plan.handle, inv, 0, 0, stage, layout) == 0
        want.append(((stage, layout), (stage, layout)))
    assert mb.variants() == want
    mb.build()
    for split in (None, [9, 4, 2]):
        mb.set_split(split)
        for e in mb.entries:
            e["y"].zero_()
            e["xr"].zero_()
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        mb.forward(status=st)
        mb.inverse(status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        check_against_oracle(orc, mb, datas)
    mb.set_split(None)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = mb.graph(status=st)
    for e in mb.entries:
        e["y"].zero_()
        e["xr"].zero_()
    g.launch()
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_against_oracle(orc, mb, datas)
    g.close()


def test_mixed_layout_variant_mapping(gpu):
    """A tuning whose pair the single launch lacks runs the first entry of
    its layout, else layout 0 with its default staging; stage -1 reads as
    the layout's default."""
    from paper_2505_21728_gb300 import inputs
    cases = {4: [((-1, 0), (0, 0)), ((2, 0), (0, 0)), ((2, 2), (0, 2)), ((0, 1), (0, 0)),
                 ((1, 3), (0, 0)), ((-1, 2), (0, 2))],
             6: [((-1, 0), (1, 0)), ((3, 0), (1, 0)), ((1, 3), (0, 3)), ((2, 3), (2, 3)),
                 ((0, 1), (1, 0)), ((-1, 3), (0, 3))],
             8: [((-1, 0), (0, 0)), ((3, 0), (0, 0)), ((2, 5), (0, 5)), ((1, 4), (0, 4)),
                 ((0, 2), (0, 0)), ((-1, 5), (0, 5))]}
    for log2n, pairs in cases.items():
        N = 1 << log2n
        q = inputs.angle_indices(3, 2, log2n, seed=log2n)
        plan = gpu.Plan(log2n, 2, q, inputs.permutations(3, 2, N, seed=log2n))
        for (stage, layout), expect in pairs:
            assert gpu.hygt_batch_set_tuning(plan.handle, 1, 0, 0, stage, layout) == 0
            assert gpu.hygt_mixed_class_variant(plan.handle, 1) == expect, (log2n, stage, layout)
        plan.close()
    # N = 32 has no class in a mixed launch
    q = inputs.angle_indices(1, 2, 5, seed=5)
    plan = gpu.Plan(5, 2, q, inputs.permutations(1, 2, 32, seed=5))
    with pytest.raises(RuntimeError):
        gpu.hygt_mixed_class_variant(plan.handle, 0)
    plan.close()


def test_mixed_separate_launches_with_dynamic_tails(gpu, orc):
    """Per-class launches with dynamic tails on the 8x8 and 16x16 classes
    (and the 4x4 class in the set-interleaved order), graph-replayed twice:
    every block bit-exact."""
    import torch
    from paper_2505_21728_gb300 import workloads
    w = workloads.get_mixed("mixed_frame_2160p16", scale_down=40)
    mb, datas = make_mixed(gpu, w)
    for e in mb.entries:
        plan = e["plan"]
        for inv in (0, 1):
            if plan.log2n == 4:
                assert gpu.hygt_batch_set_tuning(plan.handle, inv, 4, 0, 4, 2) == 0
            else:
                lay = 3 if plan.log2n == 6 else 5
                assert gpu.hygt_batch_set_tuning(plan.handle, inv, 0, 0, 0, lay) == 0
                assert gpu.hygt_batch_set_tail(plan.handle, inv, 16) == 0
    mb.set_split([-1, -1, -1])
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = mb.graph(status=st)
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_against_oracle(orc, mb, datas)
    g.close()
