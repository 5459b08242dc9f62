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
