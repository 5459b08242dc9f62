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
    assert len(split) == 3 and all(c >= 1 for c in split)
    assert sum(split) == gpu.hygt_mixed_ctas()
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
