"""Host logic of the mixed-launch autotuner (no GPU): the timing call is
replaced by a cost model, and the tuner must find the mode and CTA split
that the model makes fastest.

Model: class c alone on all G CTAs takes t_c; on a concurrent share of
n_c CTAs it takes t_c G / n_c (linear scaling), and the concurrent launch
ends with its slowest class; the sequential launch takes sum(t_c) times a
penalty; the separate launches take sum(t_c) times another.
"""
import pytest

from paper_2505_21728_gb300 import build as hb

G = 152


@pytest.fixture(scope="module")
def at():
    hb.build()
    from paper_2505_21728_gb300 import autotune
    return autotune


class _FakeMixed:
    def __init__(self, hygt, counts):
        self.n = len(counts)
        self.classes = (hygt.MixedClass * self.n)()
        for i, c in enumerate(counts):
            self.classes[i].nblocks = c
        self.entries = [{} for _ in counts]
        self.split = None

    def set_split(self, split):
        self.split = None if split is None else list(split)


def _model(alone, seq_factor, sep_factor):
    def time_pair(classes, n, reps):
        ctas = [classes[i].ctas for i in range(n)]
        if n == 1:  # one class alone on all CTAs
            for c, t in alone.items():
                if classes[0].nblocks == c:
                    return t
            raise AssertionError("unknown class")
        counts = [classes[i].nblocks for i in range(n)]
        active = [i for i in range(n) if counts[i] > 0]
        times = [alone[counts[i]] for i in active]
        if all(ctas[i] == 0 for i in range(n)):
            return sum(times) * seq_factor
        if all(ctas[i] == -1 for i in range(n)):
            return sum(times) * sep_factor
        assert all(ctas[i] >= 1 for i in active) and sum(ctas[i] for i in active) <= G
        return max(alone[counts[i]] * G / ctas[i] for i in active)
    return time_pair


def _run(at, monkeypatch, alone, seq_factor, sep_factor):
    from paper_2505_21728_gb300 import hygt
    monkeypatch.setattr(at, "_time_pair", _model(alone, seq_factor, sep_factor))
    monkeypatch.setattr(at, "_key", lambda mb: "cpu-model")
    monkeypatch.setattr(at.hygt, "hygt_mixed_ctas", lambda: G)
    mb = _FakeMixed(hygt, list(alone))
    report = {}
    split = at.tune_split(mb, reps=1, use_cache=False, report=report)
    assert mb.split == split
    # the report holds the modes' times; the chosen one is the least of them
    # up to the search's 0.5% acceptance margin
    least = min(report["sequential_ms"], report["separate_ms"], report["best_concurrent_ms"])
    assert least <= report["chosen_ms"] <= least / 0.995
    return split, _model(alone, seq_factor, sep_factor)


def test_concurrent_split_balances_the_classes(at, monkeypatch):
    # block counts double as class ids; class times 0.30 / 0.20 / 0.10 ms alone
    alone = {4147200: 0.30, 725760: 0.20, 77760: 0.10}
    split, model = _run(at, monkeypatch, alone, seq_factor=1.5, sep_factor=1.5)
    assert all(c >= 1 for c in split) and sum(split) == G
    # the best a linear model allows is sum(t) (every class finishing together)
    from paper_2505_21728_gb300 import hygt
    mb = _FakeMixed(hygt, list(alone))
    for i, c in enumerate(split):
        mb.classes[i].ctas = c
    t = model(mb.classes, mb.n, 1)
    assert t <= sum(alone.values()) * 1.02
    # shares close to proportional
    for i, c in enumerate(alone):
        assert abs(split[i] - G * alone[c] / sum(alone.values())) <= 3


def test_separate_launches_win_when_cheaper(at, monkeypatch):
    alone = {1000: 0.3, 2000: 0.2, 3000: 0.1}
    split, _ = _run(at, monkeypatch, alone, seq_factor=1.2, sep_factor=0.9)
    assert split == [-1, -1, -1]


def test_sequential_launch_wins_when_cheaper(at, monkeypatch):
    alone = {1000: 0.3, 2000: 0.2, 3000: 0.1}
    split, _ = _run(at, monkeypatch, alone, seq_factor=0.8, sep_factor=1.1)
    assert split == [0, 0, 0]


def test_single_active_class_takes_every_cta(at, monkeypatch):
    from paper_2505_21728_gb300 import hygt
    monkeypatch.setattr(at, "_key", lambda mb: "cpu-model")
    monkeypatch.setattr(at.hygt, "hygt_mixed_ctas", lambda: G)

    def no_timing(*a, **k):
        raise AssertionError("nothing to time with one class")
    monkeypatch.setattr(at, "_time_pair", no_timing)
    mb = _FakeMixed(hygt, [0, 5000, 0])
    assert at.tune_split(mb, reps=1, use_cache=False) == [0, G, 0]


def test_batch_tuner_picks_the_modelled_best(at, monkeypatch):
    """tune_batch with the GPU timing replaced by a cost model: it must set
    the cheapest fitting point for each direction and skip refused ones."""
    from paper_2505_21728_gb300 import hygt
    state = {}

    def fake_set(plan, inv, w, c, s, lay=0):
        if c == 2 and w > 8:  # pretend these do not fit
            return hygt.HYGT_ERR_UNSUPPORTED
        if lay == 1 and s == 1:  # nor these
            return hygt.HYGT_ERR_UNSUPPORTED
        state[inv] = (w, c, s, lay)
        return hygt.HYGT_OK

    def fake_get(plan, inv):
        return state.get(inv, (0, 0, -1, 0)) + (12,)

    tails = {}

    def fake_set_tail(plan, inv, t):
        if t > 0 and state[inv][2] == 1:  # pretend cp.async points have no dynamic tail
            return hygt.HYGT_ERR_UNSUPPORTED
        tails[inv] = t
        return hygt.HYGT_OK

    monkeypatch.setattr(hygt, "hygt_batch_set_tuning", fake_set)
    monkeypatch.setattr(hygt, "hygt_batch_get_tuning", fake_get)
    monkeypatch.setattr(hygt, "hygt_batch_set_tail", fake_set_tail)

    class _P:
        handle, N, rounds, num_sets, log2n = 1, 64, 2, 105, 6

    class _B:
        plan, nblocks = _P(), 1000

    def model(direction, point):
        w, c, s, lay = point[:4]
        base = 1.0 + abs(w - 9) * 0.1 + (0.05 if c == 0 else 0.0)
        base -= 0.3 if lay == 1 and direction == "inverse" else 0.0
        base -= 0.2 if s == 1 and direction == "forward" else 0.0
        if len(point) > 4:  # a dynamic tail: 8/64 pays 5%, the others nothing
            base *= 0.95 if point[4] == 8 else 1.0
        return base

    res = at.tune_batch(_B(), None, None, None, use_cache=False, time_fn=model)
    assert res["forward"][:4] == (9, 1, 1, 0)
    assert res["inverse"][:4] == (9, 1, 0, 1)   # layout 1, first of the equal stages
    assert state[0] == (9, 1, 1, 0) and state[1] == (9, 1, 0, 1)
    # the forward's point has no tail; the inverse keeps the one that pays
    assert res["forward"][5] == 0 and tails[0] == 0
    assert res["inverse"][5] == 8 and tails[1] == 8
    assert abs(res["inverse"][4] - 0.95 * model("inverse", (9, 1, 0, 1))) < 1e-12


def test_batch_candidates_offer_the_interleaved_order_for_4x4_only(at):
    """Stage 4 (tasks interleaved across the sets) is a candidate for 4x4
    blocks in layouts 0 and 2, and for nothing else; the bulk stage (3) is
    offered in layout 0 only."""
    for log2n in range(2, 9):
        for lay in range(6):
            stages = {c[2] for c in at.batch_candidates(12, log2n, lay)}
            assert all(c[3] == lay for c in at.batch_candidates(12, log2n, lay))
            assert (4 in stages) == (log2n == 4 and lay in (0, 2)), (log2n, lay)
            if log2n >= 4:
                assert (3 in stages) == (lay == 0)
            else:
                assert stages == {-1}
