"""Autotuner logic on the CPU with a fake timer (selection, cache keys,
persistence), plus a GPU check that tuned knobs keep the answer."""
from __future__ import annotations

import pytest

from paper_1411_5283_gb300 import autotune as at


def test_candidates_are_valid_tunes():
    for alg in ("merge", "odd_even"):
        for W in (8, 16, 24, 32):
            cs = at.candidates(alg, W)
            assert cs
            for c in cs:
                p = c["merge_fanin"]
                t = c.get("tile", c.get("oddeven_max"))
                assert p <= 2 * t and 2 * p * (8 * (W // 8) + 4) <= 200 * 1024
                assert c["threads_per_bucket"] in (256, 512, 1024)


def test_choose_picks_fastest(tmp_path):
    cs = [{"tile": 1024}, {"tile": 2048}, {"tile": 4096}]
    times = {1024: 3.0, 2048: 1.0, 4096: 2.0}
    best, t = at.choose(lambda c: times[c["tile"]], cs)
    assert best == {"tile": 2048} and t == 1.0


def test_cache_roundtrip_and_reuse(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def fake(c):
        calls.append(c)
        return 1.0 / c["tile"]

    cs = [{"tile": 1024}, {"tile": 4096}]
    key = at.tune_key("GB300", 152, 16, "merge", 3000)
    assert key.endswith("|n4096|single")
    assert at.tune(key, fake, cs, path) == {"tile": 4096}
    assert len(calls) == 2
    assert at.tune(key, fake, cs, path) == {"tile": 4096}   # cached: no new timing
    assert len(calls) == 2
    assert at.lookup(key, path) == {"tile": 4096}
    assert at.lookup("other", path) is None
    at.tune(key, lambda c: c["tile"], cs, path, force=True)
    assert at.lookup(key, path) == {"tile": 1024}


def test_refine_sweeps_crossovers_of_the_winner(tmp_path):
    path = str(tmp_path / "tune.json")
    cs = [{"tile": 1024}, {"tile": 2048}]
    seen = []

    def fake(c):
        seen.append(dict(c))
        if "oddeven_cross" in c:
            return 0.5 + abs(c["oddeven_cross"] - 128) / 1e4  # 128 is fastest
        return 1.0 if c["tile"] == 2048 else 2.0

    best = at.tune("k", fake, cs, path, refine=at.crossover_candidates)
    assert best == {"tile": 2048, "oddeven_cross": 128}
    assert {c.get("oddeven_cross") for c in seen[2:]} == set(at.CROSSOVERS)
    assert at.load_cache(path)["k"]["tune"]["oddeven_cross"] == 128
    assert all(c["oddeven_cross"] <= 256 for c in at.crossover_candidates({"tile": 256}))


def test_size_class():
    assert at.size_class(1) == 1 and at.size_class(1000) == 1024 and at.size_class(1024) == 1024


@pytest.mark.gpu
def test_tuned_knobs_keep_the_answer(orc, tmp_path):
    from gpu_util import assert_same_answer, need_cuda, table, to_dev
    torch = need_cuda()
    import paper_1411_5283_gb300 as bs
    rec, ln = table(5, 50_000, 16, b"abcdefgh", 7)
    s = bs.Sorter(ln.size, 16)
    d_rec, d_len = to_dev(rec, torch), to_dev(ln, torch)
    path = str(tmp_path / "t.json")
    best = at.tune_records(s, d_rec, d_len, ln.size, "merge", path=path, max_candidates=6)
    assert "oddeven_cross" in best  # the crossover sweep ran and its winner is cached
    assert at.load_cache(path)[next(iter(at.load_cache(path)))]["tune"] == best
    out = s.sort_records(d_rec, d_len, ln.size, alg="merge", tune=best)
    torch.cuda.synchronize()
    assert_same_answer(*out, orc.stable_sort(orc.Words(rec, ln)), ln.size)
