"""Schedule knobs and the autotuner's cache logic (no GPU needed)."""
import pytest

import paper_1803_04880_b300 as fr
from paper_1803_04880_b300 import tune


@pytest.fixture(scope="module")
def L():
    fr.build()
    return fr.lib()


def test_schedule_validation(L):
    p = fr.Plan(4096, 3)
    assert p.schedule() == (0, 0)
    p.set_schedule(32, 300)
    assert p.schedule() == (32, 300)
    for bad in (8, 24, 512, 1000):
        with pytest.raises(fr.FragError):
            p.set_schedule(bad, 0)
    assert p.schedule() == (32, 300)
    p.set_schedule(0, 0)
    assert p.schedule() == (0, 0)
    assert L.frag_plan_set_schedule(None, 0, 0) == fr.FRAG_EINVAL


def test_size_class():
    assert tune.size_class(1) == 0
    assert tune.size_class(1 << 20) == 20
    assert tune.size_class(3 << 20) == 22  # rounds log2 to the nearest integer
    assert tune.size_class(0) == 0


def test_cache_round_trip_and_apply(tmp_path, L):
    path = str(tmp_path / "sched.json")
    assert tune.load_cache(path) == {}
    key = tune._key("B300-test", 4096, 3, 1 << 24)
    tune.save_cache({key: {"seg_rows": 64, "ctas": 296, "us": 1.0, "timings": {}}}, path)
    p = fr.Plan(4096, 3)
    assert tune.apply(p, 1 << 24, path=path, device_name="B300-test")
    assert p.schedule() == (64, 296)
    # a size in another bucket falls back to the library's choice
    assert not tune.apply(p, 1 << 12, path=path, device_name="B300-test")
    assert p.schedule() == (0, 0)


def test_candidates_cover_rows_and_grids():
    c = list(tune.candidates(148))
    assert {r for r, _ in c} == set(tune.CANDIDATE_ROWS)
    assert {g for _, g in c} == {0, 148, 296}


def test_tune_batch_picks_the_fastest_candidate():
    from paper_1803_04880_b300 import tune
    cost = {(0, 0, 0): 5.0, (64, 0, 0): 4.0, (128, 296, 0): 3.5, (256, 0, 0): 6.0, (0, 0, 1): 7.0}
    built, runs = [], []

    def make_run(rows, ctas, path):
        built.append((rows, ctas, path))
        return lambda: runs.append((rows, ctas, path))

    def clock(fn):
        fn()
        return cost[runs[-1]]

    r = tune.tune_batch(make_run, list(cost), reps=2, clock=clock)
    assert (r["seg_rows"], r["ctas"], r["path"], r["ms"]) == (128, 296, 0, 3.5)
    assert built == list(cost) and len(runs) == 3 * len(cost)  # a warm-up and two timed runs each
    assert r["timings"] == {"0/0/0": 5.0, "64/0/0": 4.0, "128/296/0": 3.5, "256/0/0": 6.0, "0/0/1": 7.0}
    cands = list(tune.batch_candidates(148))
    assert cands[:8] == [(rows, c, 0) for rows in tune.BATCH_ROWS for c in (0, 296)]
    assert cands[8:] == [(0, 0, 1), (0, 296, 1)]
