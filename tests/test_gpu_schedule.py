"""Results do not depend on the schedule (rows per unit, grid cap), alone or
in a batch whose buffers carry different schedules; the autotuner picks one
of its candidates and checks its own round trips."""
import numpy as np
import pytest

import oracle
from paper_1803_04880_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fr():
    import paper_1803_04880_b300 as m
    m.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


@pytest.mark.parametrize("rows,ctas", [(16, 0), (32, 148), (128, 0), (256, 7), (64, 1)])
def test_single_call_any_schedule(fr, rows, ctas):
    data = wl.random_bytes(600_000, rows + ctas)
    W, L = 1024, 3
    plan = fr.Plan(W, L)
    plan.set_schedule(rows, ctas)
    key = fr.Key(wl.KEY)
    d = torch.from_numpy(data).cuda()
    priv, pub = fr.protect(plan, key, 5, d)
    out = fr.recover(plan, key, 5, priv, pub, data.size)
    fr.sync_status()
    p_ref, u_ref = oracle.protect(data, W, L, wl.KEY, 5)
    assert np.array_equal(priv.cpu().numpy(), p_ref)
    assert np.array_equal(pub.cpu().numpy(), u_ref)
    assert np.array_equal(out.cpu().numpy(), data)


def test_batch_with_mixed_schedules(fr):
    key = fr.Key(wl.KEY)
    specs = [(300_000, 512, 2, (16, 0)), (70_000, 256, 4, (128, 0)), (1_000_000, 2048, 1, (64, 0)),
             (5_000, 64, 3, (0, 0))]
    entries, rentries, refs = [], [], []
    for i, (n, W, L, sched) in enumerate(specs):
        plan = fr.Plan(W, L)
        plan.set_schedule(*sched)
        data = wl.random_bytes(n, 40 + i)
        d = torch.from_numpy(data).cuda()
        _, pb, ub = plan.sizes(n)
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(n, dtype=torch.uint8, device="cuda")
        entries.append((plan, i, n, d, p, u))
        rentries.append((plan, i, n, p, u, o))
        refs.append((data, W, L))
    fr.protect_batch(entries, key)
    fr.recover_batch(rentries, key)
    fr.sync_status()
    for (plan, i, n, d, p, u), (_, _, _, _, _, o), (data, W, L) in zip(entries, rentries, refs):
        p_ref, u_ref = oracle.protect(data, W, L, wl.KEY, i)
        assert np.array_equal(p.cpu().numpy(), p_ref)
        assert np.array_equal(u.cpu().numpy(), u_ref)
        assert np.array_equal(o.cpu().numpy(), data)


def test_tuner_picks_a_candidate(fr, tmp_path):
    from paper_1803_04880_b300 import tune
    path = str(tmp_path / "sched.json")
    res = tune.tune(2048, 3, 4 << 20, reps=1, path=path)
    assert res["seg_rows"] in tune.CANDIDATE_ROWS
    assert len(res["timings"]) == len(list(tune.candidates(
        torch.cuda.get_device_properties(0).multi_processor_count)))
    plan = fr.Plan(2048, 3)
    assert tune.apply(plan, 4 << 20, path=path)
    assert plan.schedule() == (res["seg_rows"], res["ctas"])


def test_large_batch_one_fused_launch_per_level_count(fr):
    """A batch whose level counts each fill at least eight rounds of full
    fused units on the device runs its first fused pass as one launch per
    count (4-level buffers join the 3-level launch and add the second fused
    pass); its fragments equal one protect call per buffer, and its recover
    gives the bytes back."""
    key = fr.Key(wl.KEY)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    W = 4096
    strips = -(-W // 240)                      # warp strips of 240 owned columns (232 at three levels)
    need = 8.8 * sms * 16 * 32 / strips        # fused iterations per level count, with a margin
    rows = int(need * 8 / 5) + 1               # five buffers a count
    entries, rentries, singles = [], [], []
    for L in (1, 2, 3, 4):
        plan = fr.Plan(W, L)
        for k in range(5 if L < 4 else 2):
            n = W * (rows + 37 * k) + 1000 * k + 3
            nonce = 100 * L + k
            d = torch.from_numpy(wl.random_bytes(n, nonce)).cuda()
            _, pb, ub = plan.sizes(n)
            p = torch.empty(pb, dtype=torch.uint8, device="cuda")
            u = torch.empty(ub, dtype=torch.uint8, device="cuda")
            o = torch.empty(n, dtype=torch.uint8, device="cuda")
            entries.append((plan, nonce, n, d, p, u))
            rentries.append((plan, nonce, n, p, u, o))
            singles.append(fr.protect(plan, key, nonce, d))
    bp, br = fr.Batch(entries, protect=True), fr.Batch(rentries, protect=False)
    # three first-pass launches (one per level count), the second pass (the
    # 4-level buffers' levels 4) and the CTR launch, each way
    assert bp.info()[0] == 5 and br.info()[0] == 5
    bp.run(key)
    br.run(key)
    fr.sync_status()
    for (plan, nonce, n, d, p, u), (_, _, _, _, _, o), (p1, u1) in zip(entries, rentries, singles):
        what = "(L=%d, n=%d)" % (plan.levels, n)
        assert torch.equal(p, p1), "private fragment differs " + what
        assert torch.equal(u, u1), "public fragment differs " + what
        assert torch.equal(o, d), "recovered bytes differ " + what
