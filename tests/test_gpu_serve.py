"""The serving loop (continuous batching): every request's result is the same
alone and in the mix, and equals the oracle; admission by a small memory
budget still completes every request."""
import threading
import time

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


def _sizes(count, seed, lo=1024, hi=1 << 22):
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)


def _submit_poisson(fn, args, rate, seed):
    """Call fn(*a) for a in args at Poisson arrival times (from this thread)."""
    rng = np.random.default_rng(seed)
    out, t0 = [], time.perf_counter()
    t = 0.0
    for a in args:
        t += rng.exponential(1.0 / rate)
        while time.perf_counter() - t0 < t:
            time.sleep(0)
        out.append(fn(*a))
    return out


def test_mix_equals_alone_and_oracle(fr):
    from paper_1803_04880_b300.serve import Server
    sizes = _sizes(48, 7)
    datas = [torch.from_numpy(wl.random_bytes(int(n), 100 + i)).cuda() for i, n in enumerate(sizes)]
    torch.cuda.synchronize()
    with Server(wl.KEY, width=4096, levels=3, max_groups=2) as srv:
        reqs = _submit_poisson(srv.submit_protect, [(d, i) for i, d in enumerate(datas)], 4000.0, 1)
        for r in reqs:
            assert r.wait(60)
        # recover every buffer in a mix with a second round of protects
        mixed = []
        for i, (r, d) in enumerate(zip(reqs, datas)):
            mixed.append((srv.submit_recover(r.private, r.public, r.nbytes, r.nonce), d))
            if i % 3 == 0:
                mixed.append((srv.submit_protect(d, 1000 + i), None))
        for r, _ in mixed:
            assert r.wait(60)
        srv.check()
        assert srv.launches >= 2
    plan = fr.Plan(4096, 3)
    key = fr.Key(wl.KEY)
    for i, (r, d) in enumerate(zip(reqs, datas)):
        assert r.error is None and r.latency_s is not None
        p_alone, u_alone = fr.protect(plan, key, i, d)
        torch.cuda.synchronize()
        assert torch.equal(r.private, p_alone) and torch.equal(r.public, u_alone), i
        if d.numel() <= 1 << 18:
            p_ref, u_ref = oracle.protect(d.cpu().numpy(), 4096, 3, wl.KEY, i)
            assert np.array_equal(r.private.cpu().numpy(), p_ref)
            assert np.array_equal(r.public.cpu().numpy(), u_ref)
    for r, d in mixed:
        if r.kind == "recover":
            assert torch.equal(r.out, d)
        else:
            p_alone, u_alone = fr.protect(plan, key, r.nonce, r.data)
            assert torch.equal(r.private, p_alone) and torch.equal(r.public, u_alone)
    fr.sync_status()


def test_small_memory_budget_admits_in_turn(fr):
    from paper_1803_04880_b300.serve import Server
    sizes = _sizes(24, 8, lo=1 << 16, hi=1 << 21)
    datas = [torch.from_numpy(wl.random_bytes(int(n), 300 + i)).cuda() for i, n in enumerate(sizes)]
    torch.cuda.synchronize()
    with Server(wl.KEY, width=1024, levels=2, memory_budget=6 << 20, max_groups=2) as srv:
        reqs = [srv.submit_protect(d, i) for i, d in enumerate(datas)]
        for r in reqs:
            assert r.wait(60)
        backs = [srv.submit_recover(r.private, r.public, r.nbytes, r.nonce) for r in reqs]
        for r in backs:
            assert r.wait(60)
        srv.check()
        assert srv.launches >= 4  # the budget forced several groups
    for r, d in zip(backs, datas):
        assert torch.equal(r.out, d)


def test_held_requests_launch_together(fr):
    """Requests submitted while the scheduler holds are admitted as one group
    when the hold ends: one protect launch and one recover launch in all."""
    from paper_1803_04880_b300.serve import Server
    sizes = _sizes(24, 11, hi=1 << 20)
    datas = [torch.from_numpy(wl.random_bytes(int(n), 300 + i)).cuda() for i, n in enumerate(sizes)]
    torch.cuda.synchronize()
    with Server(wl.KEY, width=4096, levels=3, max_groups=2) as srv:
        with srv.held():
            first = [srv.submit_protect(d, i) for i, d in enumerate(datas)]
            time.sleep(0.05)
            assert not any(r.done for r in first)  # nothing admitted while held
        for r in first:
            assert r.wait(60)
        assert srv.launches == 1
        with srv.held():
            back = [srv.submit_recover(r.private, r.public, r.nbytes, r.nonce) for r in first]
            again = [srv.submit_protect(d, 100 + i) for i, d in enumerate(datas[:5])]
        for r in back + again:
            assert r.wait(60)
        assert srv.launches == 3  # one protect batch and one recover batch for the mixed group
        srv.check()
    for r, d in zip(back, datas):
        assert torch.equal(r.out, d)
