"""Serving loop for protect / recover requests on one GPU, with continuous
batching.

Requests arrive at any time (``submit_protect`` / ``submit_recover``, from any
thread).  A scheduler thread admits waiting requests in arrival order while
the device memory they need (their outputs plus the library's level scratch)
fits the budget, launches every admitted group as one batched call per kind
(``frag_protect_batch`` / ``frag_recover_batch``: one dependency-ordered
launch for all of the group's buffers) on one of its streams, and retires
groups whose completion event has fired.  Requests that arrive while earlier
groups are still on the GPU are admitted as soon as a stream and memory are
free, so their work overlaps on the device (up to ``max_groups`` groups in
flight).  Plans, per (width, levels), and the key schedule stay resident.

Every result is the same as that of a lone call: the transform is exact
integer arithmetic and each buffer's work is independent of the others in a
launch.  The latency of a request runs from ``submit_*`` to the scheduler
seeing its group's completion event.
"""
from __future__ import annotations

import collections
import contextlib
import threading
import time
from typing import List, Optional

import torch

from . import Key, Plan, protect_batch, recover_batch, sync_status


class Request:
    """One protect or recover request and, once ``done``, its outputs."""

    __slots__ = ("kind", "nonce", "nbytes", "plan", "data", "private", "public", "out",
                 "need", "t_submit", "t_launch", "t_done", "error", "_event", "_ready")

    def __init__(self, kind: str, plan: Plan, nonce: int, nbytes: int):
        self.kind = kind
        self.plan = plan
        self.nonce = nonce
        self.nbytes = nbytes
        self.data = self.private = self.public = self.out = None
        self.need = 0
        self.t_submit = time.perf_counter()
        self.t_launch = self.t_done = None
        self.error: Optional[BaseException] = None
        self._event = threading.Event()
        # the caller's stream position at submit: the inputs are ready there
        self._ready = torch.cuda.Event()
        self._ready.record()

    @property
    def done(self) -> bool:
        return self._event.is_set()

    def wait(self, timeout: Optional[float] = None) -> bool:
        return self._event.wait(timeout)

    @property
    def latency_s(self) -> Optional[float]:
        return None if self.t_done is None else self.t_done - self.t_submit


class _Group:
    __slots__ = ("requests", "stream", "event", "need")

    def __init__(self, requests, stream, event, need):
        self.requests, self.stream, self.event, self.need = requests, stream, event, need


class Server:
    """Continuous-batching request loop (see the module docstring).

    key: 16-byte AES key; width/levels: the default plan; memory_budget: device
    bytes the in-flight requests may hold (default: free memory at start minus
    ``reserve``); max_groups: batched groups in flight at once (one stream
    each); max_items: requests per group at most.
    """

    def __init__(self, key: bytes, width: int = 4096, levels: int = 3, device: int = 0,
                 memory_budget: Optional[int] = None, reserve: int = 4 << 30,
                 max_groups: int = 2, max_items: int = 2048):
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.key = Key(key)
        self._plans = {}
        self.default_plan = self.plan(width, levels)
        free, _ = torch.cuda.mem_get_info(self.device)
        self.budget = memory_budget if memory_budget is not None else max(0, free - reserve)
        self.max_groups = max_groups
        self.max_items = max_items
        self._streams = [torch.cuda.Stream(device=self.device) for _ in range(max_groups)]
        self._pending = collections.deque()
        self._inflight: List[_Group] = []
        self._used = 0
        self._cv = threading.Condition()
        self._stop = False
        self._hold = 0
        self.launches = 0
        self._thread = threading.Thread(target=self._loop, name="frag-serve", daemon=True)
        self._thread.start()

    # -- client side --------------------------------------------------------------

    def plan(self, width: int, levels: int) -> Plan:
        key = (width, levels)
        if key not in self._plans:
            self._plans[key] = Plan(width, levels)
        return self._plans[key]

    def _need(self, plan: Plan, kind: str, n: int) -> int:
        _, pb, ub = plan.sizes(n)
        # outputs, plus the level scratch the library allocates (at most about
        # two thirds of the padded matrix, as packed pairs) and descriptors
        scratch = (pb + ub) // 3 + (1 << 16)
        return (pb + ub if kind == "protect" else n) + scratch

    def submit_protect(self, data: torch.Tensor, nonce: int, plan: Optional[Plan] = None) -> Request:
        """Protect the bytes of a uint8 CUDA tensor (kept alive until done).
        Work the caller queued on its current stream before the call (that
        fills `data`) comes first."""
        plan = plan or self.default_plan
        r = Request("protect", plan, nonce, data.numel())
        r.data = data
        r.need = self._need(plan, "protect", r.nbytes)
        self._enqueue(r)
        return r

    def submit_recover(self, private: torch.Tensor, public: torch.Tensor, nbytes: int, nonce: int,
                       plan: Optional[Plan] = None) -> Request:
        plan = plan or self.default_plan
        r = Request("recover", plan, nonce, nbytes)
        r.private, r.public = private, public
        r.need = self._need(plan, "recover", nbytes)
        self._enqueue(r)
        return r

    def _enqueue(self, r: Request) -> None:
        with self._cv:
            if self._stop:
                raise RuntimeError("server is closed")
            self._pending.append(r)
            if not self._hold:  # a held scheduler has nothing to do yet
                self._cv.notify()

    @contextlib.contextmanager
    def held(self):
        """Admit nothing while the block runs: the requests submitted inside
        it wait and are admitted together when it ends (in arrival order,
        within the memory budget), so their grouping does not depend on how
        the scheduler thread interleaves with the submitting one."""
        with self._cv:
            self._hold += 1
        try:
            yield self
        finally:
            with self._cv:
                self._hold -= 1
                self._cv.notify()

    def close(self) -> None:
        """Finish every submitted request, then stop the scheduler."""
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._thread.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- scheduler -----------------------------------------------------------------

    def _admit(self) -> List[Request]:
        """Requests to launch now, in arrival order, within the memory budget."""
        take = []
        used = self._used
        while self._pending and len(take) < self.max_items:
            r = self._pending[0]
            if used + r.need > self.budget and (take or self._inflight):
                break  # wait for memory (a request alone always goes, so nothing starves)
            take.append(self._pending.popleft())
            used += r.need
        return take

    def _launch(self, reqs: List[Request]) -> None:
        stream = self._streams[len(self._inflight) % self.max_groups]
        busy = {id(g.stream) for g in self._inflight}
        for s in self._streams:
            if id(s) not in busy:
                stream = s
                break
        need = sum(r.need for r in reqs)
        now = time.perf_counter()
        try:
            with torch.cuda.stream(stream):
                pitems, ritems = [], []
                for r in reqs:
                    stream.wait_event(r._ready)
                    r.t_launch = now
                    if r.kind == "protect":
                        _, pb, ub = r.plan.sizes(r.nbytes)
                        r.private = torch.empty(pb, dtype=torch.uint8, device=self.device)
                        r.public = torch.empty(ub, dtype=torch.uint8, device=self.device)
                        pitems.append((r.plan, r.nonce, r.nbytes, r.data, r.private, r.public))
                    else:
                        r.out = torch.empty(r.nbytes, dtype=torch.uint8, device=self.device)
                        ritems.append((r.plan, r.nonce, r.nbytes, r.private, r.public, r.out))
                if pitems:
                    protect_batch(pitems, self.key, stream)
                    self.launches += 1
                if ritems:
                    recover_batch(ritems, self.key, stream)
                    self.launches += 1
                ev = torch.cuda.Event()
                ev.record(stream)
        except BaseException as e:  # report on every request of the group
            for r in reqs:
                r.error = e
                r.t_done = time.perf_counter()
                r._event.set()
            return
        self._inflight.append(_Group(reqs, stream, ev, need))
        self._used += need

    def _retire(self) -> bool:
        progressed = False
        for g in list(self._inflight):
            if g.event.query():
                now = time.perf_counter()
                for r in g.requests:
                    r.t_done = now
                    r._event.set()
                self._inflight.remove(g)
                self._used -= g.need
                progressed = True
        return progressed

    def check(self) -> None:
        """Raise if a kernel of the server's launches reported an error (the
        device error word is read once every group in flight has finished)."""
        for s in self._streams:
            s.synchronize()
        sync_status(self._streams[0])

    def _loop(self) -> None:
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                if self._stop and not self._pending and not self._inflight:
                    return
                free_slot = len(self._inflight) < self.max_groups
                reqs = self._admit() if free_slot and not self._hold else []
            if reqs:
                self._launch(reqs)
                continue
            if self._retire():
                continue
            with self._cv:
                # nothing to launch now: poll the groups' events, or sleep
                # until a submit when the GPU holds nothing
                self._cv.wait(timeout=20e-6 if self._inflight else 0.01)
