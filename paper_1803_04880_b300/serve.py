"""Serving loop for protect / recover requests on one GPU, with continuous
batching: a Python face on the library's server (``frag_server_*`` in
include/frag.h), whose scheduler runs as a C++ thread inside the library.

Requests arrive at any time (``submit_protect`` / ``submit_recover``, from any
thread); a submit records the caller's current stream (the work that fills
the input comes first) and queues the request -- one ctypes call.  The
library's scheduler admits waiting requests in arrival order while the device
memory they need (their outputs plus the level scratch) fits the budget and a
group stream is free, allocates their outputs, launches every admitted group
as one batched call per kind, and learns of a group's end from a host
function the group's stream runs -- no polling.  Requests that arrive while
earlier groups are on the GPU are admitted as soon as a stream and memory are
free, so their work overlaps on the device.  Plans, per (width, levels), and
the key schedule stay resident.

Every result is the same as that of a lone call: the transform is exact
integer arithmetic and each buffer's work is independent of the others in a
launch.  The latency of a request runs from its submit to the end of its
group on the device (the library's steady clock).
"""
from __future__ import annotations

import contextlib
import ctypes
from typing import Optional

import torch

from . import FRAG_ETIMEOUT, FRAG_OK, FragError, Key, Plan, _stream, check, frag_request_info, last_error, lib


class _DevBytes:
    """A device byte range as __cuda_array_interface__ (no ownership)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 2}


class _Handle:
    """Owns the library's server; destroyed when the Server and every request
    that still holds outputs are gone."""

    def __init__(self, key: Key, budget: int, max_groups: int, max_items: int):
        self.key = key  # the key must outlive the server
        self.ptr = ctypes.c_void_p()
        check(lib().frag_server_create(ctypes.byref(self.ptr), key.handle, budget, max_groups, max_items))

    def __del__(self):
        if self.ptr:
            lib().frag_server_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()


class Request:
    """One protect or recover request.  Once done: ``private`` / ``public``
    (protect) or ``out`` (recover) are uint8 CUDA tensors over the memory the
    server allocated, valid until ``release()`` (or until the request and
    every such tensor are garbage)."""

    def __init__(self, handle: _Handle, kind: str, plan: Plan, nonce: int, nbytes: int):
        self._h = handle
        self.kind = kind
        self.plan = plan
        self.nonce = nonce
        self.nbytes = nbytes
        self.id = None
        self.data = None           # protect: the input (kept alive)
        self.private = self.public = None
        self.out = None
        self.error: Optional[BaseException] = None
        self.t_submit = self.t_launch = self.t_done = None
        self._done = False
        self._released = False

    def _take(self, info: frag_request_info, status: int) -> None:
        self._done = True
        self.t_submit, self.t_launch, self.t_done = info.t_submit, info.t_launch, info.t_done
        if status != FRAG_OK:
            self.error = FragError(status, last_error())
            return
        if self.kind == "protect":
            self.private = self._view(info.d_private, info.private_bytes)
            self.public = self._view(info.d_public, info.public_bytes)
        else:
            self.out = self._view(info.d_out, info.nbytes)

    def _view(self, ptr: Optional[int], n: int) -> torch.Tensor:
        t = torch.as_tensor(_DevBytes(ptr or 0, n), device="cuda") if n else \
            torch.empty(0, dtype=torch.uint8, device="cuda")
        t._frag_request = self  # the tensor keeps the request (and so its memory) alive
        return t

    def wait(self, timeout: Optional[float] = None) -> bool:
        """True once the request is done (its outputs are ready on the GPU);
        False if timeout seconds pass first."""
        if self._done:
            return True
        info = frag_request_info()
        st = lib().frag_server_wait(self._h.ptr, self.id, -1.0 if timeout is None else float(timeout),
                                    ctypes.byref(info))
        if st == FRAG_ETIMEOUT and not info.done:
            return False
        self._take(info, st)
        return True

    @property
    def done(self) -> bool:
        return self.wait(0.0)

    @property
    def latency_s(self) -> Optional[float]:
        return None if self.t_done is None else self.t_done - self.t_submit

    def release(self) -> None:
        """Give the request's outputs back to the library's pool (after the
        work queued on the current stream)."""
        if self._released or self.id is None or not self._done:
            return
        self._released = True
        self.private = self.public = self.out = None
        if self._h.ptr:
            lib().frag_server_release(self._h.ptr, self.id, _stream(None))

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


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
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            memory_budget = max(1, free - reserve)
        self.budget = memory_budget
        self._h = _Handle(self.key, memory_budget, max_groups, max_items)
        self._closed = False

    def plan(self, width: int, levels: int) -> Plan:
        key = (width, levels)
        if key not in self._plans:
            self._plans[key] = Plan(width, levels)
        return self._plans[key]

    def submit_protect(self, data: torch.Tensor, nonce: int, plan: Optional[Plan] = None) -> Request:
        """Protect the bytes of a uint8 CUDA tensor (kept alive until done).
        Work the caller queued on its current stream before the call (that
        fills `data`) comes first."""
        plan = plan or self.default_plan
        r = Request(self._h, "protect", plan, nonce, data.numel())
        r.data = data
        rid = ctypes.c_uint64()
        check(lib().frag_server_submit_protect(self._h.ptr, plan.handle, nonce, data.data_ptr(), data.numel(),
                                               _stream(None), ctypes.byref(rid)))
        r.id = rid.value
        return r

    def submit_recover(self, private: torch.Tensor, public: torch.Tensor, nbytes: int, nonce: int,
                       plan: Optional[Plan] = None) -> Request:
        plan = plan or self.default_plan
        r = Request(self._h, "recover", plan, nonce, nbytes)
        r.private, r.public = private, public  # inputs, kept alive until done
        rid = ctypes.c_uint64()
        check(lib().frag_server_submit_recover(self._h.ptr, plan.handle, nonce, private.data_ptr(),
                                               public.data_ptr(), nbytes, _stream(None), ctypes.byref(rid)))
        r.id = rid.value
        return r

    @contextlib.contextmanager
    def held(self):
        """Admit nothing while the block runs: the requests submitted inside
        it wait and are admitted together when it ends (in arrival order,
        within the memory budget)."""
        check(lib().frag_server_hold(self._h.ptr, 1))
        try:
            yield self
        finally:
            check(lib().frag_server_hold(self._h.ptr, 0))

    @property
    def launches(self) -> int:
        n = ctypes.c_uint64()
        check(lib().frag_server_stats(self._h.ptr, ctypes.byref(n), None, None, None))
        return n.value

    def check(self) -> None:
        """Raise if a kernel of the server's launches reported an error (the
        device error word is read once every group in flight has finished)."""
        check(lib().frag_server_check(self._h.ptr))

    def close(self) -> None:
        """Finish every submitted request, then stop the scheduler (results
        stay valid until released)."""
        if not self._closed:
            self._closed = True
            check(lib().frag_server_stop(self._h.ptr))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
