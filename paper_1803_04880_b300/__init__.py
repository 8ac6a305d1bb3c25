"""Python binding of libfrag (include/frag.h): agnostic fragmentation of bytes
with a reversible integer LeGall 5/3 wavelet and AES-128-CTR on the private
LL band (Chapter 5 of arXiv 1803.04880), on one B300.

This module only marshals arguments: every step of protect / recover runs in
the CUDA kernels of libfrag.so.  PyTorch supplies device memory and streams.
There is no CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence, Tuple

_HERE = os.path.dirname(os.path.abspath(__file__))
# FRAG_LIBRARY selects another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("FRAG_LIBRARY") or os.path.join(_HERE, "libfrag.so")

FRAG_OK, FRAG_EINVAL, FRAG_EUNSUPPORTED, FRAG_ENOMEM, FRAG_ECUDA, FRAG_ETIMEOUT, FRAG_EDEVICE = range(7)
STATUS_NAMES = {0: "FRAG_OK", 1: "FRAG_EINVAL", 2: "FRAG_EUNSUPPORTED", 3: "FRAG_ENOMEM",
                4: "FRAG_ECUDA", 5: "FRAG_ETIMEOUT", 6: "FRAG_EDEVICE"}

# every symbol include/frag.h declares
EXPORTS = [
    "frag_abi_version", "frag_plan_create", "frag_plan_destroy", "frag_plan_sizes",
    "frag_plan_set_schedule", "frag_plan_get_schedule", "frag_plan_set_path", "frag_plan_get_path",
    "frag_plan_set_block", "frag_plan_get_block", "frag_plan_set_packed", "frag_plan_get_packed",
    "frag_plan_fragment_sizes", "frag_plan_set_protect_public", "frag_plan_get_protect_public",
    "frag_key_create", "frag_key_destroy",
    "frag_protect", "frag_recover", "frag_aes128_ctr", "frag_aes128_ctr_bitsliced", "frag_protect_host",
    "frag_recover_host",
    "frag_protect_batch", "frag_recover_batch", "frag_batch_create_protect",
    "frag_batch_create_recover", "frag_batch_run", "frag_batch_destroy", "frag_batch_info",
    "frag_batch_set_timing", "frag_batch_launch_times",
    "frag_get_error", "frag_check_wait_timeout", "frag_check_box_wait_timeout",
    "frag_sync_status", "frag_protect_batch_noalloc", "frag_noalloc_sync_status",
    "frag_server_create", "frag_server_stop", "frag_server_destroy", "frag_server_submit_protect",
    "frag_server_submit_recover", "frag_server_wait", "frag_server_release", "frag_server_hold",
    "frag_server_stats", "frag_server_check",
]


class FragError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


class frag_item(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("nonce", ctypes.c_uint64),
                ("nbytes", ctypes.c_uint64), ("d_in", ctypes.c_void_p),
                ("d_private", ctypes.c_void_p), ("d_public", ctypes.c_void_p)]


class frag_request_info(ctypes.Structure):
    _fields_ = [("done", ctypes.c_uint32), ("status", ctypes.c_int32), ("d_private", ctypes.c_void_p),
                ("d_public", ctypes.c_void_p), ("private_bytes", ctypes.c_uint64),
                ("public_bytes", ctypes.c_uint64), ("d_out", ctypes.c_void_p), ("nbytes", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double)]


class frag_ritem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("nonce", ctypes.c_uint64),
                ("nbytes", ctypes.c_uint64), ("d_private", ctypes.c_void_p),
                ("d_public", ctypes.c_void_p), ("d_out", ctypes.c_void_p)]


_lib = None


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """The loaded libfrag.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfrag.so is missing: build it with "
                           "paper_1803_04880_b300.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "frag_abi_version": ([], ctypes.c_int),
        "frag_plan_create": ([ctypes.POINTER(vp), u32, u32, ctypes.c_int], ctypes.c_int),
        "frag_plan_destroy": ([vp], ctypes.c_int),
        "frag_plan_sizes": ([vp, u64, ctypes.POINTER(u32), ctypes.POINTER(u64),
                             ctypes.POINTER(u64)], ctypes.c_int),
        "frag_plan_set_schedule": ([vp, u32, u32], ctypes.c_int),
        "frag_plan_get_schedule": ([vp, ctypes.POINTER(u32), ctypes.POINTER(u32)], ctypes.c_int),
        "frag_plan_set_path": ([vp, ctypes.c_int], ctypes.c_int),
        "frag_plan_set_block": ([vp, u32], ctypes.c_int),
        "frag_plan_get_block": ([vp, ctypes.POINTER(u32)], ctypes.c_int),
        "frag_plan_set_packed": ([vp, u32], ctypes.c_int),
        "frag_plan_get_packed": ([vp, ctypes.POINTER(u32)], ctypes.c_int),
        "frag_plan_fragment_sizes": ([vp, u64, ctypes.POINTER(u64)], ctypes.c_int),
        "frag_plan_set_protect_public": ([vp, u32], ctypes.c_int),
        "frag_plan_get_protect_public": ([vp, ctypes.POINTER(u32)], ctypes.c_int),
        "frag_plan_get_path": ([vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "frag_key_create": ([ctypes.POINTER(vp), ctypes.c_char_p], ctypes.c_int),
        "frag_key_destroy": ([vp], ctypes.c_int),
        "frag_protect": ([vp, vp, u64, vp, u64, vp, vp, vp], ctypes.c_int),
        "frag_recover": ([vp, vp, u64, vp, vp, u64, vp, vp], ctypes.c_int),
        "frag_aes128_ctr": ([vp, u64, vp, vp, u64, vp], ctypes.c_int),
        "frag_aes128_ctr_bitsliced": ([vp, u64, vp, vp, u64, vp], ctypes.c_int),
        "frag_protect_host": ([vp, vp, u64, vp, u64, vp, vp, vp], ctypes.c_int),
        "frag_recover_host": ([vp, vp, u64, vp, vp, u64, vp, vp], ctypes.c_int),
        "frag_protect_batch": ([ctypes.POINTER(frag_item), u32, vp, vp], ctypes.c_int),
        "frag_recover_batch": ([ctypes.POINTER(frag_ritem), u32, vp, vp], ctypes.c_int),
        "frag_batch_create_protect": ([ctypes.POINTER(vp), ctypes.POINTER(frag_item), u32],
                                      ctypes.c_int),
        "frag_batch_create_recover": ([ctypes.POINTER(vp), ctypes.POINTER(frag_ritem), u32],
                                      ctypes.c_int),
        "frag_batch_run": ([vp, vp, vp], ctypes.c_int),
        "frag_batch_destroy": ([vp], ctypes.c_int),
        "frag_batch_info": ([vp, ctypes.POINTER(u32), ctypes.POINTER(u64)], ctypes.c_int),
        "frag_batch_set_timing": ([vp, ctypes.c_int], ctypes.c_int),
        "frag_batch_launch_times": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32)],
                                    ctypes.c_int),
        "frag_get_error": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "frag_sync_status": ([vp], ctypes.c_int),
        "frag_check_wait_timeout": ([u32, vp], ctypes.c_int),
        "frag_check_box_wait_timeout": ([u32, vp], ctypes.c_int),
        "frag_protect_batch_noalloc": ([ctypes.POINTER(frag_item), u32, ctypes.c_char_p, vp],
                                       ctypes.c_int),
        "frag_noalloc_sync_status": ([vp], ctypes.c_int),
        "frag_server_create": ([ctypes.POINTER(vp), vp, u64, u32, u32], ctypes.c_int),
        "frag_server_stop": ([vp], ctypes.c_int),
        "frag_server_destroy": ([vp], ctypes.c_int),
        "frag_server_submit_protect": ([vp, vp, u64, vp, u64, vp, ctypes.POINTER(u64)], ctypes.c_int),
        "frag_server_submit_recover": ([vp, vp, u64, vp, vp, u64, vp, ctypes.POINTER(u64)], ctypes.c_int),
        "frag_server_wait": ([vp, u64, ctypes.c_double, ctypes.POINTER(frag_request_info)], ctypes.c_int),
        "frag_server_release": ([vp, u64, vp], ctypes.c_int),
        "frag_server_hold": ([vp, ctypes.c_int], ctypes.c_int),
        "frag_server_stats": ([vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u32),
                               ctypes.POINTER(u32)], ctypes.c_int),
        "frag_server_check": ([vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib().frag_get_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(status: int) -> None:
    if status != FRAG_OK:
        raise FragError(status, last_error())


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _ptr(t) -> int:
    return t.data_ptr()


class Plan:
    """Matrix width and number of levels (Sec. 5.2.1 / 5.1.1)."""

    def __init__(self, width: int, levels: int):
        h = ctypes.c_void_p()
        check(lib().frag_plan_create(ctypes.byref(h), width, levels, 0))
        self._h = h
        self.width, self.levels = width, levels

    @property
    def handle(self):
        return self._h

    def sizes(self, nbytes: int) -> Tuple[int, int, int]:
        H, pb, ub = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().frag_plan_sizes(self._h, nbytes, ctypes.byref(H), ctypes.byref(pb),
                                    ctypes.byref(ub)))
        return H.value, pb.value, ub.value

    def set_schedule(self, seg_rows: int = 0, ctas: int = 0) -> None:
        """Rows per work unit and grid cap of the streaming kernel (0 = auto)."""
        check(lib().frag_plan_set_schedule(self._h, seg_rows, ctas))

    def schedule(self) -> Tuple[int, int]:
        a, b = ctypes.c_uint32(), ctypes.c_uint32()
        check(lib().frag_plan_get_schedule(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    PATH_AUTO = 0    # levels 1..min(L, 3) fused in one pass where alignment allows
    PATH_LEVELS = 1  # every level in the dependency-ordered kernel
    PATH_FUSED_CIPHER = 2  # AUTO, with LL_L enciphered inside the fused pass that reaches it

    def set_path(self, path: int) -> None:
        """Kernels that run the levels (PATH_AUTO, PATH_LEVELS or
        PATH_FUSED_CIPHER); results do
        not depend on it."""
        check(lib().frag_plan_set_path(self._h, path))

    def path(self) -> int:
        v = ctypes.c_int()
        check(lib().frag_plan_get_path(self._h, ctypes.byref(v)))
        return v.value

    def set_block(self, block: int) -> None:
        """Block mode: every block x block block transformed on its own
        (0: the whole matrix; the CUDA path runs 8 x 8 blocks)."""
        check(lib().frag_plan_set_block(self._h, block))

    def block(self) -> int:
        v = ctypes.c_uint32()
        check(lib().frag_plan_get_block(self._h, ctypes.byref(v)))
        return v.value

    def set_packed(self, packed: bool) -> None:
        """The thesis's packed three fragments (8 x 8 blocks, two levels):
        private A (40 bits a block), public B (124) then C (480)."""
        check(lib().frag_plan_set_packed(self._h, 1 if packed else 0))

    def packed(self) -> bool:
        v = ctypes.c_uint32()
        check(lib().frag_plan_get_packed(self._h, ctypes.byref(v)))
        return bool(v.value)

    def set_protect_public(self, on: bool) -> None:
        """Packed plans: protect B and C with the keyed SHA-256 / SHA-512
        bit sequences of each block (Sec. 5.2.1)."""
        check(lib().frag_plan_set_protect_public(self._h, 1 if on else 0))

    def protect_public(self) -> bool:
        v = ctypes.c_uint32()
        check(lib().frag_plan_get_protect_public(self._h, ctypes.byref(v)))
        return bool(v.value)

    def fragment_sizes(self, nbytes: int) -> Tuple[int, int, int]:
        """(private, first public, second public) bytes of nbytes bytes."""
        v = (ctypes.c_uint64 * 3)()
        check(lib().frag_plan_fragment_sizes(self._h, nbytes, v))
        return v[0], v[1], v[2]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.frag_plan_destroy(self._h)
            self._h = None


class Key:
    """AES-128 key with round keys resident on the device."""

    def __init__(self, key: bytes):
        key = bytes(key)
        if len(key) != 16:
            raise ValueError("AES-128 key must be 16 bytes")
        h = ctypes.c_void_p()
        check(lib().frag_key_create(ctypes.byref(h), key))
        self._h = h

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.frag_key_destroy(self._h)
            self._h = None


def _empty(n: int, device):
    import torch
    return torch.empty(max(n, 0), dtype=torch.uint8, device=device)


def protect(plan: Plan, key: Key, nonce: int, data, nbytes: Optional[int] = None,
            private=None, public=None, stream=None):
    """Device bytes -> (private, public) uint8 device tensors."""
    n = data.numel() * data.element_size() if nbytes is None else nbytes
    if private is None or public is None:
        _, pb, ub = plan.sizes(n)
        if private is None:
            private = _empty(pb, data.device)
        if public is None:
            public = _empty(ub, data.device)
    check(lib().frag_protect(plan.handle, key.handle, nonce, _ptr(data), n, _ptr(private),
                             _ptr(public), _stream(stream)))
    return private, public


def recover(plan: Plan, key: Key, nonce: int, private, public, nbytes: int, out=None,
            stream=None):
    """(private, public) device tensors -> nbytes recovered bytes (device tensor)."""
    if out is None:
        out = _empty(nbytes, private.device)
    check(lib().frag_recover(plan.handle, key.handle, nonce, _ptr(private), _ptr(public),
                             nbytes, _ptr(out), _stream(stream)))
    return out


def aes_ctr(key: Key, nonce: int, data, out=None, stream=None):
    """Full-buffer AES-128-CTR of a device uint8 tensor (the comparator for
    the selective method; its own inverse): returns out (in place when out is
    data)."""
    if out is None:
        out = _empty(data.numel(), data.device)
    check(lib().frag_aes128_ctr(key.handle, nonce, _ptr(data), _ptr(out), data.numel(),
                                _stream(stream)))
    return out


def aes_ctr_bitsliced(key: Key, nonce: int, data, out=None, stream=None):
    """aes_ctr computed by the bitsliced kernel (the measured alternative to
    the table form); byte-identical output."""
    if out is None:
        out = _empty(data.numel(), data.device)
    check(lib().frag_aes128_ctr_bitsliced(key.handle, nonce, _ptr(data), _ptr(out), data.numel(),
                                          _stream(stream)))
    return out


def protect_host(plan: Plan, key: Key, nonce: int, data, private=None, public=None,
                 stream=None):
    """Host bytes (numpy uint8 or pinned torch CPU tensor) -> host fragments."""
    import numpy as np
    import torch
    if isinstance(data, np.ndarray):
        data = torch.from_numpy(np.ascontiguousarray(data).reshape(-1))
    n = data.numel()
    _, pb, ub = plan.sizes(n)
    if private is None:
        private = torch.empty(pb, dtype=torch.uint8)
    if public is None:
        public = torch.empty(ub, dtype=torch.uint8)
    check(lib().frag_protect_host(plan.handle, key.handle, nonce, _ptr(data), n, _ptr(private),
                                  _ptr(public), _stream(stream)))
    return private, public


def recover_host(plan: Plan, key: Key, nonce: int, private, public, nbytes: int, out=None,
                 stream=None):
    import numpy as np
    import torch
    if isinstance(private, np.ndarray):
        private = torch.from_numpy(np.ascontiguousarray(private))
    if isinstance(public, np.ndarray):
        public = torch.from_numpy(np.ascontiguousarray(public))
    if out is None:
        out = torch.empty(nbytes, dtype=torch.uint8)
    check(lib().frag_recover_host(plan.handle, key.handle, nonce, _ptr(private), _ptr(public),
                                  nbytes, _ptr(out), _stream(stream)))
    return out


def _items(entries, kind):
    arr = (kind * max(len(entries), 1))()
    for i, e in enumerate(entries):
        plan, nonce, nbytes, a, b, c = e
        arr[i] = kind(plan.handle, nonce, nbytes, _ptr(a), _ptr(b), _ptr(c))
    return arr


def protect_batch(entries: Sequence[tuple], key: Key, stream=None) -> None:
    """entries: (plan, nonce, nbytes, d_in, d_private, d_public) per buffer."""
    arr = _items(entries, frag_item)
    check(lib().frag_protect_batch(arr, len(entries), key.handle, _stream(stream)))


def recover_batch(entries: Sequence[tuple], key: Key, stream=None) -> None:
    """entries: (plan, nonce, nbytes, d_private, d_public, d_out) per buffer."""
    arr = _items(entries, frag_ritem)
    check(lib().frag_recover_batch(arr, len(entries), key.handle, _stream(stream)))


class Batch:
    """A resident work queue (frag_batch_create_*); run() launches it."""

    def __init__(self, entries: Sequence[tuple], protect: bool = True):
        h = ctypes.c_void_p()
        if protect:
            check(lib().frag_batch_create_protect(ctypes.byref(h), _items(entries, frag_item),
                                                  len(entries)))
        else:
            check(lib().frag_batch_create_recover(ctypes.byref(h), _items(entries, frag_ritem),
                                                  len(entries)))
        self._h = h
        self._keep = list(entries)  # the buffers must outlive the batch

    def run(self, key: Key, stream=None) -> None:
        check(lib().frag_batch_run(self._h, key.handle, _stream(stream)))

    def info(self) -> Tuple[int, int]:
        """(kernel launches per run, device bytes the batch holds)."""
        n, b = ctypes.c_uint32(), ctypes.c_uint64()
        check(lib().frag_batch_info(self._h, ctypes.byref(n), ctypes.byref(b)))
        return n.value, b.value

    @property
    def launches(self) -> int:
        return self.info()[0]

    KERNEL_KINDS = ("fused", "levels", "cipher", "blocks", "fused_low")

    def set_timing(self, enable: bool = True) -> None:
        """Record a CUDA event pair around each kernel launch of run()."""
        check(lib().frag_batch_set_timing(self._h, 1 if enable else 0))

    def launch_times(self) -> dict:
        """{kind: (total ms, launches)} over the timed runs since the last
        call (waits for their events)."""
        ms = (ctypes.c_double * len(self.KERNEL_KINDS))()
        n = (ctypes.c_uint32 * len(self.KERNEL_KINDS))()
        check(lib().frag_batch_launch_times(self._h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(self.KERNEL_KINDS)}

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.frag_batch_destroy(self._h)
            self._h = None


def sync_status(stream=None) -> None:
    check(lib().frag_sync_status(_stream(stream)))


def check_wait_timeout(polls: int = 2000, stream=None) -> None:
    """Enqueue one bounded wait that is bound to run out (see frag.h)."""
    check(lib().frag_check_wait_timeout(polls, _stream(stream)))


def check_box_wait_timeout(polls: int = 2000, stream=None) -> None:
    """Enqueue the box loads' bounded wait on a barrier nothing completes
    (see frag.h)."""
    check(lib().frag_check_box_wait_timeout(polls, _stream(stream)))
