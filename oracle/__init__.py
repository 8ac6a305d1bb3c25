"""The oracle: plain single-threaded C statement of the Chapter 5 method
(LeGall 5/3 integer lifting, Eq. 5.1/5.2; dyadic 2-D decomposition, Sec. 5.1.1;
AES-128-CTR on the final LL band, Sec. 5.2.1), wrapped with ctypes, and the
keyed SHA-256 / SHA-512 protection of the packed public fragments (Sec. 5.2.1)
in plain Python on top of it (sha2.py).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are its only users.  The CUDA library never loads
it, and the two share no code.  Every function is pinned by
tests/test_oracle_*.py against the thesis's printed matrix A and F(4,4)
weights, its magnitude bounds, hand-worked examples, closed forms, invariants
and the FIPS-197 / SP 800-38A vectors; SHA-2 by FIPS 180-4's example and
hashlib.  Parity unpinned: the hash-input framing of protect_keyed /
recover_keyed / keyed_block_records (which bytes enter SHA-256 and SHA-512,
and how digest bits map onto record bits), which the thesis does not give;
tests/test_oracle_sha.py checks it only by a hashlib restatement and by the
scheme's properties (exact inverse, key sensitivity, identical blocks
protected differently, errors that stay in their block).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "frag_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no vectorisation flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_lift53_fwd_1d.argtypes = [_i32p, ctypes.c_int64, _i32p]
        lib.oracle_lift53_inv_1d.argtypes = [_i32p, ctypes.c_int64, _i32p]
        lib.oracle_dwt53_fwd_2d.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        lib.oracle_dwt53_inv_2d.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        lib.oracle_aes128_expand_key.argtypes = [_u8p, _u8p]
        lib.oracle_aes128_encrypt_block.argtypes = [_u8p, _u8p, _u8p]
        lib.oracle_aes128_ctr_xor.argtypes = [_u8p, ctypes.c_uint64, ctypes.c_uint64, _u8p,
                                              ctypes.c_uint64]
        lib.oracle_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u64p,
                                     _u64p, _u64p]
        lib.oracle_protect.argtypes = [_u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       _u8p, ctypes.c_uint64, _u8p, _u8p]
        lib.oracle_recover.argtypes = [_u8p, _u8p, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, _u8p, ctypes.c_uint64, _u8p]
        lib.oracle_block_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, _u64p, _u64p, _u64p]
        lib.oracle_protect_blocks.argtypes = [_u8p, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_uint32, _u8p,
                                              ctypes.c_uint64, _u8p, _u8p]
        lib.oracle_recover_blocks.argtypes = [_u8p, _u8p, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_uint32, _u8p,
                                              ctypes.c_uint64, _u8p]
        lib.oracle_packed_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint32, _u64p, _u64p,
                                            _u64p, _u64p]
        lib.oracle_protect_packed.argtypes = [_u8p, ctypes.c_uint64, ctypes.c_uint32, _u8p,
                                              ctypes.c_uint64, _u8p, _u8p, _u8p]
        lib.oracle_recover_packed.argtypes = [_u8p, _u8p, _u8p, ctypes.c_uint64, ctypes.c_uint32,
                                              _u8p, ctypes.c_uint64, _u8p]
        for f in ("oracle_dwt53_fwd_2d", "oracle_dwt53_inv_2d", "oracle_sizes", "oracle_protect",
                  "oracle_recover", "oracle_block_sizes", "oracle_protect_blocks",
                  "oracle_recover_blocks", "oracle_packed_sizes", "oracle_protect_packed",
                  "oracle_recover_packed"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _key(key) -> np.ndarray:
    k = np.frombuffer(bytes(key), dtype=np.uint8).copy()
    if k.size != 16:
        raise ValueError("AES-128 key must be 16 bytes")
    return k


def lift53_fwd_1d(x) -> np.ndarray:
    """Eq. 5.1/5.2 on one even-length signal; returns [s | d]."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    out = np.empty_like(x)
    _load().oracle_lift53_fwd_1d(_p(x, _i32p), x.size, _p(out, _i32p))
    return out


def lift53_inv_1d(sd) -> np.ndarray:
    sd = np.ascontiguousarray(sd, dtype=np.int32)
    out = np.empty_like(sd)
    _load().oracle_lift53_inv_1d(_p(sd, _i32p), sd.size, _p(out, _i32p))
    return out


def dwt53_fwd_2d(img, levels: int) -> np.ndarray:
    """L-level dyadic 2-D transform (rows first); Mallat layout, int32."""
    a = np.array(img, dtype=np.int32, order="C", copy=True)
    st = _load().oracle_dwt53_fwd_2d(_p(a, _i32p), a.shape[0], a.shape[1], levels)
    if st:
        raise RuntimeError("oracle_dwt53_fwd_2d failed: %d" % st)
    return a


def dwt53_inv_2d(coef, levels: int) -> np.ndarray:
    a = np.array(coef, dtype=np.int32, order="C", copy=True)
    st = _load().oracle_dwt53_inv_2d(_p(a, _i32p), a.shape[0], a.shape[1], levels)
    if st:
        raise RuntimeError("oracle_dwt53_inv_2d failed: %d" % st)
    return a


def aes128_expand_key(key) -> np.ndarray:
    k = _key(key)
    rk = np.empty(176, dtype=np.uint8)
    _load().oracle_aes128_expand_key(_p(k, _u8p), _p(rk, _u8p))
    return rk


def aes128_encrypt_block(key, block) -> bytes:
    rk = aes128_expand_key(key)
    b = np.frombuffer(bytes(block), dtype=np.uint8).copy()
    out = np.empty(16, dtype=np.uint8)
    _load().oracle_aes128_encrypt_block(_p(rk, _u8p), _p(b, _u8p), _p(out, _u8p))
    return out.tobytes()


def aes128_ctr_xor(key, nonce: int, first_block: int, data) -> bytes:
    k = _key(key)
    d = np.frombuffer(bytes(data), dtype=np.uint8).copy()
    _load().oracle_aes128_ctr_xor(_p(k, _u8p), nonce, first_block, _p(d, _u8p), d.size)
    return d.tobytes()


def sizes(n: int, width: int, levels: int, block: int = 0):
    """(H, private_bytes, public_bytes) for n input bytes; block > 0: the
    block mode with B x B blocks."""
    H, pb, ub = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    if block:
        st = _load().oracle_block_sizes(n, width, levels, block, ctypes.byref(H),
                                        ctypes.byref(pb), ctypes.byref(ub))
    else:
        st = _load().oracle_sizes(n, width, levels, ctypes.byref(H), ctypes.byref(pb),
                                  ctypes.byref(ub))
    if st:
        raise ValueError("invalid plan: width=%d levels=%d block=%d" % (width, levels, block))
    return H.value, pb.value, ub.value


def protect(data, width: int, levels: int, key, nonce: int, block: int = 0):
    """Bytes -> (private fragment, public fragment), both uint8 arrays;
    block > 0: every B x B block transformed as an image of its own."""
    buf = np.ascontiguousarray(np.frombuffer(data, dtype=np.uint8) if isinstance(data, (bytes, bytearray)) else data, dtype=np.uint8).reshape(-1)
    n = buf.size
    _, pb, ub = sizes(n, width, levels, block)
    priv = np.zeros(pb, dtype=np.uint8)
    pub = np.zeros(ub, dtype=np.uint8)
    k = _key(key)
    if block:
        st = _load().oracle_protect_blocks(_p(buf, _u8p), n, width, levels, block, _p(k, _u8p),
                                           nonce, _p(priv, _u8p), _p(pub, _u8p))
    else:
        st = _load().oracle_protect(_p(buf, _u8p), n, width, levels, _p(k, _u8p), nonce,
                                    _p(priv, _u8p), _p(pub, _u8p))
    if st:
        raise RuntimeError("oracle_protect failed: %d" % st)
    return priv, pub


def recover(priv, pub, n: int, width: int, levels: int, key, nonce: int,
            block: int = 0) -> np.ndarray:
    _, pb, ub = sizes(n, width, levels, block)
    priv = np.ascontiguousarray(priv, dtype=np.uint8).reshape(-1)
    pub = np.ascontiguousarray(pub, dtype=np.uint8).reshape(-1)
    if priv.size != pb or pub.size != ub:
        raise ValueError("fragment sizes do not match the plan")
    out = np.zeros(n, dtype=np.uint8)
    k = _key(key)
    if block:
        st = _load().oracle_recover_blocks(_p(priv, _u8p), _p(pub, _u8p), n, width, levels,
                                           block, _p(k, _u8p), nonce, _p(out, _u8p))
    else:
        st = _load().oracle_recover(_p(priv, _u8p), _p(pub, _u8p), n, width, levels,
                                    _p(k, _u8p), nonce, _p(out, _u8p))
    if st:
        raise RuntimeError("oracle_recover failed: %d" % st)
    return out


# -- the thesis's packed three fragments (8 x 8 blocks, two levels) ----------

def packed_sizes(n: int, width: int):
    """(H, A bytes, B bytes, C bytes): the private fragment (40 bits a
    block), the first public fragment (124 bits a block, every block row
    starting on a byte) and the second (480 bits a block)."""
    H, a, b, c = (ctypes.c_uint64() for _ in range(4))
    st = _load().oracle_packed_sizes(n, width, ctypes.byref(H), ctypes.byref(a), ctypes.byref(b),
                                     ctypes.byref(c))
    if st:
        raise ValueError("invalid width %d for 8 x 8 blocks" % width)
    return H.value, a.value, b.value, c.value


def protect_packed(data, width: int, key, nonce: int):
    """Bytes -> (private fragment A, public fragment B || C) in the packed
    storage, both uint8 arrays."""
    buf = np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
    n = buf.size
    _, sa, sb, sc = packed_sizes(n, width)
    a = np.zeros(sa, dtype=np.uint8)
    pub = np.zeros(sb + sc, dtype=np.uint8)
    b, c = pub[:sb], pub[sb:]
    k = _key(key)
    st = _load().oracle_protect_packed(_p(buf, _u8p), n, width, _p(k, _u8p), nonce, _p(a, _u8p),
                                       _p(b, _u8p), _p(c, _u8p))
    if st:
        raise RuntimeError("oracle_protect_packed failed: %d" % st)
    return a, pub


def recover_packed(a, pub, n: int, width: int, key, nonce: int) -> np.ndarray:
    _, sa, sb, sc = packed_sizes(n, width)
    a = np.ascontiguousarray(a, dtype=np.uint8).reshape(-1)
    pub = np.ascontiguousarray(pub, dtype=np.uint8).reshape(-1)
    if a.size != sa or pub.size != sb + sc:
        raise ValueError("fragment sizes do not match")
    b, c = np.ascontiguousarray(pub[:sb]), np.ascontiguousarray(pub[sb:])
    out = np.zeros(n, dtype=np.uint8)
    k = _key(key)
    st = _load().oracle_recover_packed(_p(a, _u8p), _p(b, _u8p), _p(c, _u8p), n, width,
                                       _p(k, _u8p), nonce, _p(out, _u8p))
    if st:
        raise RuntimeError("oracle_recover_packed failed: %d" % st)
    return out


# -- keyed protection of the public fragments (Sec. 5.2.1) ------------------
# Per 8 x 8 block (idx = bi * nbx + bj, blocks row-major):
#   H1 = SHA-256(key || nonce || idx || A record),  B' = B XOR H1 (124 bits)
#   H2 = SHA-512(key || nonce || idx || B' record), C' = C XOR H2 (480 bits)
# key: the 16 AES key bytes; nonce and idx: 8 bytes each, big-endian; the A
# record is its 5 plaintext bytes and the B' record its 124 bits in 16 bytes
# (the 4 top bits zero).  Digest bit i (bit i % 8 of byte i // 8) masks bit i
# of the record, records reading bits from the least significant bit of each
# byte as in the packed storage.  Recover takes H2 from the stored B' first,
# then H1 from the deciphered A.

_B_BITS = 124
_C_BITS = 480


def _digest_bits(digest: bytes, bits: int) -> int:
    return int.from_bytes(digest, "little") & ((1 << bits) - 1)


def _xor_public(pub: np.ndarray, plain_a: bytes, H: int, width: int, key, nonce: int,
                protect: bool) -> None:
    """Protect (B -> B', C -> C') or unprotect the public fragment in place."""
    from . import sha2
    k = bytes(_key(key))
    nbx, nby = width // 8, H // 8
    brow = (_B_BITS * nbx + 7) // 8
    sb = nby * brow
    mask_b = (1 << _B_BITS) - 1
    for bi in range(nby):
        row = int.from_bytes(pub[bi * brow:(bi + 1) * brow].tobytes(), "little")
        for bj in range(nbx):
            idx = bi * nbx + bj
            prefix = k + int(nonce).to_bytes(8, "big") + idx.to_bytes(8, "big")
            h1 = _digest_bits(sha2.sha256(prefix + plain_a[5 * idx:5 * idx + 5]), _B_BITS)
            b_stored = (row >> (_B_BITS * bj)) & mask_b
            b_prot = b_stored ^ h1 if protect else b_stored
            h2 = _digest_bits(sha2.sha512(prefix + b_prot.to_bytes(16, "little")), _C_BITS)
            off = sb + 60 * idx
            c = int.from_bytes(pub[off:off + 60].tobytes(), "little") ^ h2
            pub[off:off + 60] = np.frombuffer(c.to_bytes(60, "little"), dtype=np.uint8)
            row ^= h1 << (_B_BITS * bj)
        pub[bi * brow:(bi + 1) * brow] = np.frombuffer(row.to_bytes(brow, "little"), dtype=np.uint8)


def protect_keyed(data, width: int, key, nonce: int):
    """The packed three fragments with the public ones protected by the
    keyed hashes: (A enciphered, B' || C')."""
    n = np.asarray(data).size
    H, _, _, _ = packed_sizes(n, width)
    a, pub = protect_packed(data, width, key, nonce)
    if n:
        _xor_public(pub, aes128_ctr_xor(key, nonce, 0, a), H, width, key, nonce, True)
    return a, pub


def recover_keyed(a, pub, n: int, width: int, key, nonce: int) -> np.ndarray:
    H, sa, sb, sc = packed_sizes(n, width)
    a = np.ascontiguousarray(a, dtype=np.uint8).reshape(-1)
    pub = np.array(pub, dtype=np.uint8).reshape(-1)
    if a.size != sa or pub.size != sb + sc:
        raise ValueError("fragment sizes do not match")
    if n:
        _xor_public(pub, aes128_ctr_xor(key, nonce, 0, a), H, width, key, nonce, False)
    return recover_packed(a, pub, n, width, key, nonce)


def keyed_block_records(block, key, nonce: int, idx: int):
    """One 8 x 8 block's records as block idx of a keyed buffer: (A plaintext
    5 bytes, B' as a 124-bit int, C' as a 480-bit int).  Blocks are
    transformed on their own, so any block of a large buffer can be checked
    from its 64 bytes alone."""
    from . import sha2
    blk = np.ascontiguousarray(block, dtype=np.uint8).reshape(8, 8)
    a, pub = protect_packed(blk.reshape(-1), 8, key, nonce)
    a_plain = aes128_ctr_xor(key, nonce, 0, a)
    b = int.from_bytes(pub[:16].tobytes(), "little") & ((1 << _B_BITS) - 1)
    c = int.from_bytes(pub[16:76].tobytes(), "little")
    prefix = bytes(_key(key)) + int(nonce).to_bytes(8, "big") + int(idx).to_bytes(8, "big")
    b ^= _digest_bits(sha2.sha256(prefix + a_plain), _B_BITS)
    c ^= _digest_bits(sha2.sha512(prefix + b.to_bytes(16, "little")), _C_BITS)
    return a_plain, b, c
