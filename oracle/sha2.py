"""SHA-256 and SHA-512 (FIPS 180-4), plain Python, for the oracle's
protection of the public fragments (Sec. 5.2.1: a bit sequence from SHA-256
of the private fragment and the key protects the first public fragment, one
from SHA-512 of the first protected fragment and the key the second).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/.  The round constants and
initial hash values are not typed in: they are computed here from their
definitions in FIPS 180-4 (the first 32 or 64 bits of the fractional parts of
the cube roots of the first 64 / 80 primes, and of the square roots of the
first 8 primes), with exact integer roots.  Pinned by tests/test_oracle_sha.py
against Python's hashlib.
"""
from __future__ import annotations


def _primes(count):
    out, p = [], 2
    while len(out) < count:
        if all(p % q for q in out if q * q <= p):
            out.append(p)
        p += 1
    return out


def _iroot(a, n):
    """floor(a ** (1 / n)) for integers a >= 0, n >= 2 (Newton's method)."""
    if a < 2:
        return a
    x = 1 << ((a.bit_length() + n - 1) // n)  # above the root
    while True:
        y = ((n - 1) * x + a // x ** (n - 1)) // n
        if y >= x:
            return x
        x = y


def _frac_bits(p, n, bits):
    """The first `bits` bits of the fractional part of p ** (1 / n)."""
    return _iroot(p << (n * bits), n) & ((1 << bits) - 1)


_P = _primes(80)
K256 = [_frac_bits(p, 3, 32) for p in _P[:64]]
H256 = [_frac_bits(p, 2, 32) for p in _P[:8]]
K512 = [_frac_bits(p, 3, 64) for p in _P[:80]]
H512 = [_frac_bits(p, 2, 64) for p in _P[:8]]


def _rotr(x, n, w):
    return ((x >> n) | (x << (w - n))) & ((1 << w) - 1)


def _pad(msg: bytes, block: int, lenbytes: int) -> bytes:
    """Append 1, zeros and the message length in bits (big-endian)."""
    ml = len(msg) * 8
    m = msg + b"\x80"
    m += b"\x00" * ((block - lenbytes - len(m) % block) % block)
    return m + ml.to_bytes(lenbytes, "big")


def sha256(msg: bytes) -> bytes:
    M = 0xFFFFFFFF
    h = list(H256)
    m = _pad(bytes(msg), 64, 8)
    for off in range(0, len(m), 64):
        w = [int.from_bytes(m[off + 4 * t:off + 4 * t + 4], "big") for t in range(16)]
        for t in range(16, 64):
            s0 = _rotr(w[t - 15], 7, 32) ^ _rotr(w[t - 15], 18, 32) ^ (w[t - 15] >> 3)
            s1 = _rotr(w[t - 2], 17, 32) ^ _rotr(w[t - 2], 19, 32) ^ (w[t - 2] >> 10)
            w.append((w[t - 16] + s0 + w[t - 7] + s1) & M)
        a, b, c, d, e, f, g, hh = h
        for t in range(64):
            S1 = _rotr(e, 6, 32) ^ _rotr(e, 11, 32) ^ _rotr(e, 25, 32)
            ch = (e & f) ^ (~e & g)
            t1 = (hh + S1 + ch + K256[t] + w[t]) & M
            S0 = _rotr(a, 2, 32) ^ _rotr(a, 13, 32) ^ _rotr(a, 22, 32)
            maj = (a & b) ^ (a & c) ^ (b & c)
            t2 = (S0 + maj) & M
            a, b, c, d, e, f, g, hh = (t1 + t2) & M, a, b, c, (d + t1) & M, e, f, g
        h = [(x + y) & M for x, y in zip(h, (a, b, c, d, e, f, g, hh))]
    return b"".join(x.to_bytes(4, "big") for x in h)


def sha512(msg: bytes) -> bytes:
    M = (1 << 64) - 1
    h = list(H512)
    m = _pad(bytes(msg), 128, 16)
    for off in range(0, len(m), 128):
        w = [int.from_bytes(m[off + 8 * t:off + 8 * t + 8], "big") for t in range(16)]
        for t in range(16, 80):
            s0 = _rotr(w[t - 15], 1, 64) ^ _rotr(w[t - 15], 8, 64) ^ (w[t - 15] >> 7)
            s1 = _rotr(w[t - 2], 19, 64) ^ _rotr(w[t - 2], 61, 64) ^ (w[t - 2] >> 6)
            w.append((w[t - 16] + s0 + w[t - 7] + s1) & M)
        a, b, c, d, e, f, g, hh = h
        for t in range(80):
            S1 = _rotr(e, 14, 64) ^ _rotr(e, 18, 64) ^ _rotr(e, 41, 64)
            ch = (e & f) ^ (~e & g & M)
            t1 = (hh + S1 + ch + K512[t] + w[t]) & M
            S0 = _rotr(a, 28, 64) ^ _rotr(a, 34, 64) ^ _rotr(a, 39, 64)
            maj = (a & b) ^ (a & c) ^ (b & c)
            t2 = (S0 + maj) & M
            a, b, c, d, e, f, g, hh = (t1 + t2) & M, a, b, c, (d + t1) & M, e, f, g
        h = [(x + y) & M for x, y in zip(h, (a, b, c, d, e, f, g, hh))]
    return b"".join(x.to_bytes(8, "big") for x in h)
