"""The bitsliced AES's S-box circuit (csrc/aes_bs.cuh, Boyar and Peralta's
straight-line program with its XNOR gates as XORs) evaluated gate by gate on
all 256 inputs: with the affine constant 0x63 added back it is FIPS-197's
S-box, which this test builds from its definition (the multiplicative inverse
in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1, then the affine map of Sec. 5.1.1)
and pins to the standard's printed entries."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1803_04880_b300", "csrc", "aes_bs.cuh")


def _gf_mul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a = ((a << 1) ^ 0x11B) if a & 0x80 else a << 1
        b >>= 1
    return r


def _fips_sbox():
    inv = [0] * 256
    for a in range(1, 256):
        inv[a] = next(b for b in range(1, 256) if _gf_mul(a, b) == 1)
    out = []
    for x in range(256):
        b, s = inv[x], 0
        for i in range(8):
            bit = (b >> i) ^ (b >> ((i + 4) % 8)) ^ (b >> ((i + 5) % 8)) ^ (b >> ((i + 6) % 8)) ^ \
                (b >> ((i + 7) % 8)) ^ (0x63 >> i)
            s |= (bit & 1) << i
        out.append(s)
    return out


def _circuit():
    text = open(HDR).read()
    body = text.split("// circuit-begin")[1].split("// circuit-end")[0]
    gates = []
    for line in body.strip().splitlines():
        m = re.fullmatch(r"\s*(?:const uint32_t )?(\w+) = (\w+)(?: ([&^]) (\w+))?;\s*", line)
        assert m, line
        gates.append(m.groups())  # (lhs, a, None, None) is a plain copy
    return gates


def test_circuit_shape():
    g = [x for x in _circuit() if x[2]]
    assert sum(op == "&" for _, _, op, _ in g) == 34
    assert sum(op == "^" for _, _, op, _ in g) == 94
    assert len(g) == 128


def test_circuit_is_the_sbox_without_its_constant():
    S = _fips_sbox()
    # FIPS-197 Figure 7 entries
    assert (S[0x00], S[0x01], S[0x53], S[0xFF], S[0x10]) == (0x63, 0x7C, 0xED, 0x16, 0xCA)
    gates = _circuit()
    for x in range(256):
        env = {"U%d" % i: (x >> (7 - i)) & 1 for i in range(8)}
        for lhs, a, op, b in gates:
            env[lhs] = env[a] if op is None else (env[a] & env[b]) if op == "&" else (env[a] ^ env[b])
        y = sum(env["S%d" % i] << (7 - i) for i in range(8))
        assert y ^ 0x63 == S[x], hex(x)
