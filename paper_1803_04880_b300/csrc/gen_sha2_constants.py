"""Writes sha2_constants.cuh: the SHA-256 / SHA-512 round constants and
initial hash values of FIPS 180-4, derived from their definitions (the
leading fraction bits of the cube roots of the first 64 / 80 primes and of
the square roots of the first 8), by exact integer arithmetic.

    python gen_sha2_constants.py            # rewrite the header beside this file
    python gen_sha2_constants.py --check    # exit 1 if the header differs
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "sha2_constants.cuh")


def first_primes(count):
    found = []
    cand = 2
    while len(found) < count:
        if all(cand % p for p in found if p * p <= cand):
            found.append(cand)
        cand += 1
    return found


def floor_cbrt(a):
    """Largest r with r ** 3 <= a (bisection)."""
    lo, hi = 0, 1 << (a.bit_length() // 3 + 2)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if mid ** 3 <= a:
            lo = mid
        else:
            hi = mid
    return lo


def fraction_bits(p, root, bits):
    scaled = p << (root * bits)
    r = math.isqrt(scaled) if root == 2 else floor_cbrt(scaled)
    return r % (1 << bits)


def table(name, ctype, values, digits, per_line):
    lines = ["__constant__ %s %s[%d] = {" % (ctype, name, len(values))]
    suffix = "ull" if digits == 16 else "u"
    for i in range(0, len(values), per_line):
        chunk = ", ".join("0x%0*x%s" % (digits, v, suffix) for v in values[i:i + per_line])
        lines.append("    " + chunk + ",")
    lines.append("};")
    return "\n".join(lines)


def render():
    primes = first_primes(80)
    parts = [
        "// sha2_constants.cuh -- written by gen_sha2_constants.py; do not edit.",
        "// FIPS 180-4 constants: K = leading fraction bits of the cube roots of",
        "// the first 64 (SHA-256) / 80 (SHA-512) primes, H0 = those of the square",
        "// roots of the first 8 primes.",
        "#pragma once",
        "",
        "#include <cstdint>",
        "",
        "namespace frag {",
        "namespace sha {",
        "",
        table("kSha256K", "uint32_t", [fraction_bits(p, 3, 32) for p in primes[:64]], 8, 8),
        table("kSha256H", "uint32_t", [fraction_bits(p, 2, 32) for p in primes[:8]], 8, 8),
        table("kSha512K", "uint64_t", [fraction_bits(p, 3, 64) for p in primes[:80]], 16, 4),
        table("kSha512H", "uint64_t", [fraction_bits(p, 2, 64) for p in primes[:8]], 16, 4),
        "",
        "} // namespace sha",
        "} // namespace frag",
        "",
    ]
    return "\n".join(parts)


if __name__ == "__main__":
    text = render()
    if "--check" in sys.argv:
        with open(HEADER) as f:
            sys.exit(0 if f.read() == text else 1)
    with open(HEADER, "w") as f:
        f.write(text)
