// sha2.cuh -- SHA-256 and SHA-512 (FIPS 180-4) of one padded message block,
// one lane each, and the keyed protection of a block's packed public records
// (Sec. 5.2.1: a bit sequence from SHA-256 of the block's private fragment
// and the key is XORed into its first public and protected fragment, one
// from SHA-512 of that protected fragment and the key into its second).
//
// Hash inputs per 8 x 8 block idx (blocks row-major): key (16 bytes) ||
// nonce (8 bytes, big-endian) || idx (8 bytes, big-endian) || record, where
// the record is the block's 5 plaintext A bytes (SHA-256, 37 bytes) or its
// 124 protected B bits in 16 bytes (SHA-512, 48 bytes); both messages fit
// one block, so the padding is fixed.  Digest bit i (bit i % 8 of byte
// i / 8) masks record bit i: with the records held as little-endian words
// (pack_bits.cuh), record word q takes the byte-swapped digest word q.
#pragma once

#include <cstdint>

#include "sha2_constants.cuh"

namespace frag {
namespace sha {

__device__ __forceinline__ uint32_t rotr(uint32_t x, int n) { return __funnelshift_r(x, x, n); }

__device__ __forceinline__ uint64_t rotr64(uint64_t x, int n)
{
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    uint32_t rl, rh;
    if (n < 32) {
        rl = __funnelshift_r(lo, hi, n);
        rh = __funnelshift_r(hi, lo, n);
    } else { // the halves swapped, then n - 32 more
        rl = __funnelshift_r(hi, lo, n - 32);
        rh = __funnelshift_r(lo, hi, n - 32);
    }
    return ((uint64_t)rh << 32) | rl;
}

__device__ __forceinline__ uint32_t bswap(uint32_t x) { return __byte_perm(x, 0u, 0x0123); }

// digest h of the one padded block m (the schedule is built in m)
__device__ __forceinline__ void sha256_block(uint32_t (&m)[16], uint32_t (&h)[8])
{
    uint32_t a = kSha256H[0], b = kSha256H[1], c = kSha256H[2], d = kSha256H[3];
    uint32_t e = kSha256H[4], f = kSha256H[5], g = kSha256H[6], k = kSha256H[7];
#pragma unroll
    for (int t = 0; t < 64; ++t) {
        if (t >= 16) {
            const uint32_t x = m[(t - 15) & 15], y = m[(t - 2) & 15];
            m[t & 15] += (rotr(x, 7) ^ rotr(x, 18) ^ (x >> 3)) + m[(t - 7) & 15] +
                         (rotr(y, 17) ^ rotr(y, 19) ^ (y >> 10));
        }
        const uint32_t t1 = k + (rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25)) + ((e & f) ^ (~e & g)) + kSha256K[t] +
                            m[t & 15];
        const uint32_t t2 = (rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22)) + ((a & b) ^ (a & c) ^ (b & c));
        k = g;
        g = f;
        f = e;
        e = d + t1;
        d = c;
        c = b;
        b = a;
        a = t1 + t2;
    }
    h[0] = kSha256H[0] + a;
    h[1] = kSha256H[1] + b;
    h[2] = kSha256H[2] + c;
    h[3] = kSha256H[3] + d;
    h[4] = kSha256H[4] + e;
    h[5] = kSha256H[5] + f;
    h[6] = kSha256H[6] + g;
    h[7] = kSha256H[7] + k;
}

__device__ __forceinline__ void sha512_block(uint64_t (&m)[16], uint64_t (&h)[8])
{
    uint64_t a = kSha512H[0], b = kSha512H[1], c = kSha512H[2], d = kSha512H[3];
    uint64_t e = kSha512H[4], f = kSha512H[5], g = kSha512H[6], k = kSha512H[7];
#pragma unroll
    for (int t = 0; t < 80; ++t) {
        if (t >= 16) {
            const uint64_t x = m[(t - 15) & 15], y = m[(t - 2) & 15];
            m[t & 15] += (rotr64(x, 1) ^ rotr64(x, 8) ^ (x >> 7)) + m[(t - 7) & 15] +
                         (rotr64(y, 19) ^ rotr64(y, 61) ^ (y >> 6));
        }
        const uint64_t t1 = k + (rotr64(e, 14) ^ rotr64(e, 18) ^ rotr64(e, 41)) + ((e & f) ^ (~e & g)) +
                            kSha512K[t] + m[t & 15];
        const uint64_t t2 = (rotr64(a, 28) ^ rotr64(a, 34) ^ rotr64(a, 39)) + ((a & b) ^ (a & c) ^ (b & c));
        k = g;
        g = f;
        f = e;
        e = d + t1;
        d = c;
        c = b;
        b = a;
        a = t1 + t2;
    }
    h[0] = kSha512H[0] + a;
    h[1] = kSha512H[1] + b;
    h[2] = kSha512H[2] + c;
    h[3] = kSha512H[3] + d;
    h[4] = kSha512H[4] + e;
    h[5] = kSha512H[5] + f;
    h[6] = kSha512H[6] + g;
    h[7] = kSha512H[7] + k;
}

// B ^= the first 124 bits of SHA-256(key || nonce || idx || A record)
__device__ __forceinline__ void mask_b(const uint32_t (&key)[4], uint64_t nonce, uint64_t idx,
                                       const uint32_t (&ra)[2], uint32_t (&rb)[4])
{
    uint32_t m[16], h[8];
    m[0] = key[0];
    m[1] = key[1];
    m[2] = key[2];
    m[3] = key[3];
    m[4] = (uint32_t)(nonce >> 32);
    m[5] = (uint32_t)nonce;
    m[6] = (uint32_t)(idx >> 32);
    m[7] = (uint32_t)idx;
    m[8] = bswap(ra[0]);
    m[9] = (ra[1] << 24) | 0x00800000u; // A's fifth byte, then the padding bit
#pragma unroll
    for (int i = 10; i < 15; ++i)
        m[i] = 0u;
    m[15] = 37u * 8u;
    sha256_block(m, h);
    rb[0] ^= bswap(h[0]);
    rb[1] ^= bswap(h[1]);
    rb[2] ^= bswap(h[2]);
    rb[3] ^= bswap(h[3]) & 0x0fffffffu; // 124 = 96 + 28 bits
}

// C ^= the first 480 bits of SHA-512(key || nonce || idx || B' record)
__device__ __forceinline__ void mask_c(const uint32_t (&key)[4], uint64_t nonce, uint64_t idx,
                                       const uint32_t (&rb_protected)[4], uint32_t (&rc)[15])
{
    uint64_t m[16], h[8];
    m[0] = ((uint64_t)key[0] << 32) | key[1];
    m[1] = ((uint64_t)key[2] << 32) | key[3];
    m[2] = nonce;
    m[3] = idx;
    m[4] = ((uint64_t)bswap(rb_protected[0]) << 32) | bswap(rb_protected[1]);
    m[5] = ((uint64_t)bswap(rb_protected[2]) << 32) | bswap(rb_protected[3]);
    m[6] = 0x8000000000000000ull;
#pragma unroll
    for (int i = 7; i < 15; ++i)
        m[i] = 0ull;
    m[15] = 48ull * 8ull;
    sha512_block(m, h);
#pragma unroll
    for (int q = 0; q < 15; ++q)
        rc[q] ^= bswap((uint32_t)(h[q >> 1] >> ((q & 1) ? 0 : 32)));
}

} // namespace sha
} // namespace frag
