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

// One round on the working variables a..h with schedule word w and constant
// kt: d becomes the next e and h the next a; the caller rotates the names,
// so 8 calls in a row return to the same assignment.
__device__ __forceinline__ void round256(uint32_t a, uint32_t b, uint32_t c, uint32_t &d, uint32_t e,
                                         uint32_t f, uint32_t g, uint32_t &h, uint32_t kt, uint32_t w)
{
    const uint32_t t1 = h + (rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25)) + ((e & f) ^ (~e & g)) + kt + w;
    d += t1;
    h = t1 + (rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22)) + ((a & b) ^ (a & c) ^ (b & c));
}

__device__ __forceinline__ void round512(uint64_t a, uint64_t b, uint64_t c, uint64_t &d, uint64_t e,
                                         uint64_t f, uint64_t g, uint64_t &h, uint64_t kt, uint64_t w)
{
    const uint64_t t1 = h + (rotr64(e, 14) ^ rotr64(e, 18) ^ rotr64(e, 41)) + ((e & f) ^ (~e & g)) + kt + w;
    d += t1;
    h = t1 + (rotr64(a, 28) ^ rotr64(a, 34) ^ rotr64(a, 39)) + ((a & b) ^ (a & c) ^ (b & c));
}

__device__ __forceinline__ uint32_t s256_0(uint32_t x) { return rotr(x, 7) ^ rotr(x, 18) ^ (x >> 3); }
__device__ __forceinline__ uint32_t s256_1(uint32_t x) { return rotr(x, 17) ^ rotr(x, 19) ^ (x >> 10); }
__device__ __forceinline__ uint64_t s512_0(uint64_t x) { return rotr64(x, 1) ^ rotr64(x, 8) ^ (x >> 7); }
__device__ __forceinline__ uint64_t s512_1(uint64_t x) { return rotr64(x, 19) ^ rotr64(x, 61) ^ (x >> 6); }

// Eight rounds starting at round t0 + q0 with the names in their home order
// (a..h at rounds = 0 mod 8), words m[q0..q0+7]
__device__ __forceinline__ void sha256_8(const uint32_t (&m)[16], uint32_t (&v)[8], int t0, int q0)
{
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        round256(v[(8 - j) & 7], v[(9 - j) & 7], v[(10 - j) & 7], v[(11 - j) & 7], v[(12 - j) & 7],
                 v[(13 - j) & 7], v[(14 - j) & 7], v[(15 - j) & 7], kSha256K[t0 + q0 + j], m[q0 + j]);
    }
}

__device__ __forceinline__ void sha512_8(const uint64_t (&m)[16], uint64_t (&v)[8], int t0, int q0)
{
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        round512(v[(8 - j) & 7], v[(9 - j) & 7], v[(10 - j) & 7], v[(11 - j) & 7], v[(12 - j) & 7],
                 v[(13 - j) & 7], v[(14 - j) & 7], v[(15 - j) & 7], kSha512K[t0 + q0 + j], m[q0 + j]);
    }
}

// the next 16 schedule words in place of the last 16 (word q needs words
// q - 2 and q - 7 of the new 16 and q - 15, q - 16 of the old)
template <typename T, T (*S0)(T), T (*S1)(T)>
__device__ __forceinline__ void schedule16(T (&m)[16])
{
#pragma unroll
    for (int q = 0; q < 16; ++q)
        m[q] += S0(m[(q + 1) & 15]) + m[(q + 9) & 15] + S1(m[(q + 14) & 15]);
}

// digest h of the one padded block m (the schedule is built in m): a loop
// of 16 rounds, then the next 16 schedule words, so each compression is a
// few KB of code (unrolled whole, the two compressions outgrow the
// instruction cache and the warps wait on fetches)
__device__ __forceinline__ void sha256_block(uint32_t (&m)[16], uint32_t (&h)[8])
{
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        v[i] = kSha256H[i];
#pragma unroll 1
    for (int t0 = 0;; t0 += 16) {
        sha256_8(m, v, t0, 0);
        sha256_8(m, v, t0, 8);
        if (t0 == 48)
            break;
        schedule16<uint32_t, s256_0, s256_1>(m);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
        h[i] = kSha256H[i] + v[i];
}

__device__ __forceinline__ void sha512_block(uint64_t (&m)[16], uint64_t (&h)[8])
{
    uint64_t v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        v[i] = kSha512H[i];
#pragma unroll 1
    for (int t0 = 0;; t0 += 16) {
        sha512_8(m, v, t0, 0);
        sha512_8(m, v, t0, 8);
        if (t0 == 64)
            break;
        schedule16<uint64_t, s512_0, s512_1>(m);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
        h[i] = kSha512H[i] + v[i];
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
