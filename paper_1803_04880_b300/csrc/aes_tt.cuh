// aes_tt.cuh -- AES-128 of counter blocks in the 32-bit table form, for the
// kernels that encipher the private fragment (Sec. 5.2.1: the LL band is
// encrypted with AES; AES-128 is FIPS-197).
//
// A round's SubBytes, ShiftRows and MixColumns become, per output column,
// four lookups in one 256-entry table T0 and its byte rotations T1..T3
// (FIPS-197 Sec. 5.1 restated column by column); the last round takes the
// S-box from byte 1 of the same entry, since T0[x] = (2 S[x], S[x], S[x],
// 3 S[x]) from the most significant byte down.  The table sits in shared
// memory once per lane (entry x of lane t at word 32 x + t), so the 32
// lookups of a warp always fall in 32 different banks.
//
// Counter block (CTR mode, SP 800-38A): nonce (8 bytes big-endian) followed
// by the block index (8 bytes big-endian); the keystream comes back as four
// words whose bytes are in stream order (word 0, byte 0 is keystream byte 0),
// ready to XOR into little-endian loads of the data.
#pragma once

#include "frag_internal.cuh"

namespace frag {
namespace aes {

// shared-memory words of the lane-replicated table
constexpr int kTableWords = 256 * 32;

using Keys = AesKeys;

__host__ __device__ inline uint32_t rol8_host(uint32_t w) { return (w << 8) | (w >> 24); }

// from the 44 big-endian round-key words of the key schedule
__host__ __device__ inline Keys keys_from_words(const uint32_t *rk)
{
    Keys K;
    for (int r = 0; r < 10; ++r) {
        K.k[r] = make_uint4(rk[4 * r], rk[4 * r + 1], rk[4 * r + 2], rk[4 * r + 3]);
        K.kr[r] = make_uint4(rol8_host(rk[4 * r]), rol8_host(rk[4 * r + 1]), rol8_host(rk[4 * r + 2]),
                             rol8_host(rk[4 * r + 3]));
    }
    uint32_t l[4];
    for (int i = 0; i < 4; ++i) {
        const uint32_t w = rk[40 + i];
        l[i] = (w >> 24) | ((w >> 8) & 0xff00u) | ((w << 8) & 0xff0000u) | (w << 24);
    }
    K.last_le = make_uint4(l[0], l[1], l[2], l[3]);
    return K;
}

// Table 0 into shared memory, one copy per lane: each warp of the block takes
// 32 entries with one coalesced load and writes entry x as the 32 words
// (x, lane 0..31).  The caller synchronises the block afterwards.
__device__ __forceinline__ void build_table(uint32_t *te, const uint32_t *t0)
{
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t base = (threadIdx.x >> 5) * 32; base < 256; base += (blockDim.x >> 5) * 32) {
        const uint32_t v = __ldg(t0 + base + lane);
#pragma unroll 8
        for (int k = 0; k < 32; ++k)
            te[(base + k) * 32 + lane] = __shfl_sync(0xffffffffu, v, k);
    }
}

// byte k of v, zero-extended
__device__ __forceinline__ uint32_t byte_of(uint32_t v, uint32_t k) { return __byte_perm(v, 0u, 0x4440u | k); }
// entry x of this lane's copy (tel = table + lane)
__device__ __forceinline__ uint32_t t0(const uint32_t *tel, uint32_t x) { return tel[x << 5]; }
__device__ __forceinline__ uint32_t ror8(uint32_t v) { return __byte_perm(v, v, 0x0321); }
__device__ __forceinline__ uint32_t ror16(uint32_t v) { return __byte_perm(v, v, 0x1032); }
__device__ __forceinline__ uint32_t ror24(uint32_t v) { return __byte_perm(v, v, 0x2103); }

// Keystream block `blk` of `nonce`.  K: anything with k[0..9] and last_le
// (the launch's parameters, or a copy in shared memory).
template <class KeySet>
__device__ __forceinline__ void ctr_block(const uint32_t *tel, const KeySet &K, uint64_t nonce,
                                          uint64_t blk, uint32_t ks[4])
{
    const uint4 k0 = K.k[0];
    uint32_t s0 = (uint32_t)(nonce >> 32) ^ k0.x;
    uint32_t s1 = (uint32_t)nonce ^ k0.y;
    uint32_t s2 = (uint32_t)(blk >> 32) ^ k0.z;
    uint32_t s3 = (uint32_t)blk ^ k0.w;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint4 k = K.k[r];
        const uint32_t n0 = t0(tel, byte_of(s0, 3)) ^ ror8(t0(tel, byte_of(s1, 2))) ^
                            ror16(t0(tel, byte_of(s2, 1))) ^ ror24(t0(tel, byte_of(s3, 0))) ^ k.x;
        const uint32_t n1 = t0(tel, byte_of(s1, 3)) ^ ror8(t0(tel, byte_of(s2, 2))) ^
                            ror16(t0(tel, byte_of(s3, 1))) ^ ror24(t0(tel, byte_of(s0, 0))) ^ k.y;
        const uint32_t n2 = t0(tel, byte_of(s2, 3)) ^ ror8(t0(tel, byte_of(s3, 2))) ^
                            ror16(t0(tel, byte_of(s0, 1))) ^ ror24(t0(tel, byte_of(s1, 0))) ^ k.z;
        const uint32_t n3 = t0(tel, byte_of(s3, 3)) ^ ror8(t0(tel, byte_of(s0, 2))) ^
                            ror16(t0(tel, byte_of(s1, 1))) ^ ror24(t0(tel, byte_of(s2, 0))) ^ k.w;
        s0 = n0;
        s1 = n1;
        s2 = n2;
        s3 = n3;
    }
    // last round: SubBytes (byte 1 of the entry), ShiftRows, AddRoundKey,
    // the output bytes placed straight in stream order
    auto sub4 = [&](uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
        const uint32_t lo = __byte_perm(t0(tel, byte_of(a, 3)), t0(tel, byte_of(b, 2)), 0x0051);
        const uint32_t hi = __byte_perm(t0(tel, byte_of(c, 1)), t0(tel, byte_of(d, 0)), 0x0051);
        return __byte_perm(lo, hi, 0x5410);
    };
    const uint4 kl = K.last_le;
    ks[0] = sub4(s0, s1, s2, s3) ^ kl.x;
    ks[1] = sub4(s1, s2, s3, s0) ^ kl.y;
    ks[2] = sub4(s2, s3, s0, s1) ^ kl.z;
    ks[3] = sub4(s3, s0, s1, s2) ^ kl.w;
}

// ---------------------------------------------------------------------------
// Two-table form: T0 and T2 = ror16(T0) side by side, once per lane, 64 KB at
// a shared-window address that is a multiple of 65536.  Entry x of T0 for
// lane t is at byte 256 x + 4 t of the table, of T2 at 256 x + 128 + 4 t, so
// a lookup's whole address is one byte permute: byte 0 the lane's offset,
// byte 1 the state byte, bytes 2 and 3 the table's (its low 16 bits are 0).
// With T2 a round column needs one rotation instead of three:
//   n0 = T0[a] ^ T2[c] ^ ror8(T0[b] ^ T2[d] ^ rol8(k))
// for the bytes a, b, c, d that ShiftRows brings to column 0.
// ---------------------------------------------------------------------------
constexpr uint32_t kDualBytes = 65536;

// the 64 KB-aligned window address for the table inside a block's dynamic
// shared memory that starts at window address `base`: 2 kDualBytes of it
// hold the table whatever base in 0 .. 65536 is
__device__ __forceinline__ uint32_t dual_table_at(uint32_t base) { return (base + 65535u) & ~65535u; }

__device__ __forceinline__ void sts32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// every thread of a block of THREADS threads writes its share of the 16,384
// words; all of a thread's loads are issued before its stores, so the
// build costs one round trip to L2, not one per word
template <int THREADS>
__device__ __forceinline__ void build_dual(uint32_t tab, const uint32_t *t0g)
{
    constexpr int kPer = (int)(kDualBytes / 4) / THREADS;
    static_assert(kPer * THREADS == (int)(kDualBytes / 4), "the block's threads divide the table");
    uint32_t v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k)
        v[k] = __ldg(t0g + ((threadIdx.x + (uint32_t)(k * THREADS)) >> 6));
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t i = threadIdx.x + (uint32_t)(k * THREADS);
        sts32(tab + 4 * i, ((i >> 5) & 1) ? ror16(v[k]) : v[k]);
    }
}

// the lane's lookup bases: the table's window address with byte 0 = 4 t (T0)
// or 128 + 4 t (T2)
struct Lut {
    uint32_t b0, b2;
};
__device__ __forceinline__ Lut make_lut(uint32_t tab, uint32_t lane) { return Lut{tab | (4u * lane), tab | (128u + 4u * lane)}; }

// entry (byte k of w) of the table whose lane base is `base`
template <int K>
__device__ __forceinline__ uint32_t look(uint32_t base, uint32_t w)
{
    const uint32_t a = __byte_perm(w, base, 0x7604u | ((uint32_t)K << 4));
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) { return a ^ b ^ c; }

// The round-1 outputs of a counter block depend on the nonce words (s0, s1)
// and the high block word (s2) only through constants: the column of s3's
// byte is the only term that varies.  C[j] holds the rest of column j.
struct Round1 {
    uint32_t c0, c1, c2, c3;
    uint32_t hi; // the high block word they were made for
};

template <class KeySet>
__device__ __forceinline__ Round1 round1_consts(const Lut &L, const KeySet &K, uint64_t nonce, uint32_t hi)
{
    const uint4 k0 = K.k[0], kr = K.kr[1];
    const uint32_t s0 = (uint32_t)(nonce >> 32) ^ k0.x, s1 = (uint32_t)nonce ^ k0.y, s2 = hi ^ k0.z;
    Round1 R;
    R.c0 = look<3>(L.b0, s0) ^ look<1>(L.b2, s2) ^ ror8(look<2>(L.b0, s1) ^ kr.x);
    R.c1 = look<3>(L.b0, s1) ^ ror8(look<2>(L.b0, s2) ^ look<0>(L.b2, s0) ^ kr.y);
    R.c2 = look<3>(L.b0, s2) ^ look<1>(L.b2, s0) ^ ror8(look<0>(L.b2, s1) ^ kr.z);
    R.c3 = look<1>(L.b2, s1) ^ ror8(look<2>(L.b0, s0) ^ look<0>(L.b2, s2) ^ kr.w);
    R.hi = hi;
    return R;
}

// keystream of the counter block whose low word is lo (the high word and the
// nonce are R's), bytes in stream order
template <class KeySet>
__device__ __forceinline__ void ctr_block2(const Lut &L, const KeySet &K, const Round1 &R, uint32_t lo,
                                           uint32_t ks[4])
{
    const uint32_t s3 = lo ^ K.k[0].w;
    uint32_t s0 = R.c0 ^ ror8(look<0>(L.b2, s3));
    uint32_t s1 = R.c1 ^ look<1>(L.b2, s3);
    uint32_t s2 = R.c2 ^ ror8(look<2>(L.b0, s3));
    uint32_t t3 = R.c3 ^ look<3>(L.b0, s3);
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint4 k = K.kr[r];
        const uint32_t n0 = xor3(look<3>(L.b0, s0), look<1>(L.b2, s2),
                                 ror8(xor3(look<2>(L.b0, s1), look<0>(L.b2, t3), k.x)));
        const uint32_t n1 = xor3(look<3>(L.b0, s1), look<1>(L.b2, t3),
                                 ror8(xor3(look<2>(L.b0, s2), look<0>(L.b2, s0), k.y)));
        const uint32_t n2 = xor3(look<3>(L.b0, s2), look<1>(L.b2, s0),
                                 ror8(xor3(look<2>(L.b0, t3), look<0>(L.b2, s1), k.z)));
        const uint32_t n3 = xor3(look<3>(L.b0, t3), look<1>(L.b2, s1),
                                 ror8(xor3(look<2>(L.b0, s0), look<0>(L.b2, s2), k.w)));
        s0 = n0;
        s1 = n1;
        s2 = n2;
        t3 = n3;
    }
    // last round: S[x] is byte 1 and byte 2 of T0[x], byte 0 and byte 3 of
    // T2[x]; each output byte comes from the entry that has it in place
    const uint4 kl = K.last_le;
    auto sub4 = [&](uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
        const uint32_t x = __byte_perm(look<3>(L.b2, a), look<2>(L.b0, b), 0x0050u);
        const uint32_t y = __byte_perm(look<1>(L.b0, c), look<0>(L.b2, d), 0x7200u);
        return __byte_perm(x, y, 0x7610u);
    };
    ks[0] = sub4(s0, s1, s2, t3) ^ kl.x;
    ks[1] = sub4(s1, s2, t3, s0) ^ kl.y;
    ks[2] = sub4(s2, t3, s0, s1) ^ kl.z;
    ks[3] = sub4(t3, s0, s1, s2) ^ kl.w;
}

} // namespace aes
} // namespace frag
