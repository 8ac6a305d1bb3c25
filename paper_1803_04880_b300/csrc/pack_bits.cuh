// pack_bits.cuh -- the bit records of the thesis's packed three fragments
// (Sec. 5.2.1 fragments, Sec. 5.2.3 widths) for 8 x 8 blocks at two levels.
//
// Per block: A = LL_2 - 128 as 4 x 10 bits (40); B = HL_2 and LH_2 as 10
// bits and HH_2 as 11 (124); C = HL_1, LH_1 and HH_1 as 10 bits (480).  A
// value is its two's complement in its width; a record's values follow each
// other from bit 0 (each band's 2 x 2 or 4 x 4 tile row-major, bands in the
// order above) and fill bytes from the least significant bit.  A and C hold
// one record per block (5 and 60 bytes), blocks row-major; in B the blocks
// of a block row follow each other every 124 bits and every block row starts
// on a byte.  A warp owns 32 neighbouring blocks of a block row, so its B
// records are 496 contiguous bytes, assembled from the lanes' registers
// with shuffles (or in a shared area of kPackBWords words when unaligned),
// and its A and C records are 160 and 1,920 contiguous bytes, which the
// lanes write to (read from) a shared staging area and the warp moves with
// 16-byte accesses.
#pragma once

#include <cstdint>

namespace frag {
namespace pkb {

constexpr int kPackBWords = 125; // 124 words of a warp's B records and one more read on unpack
constexpr int kErrWidth = 5;     // device error code: a coefficient outside its width

// bytes of B a block row of nbx blocks takes
__host__ __device__ inline uint64_t b_row_bytes(uint64_t nbx) { return (124 * nbx + 7) / 8; }

// the warp's B bytes: `count` from `base`, the warp's 32 blocks at bits
// 124 lane of its shared area sb (every lane of the warp calls these)
__device__ __forceinline__ void store_b(uint32_t *sb, uint8_t *base, uint32_t count, bool valid, int lane,
                                        const uint32_t (&rb)[4])
{
    for (int j = lane; j < kPackBWords; j += 32)
        sb[j] = 0u;
    __syncwarp();
    if (valid) {
        const uint32_t bit = 124u * (uint32_t)lane, q = bit >> 5, sh = bit & 31;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            atomicOr(&sb[q + i], rb[i] << sh);
            if (sh)
                atomicOr(&sb[q + i + 1], rb[i] >> (32 - sh));
        }
    }
    __syncwarp();
    const uint8_t *smb = reinterpret_cast<const uint8_t *>(sb);
    for (uint32_t j = (uint32_t)lane; j < count; j += 32)
        base[j] = smb[j];
    __syncwarp();
}

__device__ __forceinline__ void load_b(uint32_t *sb, const uint8_t *base, uint32_t count, bool valid,
                                       int lane, uint32_t (&rb)[4])
{
    uint8_t *smb = reinterpret_cast<uint8_t *>(sb);
    for (uint32_t j = (uint32_t)lane; j < count; j += 32)
        smb[j] = base[j];
    __syncwarp();
    if (valid) {
        const uint32_t bit = 124u * (uint32_t)lane, q = bit >> 5, sh = bit & 31;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            rb[i] = sh ? (sb[q + i] >> sh) | (sb[q + i + 1] << (32 - sh)) : sb[q + i];
        rb[3] &= 0x0fffffffu; // bits 124..127 are the next block's
    }
    __syncwarp();
}

// -- the same without shared memory, for a 16-byte aligned warp area ------
// The warp's 31 chunks of 128 bits: chunk j (bytes 16 j .. 16 j + 15) holds
// bits 4 j .. 123 of block j's record, then bits 0 .. 4 j + 3 of block
// j + 1's; so lane j writes (reads) chunk j with its neighbour's record (the
// previous chunk) from one shuffle.  Every lane of the warp calls these.
struct U128 {
    uint64_t lo, hi;
};

__device__ __forceinline__ U128 u128(const uint32_t (&r)[4])
{
    return {r[0] | ((uint64_t)r[1] << 32), r[2] | ((uint64_t)r[3] << 32)};
}

// 64-bit shifts whose amount may exceed 63: PTX clamps the amount to 64,
// so the result is then 0 (C++ shifts would be undefined there)
__device__ __forceinline__ uint64_t shr64z(uint64_t x, uint32_t s)
{
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}
__device__ __forceinline__ uint64_t shl64z(uint64_t x, uint32_t s)
{
    uint64_t r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}

// 128-bit shifts by 0 <= s <= 128, without branches: of the three terms of
// the word that straddles, the ones whose amount is out of range (64 - s or
// s - 64 wraps to a huge unsigned value) are 0
__device__ __forceinline__ U128 shr128(U128 x, uint32_t s)
{
    return {shr64z(x.lo, s) | shl64z(x.hi, 64u - s) | shr64z(x.hi, s - 64u), shr64z(x.hi, s)};
}

__device__ __forceinline__ U128 shl128(U128 x, uint32_t s)
{
    return {shl64z(x.lo, s), shl64z(x.hi, s) | shr64z(x.lo, 64u - s) | shl64z(x.lo, s - 64u)};
}

__device__ __forceinline__ void store_b_vec(uint8_t *base, uint32_t count, int lane, const uint32_t (&rb)[4])
{
    uint32_t nx[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        nx[i] = __shfl_down_sync(0xffffffffu, rb[i], 1); // block lane + 1 (lanes without a block hold 0)
    const U128 a = shr128(u128(rb), 4u * (uint32_t)lane);
    const U128 b = shl128(u128(nx), 124u - 4u * (uint32_t)lane);
    const uint32_t c[4] = {(uint32_t)(a.lo | b.lo), (uint32_t)((a.lo | b.lo) >> 32), (uint32_t)(a.hi | b.hi),
                           (uint32_t)((a.hi | b.hi) >> 32)};
    const uint32_t off = 16u * (uint32_t)lane;
    if (off + 16 <= count) {
        __stcs(reinterpret_cast<uint4 *>(base + off), make_uint4(c[0], c[1], c[2], c[3]));
    } else if (off < count) {
#pragma unroll
        for (uint32_t k = 0; k < 16; ++k)
            if (off + k < count)
                base[off + k] = (uint8_t)(c[k >> 2] >> (8 * (k & 3)));
    }
}

__device__ __forceinline__ void load_b_vec(const uint8_t *base, uint32_t count, bool valid, int lane,
                                           uint32_t (&rb)[4])
{
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    const uint32_t off = 16u * (uint32_t)lane;
    if (off + 16 <= count) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(base + off));
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    } else if (off < count) {
#pragma unroll
        for (uint32_t k = 0; k < 16; ++k)
            if (off + k < count)
                w[k >> 2] |= (uint32_t)__ldg(base + off + k) << (8 * (k & 3));
    }
    uint32_t pv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        pv[i] = __shfl_up_sync(0xffffffffu, w[i], 1); // chunk lane - 1
    // block j: the top 4 j bits of chunk j - 1, then chunk j (block 0: chunk 0)
    const U128 a = shr128(u128(pv), 128u - 4u * (uint32_t)lane);
    const U128 b = shl128(u128(w), 4u * (uint32_t)lane);
    if (valid) {
        rb[0] = (uint32_t)(a.lo | b.lo);
        rb[1] = (uint32_t)((a.lo | b.lo) >> 32);
        rb[2] = (uint32_t)(a.hi | b.hi);
        rb[3] = (uint32_t)((a.hi | b.hi) >> 32) & 0x0fffffffu;
    }
}

// the warp's B records out of (into) the registers: vector accesses when
// the warp's area is 16-byte aligned, else through the shared area sb
__device__ __forceinline__ void put_b(uint32_t *sb, uint8_t *base, uint32_t count, bool valid, int lane,
                                      const uint32_t (&rb)[4])
{
    if ((reinterpret_cast<uintptr_t>(base) & 15u) == 0)
        store_b_vec(base, count, lane, rb);
    else
        store_b(sb, base, count, valid, lane, rb);
}

__device__ __forceinline__ void get_b(uint32_t *sb, const uint8_t *base, uint32_t count, bool valid, int lane,
                                      uint32_t (&rb)[4])
{
    if ((reinterpret_cast<uintptr_t>(base) & 15u) == 0)
        load_b_vec(base, count, valid, lane, rb);
    else
        load_b(sb, base, count, valid, lane, rb);
}

// -- biased pairs straight to fields -------------------------------------
// The kernels carry a pair of coefficients as one word, v + 0x4000 in each
// 16-bit half (|v| < 0x4000).  0x4000 is a multiple of 2^K for the widths
// here, so the low K bits of a half are v's K-bit two's complement: a pair
// becomes its 2K-bit field (low value first) with one shift and one select,
// and both halves are range-checked with one subtraction and one mask.

// the pair's 2K-bit field: (v_lo mod 2^K) | (v_hi mod 2^K) << K
template <int K>
__device__ __forceinline__ uint32_t field2(uint32_t w)
{
    constexpr uint32_t m = (1u << K) - 1u;
    return (w & m) | ((w >> (16 - K)) & (m << K));
}

// nonzero when a half of the pair is outside [-2^(K-1), 2^(K-1)): v + 0x4000
// - (0x4000 - 2^(K-1)) is in [0, 2^K) exactly when v fits (a borrow out of
// the low half only happens when the low half is already out of range)
template <int K>
__device__ __forceinline__ uint32_t range_bits(uint32_t w)
{
    constexpr uint32_t c = (0x4000u - (1u << (K - 1))) * 0x10001u;
    constexpr uint32_t hi = (0xffffu & ~((1u << K) - 1u)) * 0x10001u;
    return (w - c) & hi;
}

// the biased pair of a 2K-bit field: flipping a K-bit two's complement's
// sign bit adds 2^(K-1), then the bias less 2^(K-1)
template <int K>
__device__ __forceinline__ uint32_t unfield2(uint32_t f)
{
    constexpr uint32_t m = (1u << K) - 1u, h = 1u << (K - 1), c = 0x4000u - h;
    const uint32_t p = (f & m) | ((f << (16 - K)) & (m << 16));
    return (p ^ (h * 0x10001u)) + c * 0x10001u;
}

// field f of `bits` bits (at most 32) into record r at bit pos, r zeroed
// first (pos and bits are constants once the callers' loops unroll)
template <int N>
__device__ __forceinline__ void ins(uint32_t (&r)[N], int pos, uint32_t f, int bits)
{
    const int q = pos >> 5, sh = pos & 31;
    r[q] |= f << sh;
    if (sh + bits > 32)
        r[q + 1] |= f >> (32 - sh);
}

template <int N>
__device__ __forceinline__ uint32_t ext(const uint32_t (&r)[N], int pos, int bits)
{
    const int q = pos >> 5, sh = pos & 31;
    const uint32_t u = (sh + bits > 32) ? __funnelshift_r(r[q], r[q + 1], (uint32_t)sh) : (r[q] >> sh);
    return bits == 32 ? u : (u & ((1u << bits) - 1u));
}

// -- a warp's A or C records between its shared staging area and memory ----
// The records of the warp's 32 blocks are contiguous (count bytes at dst /
// src); every lane of the warp calls these.  16-byte accesses when the
// global address allows, else 4-byte, else bytes.
__device__ __forceinline__ void copy_out(uint8_t *dst, const uint8_t *sm, uint32_t count, int lane)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
    uint32_t done = 0;
    if ((a & 15u) == 0) {
        const uint32_t n = count >> 4;
        for (uint32_t j = (uint32_t)lane; j < n; j += 32)
            __stcs(reinterpret_cast<uint4 *>(dst) + j, reinterpret_cast<const uint4 *>(sm)[j]);
        done = n << 4;
    } else if ((a & 3u) == 0) {
        const uint32_t n = count >> 2;
        for (uint32_t j = (uint32_t)lane; j < n; j += 32)
            __stcs(reinterpret_cast<unsigned int *>(dst) + j, reinterpret_cast<const unsigned int *>(sm)[j]);
        done = n << 2;
    }
    for (uint32_t j = done + (uint32_t)lane; j < count; j += 32)
        dst[j] = sm[j];
}

__device__ __forceinline__ void copy_in(uint8_t *sm, const uint8_t *src, uint32_t count, int lane)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    uint32_t done = 0;
    if ((a & 15u) == 0) {
        const uint32_t n = count >> 4;
        for (uint32_t j = (uint32_t)lane; j < n; j += 32)
            reinterpret_cast<uint4 *>(sm)[j] = __ldg(reinterpret_cast<const uint4 *>(src) + j);
        done = n << 4;
    } else if ((a & 3u) == 0) {
        const uint32_t n = count >> 2;
        for (uint32_t j = (uint32_t)lane; j < n; j += 32)
            reinterpret_cast<unsigned int *>(sm)[j] = __ldg(reinterpret_cast<const unsigned int *>(src) + j);
        done = n << 2;
    }
    for (uint32_t j = done + (uint32_t)lane; j < count; j += 32)
        sm[j] = __ldg(src + j);
}

// a warp's staging area: C records (15 words a block, block j at word 15 j:
// 15 is odd, so the 32 lanes' words fall in 32 banks), A records (5 bytes a
// block) and, on the way in, the raw B bytes (496 and a zero chunk)
constexpr int kStageCWords = 15 * 32;
constexpr int kStageABytes = 5 * 32;
constexpr int kStageBBytes = 512;
struct __align__(16) Stage {
    uint32_t c[kStageCWords];
    uint8_t a[kStageABytes];
};
struct __align__(16) StageIn {
    uint32_t c[kStageCWords];
    uint8_t a[kStageABytes];
    uint8_t b[kStageBBytes];
};

// A full warp of 32 blocks whose three record areas are 16-byte aligned:
// 1,920 bytes of C, 160 of A, 496 of B, all whole 16-byte pieces
constexpr uint32_t kFullC16 = 120, kFullA16 = 10, kFullB16 = 31;
__device__ __forceinline__ bool full_aligned(uint32_t nvalid, const void *a, const void *b, const void *c)
{
    return nvalid == 32 &&
           ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c)) & 15u) ==
               0;
}

// the A and C records of a full aligned warp out of its staging area: fixed
// trip counts, no loop control
__device__ __forceinline__ void copy_out_full(uint8_t *a, uint8_t *c, const Stage &st, int lane)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t j = (uint32_t)lane + 32u * k;
        if (j < kFullC16)
            __stcs(reinterpret_cast<uint4 *>(c) + j, reinterpret_cast<const uint4 *>(st.c)[j]);
    }
    if ((uint32_t)lane < kFullA16)
        __stcs(reinterpret_cast<uint4 *>(a) + lane, reinterpret_cast<const uint4 *>(st.a)[lane]);
}

// the next unit's A, B and C records of a full aligned warp into a staging
// area with cp.async (16 bytes a copy, every lane its share); the caller
// commits the group and waits for it before reading
__device__ __forceinline__ void cp16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void prefetch_full(StageIn &st, const uint8_t *a, const uint8_t *b, const uint8_t *c,
                                              int lane)
{
    const uint32_t sc = (uint32_t)__cvta_generic_to_shared(st.c);
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(st.a);
    const uint32_t sbb = (uint32_t)__cvta_generic_to_shared(st.b);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t j = (uint32_t)lane + 32u * k;
        if (j < kFullC16)
            cp16(sc + 16u * j, c + 16u * j);
    }
    if ((uint32_t)lane < kFullA16)
        cp16(sa + 16u * lane, a + 16u * lane);
    if ((uint32_t)lane < kFullB16)
        cp16(sbb + 16u * lane, b + 16u * lane);
}

// the lane's B record from the raw B bytes of its warp in shared memory
// (chunk j holds bits 4 j .. 123 of block j and the start of block j + 1's)
__device__ __forceinline__ void b_from_stage(const StageIn &st, bool valid, int lane, uint32_t (&rb)[4])
{
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if ((uint32_t)lane < kFullB16) {
        const uint4 v = reinterpret_cast<const uint4 *>(st.b)[lane];
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    }
    uint32_t pv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        pv[i] = __shfl_up_sync(0xffffffffu, w[i], 1);
    const U128 x = shr128(u128(pv), 128u - 4u * (uint32_t)lane);
    const U128 y = shl128(u128(w), 4u * (uint32_t)lane);
    if (valid) {
        rb[0] = (uint32_t)(x.lo | y.lo);
        rb[1] = (uint32_t)((x.lo | y.lo) >> 32);
        rb[2] = (uint32_t)(x.hi | y.hi);
        rb[3] = (uint32_t)((x.hi | y.hi) >> 32) & 0x0fffffffu;
    }
}

} // namespace pkb
} // namespace frag
