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
// records are 496 contiguous bytes, assembled in (or read from) a shared
// area of kPackBWords words.
#pragma once

#include <cstdint>

namespace frag {
namespace pkb {

constexpr int kPackBWords = 125; // 124 words of a warp's B records and one more read on unpack
constexpr int kErrWidth = 5;     // device error code: a coefficient outside its width

__device__ __forceinline__ bool fits(int32_t v, int width)
{
    return v >= -(1 << (width - 1)) && v < (1 << (width - 1));
}

// value v as `width` bits at bit pos of the record r (zeroed first)
template <int N>
__device__ __forceinline__ void put(uint32_t (&r)[N], int pos, int32_t v, int width)
{
    const uint32_t u = (uint32_t)v & ((1u << width) - 1u);
    const int q = pos >> 5, sh = pos & 31;
    r[q] |= u << sh;
    if (sh + width > 32)
        r[q + 1] |= u >> (32 - sh);
}

template <int N>
__device__ __forceinline__ int32_t get(const uint32_t (&r)[N], int pos, int width)
{
    const int q = pos >> 5, sh = pos & 31;
    uint32_t u = r[q] >> sh;
    if (sh + width > 32)
        u |= r[q + 1] << (32 - sh);
    return (int32_t)(u << (32 - width)) >> (32 - width); // sign-extend
}

__device__ __forceinline__ int32_t lo16(uint32_t w) { return (int32_t)(int16_t)(w & 0xffffu); }
__device__ __forceinline__ int32_t hi16(uint32_t w) { return (int32_t)(int16_t)(w >> 16); }
__device__ __forceinline__ uint32_t pair16(int32_t a, int32_t b)
{
    return ((uint32_t)a & 0xffffu) | ((uint32_t)b << 16);
}

// the two int16 halves of w at bits pos and pos + width of r; ok &= both fit
template <int N>
__device__ __forceinline__ void put_pair(uint32_t (&r)[N], int pos, uint32_t w, int width, bool &ok)
{
    ok = ok && fits(lo16(w), width) && fits(hi16(w), width);
    put(r, pos, lo16(w), width);
    put(r, pos + width, hi16(w), width);
}

// the int16 pair at bits pos and pos + width of r
template <int N>
__device__ __forceinline__ uint32_t get_pair(const uint32_t (&r)[N], int pos, int width)
{
    return pair16(get(r, pos, width), get(r, pos + width, width));
}

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

__device__ __forceinline__ U128 shr128(U128 x, uint32_t s) // 0 <= s <= 128
{
    if (s >= 128)
        return {0ull, 0ull};
    if (s >= 64)
        return {x.hi >> (s - 64), 0ull};
    if (s == 0)
        return x;
    return {(x.lo >> s) | (x.hi << (64 - s)), x.hi >> s};
}

__device__ __forceinline__ U128 shl128(U128 x, uint32_t s) // 0 <= s <= 128
{
    if (s >= 128)
        return {0ull, 0ull};
    if (s >= 64)
        return {0ull, x.lo << (s - 64)};
    if (s == 0)
        return x;
    return {x.lo << s, (x.hi << s) | (x.lo >> (64 - s))};
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
    } else {
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
    } else {
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

} // namespace pkb
} // namespace frag
