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

} // namespace pkb
} // namespace frag
