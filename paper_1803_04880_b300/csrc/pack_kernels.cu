// pack_kernels.cu -- the thesis's storage of its three fragments (Sec. 5.2.1:
// the private fragment and the first and second public and protected
// fragments; Sec. 5.2.3: the bits each coefficient takes) for 8 x 8 blocks
// at two levels, to and from the block mode's int16 layout.
//
// Per block: A = LL_2 as 4 x 10 bits (40); B = HL_2 and LH_2 as 10 bits and
// HH_2 as 11 (124); C = HL_1, LH_1 and HH_1 as 10 bits (480).  A value is its
// two's complement in its width; a record's values follow each other from bit
// 0 (each band's 2 x 2 or 4 x 4 tile row-major, bands in the order above) and
// fill bytes from the least significant bit.  A and C hold one record per
// block (5 and 60 bytes), blocks row-major; in B the blocks of a block row
// follow each other every 124 bits and every block row starts on a byte.
// The bounds of the coefficients (Sec. 5.2.3) make the widths enough; a
// value outside its width sets the device error word instead of being
// stored.
//
// One lane owns one block and a warp 32 neighbouring blocks of a block row,
// so the warp's B records are 496 contiguous bytes: they are assembled in
// shared memory (each lane ORs its bits in) and copied out a byte a lane.
#include "frag_internal.cuh"

namespace frag {
namespace pk {

constexpr int kWarps = kPackWarps;
constexpr int kThreads = 32 * kWarps;
constexpr int kBWords = 125; // a warp's 124 words of B records and one more read on unpack
constexpr int kErrWidth = 5; // device error code: a coefficient outside its width

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

// element (row, col) of an int16 band of width wl
__device__ __forceinline__ uint8_t *at(uint8_t *band, uint64_t row, uint32_t wl, uint64_t col)
{
    return band + 2 * (row * wl + col);
}

template <bool FWD>
__global__ void __launch_bounds__(kThreads) pack_kernel(PackWork w)
{
    __shared__ uint32_t sb[kWarps][kBWords];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *smb = reinterpret_cast<uint8_t *>(sb[warp]);
    const uint32_t strips = (w.nbx + 31) / 32;
    const uint64_t units = (uint64_t)w.nby * strips;
    const uint32_t W1 = w.W >> 1, W2 = w.W >> 2;
    for (uint64_t u = (uint64_t)blockIdx.x * kWarps + warp; u < units; u += (uint64_t)gridDim.x * kWarps) {
        const uint64_t bi = u / strips;
        const uint32_t s = (uint32_t)(u % strips);
        const uint32_t bj = 32 * s + lane;
        const uint32_t nvalid = min(32u, w.nbx - 32 * s);
        const bool valid = bj < w.nbx;
        const uint64_t idx = bi * w.nbx + bj;
        const uint32_t count = (124 * nvalid + 7) / 8; // bytes of B this warp owns
        uint8_t *bbase = w.b + bi * w.brow + 496ull * s;
        uint32_t ra[2] = {0u, 0u}, rb[4] = {0u, 0u, 0u, 0u}, rc[15];
#pragma unroll
        for (int i = 0; i < 15; ++i)
            rc[i] = 0u;
        if (FWD) {
            bool ok = true;
            if (valid) {
                // A: LL_2 (2 x 2)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const uint32_t v = *reinterpret_cast<const uint32_t *>(at(w.ll, 2 * bi + r, W2, 2ull * bj));
                    ok = ok && fits(lo16(v), 10) && fits(hi16(v), 10);
                    put(ra, 20 * r, lo16(v), 10);
                    put(ra, 20 * r + 10, hi16(v), 10);
                }
                // B: HL_2, LH_2 (10 bits), HH_2 (11 bits)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int width = k == 2 ? 11 : 10;
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const uint32_t v =
                            *reinterpret_cast<const uint32_t *>(at(w.band[1][k], 2 * bi + r, W2, 2ull * bj));
                        const int pos = 40 * k + 2 * r * width;
                        ok = ok && fits(lo16(v), width) && fits(hi16(v), width);
                        put(rb, pos, lo16(v), width);
                        put(rb, pos + width, hi16(v), width);
                    }
                }
                // C: HL_1, LH_1, HH_1 (4 x 4, 10 bits)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const uint2 v = *reinterpret_cast<const uint2 *>(at(w.band[0][k], 4 * bi + r, W1, 4ull * bj));
                        const int pos = 160 * k + 40 * r;
                        ok = ok && fits(lo16(v.x), 10) && fits(hi16(v.x), 10) && fits(lo16(v.y), 10) &&
                             fits(hi16(v.y), 10);
                        put(rc, pos, lo16(v.x), 10);
                        put(rc, pos + 10, hi16(v.x), 10);
                        put(rc, pos + 20, lo16(v.y), 10);
                        put(rc, pos + 30, hi16(v.y), 10);
                    }
                }
                if (!ok)
                    atomicCAS(w.err, 0, kErrWidth);
                uint8_t *pa = w.a + 5 * idx;
                pa[0] = (uint8_t)ra[0];
                pa[1] = (uint8_t)(ra[0] >> 8);
                pa[2] = (uint8_t)(ra[0] >> 16);
                pa[3] = (uint8_t)(ra[0] >> 24);
                pa[4] = (uint8_t)ra[1];
                uint8_t *pc = w.c + 60 * idx;
                if (w.cvec) {
#pragma unroll
                    for (int i = 0; i < 15; ++i)
                        reinterpret_cast<uint32_t *>(pc)[i] = rc[i];
                } else {
#pragma unroll
                    for (int i = 0; i < 60; ++i)
                        pc[i] = (uint8_t)(rc[i >> 2] >> (8 * (i & 3)));
                }
            }
            // B: OR the records into shared memory, then copy the warp's bytes out
            for (int j = lane; j < kBWords; j += 32)
                sb[warp][j] = 0u;
            __syncwarp();
            if (valid) {
                const uint32_t bit = 124u * lane, q = bit >> 5, sh = bit & 31;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    atomicOr(&sb[warp][q + i], rb[i] << sh);
                    if (sh)
                        atomicOr(&sb[warp][q + i + 1], rb[i] >> (32 - sh));
                }
            }
            __syncwarp();
            for (uint32_t j = lane; j < count; j += 32)
                bbase[j] = smb[j];
            __syncwarp();
        } else {
            // B: copy the warp's bytes in, then each lane takes its 124 bits
            for (uint32_t j = lane; j < count; j += 32)
                smb[j] = bbase[j];
            __syncwarp();
            if (valid) {
                const uint32_t bit = 124u * lane, q = bit >> 5, sh = bit & 31;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    rb[i] = sh ? (sb[warp][q + i] >> sh) | (sb[warp][q + i + 1] << (32 - sh)) : sb[warp][q + i];
                const uint8_t *pa = w.a + 5 * idx;
                ra[0] = (uint32_t)pa[0] | ((uint32_t)pa[1] << 8) | ((uint32_t)pa[2] << 16) | ((uint32_t)pa[3] << 24);
                ra[1] = pa[4];
                const uint8_t *pc = w.c + 60 * idx;
                if (w.cvec) {
#pragma unroll
                    for (int i = 0; i < 15; ++i)
                        rc[i] = reinterpret_cast<const uint32_t *>(pc)[i];
                } else {
#pragma unroll
                    for (int i = 0; i < 60; ++i)
                        rc[i >> 2] |= (uint32_t)pc[i] << (8 * (i & 3));
                }
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    *reinterpret_cast<uint32_t *>(at(w.ll, 2 * bi + r, W2, 2ull * bj)) =
                        pair16(get(ra, 20 * r, 10), get(ra, 20 * r + 10, 10));
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int width = k == 2 ? 11 : 10;
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int pos = 40 * k + 2 * r * width;
                        *reinterpret_cast<uint32_t *>(at(w.band[1][k], 2 * bi + r, W2, 2ull * bj)) =
                            pair16(get(rb, pos, width), get(rb, pos + width, width));
                    }
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int pos = 160 * k + 40 * r;
                        *reinterpret_cast<uint2 *>(at(w.band[0][k], 4 * bi + r, W1, 4ull * bj)) =
                            make_uint2(pair16(get(rc, pos, 10), get(rc, pos + 10, 10)),
                                       pair16(get(rc, pos + 20, 10), get(rc, pos + 30, 10)));
                    }
                }
            }
            __syncwarp();
        }
    }
}

} // namespace pk

cudaError_t launch_pack(bool fwd, const PackWork &w, uint32_t grid, cudaStream_t stream)
{
    if (fwd)
        pk::pack_kernel<true><<<grid, pk::kThreads, 0, stream>>>(w);
    else
        pk::pack_kernel<false><<<grid, pk::kThreads, 0, stream>>>(w);
    return cudaGetLastError();
}

} // namespace frag
