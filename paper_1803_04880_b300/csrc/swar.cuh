// swar.cuh -- packed-pair arithmetic and the row lifting of the LeGall 5/3
// filter shared by the streaming kernels.
//
// Packed pairs: each 16-bit half of a 32-bit word holds v + 0x4000 with
// |v| < 2^14, so the halves of (A + B) never carry into each other and both
// floors of a lifting step (Eq. 5.1 predict, Eq. 5.2 update) take one add, one
// shift and one mask for two columns.  Every half must hold such a value,
// even in lanes whose results are discarded: a half outside the range would
// carry into its neighbour.
#pragma once

#include <cstdint>

namespace frag {
namespace strm {

constexpr uint32_t kB2 = 0x40004000u;

__device__ __forceinline__ uint32_t pavg(uint32_t a, uint32_t b) { return ((a + b) >> 1) & 0x7fff7fffu; }
__device__ __forceinline__ uint32_t pq4(uint32_t a, uint32_t b)
{
    return ((a + b + 0x00020002u) >> 2) & 0x3fff3fffu;
}
__device__ __forceinline__ uint32_t to_i16x2(uint32_t w) { return (w + kB2) ^ 0x80008000u; }
__device__ __forceinline__ uint32_t from_i16x2(uint32_t w) { return (w ^ 0x80008000u) - kB2; }

struct Raw {
    uint32_t w[4];
};

// ---------------------------------------------------------------------------
// row lifting on packed pairs
// ---------------------------------------------------------------------------

// Lift one row along its length (Eq. 5.1 then Eq. 5.2) for the lane's four
// pairs at image columns c .. c+7: (x0, x2), (x1, x3), (x4, x6), (x5, x7) are
// formed with byte permutes; x8 and d[-1] come from the adjacent lanes.
// P[0] = (s0, s1), P[1] = (s2, s3), P[2] = (d0, d1), P[3] = (d2, d3), biased.
// BORDER: apply the symmetric extension where the row starts or ends.
template <bool BYTES, bool BORDER>
__device__ __forceinline__ void lift_row(const Raw &raw, int c, int Ws, bool edge, uint32_t (&P)[4])
{
    uint32_t e01, o01, e23, o23;
    if (BYTES) {
        // bytes into 16-bit halves with 0x40 as the high byte: v + 0x4000
        e01 = __byte_perm(raw.w[0], 0x40404040u, 0x4240);
        o01 = __byte_perm(raw.w[0], 0x40404040u, 0x4341);
        e23 = __byte_perm(raw.w[1], 0x40404040u, 0x4240);
        o23 = __byte_perm(raw.w[1], 0x40404040u, 0x4341);
    } else {
        e01 = __byte_perm(raw.w[0], raw.w[1], 0x5410);
        o01 = __byte_perm(raw.w[0], raw.w[1], 0x7632);
        e23 = __byte_perm(raw.w[2], raw.w[3], 0x5410);
        o23 = __byte_perm(raw.w[2], raw.w[3], 0x7632);
    }
    const uint32_t e01n = __shfl_down_sync(0xffffffffu, e01, 1); // (x8, x10) of the next lane
    uint32_t e12 = __byte_perm(e01, e23, 0x5432);                // (x2, x4)
    uint32_t e34 = __byte_perm(e23, e01n, 0x5432);               // (x6, x8)
    if (BORDER && edge) { // x[m] = x[m-2] for the pair that ends the row
        if (c + 2 == Ws)
            e12 = __byte_perm(e12, e01, 0x3254);
        if (c + 4 == Ws)
            e12 = __byte_perm(e12, e01, 0x7610);
        if (c + 6 == Ws)
            e34 = __byte_perm(e34, e23, 0x3254);
        if (c + 8 == Ws)
            e34 = __byte_perm(e34, e23, 0x7610);
    }
    const uint32_t d01 = o01 - pavg(e01, e12) + kB2; // Eq. 5.1
    const uint32_t d23 = o23 - pavg(e23, e34) + kB2;
    const uint32_t d23p = __shfl_up_sync(0xffffffffu, d23, 1); // (d2, d3) of the previous lane
    uint32_t dm0 = __byte_perm(d23p, d01, 0x5432);               // (d[-1], d0)
    if (BORDER && c == 0)
        dm0 = __byte_perm(d01, d01, 0x1010); // d[-1] = d[0]
    const uint32_t d12 = __byte_perm(d01, d23, 0x5432); // (d1, d2)
    P[0] = e01 + pq4(dm0, d01) - 0x20002000u; // Eq. 5.2
    P[1] = e23 + pq4(d12, d23) - 0x20002000u;
    P[2] = d01;
    P[3] = d23;
}

// Row inverse on packed pairs: w[0] = (L0, L1), w[1] = (L2, L3),
// w[2] = (H0, H1), w[3] = (H2, H3) -> samples (x0, x1), (x2, x3), (x4, x5),
// (x6, x7) of image columns c .. c+7.
template <bool BORDER>
__device__ __forceinline__ void unlift_row(const uint32_t (&w)[4], int c, int Ws, bool edge,
                                           uint32_t (&out)[4])
{
    const uint32_t h23p = __shfl_up_sync(0xffffffffu, w[3], 1);
    uint32_t hm0 = __byte_perm(h23p, w[2], 0x5432); // (H[-1], H0)
    if (BORDER && c == 0)
        hm0 = __byte_perm(w[2], w[2], 0x1010); // d[-1] = d[0]
    const uint32_t h12 = __byte_perm(w[2], w[3], 0x5432);
    const uint32_t e01 = w[0] - pq4(hm0, w[2]) + 0x20002000u; // undo Eq. 5.2
    const uint32_t e23 = w[1] - pq4(h12, w[3]) + 0x20002000u;
    const uint32_t e01n = __shfl_down_sync(0xffffffffu, e01, 1);
    uint32_t e12 = __byte_perm(e01, e23, 0x5432);
    uint32_t e34 = __byte_perm(e23, e01n, 0x5432);
    if (BORDER && edge) { // x[m] = x[m-2]
        if (c + 2 == Ws)
            e12 = __byte_perm(e12, e01, 0x3254);
        if (c + 4 == Ws)
            e12 = __byte_perm(e12, e01, 0x7610);
        if (c + 6 == Ws)
            e34 = __byte_perm(e34, e23, 0x3254);
        if (c + 8 == Ws)
            e34 = __byte_perm(e34, e23, 0x7610);
    }
    const uint32_t o01 = w[2] + pavg(e01, e12) - kB2; // undo Eq. 5.1
    const uint32_t o23 = w[3] + pavg(e23, e34) - kB2;
    out[0] = __byte_perm(e01, o01, 0x5410);
    out[1] = __byte_perm(e01, o01, 0x7632);
    out[2] = __byte_perm(e23, o23, 0x5410);
    out[3] = __byte_perm(e23, o23, 0x7632);
}

} // namespace strm
} // namespace frag
