// block_kernels.cu -- the block mode: every 8 x 8 block of the matrix is
// transformed as an image of its own (Sec. 5.2.1: each chunk is processed
// block by block, 8 x 8 in the thesis), up to three levels.
//
// One lane owns one block: it loads the block's 8 rows of 8 bytes (a warp
// takes 32 neighbouring blocks, so every row it reads is 256 contiguous
// bytes), runs every level in its registers and stores each band's tile of
// the block.  The symmetric extension applies at the block's own borders,
// so no lane needs another lane's samples: the mirrors x[8] = x[6] and
// d[-1] = d[0] are fixed byte permutes.  Rows before columns at every level
// (Eq. 5.1 predict, Eq. 5.2 update, Sec. 5.2.2), packed pairs as in the
// other kernels (each 16-bit half holds v + 0x4000).
//
// Band layout (as in the whole-matrix mode): band (l, k) is an H_l x W_l
// int16 image and block (bi, bj) fills rows [bi 8/2^l, (bi+1) 8/2^l) and
// columns [bj 8/2^l, (bj+1) 8/2^l) of it; LL_L - 128 goes to `ll`.  A
// packed buffer (two levels) instead gets the thesis's bit records of its
// three fragments straight from the registers (pack_bits.cuh): the lane
// writes its block's A and C records, the warp its 32 blocks' B records.
// A keyed buffer's B and C records are protected in the registers on the
// way out (and unprotected on the way in) with the keyed hashes of sha2.cuh.
#include "frag_internal.cuh"
#include "pack_bits.cuh"
#include "sha2.cuh"
#include "swar.cuh"

namespace frag {
namespace blk {

using strm::from_i16x2;
using strm::kB2;
using strm::pavg;
using strm::pq4;
using strm::to_i16x2;

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr uint32_t kQ4 = 0x20002000u; // the +2 of the update's floor, biased

// ---------------------------------------------------------------------------
// one row of the block, forward
// ---------------------------------------------------------------------------

// 8 bytes (w0, w1) -> P[0] = (s0, s1), P[1] = (s2, s3), P[2] = (d0, d1),
// P[3] = (d2, d3)
__device__ __forceinline__ void lift8(uint32_t w0, uint32_t w1, uint32_t (&P)[4])
{
    const uint32_t e01 = __byte_perm(w0, 0x40404040u, 0x4240); // (x0, x2)
    const uint32_t o01 = __byte_perm(w0, 0x40404040u, 0x4341); // (x1, x3)
    const uint32_t e23 = __byte_perm(w1, 0x40404040u, 0x4240); // (x4, x6)
    const uint32_t o23 = __byte_perm(w1, 0x40404040u, 0x4341); // (x5, x7)
    const uint32_t e12 = __byte_perm(e01, e23, 0x5432);         // (x2, x4)
    const uint32_t e34 = __byte_perm(e23, e23, 0x3232);         // (x6, x8 = x6)
    const uint32_t d01 = o01 - pavg(e01, e12) + kB2;            // Eq. 5.1
    const uint32_t d23 = o23 - pavg(e23, e34) + kB2;
    const uint32_t dm0 = __byte_perm(d01, d01, 0x1010);         // (d[-1] = d0, d0)
    const uint32_t d12 = __byte_perm(d01, d23, 0x5432);         // (d1, d2)
    P[0] = e01 + pq4(dm0, d01) - kQ4;                           // Eq. 5.2
    P[1] = e23 + pq4(d12, d23) - kQ4;
    P[2] = d01;
    P[3] = d23;
}

// 4 samples (w0 = (y0, y1), w1 = (y2, y3)) -> L = (s0, s1), H = (d0, d1)
__device__ __forceinline__ void lift4(uint32_t w0, uint32_t w1, uint32_t &L, uint32_t &H)
{
    const uint32_t e = __byte_perm(w0, w1, 0x5410);  // (y0, y2)
    const uint32_t o = __byte_perm(w0, w1, 0x7632);  // (y1, y3)
    const uint32_t es = __byte_perm(e, e, 0x3232);   // (y2, y4 = y2)
    const uint32_t d = o - pavg(e, es) + kB2;
    const uint32_t dm = __byte_perm(d, d, 0x1010);   // (d[-1] = d0, d0)
    L = e + pq4(dm, d) - kQ4;
    H = d;
}

// 2 samples z = (z0, z1) -> (s, d) in one word (s low, d high)
__device__ __forceinline__ uint32_t lift2(uint32_t z)
{
    const uint32_t e = z & 0xffffu, o = z >> 16;
    const uint32_t d = o - e + 0x4000u;                  // z2 = z0: o - floor((2 z0) / 2)
    const uint32_t s = e + ((2 * d + 2) >> 2) - 0x2000u; // d[-1] = d0
    return s | (d << 16);
}

// column lifting of R rows (R = 8, 4, 2) of NW words each, in place: rows
// become s rows 0..R/2-1 then d rows (per word; the top d[-1] = d[0] and the
// bottom x[R] = x[R-2] are the block's own borders)
template <int R, int NW>
__device__ __forceinline__ void col_lift(uint32_t (&x)[R][NW], uint32_t (&s)[R / 2][NW],
                                         uint32_t (&d)[R / 2][NW])
{
#pragma unroll
    for (int q = 0; q < R / 2; ++q)
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const uint32_t e1 = (2 * q + 2 < R) ? x[2 * q + 2][k] : x[2 * q][k];
            d[q][k] = x[2 * q + 1][k] - pavg(x[2 * q][k], e1) + kB2; // Eq. 5.1
        }
#pragma unroll
    for (int q = 0; q < R / 2; ++q)
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const uint32_t dm = q ? d[q - 1][k] : d[0][k];
            s[q][k] = x[2 * q][k] + pq4(dm, d[q][k]) - kQ4; // Eq. 5.2
        }
}

// inverse of col_lift: s, d rows -> R rows
template <int R, int NW>
__device__ __forceinline__ void col_unlift(const uint32_t (&s)[R / 2][NW], const uint32_t (&d)[R / 2][NW],
                                           uint32_t (&x)[R][NW])
{
#pragma unroll
    for (int q = 0; q < R / 2; ++q)
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const uint32_t dm = q ? d[q - 1][k] : d[0][k];
            x[2 * q][k] = s[q][k] - pq4(dm, d[q][k]) + kQ4; // undo Eq. 5.2
        }
#pragma unroll
    for (int q = 0; q < R / 2; ++q)
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const uint32_t e1 = (2 * q + 2 < R) ? x[2 * q + 2][k] : x[2 * q][k];
            x[2 * q + 1][k] = d[q][k] + pavg(x[2 * q][k], e1) - kB2; // undo Eq. 5.1
        }
}

// row inverses
__device__ __forceinline__ uint2 unlift8(const uint32_t (&w)[4])
{
    const uint32_t hm0 = __byte_perm(w[2], w[2], 0x1010); // (d[-1] = d0, d0)
    const uint32_t h12 = __byte_perm(w[2], w[3], 0x5432);
    const uint32_t e01 = w[0] - pq4(hm0, w[2]) + kQ4;     // undo Eq. 5.2
    const uint32_t e23 = w[1] - pq4(h12, w[3]) + kQ4;
    const uint32_t e12 = __byte_perm(e01, e23, 0x5432);
    const uint32_t e34 = __byte_perm(e23, e23, 0x3232);   // x8 = x6
    const uint32_t o01 = w[2] + pavg(e01, e12) - kB2;     // undo Eq. 5.1
    const uint32_t o23 = w[3] + pavg(e23, e34) - kB2;
    return make_uint2(__byte_perm(e01, o01, 0x6240), __byte_perm(e23, o23, 0x6240));
}

__device__ __forceinline__ void unlift4(uint32_t L, uint32_t H, uint32_t &w0, uint32_t &w1)
{
    const uint32_t hm = __byte_perm(H, H, 0x1010);
    const uint32_t e = L - pq4(hm, H) + kQ4;       // (y0, y2)
    const uint32_t es = __byte_perm(e, e, 0x3232); // (y2, y4 = y2)
    const uint32_t o = H + pavg(e, es) - kB2;      // (y1, y3)
    w0 = __byte_perm(e, o, 0x5410);
    w1 = __byte_perm(e, o, 0x7632);
}

__device__ __forceinline__ uint32_t unlift2(uint32_t w)
{
    const uint32_t s = w & 0xffffu, d = w >> 16;
    const uint32_t z0 = s - ((2 * d + 2) >> 2) + 0x2000u;
    const uint32_t z1 = d + z0 - 0x4000u;
    return z0 | (z1 << 16);
}

// ---------------------------------------------------------------------------
// band tiles
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ll_final(uint32_t w) { return to_i16x2(w - 0x00800080u); }

// row r of the tile (b values) of block (bi, bj) in an H_l x W_l int16 band
__device__ __forceinline__ uint8_t *tile_row(uint8_t *band, uint32_t Wl, uint32_t b, uint64_t bi,
                                             uint32_t bj, uint32_t r)
{
    return band + 2 * ((bi * b + r) * (uint64_t)Wl + (uint64_t)bj * b);
}

// b int16 values (w0, w1 as int16 pairs); `vec`: p is aligned to the store
__device__ __forceinline__ void st_tile(uint8_t *p, uint32_t b, uint32_t w0, uint32_t w1, bool vec)
{
    if (!vec) {
        const uint32_t h[4] = {w0 & 0xffffu, w0 >> 16, w1 & 0xffffu, w1 >> 16};
        for (uint32_t i = 0; i < b; ++i) {
            p[2 * i] = (uint8_t)h[i];
            p[2 * i + 1] = (uint8_t)(h[i] >> 8);
        }
    } else if (b == 4)
        __stcs(reinterpret_cast<uint2 *>(p), make_uint2(w0, w1));
    else if (b == 2)
        __stcs(reinterpret_cast<unsigned int *>(p), w0);
    else
        __stcs(reinterpret_cast<unsigned short *>(p), (unsigned short)w0);
}

__device__ __forceinline__ void ld_tile(const uint8_t *p, uint32_t b, uint32_t &w0, uint32_t &w1,
                                        bool vec)
{
    if (!vec) {
        uint32_t h[4] = {0, 0, 0, 0};
        for (uint32_t i = 0; i < b; ++i)
            h[i] = (uint32_t)__ldg(p + 2 * i) | ((uint32_t)__ldg(p + 2 * i + 1) << 8);
        w0 = h[0] | (h[1] << 16);
        w1 = h[2] | (h[3] << 16);
    } else if (b == 4) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        w0 = v.x;
        w1 = v.y;
    } else if (b == 2) {
        w0 = __ldg(reinterpret_cast<const unsigned int *>(p));
        w1 = 0;
    } else {
        w0 = __ldg(reinterpret_cast<const unsigned short *>(p));
        w1 = 0;
    }
}

// ---------------------------------------------------------------------------
// staged loads (the unpacked forward): each warp copies the rows of its next
// blocks into a ring of shared-memory stages with cp.async (each lane its own
// bytes, so no barrier), two blocks ahead of the one it computes
// ---------------------------------------------------------------------------
constexpr int kDepth = 3;
constexpr int kFwdStage = 8 * 256; // 8 rows x 32 lanes x 8 bytes

extern __shared__ __align__(16) uint8_t g_block_smem[];

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp8(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// plain loads of the ring (ordered after cp.async.wait_group by its memory clobber)
__device__ __forceinline__ const uint8_t *ring_ptr(uint32_t a)
{
    return g_block_smem + (a - smem_addr(g_block_smem));
}
__device__ __forceinline__ uint2 lds8(uint32_t a) { return *reinterpret_cast<const uint2 *>(ring_ptr(a)); }

// the block a lane works on, or none
struct Slot {
    const FuseBuf *b;
    uint64_t bi;
    uint32_t bj;
    bool on;  // the lane has a block in this unit
    bool vec; // aligned: staged loads and vector accesses
};

// single: the launch's lone descriptor, copied to shared memory by the block
// (a pointer to the kernel parameter itself would make the compiler copy the
// whole parameter block into local memory)
// A warp's units only grow, so it keeps the buffer its last unit fell in
// and that buffer's unit range: the next unit is usually found with one
// comparison instead of a binary search of dependent loads.
struct BufCursor {
    uint32_t lo = 0;
    uint64_t u_lo = 1, u_hi = 0; // empty: the first lookup searches
};

__device__ __forceinline__ uint32_t find_buf(const FuseWork &w, uint64_t u, BufCursor &c)
{
    if (u < c.u_lo || u >= c.u_hi) {
        uint32_t lo = 0, hi = w.nbufs;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(&w.bufs[mid].unit0) <= u)
                lo = mid;
            else
                hi = mid;
        }
        c.lo = lo;
        c.u_lo = __ldg(&w.bufs[lo].unit0);
        c.u_hi = lo + 1 < w.nbufs ? __ldg(&w.bufs[lo + 1].unit0) : w.total_units;
    }
    return c.lo;
}

__device__ __forceinline__ const FuseBuf *unit_buf(const FuseWork &w, const FuseBuf *single, uint64_t u,
                                                  uint64_t &local, BufCursor &c)
{
    if (w.nbufs == 1) {
        local = u;
        return single;
    }
    const uint32_t lo = find_buf(w, u, c);
    local = u - c.u_lo;
    return &w.bufs[lo];
}

// one unit = one block row of 32 blocks (a warp), lane = block column
__device__ __forceinline__ Slot slot_of(const FuseWork &w, const FuseBuf *single, uint64_t u, int lane,
                                       BufCursor &c)
{
    Slot sl;
    sl.on = false;
    sl.vec = false;
    sl.b = nullptr;
    sl.bi = 0;
    sl.bj = 0;
    if (u >= w.total_units)
        return sl;
    uint64_t local;
    sl.b = unit_buf(w, single, u, local, c);
    const uint32_t strips = sl.b->strips;
    if (local < (1ull << 32)) { // 32-bit division: a unit is one warp's 32 blocks, so it counts
        const uint32_t l32 = (uint32_t)local, q = l32 / strips;
        sl.bi = q;
        sl.bj = (l32 - q * strips) * 32 + lane;
    } else {
        sl.bi = local / strips;
        sl.bj = (uint32_t)(local % strips) * 32 + lane;
    }
    sl.on = sl.bj * 8 < sl.b->W;
    sl.vec = sl.b->vec != 0;
    return sl;
}

__device__ __forceinline__ void fwd_issue(const Slot &sl, uint32_t st)
{
    if (sl.on && sl.vec) {
        const FuseBuf &f = *sl.b;
        const uint64_t base = sl.bi * 8 * f.W + (uint64_t)sl.bj * 8;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint64_t off = base + (uint64_t)r * f.W;
            const uint32_t bytes = off >= f.n ? 0u : (uint32_t)(f.n - off < 8 ? f.n - off : 8);
            cp8(st + 256 * r, bytes ? f.src + off : f.src, bytes);
        }
    }
    cp_commit();
}

// ---------------------------------------------------------------------------
// one block, forward and inverse (rows from the stage, or straight from
// global memory with byte accesses when the buffer is not aligned)
// ---------------------------------------------------------------------------
// the block's 8 rows of 8 bytes from the stage, or straight from global
// memory (8-byte loads where the row is whole data and aligned)
__device__ __forceinline__ void block_rows(const FuseBuf &f, uint64_t bi, uint32_t bj, bool staged, bool vec8,
                                           uint32_t st, uint2 (&v)[8])
{
    const uint32_t W = f.W;
    const uint64_t base = bi * 8 * W + (uint64_t)bj * 8;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if (staged) {
            v[r] = lds8(st + 256 * r);
        } else if (vec8 && bi * 8 + r < f.full_rows) {
            v[r] = __ldg(reinterpret_cast<const uint2 *>(f.src + base + (uint64_t)r * W));
        } else {
            const uint64_t off = base + (uint64_t)r * W;
            uint32_t b8[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                b8[i] = off + i < f.n ? (uint32_t)__ldg(f.src + off + i) : 0u;
            v[r].x = b8[0] | (b8[1] << 8) | (b8[2] << 16) | (b8[3] << 24);
            v[r].y = b8[4] | (b8[5] << 8) | (b8[6] << 16) | (b8[7] << 24);
        }
    }
}

// VEC: the buffer's tiles are aligned to their vector widths (a compile-time
// choice, so the unaligned byte path is not issued under predicates beside
// the vector stores)
template <bool VEC>
__device__ __forceinline__ void fwd_block(const FuseBuf &f, uint64_t bi, uint32_t bj, const uint2 (&v)[8])
{
    const uint32_t W = f.W, L = f.F;
    uint32_t x1[8][4]; // row-lifted rows, 4 words each
#pragma unroll
    for (int r = 0; r < 8; ++r)
        lift8(v[r].x, v[r].y, x1[r]);
    uint32_t s1[4][4], d1[4][4];
    col_lift<8, 4>(x1, s1, d1);
    // level-1 tiles: LL_1 = s1[][0..1], HL_1 = s1[][2..3], LH_1 = d1[][0..1], HH_1 = d1[][2..3]
    const uint32_t W1 = W >> 1;
    constexpr bool vec = VEC;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        st_tile(tile_row(f.band[0][0], W1, 4, bi, bj, r), 4, to_i16x2(s1[r][2]), to_i16x2(s1[r][3]), vec);
        st_tile(tile_row(f.band[0][1], W1, 4, bi, bj, r), 4, to_i16x2(d1[r][0]), to_i16x2(d1[r][1]), vec);
        st_tile(tile_row(f.band[0][2], W1, 4, bi, bj, r), 4, to_i16x2(d1[r][2]), to_i16x2(d1[r][3]), vec);
    }
    if (L == 1) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
            st_tile(tile_row(f.ll, W1, 4, bi, bj, r), 4, ll_final(s1[r][0]), ll_final(s1[r][1]), vec);
        return;
    }
    // level 2 on the 4 x 4 LL_1
    uint32_t x2[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        lift4(s1[r][0], s1[r][1], x2[r][0], x2[r][1]);
    uint32_t s2[2][2], d2[2][2];
    col_lift<4, 2>(x2, s2, d2);
    const uint32_t W2 = W >> 2;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        st_tile(tile_row(f.band[1][0], W2, 2, bi, bj, r), 2, to_i16x2(s2[r][1]), 0, vec);
        st_tile(tile_row(f.band[1][1], W2, 2, bi, bj, r), 2, to_i16x2(d2[r][0]), 0, vec);
        st_tile(tile_row(f.band[1][2], W2, 2, bi, bj, r), 2, to_i16x2(d2[r][1]), 0, vec);
    }
    if (L == 2) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
            st_tile(tile_row(f.ll, W2, 2, bi, bj, r), 2, ll_final(s2[r][0]), 0, vec);
        return;
    }
    // level 3 on the 2 x 2 LL_2: one (s, d) word per row
    uint32_t x3[2][1];
    x3[0][0] = lift2(s2[0][0]);
    x3[1][0] = lift2(s2[1][0]);
    uint32_t s3[1][1], d3[1][1];
    col_lift<2, 1>(x3, s3, d3);
    const uint32_t W3 = W >> 3;
    const uint32_t sw = to_i16x2(s3[0][0]), dw = to_i16x2(d3[0][0]);
    st_tile(tile_row(f.band[2][0], W3, 1, bi, bj, 0), 1, sw >> 16, 0, vec); // HL_3
    st_tile(tile_row(f.band[2][1], W3, 1, bi, bj, 0), 1, dw, 0, vec);       // LH_3
    st_tile(tile_row(f.band[2][2], W3, 1, bi, bj, 0), 1, dw >> 16, 0, vec); // HH_3
    st_tile(tile_row(f.ll, W3, 1, bi, bj, 0), 1, ll_final(s3[0][0]), 0, vec);
}

template <bool VEC>
__device__ __forceinline__ void inv_block(const FuseBuf &f, uint64_t bi, uint32_t bj)
{
    constexpr bool vec = VEC;
    const uint32_t W = f.W, L = f.F;
    const uint32_t W1 = W >> 1, W2 = W >> 2, W3 = W >> 3;
    uint32_t s1[4][4], d1[4][4];
    // LL_1: from the input (one level) or from the levels above
    if (L >= 2) {
        uint32_t s2[2][2], d2[2][2];
        if (L == 3) {
            uint32_t a, b, c, e, z;
            ld_tile(tile_row(f.ll, W3, 1, bi, bj, 0), 1, a, z, vec);
            ld_tile(tile_row(f.band[2][0], W3, 1, bi, bj, 0), 1, b, z, vec);
            ld_tile(tile_row(f.band[2][1], W3, 1, bi, bj, 0), 1, c, z, vec);
            ld_tile(tile_row(f.band[2][2], W3, 1, bi, bj, 0), 1, e, z, vec);
            uint32_t s3[1][1], d3[1][1], x3[2][1];
            s3[0][0] = from_i16x2(a | (b << 16)) + 0x80u;
            d3[0][0] = from_i16x2(c | (e << 16));
            col_unlift<2, 1>(s3, d3, x3);
            s2[0][0] = unlift2(x3[0][0]);
            s2[1][0] = unlift2(x3[1][0]);
        } else {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                uint32_t w, z;
                ld_tile(tile_row(f.ll, W2, 2, bi, bj, r), 2, w, z, vec);
                s2[r][0] = from_i16x2(w) + 0x00800080u;
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            uint32_t w[3], z;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                ld_tile(tile_row(f.band[1][k], W2, 2, bi, bj, r), 2, w[k], z, vec);
            s2[r][1] = from_i16x2(w[0]);
            d2[r][0] = from_i16x2(w[1]);
            d2[r][1] = from_i16x2(w[2]);
        }
        uint32_t x2[4][2];
        col_unlift<4, 2>(s2, d2, x2);
#pragma unroll
        for (int r = 0; r < 4; ++r)
            unlift4(x2[r][0], x2[r][1], s1[r][0], s1[r][1]);
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint32_t a, b;
            ld_tile(tile_row(f.ll, W1, 4, bi, bj, r), 4, a, b, vec);
            s1[r][0] = from_i16x2(a) + 0x00800080u;
            s1[r][1] = from_i16x2(b) + 0x00800080u;
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        uint32_t v[3][2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            ld_tile(tile_row(f.band[0][k], W1, 4, bi, bj, r), 4, v[k][0], v[k][1], vec);
        s1[r][2] = from_i16x2(v[0][0]);
        s1[r][3] = from_i16x2(v[0][1]);
        d1[r][0] = from_i16x2(v[1][0]);
        d1[r][1] = from_i16x2(v[1][1]);
        d1[r][2] = from_i16x2(v[2][0]);
        d1[r][3] = from_i16x2(v[2][1]);
    }
    uint32_t x1[8][4];
    col_unlift<8, 4>(s1, d1, x1);
    const uint64_t base = bi * 8 * W + (uint64_t)bj * 8;
    const bool whole = bi * 8 + 8 <= f.full_rows && vec;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const uint2 v = unlift8(x1[r]);
        const uint64_t off = base + (uint64_t)r * W;
        if (whole) {
            __stcs(reinterpret_cast<uint2 *>(f.out + off), v);
        } else {
            for (int i = 0; i < 8 && off + i < f.n; ++i)
                f.out[off + i] = (uint8_t)((i < 4 ? v.x : v.y) >> (8 * (i & 3)));
        }
    }
}

// ---------------------------------------------------------------------------
// the packed forward (Sec. 5.2.3's records of two-level 8 x 8 blocks)
//
// A unit is a warp's 32 neighbouring blocks of a block row, one a lane.  Its
// descriptor fields are decoded once into registers (a lone buffer's straight
// from the kernel parameter), the next unit's rows are fetched into registers
// while the current one is transformed, and a unit whose 8 rows are whole
// data takes its loads without per-row tests.
// ---------------------------------------------------------------------------
struct PkUnit {
    const uint8_t *src;  // forward: the block's first byte (bi 8 W + bj 8 of the buffer)
    uint8_t *out;        // inverse: the same byte of the recovered buffer
    uint8_t *pa, *pb, *pc; // the unit's A, B and C record areas
    uint64_t n_left;     // data bytes from the block's first byte on
    uint64_t idx;        // the block's index (keyed hash input)
    uint64_t nonce;
    uint32_t W;
    uint32_t nvalid;     // blocks of the unit (0: no unit)
    bool on;             // the lane has a block
    bool whole;          // every row of the unit is data, 8-byte aligned
    bool keyed;
};

__device__ __forceinline__ uint64_t ldg64(const void *p)
{
    return __ldg(reinterpret_cast<const unsigned long long *>(p));
}

template <bool FWD>
__device__ __forceinline__ PkUnit pk_unit(const FuseWork &w, uint64_t u, int lane, BufCursor &c)
{
    PkUnit p;
    p.nvalid = 0;
    p.on = p.whole = p.keyed = false;
    p.src = nullptr;
    p.out = p.pa = p.pb = p.pc = nullptr;
    p.n_left = p.idx = p.nonce = 0;
    p.W = 8;
    if (u >= w.total_units)
        return p;
    const FuseBuf *bp = nullptr; // null: the launch's lone buffer (w.single)
    uint64_t local = u;
    if (w.nbufs != 1) {
        bp = w.bufs + find_buf(w, u, c);
        local = u - c.u_lo;
    }
    const uint8_t *src;
    uint8_t *k0, *k1, *k2;
    uint64_t n, nonce;
    uint32_t W, strips, full_rows, vec, keyed;
    if (bp) {
        src = reinterpret_cast<const uint8_t *>(ldg64(FWD ? (const void *)&bp->src : (const void *)&bp->out));
        k0 = reinterpret_cast<uint8_t *>(ldg64(&bp->pk[0]));
        k1 = reinterpret_cast<uint8_t *>(ldg64(&bp->pk[1]));
        k2 = reinterpret_cast<uint8_t *>(ldg64(&bp->pk[2]));
        n = ldg64(&bp->n);
        nonce = ldg64(&bp->nonce);
        W = __ldg(&bp->W);
        strips = __ldg(&bp->strips);
        full_rows = __ldg(&bp->full_rows);
        vec = __ldg(&bp->vec);
        keyed = __ldg(&bp->keyed);
    } else {
        src = FWD ? w.single.src : w.single.out;
        k0 = w.single.pk[0];
        k1 = w.single.pk[1];
        k2 = w.single.pk[2];
        n = w.single.n;
        nonce = w.single.nonce;
        W = w.single.W;
        strips = w.single.strips;
        full_rows = w.single.full_rows;
        vec = w.single.vec;
        keyed = w.single.keyed;
    }
    uint64_t bi;
    uint32_t s;
    if (local < (1ull << 32)) {
        const uint32_t l32 = (uint32_t)local, q = l32 / strips;
        bi = q;
        s = l32 - q * strips;
    } else {
        bi = local / strips;
        s = (uint32_t)(local % strips);
    }
    const uint32_t nbx = W >> 3, bj = 32 * s + (uint32_t)lane;
    p.W = W;
    p.nvalid = min(32u, nbx - 32 * s);
    p.on = bj < nbx;
    const uint64_t idx0 = bi * (uint64_t)nbx + 32ull * s;
    p.idx = idx0 + (uint64_t)lane;
    const uint64_t off = bi * 8 * (uint64_t)W + 8ull * bj;
    p.n_left = off < n ? n - off : 0;
    p.src = src + off;
    p.out = const_cast<uint8_t *>(src) + off;
    p.pa = k0 + 5 * idx0;
    p.pb = k1 + bi * pkb::b_row_bytes(nbx) + 496ull * s;
    p.pc = k2 + 60 * idx0;
    p.whole = vec != 0 && bi * 8 + 8 <= (uint64_t)full_rows;
    p.keyed = keyed != 0;
    p.nonce = nonce;
    return p;
}

// the lane's 8 rows of 8 bytes (bytes past the data read as zero)
__device__ __forceinline__ void pk_rows(const PkUnit &p, uint2 (&v)[8])
{
    if (p.whole) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            v[r] = __ldg(reinterpret_cast<const uint2 *>(p.src + (uint64_t)r * p.W));
        return;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        v[r] = make_uint2(0u, 0u);
        if (!p.on)
            continue;
        const uint64_t o = (uint64_t)r * p.W;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (o + i < p.n_left) {
                const uint32_t b = (uint32_t)__ldg(p.src + o + i) << (8 * (i & 3));
                if (i < 4)
                    v[r].x |= b;
                else
                    v[r].y |= b;
            }
    }
}

// The block's two levels and its three records in registers.  Only the
// level-2 values are range-checked: every level-1 detail of bytes is within
// +-510 (row predict d in [-255, 255], row update s in [-127, 383]; the
// column steps then give HH = d - floor((d + d') / 2), HL = d +
// floor((HH + HH' + 2) / 4) and LH = s - floor((s + s') / 2), each in
// [-510, 510]), so it always fits its 10 bits.
template <bool KEYED>
__device__ __forceinline__ void pk_block(const uint2 (&v)[8], bool keyed, const uint32_t (&key)[4],
                                         uint64_t nonce, uint64_t idx, uint32_t (&ra)[2], uint32_t (&rb)[4],
                                         uint32_t (&rc)[15], uint32_t &bad)
{
    uint32_t x1[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
        lift8(v[r].x, v[r].y, x1[r]);
    uint32_t s1[4][4], d1[4][4];
    col_lift<8, 4>(x1, s1, d1);
    uint32_t x2[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        lift4(s1[r][0], s1[r][1], x2[r][0], x2[r][1]);
    uint32_t s2[2][2], d2[2][2];
    col_lift<4, 2>(x2, s2, d2);
    ra[0] = ra[1] = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        rb[i] = 0u;
#pragma unroll
    for (int i = 0; i < 15; ++i)
        rc[i] = 0u;
    bad = 0u;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const uint32_t a = s2[r][0] - 0x00800080u; // LL_2 - 128
        bad |= pkb::range_bits<10>(a) | pkb::range_bits<10>(s2[r][1]) | pkb::range_bits<10>(d2[r][0]) |
               pkb::range_bits<11>(d2[r][1]);
        pkb::ins(ra, 20 * r, pkb::field2<10>(a), 20);
        pkb::ins(rb, 20 * r, pkb::field2<10>(s2[r][1]), 20);      // HL_2
        pkb::ins(rb, 40 + 20 * r, pkb::field2<10>(d2[r][0]), 20); // LH_2
        pkb::ins(rb, 80 + 22 * r, pkb::field2<11>(d2[r][1]), 22); // HH_2
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        pkb::ins(rc, 40 * r, pkb::field2<10>(s1[r][2]), 20); // HL_1
        pkb::ins(rc, 40 * r + 20, pkb::field2<10>(s1[r][3]), 20);
        pkb::ins(rc, 160 + 40 * r, pkb::field2<10>(d1[r][0]), 20); // LH_1
        pkb::ins(rc, 180 + 40 * r, pkb::field2<10>(d1[r][1]), 20);
        pkb::ins(rc, 320 + 40 * r, pkb::field2<10>(d1[r][2]), 20); // HH_1
        pkb::ins(rc, 340 + 40 * r, pkb::field2<10>(d1[r][3]), 20);
    }
    if (KEYED && keyed) { // B' = B ^ H1(A), then C' = C ^ H2(B')
        sha::mask_b(key, nonce, idx, ra, rb);
        sha::mask_c(key, nonce, idx, rb, rc);
    }
}

// Every unit of a packed launch, forward: the lane transforms its block
// while the next unit's rows load, writes its A and C records into the
// warp's staging area (C at word 15 lane: conflict-free) and its B record
// into the warp's shuffle-built chunks, and the warp moves the unit's
// records with 16-byte stores.
template <bool KEYED>
__device__ __forceinline__ void packed_fwd(const FuseWork &w, const uint32_t (&key)[4])
{
    __shared__ uint32_t sb[kWarps][pkb::kPackBWords]; // B records of an unaligned unit
    __shared__ pkb::Stage stg_all[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    pkb::Stage &stg = stg_all[warp];
    const uint64_t G = (uint64_t)gridDim.x * kWarps;
    uint64_t u = (uint64_t)blockIdx.x * kWarps + warp;
    // one unit, whose rows are in v (the next unit's are loading)
    auto unit = [&](const PkUnit &cur, const uint2 (&v)[8]) {
        uint32_t ra[2], rb[4], rc[15], bad;
        pk_block<KEYED>(v, cur.keyed, key, cur.nonce, cur.idx, ra, rb, rc, bad);
        if (bad && cur.on)
            atomicCAS(w.err, 0, pkb::kErrWidth);
        if (!cur.on) { // the B chunks take a lane without a block as zeros
#pragma unroll
            for (int i = 0; i < 4; ++i)
                rb[i] = 0u;
        }
        uint8_t *sa = stg.a + 5 * lane;
        sa[0] = (uint8_t)ra[0];
        sa[1] = (uint8_t)(ra[0] >> 8);
        sa[2] = (uint8_t)(ra[0] >> 16);
        sa[3] = (uint8_t)(ra[0] >> 24);
        sa[4] = (uint8_t)ra[1];
#pragma unroll
        for (int i = 0; i < 15; ++i)
            stg.c[15 * lane + i] = rc[i];
        pkb::put_b(sb[warp], cur.pb, (124 * cur.nvalid + 7) / 8, cur.on, lane, rb);
        __syncwarp();
        if (pkb::full_aligned(cur.nvalid, cur.pa, cur.pb, cur.pc)) {
            pkb::copy_out_full(cur.pa, cur.pc, stg, lane);
        } else {
            pkb::copy_out(cur.pa, stg.a, 5 * cur.nvalid, lane);
            pkb::copy_out(cur.pc, reinterpret_cast<const uint8_t *>(stg.c), 60 * cur.nvalid, lane);
        }
        __syncwarp(); // every lane is done with the staging area before it is refilled
    };
    BufCursor bc;
    PkUnit cur = pk_unit<true>(w, u, lane, bc);
    uint2 rows[8];
    pk_rows(cur, rows);
    for (; u < w.total_units; u += G) {
        uint2 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r)
            v[r] = rows[r];
        BufCursor fresh; // keyed launches keep no cursor across units (registers)
        const PkUnit nx = pk_unit<true>(w, u + G, lane, KEYED ? fresh : bc);
        pk_rows(nx, rows);
        unit(cur, v);
        cur = nx;
    }
}

// The block's records (A deciphered and C from the warp's staging area, B
// from the warp) back to its 8 rows of bytes: both levels undone in the
// registers, the rows stored straight from them.
template <bool KEYED>
__device__ __forceinline__ void pk_inv_block(const PkUnit &p, const pkb::StageIn &st, const uint32_t (&rb_in)[4],
                                             const uint32_t (&key)[4], int lane)
{
    const uint8_t *sa = st.a + 5 * lane;
    const uint32_t ra[2] = {(uint32_t)sa[0] | ((uint32_t)sa[1] << 8) | ((uint32_t)sa[2] << 16) |
                                ((uint32_t)sa[3] << 24),
                            (uint32_t)sa[4]};
    uint32_t rc[15];
#pragma unroll
    for (int i = 0; i < 15; ++i)
        rc[i] = st.c[15 * lane + i];
    uint32_t rb[4] = {rb_in[0], rb_in[1], rb_in[2], rb_in[3]};
    if (KEYED && p.keyed) { // C = C' ^ H2(B') first, then B = B' ^ H1(A)
        sha::mask_c(key, p.nonce, p.idx, rb, rc);
        sha::mask_b(key, p.nonce, p.idx, ra, rb);
    }
    uint32_t s1[4][4], d1[4][4];
    uint32_t s2[2][2], d2[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        s2[r][0] = pkb::unfield2<10>(pkb::ext(ra, 20 * r, 20)) + 0x00800080u;
        s2[r][1] = pkb::unfield2<10>(pkb::ext(rb, 20 * r, 20));
        d2[r][0] = pkb::unfield2<10>(pkb::ext(rb, 40 + 20 * r, 20));
        d2[r][1] = pkb::unfield2<11>(pkb::ext(rb, 80 + 22 * r, 22));
    }
    uint32_t x2[4][2];
    col_unlift<4, 2>(s2, d2, x2);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        unlift4(x2[r][0], x2[r][1], s1[r][0], s1[r][1]);
        s1[r][2] = pkb::unfield2<10>(pkb::ext(rc, 40 * r, 20));
        s1[r][3] = pkb::unfield2<10>(pkb::ext(rc, 40 * r + 20, 20));
        d1[r][0] = pkb::unfield2<10>(pkb::ext(rc, 160 + 40 * r, 20));
        d1[r][1] = pkb::unfield2<10>(pkb::ext(rc, 180 + 40 * r, 20));
        d1[r][2] = pkb::unfield2<10>(pkb::ext(rc, 320 + 40 * r, 20));
        d1[r][3] = pkb::unfield2<10>(pkb::ext(rc, 340 + 40 * r, 20));
    }
    uint32_t x1[8][4];
    col_unlift<8, 4>(s1, d1, x1);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const uint2 v = unlift8(x1[r]);
        const uint64_t o = (uint64_t)r * p.W;
        if (p.whole) {
            __stcs(reinterpret_cast<uint2 *>(p.out + o), v);
        } else {
            for (int i = 0; i < 8 && o + i < p.n_left; ++i)
                p.out[o + i] = (uint8_t)((i < 4 ? v.x : v.y) >> (8 * (i & 3)));
        }
    }
}

// Every unit of a packed launch, inverse: the warp fetches the next unit's
// A, B and C records into the other of its two staging areas with cp.async
// (a full warp whose three areas are 16-byte aligned; other units load
// synchronously) while the current unit is transformed.
template <bool KEYED>
__device__ __forceinline__ void packed_inv(const FuseWork &w, const uint32_t (&key)[4])
{
    __shared__ uint32_t sb[kWarps][pkb::kPackBWords];
    __shared__ pkb::StageIn stg_in[kWarps][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t G = (uint64_t)gridDim.x * kWarps;
    uint64_t u = (uint64_t)blockIdx.x * kWarps + warp;
    // one unit, whose records (when `full`) are landing in `st`; the next
    // unit's group was committed after this one's
    auto unit = [&](const PkUnit &cur, bool full, pkb::StageIn &st) {
        cp_wait<1>(); // this unit's group has landed
        __syncwarp();
        uint32_t rb[4] = {0u, 0u, 0u, 0u};
        if (full) {
            pkb::b_from_stage(st, cur.on, lane, rb);
        } else {
            pkb::get_b(sb[warp], cur.pb, (124 * cur.nvalid + 7) / 8, cur.on, lane, rb);
            pkb::copy_in(st.a, cur.pa, 5 * cur.nvalid, lane);
            pkb::copy_in(reinterpret_cast<uint8_t *>(st.c), cur.pc, 60 * cur.nvalid, lane);
            __syncwarp();
        }
        if (cur.on)
            pk_inv_block<KEYED>(cur, st, rb, key, lane);
        __syncwarp(); // every lane is done with this area before it is refilled
    };
    BufCursor bc;
    PkUnit cur = pk_unit<false>(w, u, lane, bc);
    bool cur_full = pkb::full_aligned(cur.nvalid, cur.pa, cur.pb, cur.pc);
    if (cur_full)
        pkb::prefetch_full(stg_in[warp][0], cur.pa, cur.pb, cur.pc, lane);
    cp_commit();
    for (uint32_t i = 0; u < w.total_units; u += G, ++i) {
        BufCursor fresh; // keyed launches keep no cursor across units (registers)
        const PkUnit nx = pk_unit<false>(w, u + G, lane, KEYED ? fresh : bc);
        const bool nx_full = pkb::full_aligned(nx.nvalid, nx.pa, nx.pb, nx.pc);
        if (nx_full)
            pkb::prefetch_full(stg_in[warp][(i + 1) & 1], nx.pa, nx.pb, nx.pc, lane);
        cp_commit();
        unit(cur, cur_full, stg_in[warp][i & 1]);
        cur = nx;
        cur_full = nx_full;
    }
    cp_wait<0>();
}

// The unpacked inverse reads four times as many tiles per block as the
// forward; it runs best with direct loads and many warps, the unpacked
// forward with the ring.  Packed launches run their own loops (packed_fwd,
// packed_inv): every buffer of such a launch is packed.
#ifndef BLOCK_PACKED_FWD_MINB
#define BLOCK_PACKED_FWD_MINB 5
#endif
#ifndef BLOCK_PACKED_INV_MINB
#define BLOCK_PACKED_INV_MINB 6
#endif
#ifndef BLOCK_FWD_MINB
#define BLOCK_FWD_MINB 6
#endif
#ifndef BLOCK_INV_MINB
#define BLOCK_INV_MINB 8
#endif
template <bool FWD, bool PACKED>
__host__ __device__ constexpr int block_min_ctas(bool keyed)
{
    return keyed ? 1 : PACKED ? (FWD ? BLOCK_PACKED_FWD_MINB : BLOCK_PACKED_INV_MINB)
                              : (FWD ? BLOCK_FWD_MINB : BLOCK_INV_MINB);
}
// the packed forward: five 4-warp blocks an SM (registers capped at 102);
// the packed inverse: six (capped at 85); the unpacked forward six, its
// inverse (direct loads, latency-bound) eight (capped at 64)
template <bool FWD, bool PACKED, bool KEYED>
__global__ void __launch_bounds__(kThreads, block_min_ctas<FWD, PACKED>(KEYED))
    block_kernel(FuseWork w)
{
    __shared__ FuseBuf s_single;
    if (threadIdx.x == 0)
        s_single = w.single;
    __syncthreads();
    uint32_t key[4] = {0u, 0u, 0u, 0u}; // the AES key's words, big-endian (keyed buffers)
    if (KEYED) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            key[i] = __ldg(w.key_words + i);
    }
    if (PACKED && !FWD) {
        grid_release();
        packed_inv<KEYED>(w, key);
        return;
    }
    if (FWD && PACKED) {
        grid_release();
        packed_fwd<KEYED>(w, key);
        return;
    }
    if (!FWD) { // the unpacked inverse: direct loads
        grid_release();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const uint64_t G = (uint64_t)gridDim.x * kWarps;
        BufCursor bc;
        for (uint64_t u = (uint64_t)blockIdx.x * kWarps + warp; u < w.total_units; u += G) {
            const Slot sl = slot_of(w, &s_single, u, lane, bc);
            if (sl.on) {
                if (sl.vec)
                    inv_block<true>(*sl.b, sl.bi, sl.bj);
                else
                    inv_block<false>(*sl.b, sl.bi, sl.bj);
            }
        }
        return;
    }
    // the unpacked forward: the rows of each unit staged with cp.async two
    // units ahead.  The next kernel (the CTR pass after a protect) may start
    // its data-independent part now; it waits for this grid before reading
    grid_release();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t stage = kFwdStage;
    const uint32_t ring = smem_addr(g_block_smem) + (uint32_t)warp * kDepth * stage;
    const uint32_t ring8 = ring + 8u * lane;
    const uint64_t G = (uint64_t)gridDim.x * kWarps;
    const uint64_t u0 = (uint64_t)blockIdx.x * kWarps + warp;
    static_assert(kDepth == 3, "the unit loop below is unrolled for three stages");
    // the blocks of the units in flight, in stages 0, 1, 2 (static indices
    // keep them in registers)
    BufCursor bc;
    Slot q0 = slot_of(w, &s_single, u0, lane, bc), q1 = slot_of(w, &s_single, u0 + G, lane, bc), q2;
    fwd_issue(q0, ring8);
    fwd_issue(q1, ring8 + stage);
    // unit i computes from stage i % 3 after issuing unit i + 2 into stage
    // (i + 2) % 3, the one unit i - 1 freed
    auto step = [&](uint64_t i, Slot &cur, Slot &ahead, int cur_k, int ahead_k) {
        ahead = slot_of(w, &s_single, u0 + (i + 2) * G, lane, bc);
        fwd_issue(ahead, ring8 + (uint32_t)ahead_k * stage);
        cp_wait<kDepth - 1>();
        if (cur.on) {
            const FuseBuf &f = *cur.b;
            uint2 v[8];
            block_rows(f, cur.bi, cur.bj, cur.vec, false, ring8 + (uint32_t)cur_k * stage, v);
            if (cur.vec)
                fwd_block<true>(f, cur.bi, cur.bj, v);
            else
                fwd_block<false>(f, cur.bi, cur.bj, v);
        }
    };
    for (uint64_t i = 0; u0 + i * G < w.total_units; i += 3) {
        step(i, q0, q2, 0, 2);
        if (u0 + (i + 1) * G >= w.total_units)
            break;
        step(i + 1, q1, q0, 1, 0);
        if (u0 + (i + 2) * G >= w.total_units)
            break;
        step(i + 2, q2, q1, 2, 1);
    }
    cp_wait<0>();
}

size_t smem_bytes(bool fwd, bool packed) { return fwd && !packed ? (size_t)kWarps * kDepth * kFwdStage : 0; }

template <bool FWD, bool PACKED, bool KEYED>
cudaError_t set_attr()
{
    static std::atomic<uint64_t> done{0};
    return smem_attr_once((const void *)block_kernel<FWD, PACKED, KEYED>, (int)smem_bytes(FWD, PACKED), done);
}

template <bool FWD, bool PACKED, bool KEYED>
cudaError_t launch(const FuseWork &w, uint32_t grid, cudaStream_t stream)
{
    cudaError_t e = set_attr<FWD, PACKED, KEYED>();
    if (e != cudaSuccess)
        return e;
    block_kernel<FWD, PACKED, KEYED><<<grid, kThreads, smem_bytes(FWD, PACKED), stream>>>(w);
    return cudaGetLastError();
}

template <bool FWD, bool PACKED, bool KEYED>
cudaError_t occupancy(int *blocks_per_sm)
{
    cudaError_t e = set_attr<FWD, PACKED, KEYED>();
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, (const void *)block_kernel<FWD, PACKED, KEYED>, kThreads, smem_bytes(FWD, PACKED));
}

template <bool FWD>
cudaError_t launch_dir(bool packed, bool keyed, const FuseWork &w, uint32_t grid, cudaStream_t stream)
{
    if (!packed)
        return launch<FWD, false, false>(w, grid, stream);
    return keyed ? launch<FWD, true, true>(w, grid, stream) : launch<FWD, true, false>(w, grid, stream);
}

template <bool FWD>
cudaError_t occupancy_dir(bool packed, bool keyed, int *blocks_per_sm)
{
    if (!packed)
        return occupancy<FWD, false, false>(blocks_per_sm);
    return keyed ? occupancy<FWD, true, true>(blocks_per_sm) : occupancy<FWD, true, false>(blocks_per_sm);
}

} // namespace blk

cudaError_t launch_blocks(bool fwd, bool packed, bool keyed, const FuseWork &w, uint32_t grid,
                          cudaStream_t stream)
{
    return fwd ? blk::launch_dir<true>(packed, keyed, w, grid, stream)
               : blk::launch_dir<false>(packed, keyed, w, grid, stream);
}

cudaError_t block_occupancy(bool fwd, bool packed, bool keyed, int *blocks_per_sm)
{
    return fwd ? blk::occupancy_dir<true>(packed, keyed, blocks_per_sm)
               : blk::occupancy_dir<false>(packed, keyed, blocks_per_sm);
}

} // namespace frag
