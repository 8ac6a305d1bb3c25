// fused_kernels.cu -- up to three LeGall 5/3 levels of a buffer in one pass
// down its rows, every intermediate LL band kept in registers.
//
// Work unit = (buffer, warp strip sx, row segment sy).  A warp owns a strip
// of level-0 columns: lane k holds 8 consecutive samples of every row, lanes
// 0 .. halo-1 and 31 only supply neighbours (the lifting taps of the levels
// above shrink the valid span by about one lane per side), so a strip owns
// 8 (31 - halo) columns.  The unit streams down its rows in iterations of 8
// level-0 rows:
//
//   forward   iteration t reads rows 8t-1 .. 8t+6 and, rows before columns
//             at every level (Sec. 5.2.2; Eq. 5.1 predict, Eq. 5.2 update):
//               level 1: four row pairs -> level-1 rows 4t-1 .. 4t+2
//               level 2: their LL_1 rows -> level-2 rows 2t-1, 2t
//               level 3: their LL_2 rows -> level-3 row t-1
//             The column lifting of each level carries (e0, d[-1]) from one
//             pair to the next, so a level's rows come out as soon as its two
//             input rows exist.  A unit first runs F iterations that store
//             nothing: they rebuild the column state of every level above
//             its first row (the lifting's support grows by two rows per
//             level).
//   inverse   iteration t consumes level-3 row t, level-2 rows 2t-1, 2t and
//             level-1 rows 4t-3 .. 4t; the column inverse of each level
//             (undo Eq. 5.2, then Eq. 5.1) emits two rows of the level below
//             per coefficient row, the row inverse makes them LL samples, and
//             level 1 ends in level-0 rows 8t-7 .. 8t.  A unit first runs one
//             iteration (two with three levels) that stores nothing.
//
// Loads: each lane copies its own 8 (or 4) bytes of every row it needs into a
// per-warp ring of shared-memory stages with cp.async, two iterations ahead,
// and reads back only what it copied, so no barrier is needed.  Rows past the
// data read as zeros (zero-filled copies); rows and lanes outside the matrix
// are not loaded, and the symmetric extension (x[-1] = x[1], x[m] = x[m-2],
// hence d[-1] = d[0]) is applied at each level's own borders.
//
// Output: the detail bands of every fused level go straight to the public
// fragment; LL_F goes to the private fragment as LL_L - 128 (int16) when F is
// the last level, else to scratch as biased 16-bit values (the packed-pair
// layout the dependency-ordered kernel reads for the levels above).
#include "frag_internal.cuh"
#include "swar.cuh"

namespace frag {
namespace fuse {

using strm::from_i16x2;
using strm::kB2;
using strm::lift_row;
using strm::pavg;
using strm::pq4;
using strm::Raw;
using strm::to_i16x2;
using strm::unlift_row;

constexpr int kWarps = kFuseWarps;
constexpr int kThreads = 32 * kWarps;
constexpr int kDepth = kFuseDepth;
constexpr int kFwdStage = 8 * 256; // 8 level-0 rows x 32 lanes x 8 bytes
// inverse stage: level-1 rows j = 0..3, bands HL/LH/HH, 8 bytes a lane, then
// region X: level-1 LL rows (one level), or level-2 rows k = 0..1 of the three
// bands (4 bytes a lane) followed by LL_2 rows (two levels) or the four
// level-3 words (three levels)
constexpr int kInvX = 12 * 256;
constexpr int kInvL2Ll = kInvX + 6 * 128;
constexpr int kInvL3 = kInvX + 6 * 128;
constexpr int kInvStage = kInvL3 + 4 * 128;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// cp.async of `size` bytes (4 or 8) of which the first `bytes` are read and
// the rest zero-filled
__device__ __forceinline__ void cp8(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp4(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ uint2 lds8(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds4(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

// int16 stores at element index idx of a band (streaming: never re-read here)
__device__ __forceinline__ void st8(uint8_t *band, uint64_t idx, uint32_t a, uint32_t b)
{
    __stcs(reinterpret_cast<uint2 *>(band + 2 * idx), make_uint2(a, b));
}
__device__ __forceinline__ void st4(uint8_t *band, uint64_t idx, uint32_t a)
{
    __stcs(reinterpret_cast<unsigned int *>(band + 2 * idx), a);
}
__device__ __forceinline__ void st2(uint8_t *band, uint64_t idx, uint32_t a)
{
    __stcs(reinterpret_cast<unsigned short *>(band + 2 * idx), (unsigned short)a);
}

// ---------------------------------------------------------------------------
// row lifting of the coarser levels
// ---------------------------------------------------------------------------

// Level-2 row lift of the lane's four LL_1 samples y0..y3 (columns c .. c+3
// of a row of Wd samples; w0 = (y0, y1), w1 = (y2, y3)): L = (s0, s1),
// H = (d0, d1).  y4 and d[-1] come from the adjacent lanes.
__device__ __forceinline__ void lift4(uint32_t w0, uint32_t w1, int c, int Wd, bool edge,
                                      uint32_t &L, uint32_t &H)
{
    const uint32_t e = __byte_perm(w0, w1, 0x5410); // (y0, y2)
    const uint32_t o = __byte_perm(w0, w1, 0x7632); // (y1, y3)
    const uint32_t en = __shfl_down_sync(0xffffffffu, e, 1);
    uint32_t es = __byte_perm(e, en, 0x5432); // (y2, y4)
    if (edge) {                               // x[m] = x[m-2]
        if (c + 2 == Wd)
            es = __byte_perm(e, es, 0x7610);
        if (c + 4 == Wd)
            es = __byte_perm(es, e, 0x7610);
    }
    const uint32_t d = o - pavg(e, es) + kB2; // Eq. 5.1
    const uint32_t dpl = __shfl_up_sync(0xffffffffu, d, 1);
    uint32_t dm = __byte_perm(dpl, d, 0x5432); // (d[-1], d0)
    if (c == 0)
        dm = __byte_perm(d, d, 0x1010); // d[-1] = d[0]
    L = e + pq4(dm, d) - 0x20002000u;   // Eq. 5.2
    H = d;
}

// Level-3 row lift of the lane's two LL_2 samples z = (z0, z1) at columns
// c, c+1: returns (s, d) of the pair in one word (s low, d high).
__device__ __forceinline__ uint32_t lift2(uint32_t z, int c, int Wd, bool edge)
{
    const uint32_t zn = __shfl_down_sync(0xffffffffu, z, 1);
    const uint32_t e = z & 0xffffu, o = z >> 16;
    const uint32_t en = (edge && c + 2 == Wd) ? e : (zn & 0xffffu);
    const uint32_t d = o - ((e + en) >> 1) + 0x4000u; // Eq. 5.1
    uint32_t dp = __shfl_up_sync(0xffffffffu, d, 1);
    if (c == 0)
        dp = d;
    const uint32_t s = e + ((dp + d + 2) >> 2) - 0x2000u; // Eq. 5.2
    return s | (d << 16);
}

// Level-3 row inverse: (s, d) word of a row-lifted LL_2 row -> (z0, z1)
__device__ __forceinline__ uint32_t unlift2(uint32_t w, int c, int Wd, bool edge)
{
    const uint32_t s = w & 0xffffu, d = w >> 16;
    uint32_t dp = __shfl_up_sync(0xffffffffu, d, 1);
    if (c == 0)
        dp = d;
    const uint32_t z0 = s - ((dp + d + 2) >> 2) + 0x2000u; // undo Eq. 5.2
    uint32_t zn = __shfl_down_sync(0xffffffffu, z0, 1);
    if (edge && c + 2 == Wd)
        zn = z0;
    const uint32_t z1 = d + ((z0 + zn) >> 1) - 0x4000u; // undo Eq. 5.1
    return z0 | (z1 << 16);
}

// Level-2 row inverse: L = (s0, s1), H = (d0, d1) -> w0 = (y0, y1), w1 = (y2, y3)
__device__ __forceinline__ void unlift4(uint32_t L, uint32_t H, int c, int Wd, bool edge,
                                        uint32_t &w0, uint32_t &w1)
{
    const uint32_t hp = __shfl_up_sync(0xffffffffu, H, 1);
    uint32_t hm = __byte_perm(hp, H, 0x5432); // (d[-1], d0)
    if (c == 0)
        hm = __byte_perm(H, H, 0x1010);
    const uint32_t e = L - pq4(hm, H) + 0x20002000u; // undo Eq. 5.2: (y0, y2)
    const uint32_t en = __shfl_down_sync(0xffffffffu, e, 1);
    uint32_t es = __byte_perm(e, en, 0x5432); // (y2, y4)
    if (edge) {
        if (c + 2 == Wd)
            es = __byte_perm(e, es, 0x7610);
        if (c + 4 == Wd)
            es = __byte_perm(es, e, 0x7610);
    }
    const uint32_t o = H + pavg(e, es) - kB2; // undo Eq. 5.1: (y1, y3)
    w0 = __byte_perm(e, o, 0x5410);
    w1 = __byte_perm(e, o, 0x7632);
}

// ---------------------------------------------------------------------------
// forward unit
// ---------------------------------------------------------------------------

// the level-0 rows of iteration t into its stage: rows 8t-1 .. 8t+6
__device__ __forceinline__ void fwd_issue(const FuseBuf &b, int t, int t_end, int c0, bool loads,
                                          uint32_t ring_lane)
{
    if (t < t_end && loads) {
        const uint32_t st = ring_lane + (uint32_t)(t % kDepth) * kFwdStage;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = 8 * t - 1 + j;
            if (r >= 0 && r < (int)b.H) {
                const uint64_t off = (uint64_t)r * b.W + (uint64_t)c0;
                const uint32_t bytes = off >= b.n ? 0u : (uint32_t)(b.n - off < 8 ? b.n - off : 8);
                cp8(st + 256 * j, bytes ? b.src + off : b.src, bytes);
            }
        }
    }
    cp_commit();
}

// LL_F of the final level: LL - 128 as int16 (both halves of each word)
__device__ __forceinline__ uint32_t ll_final(uint32_t w) { return to_i16x2(w - 0x00800080u); }

__device__ __forceinline__ void fwd_unit(const FuseBuf &b, uint32_t sx, uint32_t sy, uint32_t ring_lane,
                                      int lane)
{
    const int h = (int)b.halo;
    const int SW = 8 * (31 - h);
    const int W = (int)b.W, H = (int)b.H, F = (int)b.F;
    const int c0 = (int)sx * SW + 8 * (lane - h);
    const bool loads = c0 >= 0 && c0 < W;
    const bool own = lane >= h && lane <= 30 && c0 < W;
    const bool edge = (int)sx * SW + 8 * (32 - h) >= W;
    const int W1 = W >> 1, H1 = H >> 1, W2 = W >> 2, H2 = H >> 2, W3 = W >> 3, H3 = H >> 3;
    const int c1 = c0 >> 1, c2 = c0 >> 2, c3 = c0 >> 3;
    const bool fin = b.ll_final != 0;
    const int t_begin = (int)(sy * b.seg_iters);
    const int t_end = min(t_begin + (int)b.seg_iters, (int)b.iters);
    const int t_first = max(t_begin - F, 0);

#pragma unroll
    for (int k = 0; k < kDepth - 1; ++k)
        fwd_issue(b, t_first + k, t_end, c0, loads, ring_lane);

    uint32_t e0[4], dp[4], e2L = kB2, e2H = kB2, p2L = kB2, p2H = kB2, e3 = kB2, p3 = kB2;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        e0[k] = dp[k] = kB2;

    for (int t = t_first; t < t_end; ++t) {
        fwd_issue(b, t + kDepth - 1, t_end, c0, loads, ring_lane);
        cp_wait<kDepth - 1>();
        const uint32_t st = ring_lane + (uint32_t)(t % kDepth) * kFwdStage;
        uint2 raw[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            raw[j] = lds8(st + 256 * j);
        const bool store = own && t >= t_begin;

        // level 1: pairs (8t-1+2j, 8t+2j) -> level-1 row 4t-1+j
        uint32_t y[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Raw ro, re;
            ro.w[0] = raw[2 * j].x;
            ro.w[1] = raw[2 * j].y;
            ro.w[2] = ro.w[3] = 0;
            re.w[0] = raw[2 * j + 1].x;
            re.w[1] = raw[2 * j + 1].y;
            re.w[2] = re.w[3] = 0;
            uint32_t Po[4], Pe[4];
            lift_row<true, true>(ro, c0, W, edge, Po);
            lift_row<true, true>(re, c0, W, edge, Pe);
            const int q = 4 * t - 1 + j;
            if (8 * t + 2 * j == H) { // x[m] = x[m-2] at the bottom border
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    Pe[k] = e0[k];
            }
            uint32_t dv[4], sv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                dv[k] = Po[k] - pavg(e0[k], Pe[k]) + kB2; // Eq. 5.1 down the columns
            if (q == 0) {                                 // d[-1] = d[0] at the top border
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    dp[k] = dv[k];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                sv[k] = e0[k] + pq4(dp[k], dv[k]) - 0x20002000u; // Eq. 5.2 down the columns
                e0[k] = Pe[k];
                dp[k] = dv[k];
            }
            if (store && (unsigned)q < (unsigned)H1) {
                const uint64_t idx = (uint64_t)q * (uint64_t)W1 + (uint64_t)c1;
                st8(b.band[0][0], idx, to_i16x2(sv[2]), to_i16x2(sv[3])); // HL_1
                st8(b.band[0][1], idx, to_i16x2(dv[0]), to_i16x2(dv[1])); // LH_1
                st8(b.band[0][2], idx, to_i16x2(dv[2]), to_i16x2(dv[3])); // HH_1
                if (F == 1) {
                    if (fin)
                        st8(b.ll, idx, ll_final(sv[0]), ll_final(sv[1]));
                    else
                        st8(b.ll, idx, sv[0], sv[1]);
                }
            }
            y[j][0] = sv[0];
            y[j][1] = sv[1];
        }
        if (F < 2)
            continue;

        // level 2: LL_1 pairs (4t-1+2k, 4t+2k) -> level-2 row 2t-1+k
        uint32_t z[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint32_t Lo, Ho, Le, He;
            lift4(y[2 * k][0], y[2 * k][1], c1, W1, edge, Lo, Ho);
            lift4(y[2 * k + 1][0], y[2 * k + 1][1], c1, W1, edge, Le, He);
            const int q2 = 2 * t - 1 + k;
            if (4 * t + 2 * k == H1) {
                Le = e2L;
                He = e2H;
            }
            const uint32_t dL = Lo - pavg(e2L, Le) + kB2, dH = Ho - pavg(e2H, He) + kB2;
            if (q2 == 0) {
                p2L = dL;
                p2H = dH;
            }
            const uint32_t sL = e2L + pq4(p2L, dL) - 0x20002000u;
            const uint32_t sH = e2H + pq4(p2H, dH) - 0x20002000u;
            e2L = Le;
            e2H = He;
            p2L = dL;
            p2H = dH;
            if (store && (unsigned)q2 < (unsigned)H2) {
                const uint64_t idx = (uint64_t)q2 * (uint64_t)W2 + (uint64_t)c2;
                st4(b.band[1][0], idx, to_i16x2(sH)); // HL_2
                st4(b.band[1][1], idx, to_i16x2(dL)); // LH_2
                st4(b.band[1][2], idx, to_i16x2(dH)); // HH_2
                if (F == 2)
                    st4(b.ll, idx, fin ? ll_final(sL) : sL);
            }
            z[k] = sL;
        }
        if (F < 3)
            continue;

        // level 3: LL_2 pair (2t-1, 2t) -> level-3 row t-1
        {
            const uint32_t wo = lift2(z[0], c2, W2, edge);
            uint32_t we = lift2(z[1], c2, W2, edge);
            const int q3 = t - 1;
            if (2 * t == H2)
                we = e3;
            const uint32_t d3 = wo - pavg(e3, we) + kB2;
            if (q3 == 0)
                p3 = d3;
            const uint32_t s3 = e3 + pq4(p3, d3) - 0x20002000u;
            e3 = we;
            p3 = d3;
            if (store && (unsigned)q3 < (unsigned)H3) {
                const uint64_t idx = (uint64_t)q3 * (uint64_t)W3 + (uint64_t)c3;
                const uint32_t sw = to_i16x2(s3), dw = to_i16x2(d3);
                st2(b.band[2][0], idx, sw >> 16); // HL_3
                st2(b.band[2][1], idx, dw);       // LH_3
                st2(b.band[2][2], idx, dw >> 16); // HH_3
                st2(b.ll, idx, fin ? ll_final(s3) : s3);
            }
        }
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// inverse unit
// ---------------------------------------------------------------------------

// int16 word(s) of the input -> biased values; LL_L - 128 gets its 128 back
__device__ __forceinline__ uint32_t in16(uint32_t w) { return from_i16x2(w); }

// the coefficient rows iteration t consumes, into its stage
__device__ __forceinline__ void inv_issue(const FuseBuf &b, int t, int t_end, int c0, bool loads,
                                          uint32_t ring8, uint32_t ring4)
{
    if (t < t_end && loads) {
        const int F = (int)b.F;
        const uint32_t so = (uint32_t)(t % kDepth) * kInvStage;
        const uint32_t W1 = b.W >> 1, H1 = b.H >> 1, W2 = b.W >> 2, H2 = b.H >> 2;
        const uint32_t c1 = (uint32_t)c0 >> 1, c2 = (uint32_t)c0 >> 2;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = 4 * t - 3 + j;
            if (q >= 0 && q < (int)H1) {
                const uint64_t off = 2ull * ((uint64_t)q * W1 + c1);
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    cp8(ring8 + so + 256 * (3 * j + k), b.band[0][k] + off, 8);
                if (F == 1)
                    cp8(ring8 + so + kInvX + 256 * j, b.ll + off, 8);
            }
        }
        if (F >= 2) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = 2 * t - 1 + k;
                if (q >= 0 && q < (int)H2) {
                    const uint64_t off = 2ull * ((uint64_t)q * W2 + c2);
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        cp4(ring4 + so + kInvX + 128 * (3 * k + m), b.band[1][m] + off, 4);
                    if (F == 2)
                        cp4(ring4 + so + kInvL2Ll + 128 * k, b.ll + off, 4);
                }
            }
        }
        if (F == 3 && t < (int)(b.H >> 3)) {
            // one int16 per lane: copy the aligned word that holds it (band
            // bases are 4-byte aligned, so the word stays inside the band)
            const uint64_t e = (uint64_t)t * (b.W >> 3) + ((uint32_t)c0 >> 3);
            const uint64_t off = 2ull * (e & ~1ull);
            const uint32_t bytes = (e & 1ull) ? 4u : 2u;
#pragma unroll
            for (int m = 0; m < 3; ++m)
                cp4(ring4 + so + kInvL3 + 128 * m, b.band[2][m] + off, bytes);
            cp4(ring4 + so + kInvL3 + 128 * 3, b.ll + off, bytes);
        }
    }
    cp_commit();
}

// eager column inverse of one coefficient row q of a level (words of the
// lane): xe = x[2q], xo = x[2q-1]; (xp, dp) = (x[2q-2], d[q-1]) carried.
// top: q == 0 (d[-1] = d[0]); bottom: q is one past the last row (x[2q] =
// x[2q-2], only the odd row is real)
__device__ __forceinline__ void col_inv(uint32_t s, uint32_t d, bool top, bool bottom, uint32_t &xp,
                                        uint32_t &dp, uint32_t &xo, uint32_t &xe)
{
    if (top)
        dp = d;
    xe = bottom ? xp : s - pq4(dp, d) + 0x20002000u; // undo Eq. 5.2
    xo = dp + pavg(xp, xe) - kB2;                    // undo Eq. 5.1
    xp = xe;
    dp = d;
}

// 8 recovered bytes of row r at column c0 (biased halves: the low byte of
// each is the byte)
__device__ __forceinline__ void store_bytes(const FuseBuf &b, int r, int c0, const uint32_t (&p)[4])
{
    const uint64_t g = (uint64_t)r * b.W + (uint64_t)c0;
    if (g >= b.n)
        return;
    const uint32_t w0 = __byte_perm(p[0], p[1], 0x6420);
    const uint32_t w1 = __byte_perm(p[2], p[3], 0x6420);
    if (g + 8 <= b.n) {
        __stcs(reinterpret_cast<uint2 *>(b.out + g), make_uint2(w0, w1));
    } else {
        for (int i = 0; i < 8 && g + (uint64_t)i < b.n; ++i)
            b.out[g + i] = (uint8_t)((i < 4 ? w0 : w1) >> (8 * (i & 3)));
    }
}

__device__ __forceinline__ void inv_unit(const FuseBuf &b, uint32_t sx, uint32_t sy, uint32_t ring_lane8,
                                      uint32_t ring_lane4, int lane)
{
    const int h = (int)b.halo;
    const int SW = 8 * (31 - h);
    const int W = (int)b.W, H = (int)b.H, F = (int)b.F;
    const int c0 = (int)sx * SW + 8 * (lane - h);
    const bool loads = c0 >= 0 && c0 < W;
    const bool own = lane >= h && lane <= 30 && c0 < W;
    const bool edge = (int)sx * SW + 8 * (32 - h) >= W;
    const int W1 = W >> 1, H1 = H >> 1, W2 = W >> 2, H2 = H >> 2, W3 = W >> 3, H3 = H >> 3;
    const int c1 = c0 >> 1, c2 = c0 >> 2, c3 = c0 >> 3;
    const uint32_t llb = b.ll_final ? 0x00800080u : 0u; // LL_L - 128 -> LL_L
    const int t_begin = (int)(sy * b.seg_iters);
    const int t_end = min(t_begin + (int)b.seg_iters, (int)b.iters);
    const int t_first = max(t_begin - (F == 3 ? 2 : 1), 0);

#pragma unroll
    for (int k = 0; k < kDepth - 1; ++k)
        inv_issue(b, t_first + k, t_end, c0, loads, ring_lane8, ring_lane4);

    uint32_t x1[4], d1[4], x2[2], d2[2], x3 = kB2, d3 = kB2;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        x1[k] = d1[k] = kB2;
    x2[0] = x2[1] = d2[0] = d2[1] = kB2;

    for (int t = t_first; t < t_end; ++t) {
        inv_issue(b, t + kDepth - 1, t_end, c0, loads, ring_lane8, ring_lane4);
        cp_wait<kDepth - 1>();
        const uint32_t so = (uint32_t)(t % kDepth) * kInvStage;
        const uint32_t s8 = ring_lane8 + so, s4 = ring_lane4 + so;
        const bool store = own && t >= t_begin;

        // level 3: row t -> LL_2 rows 2t-1, 2t
        uint32_t z[2];
        if (F == 3) {
            const uint32_t sh = 16u * (uint32_t)(((uint64_t)t * (uint64_t)W3 + (uint64_t)c3) & 1ull);
            const uint32_t hl = (lds4(s4 + kInvL3) >> sh) & 0xffffu;
            const uint32_t lh = (lds4(s4 + kInvL3 + 128) >> sh) & 0xffffu;
            const uint32_t hh = (lds4(s4 + kInvL3 + 256) >> sh) & 0xffffu;
            const uint32_t ll = (lds4(s4 + kInvL3 + 384) >> sh) & 0xffffu;
            const uint32_t s = b.ll_final ? in16(ll | (hl << 16)) + 0x80u : ((ll | (in16(hl << 16) & 0xffff0000u)));
            const uint32_t d = in16(lh | (hh << 16));
            uint32_t xo, xe;
            col_inv(s, d, t == 0, t == H3, x3, d3, xo, xe);
            z[0] = unlift2(xo, c2, W2, edge);
            z[1] = unlift2(xe, c2, W2, edge);
        }

        // level 2: rows 2t-1+k -> LL_1 rows 4t-3+2k, 4t-2+2k
        uint32_t y[4][2];
        if (F >= 2) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q2 = 2 * t - 1 + k;
                const uint32_t hl = in16(lds4(s4 + kInvX + 128 * (3 * k)));
                const uint32_t lh = in16(lds4(s4 + kInvX + 128 * (3 * k + 1)));
                const uint32_t hh = in16(lds4(s4 + kInvX + 128 * (3 * k + 2)));
                uint32_t ll;
                if (F == 3)
                    ll = z[k];
                else if (b.ll_final)
                    ll = in16(lds4(s4 + kInvL2Ll + 128 * k)) + llb;
                else
                    ll = lds4(s4 + kInvL2Ll + 128 * k);
                uint32_t oL, eL, oH, eH;
                col_inv(ll, lh, q2 == 0, q2 == H2, x2[0], d2[0], oL, eL);
                col_inv(hl, hh, q2 == 0, q2 == H2, x2[1], d2[1], oH, eH);
                unlift4(oL, oH, c1, W1, edge, y[2 * k][0], y[2 * k][1]);
                unlift4(eL, eH, c1, W1, edge, y[2 * k + 1][0], y[2 * k + 1][1]);
            }
        }

        // level 1: rows 4t-3+j -> level-0 rows 8t-7+2j, 8t-6+2j
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = 4 * t - 3 + j;
            const uint2 hl = lds8(s8 + 256 * (3 * j));
            const uint2 lh = lds8(s8 + 256 * (3 * j + 1));
            const uint2 hh = lds8(s8 + 256 * (3 * j + 2));
            uint32_t s[4], d[4];
            if (F == 1) {
                const uint2 ll = lds8(s8 + kInvX + 256 * j);
                s[0] = b.ll_final ? in16(ll.x) + llb : ll.x;
                s[1] = b.ll_final ? in16(ll.y) + llb : ll.y;
            } else {
                s[0] = y[j][0];
                s[1] = y[j][1];
            }
            s[2] = in16(hl.x);
            s[3] = in16(hl.y);
            d[0] = in16(lh.x);
            d[1] = in16(lh.y);
            d[2] = in16(hh.x);
            d[3] = in16(hh.y);
            uint32_t xo[4], xe[4];
#pragma unroll
            for (int m = 0; m < 4; ++m)
                col_inv(s[m], d[m], q == 0, q == H1, x1[m], d1[m], xo[m], xe[m]);
            uint32_t vo[4], ve[4];
            unlift_row<true>(xo, c0, W, edge, vo);
            unlift_row<true>(xe, c0, W, edge, ve);
            const int r = 2 * q - 1;
            if (store && r >= 0 && r < H)
                store_bytes(b, r, c0, vo);
            if (store && r + 1 >= 0 && r + 1 < H)
                store_bytes(b, r + 1, c0, ve);
        }
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// kernel: warp-granular units, static round robin over the grid's warps
// ---------------------------------------------------------------------------
__device__ __forceinline__ const FuseBuf *unit_buf(const FuseWork &w, uint64_t u, uint64_t &local)
{
    if (w.nbufs == 1) {
        local = u;
        return &w.single;
    }
    uint32_t lo = 0, hi = w.nbufs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&w.bufs[mid].unit0) <= u)
            lo = mid;
        else
            hi = mid;
    }
    local = u - __ldg(&w.bufs[lo].unit0);
    return &w.bufs[lo];
}

template <bool FWD>
__global__ void __launch_bounds__(kThreads) fuse_kernel(FuseWork w)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ring = smem_addr(smem) + (uint32_t)warp * kDepth * (FWD ? kFwdStage : kInvStage);
    const uint64_t G = (uint64_t)gridDim.x * kWarps;
    for (uint64_t u = (uint64_t)blockIdx.x * kWarps + warp; u < w.total_units; u += G) {
        uint64_t local;
        const FuseBuf *bp = unit_buf(w, u, local);
        const FuseBuf b = *bp;
        const uint32_t sy = (uint32_t)(local / b.strips), sx = (uint32_t)(local % b.strips);
        if (FWD)
            fwd_unit(b, sx, sy, ring + 8u * lane, lane);
        else
            inv_unit(b, sx, sy, ring + 8u * lane, ring + 4u * lane, lane);
    }
}

size_t smem_bytes(bool fwd) { return (size_t)kWarps * kDepth * (fwd ? kFwdStage : kInvStage); }

template <bool FWD>
cudaError_t set_attr()
{
    return cudaFuncSetAttribute((const void *)fuse_kernel<FWD>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(FWD));
}

} // namespace fuse

cudaError_t launch_fuse(bool fwd, const FuseWork &w, uint32_t grid, cudaStream_t stream)
{
    cudaError_t e = fwd ? fuse::set_attr<true>() : fuse::set_attr<false>();
    if (e != cudaSuccess)
        return e;
    if (fwd)
        fuse::fuse_kernel<true><<<grid, fuse::kThreads, fuse::smem_bytes(true), stream>>>(w);
    else
        fuse::fuse_kernel<false><<<grid, fuse::kThreads, fuse::smem_bytes(false), stream>>>(w);
    return cudaGetLastError();
}

cudaError_t fuse_occupancy(bool fwd, int *blocks_per_sm)
{
    cudaError_t e = fwd ? fuse::set_attr<true>() : fuse::set_attr<false>();
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, fwd ? (const void *)fuse::fuse_kernel<true> : (const void *)fuse::fuse_kernel<false>,
        fuse::kThreads, fuse::smem_bytes(fwd));
}

} // namespace frag
