// stream_kernels.cu -- every LeGall 5/3 level of one or many buffers, and the
// AES-128-CTR pass over their private fragments, in one launch.
//
// Work units (the host lists them so that every unit's producers come first):
//   level unit   (buffer, level l, strip, row segment): a warp takes a strip of
//                256 columns of the level-(l-1) image and streams down the
//                rows of its segment.
//                forward: lane t loads 8 consecutive samples of a row; the row
//                lifting (Eq. 5.1 predict, then Eq. 5.2 update; rows before
//                columns, Sec. 5.2.2) runs on packed pairs, the neighbours x8
//                and d[-1] taken from the adjacent lanes by warp shuffles; the
//                column lifting then runs on those packed pairs in registers.
//                HL_l / LH_l / HH_l go straight to the public fragment, LL_l
//                to scratch (packed pairs) or, at the last level, as
//                LL_L - 128 (int16 LE) to the private fragment.
//                inverse: the exact reverse (undo Eq. 5.2, then Eq. 5.1, down
//                the columns, then along the rows) gives LL_{l-1} (scratch) or
//                the recovered bytes.
//   cipher unit  the 16-byte blocks of the private fragment that start in one
//                row segment of LL_L, XORed with the AES-128 keystream of the
//                counter block nonce || block index, one block per lane.
//                forward: in place, after the last level wrote those rows;
//                inverse: into a plaintext copy that the top level reads.
//
// Lanes 0 and 31 of a warp only supply neighbours: lanes 1..30 own the
// strip's 240 columns.  Rows above a segment are re-lifted to restart the
// column stream.  The symmetric extension (x[-1] = x[1], x[m] = x[m-2], hence
// d[-1] = d[0]) applies only at the image borders.  A unit away from every
// border runs a branch-free loop that keeps several row pairs of loads in
// flight; the others run the general loop with bounds checks and the border
// rules.
//
// Packed pairs: each 16-bit half holds v + 0x4000 (|v| < 2^14); the halves of
// (A + B) never carry into each other, so both floors of a lifting step take
// one add, one shift and one mask for two columns.
//
// A unit whose input another unit of the launch writes waits (lane 0, bounded
// spin) until the producer row segments are complete and then reads that data
// with L2-coherent loads.  A wait that runs out sets the error word to 3
// (FRAG_ETIMEOUT) and skips the unit, which is still reported complete so that
// no consumer waits forever.
#include "frag_internal.cuh"

namespace frag {

struct AesTab {
    uint32_t T[4][256];
    uint32_t S[256];
    uint32_t rk[44];
};

// AES-128 encryption of the counter block nonce || blk (FIPS-197 cipher,
// 32-bit table form), big-endian words.
__device__ __forceinline__ void aes_block(const AesTab &a, uint64_t nonce, uint64_t blk,
                                          uint32_t ks[4])
{
    uint32_t s0 = (uint32_t)(nonce >> 32) ^ a.rk[0];
    uint32_t s1 = (uint32_t)nonce ^ a.rk[1];
    uint32_t s2 = (uint32_t)(blk >> 32) ^ a.rk[2];
    uint32_t s3 = (uint32_t)blk ^ a.rk[3];
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint32_t t0 = a.T[0][s0 >> 24] ^ a.T[1][(s1 >> 16) & 255] ^
                            a.T[2][(s2 >> 8) & 255] ^ a.T[3][s3 & 255] ^ a.rk[4 * r];
        const uint32_t t1 = a.T[0][s1 >> 24] ^ a.T[1][(s2 >> 16) & 255] ^
                            a.T[2][(s3 >> 8) & 255] ^ a.T[3][s0 & 255] ^ a.rk[4 * r + 1];
        const uint32_t t2 = a.T[0][s2 >> 24] ^ a.T[1][(s3 >> 16) & 255] ^
                            a.T[2][(s0 >> 8) & 255] ^ a.T[3][s1 & 255] ^ a.rk[4 * r + 2];
        const uint32_t t3 = a.T[0][s3 >> 24] ^ a.T[1][(s0 >> 16) & 255] ^
                            a.T[2][(s1 >> 8) & 255] ^ a.T[3][s2 & 255] ^ a.rk[4 * r + 3];
        s0 = t0;
        s1 = t1;
        s2 = t2;
        s3 = t3;
    }
    ks[0] = ((a.S[s0 >> 24] << 24) | (a.S[(s1 >> 16) & 255] << 16) |
             (a.S[(s2 >> 8) & 255] << 8) | a.S[s3 & 255]) ^ a.rk[40];
    ks[1] = ((a.S[s1 >> 24] << 24) | (a.S[(s2 >> 16) & 255] << 16) |
             (a.S[(s3 >> 8) & 255] << 8) | a.S[s0 & 255]) ^ a.rk[41];
    ks[2] = ((a.S[s2 >> 24] << 24) | (a.S[(s3 >> 16) & 255] << 16) |
             (a.S[(s0 >> 8) & 255] << 8) | a.S[s1 & 255]) ^ a.rk[42];
    ks[3] = ((a.S[s3 >> 24] << 24) | (a.S[(s0 >> 16) & 255] << 16) |
             (a.S[(s1 >> 8) & 255] << 8) | a.S[s2 & 255]) ^ a.rk[43];
}

namespace strm {

// row pairs of loads kept in flight by an interior unit, and resident blocks
// of 256 threads per SM the kernel is compiled for (tuning knobs)
#ifndef FRAG_PREFETCH_BYTES
#define FRAG_PREFETCH_BYTES 4
#endif
#ifndef FRAG_PREFETCH_PACKED
#define FRAG_PREFETCH_PACKED 2
#endif
#ifndef FRAG_PREFETCH_INV
#define FRAG_PREFETCH_INV 2
#endif
#ifndef FRAG_PREFETCH_GENERAL
#define FRAG_PREFETCH_GENERAL 1
#endif
#ifndef FRAG_BLOCKS_PER_SM
#define FRAG_BLOCKS_PER_SM 3
#endif

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
        e01 = __byte_perm(raw.w[0], 0, 0x4240) + kB2;
        o01 = __byte_perm(raw.w[0], 0, 0x4341) + kB2;
        e23 = __byte_perm(raw.w[1], 0, 0x4240) + kB2;
        o23 = __byte_perm(raw.w[1], 0, 0x4341) + kB2;
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

// one row pair down the columns, forward: rows o (odd) and e1 (next even) of
// the pair, (e0, dp) carried; sv = s of the pair, dv = d of the pair
__device__ __forceinline__ void col_step(const uint32_t (&o)[4], const uint32_t (&e1)[4],
                                         uint32_t (&e0)[4], uint32_t (&dp)[4], bool top,
                                         uint32_t (&sv)[4], uint32_t (&dv)[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k)
        dv[k] = o[k] - pavg(e0[k], e1[k]) + kB2; // Eq. 5.1 down the columns
    if (top) {                                   // d[-1] = d[0] at the top border
#pragma unroll
        for (int k = 0; k < 4; ++k)
            dp[k] = dv[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        sv[k] = e0[k] + pq4(dp[k], dv[k]) - 0x20002000u; // Eq. 5.2 down the columns
        e0[k] = e1[k];
        dp[k] = dv[k];
    }
}

// LL words of a pair for the output: scratch keeps packed pairs; the last
// level writes LL_L - 128 as int16 (the level shift moves only LL_L)
template <bool FINAL>
__device__ __forceinline__ uint2 ll_out(const uint32_t (&sv)[4])
{
    if (FINAL)
        return make_uint2(to_i16x2(sv[0] - 0x00800080u), to_i16x2(sv[1] - 0x00800080u));
    return make_uint2(sv[0], sv[1]);
}

// ---------------------------------------------------------------------------
// general-path memory helpers (bounds checked)
// ---------------------------------------------------------------------------

// 8 source samples of row r at columns c .. c+7 of the level-(l-1) image.
// Bytes past n (or outside the image) are 0; packed samples outside the
// image are the biased 0.
template <bool BYTES>
__device__ __forceinline__ Raw load_row(const LevelJob &j, int r, int c, bool vec)
{
    Raw raw;
    if (BYTES) {
        raw.w[2] = raw.w[3] = 0;
        const uint64_t base = (uint64_t)r * (uint64_t)j.Ws;
        if (r < (int)j.Hs && vec && c >= 0 && c + 8 <= (int)j.Ws && base + (uint64_t)c + 8 <= j.n) {
            const uint2 t = __ldg(reinterpret_cast<const uint2 *>(j.src + base + c));
            raw.w[0] = t.x;
            raw.w[1] = t.y;
        } else {
            uint32_t b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int cc = c + i;
                b[i] = (r < (int)j.Hs && cc >= 0 && cc < (int)j.Ws && base + (uint64_t)cc < j.n)
                           ? (uint32_t)__ldg(j.src + base + (uint64_t)cc)
                           : 0u;
            }
            raw.w[0] = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
            raw.w[1] = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
        }
    } else {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(j.src);
        const int wpr = (int)j.Ws / 2, w0 = c >> 1;
        const uint64_t base = (uint64_t)r * (uint64_t)wpr;
        if (r < (int)j.Hs && vec && c >= 0 && c + 8 <= (int)j.Ws) {
            const uint4 t = __ldcg(reinterpret_cast<const uint4 *>(src + base + w0));
            raw.w[0] = t.x;
            raw.w[1] = t.y;
            raw.w[2] = t.z;
            raw.w[3] = t.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int ww = w0 + i;
                raw.w[i] = (r < (int)j.Hs && ww >= 0 && ww < wpr) ? __ldcg(src + base + ww) : kB2;
            }
        }
    }
    return raw;
}

// store 4 int16 values (2 words of int16 pairs) at (y, x .. x+3) of a band
__device__ __forceinline__ void store4(uint8_t *band, int Wl, int y, int x, uint32_t u, uint32_t v,
                                       int nval)
{
    uint8_t *dst = band + 2ull * ((uint64_t)y * (uint64_t)Wl + (uint64_t)x);
    if (nval == 4 && ((uintptr_t)dst & 7u) == 0) {
        *reinterpret_cast<uint2 *>(dst) = make_uint2(u, v);
    } else {
        const uint32_t h[4] = {u & 0xffffu, u >> 16, v & 0xffffu, v >> 16};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (i < nval) {
                dst[2 * i] = (uint8_t)h[i];
                dst[2 * i + 1] = (uint8_t)(h[i] >> 8);
            }
    }
}

// ---------------------------------------------------------------------------
// forward level unit
// ---------------------------------------------------------------------------
template <bool BYTES, bool FINAL>
__device__ void fwd_unit(const LevelJob &j, int sx, int sy, int lane)
{
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const int c = 240 * sx - 8 + 8 * lane; // first column of this lane
    const int q0 = sy * (int)j.seg_pairs;
    const int q1 = min(q0 + (int)j.seg_pairs, Hs / 2);
    const int Wl = Ws / 2;
    const int x = c / 2; // level-l column of the lane's first value
    const bool edge = (240 * sx + 248 >= Ws);
    const int n_it = q1 - q0;

    uint32_t e0[4], dp[4];
    const bool interior =
        sx >= 1 && !edge && q0 >= 1 && 2 * q1 < Hs && (Wl & 3) == 0 && (j.Ws & 7u) == 0 &&
        ((((uintptr_t)j.hl | (uintptr_t)j.lh | (uintptr_t)j.hh | (uintptr_t)j.ll) & 7u) == 0) &&
        (BYTES ? (((uintptr_t)j.src & 7u) == 0 &&
                  (uint64_t)(2 * q1) * (uint64_t)Ws + (uint64_t)(240 * sx + 248) <= j.n)
               : (((uintptr_t)j.src & 15u) == 0));
    if (interior) {
        // every row of the segment and its halo exists and holds data, no
        // border rule applies, and every lane's addresses lie inside the
        // buffers (lanes 0 and 31 only skip their stores)
        constexpr int D = BYTES ? FRAG_PREFETCH_BYTES : FRAG_PREFETCH_PACKED;
        const uint64_t pitch = BYTES ? (uint64_t)Ws : 2ull * (uint64_t)Ws;
        const uint8_t *rp = j.src + (uint64_t)(2 * q0 - 2) * pitch + (BYTES ? c : 2 * c);
        auto ld = [&](const uint8_t *p) -> Raw {
            Raw r;
            if (BYTES) {
                const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
                r.w[0] = t.x;
                r.w[1] = t.y;
                r.w[2] = r.w[3] = 0;
            } else {
                const uint4 t = __ldcg(reinterpret_cast<const uint4 *>(p));
                r.w[0] = t.x;
                r.w[1] = t.y;
                r.w[2] = t.z;
                r.w[3] = t.w;
            }
            return r;
        };
        Raw ra[D], rb[D];
        {
            const Raw rm2 = ld(rp), rm1 = ld(rp + pitch), r0 = ld(rp + 2 * pitch);
            rp += 3 * pitch; // row 2 q0 + 1
#pragma unroll
            for (int s = 0; s < D; ++s) {
                if (s < n_it) {
                    ra[s] = ld(rp);
                    rb[s] = ld(rp + pitch);
                } else {
                    ra[s] = rb[s] = Raw{{0u, 0u, 0u, 0u}};
                }
                rp += 2 * pitch;
            }
            uint32_t a[4], o[4];
            lift_row<BYTES, false>(r0, c, Ws, false, e0);
            lift_row<BYTES, false>(rm2, c, Ws, false, a);
            lift_row<BYTES, false>(rm1, c, Ws, false, o);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                dp[i] = o[i] - pavg(a[i], e0[i]) + kB2;
        }
        const bool own = lane >= 1 && lane <= 30;
        const uint64_t ostep = 2ull * (uint64_t)Wl; // bytes per band row
        const uint64_t o0 = 2ull * ((uint64_t)q0 * (uint64_t)Wl + (uint64_t)x);
        uint8_t *phl = j.hl + o0, *plh = j.lh + o0, *phh = j.hh + o0, *pll = j.ll + o0;
        auto step = [&](const Raw &c1, const Raw &c2) {
            uint32_t o[4], e1[4], sv[4], dv[4];
            lift_row<BYTES, false>(c1, c, Ws, false, o);
            lift_row<BYTES, false>(c2, c, Ws, false, e1);
            col_step(o, e1, e0, dp, false, sv, dv);
            // sv[0..1] = LL, sv[2..3] = HL, dv[0..1] = LH, dv[2..3] = HH
            if (own) {
                *reinterpret_cast<uint2 *>(phl) = make_uint2(to_i16x2(sv[2]), to_i16x2(sv[3]));
                *reinterpret_cast<uint2 *>(plh) = make_uint2(to_i16x2(dv[0]), to_i16x2(dv[1]));
                *reinterpret_cast<uint2 *>(phh) = make_uint2(to_i16x2(dv[2]), to_i16x2(dv[3]));
                *reinterpret_cast<uint2 *>(pll) = ll_out<FINAL>(sv);
            }
            phl += ostep;
            plh += ostep;
            phh += ostep;
            pll += ostep;
        };
        // whole groups of D row pairs: slot s is consumed, then refilled D
        // row pairs ahead (predicated loads, straight-line code)
        int i = 0;
        for (; i + D <= n_it; i += D) {
#pragma unroll
            for (int s = 0; s < D; ++s) {
                const Raw c1 = ra[s], c2 = rb[s];
                if (i + s + D < n_it) {
                    ra[s] = ld(rp);
                    rb[s] = ld(rp + pitch);
                }
                rp += 2 * pitch;
                step(c1, c2);
            }
        }
        // the last n_it mod D row pairs are already loaded
#pragma unroll
        for (int s = 0; s < D - 1; ++s)
            if (i + s < n_it)
                step(ra[s], rb[s]);
        return;
    }

    // general path: bounds checks and the border rules, a shorter ring of
    // loads in flight (its checked loads need more registers)
    constexpr int D = FRAG_PREFETCH_GENERAL;
    const bool vec = BYTES ? (((j.Ws & 7u) == 0) && (((uintptr_t)j.src & 7u) == 0))
                           : (((j.Ws & 7u) == 0) && (((uintptr_t)j.src & 15u) == 0));
    const bool own = lane >= 1 && lane <= 30 && x < Wl;
    const int nval = min(4, Wl - x);
    Raw ra[D], rb[D];
    {
        uint32_t a[4], o[4];
        const Raw r0 = load_row<BYTES>(j, 2 * q0, c, vec);
        const Raw rm2 = load_row<BYTES>(j, max(2 * q0 - 2, 0), c, vec);
        const Raw rm1 = load_row<BYTES>(j, max(2 * q0 - 1, 0), c, vec);
#pragma unroll
        for (int s = 0; s < D; ++s) {
            if (s < n_it) {
                ra[s] = load_row<BYTES>(j, 2 * (q0 + s) + 1, c, vec);
                rb[s] = load_row<BYTES>(j, 2 * (q0 + s) + 2, c, vec);
            } else {
                ra[s] = rb[s] = Raw{{0u, 0u, 0u, 0u}};
            }
        }
        lift_row<BYTES, true>(r0, c, Ws, edge, e0);
        lift_row<BYTES, true>(rm2, c, Ws, edge, a);
        lift_row<BYTES, true>(rm1, c, Ws, edge, o);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            dp[i] = o[i] - pavg(a[i], e0[i]) + kB2;
    }
    auto gstep = [&](int q, const Raw &c1, const Raw &c2) {
        uint32_t o[4], e1[4], dv[4], sv[4];
        lift_row<BYTES, true>(c1, c, Ws, edge, o);
        if (2 * q + 2 == Hs) { // x[m] = x[m-2] at the bottom border
#pragma unroll
            for (int k = 0; k < 4; ++k)
                e1[k] = e0[k];
        } else {
            lift_row<BYTES, true>(c2, c, Ws, edge, e1);
        }
        col_step(o, e1, e0, dp, q == 0, sv, dv);
        if (own) {
            store4(j.hl, Wl, q, x, to_i16x2(sv[2]), to_i16x2(sv[3]), nval);
            store4(j.lh, Wl, q, x, to_i16x2(dv[0]), to_i16x2(dv[1]), nval);
            store4(j.hh, Wl, q, x, to_i16x2(dv[2]), to_i16x2(dv[3]), nval);
            const uint2 ll = ll_out<FINAL>(sv);
            if (FINAL) {
                store4(j.ll, Wl, q, x, ll.x, ll.y, nval);
            } else {
                // packed scratch rows have Wl / 2 words (Wl is even below the last level)
                uint32_t *p = reinterpret_cast<uint32_t *>(j.ll) + (uint64_t)q * (uint64_t)(Wl / 2) + x / 2;
                if (nval == 4 && ((uintptr_t)p & 7u) == 0) {
                    *reinterpret_cast<uint2 *>(p) = ll;
                } else {
                    p[0] = ll.x;
                    if (nval > 2)
                        p[1] = ll.y;
                }
            }
        }
    };
    int i = 0;
    for (; i + D <= n_it; i += D) {
#pragma unroll
        for (int s = 0; s < D; ++s) {
            const Raw c1 = ra[s], c2 = rb[s];
            if (i + s + D < n_it) {
                ra[s] = load_row<BYTES>(j, 2 * (q0 + i + s + D) + 1, c, vec);
                rb[s] = load_row<BYTES>(j, 2 * (q0 + i + s + D) + 2, c, vec);
            }
            gstep(q0 + i + s, c1, c2);
        }
    }
#pragma unroll
    for (int s = 0; s < D - 1; ++s)
        if (i + s < n_it)
            gstep(q0 + i + s, ra[s], rb[s]);
}

// ---------------------------------------------------------------------------
// inverse level unit
// ---------------------------------------------------------------------------
struct Coef {
    uint32_t sl[2], dl[2], sh[2], dh[2]; // low s (LL), low d (LH), high s (HL), high d (HH)
};

// 4 int16 values at (y, x .. x+3) of an int16 array of Hl x Wl, as two words
// of int16 pairs; 0 outside the array
__device__ __forceinline__ void load4(const uint8_t *band, int Hl, int Wl, int y, int x, bool vec,
                                      bool coherent, uint32_t &a, uint32_t &b)
{
    if (y >= Hl || x < 0 || x >= Wl) {
        a = b = 0;
        return;
    }
    const uint8_t *p = band + 2ull * ((uint64_t)y * (uint64_t)Wl + (uint64_t)x);
    if (vec && x + 4 <= Wl && ((uintptr_t)p & 7u) == 0) {
        const uint2 t = coherent ? __ldcg(reinterpret_cast<const uint2 *>(p))
                                 : __ldg(reinterpret_cast<const uint2 *>(p));
        a = t.x;
        b = t.y;
    } else {
        uint32_t h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t v = 0;
            if (x + i < Wl)
                v = coherent ? ((uint32_t)__ldcg(p + 2 * i) | ((uint32_t)__ldcg(p + 2 * i + 1) << 8))
                             : ((uint32_t)__ldg(p + 2 * i) | ((uint32_t)__ldg(p + 2 * i + 1) << 8));
            h[i] = v;
        }
        a = h[0] | (h[1] << 16);
        b = h[2] | (h[3] << 16);
    }
}

// coefficients of row k: the detail bands, and LL_l from the packed scratch
// or, at the top level, LL_L - 128 as int16 (the deciphered private fragment)
template <bool TOP>
__device__ __forceinline__ Coef load_coef(const LevelJob &j, int k, int x, bool vec)
{
    const int Hl = (int)j.Hs / 2, Wl = (int)j.Ws / 2;
    Coef cf;
    uint32_t a, b;
    load4(j.lh, Hl, Wl, k, x, vec, false, a, b);
    cf.dl[0] = from_i16x2(a);
    cf.dl[1] = from_i16x2(b);
    load4(j.hl, Hl, Wl, k, x, vec, false, a, b);
    cf.sh[0] = from_i16x2(a);
    cf.sh[1] = from_i16x2(b);
    load4(j.hh, Hl, Wl, k, x, vec, false, a, b);
    cf.dh[0] = from_i16x2(a);
    cf.dh[1] = from_i16x2(b);
    if (TOP) {
        load4(j.ll_in, Hl, Wl, k, x, vec, true, a, b);
        cf.sl[0] = from_i16x2(a) + 0x00800080u;
        cf.sl[1] = from_i16x2(b) + 0x00800080u;
    } else {
        const uint32_t *ll = reinterpret_cast<const uint32_t *>(j.ll_in);
        const int wpr = Wl / 2;
        if (k >= Hl || x < 0 || x >= Wl) {
            cf.sl[0] = cf.sl[1] = kB2;
        } else {
            const uint32_t *p = ll + (uint64_t)k * (uint64_t)wpr + x / 2;
            if (vec && x + 4 <= Wl && ((uintptr_t)p & 7u) == 0) {
                const uint2 t = __ldcg(reinterpret_cast<const uint2 *>(p));
                cf.sl[0] = t.x;
                cf.sl[1] = t.y;
            } else {
                cf.sl[0] = __ldcg(p);
                cf.sl[1] = (x + 2 < Wl) ? __ldcg(p + 1) : kB2;
            }
        }
    }
    return cf;
}

template <bool BYTES_OUT>
__device__ __forceinline__ void store_row(const LevelJob &j, int r, int c, bool own, int nv,
                                          const uint32_t (&p)[4])
{
    if (!own)
        return;
    const int Ws = (int)j.Ws;
    if (BYTES_OUT) {
        // biased 0x4000 + b: the low byte of each half is the recovered byte
        const uint64_t g = (uint64_t)r * (uint64_t)Ws + (uint64_t)c;
        if (g >= j.n)
            return;
        uint8_t *dst = j.out + g;
        const uint32_t w0 = __byte_perm(p[0], p[1], 0x6420);
        const uint32_t w1 = __byte_perm(p[2], p[3], 0x6420);
        if (nv == 8 && g + 8 <= j.n && ((uintptr_t)dst & 7u) == 0) {
            *reinterpret_cast<uint2 *>(dst) = make_uint2(w0, w1);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < nv && g + i < j.n)
                    dst[i] = (uint8_t)((i < 4 ? w0 : w1) >> (8 * (i & 3)));
        }
    } else {
        uint32_t *dst = reinterpret_cast<uint32_t *>(j.out) + (uint64_t)r * (uint64_t)(Ws / 2) + c / 2;
        if (nv == 8 && ((uintptr_t)dst & 15u) == 0) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(p[0], p[1], p[2], p[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (2 * i < nv)
                    dst[i] = p[i];
        }
    }
}

// one row pair down the columns, inverse: xe (even row of pair k) and d0 (d of
// pair k) carried, c1 = the coefficients of pair k + 1; returns the even row
// ev and the odd row xo of pair k (still row-lifted)
__device__ __forceinline__ void col_unstep(const Coef &c1, bool bottom, uint32_t (&xe)[4],
                                           uint32_t (&d0)[4], uint32_t (&ev)[4], uint32_t (&xo)[4])
{
    const uint32_t s1[4] = {c1.sl[0], c1.sl[1], c1.sh[0], c1.sh[1]};
    const uint32_t d1[4] = {c1.dl[0], c1.dl[1], c1.dh[0], c1.dh[1]};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t xe1 = s1[m] - pq4(d0[m], d1[m]) + 0x20002000u; // undo Eq. 5.2
        xo[m] = d0[m] + pavg(xe[m], bottom ? xe[m] : xe1) - kB2;     // undo Eq. 5.1
        ev[m] = xe[m];
        xe[m] = xe1;
        d0[m] = d1[m];
    }
}

template <bool TOP, bool BYTES_OUT>
__device__ void inv_unit(const LevelJob &j, int sx, int sy, int lane)
{
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const int c = 240 * sx - 8 + 8 * lane; // first output column of this lane
    const int x = c >> 1;                  // first coefficient column
    const int k0 = sy * (int)j.seg_pairs;
    const int k1 = min(k0 + (int)j.seg_pairs, Hs / 2);
    const int Wl = Ws / 2, Hl = Hs / 2;
    const bool edge = (240 * sx + 248 >= Ws);
    const int n_it = k1 - k0;

    uint32_t xe[4], d0[4];
    const bool interior =
        sx >= 1 && !edge && k0 >= 1 && k1 <= Hl - 1 && (Wl & 3) == 0 && (j.Ws & 7u) == 0 &&
        ((((uintptr_t)j.hl | (uintptr_t)j.lh | (uintptr_t)j.hh | (uintptr_t)j.ll_in) & 7u) == 0) &&
        (BYTES_OUT ? (((uintptr_t)j.out & 7u) == 0 &&
                      (uint64_t)(2 * k1 - 1) * (uint64_t)Ws + (uint64_t)(240 * sx + 248) <= j.n)
                   : (((uintptr_t)j.out & 15u) == 0));
    if (interior) {
        constexpr int D = FRAG_PREFETCH_INV; // coefficient rows of loads in flight
        const uint64_t cstep = 2ull * (uint64_t)Wl; // bytes per coefficient row
        const uint64_t cb = 2ull * ((uint64_t)(k0 - 1) * (uint64_t)Wl + (uint64_t)x);
        const uint8_t *pll = j.ll_in + cb, *plh = j.lh + cb, *phl = j.hl + cb, *phh = j.hh + cb;
        auto ld = [&]() -> Coef {
            Coef cf;
            const uint2 a = __ldcg(reinterpret_cast<const uint2 *>(pll));
            const uint2 b = __ldg(reinterpret_cast<const uint2 *>(plh));
            const uint2 h = __ldg(reinterpret_cast<const uint2 *>(phl));
            const uint2 d = __ldg(reinterpret_cast<const uint2 *>(phh));
            cf.sl[0] = TOP ? from_i16x2(a.x) + 0x00800080u : a.x;
            cf.sl[1] = TOP ? from_i16x2(a.y) + 0x00800080u : a.y;
            cf.dl[0] = from_i16x2(b.x);
            cf.dl[1] = from_i16x2(b.y);
            cf.sh[0] = from_i16x2(h.x);
            cf.sh[1] = from_i16x2(h.y);
            cf.dh[0] = from_i16x2(d.x);
            cf.dh[1] = from_i16x2(d.y);
            pll += cstep;
            plh += cstep;
            phl += cstep;
            phh += cstep;
            return cf;
        };
        Coef ring[D];
        {
            const Coef prev = ld(); // row k0 - 1
            const Coef cur = ld();  // row k0
#pragma unroll
            for (int s = 0; s < D; ++s) {
                if (s < n_it)
                    ring[s] = ld(); // rows k0 + 1 ..
                else
                    ring[s] = cur;
            }
            const uint32_t dm[4] = {prev.dl[0], prev.dl[1], prev.dh[0], prev.dh[1]};
            const uint32_t s[4] = {cur.sl[0], cur.sl[1], cur.sh[0], cur.sh[1]};
            d0[0] = cur.dl[0];
            d0[1] = cur.dl[1];
            d0[2] = cur.dh[0];
            d0[3] = cur.dh[1];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                xe[i] = s[i] - pq4(dm[i], d0[i]) + 0x20002000u;
        }
        const bool own = lane >= 1 && lane <= 30;
        const uint64_t rstep = BYTES_OUT ? (uint64_t)Ws : 2ull * (uint64_t)Ws; // bytes per output row
        uint8_t *po = j.out + (uint64_t)(2 * k0) * rstep + (BYTES_OUT ? c : 2 * c);
        auto step = [&](const Coef &c1) {
            uint32_t ev[4], xo[4], ve[4], vo[4];
            col_unstep(c1, false, xe, d0, ev, xo);
            unlift_row<false>(ev, c, Ws, false, ve);
            unlift_row<false>(xo, c, Ws, false, vo);
            if (own) {
                if (BYTES_OUT) {
                    *reinterpret_cast<uint2 *>(po) = make_uint2(__byte_perm(ve[0], ve[1], 0x6420),
                                                                __byte_perm(ve[2], ve[3], 0x6420));
                    *reinterpret_cast<uint2 *>(po + rstep) = make_uint2(
                        __byte_perm(vo[0], vo[1], 0x6420), __byte_perm(vo[2], vo[3], 0x6420));
                } else {
                    *reinterpret_cast<uint4 *>(po) = make_uint4(ve[0], ve[1], ve[2], ve[3]);
                    *reinterpret_cast<uint4 *>(po + rstep) = make_uint4(vo[0], vo[1], vo[2], vo[3]);
                }
            }
            po += 2 * rstep;
        };
        int i = 0;
        for (; i + D <= n_it; i += D) {
#pragma unroll
            for (int s = 0; s < D; ++s) {
                const Coef c1 = ring[s];
                if (i + s + D < n_it)
                    ring[s] = ld();
                step(c1);
            }
        }
#pragma unroll
        for (int s = 0; s < D - 1; ++s)
            if (i + s < n_it)
                step(ring[s]);
        return;
    }

    // general path: bounds checks and the border rules, a shorter ring of
    // loads in flight
    constexpr int D = FRAG_PREFETCH_GENERAL;
    const bool vec = ((j.Ws & 7u) == 0);
    const bool own = lane >= 1 && lane <= 30 && c < Ws;
    const int nv = min(8, Ws - c);
    Coef ring[D];
    {
        const Coef cur = load_coef<TOP>(j, k0, x, vec);
        const Coef prev = load_coef<TOP>(j, max(k0 - 1, 0), x, vec);
        const uint32_t dm[4] = {k0 == 0 ? cur.dl[0] : prev.dl[0], k0 == 0 ? cur.dl[1] : prev.dl[1],
                                k0 == 0 ? cur.dh[0] : prev.dh[0], k0 == 0 ? cur.dh[1] : prev.dh[1]};
        const uint32_t s[4] = {cur.sl[0], cur.sl[1], cur.sh[0], cur.sh[1]};
        d0[0] = cur.dl[0];
        d0[1] = cur.dl[1];
        d0[2] = cur.dh[0];
        d0[3] = cur.dh[1];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            xe[i] = s[i] - pq4(dm[i], d0[i]) + 0x20002000u; // undo Eq. 5.2 down the columns
#pragma unroll
        for (int t = 0; t < D; ++t)
            ring[t] = t < n_it ? load_coef<TOP>(j, k0 + 1 + t, x, vec) : cur;
    }
    auto gstep = [&](int k, const Coef &c1) {
        uint32_t ev[4], xo[4], ve[4], vo[4];
        col_unstep(c1, 2 * k + 2 == Hs, xe, d0, ev, xo); // x[m] = x[m-2] at the bottom
        unlift_row<true>(ev, c, Ws, edge, ve);
        unlift_row<true>(xo, c, Ws, edge, vo);
        store_row<BYTES_OUT>(j, 2 * k, c, own, nv, ve);
        store_row<BYTES_OUT>(j, 2 * k + 1, c, own, nv, vo);
    };
    int i = 0;
    for (; i + D <= n_it; i += D) {
#pragma unroll
        for (int t = 0; t < D; ++t) {
            const Coef c1 = ring[t];
            if (i + t + D < n_it)
                ring[t] = load_coef<TOP>(j, k0 + 1 + i + t + D, x, vec);
            gstep(k0 + i + t, c1);
        }
    }
#pragma unroll
    for (int t = 0; t < D - 1; ++t)
        if (i + t < n_it)
            gstep(k0 + i + t, ring[t]);
}

// ---------------------------------------------------------------------------
// cipher unit: AES-128-CTR over the private fragment (LL_L, int16 LE, rows of
// 2 Ws bytes).  Segment sy owns the blocks that start in its rows [q0, q1);
// strip sx of it takes kCipherBlocks of them, one per lane at a time.
// out = in XOR keystream (in may equal out).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cipher_range(const LevelJob &j, int sx, int sy, uint64_t &bs,
                                             uint64_t &be)
{
    const uint64_t rowb = 2ull * j.Ws;
    const uint64_t q0 = (uint64_t)sy * j.seg_pairs;
    const uint64_t q1 = min(q0 + (uint64_t)j.seg_pairs, (uint64_t)j.Hs);
    const uint64_t b0 = (q0 * rowb + 15) / 16, b1 = (q1 * rowb + 15) / 16;
    bs = min(b0 + (uint64_t)sx * kCipherBlocks, b1);
    be = min(bs + kCipherBlocks, b1);
}

__device__ void cipher_unit(const LevelJob &j, int sx, int sy, const AesTab &aes, int lane,
                            const uint8_t *in, uint8_t *out, bool coherent)
{
    const uint64_t total = 2ull * j.Ws * j.Hs;
    uint64_t bs, be;
    cipher_range(j, sx, sy, bs, be);
    const bool vec = (((uintptr_t)in | (uintptr_t)out) & 15u) == 0;
    for (uint64_t b = bs + lane; b < be; b += 32) {
        uint32_t ks[4];
        aes_block(aes, j.nonce, b, ks);
        const uint64_t o = 16 * b;
        if (vec && o + 16 <= total) {
            const uint4 t = coherent ? __ldcg(reinterpret_cast<const uint4 *>(in + o))
                                     : __ldg(reinterpret_cast<const uint4 *>(in + o));
            uint4 r; // keystream bytes in stream order = big-endian words
            r.x = t.x ^ __byte_perm(ks[0], 0, 0x0123);
            r.y = t.y ^ __byte_perm(ks[1], 0, 0x0123);
            r.z = t.z ^ __byte_perm(ks[2], 0, 0x0123);
            r.w = t.w ^ __byte_perm(ks[3], 0, 0x0123);
            *reinterpret_cast<uint4 *>(out + o) = r;
        } else {
            for (int i = 0; i < 16 && o + (uint64_t)i < total; ++i) {
                const uint8_t v = coherent ? __ldcg(in + o + i) : __ldg(in + o + i);
                out[o + i] = (uint8_t)(v ^ (uint8_t)(ks[i >> 2] >> (24 - 8 * (i & 3))));
            }
        }
    }
}

} // namespace strm

// ---------------------------------------------------------------------------
// kernel: persistent warps over a dependency-ordered queue of units
// ---------------------------------------------------------------------------
constexpr int kStreamThreads = 256;

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// lane 0: wait until done[lo .. hi] all reach `target`.  Polls are relaxed
// loads with a growing sleep between them (no cache invalidation per poll);
// one acquire fence orders the unit's reads after the counts it saw.
__device__ __forceinline__ bool wait_segments(const unsigned *done, uint32_t lo, uint32_t hi,
                                              unsigned target, uint32_t spin_limit, int *err)
{
    uint32_t it = 0, ns = 128;
    for (uint32_t s = lo; s <= hi; ++s) {
        while (ld_relaxed(done + s) < target) {
            if (++it > spin_limit) {
                atomicCAS(err, 0, 3);
                return false;
            }
            __nanosleep(ns);
            ns = min(2 * ns, 2048u);
        }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return true;
}

__device__ __forceinline__ const LevelJob &dag_job(const DagWork &w, uint32_t i)
{
    return w.n_inline ? w.inline_jobs[i] : w.jobs[i];
}

// Implicit order for one buffer: job m (in processing order) runs its segment
// sy in round sy + m * lag; rounds in order, jobs in order within a round,
// strips within a job.  All jobs have the same segment count.
__device__ __forceinline__ void implicit_unit(const DagWork &w, uint64_t t, uint32_t &job,
                                              uint32_t &sx, uint32_t &sy)
{
    const int n = (int)w.n_inline;
    const int NS = (int)w.inline_jobs[0].segs;
    const int lag = (int)w.lag;
    auto before = [&](int r) -> uint64_t { // units in rounds < r
        uint64_t c = 0;
        for (int m = 0; m < n; ++m)
            c += (uint64_t)w.inline_jobs[m].strips * (uint64_t)min(max(r - lag * m, 0), NS);
        return c;
    };
    int lo = 0, hi = NS + lag * (n - 1); // before(lo) <= t < before(hi)
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (before(mid) <= t)
            lo = mid;
        else
            hi = mid;
    }
    uint64_t off = t - before(lo);
    job = 0;
    sx = sy = 0;
    for (int m = 0; m < n; ++m) {
        const int seg = lo - lag * m;
        if (seg < 0 || seg >= NS)
            continue;
        const uint64_t st = w.inline_jobs[m].strips;
        if (off < st) {
            job = (uint32_t)m;
            sx = (uint32_t)off;
            sy = (uint32_t)seg;
            return;
        }
        off -= st;
    }
}

// Segments [slo, shi] of producer p that write the data unit (j, sy) reads.
template <bool FWD>
__device__ __forceinline__ void producer_segments(const LevelJob &j, const LevelJob &p, int sx,
                                                  int sy, uint32_t &slo, uint32_t &shi)
{
    if (j.kind == kJobCipher) {
        // forward cipher after the last level: the LL_L rows its blocks touch
        const uint64_t rowb = 2ull * j.Ws;
        uint64_t bs, be;
        strm::cipher_range(j, sx, sy, bs, be);
        if (be == bs) { // nothing to do: wait for nothing
            slo = 1;
            shi = 0;
            return;
        }
        const uint64_t last = min(16 * be, rowb * j.Hs) - 1; // last byte touched
        slo = (uint32_t)(((16 * bs) / rowb) / p.seg_pairs);
        shi = (uint32_t)((last / rowb) / p.seg_pairs);
        return;
    }
    if (FWD) {
        // source rows 2 q0 - 2 .. 2 q1 of the level-(l-1) image = LL_{l-1} rows
        const int q0 = sy * (int)j.seg_pairs;
        const int q1 = min(q0 + (int)j.seg_pairs, (int)j.Hs / 2);
        slo = (uint32_t)(max(2 * q0 - 2, 0) / (int)p.seg_pairs);
        shi = (uint32_t)(min(2 * q1, (int)j.Hs - 1) / (int)p.seg_pairs);
        return;
    }
    // inverse: coefficient rows k0 - 1 .. k1 of LL_l
    const int k0 = sy * (int)j.seg_pairs;
    const int k1 = min(k0 + (int)j.seg_pairs, (int)j.Hs / 2);
    const int Hl = (int)j.Hs / 2;
    const int rlo = max(k0 - 1, 0), rhi = min(k1, Hl - 1);
    if (p.kind == kJobCipher) {
        // deciphered rows: a row is complete once every block overlapping it
        // is; block b belongs to the segment of the row it starts in
        const uint64_t rowb = 2ull * p.Ws;
        const uint64_t blo = ((uint64_t)rlo * rowb) / 16;
        const uint64_t bhi = (((uint64_t)rhi + 1) * rowb - 1) / 16;
        slo = (uint32_t)(((16 * blo) / rowb) / p.seg_pairs);
        shi = (uint32_t)(((16 * bhi) / rowb) / p.seg_pairs);
        return;
    }
    // the previous inverse level's segment s writes LL_l rows
    // [2 s seg_pairs, 2 (s + 1) seg_pairs)
    slo = (uint32_t)(rlo / (2 * (int)p.seg_pairs));
    shi = (uint32_t)(rhi / (2 * (int)p.seg_pairs));
}

// true if the unit may run (its producers are complete)
template <bool FWD>
__device__ __forceinline__ bool wait_producers(const DagWork &w, const LevelJob &j, int sx, int sy,
                                               int lane)
{
    int ok = 1;
    if (j.dep >= 0) {
        if (lane == 0) {
            const LevelJob &p = dag_job(w, (uint32_t)j.dep);
            uint32_t slo, shi;
            producer_segments<FWD>(j, p, sx, sy, slo, shi);
            shi = min(shi, p.segs - 1);
            ok = slo > shi ||
                         wait_segments(w.done + p.done_off, slo, shi, p.strips, w.spin_limit, w.err)
                     ? 1
                     : 0;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
    }
    return ok != 0;
}

template <bool FWD>
__global__ void __launch_bounds__(kStreamThreads, FRAG_BLOCKS_PER_SM) dag_kernel(DagWork w)
{
    __shared__ AesTab aes;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kAesWords; i += blockDim.x)
        (&aes.T[0][0])[i] = w.aes_tables[i];
    for (int i = threadIdx.x; i < 44; i += blockDim.x)
        aes.rk[i] = w.round_keys[i];
    __syncthreads();
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0)
            t = atomicAdd(w.queue, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= w.total_units)
            break;
        uint32_t ji, ux, uy;
        if (w.n_inline) {
            implicit_unit(w, t, ji, ux, uy);
        } else {
            const DagUnit un = w.units[t];
            ji = un.job;
            ux = un.sx;
            uy = un.sy;
        }
        const LevelJob j = dag_job(w, ji);
        const int sx = (int)ux, sy = (int)uy;
        if (wait_producers<FWD>(w, j, sx, sy, lane)) {
            if (j.kind == kJobCipher) {
                if (FWD)
                    strm::cipher_unit(j, sx, sy, aes, lane, j.ll, j.ll, true); // in place
                else
                    strm::cipher_unit(j, sx, sy, aes, lane, j.ll_in, j.out, false);
            } else if (FWD) {
                if (j.src_bytes) {
                    if (j.final_level)
                        strm::fwd_unit<true, true>(j, sx, sy, lane);
                    else
                        strm::fwd_unit<true, false>(j, sx, sy, lane);
                } else {
                    if (j.final_level)
                        strm::fwd_unit<false, true>(j, sx, sy, lane);
                    else
                        strm::fwd_unit<false, false>(j, sx, sy, lane);
                }
            } else {
                if (j.top_level) {
                    if (j.out_bytes)
                        strm::inv_unit<true, true>(j, sx, sy, lane);
                    else
                        strm::inv_unit<true, false>(j, sx, sy, lane);
                } else {
                    if (j.out_bytes)
                        strm::inv_unit<false, true>(j, sx, sy, lane);
                    else
                        strm::inv_unit<false, false>(j, sx, sy, lane);
                }
            }
        }
        // publish: every lane's stores before the count (jobs that nothing
        // in the launch reads skip it)
        if (j.publish) {
            __threadfence();
            __syncwarp();
            if (lane == 0)
                atomicAdd(w.done + j.done_off + sy, 1u);
        }
    }
}

cudaError_t launch_dag(bool fwd, const DagWork &w, uint32_t grid, cudaStream_t stream)
{
    if (fwd)
        dag_kernel<true><<<grid, kStreamThreads, 0, stream>>>(w);
    else
        dag_kernel<false><<<grid, kStreamThreads, 0, stream>>>(w);
    return cudaGetLastError();
}

cudaError_t dag_occupancy(bool fwd, int *blocks_per_sm)
{
    const void *fn = fwd ? (const void *)dag_kernel<true> : (const void *)dag_kernel<false>;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kStreamThreads, 0);
}

// A lone wait on a counter nothing increments: lets a test check that a wait
// that runs out reports FRAG_ETIMEOUT and returns.
__global__ void stall_probe_kernel(const unsigned *ctr, uint32_t spin_limit, int *err)
{
    if (threadIdx.x == 0)
        wait_segments(ctr, 0, 0, 1u, spin_limit, err);
}

cudaError_t launch_stall_probe(const unsigned *ctr, uint32_t spin_limit, int *err,
                               cudaStream_t stream)
{
    stall_probe_kernel<<<1, 32, 0, stream>>>(ctr, spin_limit, err);
    return cudaGetLastError();
}

} // namespace frag
