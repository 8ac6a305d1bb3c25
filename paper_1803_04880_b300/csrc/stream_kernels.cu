// stream_kernels.cu -- every LeGall 5/3 level of one or many buffers, and the
// AES-128-CTR pass over their private fragments, in one launch.
//
// A CTA is four consumer warps and one producer warp.  Work units (the host
// lists them so that every unit's producers come first):
//   level unit   (buffer, level l, tile, row segment): the tile is 960
//                columns of the level-(l-1) image, one 256-column strip per
//                consumer warp (lanes 1..30 own 240 columns, lanes 0 and 31
//                supply neighbours), and the unit streams down the rows of its
//                segment.
//                forward: a lane takes 8 consecutive samples of a row; the row
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
//   cipher unit  512 of the 16-byte blocks of the private fragment, XORed with
//                the AES-128 keystream of the counter block nonce || block
//                index, one block per lane at a time.  forward: in place, after
//                the last level wrote those rows; inverse: into a plaintext copy
//                that the top level reads.
//
// Data movement: the producer warp (one elected lane) dequeues units, waits
// for their producers, and streams each unit's rows (forward: image rows,
// inverse: one row of each of LL, LH, HL, HH) into a ring of shared-memory
// stages with bulk asynchronous copies (cp.async.bulk, completion counted in
// bytes on the stage's mbarrier), so many kilobytes per CTA are in flight
// without registers.  Consumers wait on a stage's "full" barrier, take their
// samples into registers and release the stage on its "empty" barrier.  A
// tile reads rows about 1 KB wide, which the DRAM serves far better than the
// 256-byte pieces of a single warp strip.  Units whose rows are not whole
// aligned runs (unaligned buffers or pitches, rows past the end of the data)
// run the general path instead: each consumer warp loads its own strip with
// bounds checks.
//
// The symmetric extension (x[-1] = x[1], x[m] = x[m-2], hence d[-1] = d[0])
// applies only at the image borders; rows above a segment are re-lifted to
// restart the column stream.
//
// Packed pairs: each 16-bit half holds v + 0x4000 (|v| < 2^14); the halves of
// (A + B) never carry into each other, so both floors of a lifting step take
// one add, one shift and one mask for two columns.
//
// Each consumer warp reports its share of a unit complete on the segment's
// counter (fence, then atomic add); there is no barrier across warps.  Every
// wait is bounded.  A dependency wait that runs out sets the error word to 3
// (FRAG_ETIMEOUT) and the unit is skipped but still reported complete, so no
// consumer waits forever; a stage wait that runs out sets the error word to 4
// and the CTA stops (the producer first waits, bounded, for its copies).
#include "frag_internal.cuh"
#include "swar.cuh"

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

// tuning knobs: ring stages per CTA, KiB per stage, resident CTAs per SM the
// kernel is compiled for
#ifndef FRAG_STAGES
#define FRAG_STAGES 3
#endif
#ifndef FRAG_STAGE_KB
#define FRAG_STAGE_KB 16
#endif
#ifndef FRAG_CTAS_PER_SM
#define FRAG_CTAS_PER_SM 4
#endif

constexpr int kConsumerWarps = (int)kTileStrips;
constexpr int kCtaThreads = 32 * (kConsumerWarps + 1);
constexpr int kStages = FRAG_STAGES;
// A stage is a run of row slots: forward 1 KB (byte rows) or 2 KB (packed
// rows) per image row, inverse 4 KB per coefficient row (LL, LH, HL, HH in
// 1 KB slots).  Few large stages keep the handshakes per byte low.
constexpr int kStageBytes = FRAG_STAGE_KB * 1024;
constexpr int kCoefSlot = 1024;
constexpr int kCoefRow = 4 * kCoefSlot;
constexpr int kTileCols = kConsumerWarps * kStripCols; // 960
constexpr uint32_t kStageSpin = 1u << 23;              // tests of a stage barrier before giving up

// stage kinds
constexpr uint32_t kModeEnd = 0;      // no more units
constexpr uint32_t kModeBulk = 1;     // rows streamed into the ring
constexpr uint32_t kModeGeneral = 3;  // consumers load their own strips (bounds checked)
constexpr uint32_t kModeCipher = 4;   // AES-CTR blocks
constexpr uint32_t kModeSkip = 5;     // a dependency wait ran out: report complete, do nothing

// written by the producer into the first stage of every unit
struct StageHdr {
    LevelJob job;
    uint32_t x, y, mode, pad;
};

namespace strm {

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
__device__ __forceinline__ uint2 ll_out(bool final_level, const uint32_t (&sv)[4])
{
    if (final_level)
        return make_uint2(to_i16x2(sv[0] - 0x00800080u), to_i16x2(sv[1] - 0x00800080u));
    return make_uint2(sv[0], sv[1]);
}

// ---------------------------------------------------------------------------
// bounds-checked global memory helpers (general path)
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

// the four outputs of one row pair of one lane (checked stores)
__device__ __forceinline__ void fwd_store(const LevelJob &j, int Wl, int q, int x, int nval,
                                          const uint32_t (&sv)[4], const uint32_t (&dv)[4])
{
    // sv[0..1] = LL, sv[2..3] = HL, dv[0..1] = LH, dv[2..3] = HH
    store4(j.hl, Wl, q, x, to_i16x2(sv[2]), to_i16x2(sv[3]), nval);
    store4(j.lh, Wl, q, x, to_i16x2(dv[0]), to_i16x2(dv[1]), nval);
    store4(j.hh, Wl, q, x, to_i16x2(dv[2]), to_i16x2(dv[3]), nval);
    const uint2 ll = ll_out(j.final_level, sv);
    if (j.final_level) {
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

// ---------------------------------------------------------------------------
// forward level: general path (one warp, one 256-column strip)
// ---------------------------------------------------------------------------
template <bool BYTES>
__device__ void fwd_general(const LevelJob &j, int sx, int sy, int lane)
{
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const int c = kStripCols * sx - 8 + 8 * lane; // first column of this lane
    const int q0 = sy * (int)j.seg_pairs;
    const int q1 = min(q0 + (int)j.seg_pairs, Hs / 2);
    const int Wl = Ws / 2;
    const int x = c / 2; // level-l column of the lane's first value
    const bool edge = (kStripCols * sx + 248 >= Ws);
    const bool vec = BYTES ? (((j.Ws & 7u) == 0) && (((uintptr_t)j.src & 7u) == 0))
                           : (((j.Ws & 7u) == 0) && (((uintptr_t)j.src & 15u) == 0));
    const bool own = lane >= 1 && lane <= 30 && x < Wl;
    const int nval = min(4, Wl - x);
    uint32_t e0[4], dp[4];
    {
        uint32_t a[4], o[4];
        const Raw r0 = load_row<BYTES>(j, 2 * q0, c, vec);
        const Raw rm2 = load_row<BYTES>(j, max(2 * q0 - 2, 0), c, vec);
        const Raw rm1 = load_row<BYTES>(j, max(2 * q0 - 1, 0), c, vec);
        lift_row<BYTES, true>(r0, c, Ws, edge, e0);
        lift_row<BYTES, true>(rm2, c, Ws, edge, a);
        lift_row<BYTES, true>(rm1, c, Ws, edge, o);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            dp[i] = o[i] - pavg(a[i], e0[i]) + kB2;
    }
    Raw n1 = load_row<BYTES>(j, 2 * q0 + 1, c, vec);
    Raw n2 = load_row<BYTES>(j, 2 * q0 + 2, c, vec);
    for (int q = q0; q < q1; ++q) {
        const Raw c1 = n1, c2 = n2;
        if (q + 1 < q1) {
            n1 = load_row<BYTES>(j, 2 * q + 3, c, vec);
            n2 = load_row<BYTES>(j, 2 * q + 4, c, vec);
        }
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
        if (own)
            fwd_store(j, Wl, q, x, nval, sv, dv);
    }
}

// ---------------------------------------------------------------------------
// inverse level: general path
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
    if (j.top_level) {
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

// start of the column inverse at pair k0: xe = even row of pair k0, d0 = d of
// pair k0 (prev = coefficients of pair k0 - 1, ignored at the top border)
__device__ __forceinline__ void col_unstart(const Coef &prev, const Coef &cur, bool top,
                                            uint32_t (&xe)[4], uint32_t (&d0)[4])
{
    const uint32_t dm[4] = {top ? cur.dl[0] : prev.dl[0], top ? cur.dl[1] : prev.dl[1],
                            top ? cur.dh[0] : prev.dh[0], top ? cur.dh[1] : prev.dh[1]};
    const uint32_t s[4] = {cur.sl[0], cur.sl[1], cur.sh[0], cur.sh[1]};
    d0[0] = cur.dl[0];
    d0[1] = cur.dl[1];
    d0[2] = cur.dh[0];
    d0[3] = cur.dh[1];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        xe[i] = s[i] - pq4(dm[i], d0[i]) + 0x20002000u; // undo Eq. 5.2 down the columns
}

template <bool BYTES_OUT>
__device__ void inv_general(const LevelJob &j, int sx, int sy, int lane)
{
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const int c = kStripCols * sx - 8 + 8 * lane; // first output column of this lane
    const int x = c >> 1;                         // first coefficient column
    const int k0 = sy * (int)j.seg_pairs;
    const int k1 = min(k0 + (int)j.seg_pairs, Hs / 2);
    const bool edge = (kStripCols * sx + 248 >= Ws);
    const bool vec = ((j.Ws & 7u) == 0);
    const bool own = lane >= 1 && lane <= 30 && c < Ws;
    const int nv = min(8, Ws - c);
    uint32_t xe[4], d0[4];
    {
        const Coef cur = load_coef(j, k0, x, vec);
        const Coef prev = load_coef(j, max(k0 - 1, 0), x, vec);
        col_unstart(prev, cur, k0 == 0, xe, d0);
    }
    Coef nxt = load_coef(j, k0 + 1, x, vec);
    for (int k = k0; k < k1; ++k) {
        const Coef c1 = nxt;
        if (k + 1 < k1)
            nxt = load_coef(j, k + 2, x, vec);
        uint32_t ev[4], xo[4], ve[4], vo[4];
        col_unstep(c1, 2 * k + 2 == Hs, xe, d0, ev, xo); // x[m] = x[m-2] at the bottom
        unlift_row<true>(ev, c, Ws, edge, ve);
        unlift_row<true>(xo, c, Ws, edge, vo);
        store_row<BYTES_OUT>(j, 2 * k, c, own, nv, ve);
        store_row<BYTES_OUT>(j, 2 * k + 1, c, own, nv, vo);
    }
}

// ---------------------------------------------------------------------------
// cipher: AES-128-CTR over the private fragment (LL_L, int16 LE, rows of
// 2 Ws bytes).  Segment sy owns the blocks that start in its rows [q0, q1);
// unit sx of it takes kCipherBlocks of them, an equal share per consumer
// warp, one per lane at a time.  out = in XOR keystream (in may equal out).
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

__device__ void cipher_warp(const LevelJob &j, int sx, int sy, int w, const AesTab &aes, int lane,
                            const uint8_t *in, uint8_t *out, bool coherent)
{
    const uint64_t total = 2ull * j.Ws * j.Hs;
    uint64_t bs, be;
    cipher_range(j, sx, sy, bs, be);
    constexpr uint32_t per_warp = kCipherBlocks / kConsumerWarps;
    const uint64_t ws = min(bs + (uint64_t)w * per_warp, be), we = min(ws + per_warp, be);
    const bool vec = (((uintptr_t)in | (uintptr_t)out) & 15u) == 0;
    for (uint64_t b = ws + lane; b < we; b += 32) {
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
// shared-memory stage ring
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// one test of the phase; the thread may sleep up to about 1 us for it first
__device__ __forceinline__ bool mbar_try_wait(const uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity), "n"(1000)
                 : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity; false if it ran out
__device__ __forceinline__ bool mbar_wait(const uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < kStageSpin; ++it)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy of `bytes` (16-byte aligned addresses, size a
// multiple of 16), completion counted on `bar`
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                     "r"(smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

struct Ring {
    uint8_t *data;   // kStages x kStageBytes
    uint64_t *full;  // producer arrival + copied bytes
    uint64_t *empty; // one arrival per consumer warp
    StageHdr *hdr;
    int *err;
};

// consumer side: wait until stage `it` is full (all lanes); nullptr if the
// wait ran out (error word set).  A phase, once complete, stays visible until
// this warp releases the stage, so a lane that gave up just before another saw
// it complete looks again.
__device__ __forceinline__ const uint8_t *ring_wait(Ring r, uint32_t it)
{
    const uint32_t s = it % kStages, parity = (it / kStages) & 1u;
    bool ok = mbar_wait(r.full + s, parity);
    if (__any_sync(0xffffffffu, ok) && !ok)
        ok = mbar_wait(r.full + s, parity);
    if (!__all_sync(0xffffffffu, ok)) {
        if ((threadIdx.x & 31) == 0)
            atomicCAS(r.err, 0, 4);
        return nullptr;
    }
    return r.data + s * kStageBytes;
}

// consumer side: this warp is done reading stage `it`
__device__ __forceinline__ void ring_release(Ring r, uint32_t it)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0)
        mbar_arrive(r.empty + it % kStages);
}

// ---------------------------------------------------------------------------
// bulk consumers (one warp, one strip of the tile)
// ---------------------------------------------------------------------------
namespace strm {

// The stages of one unit, read in order: a warp holds one stage at a time and
// releases it when it moves on.
struct Cursor {
    Ring ring;
    uint32_t base;     // ring index of the unit's first stage
    int cur;           // stage of the unit held now
    const uint8_t *st; // its data

    __device__ __forceinline__ Cursor(Ring r, uint32_t b, const uint8_t *first)
        : ring(r), base(b), cur(0), st(first)
    {
    }

    // move to the next stage; false if the wait ran out
    __device__ __forceinline__ bool next()
    {
        ring_release(ring, base + cur);
        ++cur;
        st = ring_wait(ring, base + cur);
        return st != nullptr;
    }

    __device__ __forceinline__ void finish(uint32_t &it, int nstages)
    {
        ring_release(ring, base + cur);
        it = base + nstages;
    }
};

// a warp with no strip in the tile still takes part in every stage
__device__ __forceinline__ bool skip_stages(Ring ring, uint32_t &it, int nstages)
{
    ring_release(ring, it);
    for (int k = 1; k < nstages; ++k) {
        if (ring_wait(ring, it + k) == nullptr)
            return false;
        ring_release(ring, it + k);
    }
    it += nstages;
    return true;
}

// samples of the lane from a row slot: the slot holds columns [C0 - 16, ...)
// of the row; the lane's columns start `off` bytes into the slot
template <bool BYTES>
__device__ __forceinline__ Raw slot_row(const uint8_t *slot, int off)
{
    Raw r;
    if (BYTES) {
        const uint2 t = *reinterpret_cast<const uint2 *>(slot + off);
        r.w[0] = t.x;
        r.w[1] = t.y;
        r.w[2] = r.w[3] = 0;
    } else {
        const uint4 t = *reinterpret_cast<const uint4 *>(slot + off);
        r.w[0] = t.x;
        r.w[1] = t.y;
        r.w[2] = t.z;
        r.w[3] = t.w;
    }
    return r;
}

template <bool BYTES>
__host__ __device__ constexpr int fwd_slot_bytes()
{
    return BYTES ? 1024 : 2048;
}

// The symmetric extension at the column borders, written into a row slot
// before it is read: x[-k] = x[k] for k = 1..8 (the halo lane's samples: the
// lifting needs x[-2], x[-1] for d[-1] = d[0], and every packed half must
// hold an in-range value so that no carry crosses into its neighbour) and
// x[Ws] = x[Ws - 2].  The slot holds columns [C0 - 16, ...); the copy leaves
// those positions unwritten, and only the border warp's own lanes use them.
template <bool BYTES>
__device__ __forceinline__ void mirror_slot(uint8_t *slot, bool left, int right_col)
{
    constexpr int e = BYTES ? 1 : 2; // bytes per sample
#pragma unroll
    for (int b = 0; b < e; ++b) {
        if (left) {
#pragma unroll
            for (int k = 1; k <= 8; ++k)
                slot[(16 - k) * e + b] = slot[(16 + k) * e + b];
        }
        if (right_col >= 0)
            slot[(right_col + 16) * e + b] = slot[(right_col + 14) * e + b];
    }
}

// Forward bulk unit.  Row slot u = 1 .. 2 n + 3 of the unit holds image row
// 2 q0 - 3 + u (slot 0 stays empty so that every row pair 2q+1, 2q+2 sits in
// one stage; rows outside the image are not copied and not used), rps slots
// per stage; stage 0 (already waited for) is at `it`.  The warps that hold
// a column border mirror the samples beyond it into the slot first, so every
// row lifts with the interior formula; bulk units have whole aligned rows, so
// the outputs leave as plain vector stores.  Returns false if a stage wait
// ran out.
template <bool BYTES>
__device__ bool fwd_bulk(const LevelJob &j, int tx, int sy, int w, int lane, Ring ring,
                         uint32_t &it, const uint8_t *st0)
{
    constexpr int slot = fwd_slot_bytes<BYTES>(), rps = kStageBytes / slot;
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const int sx = kConsumerWarps * tx + w;
    const int C0 = kTileCols * tx;
    const int c = kStripCols * sx - 8 + 8 * lane;
    const int off = (kStripCols * w + 8 + 8 * lane) * (BYTES ? 1 : 2); // byte offset of c in a slot
    const int q0 = sy * (int)j.seg_pairs;
    const int q1 = min(q0 + (int)j.seg_pairs, Hs / 2);
    const int n_it = q1 - q0;
    const int nstages = (2 * n_it + 4 + rps - 1) / rps;
    if (sx >= (int)j.wstrips)
        return skip_stages(ring, it, nstages);
    const int Wl = Ws / 2;
    const int x = c / 2;
    const bool own = lane >= 1 && lane <= 30 && x < Wl;
    const bool top = q0 == 0, bottom = 2 * q1 >= Hs, final_level = j.final_level;
    // border work of this warp (uniform): left border, right border column
    const bool left = sx == 0;
    const int right_col = (kStripCols * sx + 248 >= Ws) ? Ws - C0 : -1;
    const bool border = left || right_col >= 0;
    auto row = [&](const uint8_t *slot_base) -> Raw {
        if (border) {
            if (lane == 0)
                mirror_slot<BYTES>(const_cast<uint8_t *>(slot_base), left, right_col);
            __syncwarp();
            asm volatile("" ::: "memory"); // the slot reads below come after the patch
        }
        return slot_row<BYTES>(slot_base, off);
    };
    Cursor cu(ring, it, st0);
    uint32_t e0[4], dp[4];
    {
        const Raw rm2 = row(cu.st + 1 * slot);
        const Raw rm1 = row(cu.st + 2 * slot);
        const Raw r0 = row(cu.st + 3 * slot);
        uint32_t a[4], o[4];
        lift_row<BYTES, false>(r0, c, Ws, false, e0);
        lift_row<BYTES, false>(rm2, c, Ws, false, a);
        lift_row<BYTES, false>(rm1, c, Ws, false, o);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            dp[i] = o[i] - pavg(a[i], e0[i]) + kB2; // (replaced at the top border)
    }
    const uint64_t ostep = 2ull * (uint64_t)Wl;
    const uint64_t o0 = 2ull * ((uint64_t)q0 * (uint64_t)Wl + (uint64_t)x);
    uint8_t *phl = j.hl + o0, *plh = j.lh + o0, *phh = j.hh + o0, *pll = j.ll + o0;
    const uint8_t *p = cu.st + 4 * slot; // slot of row 2 q0 + 1
    int left_slots = rps - 4;            // slots of the held stage still to read
    for (int q = q0; q < q1; ++q) {
        if (left_slots == 0) {
            if (!cu.next())
                return false;
            p = cu.st;
            left_slots = rps;
        }
        const Raw c1 = row(p), c2 = row(p + slot);
        p += 2 * slot;
        left_slots -= 2;
        uint32_t o[4], e1[4], sv[4], dv[4];
        lift_row<BYTES, false>(c1, c, Ws, false, o);
        if (bottom && 2 * q + 2 == Hs) { // x[m] = x[m-2] at the bottom border
#pragma unroll
            for (int k = 0; k < 4; ++k)
                e1[k] = e0[k];
        } else {
            lift_row<BYTES, false>(c2, c, Ws, false, e1);
        }
        col_step(o, e1, e0, dp, top && q == 0, sv, dv);
        // sv[0..1] = LL, sv[2..3] = HL, dv[0..1] = LH, dv[2..3] = HH
        if (own) {
            *reinterpret_cast<uint2 *>(phl) = make_uint2(to_i16x2(sv[2]), to_i16x2(sv[3]));
            *reinterpret_cast<uint2 *>(plh) = make_uint2(to_i16x2(dv[0]), to_i16x2(dv[1]));
            *reinterpret_cast<uint2 *>(phh) = make_uint2(to_i16x2(dv[2]), to_i16x2(dv[3]));
            *reinterpret_cast<uint2 *>(pll) = ll_out(final_level, sv);
        }
        phl += ostep;
        plh += ostep;
        phh += ostep;
        pll += ostep;
    }
    cu.finish(it, nstages);
    return true;
}

// coefficients of the lane from a coefficient-row slot: four 1 KB arrays (LL,
// LH, HL, HH), each holding coefficient columns [C0/2 - 8, ...) of one row
__device__ __forceinline__ Coef slot_coef(const uint8_t *st, int off, bool top)
{
    const uint2 a = *reinterpret_cast<const uint2 *>(st + off);
    const uint2 b = *reinterpret_cast<const uint2 *>(st + kCoefSlot + off);
    const uint2 h = *reinterpret_cast<const uint2 *>(st + 2 * kCoefSlot + off);
    const uint2 d = *reinterpret_cast<const uint2 *>(st + 3 * kCoefSlot + off);
    Coef cf;
    cf.sl[0] = top ? from_i16x2(a.x) + 0x00800080u : a.x;
    cf.sl[1] = top ? from_i16x2(a.y) + 0x00800080u : a.y;
    cf.dl[0] = from_i16x2(b.x);
    cf.dl[1] = from_i16x2(b.y);
    cf.sh[0] = from_i16x2(h.x);
    cf.sh[1] = from_i16x2(h.y);
    cf.dh[0] = from_i16x2(d.x);
    cf.dh[1] = from_i16x2(d.y);
    return cf;
}

// Inverse bulk unit.  Unit rows t = 0 .. n + 1 are coefficient rows k0 - 1 + t
// (rows outside the bands are not copied and not used), kStageBytes /
// kCoefRow per stage; stage 0 (already waited for) is at `it`.  Stores are
// checked and the symmetric extension applies where a strip reaches a
// border.  Returns false if a stage wait ran out.
template <bool BYTES_OUT>
__device__ bool inv_bulk(const LevelJob &j, int tx, int sy, int w, int lane, Ring ring,
                         uint32_t &it, const uint8_t *st0)
{
    constexpr int rps = kStageBytes / kCoefRow;
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const int sx = kConsumerWarps * tx + w;
    const int c = kStripCols * sx - 8 + 8 * lane;
    const int off = 2 * (kStripCols / 2 * w + 4 + 4 * lane); // slot byte offset of coefficient c/2
    const int k0 = sy * (int)j.seg_pairs;
    const int k1 = min(k0 + (int)j.seg_pairs, Hs / 2);
    const int n_it = k1 - k0;
    const int nstages = (n_it + 2 + rps - 1) / rps;
    if (sx >= (int)j.wstrips)
        return skip_stages(ring, it, nstages);
    const bool edge = (kStripCols * sx + 248 >= Ws);
    const bool own = lane >= 1 && lane <= 30 && c < Ws;
    const int nv = min(8, Ws - c);
    const bool bottom = 2 * k1 >= Hs, top_level = j.top_level;
    Cursor cu(ring, it, st0);
    uint32_t xe[4], d0[4];
    {
        const Coef prev = slot_coef(cu.st + off, 0, top_level);
        const Coef cur = slot_coef(cu.st + kCoefRow + off, 0, top_level);
        col_unstart(prev, cur, k0 == 0, xe, d0);
    }
    const uint8_t *p = cu.st + 2 * kCoefRow + off;
    int left = rps - 2;
    for (int k = k0; k < k1; ++k) {
        if (left == 0) {
            if (!cu.next())
                return false;
            p = cu.st + off;
            left = rps;
        }
        const Coef c1 = slot_coef(p, 0, top_level);
        p += kCoefRow;
        --left;
        uint32_t ev[4], xo[4], ve[4], vo[4];
        col_unstep(c1, bottom && 2 * k + 2 == Hs, xe, d0, ev, xo);
        unlift_row<true>(ev, c, Ws, edge, ve);
        unlift_row<true>(xo, c, Ws, edge, vo);
        store_row<BYTES_OUT>(j, 2 * k, c, own, nv, ve);
        store_row<BYTES_OUT>(j, 2 * k + 1, c, own, nv, vo);
    }
    cu.finish(it, nstages);
    return true;
}

} // namespace strm

// ---------------------------------------------------------------------------
// work queue, dependencies
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// wait until done[lo .. hi] all reach `target`.  Polls are relaxed loads with
// a growing sleep between them (no cache invalidation per poll); one acquire
// fence orders what follows after the counts seen.
__device__ __forceinline__ bool wait_segments(const unsigned *done, uint32_t lo, uint32_t hi,
                                              unsigned target, uint32_t spin_limit, int *err)
{
    uint32_t it = 0, ns = 64;
    for (uint32_t s = lo; s <= hi; ++s) {
        while (ld_relaxed(done + s) < target) {
            if (++it > spin_limit) {
                atomicCAS(err, 0, 3);
                return false;
            }
            __nanosleep(ns);
            ns = min(2 * ns, 1024u);
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
// units within a job.  All jobs have the same segment count.
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

// Segments [slo, shi] of job j.dep that write the data unit (j, sx, sy) reads.
template <bool FWD>
__device__ __forceinline__ void producer_segments(const LevelJob &j, int sx, int sy, uint32_t &slo,
                                                  uint32_t &shi)
{
    const uint32_t p_seg_pairs = j.dep_seg_pairs;
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
        slo = (uint32_t)(((16 * bs) / rowb) / p_seg_pairs);
        shi = (uint32_t)((last / rowb) / p_seg_pairs);
        return;
    }
    if (FWD) {
        // source rows 2 q0 - 2 .. 2 q1 of the level-(l-1) image = LL_{l-1} rows
        const int q0 = sy * (int)j.seg_pairs;
        const int q1 = min(q0 + (int)j.seg_pairs, (int)j.Hs / 2);
        slo = (uint32_t)(max(2 * q0 - 2, 0) / (int)p_seg_pairs);
        shi = (uint32_t)(min(2 * q1, (int)j.Hs - 1) / (int)p_seg_pairs);
        return;
    }
    // inverse: coefficient rows k0 - 1 .. k1 of LL_l
    const int k0 = sy * (int)j.seg_pairs;
    const int k1 = min(k0 + (int)j.seg_pairs, (int)j.Hs / 2);
    const int Hl = (int)j.Hs / 2;
    const int rlo = max(k0 - 1, 0), rhi = min(k1, Hl - 1);
    if (j.dep_kind == kJobCipher) {
        // deciphered rows: a row is complete once every block overlapping it
        // is; block b belongs to the segment of the row it starts in
        const uint64_t rowb = 2ull * j.dep_Ws;
        const uint64_t blo = ((uint64_t)rlo * rowb) / 16;
        const uint64_t bhi = (((uint64_t)rhi + 1) * rowb - 1) / 16;
        slo = (uint32_t)(((16 * blo) / rowb) / p_seg_pairs);
        shi = (uint32_t)(((16 * bhi) / rowb) / p_seg_pairs);
        return;
    }
    // the previous inverse level's segment s writes LL_l rows
    // [2 s seg_pairs, 2 (s + 1) seg_pairs)
    slo = (uint32_t)(rlo / (2 * (int)p_seg_pairs));
    shi = (uint32_t)(rhi / (2 * (int)p_seg_pairs));
}

// ---------------------------------------------------------------------------
// producer: one elected lane of the producer warp
// ---------------------------------------------------------------------------
struct Producer {
    Ring ring;
    uint32_t it = 0; // stages issued

    __device__ explicit Producer(Ring r) : ring(r) {}

    // claim the next stage (bounded wait for the consumers to release it)
    __device__ __forceinline__ uint8_t *claim(uint32_t &s)
    {
        s = it % kStages;
        if (it >= (uint32_t)kStages && !mbar_wait(ring.empty + s, ((it / kStages) - 1) & 1u)) {
            atomicCAS(ring.err, 0, 4);
            return nullptr;
        }
        // the consumers' reads of the previous contents come before the copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        return ring.data + s * kStageBytes;
    }

    // the header of a unit's first stage: the job descriptor and the unit
    __device__ __forceinline__ void header(uint32_t s, const LevelJob &job, uint32_t x, uint32_t y,
                                           uint32_t mode)
    {
        StageHdr &h = ring.hdr[s];
        h.job = job;
        h.x = x;
        h.y = y;
        h.mode = mode;
    }

    // a stage holding only a header
    __device__ __forceinline__ bool emit(const LevelJob &job, uint32_t x, uint32_t y, uint32_t mode)
    {
        uint32_t s;
        if (claim(s) == nullptr)
            return false;
        header(s, job, x, y, mode);
        mbar_arrive(ring.full + s);
        ++it;
        return true;
    }

    // the end-of-work stage
    __device__ __forceinline__ bool finish()
    {
        uint32_t s;
        if (claim(s) == nullptr)
            return false;
        ring.hdr[s].mode = kModeEnd;
        mbar_arrive(ring.full + s);
        ++it;
        return true;
    }

    // wait (bounded) for the copies of the last stages issued
    __device__ void drain()
    {
        const uint32_t first = it > (uint32_t)kStages ? it - kStages : 0;
        for (uint32_t i = first; i < it; ++i)
            mbar_wait(ring.full + i % kStages, (i / kStages) & 1u);
    }
};

// Forward bulk stages of unit (j, tx, sy): row slot u = 1 .. 2 n + 3 holds
// image row 2 q0 - 3 + u, copied as columns [C0 - 16, C0 + 976) clipped to the
// image (element size 1 for bytes, 2 for packed pairs).
__device__ bool produce_fwd(Producer &pr, const LevelJob &j, int tx, int sy, uint32_t mode)
{
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const bool bytes_src = j.src_bytes;
    const uint32_t esz = bytes_src ? 1u : 2u;
    const int slot = bytes_src ? strm::fwd_slot_bytes<true>() : strm::fwd_slot_bytes<false>();
    const int rps = kStageBytes / slot;
    const int C0 = kTileCols * tx;
    const int lo = max(C0 - 16, 0), hi = min(C0 + kTileCols + 16, Ws);
    const uint32_t bytes = (uint32_t)(hi - lo) * esz;
    const uint32_t dst = (uint32_t)(lo - (C0 - 16)) * esz;
    const int q0 = sy * (int)j.seg_pairs;
    const int q1 = min(q0 + (int)j.seg_pairs, Hs / 2);
    // slot u = 1 .. 2 n + 3 holds image row r0 + u (slot 0 stays empty)
    const int U = 2 * (q1 - q0) + 4, r0 = 2 * q0 - 3;
    for (int u0 = 0; u0 < U; u0 += rps) {
        const int u1 = min(u0 + rps, U);
        uint32_t s;
        uint8_t *st = pr.claim(s);
        if (st == nullptr)
            return false;
        if (u0 == 0)
            pr.header(s, j, (uint32_t)tx, (uint32_t)sy, mode);
        // rows of the image in this stage: [ra, rb)
        const int ra = max(r0 + max(u0, 1), 0), rb = min(r0 + u1, Hs);
        if (rb <= ra) {
            mbar_arrive(pr.ring.full + s);
        } else {
            mbar_arrive_tx(pr.ring.full + s, (uint32_t)(rb - ra) * bytes);
            for (int r = ra; r < rb; ++r)
                bulk_copy(st + (r - r0 - u0) * slot + dst, j.src + ((uint64_t)r * Ws + lo) * esz,
                          bytes, pr.ring.full + s);
        }
        ++pr.it;
    }
    return true;
}

// Inverse bulk stages of unit (j, tx, sy): unit rows t = 0 .. n + 1 are
// coefficient rows k0 - 1 + t of LL, LH, HL, HH, columns [C0/2 - 8,
// C0/2 + 488) clipped to the band, one 4 KB coefficient-row slot each.
__device__ bool produce_inv(Producer &pr, const LevelJob &j, int tx, int sy, uint32_t mode)
{
    constexpr int rps = kStageBytes / kCoefRow;
    const int Hl = (int)j.Hs / 2, Wl = (int)j.Ws / 2;
    const int X0 = kTileCols / 2 * tx - 8;
    const int lo = max(X0, 0), hi = min(X0 + kTileCols / 2 + 16, Wl);
    const uint32_t bytes = 2u * (uint32_t)(hi - lo);
    const uint32_t dst = 2u * (uint32_t)(lo - X0);
    const int k0 = sy * (int)j.seg_pairs;
    const int k1 = min(k0 + (int)j.seg_pairs, Hl);
    const int T = k1 - k0 + 2, r0 = k0 - 1;
    const uint8_t *arr[4] = {j.ll_in, j.lh, j.hl, j.hh};
    for (int t0 = 0; t0 < T; t0 += rps) {
        const int t1 = min(t0 + rps, T);
        uint32_t s;
        uint8_t *st = pr.claim(s);
        if (st == nullptr)
            return false;
        if (t0 == 0)
            pr.header(s, j, (uint32_t)tx, (uint32_t)sy, mode);
        const int ra = max(r0 + t0, 0), rb = min(r0 + t1, Hl);
        if (rb <= ra) {
            mbar_arrive(pr.ring.full + s);
        } else {
            mbar_arrive_tx(pr.ring.full + s, (uint32_t)(rb - ra) * 4u * bytes);
            for (int r = ra; r < rb; ++r) {
                const uint64_t o = 2ull * ((uint64_t)r * Wl + lo);
                uint8_t *row = st + (r - r0 - t0) * kCoefRow + dst;
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    bulk_copy(row + a * kCoefSlot, arr[a] + o, bytes, pr.ring.full + s);
            }
        }
        ++pr.it;
    }
    return true;
}

// Which path unit (j, tx, sy) takes: bulk rows need whole aligned runs (the
// host sets j.bulk when bases and pitches allow it); forward byte sources also
// need every row read to lie before n.
template <bool FWD>
__device__ __forceinline__ uint32_t unit_mode(const LevelJob &j, int sy)
{
    if (!j.bulk)
        return kModeGeneral;
    if (FWD && j.src_bytes) {
        const int Hs = (int)j.Hs;
        const int p1 = min(sy * (int)j.seg_pairs + (int)j.seg_pairs, Hs / 2);
        if ((uint64_t)(min(2 * p1, Hs - 1) + 1) * (uint64_t)j.Ws > j.n)
            return kModeGeneral;
    }
    return kModeBulk;
}

// unit t of the launch: (job, x, y)
__device__ __forceinline__ void unit_at(const DagWork &w, uint64_t t, uint32_t &ji, uint32_t &ux,
                                        uint32_t &uy)
{
    if (w.n_inline) {
        implicit_unit(w, t, ji, ux, uy);
    } else {
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(w.units + t));
        ji = u.x;
        ux = u.y;
        uy = u.z;
    }
}

// job descriptor i, through the read-only cache for a batch
__device__ __forceinline__ LevelJob load_job(const DagWork &w, uint32_t i)
{
    if (w.n_inline)
        return w.inline_jobs[i];
    LevelJob j;
    const uint4 *src = reinterpret_cast<const uint4 *>(w.jobs + i);
    uint4 *dst = reinterpret_cast<uint4 *>(&j);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(LevelJob) / 16); ++k)
        dst[k] = __ldg(src + k);
    return j;
}

// The producer claims units from the queue, one ahead: the claim of the next
// unit and its index are in flight while the current unit streams.  A CTA
// only ever holds the unit it streams and the one after it, both later in
// the queue than everything they wait for, so every wait ends once earlier
// units finish -- whether or not the whole grid is resident.
template <bool FWD>
__device__ void producer_loop(const DagWork &w, Ring ring)
{
    Producer pr(ring);
    unsigned long long t = atomicAdd(w.queue, 1ull);
    uint32_t ji = 0, ux = 0, uy = 0;
    if (t < w.total_units)
        unit_at(w, t, ji, ux, uy);
    while (t < w.total_units) {
        const unsigned long long nt = atomicAdd(w.queue, 1ull);
        const LevelJob j = load_job(w, ji);
        bool ok = true;
        if (j.dep >= 0) {
            uint32_t slo, shi;
            producer_segments<FWD>(j, (int)ux, (int)uy, slo, shi);
            shi = min(shi, j.dep_segs - 1);
            if (slo <= shi)
                ok = wait_segments(w.done + j.dep_done_off, slo, shi, j.dep_units * kConsumerWarps,
                                   w.spin_limit, w.err);
            // what other CTAs wrote through the generic proxy is read next by bulk copies
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        bool fine;
        if (!ok) {
            fine = pr.emit(j, ux, uy, kModeSkip);
        } else if (j.kind == kJobCipher) {
            fine = pr.emit(j, ux, uy, kModeCipher);
        } else {
            const uint32_t mode = unit_mode<FWD>(j, (int)uy);
            if (mode == kModeGeneral)
                fine = pr.emit(j, ux, uy, kModeGeneral);
            else
                fine = FWD ? produce_fwd(pr, j, (int)ux, (int)uy, mode)
                           : produce_inv(pr, j, (int)ux, (int)uy, mode);
        }
        if (!fine) { // a stage wait ran out: stop issuing, let the copies land
            pr.drain();
            return;
        }
        t = nt;
        if (t < w.total_units)
            unit_at(w, t, ji, ux, uy);
    }
    pr.finish();
}

// ---------------------------------------------------------------------------
// consumers
// ---------------------------------------------------------------------------
template <bool FWD>
__device__ bool run_bulk(const LevelJob &j, int tx, int sy, int w, int lane, Ring ring,
                         uint32_t &it, const uint8_t *st0)
{
    if (FWD)
        return j.src_bytes ? strm::fwd_bulk<true>(j, tx, sy, w, lane, ring, it, st0)
                           : strm::fwd_bulk<false>(j, tx, sy, w, lane, ring, it, st0);
    return j.out_bytes ? strm::inv_bulk<true>(j, tx, sy, w, lane, ring, it, st0)
                       : strm::inv_bulk<false>(j, tx, sy, w, lane, ring, it, st0);
}

template <bool FWD>
__device__ void run_general(const LevelJob &j, int tx, int sy, int w, int lane)
{
    const int sx = kConsumerWarps * tx + w;
    if (sx >= (int)j.wstrips)
        return;
    if (FWD) {
        if (j.src_bytes)
            strm::fwd_general<true>(j, sx, sy, lane);
        else
            strm::fwd_general<false>(j, sx, sy, lane);
    } else {
        if (j.out_bytes)
            strm::inv_general<true>(j, sx, sy, lane);
        else
            strm::inv_general<false>(j, sx, sy, lane);
    }
}

template <bool FWD>
__device__ void consumer_loop(const DagWork &w, Ring ring, const AesTab &aes, int warp,
                              int lane)
{
    uint32_t it = 0;
    for (;;) {
        const uint8_t *st = ring_wait(ring, it);
        if (st == nullptr)
            return;
        const StageHdr &h = ring.hdr[it % kStages];
        const uint32_t mode = h.mode;
        if (mode == kModeEnd)
            return;
        // copied out before the stage is released
        const LevelJob j = h.job;
        const int tx = (int)h.x, sy = (int)h.y;
        if (mode == kModeBulk) {
            if (!run_bulk<FWD>(j, tx, sy, warp, lane, ring, it, st))
                return;
        } else {
            ring_release(ring, it++);
            if (mode == kModeCipher) {
                if (FWD)
                    strm::cipher_warp(j, tx, sy, warp, aes, lane, j.ll, j.ll, true); // in place
                else
                    strm::cipher_warp(j, tx, sy, warp, aes, lane, j.ll_in, j.out, false);
            } else if (mode == kModeGeneral) {
                run_general<FWD>(j, tx, sy, warp, lane);
            } // kModeSkip: nothing
        }
        // publish: each consumer warp counts itself once its stores are
        // visible (a segment is complete at strips x kConsumerWarps), also to
        // the bulk copies (async proxy) that consumers of this data use; jobs
        // that nothing in the launch reads skip it
        if (j.publish) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            __threadfence();
            __syncwarp();
            if (lane == 0)
                atomicAdd(w.done + j.done_off + sy, 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// kernel: persistent CTAs over a dependency-ordered queue of units
// ---------------------------------------------------------------------------
// dynamic shared memory: the stages, then AES tables, barriers, headers
constexpr size_t kSmemData = (size_t)kStages * kStageBytes;
constexpr size_t kSmemAes = kSmemData;
constexpr size_t kSmemBars = kSmemAes + (sizeof(AesTab) + 15) / 16 * 16;
constexpr size_t kSmemHdr = kSmemBars + 16 * (size_t)kStages;
constexpr size_t kSmemBytes = kSmemHdr + sizeof(StageHdr) * (size_t)kStages;

template <bool FWD>
__global__ void __launch_bounds__(kCtaThreads, FRAG_CTAS_PER_SM) dag_kernel(DagWork w)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *data = smem;
    AesTab &aes = *reinterpret_cast<AesTab *>(smem + kSmemAes);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kSmemBars);
    uint64_t *empty = full + kStages;
    StageHdr *hdr = reinterpret_cast<StageHdr *>(smem + kSmemHdr);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        // all of a thread's table loads in flight at once
        constexpr int kTabIters = (kAesWords + kCtaThreads - 1) / kCtaThreads;
        uint32_t tv[kTabIters];
#pragma unroll
        for (int k = 0; k < kTabIters; ++k) {
            const int i = (int)threadIdx.x + k * kCtaThreads;
            tv[k] = i < kAesWords ? __ldg(w.aes_tables + i) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kTabIters; ++k) {
            const int i = (int)threadIdx.x + k * kCtaThreads;
            if (i < kAesWords)
                (&aes.T[0][0])[i] = tv[k];
        }
    }
    for (int i = threadIdx.x; i < 44; i += blockDim.x)
        aes.rk[i] = w.round_keys[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + s)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(empty + s)),
                         "n"(kConsumerWarps)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const Ring ring{data, full, empty, hdr, w.err};
    if (warp == kConsumerWarps) {
        if (lane == 0)
            producer_loop<FWD>(w, ring);
    } else {
        consumer_loop<FWD>(w, ring, aes, warp, lane);
    }
}

static cudaError_t dag_attr(bool fwd)
{
    static std::atomic<uint64_t> done[2] = {{0}, {0}};
    const void *fn = fwd ? (const void *)dag_kernel<true> : (const void *)dag_kernel<false>;
    return smem_attr_once(fn, (int)kSmemBytes, done[fwd ? 1 : 0]);
}

cudaError_t launch_dag(bool fwd, const DagWork &w, uint32_t grid, cudaStream_t stream)
{
    cudaError_t e = dag_attr(fwd);
    if (e != cudaSuccess)
        return e;
    if (fwd)
        dag_kernel<true><<<grid, kCtaThreads, kSmemBytes, stream>>>(w);
    else
        dag_kernel<false><<<grid, kCtaThreads, kSmemBytes, stream>>>(w);
    return cudaGetLastError();
}

cudaError_t dag_occupancy(bool fwd, int *blocks_per_sm)
{
    cudaError_t e = dag_attr(fwd);
    if (e != cudaSuccess)
        return e;
    const void *fn = fwd ? (const void *)dag_kernel<true> : (const void *)dag_kernel<false>;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kCtaThreads, kSmemBytes);
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
