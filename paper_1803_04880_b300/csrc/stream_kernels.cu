// stream_kernels.cu -- one LeGall 5/3 level per launch, streamed by warps.
//
// A launch runs level l of one or many buffers.  Its work units are
// (buffer, strip, segment): a warp takes a strip of 256 columns of the
// level-(l-1) image and a segment of rows, and streams down the rows:
//
//   forward  lane t loads 8 consecutive samples of a row, lifts the row
//            (Eq. 5.1 predict, then Eq. 5.2 update; rows before columns,
//            Sec. 5.2.2) with its neighbours' samples taken by warp shuffles,
//            and packs its 4 low and 4 high results two per 32-bit word; the
//            column lifting then runs on those packed pairs in registers,
//            two row pairs of state per lane.  HL_l / LH_l / HH_l go straight
//            to the public fragment, LL_l to a scratch array (packed pairs)
//            or, at the last level, through AES-128-CTR to the private
//            fragment.
//   inverse  the exact reverse: the column inverse (undo Eq. 5.2, then Eq. 5.1)
//            on packed pairs read from LL_l (scratch, or the decrypted
//            private fragment at the top level) and the detail bands, then
//            the row inverse with shuffles; the result is LL_{l-1} (scratch)
//            or the recovered bytes.
//
// Lanes 0 and 31 of a warp only supply neighbours: lanes 1..30 own the
// strip's 240 columns, so strips advance by 240 and no value ever needs a
// lane outside the warp.  Rows above a segment are re-lifted (two rows) to
// restart the column stream.  The symmetric extension (x[-1] = x[1],
// x[m] = x[m-2], hence d[-1] = d[0]) applies only at the image borders.
//
// Packed pairs: each 16-bit half holds v + 0x4000 (|v| < 2^14); the halves of
// (A + B) never carry into each other, so both floors of a lifting step take
// one add, one shift and one mask for two columns.
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

// Keystream bytes [o, o + 8) (o even), as two little-endian words.  The
// bytes come from the 32-byte stream block(o / 16) || block(o / 16 + 1).
__device__ __forceinline__ void keystream8(const AesTab &a, uint64_t nonce, uint64_t o,
                                           uint32_t &k0, uint32_t &k1)
{
    uint32_t ks[4], kb[4] = {0u, 0u, 0u, 0u};
    const uint64_t b0 = o >> 4;
    const int m = (int)(o & 15);
    aes_block(a, nonce, b0, ks);
    if (m > 8)
        aes_block(a, nonce, b0 + 1, kb);
    // little-endian words of the 32-byte stream
    const uint32_t w0 = __byte_perm(ks[0], 0, 0x0123), w1 = __byte_perm(ks[1], 0, 0x0123);
    const uint32_t w2 = __byte_perm(ks[2], 0, 0x0123), w3 = __byte_perm(ks[3], 0, 0x0123);
    const uint32_t w4 = __byte_perm(kb[0], 0, 0x0123), w5 = __byte_perm(kb[1], 0, 0x0123);
    const int wi = m >> 2, sh = 8 * (m & 3);
    const uint32_t p0 = wi == 0 ? w0 : (wi == 1 ? w1 : (wi == 2 ? w2 : w3));
    const uint32_t p1 = wi == 0 ? w1 : (wi == 1 ? w2 : (wi == 2 ? w3 : w4));
    const uint32_t p2 = wi == 0 ? w2 : (wi == 1 ? w3 : (wi == 2 ? w4 : w5));
    k0 = __funnelshift_r(p0, p1, sh);
    k1 = __funnelshift_r(p1, p2, sh);
}

namespace strm {

constexpr uint32_t kB2 = 0x40004000u;

__device__ __forceinline__ uint32_t pack2(int lo, int hi)
{
    return __byte_perm((uint32_t)lo, (uint32_t)hi, 0x5410);
}
__device__ __forceinline__ uint32_t pavg(uint32_t a, uint32_t b) { return ((a + b) >> 1) & 0x7fff7fffu; }
__device__ __forceinline__ uint32_t pq4(uint32_t a, uint32_t b)
{
    return ((a + b + 0x00020002u) >> 2) & 0x3fff3fffu;
}
__device__ __forceinline__ uint32_t to_i16x2(uint32_t w) { return (w + kB2) ^ 0x80008000u; }
__device__ __forceinline__ uint32_t from_i16x2(uint32_t w) { return (w ^ 0x80008000u) - kB2; }
__device__ __forceinline__ int lo16(uint32_t w) { return (int)(w & 0xffffu); }
__device__ __forceinline__ int hi16(uint32_t w) { return (int)(w >> 16); }

// ---------------------------------------------------------------------------
// raw row loads (issued ahead of use)
// ---------------------------------------------------------------------------
struct Raw {
    uint32_t w[4];
};

// 8 source samples of row r at columns c .. c+7 of the level-(l-1) image.
// Byte sources: samples past n (or outside the image) are 0; packed sources:
// outside the image they are the biased 0 (0x4000).
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

// Lift one row along its length (Eq. 5.1 then Eq. 5.2) for the lane's four
// pairs at image columns c .. c+7, on packed pairs: (x0, x2), (x1, x3),
// (x4, x6), (x5, x7) are formed with byte permutes, the neighbours x8 and
// d[-1] come from the adjacent lanes.  Returns P[0] = (s0, s1),
// P[1] = (s2, s3), P[2] = (d0, d1), P[3] = (d2, d3), all biased.
template <bool BYTES>
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
    if (edge) { // x[m] = x[m-2] for the pair that ends the row
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
    if (c == 0)
        dm0 = __byte_perm(d01, d01, 0x1010); // d[-1] = d[0]
    const uint32_t d12 = __byte_perm(d01, d23, 0x5432); // (d1, d2)
    P[0] = e01 + pq4(dm0, d01) - 0x20002000u; // Eq. 5.2
    P[1] = e23 + pq4(d12, d23) - 0x20002000u;
    P[2] = d01;
    P[3] = d23;
}

// store 4 int16 values (2 packed biased pairs) to a band at (y, x .. x+3)
__device__ __forceinline__ void store4(uint8_t *band, int Wl, int y, int x, uint32_t a, uint32_t b,
                                       int nval)
{
    uint8_t *dst = band + 2ull * ((uint64_t)y * (uint64_t)Wl + (uint64_t)x);
    const uint32_t u = to_i16x2(a), v = to_i16x2(b);
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
// forward unit: one strip x one segment of level l
// ---------------------------------------------------------------------------
template <bool BYTES, bool FINAL>
__device__ void fwd_unit(const LevelJob &j, int sx, int sy, const AesTab &aes, int lane)
{
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const int c = 240 * sx - 8 + 8 * lane;        // first column of this lane
    const int q0 = sy * (int)j.seg_pairs;
    const int q1 = min(q0 + (int)j.seg_pairs, Hs / 2);
    const bool edge = (240 * sx + 248 >= Ws);      // strip reaches the right border
    const bool vec = BYTES ? (((j.Ws & 7u) == 0) && (((uintptr_t)j.src & 7u) == 0))
                           : (((j.Ws & 7u) == 0) && (((uintptr_t)j.src & 15u) == 0));
    const int Wl = Ws / 2;
    const int x = c / 2;                            // level-l column of the lane's first value
    const bool own = lane >= 1 && lane <= 30 && x < Wl;
    const int nval = min(4, Wl - x);

    uint32_t e0[4], dp[4];
    {
        uint32_t a[4], o[4];
        const Raw r0 = load_row<BYTES>(j, 2 * q0, c, vec);
        const Raw rm2 = load_row<BYTES>(j, max(2 * q0 - 2, 0), c, vec);
        const Raw rm1 = load_row<BYTES>(j, max(2 * q0 - 1, 0), c, vec);
        lift_row<BYTES>(r0, c, Ws, edge, e0);
        lift_row<BYTES>(rm2, c, Ws, edge, a);
        lift_row<BYTES>(rm1, c, Ws, edge, o);
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
        lift_row<BYTES>(c1, c, Ws, edge, o);
        if (2 * q + 2 == Hs) { // x[m] = x[m-2] at the bottom border
#pragma unroll
            for (int i = 0; i < 4; ++i)
                e1[i] = e0[i];
        } else {
            lift_row<BYTES>(c2, c, Ws, edge, e1);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            dv[i] = o[i] - pavg(e0[i], e1[i]) + kB2; // Eq. 5.1 down the columns
        if (q == 0) {                                // d[-1] = d[0] at the top border
#pragma unroll
            for (int i = 0; i < 4; ++i)
                dp[i] = dv[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            sv[i] = e0[i] + pq4(dp[i], dv[i]) - 0x20002000u; // Eq. 5.2 down the columns
        if (own) {
            // sv[0..1] = LL, sv[2..3] = HL, dv[0..1] = LH, dv[2..3] = HH
            store4(j.hl, Wl, q, x, sv[2], sv[3], nval);
            store4(j.lh, Wl, q, x, dv[0], dv[1], nval);
            store4(j.hh, Wl, q, x, dv[2], dv[3], nval);
            if (!FINAL) {
                uint32_t *ll = reinterpret_cast<uint32_t *>(j.ll) + (uint64_t)q * (uint64_t)(Wl / 2) + x / 2;
                if (nval == 4 && ((uintptr_t)ll & 7u) == 0) {
                    *reinterpret_cast<uint2 *>(ll) = make_uint2(sv[0], sv[1]);
                } else {
                    ll[0] = sv[0];
                    if (nval > 2)
                        ll[1] = sv[1];
                }
            }
        }
        if (FINAL) {
            // private fragment: LL - 128 as int16 LE, XOR AES-CTR keystream
            const uint64_t o8 = 2ull * ((uint64_t)q * (uint64_t)Wl + (uint64_t)x);
            uint32_t k0 = 0, k1 = 0;
            if (own)
                keystream8(aes, j.nonce, o8, k0, k1);
            if (own) {
                const uint32_t u = to_i16x2(sv[0] - 0x00800080u) ^ k0;
                const uint32_t v = to_i16x2(sv[1] - 0x00800080u) ^ k1;
                uint8_t *dst = j.ll + o8;
                if (nval == 4 && ((uintptr_t)dst & 7u) == 0) {
                    *reinterpret_cast<uint2 *>(dst) = make_uint2(u, v);
                } else {
                    const uint32_t bytes[2] = {u, v};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < 2 * nval)
                            dst[i] = (uint8_t)(bytes[i >> 2] >> (8 * (i & 3)));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            e0[i] = e1[i];
            dp[i] = dv[i];
        }
    }
}

// ---------------------------------------------------------------------------
// inverse unit
// ---------------------------------------------------------------------------
struct Coef {
    uint32_t sl[2], dl[2], sh[2], dh[2]; // low s (LL), low d (LH), high s (HL), high d (HH)
};

__device__ __forceinline__ void load4(const uint8_t *band, int Hl, int Wl, int y, int x, bool vec,
                                      uint32_t &a, uint32_t &b)
{
    if (y >= Hl || x < 0 || x >= Wl) {
        a = b = kB2;
        return;
    }
    const uint8_t *p = band + 2ull * ((uint64_t)y * (uint64_t)Wl + (uint64_t)x);
    if (vec && x + 4 <= Wl && ((uintptr_t)p & 7u) == 0) {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
        a = from_i16x2(t.x);
        b = from_i16x2(t.y);
    } else {
        uint32_t h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            h[i] = (x + i < Wl) ? ((uint32_t)__ldg(p + 2 * i) | ((uint32_t)__ldg(p + 2 * i + 1) << 8))
                                : 0u;
        a = from_i16x2(h[0] | (h[1] << 16));
        b = from_i16x2(h[2] | (h[3] << 16));
    }
}

template <bool TOP>
__device__ __forceinline__ Coef load_coef(const LevelJob &j, int k, int x, bool vec, const AesTab &aes)
{
    const int Hl = (int)j.Hs / 2, Wl = (int)j.Ws / 2;
    Coef cf;
    load4(j.lh, Hl, Wl, k, x, vec, cf.dl[0], cf.dl[1]);
    load4(j.hl, Hl, Wl, k, x, vec, cf.sh[0], cf.sh[1]);
    load4(j.hh, Hl, Wl, k, x, vec, cf.dh[0], cf.dh[1]);
    if (TOP) {
        // decrypt LL_L from the private fragment, add back 128
        cf.sl[0] = cf.sl[1] = kB2;
        if (k < Hl && x >= 0 && x < Wl) {
            const uint64_t o8 = 2ull * ((uint64_t)k * (uint64_t)Wl + (uint64_t)x);
            uint32_t k0, k1;
            keystream8(aes, j.nonce, o8, k0, k1);
            const uint8_t *p = j.ll_in + o8;
            uint32_t c0, c1;
            if (vec && x + 4 <= Wl && ((uintptr_t)p & 7u) == 0) {
                const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
                c0 = t.x;
                c1 = t.y;
            } else {
                uint32_t b[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    b[i] = (x + (i >> 1) < Wl) ? (uint32_t)__ldg(p + i) : 0u;
                c0 = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
                c1 = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
            }
            cf.sl[0] = from_i16x2(c0 ^ k0) + 0x00800080u;
            cf.sl[1] = from_i16x2(c1 ^ k1) + 0x00800080u;
        }
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

// Row inverse of one row on packed pairs: w[0] = (L0, L1), w[1] = (L2, L3),
// w[2] = (H0, H1), w[3] = (H2, H3); returns the 8 samples of image columns
// c .. c+7 as packed pairs (x0, x1), (x2, x3), (x4, x5), (x6, x7).
__device__ __forceinline__ void unlift_row(const uint32_t (&w)[4], int c, int Ws, bool edge,
                                           uint32_t (&out)[4])
{
    const uint32_t h23p = __shfl_up_sync(0xffffffffu, w[3], 1);
    uint32_t hm0 = __byte_perm(h23p, w[2], 0x5432); // (H[-1], H0)
    if (c == 0)
        hm0 = __byte_perm(w[2], w[2], 0x1010); // d[-1] = d[0]
    const uint32_t h12 = __byte_perm(w[2], w[3], 0x5432);
    const uint32_t e01 = w[0] - pq4(hm0, w[2]) + 0x20002000u; // undo Eq. 5.2
    const uint32_t e23 = w[1] - pq4(h12, w[3]) + 0x20002000u;
    const uint32_t e01n = __shfl_down_sync(0xffffffffu, e01, 1);
    uint32_t e12 = __byte_perm(e01, e23, 0x5432);
    uint32_t e34 = __byte_perm(e23, e01n, 0x5432);
    if (edge) { // x[m] = x[m-2]
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

template <bool TOP, bool BYTES_OUT>
__device__ void inv_unit(const LevelJob &j, int sx, int sy, const AesTab &aes, int lane)
{
    const int Ws = (int)j.Ws, Hs = (int)j.Hs;
    const int c = 240 * sx - 8 + 8 * lane; // first output column of this lane
    const int x = c >> 1;                  // first coefficient column
    const int k0 = sy * (int)j.seg_pairs;
    const int k1 = min(k0 + (int)j.seg_pairs, Hs / 2);
    const bool edge = (240 * sx + 248 >= Ws);
    const bool vec = ((j.Ws & 7u) == 0);
    const bool own = lane >= 1 && lane <= 30 && c < Ws;
    const int nv = min(8, Ws - c);

    Coef cur = load_coef<TOP>(j, k0, x, vec, aes);
    uint32_t xe[4], d0[4];
    {
        const Coef prev = load_coef<TOP>(j, max(k0 - 1, 0), x, vec, aes);
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
    }
    Coef nxt = load_coef<TOP>(j, k0 + 1, x, vec, aes);
    for (int k = k0; k < k1; ++k) {
        const Coef c1 = nxt;
        if (k + 1 < k1)
            nxt = load_coef<TOP>(j, k + 2, x, vec, aes);
        const uint32_t s1[4] = {c1.sl[0], c1.sl[1], c1.sh[0], c1.sh[1]};
        const uint32_t d1[4] = {c1.dl[0], c1.dl[1], c1.dh[0], c1.dh[1]};
        uint32_t xe1[4], xo[4];
        const bool bottom = (2 * k + 2 == Hs); // x[m] = x[m-2]
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xe1[i] = s1[i] - pq4(d0[i], d1[i]) + 0x20002000u;
            xo[i] = d0[i] + pavg(xe[i], bottom ? xe[i] : xe1[i]) - kB2; // undo Eq. 5.1
        }
        uint32_t ve[4], vo[4];
        unlift_row(xe, c, Ws, edge, ve);
        unlift_row(xo, c, Ws, edge, vo);
        store_row<BYTES_OUT>(j, 2 * k, c, own, nv, ve);
        store_row<BYTES_OUT>(j, 2 * k + 1, c, own, nv, vo);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xe[i] = xe1[i];
            d0[i] = d1[i];
        }
    }
}

} // namespace strm

// ---------------------------------------------------------------------------
// kernel: persistent warps over a dependency-ordered queue of units
// ---------------------------------------------------------------------------
// All levels of all buffers of a call run in one launch.  The queue lists
// units so that every unit's producers come before it; a unit whose input is
// another level's LL waits (lane 0, bounded spin) until the producer row
// segments it reads are complete, so the coarse levels stream right behind
// the fine ones.  A wait that runs out sets the error word to 3
// (FRAG_ETIMEOUT) and the unit is skipped but still reported complete, so no
// consumer can wait forever.
constexpr int kStreamThreads = 256;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// lane 0: wait until done[lo .. hi] all reach `target`
__device__ __forceinline__ bool wait_segments(const unsigned *done, uint32_t lo, uint32_t hi,
                                              unsigned target, uint32_t spin_limit, int *err)
{
    for (uint32_t s = lo; s <= hi; ++s) {
        uint32_t it = 0;
        while (ld_acquire(done + s) < target) {
            if (++it > spin_limit) {
                atomicCAS(err, 0, 3);
                return false;
            }
            __nanosleep(100);
        }
    }
    return true;
}

__device__ __forceinline__ const LevelJob &dag_job(const DagWork &w, uint32_t i)
{
    return w.n_inline ? w.inline_jobs[i] : w.jobs[i];
}

// Implicit order for one buffer: job m (m-th level in processing order) runs
// its segment sy in round sy + m * lag; rounds are listed in order, levels in
// order within a round, strips within a level.  All jobs have the same
// segment count.
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

// true if the unit may run (its producers are complete)
template <bool FWD>
__device__ __forceinline__ bool wait_producers(const DagWork &w, const LevelJob &j, int sy, int lane)
{
    int ok = 1;
    if (j.dep >= 0) {
        if (lane == 0) {
            const LevelJob &p = dag_job(w, (uint32_t)j.dep);
            int rlo, rhi; // producer segments covering the LL rows this unit reads
            if (FWD) {
                const int q0 = sy * (int)j.seg_pairs;
                const int q1 = min(q0 + (int)j.seg_pairs, (int)j.Hs / 2);
                rlo = max(2 * q0 - 2, 0) / (int)p.seg_pairs;
                rhi = min(2 * q1, (int)j.Hs - 1) / (int)p.seg_pairs;
            } else {
                const int k0 = sy * (int)j.seg_pairs;
                const int k1 = min(k0 + (int)j.seg_pairs, (int)j.Hs / 2);
                const int Hl = (int)j.Hs / 2;
                rlo = (max(k0 - 1, 0) / 2) / (int)p.seg_pairs;
                rhi = (min(k1 + 1, Hl - 1) / 2) / (int)p.seg_pairs;
            }
            ok = wait_segments(w.done + p.done_off, (uint32_t)rlo, (uint32_t)rhi, p.strips,
                               w.spin_limit, w.err)
                     ? 1
                     : 0;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
    }
    return ok != 0;
}

template <bool FWD>
__global__ void __launch_bounds__(kStreamThreads, 2) dag_kernel(DagWork w)
{
    __shared__ AesTab aes;
    for (int i = threadIdx.x; i < kAesWords; i += blockDim.x)
        (&aes.T[0][0])[i] = w.aes_tables[i];
    for (int i = threadIdx.x; i < 44; i += blockDim.x)
        aes.rk[i] = w.round_keys[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
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
        if (wait_producers<FWD>(w, j, sy, lane)) {
            if (FWD) {
                if (j.src_bytes) {
                    if (j.final_level)
                        strm::fwd_unit<true, true>(j, sx, sy, aes, lane);
                    else
                        strm::fwd_unit<true, false>(j, sx, sy, aes, lane);
                } else {
                    if (j.final_level)
                        strm::fwd_unit<false, true>(j, sx, sy, aes, lane);
                    else
                        strm::fwd_unit<false, false>(j, sx, sy, aes, lane);
                }
            } else {
                if (j.top_level) {
                    if (j.out_bytes)
                        strm::inv_unit<true, true>(j, sx, sy, aes, lane);
                    else
                        strm::inv_unit<true, false>(j, sx, sy, aes, lane);
                } else {
                    if (j.out_bytes)
                        strm::inv_unit<false, true>(j, sx, sy, aes, lane);
                    else
                        strm::inv_unit<false, false>(j, sx, sy, aes, lane);
                }
            }
        }
        // publish: every lane's stores before the count
        __threadfence();
        __syncwarp();
        if (lane == 0)
            atomicAdd(w.done + j.done_off + sy, 1u);
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
