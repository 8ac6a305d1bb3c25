// fast_tiles.cuh -- the forward tile body of the allocation-free protect, for
// buffers of 1 to 5 levels, built from a row pass and a packed-pair column
// pass per level (included by tile_kernels.cu).
//
// A CTA of 512 threads owns a T x T tile and lifts it inside a KW x KW window
// (T plus a halo before and after it in each direction) held in shared
// memory.  Per level:
//
//   row pass     every row of the level's input window is lifted once along
//                the row (Eq. 5.1 predict, Eq. 5.2 update; rows come first,
//                Sec. 5.2.2) by scalar code; the low-pass and high-pass
//                results go to shared memory as two halves of the row,
//                packed two columns per 32-bit word;
//   column pass  each work item streams down a strip of packed words and
//                lifts the columns two at a time with 32-bit integer ops;
//                detail bands go straight to HBM, LL_l stays in shared
//                memory as the next level's input.
//
// Packed pairs: each 16-bit half holds v + 0x4000 with |v| < 2^14.  Sums of
// two halves stay below 2^16, so floor((a + b) / 2) of both halves is
// ((A + B) >> 1) & 0x7fff7fff and floor((a + b + 2) / 4) is
// ((A + B + 0x00020002) >> 2) & 0x3fff3fff, each exact per half.  Every value
// the transform produces from bytes, at any of the five levels, is far inside
// that range (LL_l stays within a few times the byte range, details within a
// few times LL_{l-1}'s); window positions outside the image read zero bytes
// and are lifted from bounded data as well.
//
// Window positions outside the image or outside the dependency cone of the
// owned tile compute values that are never stored; the symmetric extension is
// applied exactly at the image borders (Eq. 5.1's x_ext).
#pragma once

namespace frag {
namespace fast {

// Window geometry of an L-level tile.  A level-l pair k (s at 2k, d at
// 2k + 1 of its input lattice) reads input samples 2k - 2 .. 2k + 2, so the
// level-L outputs of a tile depend on level-0 pixels from 2 (2^L - 1) before
// the tile to 2^L - 2 after it.  The window adds a leading halo kH of at
// least the first (a multiple of 2^L, so the window origin sits on every
// level's lattice) and a trailing halo kR of at least 2^L - 1, in both
// directions.  KW / 2^(L-1) is a multiple of 4 so that every level's rows
// split into whole packed words in two equal halves.
//   L = 1..3: 256-pixel tile, halos 16 / 16, 288-pixel window
//   L = 4:    240-pixel tile, halos 32 / 16, 288-pixel window
//   L = 5:    160-pixel tile, halos 64 / 32, 256-pixel window
template <int L>
struct Geom {
    static constexpr int kH = L <= 3 ? 16 : (L == 4 ? 32 : 64);
    static constexpr int kR = L <= 4 ? 16 : 32;
    static constexpr int kW = L <= 4 ? 288 : 256;
    static constexpr int kT = kW - kH - kR;
    __host__ __device__ static constexpr int side(int l) { return kW >> l; }
    // shared memory (words): region X holds R_l (row-lifted rows of level l:
    // side(l-1) rows x side(l) words, low half then high half) and A_2 ..
    // A_L; A_1 (LL_1, side(1) rows x side(1)/2 words) follows X
    static constexpr int kXWords = side(1) * side(0);
    static constexpr int kA1Words = side(1) * side(1) / 2;
    // A_l (l >= 2) sits after R_2, each LL band after the one before it
    __host__ __device__ static constexpr int a_off(int l)
    {
        return l <= 2 ? side(1) * side(2) : a_off(l - 1) + side(l - 1) * side(l - 1) / 2;
    }
    static constexpr int kWords = kXWords + kA1Words;
    static_assert(kH >= 2 * ((1 << L) - 1) && kH % (1 << L) == 0 && kR >= (1 << L) - 1 &&
                      kT % (1 << L) == 0, "halo");
    static_assert((kW >> (L - 1)) % 4 == 0, "whole packed words at every level");
    static_assert(a_off(L + 1) <= kXWords, "A_2 .. A_L must fit in region X");
    static_assert(side(2) * side(3) <= a_off(2), "R_3 must not reach A_2");
};

constexpr uint32_t kB2 = 0x40004000u; // bias of both halves of a packed pair

__device__ __forceinline__ uint32_t pack2(int lo, int hi)
{
    return __byte_perm((uint32_t)lo, (uint32_t)hi, 0x5410);
}

// floor((a + b) / 2) of both halves (biased in, biased out)
__device__ __forceinline__ uint32_t pavg(uint32_t a, uint32_t b)
{
    return ((a + b) >> 1) & 0x7fff7fffu;
}

// floor((a + b + 2) / 4) + 0x2000 of both halves (biased in)
__device__ __forceinline__ uint32_t pq4(uint32_t a, uint32_t b)
{
    return ((a + b + 0x00020002u) >> 2) & 0x3fff3fffu;
}

// packed pair (biased) -> two int16 little-endian values
__device__ __forceinline__ uint32_t to_i16x2(uint32_t w) { return (w + kB2) ^ 0x80008000u; }
// two int16 -> packed pair (biased)
__device__ __forceinline__ uint32_t from_i16x2(uint32_t w) { return (w ^ 0x80008000u) - kB2; }

struct Geo {
    int W, H;     // level-0 image
    int C0, R0;   // owned tile origin
    int wc0, wr0; // window origin = C0 - kH, R0 - kH (multiples of 2^L, may be < 0)
    uint32_t L;   // levels of the buffer (band order)
};

template <int L>
__device__ __forceinline__ Geo make_geo(const Job &j, uint32_t tx, uint32_t ty)
{
    Geo g;
    g.W = (int)j.W;
    g.H = (int)j.H;
    g.C0 = (int)tx * Geom<L>::kT;
    g.R0 = (int)ty * Geom<L>::kT;
    g.wc0 = g.C0 - Geom<L>::kH;
    g.wr0 = g.R0 - Geom<L>::kH;
    g.L = j.L;
    return g;
}

// Store N int16 values (given as N/2 packed biased pairs) to dst, vectorised
// when the whole run is owned and aligned.
template <int NW>
__device__ __forceinline__ void store_pairs(uint8_t *band, int Wl, int y, int x0, int ox0, int ox1,
                                            const uint32_t (&w)[NW])
{
    uint8_t *dst = band + 2ull * ((uint64_t)y * (uint64_t)Wl + (uint64_t)x0);
    uint32_t v[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i)
        v[i] = to_i16x2(w[i]);
    const bool all = x0 >= ox0 && x0 + 2 * NW <= ox1;
    if (all && NW == 4 && ((uintptr_t)dst & 15u) == 0) {
        *reinterpret_cast<uint4 *>(dst) = make_uint4(v[0], v[1 % NW], v[2 % NW], v[3 % NW]);
    } else if (all && NW == 2 && ((uintptr_t)dst & 7u) == 0) {
        *reinterpret_cast<uint2 *>(dst) = make_uint2(v[0], v[1 % NW]);
    } else if (all && NW == 1 && ((uintptr_t)dst & 3u) == 0) {
        *reinterpret_cast<uint32_t *>(dst) = v[0];
    } else {
#pragma unroll
        for (int i = 0; i < 2 * NW; ++i) {
            const int x = x0 + i;
            if (x < ox0 || x >= ox1)
                continue;
            const uint32_t h = (v[i >> 1] >> (16 * (i & 1))) & 0xffffu;
            dst[2 * i] = (uint8_t)(h & 255u);
            dst[2 * i + 1] = (uint8_t)(h >> 8);
        }
    }
}

// up to 4 consecutive words of shared memory (n = 1, 2 or 4; p aligned to n words)
template <int N>
__device__ __forceinline__ void ld_words(const uint32_t *p, uint32_t (&v)[N])
{
    if (N == 4) {
        const uint4 t = *reinterpret_cast<const uint4 *>(p);
        v[0] = t.x;
        v[1 % N] = t.y;
        v[2 % N] = t.z;
        v[3 % N] = t.w;
    } else if (N == 2) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        v[0] = t.x;
        v[1 % N] = t.y;
    } else {
        v[0] = p[0];
    }
}

template <int N>
__device__ __forceinline__ void st_words(uint32_t *p, const uint32_t (&v)[N])
{
    if (N == 4)
        *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1 % N], v[2 % N], v[3 % N]);
    else if (N == 2)
        *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1 % N]);
    else
        p[0] = v[0];
}

// ---------------------------------------------------------------------------
// row passes (scalar): CV input values per item
// ---------------------------------------------------------------------------

// Lift one run: x[0..CV+2] are the samples at window columns c-2 .. c+CV,
// ic the image column of sample c (even).  Returns CV/2 s and d values.
template <int CV>
__device__ __forceinline__ void lift_run(const int (&x)[CV + 3], int ic, int Wm, int (&s)[CV / 2],
                                         int (&d)[CV / 2])
{
    int dm1 = x[1] - ((x[0] + x[2]) >> 1);
#pragma unroll
    for (int i = 0; i < CV / 2; ++i) {
        const int xr = (ic + 2 * i + 2 == Wm) ? x[2 * i + 2] : x[2 * i + 4]; // x[m] = x[m-2]
        d[i] = x[2 * i + 3] - ((x[2 * i + 2] + xr) >> 1);
    }
#pragma unroll
    for (int i = 0; i < CV / 2; ++i) {
        // the image's first column may fall anywhere in the run: d[-1] = d[0]
        const int dl = (ic + 2 * i == 0) ? d[i] : (i == 0 ? dm1 : d[i - 1]);
        s[i] = x[2 * i + 2] + ((dl + d[i] + 2) >> 2);
    }
}

// level-1 row pass: bytes from HBM -> R_1 (low words then high words per row)
template <int L>
__device__ void fwd_row_pass_bytes(const Job &j, const Geo &g, uint32_t *R)
{
    using G = Geom<L>;
    constexpr int CV = 16, CH = G::kW / CV; // chunks per window row
    constexpr int RW = G::side(1);          // words per R_1 row (half low, half high)
    static_assert(G::kW % CV == 0, "whole chunks");
    const bool vec = ((j.W & 15u) == 0) && (((uintptr_t)j.in & 15u) == 0);
    for (int it = threadIdx.x; it < G::kW * CH; it += blockDim.x) {
        const int r = it / CH, k = it - r * CH;
        const int Rr = g.wr0 + r, c = g.wc0 + CV * k;
        int x[CV + 3];
        if (Rr >= 0 && Rr < g.H) {
            const uint64_t base = (uint64_t)Rr * (uint64_t)g.W;
            if (vec && c >= 4 && c + CV + 4 <= g.W && base + (uint64_t)c + CV + 4 <= j.n) {
                const uint8_t *p = j.in + base + c;
                const uint4 m = __ldg(reinterpret_cast<const uint4 *>(p));
                const uint32_t lw = __ldg(reinterpret_cast<const uint32_t *>(p - 4));
                const uint32_t rw = __ldg(reinterpret_cast<const uint32_t *>(p + CV));
                x[0] = (int)((lw >> 16) & 255u);
                x[1] = (int)(lw >> 24);
                const uint32_t mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int t = 0; t < CV; ++t)
                    x[2 + t] = (int)((mm[t >> 2] >> (8 * (t & 3))) & 255u);
                x[CV + 2] = (int)(rw & 255u);
            } else {
#pragma unroll
                for (int t = 0; t < CV + 3; ++t) {
                    const int cc = c - 2 + t;
                    x[t] = (cc >= 0 && cc < g.W && base + (uint64_t)cc < j.n)
                               ? (int)__ldg(j.in + base + (uint64_t)cc)
                               : 0;
                }
            }
        } else {
#pragma unroll
            for (int t = 0; t < CV + 3; ++t)
                x[t] = 0;
        }
        int s[CV / 2], d[CV / 2];
        lift_run<CV>(x, c, g.W, s, d);
        uint32_t *row = R + r * RW;
        uint4 lo, hi;
        // unbiased values: pack as int16 pairs, then move to the biased form
        lo.x = from_i16x2(pack2(s[0], s[1]));
        lo.y = from_i16x2(pack2(s[2], s[3]));
        lo.z = from_i16x2(pack2(s[4], s[5]));
        lo.w = from_i16x2(pack2(s[6], s[7]));
        hi.x = from_i16x2(pack2(d[0], d[1]));
        hi.y = from_i16x2(pack2(d[2], d[3]));
        hi.z = from_i16x2(pack2(d[4], d[5]));
        hi.w = from_i16x2(pack2(d[6], d[7]));
        *reinterpret_cast<uint4 *>(row + 4 * k) = lo;
        *reinterpret_cast<uint4 *>(row + RW / 2 + 4 * k) = hi;
    }
}

// values per item of the level-l packed row pass over IN values a row: 16
// at level 2, else 8, or 4 when 8 does not divide the row
__host__ __device__ constexpr int row_cv(int IN, int l)
{
    return (l == 2 && IN % 16 == 0) ? 16 : (IN % 8 == 0 ? 8 : 4);
}

// level-l row pass (l >= 2): A_{l-1} (packed, biased) -> R_l
template <int L, int l>
__device__ void fwd_row_pass_packed(const Geo &g, const uint32_t *A, uint32_t *R)
{
    using G = Geom<L>;
    constexpr int IN = G::side(l - 1);   // values per input row (= rows)
    constexpr int CV = row_cv(IN, l);    // values per item
    constexpr int NW = CV / 2;           // input words per item
    constexpr int AW = IN / 2;           // words per input row
    constexpr int CH = IN / CV;          // items per row
    constexpr int RW = G::side(l);       // words per R_l row
    static_assert(IN % CV == 0 && AW % (NW < 4 ? NW : 4) == 0, "aligned whole items");
    const int wc = g.wc0 >> (l - 1), Wm = g.W >> (l - 1);
    for (int it = threadIdx.x; it < IN * CH; it += blockDim.x) {
        const int r = it / CH, k = it - r * CH;
        const uint32_t *arow = A + r * AW;
        const int w0 = k * NW;
        uint32_t m[NW];
#pragma unroll
        for (int i = 0; i < NW; i += (NW < 4 ? NW : 4)) {
            uint32_t t[NW < 4 ? NW : 4];
            ld_words<(NW < 4 ? NW : 4)>(arow + w0 + i, t);
#pragma unroll
            for (int q = 0; q < (NW < 4 ? NW : 4); ++q)
                m[i + q] = t[q];
        }
        const uint32_t lw = arow[max(w0 - 1, 0)];
        const uint32_t rw = arow[min(w0 + NW, AW - 1)];
        int x[CV + 3];
        x[0] = (int)(lw & 0xffffu);
        x[1] = (int)(lw >> 16);
#pragma unroll
        for (int t = 0; t < NW; ++t) {
            x[2 + 2 * t] = (int)(m[t] & 0xffffu);
            x[3 + 2 * t] = (int)(m[t] >> 16);
        }
        x[CV + 2] = (int)(rw & 0xffffu);
        int s[CV / 2], d[CV / 2];
        lift_run<CV>(x, wc + CV * k, Wm, s, d); // s stays biased, d comes out unbiased
        uint32_t *row = R + r * RW;
#pragma unroll
        for (int i = 0; i < CV / 4; ++i) {
            row[(CV / 4) * k + i] = pack2(s[2 * i], s[2 * i + 1]);
            row[RW / 2 + (CV / 4) * k + i] = from_i16x2(pack2(d[2 * i], d[2 * i + 1]));
        }
    }
}

// ---------------------------------------------------------------------------
// column pass (packed pairs)
// ---------------------------------------------------------------------------

// words per item of a column pass over rows of `half` words a half: 4, or 2
// or 1 where 4 does not divide the half (an item stays within one half)
__host__ __device__ constexpr int col_cw(int half) { return half % 4 == 0 ? 4 : (half % 2 == 0 ? 2 : 1); }
// row pairs per item: 12 at level 1 (8 where 12 does not divide the pairs),
// 4 at level 2, else 2
__host__ __device__ constexpr int col_pairs(int pairs, int l)
{
    return l == 1 ? (pairs % 12 == 0 ? 12 : 8) : (l == 2 ? 4 : 2);
}

template <int L, int l>
__device__ void fwd_col_pass(const Geo &g, const uint32_t *R, uint32_t *A, uint8_t *pub)
{
    using G = Geom<L>;
    constexpr int RW = G::side(l);              // words per R_l row
    constexpr int CW = col_cw(RW / 2);          // words per item
    constexpr int ROWS = G::side(l - 1);        // R_l rows
    constexpr int PAIRS = G::side(l);           // row pairs
    constexpr int S = col_pairs(PAIRS, l);
    constexpr int CH = RW / CW;
    constexpr int SEGS = PAIRS / S;
    static_assert(PAIRS % S == 0 && (RW / 2) % CW == 0, "partition");
    const int wr = g.wr0 >> (l - 1), Hm = g.H >> (l - 1);
    const int wcl = g.wc0 >> l, wrl = g.wr0 >> l;
    const int Wl = g.W >> l;
    const int ox0 = g.C0 >> l, ox1 = min(g.C0 + G::kT, g.W) >> l;
    const int oy0 = g.R0 >> l, oy1 = min(g.R0 + G::kT, g.H) >> l;
    uint8_t *band_hl = pub + band_offset(g.H, g.W, g.L, l, 0);
    uint8_t *band_lh = pub + band_offset(g.H, g.W, g.L, l, 1);
    uint8_t *band_hh = pub + band_offset(g.H, g.W, g.L, l, 2);

    for (int it = threadIdx.x; it < CH * SEGS; it += blockDim.x) {
        const int c = it % CH, sy = it / CH;
        const int w0 = c * CW;
        const bool high = w0 >= RW / 2;
        const int x0 = wcl + 2 * (w0 - (high ? RW / 2 : 0)); // level-l image column
        const int q0 = sy * S;
        auto rowv = [&](int r, uint32_t (&v)[CW]) {
            r = min(max(r, 0), ROWS - 1);
            ld_words<CW>(R + r * RW + w0, v);
        };
        uint32_t e0[CW], o[CW], e1[CW], dp[CW], dv[CW], sv[CW];
        rowv(2 * q0, e0);
        {
            uint32_t a[CW];
            rowv(2 * q0 - 2, a);
            rowv(2 * q0 - 1, o);
#pragma unroll
            for (int i = 0; i < CW; ++i)
                dp[i] = o[i] - pavg(a[i], e0[i]) + kB2;
        }
        for (int q = q0; q < q0 + S; ++q) {
            rowv(2 * q + 1, o);
            if (wr + 2 * q + 2 == Hm) { // x[m] = x[m-2]
#pragma unroll
                for (int i = 0; i < CW; ++i)
                    e1[i] = e0[i];
            } else {
                rowv(2 * q + 2, e1);
            }
#pragma unroll
            for (int i = 0; i < CW; ++i)
                dv[i] = o[i] - pavg(e0[i], e1[i]) + kB2; // Eq. 5.1
            if (wr + 2 * q == 0) {                       // d[-1] = d[0]
#pragma unroll
                for (int i = 0; i < CW; ++i)
                    dp[i] = dv[i];
            }
#pragma unroll
            for (int i = 0; i < CW; ++i)
                sv[i] = e0[i] + pq4(dp[i], dv[i]) - 0x20002000u; // Eq. 5.2
            const int y = wrl + q;
            const bool yown = y >= oy0 && y < oy1;
            if (!high) {
                st_words<CW>(A + q * (RW / 2) + w0, sv);
                if (yown)
                    store_pairs<CW>(band_lh, Wl, y, x0, ox0, ox1, dv);
            } else if (yown) {
                store_pairs<CW>(band_hl, Wl, y, x0, ox0, ox1, sv);
                store_pairs<CW>(band_hh, Wl, y, x0, ox0, ox1, dv);
            }
#pragma unroll
            for (int i = 0; i < CW; ++i) {
                e0[i] = e1[i];
                dp[i] = dv[i];
            }
        }
    }
}

// owned part of LL_L (packed in A) -> private fragment, AES-CTR
template <int L>
__device__ void fwd_store_private(const Job &j, const Geo &g, const uint32_t *A, const AesSmem &aes)
{
    using G = Geom<L>;
    constexpr int AW = G::side(L) / 2;
    const int WL = g.W >> L;
    const int X0 = g.C0 >> L, X1 = min(g.C0 + G::kT, g.W) >> L;
    const int Y0 = g.R0 >> L, Y1 = min(g.R0 + G::kT, g.H) >> L;
    const int wcL = g.wc0 >> L, wrL = g.wr0 >> L;
    const int bpr = (2 * (X1 - X0) + 15) / 16 + 1;
    const int rows = Y1 - Y0;
    for (int idx = threadIdx.x; idx < rows * bpr; idx += blockDim.x) {
        const int yy = idx / bpr, jb = idx - yy * bpr;
        const int y = Y0 + yy;
        const uint64_t rowo = 2ull * (uint64_t)y * (uint64_t)WL;
        const uint64_t start = rowo + 2ull * X0, end = rowo + 2ull * X1;
        const uint64_t blk = start / 16 + (uint64_t)jb;
        if (blk * 16 >= end)
            continue;
        uint32_t ks[4];
        aes_ctr_block(aes, j.nonce, blk, ks);
        uint8_t c[16];
        bool full = true;
#pragma unroll
        for (int k = 0; k < 16; k += 2) {
            const uint64_t o = blk * 16 + k;
            if (o < start || o >= end) {
                full = false;
                c[k] = c[k + 1] = 0;
                continue;
            }
            const int x = (int)((o - rowo) / 2) - wcL;
            const uint32_t w = A[(y - wrL) * AW + (x >> 1)];
            const int v = (int)((w >> (16 * (x & 1))) & 0xffffu) - 0x4000 - 128;
            c[k] = (uint8_t)(((uint32_t)v & 255u) ^ ks_byte(ks, k));
            c[k + 1] = (uint8_t)((((uint32_t)v >> 8) & 255u) ^ ks_byte(ks, k + 1));
        }
        uint8_t *dst = j.priv + blk * 16;
        if (full && ((uintptr_t)dst & 15u) == 0) {
            uint4 w;
            w.x = c[0] | (c[1] << 8) | (c[2] << 16) | ((uint32_t)c[3] << 24);
            w.y = c[4] | (c[5] << 8) | (c[6] << 16) | ((uint32_t)c[7] << 24);
            w.z = c[8] | (c[9] << 8) | (c[10] << 16) | ((uint32_t)c[11] << 24);
            w.w = c[12] | (c[13] << 8) | (c[14] << 16) | ((uint32_t)c[15] << 24);
            *reinterpret_cast<uint4 *>(dst) = w;
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const uint64_t o = blk * 16 + k;
                if (o >= start && o < end)
                    j.priv[o] = c[k];
            }
        }
    }
}

// levels l .. L: row pass from A_{l-1}, column pass into A_l
template <int L, int l>
__device__ __forceinline__ void fwd_levels(const Geo &g, uint32_t *S, uint8_t *pub)
{
    if constexpr (l <= L) {
        using G = Geom<L>;
        fwd_row_pass_packed<L, l>(g, l == 2 ? S + G::kXWords : S + G::a_off(l - 1), S);
        __syncthreads();
        fwd_col_pass<L, l>(g, S, S + G::a_off(l), pub);
        __syncthreads();
        fwd_levels<L, l + 1>(g, S, pub);
    }
}

// One owned tile of an L-level buffer: every level in the window in shared
// memory S (Geom<L>::kWords words), then the private fragment's share.
template <int L>
__device__ void fwd_tile(const Job &j, uint32_t tx, uint32_t ty, uint32_t *S, const AesSmem &aes)
{
    using G = Geom<L>;
    const Geo g = make_geo<L>(j, tx, ty);
    fwd_row_pass_bytes<L>(j, g, S);
    __syncthreads();
    fwd_col_pass<L, 1>(g, S, S + G::kXWords, j.pub);
    __syncthreads();
    fwd_levels<L, 2>(g, S, j.pub);
    fwd_store_private<L>(j, g, L == 1 ? S + G::kXWords : S + G::a_off(L), aes);
}

} // namespace fast
} // namespace frag
