// fast_tiles.cuh -- tile bodies for buffers of up to three levels, built from
// a row pass and a packed-pair column pass (included by tile_kernels.cu).
//
// A CTA of 512 threads owns a 256 x 256 tile; its window adds 16 pixels of
// lifting halo on every side (288 x 288).  Per level:
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
// the transform produces from bytes (or from valid fragments) is far inside
// that range; window halo positions are lifted from bounded data as well.
//
// The inverse mirrors this: a column-inverse pass (undo Eq. 5.2, then
// Eq. 5.1, two columns per op, details read from HBM) writes the row-lifted
// rows, and a scalar row-inverse pass writes LL_{l-1} or the output bytes.
//
// Window positions outside the image or outside the dependency cone of the
// owned tile compute values that are never stored; the symmetric extension is
// applied exactly at the image borders (Eq. 5.1's x_ext).
#pragma once

namespace frag {
namespace fast {

constexpr int kT = 256;        // owned tile side (pixels)
constexpr int kH = 16;         // halo on every side
constexpr int kW = kT + 2 * kH; // window side at level 0: 288
__host__ __device__ constexpr int side(int l) { return kW >> l; } // 288, 144, 72, 36

constexpr uint32_t kB2 = 0x40004000u; // bias of both halves of a packed pair

// shared memory (words): region X holds R_l (row-lifted rows of level l:
// side(l-1) rows x side(l) words, low half then high half) and A2 / A3; A1
// (LL_1, side(1) rows x side(1)/2 words) has its own array
constexpr int kXWords = side(1) * side(0);                    // 41472 (= R_1)
constexpr int kA1Words = side(1) * side(1) / 2;               // 10368
constexpr int kA2Off = side(1) * side(2);                     // after R_2: 10368
constexpr int kA3Off = kA2Off + side(2) * side(2) / 2;        // 12960
static_assert(kA3Off + side(3) * side(3) / 2 <= kXWords, "A2/A3 must fit in region X");
static_assert(side(2) * side(3) <= kA2Off, "R_3 must not reach A2");

struct Smem {
    uint32_t x[kXWords];
    uint32_t a1[kA1Words];
};

__device__ __forceinline__ uint32_t *a_arr(Smem &sm, int l)
{
    return l == 1 ? sm.a1 : (l == 2 ? sm.x + kA2Off : sm.x + kA3Off);
}

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
    int wc0, wr0; // window origin = C0 - 16, R0 - 16 (multiples of 16, may be < 0)
    uint32_t L;   // levels of the buffer (band order)
};

__device__ __forceinline__ Geo make_geo(const Job &j, uint32_t tx, uint32_t ty)
{
    Geo g;
    g.W = (int)j.W;
    g.H = (int)j.H;
    g.C0 = (int)tx * kT;
    g.R0 = (int)ty * kT;
    g.wc0 = g.C0 - kH;
    g.wr0 = g.R0 - kH;
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

// Load N = 2 * NW int16 values of a band row (0 outside the band) as packed
// biased pairs.
template <int NW>
__device__ __forceinline__ void load_pairs(const uint8_t *band, int Hl, int Wl, int y, int x0,
                                           uint32_t (&w)[NW])
{
    if (y < 0 || y >= Hl) {
#pragma unroll
        for (int i = 0; i < NW; ++i)
            w[i] = kB2;
        return;
    }
    const uint8_t *src = band + 2ull * ((uint64_t)y * (uint64_t)Wl + (uint64_t)x0);
    const bool inside = x0 >= 0 && x0 + 2 * NW <= Wl;
    if (inside && NW == 4 && ((uintptr_t)src & 15u) == 0) {
        const uint4 t = __ldg(reinterpret_cast<const uint4 *>(src));
        const uint32_t a[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < NW; ++i)
            w[i] = from_i16x2(a[i]);
    } else if (inside && NW == 2 && ((uintptr_t)src & 7u) == 0) {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(src));
        const uint32_t a[2] = {t.x, t.y};
#pragma unroll
        for (int i = 0; i < NW; ++i)
            w[i] = from_i16x2(a[i]);
    } else {
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            uint32_t h[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int x = x0 + 2 * i + k;
                h[k] = (x >= 0 && x < Wl)
                           ? ((uint32_t)__ldg(src + 4 * i + 2 * k) |
                              ((uint32_t)__ldg(src + 4 * i + 2 * k + 1) << 8))
                           : 0u;
            }
            w[i] = from_i16x2(h[0] | (h[1] << 16));
        }
    }
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
__device__ void fwd_row_pass_bytes(const Job &j, const Geo &g, uint32_t *R)
{
    constexpr int CV = 16, CH = kW / CV; // 18 chunks per window row
    constexpr int RW = side(1);          // words per R_1 row (72 low + 72 high)
    const bool vec = ((j.W & 15u) == 0) && (((uintptr_t)j.in & 15u) == 0);
    for (int it = threadIdx.x; it < kW * CH; it += blockDim.x) {
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

// level-l row pass (l >= 2): A_{l-1} (packed, biased) -> R_l
template <int l>
__device__ void fwd_row_pass_packed(const Geo &g, const uint32_t *A, uint32_t *R)
{
    constexpr int CV = l == 2 ? 16 : 8;  // values per item
    constexpr int NW = CV / 2;           // input words per item
    constexpr int IN = side(l - 1);      // values per input row (= rows)
    constexpr int AW = IN / 2;           // words per input row
    constexpr int CH = IN / CV;          // 9
    constexpr int RW = side(l);          // words per R_l row
    const int wc = g.wc0 >> (l - 1), Wm = g.W >> (l - 1);
    for (int it = threadIdx.x; it < IN * CH; it += blockDim.x) {
        const int r = it / CH, k = it - r * CH;
        const uint32_t *arow = A + r * AW;
        const int w0 = k * NW;
        uint32_t m[NW];
#pragma unroll
        for (int i = 0; i < NW; i += 4) {
            if (NW - i >= 4) {
                const uint4 t = *reinterpret_cast<const uint4 *>(arow + w0 + i);
                m[i] = t.x;
                m[(i + 1) % NW] = t.y;
                m[(i + 2) % NW] = t.z;
                m[(i + 3) % NW] = t.w;
            }
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
// forward column pass (packed pairs)
// ---------------------------------------------------------------------------
template <int l>
__device__ void fwd_col_pass(const Geo &g, const uint32_t *R, uint32_t *A, uint8_t *pub)
{
    constexpr int CW = l == 3 ? 2 : 4;          // words per item
    constexpr int S = l == 1 ? 12 : (l == 2 ? 4 : 2);
    constexpr int RW = side(l);                 // words per R_l row
    constexpr int ROWS = side(l - 1);           // R_l rows
    constexpr int PAIRS = side(l);              // row pairs
    constexpr int CH = RW / CW;
    constexpr int SEGS = PAIRS / S;
    static_assert(PAIRS % S == 0 && RW % CW == 0, "partition");
    const int wr = g.wr0 >> (l - 1), Hm = g.H >> (l - 1);
    const int wcl = g.wc0 >> l, wrl = g.wr0 >> l;
    const int Wl = g.W >> l;
    const int ox0 = g.C0 >> l, ox1 = min(g.C0 + kT, g.W) >> l;
    const int oy0 = g.R0 >> l, oy1 = min(g.R0 + kT, g.H) >> l;
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
            const uint32_t *p = R + r * RW + w0;
            if (CW == 4) {
                const uint4 t = *reinterpret_cast<const uint4 *>(p);
                v[0] = t.x;
                v[1 % CW] = t.y;
                v[2 % CW] = t.z;
                v[3 % CW] = t.w;
            } else {
                const uint2 t = *reinterpret_cast<const uint2 *>(p);
                v[0] = t.x;
                v[1 % CW] = t.y;
            }
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
                uint32_t *dst = A + q * (RW / 2) + w0;
                if (CW == 4)
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(sv[0], sv[1 % CW], sv[2 % CW], sv[3 % CW]);
                else
                    *reinterpret_cast<uint2 *>(dst) = make_uint2(sv[0], sv[1 % CW]);
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
    constexpr int AW = side(L) / 2;
    const int WL = g.W >> L;
    const int X0 = g.C0 >> L, X1 = min(g.C0 + kT, g.W) >> L;
    const int Y0 = g.R0 >> L, Y1 = min(g.R0 + kT, g.H) >> L;
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

template <int L>
__device__ void fwd_tile_fast(const Job &j, uint32_t tx, uint32_t ty, Smem &sm, const AesSmem &aes)
{
    const Geo g = make_geo(j, tx, ty);
    fwd_row_pass_bytes(j, g, sm.x);
    __syncthreads();
    fwd_col_pass<1>(g, sm.x, sm.a1, j.pub);
    __syncthreads();
    if (L >= 2) {
        fwd_row_pass_packed<2>(g, sm.a1, sm.x);
        __syncthreads();
        fwd_col_pass<2>(g, sm.x, sm.x + kA2Off, j.pub);
        __syncthreads();
    }
    if (L >= 3) {
        fwd_row_pass_packed<3>(g, sm.x + kA2Off, sm.x);
        __syncthreads();
        fwd_col_pass<3>(g, sm.x, sm.x + kA3Off, j.pub);
        __syncthreads();
    }
    fwd_store_private<L>(j, g, a_arr(sm, L), aes);
}

// ---------------------------------------------------------------------------
// inverse
// ---------------------------------------------------------------------------

// Column inverse of level l: A_l + detail bands -> R_l (row-lifted rows).
template <int l>
__device__ void inv_col_pass(const Geo &g, const uint32_t *A, uint32_t *R, const uint8_t *pub)
{
    constexpr int CW = l == 3 ? 2 : 4;
    constexpr int S = l == 1 ? 12 : (l == 2 ? 4 : 2);
    constexpr int RW = side(l);
    constexpr int PAIRS = side(l);
    constexpr int CH = RW / CW;
    constexpr int SEGS = PAIRS / S;
    const int wrl = g.wr0 >> l, wcl = g.wc0 >> l;
    const int Hm = g.H >> (l - 1);
    const int Hl = g.H >> l, Wl = g.W >> l;
    const uint8_t *band_hl = pub + band_offset(g.H, g.W, g.L, l, 0);
    const uint8_t *band_lh = pub + band_offset(g.H, g.W, g.L, l, 1);
    const uint8_t *band_hh = pub + band_offset(g.H, g.W, g.L, l, 2);

    for (int it = threadIdx.x; it < CH * SEGS; it += blockDim.x) {
        const int c = it % CH, sy = it / CH;
        const int w0 = c * CW;
        const bool high = w0 >= RW / 2;
        const int wl = w0 - (high ? RW / 2 : 0); // word within the half
        const int x0 = wcl + 2 * wl;
        const int q0 = sy * S;
        // coefficients of row pair k: s (even row) and d (odd row)
        auto coeffs = [&](int k, uint32_t (&s)[CW], uint32_t (&d)[CW]) {
            const int y = wrl + k;
            if (!high) {
                const int kk = min(max(k, 0), PAIRS - 1);
                const uint32_t *p = A + kk * (RW / 2) + wl;
#pragma unroll
                for (int i = 0; i < CW; ++i)
                    s[i] = p[i];
                load_pairs<CW>(band_lh, Hl, Wl, y, x0, d);
            } else {
                load_pairs<CW>(band_hl, Hl, Wl, y, x0, s);
                load_pairs<CW>(band_hh, Hl, Wl, y, x0, d);
            }
        };
        uint32_t s0[CW], d0[CW], s1[CW], d1[CW], xe[CW], xe1[CW];
        coeffs(q0 - 1, s1, d1); // d[q0-1] in d1
        coeffs(q0, s0, d0);
        if (wrl + q0 == 0) { // d[-1] = d[0]
#pragma unroll
            for (int i = 0; i < CW; ++i)
                d1[i] = d0[i];
        }
#pragma unroll
        for (int i = 0; i < CW; ++i)
            xe[i] = s0[i] - pq4(d1[i], d0[i]) + 0x20002000u; // undo Eq. 5.2
        for (int q = q0; q < q0 + S; ++q) {
            coeffs(q + 1, s1, d1);
            const bool first = (wrl + q + 1 == 0);
#pragma unroll
            for (int i = 0; i < CW; ++i)
                xe1[i] = s1[i] - pq4(first ? d1[i] : d0[i], d1[i]) + 0x20002000u;
            const bool bottom = (2 * (wrl + q) + 2 == Hm); // x[m] = x[m-2]
            uint32_t xo[CW];
#pragma unroll
            for (int i = 0; i < CW; ++i)
                xo[i] = d0[i] + pavg(xe[i], bottom ? xe[i] : xe1[i]) - kB2; // undo Eq. 5.1
            uint32_t *re = R + (2 * q) * RW + w0;
            uint32_t *ro = re + RW;
            if (CW == 4) {
                *reinterpret_cast<uint4 *>(re) = make_uint4(xe[0], xe[1 % CW], xe[2 % CW], xe[3 % CW]);
                *reinterpret_cast<uint4 *>(ro) = make_uint4(xo[0], xo[1 % CW], xo[2 % CW], xo[3 % CW]);
            } else {
                *reinterpret_cast<uint2 *>(re) = make_uint2(xe[0], xe[1 % CW]);
                *reinterpret_cast<uint2 *>(ro) = make_uint2(xo[0], xo[1 % CW]);
            }
#pragma unroll
            for (int i = 0; i < CW; ++i) {
                xe[i] = xe1[i];
                d0[i] = d1[i];
            }
        }
    }
}

// Row inverse of level l: R_l -> A_{l-1} (l >= 2) or the output bytes (l = 1).
template <int l>
__device__ void inv_row_pass(const Job &j, const Geo &g, const uint32_t *R, uint32_t *Aout)
{
    constexpr int P = l == 3 ? 4 : 8;  // pairs per item
    constexpr int RW = side(l);        // words per R_l row
    constexpr int HW = RW / 2;         // words per half
    constexpr int ROWS = side(l - 1);
    constexpr int CH = side(l) / P;    // items per row
    const int wcl = g.wc0 >> l;
    const int Wm = g.W >> (l - 1);
    for (int it = threadIdx.x; it < ROWS * CH; it += blockDim.x) {
        const int r = it / CH, k = it - r * CH;
        const int p0 = k * P; // first pair (level-l window column)
        const uint32_t *row = R + r * RW;
        // low values L[p0 .. p0+P], high values H[p0-1 .. p0+P]
        int Lv[P + 2], Hv[P + 4];
        {
            const int lw = p0 / 2;
#pragma unroll
            for (int t = 0; t < P / 2; ++t) {
                const uint32_t w = row[lw + t];
                Lv[2 * t] = (int)(w & 0xffffu);
                Lv[2 * t + 1] = (int)(w >> 16);
                const uint32_t h = row[HW + lw + t];
                Hv[2 + 2 * t] = (int)(h & 0xffffu);
                Hv[3 + 2 * t] = (int)(h >> 16);
            }
            const uint32_t ln = row[min(lw + P / 2, HW - 1)];
            Lv[P] = (int)(ln & 0xffffu);
            Lv[P + 1] = (int)(ln >> 16);
            const uint32_t hp = row[HW + max(lw - 1, 0)];
            Hv[0] = (int)(hp & 0xffffu);
            Hv[1] = (int)(hp >> 16);
            const uint32_t hn = row[HW + min(lw + P / 2, HW - 1)];
            Hv[P + 2] = (int)(hn & 0xffffu);
            Hv[P + 3] = (int)(hn >> 16);
        }
        // Hv[1 + i] is H[p0 + i - 1]
        int ev[P + 1], out[2 * P];
#pragma unroll
        for (int i = 0; i <= P; ++i) {
            const int hl = (wcl + p0 + i == 0) ? Hv[2 + i] : Hv[1 + i]; // d[-1] = d[0]
            ev[i] = Lv[i] - ((hl + Hv[2 + i] + 2) >> 2) + 0x2000;     // undo Eq. 5.2 (biased)
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int xr = (2 * (wcl + p0 + i) + 2 == Wm) ? ev[i] : ev[i + 1]; // x[m] = x[m-2]
            out[2 * i] = ev[i];
            out[2 * i + 1] = Hv[2 + i] + ((ev[i] + xr) >> 1) - 0x4000; // undo Eq. 5.1 (biased)
        }
        if (l > 1) {
            uint32_t *dst = Aout + r * (ROWS / 2) + p0;
#pragma unroll
            for (int i = 0; i < P; ++i)
                dst[i] = pack2(out[2 * i], out[2 * i + 1]);
        } else {
            const int Rr = g.wr0 + r, C = g.wc0 + 2 * p0;
            if (Rr < g.R0 || Rr >= min(g.R0 + kT, g.H) || C < g.C0 || C >= g.C0 + kT || C >= g.W)
                continue;
            const uint64_t go = (uint64_t)Rr * (uint64_t)g.W + (uint64_t)C;
            uint8_t *dst = j.out + go;
            // biased values 0x4000 + b: the low byte is the recovered byte
            if (C + 2 * P <= g.W && go + 2 * P <= j.n && ((uintptr_t)dst & 15u) == 0) {
                uint32_t wv[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint32_t a = __byte_perm((uint32_t)out[4 * t], (uint32_t)out[4 * t + 1], 0x0040);
                    const uint32_t b = __byte_perm((uint32_t)out[4 * t + 2], (uint32_t)out[4 * t + 3], 0x0040);
                    wv[t] = __byte_perm(a, b, 0x5410);
                }
                *reinterpret_cast<uint4 *>(dst) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 2 * P; ++i)
                    if (C + i < g.W && go + i < j.n)
                        dst[i] = (uint8_t)out[i];
            }
        }
    }
}

// LL_L window from the private fragment: decrypt, add back 128, pack biased.
template <int L>
__device__ void inv_load_private(const Job &j, const Geo &g, uint32_t *A, const AesSmem &aes)
{
    constexpr int SD = side(L), AW = SD / 2;
    for (int i = threadIdx.x; i < SD * AW; i += blockDim.x)
        A[i] = kB2; // positions outside the image: value 0
    __syncthreads();
    const int WL = g.W >> L, HL = g.H >> L;
    const int wcL = g.wc0 >> L, wrL = g.wr0 >> L;
    const int xa = max(wcL, 0), xb = min(wcL + SD, WL);
    if (xb <= xa)
        return;
    const int bpr = (2 * (xb - xa) + 15) / 16 + 1;
    uint16_t *A16 = reinterpret_cast<uint16_t *>(A);
    for (int idx = threadIdx.x; idx < SD * bpr; idx += blockDim.x) {
        const int k = idx / bpr, jb = idx - k * bpr;
        const int y = wrL + k;
        if (y < 0 || y >= HL)
            continue;
        const uint64_t rowo = 2ull * (uint64_t)y * (uint64_t)WL;
        const uint64_t start = rowo + 2ull * xa, end = rowo + 2ull * xb;
        const uint64_t blk = start / 16 + (uint64_t)jb;
        if (blk * 16 >= end)
            continue;
        uint32_t ks[4];
        aes_ctr_block(aes, j.nonce, blk, ks);
#pragma unroll
        for (int kk = 0; kk < 16; kk += 2) {
            const uint64_t o = blk * 16 + kk;
            if (o < start || o >= end)
                continue;
            const uint32_t lo8 = __ldg(j.priv_in + o) ^ ks_byte(ks, kk);
            const uint32_t hi8 = __ldg(j.priv_in + o + 1) ^ ks_byte(ks, kk + 1);
            const int v = (int)(int16_t)(uint16_t)(lo8 | (hi8 << 8)) + 128 + 0x4000;
            const int x = (int)((o - rowo) / 2) - wcL;
            A16[k * SD + x] = (uint16_t)v;
        }
    }
}

template <int L>
__device__ void inv_tile_fast(const Job &j, uint32_t tx, uint32_t ty, Smem &sm, const AesSmem &aes)
{
    const Geo g = make_geo(j, tx, ty);
    inv_load_private<L>(j, g, a_arr(sm, L), aes);
    __syncthreads();
    if (L >= 3) {
        inv_col_pass<3>(g, sm.x + kA3Off, sm.x, j.pub_in);
        __syncthreads();
        inv_row_pass<3>(j, g, sm.x, sm.x + kA2Off);
        __syncthreads();
    }
    if (L >= 2) {
        inv_col_pass<2>(g, sm.x + kA2Off, sm.x, j.pub_in);
        __syncthreads();
        inv_row_pass<2>(j, g, sm.x, sm.a1);
        __syncthreads();
    }
    inv_col_pass<1>(g, sm.a1, sm.x, j.pub_in);
    __syncthreads();
    inv_row_pass<1>(j, g, sm.x, nullptr);
}

} // namespace fast
} // namespace frag
