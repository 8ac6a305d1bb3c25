// fast_tiles.cuh -- register-streaming tile bodies for buffers of up to three
// levels (included by tile_kernels.cu).
//
// Forward: a CTA stages a 248 x 248 byte window (the 224 x 224 owned tile
// plus 16 pixels of lifting halo above / left and 8 below / right) in shared
// memory.  For each level, each of 248 work items owns G column pairs and S
// row pairs of that level's input window: it lifts every row it needs on the
// fly (Eq. 5.1 then Eq. 5.2 along the row, rows before columns as in
// Sec. 5.2.2) and streams the column lifting down its rows in registers.
// Detail coefficients of owned positions go straight from registers to HBM;
// only the compact LL_l goes back to shared memory as the next level's input.
//
// Inverse: the mirror image.  A CTA owns a 224 x 224 output tile with a
// 16-pixel halo on each side (256 x 256 window).  For each level from the
// coarsest down, each of 256 work items streams the column inverse (undo
// Eq. 5.2, then Eq. 5.1) down G + 1 low and G + 2 high columns, reading LL_l
// from shared memory and the detail bands from HBM, then undoes the row
// lifting of the two rows it just produced in registers and writes LL_{l-1}
// (shared memory) or the recovered bytes (HBM).
//
// Window positions outside the image hold garbage that is never part of the
// dependency cone of an owned output; the symmetric extension is applied
// exactly at the image borders.  Every shared-memory array is padded so that
// neighbour reads at the window edge stay inside it.
#pragma once

namespace frag {
namespace fast {

constexpr int kT = 224;                // owned tile side (pixels), multiple of 32
constexpr int kFH = 16;                // forward halo above / left
constexpr int kFW = kT + kFH + 8;      // forward window side: 248
constexpr int kBP = 256;               // byte window pitch
constexpr int kIH = 16;                // inverse halo on every side
constexpr int kIW = kT + 2 * kIH;      // inverse window side: 256
constexpr int kItemsF = 31 * 8;        // forward work items per level
constexpr int kItemsI = 32 * 8;        // inverse work items per level

// padded compact int16 arrays: pitch = side + 4, element (r, c) at
// [(r + 1) * pitch + c + 2], one spare row above and below
__host__ __device__ constexpr int pitch_of(int side) { return side + 4; }
__host__ __device__ constexpr int words_of(int side) { return pitch_of(side) * (side + 2); }

struct FwdSmem {
    uint8_t front[16];               // absorbs the (garbage) reads left of column 0
    uint8_t bytes[(kFW + 1) * kBP];  // the byte window (+1 spare row)
    int16_t a1[words_of(kFW / 2)];
    int16_t a2[words_of(kFW / 4)];
    int16_t a3[words_of(kFW / 8)];
};

struct InvSmem {
    int16_t a0[words_of(kIW / 2)]; // LL_1 window (reconstructed from level 2)
    int16_t a1[words_of(kIW / 4)]; // LL_2 window
    int16_t a2[words_of(kIW / 8)]; // LL_3 window (decrypted private fragment)
};

template <typename T> __device__ __forceinline__ int ld_val(const T *p, int i) { return (int)p[i]; }

__device__ __forceinline__ int16_t *cell(int16_t *a, int side, int r, int c)
{
    return a + (r + 1) * pitch_of(side) + c + 2;
}

// store G int16 values at dst (any alignment), vectorised when aligned
template <int G> __device__ __forceinline__ void store_i16(uint8_t *dst, const int (&v)[G])
{
    const uintptr_t a = (uintptr_t)dst;
    if (G == 4 && (a & 7) == 0) {
        uint2 w;
        w.x = ((uint32_t)v[0] & 0xffffu) | ((uint32_t)v[1] << 16);
        w.y = ((uint32_t)v[2 % G] & 0xffffu) | ((uint32_t)v[3 % G] << 16);
        *reinterpret_cast<uint2 *>(dst) = w;
    } else if (G == 2 && (a & 3) == 0) {
        *reinterpret_cast<uint32_t *>(dst) = ((uint32_t)v[0] & 0xffffu) | ((uint32_t)v[1 % G] << 16);
    } else if (G == 1 && (a & 1) == 0) {
        *reinterpret_cast<int16_t *>(dst) = (int16_t)v[0];
    } else {
#pragma unroll
        for (int i = 0; i < G; ++i) {
            dst[2 * i] = (uint8_t)(v[i] & 255);
            dst[2 * i + 1] = (uint8_t)((v[i] >> 8) & 255);
        }
    }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

// Row lifting of G pairs starting at pair p0 of one window row (Eq. 5.1, 5.2).
// ic = image column of the row's sample 2 * p0; Wm = image row length.
template <int G, typename T>
__device__ __forceinline__ void row_lift(const T *row, int p0, int ic, int Wm, int (&s)[G],
                                         int (&d)[G])
{
    int x[2 * G + 3];
#pragma unroll
    for (int t = 0; t < 2 * G + 3; ++t)
        x[t] = ld_val(row, 2 * p0 - 2 + t);
    int dm1 = x[1] - ((x[0] + x[2]) >> 1);
#pragma unroll
    for (int i = 0; i < G; ++i) {
        const int xr = (ic + 2 * i + 2 == Wm) ? x[2 * i + 2] : x[2 * i + 4]; // x[m] = x[m-2]
        d[i] = x[2 * i + 3] - ((x[2 * i + 2] + xr) >> 1);
    }
    if (ic == 0)
        dm1 = d[0]; // d[-1] = d[0]
#pragma unroll
    for (int i = 0; i < G; ++i)
        s[i] = x[2 * i + 2] + (((i == 0 ? dm1 : d[i - 1]) + d[i] + 2) >> 2);
}

struct FwdGeo {
    int W, H;        // level-0 image
    int C0, R0;      // owned tile origin (level 0)
    int wc0, wr0;    // window origin (level 0), multiples of 16, may be negative
    uint8_t *pub;
    uint32_t L;      // total levels of the buffer (band order)
};

// One forward level l (1..3) over the window.  `in` is the level-(l-1)
// window (bytes at l = 1), `out` the compact LL_l window.
template <int l, typename T>
__device__ void fwd_level(const T *in, int in_pitch, int16_t *out, const FwdGeo &g)
{
    constexpr int G = 4 >> (l - 1);
    constexpr int S = 16 >> (l - 1);
    constexpr int EIN = kFW >> (l - 1); // input window side
    constexpr int PAIRS = EIN / 2;      // = output window side
    constexpr int GROUPS = PAIRS / G;   // 31
    constexpr int SEGS = (PAIRS + S - 1) / S;
    const int wc = g.wc0 >> (l - 1), wr = g.wr0 >> (l - 1); // level l-1 window origin
    const int Wm = g.W >> (l - 1), Hm = g.H >> (l - 1);
    const int Wl = g.W >> l;
    const int ox0 = g.C0 >> l, ox1 = min(g.C0 + kT, g.W) >> l;
    const int oy0 = g.R0 >> l, oy1 = min(g.R0 + kT, g.H) >> l;
    uint8_t *band_hl = g.pub + band_offset(g.H, g.W, g.L, l, 0);
    uint8_t *band_lh = g.pub + band_offset(g.H, g.W, g.L, l, 1);
    uint8_t *band_hh = g.pub + band_offset(g.H, g.W, g.L, l, 2);

    for (int it = threadIdx.x; it < GROUPS * SEGS; it += blockDim.x) {
        const int gx = it % GROUPS, sy = it / GROUPS;
        const int p0 = gx * G, q0 = sy * S, q1 = min(q0 + S, PAIRS);
        const int ic = wc + 2 * p0;
        auto lift = [&](int row, int (&s)[G], int (&d)[G]) {
            row = min(max(row, 0), EIN - 1);
            row_lift<G>(in + row * in_pitch, p0, ic, Wm, s, d);
        };
        int e0s[G], e0d[G], os[G], od[G], e1s[G], e1d[G], dps[G], dpd[G];
        lift(2 * q0, e0s, e0d);
        {
            int as[G], ad[G], bs[G], bd[G];
            lift(2 * q0 - 2, as, ad);
            lift(2 * q0 - 1, bs, bd);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                dps[i] = bs[i] - ((as[i] + e0s[i]) >> 1);
                dpd[i] = bd[i] - ((ad[i] + e0d[i]) >> 1);
            }
        }
        const int x0 = (wc >> 1) + p0; // level-l image column of pair p0
        const bool cols_owned = x0 >= ox0 && x0 + G <= ox1;
        for (int q = q0; q < q1; ++q) {
            lift(2 * q + 1, os, od);
            if (wr + 2 * q + 2 == Hm) { // x[m] = x[m-2] at the bottom border
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    e1s[i] = e0s[i];
                    e1d[i] = e0d[i];
                }
            } else {
                lift(2 * q + 2, e1s, e1d);
            }
            int dvs[G], dvd[G], svs[G], svd[G];
#pragma unroll
            for (int i = 0; i < G; ++i) {
                dvs[i] = os[i] - ((e0s[i] + e1s[i]) >> 1);
                dvd[i] = od[i] - ((e0d[i] + e1d[i]) >> 1);
            }
            if (wr + 2 * q == 0) { // d[-1] = d[0] at the top border
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    dps[i] = dvs[i];
                    dpd[i] = dvd[i];
                }
            }
#pragma unroll
            for (int i = 0; i < G; ++i) {
                svs[i] = e0s[i] + ((dps[i] + dvs[i] + 2) >> 2);
                svd[i] = e0d[i] + ((dpd[i] + dvd[i] + 2) >> 2);
            }
            // LL_l into the next level's window
            int16_t *o = cell(out, PAIRS, q, p0);
#pragma unroll
            for (int i = 0; i < G; ++i)
                o[i] = (int16_t)svs[i];
            // HL_l (low rows, high cols), LH_l (high rows, low cols), HH_l
            const int y = (wr >> 1) + q;
            if (y >= oy0 && y < oy1) {
                const uint64_t off = 2ull * ((uint64_t)y * (uint64_t)Wl + (uint64_t)x0);
                if (cols_owned) {
                    store_i16<G>(band_hl + off, svd);
                    store_i16<G>(band_lh + off, dvs);
                    store_i16<G>(band_hh + off, dvd);
                } else {
#pragma unroll
                    for (int i = 0; i < G; ++i) {
                        if (x0 + i < ox0 || x0 + i >= ox1)
                            continue;
                        const int a[1] = {svd[i]}, b[1] = {dvs[i]}, c[1] = {dvd[i]};
                        store_i16<1>(band_hl + off + 2 * i, a);
                        store_i16<1>(band_lh + off + 2 * i, b);
                        store_i16<1>(band_hh + off + 2 * i, c);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < G; ++i) {
                e0s[i] = e1s[i];
                e0d[i] = e1d[i];
                dps[i] = dvs[i];
                dpd[i] = dvd[i];
            }
        }
    }
}

// Load the byte window: rows wr0 .. wr0 + kFW - 1, columns wc0 .. wc0 + 255.
// Bytes past n (and outside the image) read as 0.
__device__ __forceinline__ void fwd_load(const Job &j, const FwdGeo &g, FwdSmem &sm)
{
    const bool vec = ((j.W & 15u) == 0) && (((uintptr_t)j.in & 15u) == 0);
    constexpr int CH = kBP / 16;
    for (int idx = threadIdx.x; idx < kFW * CH; idx += blockDim.x) {
        const int r = idx / CH, k = idx - r * CH;
        const int R = g.wr0 + r, c = g.wc0 + 16 * k;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (R >= 0 && R < g.H && c < g.W && c + 16 > 0) {
            const uint64_t base = (uint64_t)R * (uint64_t)g.W;
            if (vec && c >= 0 && c + 16 <= g.W && base + (uint64_t)c + 16 <= j.n) {
                v = __ldg(reinterpret_cast<const uint4 *>(j.in + base + c));
            } else {
                uint8_t b[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int cc = c + t;
                    b[t] = (cc >= 0 && cc < g.W && base + (uint64_t)cc < j.n)
                               ? __ldg(j.in + base + (uint64_t)cc)
                               : 0;
                }
                v.x = b[0] | (b[1] << 8) | (b[2] << 16) | ((uint32_t)b[3] << 24);
                v.y = b[4] | (b[5] << 8) | (b[6] << 16) | ((uint32_t)b[7] << 24);
                v.z = b[8] | (b[9] << 8) | (b[10] << 16) | ((uint32_t)b[11] << 24);
                v.w = b[12] | (b[13] << 8) | (b[14] << 16) | ((uint32_t)b[15] << 24);
            }
        }
        *reinterpret_cast<uint4 *>(sm.bytes + r * kBP + 16 * k) = v;
    }
}

// Encrypt and store the owned part of LL_L (window array a, side `side`).
template <int L>
__device__ void fwd_store_private(const Job &j, const FwdGeo &g, int16_t *a, const AesSmem &aes)
{
    constexpr int side = kFW >> L;
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
            const int x = (int)((o - rowo) / 2);
            const int v = (int)*cell(a, side, y - wrL, x - wcL) - 128;
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
__device__ void fwd_tile_fast(const Job &j, uint32_t tx, uint32_t ty, FwdSmem &sm,
                              const AesSmem &aes)
{
    FwdGeo g;
    g.W = (int)j.W;
    g.H = (int)j.H;
    g.C0 = (int)tx * kT;
    g.R0 = (int)ty * kT;
    g.wc0 = g.C0 - kFH;
    g.wr0 = g.R0 - kFH;
    g.pub = j.pub;
    g.L = j.L;
    fwd_load(j, g, sm);
    __syncthreads();
    fwd_level<1>(sm.bytes, kBP, sm.a1, g);
    __syncthreads();
    if (L >= 2) {
        fwd_level<2>(cell(sm.a1, kFW / 2, 0, 0), pitch_of(kFW / 2), sm.a2, g);
        __syncthreads();
    }
    if (L >= 3) {
        fwd_level<3>(cell(sm.a2, kFW / 4, 0, 0), pitch_of(kFW / 4), sm.a3, g);
        __syncthreads();
    }
    int16_t *ll = L == 1 ? sm.a1 : (L == 2 ? sm.a2 : sm.a3);
    fwd_store_private<L>(j, g, ll, aes);
}

// ---------------------------------------------------------------------------
// inverse
// ---------------------------------------------------------------------------

struct InvGeo {
    int W, H;
    int C0, R0;   // owned output tile origin (level 0)
    int wc0, wr0; // window origin (level 0) = C0 - 16, R0 - 16
    const uint8_t *pub;
    uint32_t L;
};

// a detail coefficient of band base `b` (level-l dims Hl x Wl) or 0 outside
__device__ __forceinline__ int coef(const uint8_t *b, int y, int x, int Hl, int Wl)
{
    if (y < 0 || y >= Hl || x < 0 || x >= Wl)
        return 0;
    const uint8_t *p = b + 2ull * ((uint64_t)y * (uint64_t)Wl + (uint64_t)x);
    if (((uintptr_t)p & 1u) == 0)
        return (int)__ldg(reinterpret_cast<const int16_t *>(p));
    return (int)(int16_t)(uint16_t)((uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 8));
}

// One inverse level l: LL_l window `ll` (side 256 >> l) + detail bands ->
// LL_{l-1} window `out` (side 256 >> (l-1)), or bytes to HBM when l == 1.
template <int l>
__device__ void inv_level(const int16_t *ll, int16_t *out, const Job &j, const InvGeo &g)
{
    constexpr int G = 4 >> (l - 1);
    constexpr int S = 16 >> (l - 1);
    constexpr int PAIRS = kIW >> l;   // level-l window side: 128, 64, 32
    constexpr int GROUPS = PAIRS / G; // 32
    constexpr int SEGS = PAIRS / S;   // 8
    constexpr int NL = G + 1, NH = G + 2;
    const int wcl = g.wc0 >> l, wrl = g.wr0 >> l;             // level-l window origin
    const int Wm = g.W >> (l - 1), Hm = g.H >> (l - 1);       // level l-1 image
    const int Wl = g.W >> l, Hl = g.H >> l;
    const uint8_t *band_hl = g.pub + band_offset(g.H, g.W, g.L, l, 0);
    const uint8_t *band_lh = g.pub + band_offset(g.H, g.W, g.L, l, 1);
    const uint8_t *band_hh = g.pub + band_offset(g.H, g.W, g.L, l, 2);

    for (int it = threadIdx.x; it < GROUPS * SEGS; it += blockDim.x) {
        const int gx = it % GROUPS, sy = it / GROUPS;
        const int p0 = gx * G, q0 = sy * S;
        // low columns p0 .. p0+G (s from LL_l, d from LH_l); high columns
        // p0-1 .. p0+G (s from HL_l, d from HH_l)
        auto load_row = [&](int k, int (&ls)[NL], int (&ld)[NL], int (&hs)[NH], int (&hd)[NH]) {
            const int kk = min(max(k, -1), PAIRS); // padded rows of `ll`
            const int y = wrl + k;
#pragma unroll
            for (int i = 0; i < NL; ++i) {
                ls[i] = (int)*cell(const_cast<int16_t *>(ll), PAIRS, kk, p0 + i);
                ld[i] = coef(band_lh, y, wcl + p0 + i, Hl, Wl);
            }
#pragma unroll
            for (int i = 0; i < NH; ++i) {
                hs[i] = coef(band_hl, y, wcl + p0 - 1 + i, Hl, Wl);
                hd[i] = coef(band_hh, y, wcl + p0 - 1 + i, Hl, Wl);
            }
        };
        int ls[NL], ld[NL], hs[NH], hd[NH];     // coefficients of row pair q (then q+1)
        int lxe[NL], hxe[NH];                   // reconstructed even rows x[2q]
        int ldp[NL], hdp[NH];                   // d[q-1]
        load_row(q0 - 1, ls, ld, hs, hd);
#pragma unroll
        for (int i = 0; i < NL; ++i)
            ldp[i] = ld[i];
#pragma unroll
        for (int i = 0; i < NH; ++i)
            hdp[i] = hd[i];
        load_row(q0, ls, ld, hs, hd);
        if (wrl + q0 == 0) { // d[-1] = d[0]
#pragma unroll
            for (int i = 0; i < NL; ++i)
                ldp[i] = ld[i];
#pragma unroll
            for (int i = 0; i < NH; ++i)
                hdp[i] = hd[i];
        }
#pragma unroll
        for (int i = 0; i < NL; ++i)
            lxe[i] = ls[i] - ((ldp[i] + ld[i] + 2) >> 2);
#pragma unroll
        for (int i = 0; i < NH; ++i)
            hxe[i] = hs[i] - ((hdp[i] + hd[i] + 2) >> 2);

        for (int q = q0; q < q0 + S; ++q) {
            int ns[NL], nd[NL], nhs[NH], nhd[NH];
            load_row(q + 1, ns, nd, nhs, nhd);
            int lxn[NL], hxn[NH], lxo[NL], hxo[NH];
            const bool bottom = (2 * (wrl + q) + 2 == Hm); // x[m] = x[m-2]
            const bool first = (wrl + q + 1 == 0);         // d[-1] = d[0] for the next pair
#pragma unroll
            for (int i = 0; i < NL; ++i) {
                lxn[i] = ns[i] - (((first ? nd[i] : ld[i]) + nd[i] + 2) >> 2);
                lxo[i] = ld[i] + ((lxe[i] + (bottom ? lxe[i] : lxn[i])) >> 1);
            }
#pragma unroll
            for (int i = 0; i < NH; ++i) {
                hxn[i] = nhs[i] - (((first ? nhd[i] : hd[i]) + nhd[i] + 2) >> 2);
                hxo[i] = hd[i] + ((hxe[i] + (bottom ? hxe[i] : hxn[i])) >> 1);
            }
            // undo the row lifting of rows 2q (lxe / hxe) and 2q+1 (lxo / hxo)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int *Lv = half ? lxo : lxe;
                const int *Hv = half ? hxo : hxe;
                int ev[NL], xo[2 * G];
#pragma unroll
                for (int i = 0; i < NL; ++i) {
                    const int hl = (wcl + p0 + i == 0) ? Hv[i + 1] : Hv[i]; // d[-1] = d[0]
                    ev[i] = Lv[i] - ((hl + Hv[i + 1] + 2) >> 2);
                }
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    const int xr = (2 * (wcl + p0 + i) + 2 == Wm) ? ev[i] : ev[i + 1];
                    xo[2 * i] = ev[i];
                    xo[2 * i + 1] = Hv[i + 1] + ((ev[i] + xr) >> 1);
                }
                const int r = 2 * q + half; // window row at level l-1
                if (l > 1) {
                    int16_t *o = cell(out, 2 * PAIRS, r, 2 * p0);
#pragma unroll
                    for (int i = 0; i < 2 * G; ++i)
                        o[i] = (int16_t)xo[i];
                } else {
                    const int R = g.wr0 + r, C = g.wc0 + 2 * p0;
                    if (R >= g.R0 && R < min(g.R0 + kT, g.H) && C >= g.C0 &&
                        C + 2 * G <= g.C0 + kT && C < g.W) {
                        const uint64_t go = (uint64_t)R * (uint64_t)g.W + (uint64_t)C;
                        uint8_t *dst = j.out + go;
                        if (C + 2 * G <= g.W && go + 2 * G <= j.n && ((uintptr_t)dst & 7u) == 0) {
                            uint2 w;
                            w.x = (xo[0] & 255) | ((xo[1] & 255) << 8) | ((xo[2] & 255) << 16) |
                                  ((uint32_t)(xo[3] & 255) << 24);
                            w.y = (xo[4] & 255) | ((xo[5] & 255) << 8) | ((xo[6] & 255) << 16) |
                                  ((uint32_t)(xo[7] & 255) << 24);
                            *reinterpret_cast<uint2 *>(dst) = w;
                        } else {
#pragma unroll
                            for (int i = 0; i < 2 * G; ++i)
                                if (C + i < g.W && go + i < j.n)
                                    dst[i] = (uint8_t)xo[i];
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NL; ++i) {
                lxe[i] = lxn[i];
                ld[i] = nd[i];
            }
#pragma unroll
            for (int i = 0; i < NH; ++i) {
                hxe[i] = hxn[i];
                hd[i] = nhd[i];
            }
        }
    }
}

// Decrypt the window's part of LL_L into `a` (side 256 >> L), adding back 128.
template <int L>
__device__ void inv_load_private(const Job &j, const InvGeo &g, int16_t *a, const AesSmem &aes)
{
    constexpr int side = kIW >> L;
    const int WL = g.W >> L, HL = g.H >> L;
    const int wcL = g.wc0 >> L, wrL = g.wr0 >> L;
    const int xa = max(wcL, 0), xb = min(wcL + side, WL); // columns [xa, xb)
    const int bpr = (2 * (xb - xa) + 15) / 16 + 1;
    for (int idx = threadIdx.x; idx < side * bpr; idx += blockDim.x) {
        const int k = idx / bpr, jb = idx - k * bpr;
        const int y = wrL + k;
        if (y < 0 || y >= HL || xb <= xa)
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
            const int v = (int)(int16_t)(uint16_t)(lo8 | (hi8 << 8)) + 128;
            const int x = (int)((o - rowo) / 2);
            *cell(a, side, k, x - wcL) = (int16_t)v;
        }
    }
}

template <int L>
__device__ void inv_tile_fast(const Job &j, uint32_t tx, uint32_t ty, InvSmem &sm,
                              const AesSmem &aes)
{
    InvGeo g;
    g.W = (int)j.W;
    g.H = (int)j.H;
    g.C0 = (int)tx * kT;
    g.R0 = (int)ty * kT;
    g.wc0 = g.C0 - kIH;
    g.wr0 = g.R0 - kIH;
    g.pub = j.pub_in;
    g.L = j.L;
    int16_t *top = L == 1 ? sm.a0 : (L == 2 ? sm.a1 : sm.a2);
    inv_load_private<L>(j, g, top, aes);
    __syncthreads();
    if (L >= 3) {
        inv_level<3>(sm.a2, sm.a1, j, g);
        __syncthreads();
    }
    if (L >= 2) {
        inv_level<2>(sm.a1, sm.a0, j, g);
        __syncthreads();
    }
    inv_level<1>(sm.a0, nullptr, j, g);
}

} // namespace fast
} // namespace frag
