/*
 * frag_oracle.c -- the oracle: a plain, slow, single-threaded CPU statement of
 * the agnostic DWT fragmentation method (Chapter 5 of the thesis
 * "An Efficient Data Protection Architecture Based on Fragmentation and
 * Encryption", arXiv 1803.04880).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this code.  It shares no source, header,
 * table or constant generator with the CUDA library, and the library never
 * calls it.
 *
 * What it computes, step by step, in the order the thesis gives:
 *   1. bytes -> H x W matrix, row-major; bytes past n are virtual zeros
 *      (Sec. 5.2.1: every byte is treated as an 8-bit pixel of a gray image;
 *      the matrix size is configurable).
 *   2. level shift v = b - 128 (Sec. 5.2.3: 0..255 is treated as -128..127).
 *   3. per level l = 1..L on the current LL region: every row with the 1-D
 *      5/3 lifting of Eq. 5.1 / Eq. 5.2, then every column (horizontal first,
 *      Sec. 5.2.2); the next level works on the top-left LL quarter only
 *      (dyadic decomposition, Sec. 5.1.1).
 *   4. private fragment = LL_L as int16 little-endian, row-major, XORed with
 *      an AES-128-CTR keystream (Sec. 5.2.1 names AES-128 for the private
 *      fragment; CTR is the parallel AES mode of Sec. 2.3).
 *   5. public fragment = the detail bands as int16 little-endian, coarsest
 *      level first: HL_L, LH_L, HH_L, HL_{L-1}, ..., HH_1, each row-major.
 *   6. recovery = decrypt LL_L, then the exact inverse lifting, levels L..1,
 *      columns before rows within a level, then +128 (Sec. 5.2.3: the 5/3
 *      filter maps integers to integers and is lossless).
 *
 * Readings taken where the thesis is ambiguous or misprinted:
 *   - Eq. 5.2 prints a minus before the floor; the update adds it.  Only the
 *     plus sign reproduces the thesis's own 8x8 level-1 matrix A and its
 *     F(4,4) weights (Sec. 5.2.2), and it is the JPEG 2000 form.
 *   - x_ext of Eq. 5.1 is the whole-sample symmetric extension:
 *     x[-1] = x[1], x[m] = x[m-2], hence d[-1] = d[0] (matches A).
 *   - floor is "the largest integer not exceeding" (text under Eq. 5.2),
 *     written here as an explicit floor, not as C's truncating division.
 *   - H is ceil(n / W) rounded up to a multiple of 2^L; W must be a multiple
 *     of 2^L, so every 1-D length at every level is even and >= 2.
 *   - AES-CTR counter block = nonce (8 bytes, big-endian) || block index
 *     (8 bytes, big-endian), block index = byte offset / 16 from 0; a short
 *     last block uses a prefix of its keystream block.
 *
 * Block mode (Sec. 5.2.1): every B x B block (8 x 8 in the thesis) of the
 * matrix is transformed as an image of its own; the band images keep the
 * whole-matrix shapes, block (bi, bj) filling one tile of each.
 *
 * Pins (tests/test_oracle_*.py): the thesis's matrix A and F(4,4) weights,
 * its magnitude bounds (as recomputed where misprinted), a hand-worked 2x2
 * example that fixes the row-before-column order, closed forms for length 2,
 * constant and ramp inputs, level-shift invariance, exact round trips,
 * FIPS-197 Appendix C.1 and SP 800-38A F.5.1 vectors.  Parity unpinned: none.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ERANGE 2
#define ORACLE_ENOMEM 3

/* floor(v / 2^sh) for any sign, written out (Eq. 5.1/5.2 floors). */
static int32_t floor_shift(int64_t v, int sh)
{
    int64_t q = (int64_t)1 << sh;
    if (v >= 0)
        return (int32_t)(v / q);
    return (int32_t)(-((-v + q - 1) / q));
}

/* ---------------------------------------------------------------------- */
/* 1-D LeGall 5/3 lifting, Eq. 5.1 (predict) and Eq. 5.2 (update).         */
/* ---------------------------------------------------------------------- */

/* Forward on x[0..m), m even >= 2.  out[0..m/2) = s (low), out[m/2..m) = d
 * (high).  x and out must not overlap. */
void oracle_lift53_fwd_1d(const int32_t *x, int64_t m, int32_t *out)
{
    int64_t h = m / 2, k;
    int32_t *s = out, *d = out + h;
    /* Eq. 5.1: every odd sample minus the floored mean of its even
     * neighbours; x[m] is the mirror x[m-2]. */
    for (k = 0; k < h; k++) {
        int64_t right = (2 * k + 2 < m) ? x[2 * k + 2] : x[m - 2];
        d[k] = x[2 * k + 1] - floor_shift((int64_t)x[2 * k] + right, 1);
    }
    /* Eq. 5.2 (plus sign): every even sample plus the floored quarter of its
     * two neighbouring details, +2 for rounding; d[-1] is the mirror d[0]. */
    for (k = 0; k < h; k++) {
        int64_t left = (k > 0) ? d[k - 1] : d[0];
        s[k] = x[2 * k] + floor_shift(left + d[k] + 2, 2);
    }
}

/* Inverse of oracle_lift53_fwd_1d: in[0..m/2) = s, in[m/2..m) = d. */
void oracle_lift53_inv_1d(const int32_t *in, int64_t m, int32_t *x)
{
    int64_t h = m / 2, k;
    const int32_t *s = in, *d = in + h;
    /* undo the update first: even samples */
    for (k = 0; k < h; k++) {
        int64_t left = (k > 0) ? d[k - 1] : d[0];
        x[2 * k] = s[k] - floor_shift(left + d[k] + 2, 2);
    }
    /* then undo the predict: odd samples */
    for (k = 0; k < h; k++) {
        int64_t right = (2 * k + 2 < m) ? x[2 * k + 2] : x[m - 2];
        x[2 * k + 1] = d[k] + floor_shift((int64_t)x[2 * k] + right, 1);
    }
}

/* ---------------------------------------------------------------------- */
/* 2-D dyadic transform (Sec. 5.1.1, Sec. 5.2.2).                          */
/* ---------------------------------------------------------------------- */

/* In place on a (H x W, row-major, int32).  Level l transforms the top-left
 * (H >> (l-1)) x (W >> (l-1)) region: all its rows, then all its columns.
 * Result is the Mallat layout: LL_L top-left, then for each level l the
 * HL_l (top-right), LH_l (bottom-left), HH_l (bottom-right) quadrants of the
 * level-l region. */
int oracle_dwt53_fwd_2d(int32_t *a, int64_t H, int64_t W, int L)
{
    int l;
    int64_t r, c, n = (H > W ? H : W);
    int32_t *line = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *res = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!line || !res) {
        free(line);
        free(res);
        return ORACLE_ENOMEM;
    }
    for (l = 1; l <= L; l++) {
        int64_t h = H >> (l - 1), w = W >> (l - 1);
        for (r = 0; r < h; r++) { /* horizontal direction first */
            for (c = 0; c < w; c++)
                line[c] = a[r * W + c];
            oracle_lift53_fwd_1d(line, w, res);
            for (c = 0; c < w; c++)
                a[r * W + c] = res[c];
        }
        for (c = 0; c < w; c++) { /* then the vertical direction */
            for (r = 0; r < h; r++)
                line[r] = a[r * W + c];
            oracle_lift53_fwd_1d(line, h, res);
            for (r = 0; r < h; r++)
                a[r * W + c] = res[r];
        }
    }
    free(line);
    free(res);
    return ORACLE_OK;
}

/* Exact inverse of oracle_dwt53_fwd_2d: levels L..1, columns then rows. */
int oracle_dwt53_inv_2d(int32_t *a, int64_t H, int64_t W, int L)
{
    int l;
    int64_t r, c, n = (H > W ? H : W);
    int32_t *line = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *res = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!line || !res) {
        free(line);
        free(res);
        return ORACLE_ENOMEM;
    }
    for (l = L; l >= 1; l--) {
        int64_t h = H >> (l - 1), w = W >> (l - 1);
        for (c = 0; c < w; c++) {
            for (r = 0; r < h; r++)
                line[r] = a[r * W + c];
            oracle_lift53_inv_1d(line, h, res);
            for (r = 0; r < h; r++)
                a[r * W + c] = res[r];
        }
        for (r = 0; r < h; r++) {
            for (c = 0; c < w; c++)
                line[c] = a[r * W + c];
            oracle_lift53_inv_1d(line, w, res);
            for (c = 0; c < w; c++)
                a[r * W + c] = res[c];
        }
    }
    free(line);
    free(res);
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------- */
/* AES-128 (FIPS-197), byte oriented, with every table derived here.       */
/* ---------------------------------------------------------------------- */

/* multiplication by x in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1 (FIPS-197
 * Sec. 4.2.1) */
static uint8_t gf_xtime(uint8_t a)
{
    return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0x00));
}

static uint8_t gf_mul(uint8_t a, uint8_t b)
{
    uint8_t p = 0;
    while (b) {
        if (b & 1)
            p ^= a;
        a = gf_xtime(a);
        b >>= 1;
    }
    return p;
}

static uint8_t rotl8(uint8_t v, int s)
{
    return (uint8_t)((v << s) | (v >> (8 - s)));
}

/* S-box entry (FIPS-197 Sec. 5.1.1): multiplicative inverse (a^254, with 0
 * mapped to 0) followed by the affine transformation. */
static uint8_t aes_sbox_entry(uint8_t a)
{
    uint8_t inv = 1, base = a;
    int e = 254;
    if (a == 0)
        inv = 0;
    else {
        while (e) {
            if (e & 1)
                inv = gf_mul(inv, base);
            base = gf_mul(base, base);
            e >>= 1;
        }
    }
    return (uint8_t)(inv ^ rotl8(inv, 1) ^ rotl8(inv, 2) ^ rotl8(inv, 3) ^ rotl8(inv, 4) ^ 0x63);
}

static uint8_t g_sbox[256];
static int g_sbox_ready = 0;

static void aes_init_sbox(void)
{
    int i;
    if (g_sbox_ready)
        return;
    for (i = 0; i < 256; i++)
        g_sbox[i] = aes_sbox_entry((uint8_t)i);
    g_sbox_ready = 1;
}

/* Key expansion for Nk = 4, Nr = 10 (FIPS-197 Sec. 5.2): 176 bytes. */
void oracle_aes128_expand_key(const uint8_t key[16], uint8_t rk[176])
{
    int i, j;
    uint8_t rcon = 1;
    aes_init_sbox();
    memcpy(rk, key, 16);
    for (i = 4; i < 44; i++) {
        uint8_t t[4];
        for (j = 0; j < 4; j++)
            t[j] = rk[4 * (i - 1) + j];
        if (i % 4 == 0) {
            uint8_t first = t[0]; /* RotWord */
            t[0] = t[1];
            t[1] = t[2];
            t[2] = t[3];
            t[3] = first;
            for (j = 0; j < 4; j++) /* SubWord */
                t[j] = g_sbox[t[j]];
            t[0] ^= rcon; /* Rcon[i/4] = x^(i/4 - 1) */
            rcon = gf_xtime(rcon);
        }
        for (j = 0; j < 4; j++)
            rk[4 * i + j] = (uint8_t)(rk[4 * (i - 4) + j] ^ t[j]);
    }
}

/* Cipher (FIPS-197 Sec. 5.1).  state[r + 4c] is byte r of column c. */
void oracle_aes128_encrypt_block(const uint8_t rk[176], const uint8_t in[16], uint8_t out[16])
{
    uint8_t s[16], t[16];
    int round, i, c, r;
    aes_init_sbox();
    for (i = 0; i < 16; i++)
        s[i] = (uint8_t)(in[i] ^ rk[i]);
    for (round = 1; round <= 10; round++) {
        for (i = 0; i < 16; i++) /* SubBytes */
            s[i] = g_sbox[s[i]];
        for (r = 0; r < 4; r++) /* ShiftRows: row r rotates left by r */
            for (c = 0; c < 4; c++)
                t[r + 4 * c] = s[r + 4 * ((c + r) % 4)];
        memcpy(s, t, 16);
        if (round != 10) { /* MixColumns */
            for (c = 0; c < 4; c++) {
                uint8_t a0 = s[4 * c], a1 = s[4 * c + 1], a2 = s[4 * c + 2], a3 = s[4 * c + 3];
                s[4 * c + 0] = (uint8_t)(gf_mul(a0, 2) ^ gf_mul(a1, 3) ^ a2 ^ a3);
                s[4 * c + 1] = (uint8_t)(a0 ^ gf_mul(a1, 2) ^ gf_mul(a2, 3) ^ a3);
                s[4 * c + 2] = (uint8_t)(a0 ^ a1 ^ gf_mul(a2, 2) ^ gf_mul(a3, 3));
                s[4 * c + 3] = (uint8_t)(gf_mul(a0, 3) ^ a1 ^ a2 ^ gf_mul(a3, 2));
            }
        }
        for (i = 0; i < 16; i++) /* AddRoundKey */
            s[i] ^= rk[16 * round + i];
    }
    memcpy(out, s, 16);
}

/* CTR: data[i] ^= keystream byte (first_block*16 + i).  Counter block for
 * block b = nonce (big-endian) || b (big-endian). */
void oracle_aes128_ctr_xor(const uint8_t key[16], uint64_t nonce, uint64_t first_block,
                           uint8_t *data, uint64_t len)
{
    uint8_t rk[176], ctr[16], ks[16];
    uint64_t off, b;
    int i;
    oracle_aes128_expand_key(key, rk);
    for (off = 0; off < len; off += 16) {
        b = first_block + off / 16;
        for (i = 0; i < 8; i++) {
            ctr[i] = (uint8_t)(nonce >> (56 - 8 * i));
            ctr[8 + i] = (uint8_t)(b >> (56 - 8 * i));
        }
        oracle_aes128_encrypt_block(rk, ctr, ks);
        for (i = 0; i < 16 && off + (uint64_t)i < len; i++)
            data[off + (uint64_t)i] ^= ks[i];
    }
}

/* ---------------------------------------------------------------------- */
/* Fragment layout and the two public operations.                          */
/* ---------------------------------------------------------------------- */

int oracle_sizes(uint64_t n, uint32_t W, uint32_t L, uint64_t *H, uint64_t *priv_bytes,
                 uint64_t *pub_bytes)
{
    uint64_t rows, step;
    if (W == 0 || L == 0 || L > 16 || (W % (1u << L)) != 0)
        return ORACLE_EINVAL;
    step = (uint64_t)1 << L;
    rows = (n + W - 1) / W;
    rows = (rows + step - 1) / step * step;
    *H = rows;
    *priv_bytes = 2 * (rows >> L) * (uint64_t)(W >> L);
    *pub_bytes = 2 * (rows * (uint64_t)W) - *priv_bytes;
    return ORACLE_OK;
}

static int put_i16(uint8_t *dst, int32_t v)
{
    if (v < -32768 || v > 32767)
        return ORACLE_ERANGE;
    dst[0] = (uint8_t)((uint32_t)v & 0xff);
    dst[1] = (uint8_t)(((uint32_t)v >> 8) & 0xff);
    return ORACLE_OK;
}

static int32_t get_i16(const uint8_t *src)
{
    return (int32_t)(int16_t)(uint16_t)(src[0] | (src[1] << 8));
}

/* copy one band (rows [r0, r0+h), cols [c0, c0+w) of a) to int16 LE */
static int store_band(const int32_t *a, int64_t W, int64_t r0, int64_t c0, int64_t h, int64_t w,
                      uint8_t *dst)
{
    int64_t r, c;
    for (r = 0; r < h; r++)
        for (c = 0; c < w; c++)
            if (put_i16(dst + 2 * (r * w + c), a[(r0 + r) * W + c0 + c]) != ORACLE_OK)
                return ORACLE_ERANGE;
    return ORACLE_OK;
}

static void load_band(int32_t *a, int64_t W, int64_t r0, int64_t c0, int64_t h, int64_t w,
                      const uint8_t *src)
{
    int64_t r, c;
    for (r = 0; r < h; r++)
        for (c = 0; c < w; c++)
            a[(r0 + r) * W + c0 + c] = get_i16(src + 2 * (r * w + c));
}

int oracle_protect(const uint8_t *in, uint64_t n, uint32_t W, uint32_t L, const uint8_t key[16],
                   uint64_t nonce, uint8_t *priv, uint8_t *pub)
{
    uint64_t H, pb, ub, i;
    int64_t Hl, Wl;
    int32_t *a;
    int l, st;
    uint8_t *p;
    if (oracle_sizes(n, W, L, &H, &pb, &ub) != ORACLE_OK)
        return ORACLE_EINVAL;
    if (n == 0)
        return ORACLE_OK;
    a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H * W));
    if (!a)
        return ORACLE_ENOMEM;
    for (i = 0; i < H * W; i++) /* map + level shift; past n the byte is 0 */
        a[i] = (int32_t)(i < n ? in[i] : 0) - 128;
    st = oracle_dwt53_fwd_2d(a, (int64_t)H, (int64_t)W, (int)L);
    if (st != ORACLE_OK) {
        free(a);
        return st;
    }
    Hl = (int64_t)(H >> L);
    Wl = (int64_t)(W >> L);
    st = store_band(a, W, 0, 0, Hl, Wl, priv); /* LL_L */
    if (st == ORACLE_OK)
        oracle_aes128_ctr_xor(key, nonce, 0, priv, pb);
    p = pub;
    for (l = (int)L; l >= 1 && st == ORACLE_OK; l--) {
        int64_t h = (int64_t)(H >> l), w = (int64_t)(W >> l);
        st = store_band(a, W, 0, w, h, w, p); /* HL_l: top-right */
        p += 2 * h * w;
        if (st == ORACLE_OK)
            st = store_band(a, W, h, 0, h, w, p); /* LH_l: bottom-left */
        p += 2 * h * w;
        if (st == ORACLE_OK)
            st = store_band(a, W, h, w, h, w, p); /* HH_l: bottom-right */
        p += 2 * h * w;
    }
    free(a);
    return st;
}

int oracle_recover(const uint8_t *priv, const uint8_t *pub, uint64_t n, uint32_t W, uint32_t L,
                   const uint8_t key[16], uint64_t nonce, uint8_t *out)
{
    uint64_t H, pb, ub, i;
    int64_t Hl, Wl;
    int32_t *a;
    uint8_t *plain;
    const uint8_t *p;
    int l, st;
    if (oracle_sizes(n, W, L, &H, &pb, &ub) != ORACLE_OK)
        return ORACLE_EINVAL;
    if (n == 0)
        return ORACLE_OK;
    a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H * W));
    plain = (uint8_t *)malloc((size_t)pb);
    if (!a || !plain) {
        free(a);
        free(plain);
        return ORACLE_ENOMEM;
    }
    memcpy(plain, priv, (size_t)pb);
    oracle_aes128_ctr_xor(key, nonce, 0, plain, pb);
    Hl = (int64_t)(H >> L);
    Wl = (int64_t)(W >> L);
    load_band(a, W, 0, 0, Hl, Wl, plain);
    p = pub;
    for (l = (int)L; l >= 1; l--) {
        int64_t h = (int64_t)(H >> l), w = (int64_t)(W >> l);
        load_band(a, W, 0, w, h, w, p);
        p += 2 * h * w;
        load_band(a, W, h, 0, h, w, p);
        p += 2 * h * w;
        load_band(a, W, h, w, h, w, p);
        p += 2 * h * w;
    }
    st = oracle_dwt53_inv_2d(a, (int64_t)H, (int64_t)W, (int)L);
    for (i = 0; i < n && st == ORACLE_OK; i++) {
        int32_t v = a[i] + 128;
        if (v < 0 || v > 255)
            st = ORACLE_ERANGE;
        else
            out[i] = (uint8_t)v;
    }
    free(a);
    free(plain);
    return st;
}

/* ---------------------------------------------------------------------- */
/* Block mode (Sec. 5.2.1): the data is cut into chunks seen as matrices    */
/* and every matrix is processed block by block (8 x 8 in the thesis, "the */
/* block size chosen can be changed"), each block being transformed as an  */
/* image of its own: L levels inside the block, the symmetric extension at  */
/* the block's own borders.  Layout (a reading): band (l, k) of the whole   */
/* matrix keeps its H_l x W_l shape and block (bi, bj) fills the tile of    */
/* rows [bi B/2^l, (bi+1) B/2^l) and columns [bj B/2^l, (bj+1) B/2^l) of    */
/* it; the fragments are then stored exactly as in the whole-matrix mode.   */
/* ---------------------------------------------------------------------- */

/* H = ceil(n / W) rounded up to a multiple of B; W must be a multiple of B
 * and B a multiple of 2^L */
int oracle_block_sizes(uint64_t n, uint32_t W, uint32_t L, uint32_t B, uint64_t *H,
                       uint64_t *priv_bytes, uint64_t *pub_bytes)
{
    uint64_t rows;
    if (W == 0 || L == 0 || L > 16 || B == 0 || (B % (1u << L)) != 0 || (W % B) != 0)
        return ORACLE_EINVAL;
    rows = (n + W - 1) / W;
    rows = (rows + B - 1) / B * B;
    *H = rows;
    *priv_bytes = 2 * (rows >> L) * (uint64_t)(W >> L);
    *pub_bytes = 2 * (rows * (uint64_t)W) - *priv_bytes;
    return ORACLE_OK;
}

/* move the bands of one transformed block (Mallat layout in blk, B x B)
 * to (to_global = 1) or from (0) their tiles in the whole-matrix Mallat
 * layout of a (H x W) */
static void block_tiles(int32_t *a, int64_t H, int64_t W, int32_t *blk, int64_t B, int L,
                        int64_t bi, int64_t bj, int to_global)
{
    int l, k;
    int64_t r, c;
    for (l = L; l >= 1; l--) {
        const int64_t b = B >> l, Hl = H >> l, Wl = W >> l;
        for (k = (l == L ? -1 : 0); k < 3; k++) {
            /* k = -1: LL_L; 0: HL (top-right); 1: LH (bottom-left); 2: HH */
            const int64_t br = (k == 1 || k == 2) ? b : 0, bc = (k == 0 || k == 2) ? b : 0;
            const int64_t gr = (k == 1 || k == 2) ? Hl : 0, gc = (k == 0 || k == 2) ? Wl : 0;
            for (r = 0; r < b; r++)
                for (c = 0; c < b; c++) {
                    int32_t *g = &a[(gr + bi * b + r) * W + gc + bj * b + c];
                    int32_t *t = &blk[(br + r) * B + bc + c];
                    if (to_global)
                        *g = *t;
                    else
                        *t = *g;
                }
        }
    }
}

/* block-mode transform of the level-shifted matrix a, in place, forward or
 * inverse */
static int blocks_2d(int32_t *a, int64_t H, int64_t W, int L, int64_t B, int fwd)
{
    int64_t bi, bj, r, c;
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H * W));
    int32_t *blk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(B * B));
    int st = ORACLE_OK;
    if (!src || !blk) {
        free(src);
        free(blk);
        return ORACLE_ENOMEM;
    }
    memcpy(src, a, sizeof(int32_t) * (size_t)(H * W));
    for (bi = 0; bi < H / B && st == ORACLE_OK; bi++)
        for (bj = 0; bj < W / B && st == ORACLE_OK; bj++) {
            if (fwd) {
                for (r = 0; r < B; r++)
                    for (c = 0; c < B; c++)
                        blk[r * B + c] = src[(bi * B + r) * W + bj * B + c];
                st = oracle_dwt53_fwd_2d(blk, B, B, L);
                block_tiles(a, H, W, blk, B, L, bi, bj, 1);
            } else {
                block_tiles(src, H, W, blk, B, L, bi, bj, 0);
                st = oracle_dwt53_inv_2d(blk, B, B, L);
                for (r = 0; r < B; r++)
                    for (c = 0; c < B; c++)
                        a[(bi * B + r) * W + bj * B + c] = blk[r * B + c];
            }
        }
    free(src);
    free(blk);
    return st;
}

/* whole-matrix Mallat image <-> fragments (shared by both modes' callers) */
static int store_fragments(const int32_t *a, uint64_t H, uint32_t W, uint32_t L,
                           const uint8_t key[16], uint64_t nonce, uint64_t pb, uint8_t *priv,
                           uint8_t *pub)
{
    int l, st;
    uint8_t *p = pub;
    st = store_band(a, W, 0, 0, (int64_t)(H >> L), (int64_t)(W >> L), priv); /* LL_L */
    if (st == ORACLE_OK)
        oracle_aes128_ctr_xor(key, nonce, 0, priv, pb);
    for (l = (int)L; l >= 1 && st == ORACLE_OK; l--) {
        int64_t h = (int64_t)(H >> l), w = (int64_t)(W >> l);
        st = store_band(a, W, 0, w, h, w, p);
        p += 2 * h * w;
        if (st == ORACLE_OK)
            st = store_band(a, W, h, 0, h, w, p);
        p += 2 * h * w;
        if (st == ORACLE_OK)
            st = store_band(a, W, h, w, h, w, p);
        p += 2 * h * w;
    }
    return st;
}

int oracle_protect_blocks(const uint8_t *in, uint64_t n, uint32_t W, uint32_t L, uint32_t B,
                          const uint8_t key[16], uint64_t nonce, uint8_t *priv, uint8_t *pub)
{
    uint64_t H, pb, ub, i;
    int32_t *a;
    int st;
    if (oracle_block_sizes(n, W, L, B, &H, &pb, &ub) != ORACLE_OK)
        return ORACLE_EINVAL;
    if (n == 0)
        return ORACLE_OK;
    a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H * W));
    if (!a)
        return ORACLE_ENOMEM;
    for (i = 0; i < H * W; i++) /* map + level shift; past n the byte is 0 */
        a[i] = (int32_t)(i < n ? in[i] : 0) - 128;
    st = blocks_2d(a, (int64_t)H, (int64_t)W, (int)L, (int64_t)B, 1);
    if (st == ORACLE_OK)
        st = store_fragments(a, H, W, L, key, nonce, pb, priv, pub);
    free(a);
    return st;
}

int oracle_recover_blocks(const uint8_t *priv, const uint8_t *pub, uint64_t n, uint32_t W,
                          uint32_t L, uint32_t B, const uint8_t key[16], uint64_t nonce,
                          uint8_t *out)
{
    uint64_t H, pb, ub, i;
    int32_t *a;
    uint8_t *plain;
    const uint8_t *p;
    int l, st;
    if (oracle_block_sizes(n, W, L, B, &H, &pb, &ub) != ORACLE_OK)
        return ORACLE_EINVAL;
    if (n == 0)
        return ORACLE_OK;
    a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H * W));
    plain = (uint8_t *)malloc((size_t)pb);
    if (!a || !plain) {
        free(a);
        free(plain);
        return ORACLE_ENOMEM;
    }
    memcpy(plain, priv, (size_t)pb);
    oracle_aes128_ctr_xor(key, nonce, 0, plain, pb);
    load_band(a, W, 0, 0, (int64_t)(H >> L), (int64_t)(W >> L), plain);
    p = pub;
    for (l = (int)L; l >= 1; l--) {
        int64_t h = (int64_t)(H >> l), w = (int64_t)(W >> l);
        load_band(a, W, 0, w, h, w, p);
        p += 2 * h * w;
        load_band(a, W, h, 0, h, w, p);
        p += 2 * h * w;
        load_band(a, W, h, w, h, w, p);
        p += 2 * h * w;
    }
    st = blocks_2d(a, (int64_t)H, (int64_t)W, (int)L, (int64_t)B, 0);
    for (i = 0; i < n && st == ORACLE_OK; i++) {
        int32_t v = a[i] + 128;
        if (v < 0 || v > 255)
            st = ORACLE_ERANGE;
        else
            out[i] = (uint8_t)v;
    }
    free(a);
    free(plain);
    return st;
}

/* ---------------------------------------------------------------------- */
/* The thesis's three fragments in its own storage (Sec. 5.2.1 and Sec.    */
/* 5.2.3, "Evaluation of the storage necessary for DWT"): 8 x 8 blocks, two */
/* levels; per block the private fragment LL_2 takes 4 x 10 bits (40), the  */
/* first public fragment HL_2 and LH_2 at 10 bits and HH_2 at 11 bits      */
/* (40 + 40 + 44 = 124), the second public fragment the 48 level-1 details */
/* at 10 bits (480): 644 bits for the block's 512.  The bounds of the      */
/* level-2 coefficients (338 / 468 / 648) and of level 1 (every detail     */
/* within +-510 by the floors of Eq. 5.1 / 5.2) are what make the widths    */
/* enough; a value outside its width is reported, never stored.            */
/*                                                                          */
/* Layout (a reading: the thesis gives the widths, not the order):          */
/*   - a value is its two's complement in `width` bits; a record's values   */
/*     follow each other from bit 0, each band's tile row-major, and a      */
/*     record's bits fill bytes from the least significant bit;             */
/*   - A (private, then AES-128-CTR as every private fragment): one 5-byte  */
/*     record per block, blocks row-major;                                  */
/*   - B (first public): the blocks of a block row follow each other every  */
/*     124 bits, and every block row starts on a byte (ceil(124 nbx / 8)    */
/*     bytes a row);                                                        */
/*   - C (second public): one 60-byte record per block, blocks row-major;   */
/*     the public fragment of the call is B followed by C.                  */
/* ---------------------------------------------------------------------- */

#define PK_B 8
#define PK_L 2

int oracle_packed_sizes(uint64_t n, uint32_t W, uint64_t *H, uint64_t *a_bytes, uint64_t *b_bytes,
                        uint64_t *c_bytes)
{
    uint64_t pb, ub, nbx, nby;
    if (oracle_block_sizes(n, W, PK_L, PK_B, H, &pb, &ub) != ORACLE_OK)
        return ORACLE_EINVAL;
    nbx = W / PK_B;
    nby = *H / PK_B;
    *a_bytes = 5 * nbx * nby;
    *b_bytes = nby * ((124 * nbx + 7) / 8);
    *c_bytes = 60 * nbx * nby;
    return ORACLE_OK;
}

/* value v as `width` bits at bit position pos of buf (buf zeroed first) */
static int put_bits(uint8_t *buf, uint64_t pos, int32_t v, int width)
{
    int i;
    const int32_t lo = -(1 << (width - 1)), hi = (1 << (width - 1)) - 1;
    if (v < lo || v > hi)
        return ORACLE_ERANGE;
    for (i = 0; i < width; i++)
        if (((uint32_t)v >> i) & 1u)
            buf[(pos + (uint64_t)i) / 8] |= (uint8_t)(1u << ((pos + (uint64_t)i) % 8));
    return ORACLE_OK;
}

static int32_t get_bits(const uint8_t *buf, uint64_t pos, int width)
{
    int i;
    uint32_t u = 0;
    for (i = 0; i < width; i++)
        u |= (uint32_t)((buf[(pos + (uint64_t)i) / 8] >> ((pos + (uint64_t)i) % 8)) & 1u) << i;
    if (u & (1u << (width - 1))) /* sign */
        return (int32_t)u - (int32_t)(1u << width);
    return (int32_t)u;
}

/* the values of one block's three records, in record order, with their
 * widths: walks the block's Mallat layout (blk, 8 x 8) in the order above */
static void record_fields(int rec, int64_t idx[48], int width[48], int *count)
{
    int k = 0, t, r, c;
    if (rec == 0) { /* A: LL_2 at rows 0..1, cols 0..1 */
        for (r = 0; r < 2; r++)
            for (c = 0; c < 2; c++, k++) {
                idx[k] = r * PK_B + c;
                width[k] = 10;
            }
    } else if (rec == 1) { /* B: HL_2 (top-right), LH_2 (bottom-left), HH_2 */
        for (t = 0; t < 3; t++)
            for (r = 0; r < 2; r++)
                for (c = 0; c < 2; c++, k++) {
                    idx[k] = (r + (t >= 1 ? 2 : 0)) * PK_B + c + (t != 1 ? 2 : 0);
                    width[k] = t == 2 ? 11 : 10;
                }
    } else { /* C: HL_1, LH_1, HH_1 (4 x 4 each) */
        for (t = 0; t < 3; t++)
            for (r = 0; r < 4; r++)
                for (c = 0; c < 4; c++, k++) {
                    idx[k] = (r + (t >= 1 ? 4 : 0)) * PK_B + c + (t != 1 ? 4 : 0);
                    width[k] = 10;
                }
    }
    *count = k;
}

/* bit position of block (bi, bj)'s record rec */
static uint64_t record_pos(int rec, uint64_t bi, uint64_t bj, uint64_t nbx)
{
    if (rec == 0)
        return 40 * (bi * nbx + bj);
    if (rec == 1)
        return 8 * (bi * ((124 * nbx + 7) / 8)) + 124 * bj;
    return 480 * (bi * nbx + bj);
}

int oracle_protect_packed(const uint8_t *in, uint64_t n, uint32_t W, const uint8_t key[16],
                          uint64_t nonce, uint8_t *a_out, uint8_t *b_out, uint8_t *c_out)
{
    uint64_t H, sa, sb, sc, i, bi, bj, nbx;
    int32_t *a, blk[PK_B * PK_B];
    int st = ORACLE_OK, rec, k, cnt;
    int64_t idx[48];
    int width[48];
    uint8_t *outs[3];
    if (oracle_packed_sizes(n, W, &H, &sa, &sb, &sc) != ORACLE_OK)
        return ORACLE_EINVAL;
    if (n == 0)
        return ORACLE_OK;
    a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H * W));
    if (!a)
        return ORACLE_ENOMEM;
    for (i = 0; i < H * W; i++) /* map + level shift; past n the byte is 0 */
        a[i] = (int32_t)(i < n ? in[i] : 0) - 128;
    st = blocks_2d(a, (int64_t)H, (int64_t)W, PK_L, PK_B, 1);
    memset(a_out, 0, (size_t)sa);
    memset(b_out, 0, (size_t)sb);
    memset(c_out, 0, (size_t)sc);
    outs[0] = a_out;
    outs[1] = b_out;
    outs[2] = c_out;
    nbx = W / PK_B;
    for (bi = 0; bi < H / PK_B && st == ORACLE_OK; bi++)
        for (bj = 0; bj < nbx && st == ORACLE_OK; bj++) {
            block_tiles(a, (int64_t)H, (int64_t)W, blk, PK_B, PK_L, (int64_t)bi, (int64_t)bj, 0);
            for (rec = 0; rec < 3 && st == ORACLE_OK; rec++) {
                uint64_t pos = record_pos(rec, bi, bj, nbx);
                record_fields(rec, idx, width, &cnt);
                for (k = 0; k < cnt && st == ORACLE_OK; k++) {
                    st = put_bits(outs[rec], pos, blk[idx[k]], width[k]);
                    pos += (uint64_t)width[k];
                }
            }
        }
    if (st == ORACLE_OK)
        oracle_aes128_ctr_xor(key, nonce, 0, a_out, sa);
    free(a);
    return st;
}

int oracle_recover_packed(const uint8_t *a_in, const uint8_t *b_in, const uint8_t *c_in, uint64_t n,
                          uint32_t W, const uint8_t key[16], uint64_t nonce, uint8_t *out)
{
    uint64_t H, sa, sb, sc, i, bi, bj, nbx;
    int32_t *a, blk[PK_B * PK_B];
    uint8_t *plain;
    const uint8_t *ins[3];
    int st = ORACLE_OK, rec, k, cnt;
    int64_t idx[48];
    int width[48];
    if (oracle_packed_sizes(n, W, &H, &sa, &sb, &sc) != ORACLE_OK)
        return ORACLE_EINVAL;
    if (n == 0)
        return ORACLE_OK;
    a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(H * W));
    plain = (uint8_t *)malloc((size_t)sa);
    if (!a || !plain) {
        free(a);
        free(plain);
        return ORACLE_ENOMEM;
    }
    memcpy(plain, a_in, (size_t)sa);
    oracle_aes128_ctr_xor(key, nonce, 0, plain, sa);
    ins[0] = plain;
    ins[1] = b_in;
    ins[2] = c_in;
    nbx = W / PK_B;
    for (bi = 0; bi < H / PK_B; bi++)
        for (bj = 0; bj < nbx; bj++) {
            for (k = 0; k < PK_B * PK_B; k++)
                blk[k] = 0;
            for (rec = 0; rec < 3; rec++) {
                uint64_t pos = record_pos(rec, bi, bj, nbx);
                record_fields(rec, idx, width, &cnt);
                for (k = 0; k < cnt; k++) {
                    blk[idx[k]] = get_bits(ins[rec], pos, width[k]);
                    pos += (uint64_t)width[k];
                }
            }
            block_tiles(a, (int64_t)H, (int64_t)W, blk, PK_B, PK_L, (int64_t)bi, (int64_t)bj, 1);
        }
    st = blocks_2d(a, (int64_t)H, (int64_t)W, PK_L, PK_B, 0);
    for (i = 0; i < n && st == ORACLE_OK; i++) {
        int32_t v = a[i] + 128;
        if (v < 0 || v > 255)
            st = ORACLE_ERANGE;
        else
            out[i] = (uint8_t)v;
    }
    free(a);
    free(plain);
    return st;
}
