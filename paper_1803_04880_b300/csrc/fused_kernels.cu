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
//             level), computing only what that state needs (fwd_warm).
//   inverse   iteration t consumes level-3 row t, level-2 rows 2t-1, 2t and
//             level-1 rows 4t-3 .. 4t; the column inverse of each level
//             (undo Eq. 5.2, then Eq. 5.1) emits two rows of the level below
//             per coefficient row, the row inverse makes them LL samples, and
//             level 1 ends in level-0 rows 8t-7 .. 8t.  A unit first runs one
//             iteration that stores nothing and only rebuilds the column
//             state (inv_warm; with three levels it also loads the level-3 d
//             row two above its first).
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
#include "aes_tt.cuh"
#include "frag_internal.cuh"
#include "swar.cuh"

namespace frag {
namespace fuse {

using strm::from_i16x2;
using strm::kB2;
using strm::pavg;
using strm::pq4;
using strm::to_i16x2;


// warps per CTA (each warp runs its own units): a launch that enciphers
// keeps one CTA an SM around its AES table; otherwise the forward passes
// measured fastest as one CTA of 16 warps an SM, the inverse and the small
// second pass as four CTAs of 4 warps
#ifndef FUSE_FWD_WARPS
#define FUSE_FWD_WARPS 16
#endif
#ifndef FUSE_INV_WARPS
#define FUSE_INV_WARPS 4
#endif
#ifndef FUSE_PK_WARPS
#define FUSE_PK_WARPS 4
#endif
template <bool FWD, bool PK, bool CIPH>
__host__ __device__ constexpr int cta_warps()
{
    return CIPH ? 16 : PK ? FUSE_PK_WARPS : FWD ? FUSE_FWD_WARPS : FUSE_INV_WARPS;
}
// stages per warp (iterations in flight + the one being read) and resident
// CTAs per SM the register budget is cut for, per direction
#ifndef FUSE_FWD_DEPTH
#define FUSE_FWD_DEPTH 3
#endif
#ifndef FUSE_INV_DEPTH
#define FUSE_INV_DEPTH 2
#endif
constexpr int kFwdDepth = FUSE_FWD_DEPTH;
constexpr int kInvDepth = FUSE_INV_DEPTH;
constexpr int kFwdStage = 8 * 256; // 8 level-0 rows x 32 lanes x 8 bytes
// packed samples (a second pass over LL_3, 16-bit values): 16 bytes a lane,
// two stages (the shared memory of three does not fit beside the AES table)
constexpr int kFwdStagePk = 8 * 512;
constexpr int kFwdDepthPk = 2;
template <bool PK>
__host__ __device__ constexpr int fwd_stage() { return PK ? kFwdStagePk : kFwdStage; }
template <bool PK>
__host__ __device__ constexpr int fwd_depth() { return PK ? kFwdDepthPk : kFwdDepth; }
// inverse stage: the level-1 bands HL/LH/HH, rows j = 0..3, 8 bytes a lane --
// with box loads each band a box of 4 rows of 272 bytes (136 int16 from the
// 16-byte-aligned column just left of the strip's first lane; lane l's 8
// bytes at 8 + 8 l) on a 128-byte boundary, the layout a TMA box load writes
// -- then region X: level-1 LL rows (one level), or level-2 rows k = 0..1
// of the three bands (4 bytes a lane) followed by LL_2 rows (two levels) or
// the four level-3 words (three levels)
constexpr int kL1Row = 272;
constexpr int kL1Box = 9 * 128; // 4 rows of 272 bytes, rounded up to 128
// BOX: the layout the level-1 box loads need (a launch that uses them);
// otherwise rows of 256 bytes, lane l's 8 bytes at 8 l, row slot 3 j + k
template <bool BOX>
__host__ __device__ constexpr int l1_at(int j, int k) { return BOX ? 8 + kL1Box * k + kL1Row * j : 256 * (3 * j + k); }
template <bool BOX>
__host__ __device__ constexpr int inv_x() { return BOX ? 3 * kL1Box : 12 * 256; }
template <bool BOX>
__host__ __device__ constexpr int inv_l2ll() { return inv_x<BOX>() + 6 * 128; }
template <bool BOX>
__host__ __device__ constexpr int inv_l3() { return inv_x<BOX>() + 6 * 128; }
template <bool BOX>
__host__ __device__ constexpr int inv_stage() { return inv_l3<BOX>() + 4 * 128; }

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
__device__ __forceinline__ void cp16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// TMA box loads of the inverse's level-1 bands: one mbarrier a stage and warp
// (arrival count 1: the issuing lane's expect_tx), completed by the bytes of
// the stage's three boxes
constexpr uint32_t kL1TmaBytes = 3 * 4 * kL1Row;
constexpr uint32_t kTmaSpinLimit = 1u << 22; // polls of a stage's barrier before giving up
constexpr int kErrTmaWait = 7;               // device error word: a box load that did not arrive
__device__ __forceinline__ void mbar_init(uint32_t a)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(a), "r"(parity)
                 : "memory");
    return ok != 0;
}
// the lanes of a warp poll a stage barrier together until its phase `par`
// completes, at most `limit` polls (so they agree on the outcome); false: it
// did not complete
__device__ __forceinline__ bool box_wait(uint32_t bar, uint32_t par, uint32_t limit)
{
    uint32_t polls = 0;
    while (!__all_sync(0xffffffffu, mbar_try(bar, par)))
        if (++polls == limit)
            return false;
    return true;
}
// generic-proxy reads of the stage before the async proxy overwrites it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// box (x, y) of a 2D map into shared memory at dst (128-byte aligned); x a
// multiple of 8 values (16 bytes)
__device__ __forceinline__ void tma2d(uint32_t dst, const CUtensorMap *m, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// Shared-memory reads of the stage ring as ordinary loads, so the compiler
// may schedule them freely; they stay after cp.async.wait_group, whose asm
// clobbers memory.  `a` is a shared-window address like the cp.async
// destinations.
extern __shared__ __align__(128) uint8_t g_fuse_smem[];
__device__ __forceinline__ const uint8_t *ring_ptr(uint32_t a)
{
    return g_fuse_smem + (a - (uint32_t)__cvta_generic_to_shared(g_fuse_smem));
}
__device__ __forceinline__ uint2 lds8(uint32_t a) { return *reinterpret_cast<const uint2 *>(ring_ptr(a)); }
__device__ __forceinline__ uint32_t lds4(uint32_t a) { return *reinterpret_cast<const uint32_t *>(ring_ptr(a)); }
__device__ __forceinline__ uint32_t lds2(uint32_t a) { return *reinterpret_cast<const uint16_t *>(ring_ptr(a)); }

// ---------------------------------------------------------------------------
// AES-128-CTR of the private fragment while LL_L is on chip (Sec. 5.2.1: the
// private fragment is encrypted with AES)
//
// The keystream does not depend on the data, so a warp computes it ahead of
// the rows that need it, 32 blocks at a time (one a lane, every lane busy),
// into a ring of 16-byte slots in shared memory; the lanes then XOR their LL
// words with it right before the store (protect) or right after the load
// (recover).  The slots follow the LL rows of the unit in order: row r takes
// nb slots, the blocks of the private fragment from the one that holds the
// warp's first LL column of that row on (nb covers the warp's 32 lanes of
// columns whatever the row's offset modulo 16 bytes), so slot
// (r - r_first) nb + (block - first block of row r) holds a block of row r.
// Before an iteration the warp fills the ring up to the last row the
// iteration touches; the ring keeps the iteration's slots (at most 4 rows of
// 17) and the up to 31 filled ahead.
// ---------------------------------------------------------------------------
constexpr int kKsSlots = 128;
constexpr int kKsBytes = 16 * kKsSlots;
constexpr int kTableBytes = 4 * aes::kTableWords;

struct Ks {
    uint32_t ring;       // this warp's keystream ring (shared-window address)
    uint32_t nb;         // slots a row takes
    uint32_t q32, r32;   // 32 = q32 nb + r32
    uint32_t produced;   // slots filled so far
    uint32_t prow, pmod; // the slot this lane fills next: block pmod of row r_first + prow
    uint32_t col_lo;     // first LL column of the warp's lanes
    uint64_t r_first;    // LL row of slot 0
    uint64_t WF;         // LL row length
};

__device__ __forceinline__ Ks ks_init(const FuseBuf &b, uint32_t sx, int lane, uint32_t ring, int r_first)
{
    Ks K;
    const int h = (int)b.halo;
    const int c_first = (int)sx * 8 * (31 - h) - 8 * h; // lane 0's first level-0 column
    const uint32_t lo = (uint32_t)max(c_first, 0) >> b.F;
    const uint32_t hi = (uint32_t)min(c_first + 256, (int)b.W) >> b.F;
    K.ring = ring;
    K.col_lo = lo;
    K.nb = ((hi - lo + 7) >> 3) + 1;
    K.q32 = 32u / K.nb;
    K.r32 = 32u - K.q32 * K.nb;
    K.produced = 0;
    K.prow = (uint32_t)lane / K.nb;
    K.pmod = (uint32_t)lane - K.prow * K.nb;
    K.r_first = (uint64_t)max(r_first, 0);
    K.WF = b.W >> b.F;
    return K;
}

// fill the ring through slot upto - 1 (warp-uniform)
__device__ __forceinline__ void ks_fill(Ks &K, uint32_t upto, const uint32_t *tel, const AesKeys &keys,
                                        uint64_t nonce, int lane)
{
    while (K.produced < upto) {
        const uint64_t r = K.r_first + K.prow;
        const uint64_t blk = ((r * K.WF + K.col_lo) >> 3) + K.pmod;
        uint32_t ks[4];
        aes::ctr_block(tel, keys, nonce, blk, ks);
        __syncwarp(); // every lane is done with the slots about to be refilled
        const uint32_t a = K.ring + ((K.produced + (uint32_t)lane) & (kKsSlots - 1)) * 16;
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(ks[0]), "r"(ks[1]),
                     "r"(ks[2]), "r"(ks[3])
                     : "memory");
        __syncwarp();
        K.prow += K.q32;
        K.pmod += K.r32;
        if (K.pmod >= K.nb) {
            K.pmod -= K.nb;
            ++K.prow;
        }
        K.produced += 32;
    }
}

// shared-window address of the keystream bytes of LL element e of row r
// (rows below r_first, which no lane uses, land on some slot of the ring)
__device__ __forceinline__ uint32_t ks_at(const Ks &K, uint64_t r, uint64_t e)
{
    const uint32_t slot = (uint32_t)(r - K.r_first) * K.nb +
                          (uint32_t)((e >> 3) - ((r * K.WF + K.col_lo) >> 3));
    return K.ring + (slot & (kKsSlots - 1)) * 16 + ((uint32_t)e & 7u) * 2;
}

// int16 stores at element index idx of a band (streaming: never re-read
// here), predicated on p: a lane with p false issues the store but writes
// nothing, so the lanes that do not own their columns (and the warm-up
// iterations) need no branch around a group of stores
__device__ __forceinline__ void pst8(bool p, uint8_t *band, uint64_t idx, uint32_t a, uint32_t b)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t"
                 "@q st.global.cs.v2.b32 [%1], {%2, %3};\n\t}" ::"r"((uint32_t)p),
                 "l"(band + 2 * idx), "r"(a), "r"(b));
}
__device__ __forceinline__ void pst4(bool p, uint8_t *band, uint64_t idx, uint32_t a)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t"
                 "@q st.global.cs.b32 [%1], %2;\n\t}" ::"r"((uint32_t)p),
                 "l"(band + 2 * idx), "r"(a));
}
__device__ __forceinline__ void pst2(bool p, uint8_t *band, uint64_t idx, uint32_t a)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t"
                 "@q st.global.cs.b16 [%1], %2;\n\t}" ::"r"((uint32_t)p),
                 "l"(band + 2 * idx), "h"((unsigned short)a));
}
// raw byte addresses: 8 bytes streaming, 16 bytes L2-cached (a scratch the
// next pass reads)
__device__ __forceinline__ void pst8b(bool p, uint8_t *at, uint2 v)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t"
                 "@q st.global.cs.v2.b32 [%1], {%2, %3};\n\t}" ::"r"((uint32_t)p),
                 "l"(at), "r"(v.x), "r"(v.y));
}
__device__ __forceinline__ void pst16b(bool p, uint8_t *at, uint4 v)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t"
                 "@q st.global.cg.v4.b32 [%1], {%2, %3, %4, %5};\n\t}" ::"r"((uint32_t)p),
                 "l"(at), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w));
}

// Store-ready bias.  A detail word that goes to a band is kept as
// v + 0x8000 per half (the usual bias plus 0x4000), so its int16 form is one
// XOR.  The lifting steps that read such a word fold the extra 0x40004000
// into their add constants: a chain of 32-bit adds and subtractions of
// packed words is exact whenever every half of the final result is in
// [0, 2^16), whatever the intermediate carries.
constexpr uint32_t kQ = 0x80008000u; // v + 0x8000 per half, from v - 0x8000 per half
__device__ __forceinline__ uint32_t q_i16(uint32_t w) { return w ^ kQ; } // to int16 pairs
// pq4 of two store-ready words: ((a + b - 0x80008000) + 0x20002) >> 2, masked
__device__ __forceinline__ uint32_t pq4q(uint32_t a, uint32_t b)
{
    return ((a + b + 0x80018002u) >> 2) & 0x3fff3fffu;
}

// ---------------------------------------------------------------------------
// row lifting with the borders folded into byte-permute selectors
//
// With W a multiple of 8 a lane's 8 level-0 columns are all inside the row
// or all outside, so only two lanes of a strip meet a border at any level:
// the lane holding column 0 (left: d[-1] = d[0]) and the lane holding the
// last 8 columns (right: x[m] = x[m-2]).  Each lane keeps two selectors for
// the whole unit: sL picks (d[-1], d0) or (d0, d0), sR picks (x[m-2], x[m])
// or (x[m-2], x[m-2]); the other permutes never change.
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kSelNext = 0x5432; // (high half of a, low half of b)
constexpr uint32_t kSelRight = 0x3232; // high half of a, twice
constexpr uint32_t kSelLeft = 0x5454;  // low half of b, twice

struct Lane {
    int c0;         // level-0 column of the lane's first sample
    bool loads;     // the lane's columns are inside the matrix
    bool own;       // the lane's results belong to this strip
    bool first;     // the lane holds column 0
    bool last;      // the lane holds the last 8 columns
    uint32_t sL, sR;
};

__device__ __forceinline__ Lane make_lane(const FuseBuf &b, uint32_t sx, int lane)
{
    Lane ln;
    const int h = (int)b.halo;
    ln.c0 = (int)sx * 8 * (31 - h) + 8 * (lane - h);
    ln.loads = ln.c0 >= 0 && ln.c0 < (int)b.W;
    ln.own = lane >= h && lane <= 30 && ln.c0 < (int)b.W;
    ln.first = ln.c0 == 0;
    ln.last = ln.c0 + 8 == (int)b.W;
    ln.sL = ln.first ? kSelLeft : kSelNext;
    ln.sR = ln.last ? kSelRight : kSelNext;
    return ln;
}

// Level-1 row lift of the lane's 8 bytes (w0, w1) = x0..x7: P[0] = (s0, s1),
// P[1] = (s2, s3), P[2] = (d0, d1), P[3] = (d2, d3), biased; x8 and d[-1]
// come from the adjacent lanes
__device__ __forceinline__ void lift8(uint32_t w0, uint32_t w1, uint32_t sR, uint32_t sL,
                                      uint32_t (&P)[4])
{
    // bytes into 16-bit halves with 0x40 as the high byte: v + 0x4000
    const uint32_t e01 = __byte_perm(w0, 0x40404040u, 0x4240);
    const uint32_t o01 = __byte_perm(w0, 0x40404040u, 0x4341);
    const uint32_t e23 = __byte_perm(w1, 0x40404040u, 0x4240);
    const uint32_t o23 = __byte_perm(w1, 0x40404040u, 0x4341);
    const uint32_t e01n = __shfl_down_sync(kFull, e01, 1);
    const uint32_t e12 = __byte_perm(e01, e23, kSelNext); // (x2, x4)
    const uint32_t e34 = __byte_perm(e23, e01n, sR);      // (x6, x8)
    const uint32_t d01 = o01 - pavg(e01, e12) + kB2;      // Eq. 5.1
    const uint32_t d23 = o23 - pavg(e23, e34) + kB2;
    const uint32_t d23p = __shfl_up_sync(kFull, d23, 1);
    const uint32_t dm0 = __byte_perm(d23p, d01, sL);      // (d[-1], d0)
    const uint32_t d12 = __byte_perm(d01, d23, kSelNext); // (d1, d2)
    P[0] = e01 + pq4(dm0, d01) - 0x20002000u;             // Eq. 5.2
    P[1] = e23 + pq4(d12, d23) - 0x20002000u;
    P[2] = d01;
    P[3] = d23;
}

// The same lift on 8 packed 16-bit samples (w0 = (x0, x1) .. w3 = (x6, x7))
__device__ __forceinline__ void lift8p(const uint4 &w, uint32_t sR, uint32_t sL, uint32_t (&P)[4])
{
    const uint32_t e01 = __byte_perm(w.x, w.y, 0x5410); // (x0, x2)
    const uint32_t o01 = __byte_perm(w.x, w.y, 0x7632); // (x1, x3)
    const uint32_t e23 = __byte_perm(w.z, w.w, 0x5410); // (x4, x6)
    const uint32_t o23 = __byte_perm(w.z, w.w, 0x7632); // (x5, x7)
    const uint32_t e01n = __shfl_down_sync(kFull, e01, 1);
    const uint32_t e12 = __byte_perm(e01, e23, kSelNext);
    const uint32_t e34 = __byte_perm(e23, e01n, sR);
    const uint32_t d01 = o01 - pavg(e01, e12) + kB2;
    const uint32_t d23 = o23 - pavg(e23, e34) + kB2;
    const uint32_t d23p = __shfl_up_sync(kFull, d23, 1);
    const uint32_t dm0 = __byte_perm(d23p, d01, sL);
    const uint32_t d12 = __byte_perm(d01, d23, kSelNext);
    P[0] = e01 + pq4(dm0, d01) - 0x20002000u;
    P[1] = e23 + pq4(d12, d23) - 0x20002000u;
    P[2] = d01;
    P[3] = d23;
}

// Level-1 row inverse to packed samples: (x0, x1) .. (x6, x7)
__device__ __forceinline__ uint4 unlift8p(const uint32_t (&w)[4], uint32_t sR, uint32_t sL)
{
    const uint32_t h23p = __shfl_up_sync(kFull, w[3], 1);
    const uint32_t hm0 = __byte_perm(h23p, w[2], sL);
    const uint32_t h12 = __byte_perm(w[2], w[3], kSelNext);
    const uint32_t e01 = w[0] - pq4(hm0, w[2]) + 0x20002000u;
    const uint32_t e23 = w[1] - pq4(h12, w[3]) + 0x20002000u;
    const uint32_t e01n = __shfl_down_sync(kFull, e01, 1);
    const uint32_t e12 = __byte_perm(e01, e23, kSelNext);
    const uint32_t e34 = __byte_perm(e23, e01n, sR);
    const uint32_t o01 = w[2] + pavg(e01, e12) - kB2;
    const uint32_t o23 = w[3] + pavg(e23, e34) - kB2;
    return make_uint4(__byte_perm(e01, o01, 0x5410), __byte_perm(e01, o01, 0x7632),
                      __byte_perm(e23, o23, 0x5410), __byte_perm(e23, o23, 0x7632));
}

// Level-1 row inverse: w[0..1] = L words, w[2..3] = H words -> the 8 bytes
__device__ __forceinline__ uint2 unlift8(const uint32_t (&w)[4], uint32_t sR, uint32_t sL)
{
    const uint32_t h23p = __shfl_up_sync(kFull, w[3], 1);
    const uint32_t hm0 = __byte_perm(h23p, w[2], sL); // (d[-1], d0)
    const uint32_t h12 = __byte_perm(w[2], w[3], kSelNext);
    const uint32_t e01 = w[0] - pq4(hm0, w[2]) + 0x20002000u; // undo Eq. 5.2
    const uint32_t e23 = w[1] - pq4(h12, w[3]) + 0x20002000u;
    const uint32_t e01n = __shfl_down_sync(kFull, e01, 1);
    const uint32_t e12 = __byte_perm(e01, e23, kSelNext);
    const uint32_t e34 = __byte_perm(e23, e01n, sR);
    const uint32_t o01 = w[2] + pavg(e01, e12) - kB2; // undo Eq. 5.1
    const uint32_t o23 = w[3] + pavg(e23, e34) - kB2;
    // biased halves: the low byte of each is the recovered byte
    return make_uint2(__byte_perm(e01, o01, 0x6240), __byte_perm(e23, o23, 0x6240));
}

// Level-2 row lift of the lane's four LL_1 samples (w0 = (y0, y1),
// w1 = (y2, y3)): L = (s0, s1), H = (d0, d1)
__device__ __forceinline__ void lift4(uint32_t w0, uint32_t w1, uint32_t sR, uint32_t sL,
                                      uint32_t &L, uint32_t &H)
{
    const uint32_t e = __byte_perm(w0, w1, 0x5410); // (y0, y2)
    const uint32_t o = __byte_perm(w0, w1, 0x7632); // (y1, y3)
    const uint32_t en = __shfl_down_sync(kFull, e, 1);
    const uint32_t es = __byte_perm(e, en, sR);    // (y2, y4)
    const uint32_t d = o - pavg(e, es) + kB2;      // Eq. 5.1
    const uint32_t dpl = __shfl_up_sync(kFull, d, 1);
    const uint32_t dm = __byte_perm(dpl, d, sL);   // (d[-1], d0)
    L = e + pq4(dm, d) - 0x20002000u;              // Eq. 5.2
    H = d;
}

// Level-2 row inverse: L = (s0, s1), H = (d0, d1) -> w0 = (y0, y1), w1 = (y2, y3)
__device__ __forceinline__ void unlift4(uint32_t L, uint32_t H, uint32_t sR, uint32_t sL,
                                        uint32_t &w0, uint32_t &w1)
{
    const uint32_t hp = __shfl_up_sync(kFull, H, 1);
    const uint32_t hm = __byte_perm(hp, H, sL);      // (d[-1], d0)
    const uint32_t e = L - pq4(hm, H) + 0x20002000u; // undo Eq. 5.2: (y0, y2)
    const uint32_t en = __shfl_down_sync(kFull, e, 1);
    const uint32_t es = __byte_perm(e, en, sR);      // (y2, y4)
    const uint32_t o = H + pavg(e, es) - kB2;        // undo Eq. 5.1: (y1, y3)
    w0 = __byte_perm(e, o, 0x5410);
    w1 = __byte_perm(e, o, 0x7632);
}

// Level-3 row lift of the lane's two LL_2 samples z = (z0, z1): returns
// (s, d) of the pair in one word (s low, d high)
__device__ __forceinline__ uint32_t lift2(uint32_t z, bool first, bool last)
{
    const uint32_t zn = __shfl_down_sync(kFull, z, 1);
    const uint32_t e = z & 0xffffu, o = z >> 16;
    const uint32_t en = last ? e : (zn & 0xffffu);
    const uint32_t d = o - ((e + en) >> 1) + 0x4000u; // Eq. 5.1
    const uint32_t dpl = __shfl_up_sync(kFull, d, 1);
    const uint32_t dp = first ? d : dpl;
    const uint32_t s = e + ((dp + d + 2) >> 2) - 0x2000u; // Eq. 5.2
    return s | (d << 16);
}

// Level-3 row inverse: (s, d) word of a row-lifted LL_2 row -> (z0, z1)
__device__ __forceinline__ uint32_t unlift2(uint32_t w, bool first, bool last)
{
    const uint32_t s = w & 0xffffu, d = w >> 16;
    const uint32_t dpl = __shfl_up_sync(kFull, d, 1);
    const uint32_t dp = first ? d : dpl;
    const uint32_t z0 = s - ((dp + d + 2) >> 2) + 0x2000u; // undo Eq. 5.2
    const uint32_t zn = __shfl_down_sync(kFull, z0, 1);
    const uint32_t z2 = last ? z0 : zn;
    const uint32_t z1 = d + ((z0 + z2) >> 1) - 0x4000u; // undo Eq. 5.1
    return z0 | (z1 << 16);
}

// ---------------------------------------------------------------------------
// forward unit
// ---------------------------------------------------------------------------

// the level-0 rows of iteration t into its stage: rows 8t-1 .. 8t+6
template <bool PK>
__device__ __forceinline__ void fwd_issue(const FuseBuf &b, const Lane &ln, int t, int t_end,
                                          uint32_t ring_lane)
{
    if (PK) {
        // packed samples: every row of the matrix is whole (no byte tail)
        if (t < t_end && ln.loads) {
            const uint32_t st = ring_lane + (uint32_t)(t % kFwdDepthPk) * kFwdStagePk;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = 8 * t - 1 + j;
                if (r >= 0 && r < (int)b.H)
                    cp16(st + 512 * j, b.src + 2 * ((uint64_t)r * b.W + (uint64_t)ln.c0));
            }
        }
        cp_commit();
        return;
    }
    if (t < t_end && ln.loads) {
        const uint32_t st = ring_lane + (uint32_t)(t % kFwdDepth) * kFwdStage;
        const int r0 = 8 * t - 1;
        if (r0 >= 0 && r0 + 8 <= (int)b.full_rows) { // eight whole rows of data
            const uint8_t *p = b.src + (uint64_t)r0 * b.W + (uint64_t)ln.c0;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                cp8(st + 256 * j, p + (uint64_t)j * b.W, 8);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = r0 + j;
                if (r >= 0 && r < (int)b.H) {
                    const uint64_t off = (uint64_t)r * b.W + (uint64_t)ln.c0;
                    const uint32_t bytes =
                        off >= b.n ? 0u : (uint32_t)(b.n - off < 8 ? b.n - off : 8);
                    cp8(st + 256 * j, bytes ? b.src + off : b.src, bytes);
                }
            }
        }
    }
    cp_commit();
}

// LL_F of the final level: LL - 128 as int16 (both halves of each word)
__device__ __forceinline__ uint32_t ll_final(uint32_t w) { return to_i16x2(w - 0x00800080u); }

struct FwdState {
    uint32_t e0[4], dp[4]; // level 1: even row, d of the previous pair (store-ready)
    uint32_t e2L, e2H, p2L, p2H; // level 2 (p2L, p2H store-ready)
    uint32_t e3, p3;
};

// One iteration (rows 8t-1 .. 8t+6 in stage st).  CHECK: the iteration may
// meet the top (a level's row 0) or the bottom (a level's last row) of the
// matrix; no other iteration does, and none stores a row outside it.
template <bool CHECK, bool PK, bool CIPH, int FL>
__device__ __forceinline__ void fwd_iter(const FuseBuf &b, const Lane &ln, int t, uint32_t st,
                                         bool store, FwdState &S, const Ks &K)
{
    const int W = (int)b.W, H = (int)b.H;
    const int F = FL ? FL : (int)b.F;
    const int W1 = W >> 1, H1 = H >> 1, W2 = W >> 2, H2 = H >> 2, W3 = W >> 3, H3 = H >> 3;
    const bool fin = b.ll_final != 0;
    const bool ciph = CIPH && b.cipher != 0; // LL_F is the private fragment, enciphered here
    uint2 raw[8];
    uint4 rawp[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (PK)
            rawp[j] = *reinterpret_cast<const uint4 *>(ring_ptr(st + 512 * j));
        else
            raw[j] = lds8(st + 256 * j);
    }

    // level 1: pairs (8t-1+2j, 8t+2j) -> level-1 row 4t-1+j
    uint32_t y[4][2];
    const uint64_t col1 = (uint64_t)(ln.c0 >> 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t Po[4], Pe[4];
        if (PK) {
            lift8p(rawp[2 * j], ln.sR, ln.sL, Po);
            lift8p(rawp[2 * j + 1], ln.sR, ln.sL, Pe);
        } else {
            lift8(raw[2 * j].x, raw[2 * j].y, ln.sR, ln.sL, Po);
            lift8(raw[2 * j + 1].x, raw[2 * j + 1].y, ln.sR, ln.sL, Pe);
        }
        const int q = 4 * t - 1 + j;
        if (CHECK && 8 * t + 2 * j == H) { // x[m] = x[m-2] at the bottom border
#pragma unroll
            for (int k = 0; k < 4; ++k)
                Pe[k] = S.e0[k];
        }
        // d store-ready (LH_1, HH_1), and so the carried d[-1]
        uint32_t dv[4], sv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            dv[k] = Po[k] - pavg(S.e0[k], Pe[k]) + kQ; // Eq. 5.1 down the columns
        if (CHECK && q == 0) {                         // d[-1] = d[0] at the top border
#pragma unroll
            for (int k = 0; k < 4; ++k)
                S.dp[k] = dv[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // Eq. 5.2 down the columns: LL_1 (k < 2) biased, HL_1 store-ready
            const uint32_t u = S.e0[k] + pq4q(S.dp[k], dv[k]);
            sv[k] = k < 2 ? u - 0x20002000u : u + 0x20002000u;
            S.e0[k] = Pe[k];
            S.dp[k] = dv[k];
        }
        {
            const uint64_t idx = (uint64_t)q * (uint64_t)W1 + col1;
            const bool p = store && (!CHECK || (unsigned)q < (unsigned)H1);
            pst8(p, b.band[0][0], idx, q_i16(sv[2]), q_i16(sv[3])); // HL_1
            pst8(p, b.band[0][1], idx, q_i16(dv[0]), q_i16(dv[1])); // LH_1
            pst8(p, b.band[0][2], idx, q_i16(dv[2]), q_i16(dv[3])); // HH_1
            if (F == 1) {
                if (fin) {
                    uint32_t l0 = ll_final(sv[0]), l1 = ll_final(sv[1]);
                    if (ciph) {
                        const uint2 k = lds8(ks_at(K, (uint64_t)q, idx));
                        l0 ^= k.x;
                        l1 ^= k.y;
                    }
                    pst8(p, b.ll, idx, l0, l1);
                } else {
                    pst8(p, b.ll, idx, sv[0], sv[1]);
                }
            }
        }
        y[j][0] = sv[0];
        y[j][1] = sv[1];
    }
    if (F < 2)
        return;

    // level 2: LL_1 pairs (4t-1+2k, 4t+2k) -> level-2 row 2t-1+k
    uint32_t z[2];
    const uint64_t col2 = (uint64_t)(ln.c0 >> 2);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        uint32_t Lo, Ho, Le, He;
        lift4(y[2 * k][0], y[2 * k][1], ln.sR, ln.sL, Lo, Ho);
        lift4(y[2 * k + 1][0], y[2 * k + 1][1], ln.sR, ln.sL, Le, He);
        const int q2 = 2 * t - 1 + k;
        if (CHECK && 4 * t + 2 * k == H1) {
            Le = S.e2L;
            He = S.e2H;
        }
        // dL, dH (LH_2, HH_2) and sH (HL_2) store-ready, sL (LL_2) biased
        const uint32_t dL = Lo - pavg(S.e2L, Le) + kQ, dH = Ho - pavg(S.e2H, He) + kQ;
        if (CHECK && q2 == 0) {
            S.p2L = dL;
            S.p2H = dH;
        }
        const uint32_t sL = S.e2L + pq4q(S.p2L, dL) - 0x20002000u;
        const uint32_t sH = S.e2H + pq4q(S.p2H, dH) + 0x20002000u;
        S.e2L = Le;
        S.e2H = He;
        S.p2L = dL;
        S.p2H = dH;
        {
            const uint64_t idx = (uint64_t)q2 * (uint64_t)W2 + col2;
            const bool p = store && (!CHECK || (unsigned)q2 < (unsigned)H2);
            pst4(p, b.band[1][0], idx, q_i16(sH)); // HL_2
            pst4(p, b.band[1][1], idx, q_i16(dL)); // LH_2
            pst4(p, b.band[1][2], idx, q_i16(dH)); // HH_2
            if (F == 2) {
                uint32_t v = fin ? ll_final(sL) : sL;
                if (ciph)
                    v ^= lds4(ks_at(K, (uint64_t)q2, idx));
                pst4(p, b.ll, idx, v);
            }
        }
        z[k] = sL;
    }
    if (F < 3)
        return;

    // level 3: LL_2 pair (2t-1, 2t) -> level-3 row t-1
    const uint32_t wo = lift2(z[0], ln.first, ln.last);
    uint32_t we = lift2(z[1], ln.first, ln.last);
    const int q3 = t - 1;
    if (CHECK && 2 * t == H2)
        we = S.e3;
    const uint32_t d3 = wo - pavg(S.e3, we) + kB2;
    if (CHECK && q3 == 0)
        S.p3 = d3;
    const uint32_t s3 = S.e3 + pq4(S.p3, d3) - 0x20002000u;
    S.e3 = we;
    S.p3 = d3;
    {
        const uint64_t idx = (uint64_t)q3 * (uint64_t)W3 + (uint64_t)(ln.c0 >> 3);
        const bool p = store && (!CHECK || (unsigned)q3 < (unsigned)H3);
        const uint32_t sw = to_i16x2(s3), dw = to_i16x2(d3);
        pst2(p, b.band[2][0], idx, sw >> 16); // HL_3
        pst2(p, b.band[2][1], idx, dw);       // LH_3
        pst2(p, b.band[2][2], idx, dw >> 16); // HH_3
        uint32_t v = fin ? ll_final(s3) : s3;
        if (ciph)
            v ^= lds2(ks_at(K, (uint64_t)q3, idx));
        pst2(p, b.ll, idx, v);
    }
}

// A warm-up iteration away from the matrix's top and bottom (t >= 2, before
// the last two): it rebuilds only the state the next iteration reads.
//   first: the unit's first iteration (F before its first stored row) --
//          the level-1 column state and the even row level 2 reads next,
//          from rows 8t+2 .. 8t+6 (8t+4 .. 8t+6 with one level);
//   last:  the iteration right before the first stored row -- every word of
//          the state;
//   else:  the LL halves of levels 1 and 2 and level 3's even row.
// The row-H halves of the level-1 column lifting, the level-2 H column and
// the level-3 column are read again only through state the last warm-up
// iteration rebuilds from the rows it holds, and no band is written.
template <bool PK, int FL>
__device__ __forceinline__ void fwd_warm(const FuseBuf &b, const Lane &ln, uint32_t st, bool first, bool last,
                                         FwdState &S)
{
    const int F = FL ? FL : (int)b.F;
    auto lift = [&](int r, uint32_t(&P)[4]) {
        if (PK) {
            lift8p(*reinterpret_cast<const uint4 *>(ring_ptr(st + 512 * r)), ln.sR, ln.sL, P);
        } else {
            const uint2 w = lds8(st + 256 * r);
            lift8(w.x, w.y, ln.sR, ln.sL, P);
        }
    };
    // level 1: pairs j0 .. 3 of rows (8t-1+2j, 8t+2j)
    const int j0 = first ? (F == 1 ? 3 : 2) : 0;
    if (first) {
        uint32_t P[4];
        lift(2 * j0 - 1, P); // the even row before pair j0
#pragma unroll
        for (int k = 0; k < 4; ++k)
            S.e0[k] = P[k];
    }
    uint32_t y[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j < j0)
            continue;
        uint32_t Po[4], Pe[4];
        lift(2 * j, Po);
        lift(2 * j + 1, Pe);
        if (last && j == 3) {
#pragma unroll
            for (int k = 2; k < 4; ++k)
                S.dp[k] = Po[k] - pavg(S.e0[k], Pe[k]) + kQ;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint32_t dv = Po[k] - pavg(S.e0[k], Pe[k]) + kQ; // Eq. 5.1
            y[j][k] = S.e0[k] + pq4q(S.dp[k], dv) - 0x20002000u;   // Eq. 5.2: LL_1
            S.dp[k] = dv;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            S.e0[k] = Pe[k];
    }
    if (F < 2)
        return;
    if (first) { // level 2 reads only the even row next
        lift4(y[3][0], y[3][1], ln.sR, ln.sL, S.e2L, S.e2H);
        return;
    }
    // level 2: the L column (LL_2 for level 3), the H column's d only last
    uint32_t z[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        uint32_t Lo, Ho, Le, He;
        lift4(y[2 * k][0], y[2 * k][1], ln.sR, ln.sL, Lo, Ho);
        lift4(y[2 * k + 1][0], y[2 * k + 1][1], ln.sR, ln.sL, Le, He);
        const uint32_t dL = Lo - pavg(S.e2L, Le) + kQ;
        z[k] = S.e2L + pq4q(S.p2L, dL) - 0x20002000u;
        if (last && k == 1)
            S.p2H = Ho - pavg(S.e2H, He) + kQ;
        S.e2L = Le;
        S.e2H = He;
        S.p2L = dL;
    }
    if (F < 3)
        return;
    // level 3: the even row, and the column's d last
    const uint32_t we = lift2(z[1], ln.first, ln.last);
    if (last)
        S.p3 = lift2(z[0], ln.first, ln.last) - pavg(S.e3, we) + kB2;
    S.e3 = we;
}

template <bool PK, bool CIPH, int FL>
__device__ __forceinline__ void fwd_unit(const FuseBuf &b, uint32_t sx, uint32_t sy, uint32_t ring_lane,
                                         int lane, uint32_t ks_ring, const uint32_t *tel, const AesKeys &keys)
{
    const Lane ln = make_lane(b, sx, lane);
    const int t_begin = (int)(sy * b.seg_iters);
    const int t_end = min(t_begin + (int)b.seg_iters, (int)b.iters);
    const int F = FL ? FL : (int)b.F;
    const int t_first = max(t_begin - F, 0);
    const int t_fast_end = (int)b.iters - 2; // iterations t >= 2 and below this skip the checks
    // LL rows a stored iteration t writes: R t - 1 .. R t + R - 2
    const int R = 8 >> F;
    Ks K = {};
    if (CIPH && b.cipher)
        K = ks_init(b, sx, lane, ks_ring, R * t_begin - 1);

#pragma unroll
    for (int k = 0; k < fwd_depth<PK>() - 1; ++k)
        fwd_issue<PK>(b, ln, t_first + k, t_end, ring_lane);

    FwdState S; // zeros, in each word's form
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        S.e0[k] = kB2;
        S.dp[k] = kQ;
    }
    S.e2L = S.e2H = S.e3 = S.p3 = kB2;
    S.p2L = S.p2H = kQ;

    for (int t = t_first; t < t_end; ++t) {
        fwd_issue<PK>(b, ln, t + fwd_depth<PK>() - 1, t_end, ring_lane);
        // the keystream of the iteration's LL rows (while its loads land)
        if (CIPH && b.cipher && t >= t_begin)
            ks_fill(K, (uint32_t)((uint64_t)(R * t + R - 1) - K.r_first) * K.nb, tel, keys, b.nonce, lane);
        cp_wait<fwd_depth<PK>() - 1>();
        const uint32_t st = ring_lane + (uint32_t)(t % fwd_depth<PK>()) * fwd_stage<PK>();
        const bool store = ln.own && t >= t_begin;
        if (t >= 2 && t < t_fast_end) {
            if (t < t_begin)
                fwd_warm<PK, FL>(b, ln, st, t == t_first && t_first == t_begin - F, t == t_begin - 1, S);
            else
                fwd_iter<false, PK, CIPH, FL>(b, ln, t, st, store, S, K);
        } else {
            fwd_iter<true, PK, CIPH, FL>(b, ln, t, st, store, S, K);
        }
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// inverse unit
// ---------------------------------------------------------------------------

// int16 word(s) of the input -> biased values
__device__ __forceinline__ uint32_t in16(uint32_t w) { return from_i16x2(w); }

// every row iteration t reads inside its level: no per-row tests
template <int FL>
__device__ __forceinline__ bool inv_inside(const FuseBuf &b, int t)
{
    const int F = FL ? FL : (int)b.F;
    return t >= 1 && 4 * t < (int)(b.H >> 1) && (F < 2 || 2 * t < (int)(b.H >> 2)) &&
           (F < 3 || t < (int)(b.H >> 3));
}

// The level-1 box loads of a lone buffer's first inverse pass: in an
// iteration whose rows are all inside, lane 0 loads the three level-1 bands'
// rows as three TMA boxes into the stage (the bytes the per-lane copies would
// write, and the lanes outside the matrix read zeros) and the lanes wait on
// the stage's barrier instead of copying them.
struct Tma {
    const CUtensorMap *map; // the three level-1 band maps (nullptr: per-lane copies)
    uint32_t ring;          // the warp's stage ring (128-byte aligned)
    uint32_t bar;           // the warp's barriers, one a stage
    int x0;                 // box origin: the level-1 column 4 left of lane 0's first
    bool leader;            // lane 0
};

// the coefficient rows iteration t consumes, into its stage
template <int FL, bool BOX>
__device__ __forceinline__ void inv_issue(const FuseBuf &b, const Lane &ln, int t, int t_end,
                                          uint32_t ring8, uint32_t ring4, const Tma &tm)
{
    const bool inside = inv_inside<FL>(b, t);
    const bool box = BOX && tm.map != nullptr && t < t_end && inside;
    if (box) {
        // every lane has read the stage's last contents (iteration t - 2)
        __syncwarp();
        if (tm.leader) {
            const uint32_t st = (uint32_t)(t % kInvDepth);
            const uint32_t bar = tm.bar + 8u * st;
            fence_proxy_async();
            mbar_expect(bar, kL1TmaBytes);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                tma2d(tm.ring + st * inv_stage<BOX>() + kL1Box * k, tm.map + k, tm.x0, 4 * t - 3, bar);
        }
    }
    if (t < t_end && ln.loads) {
        const int F = FL ? FL : (int)b.F;
        const uint32_t so = (uint32_t)(t % kInvDepth) * inv_stage<BOX>();
        const uint32_t W1 = b.W >> 1, H1 = b.H >> 1, W2 = b.W >> 2, H2 = b.H >> 2;
        const uint32_t c1 = (uint32_t)ln.c0 >> 1, c2 = (uint32_t)ln.c0 >> 2;
        if (inside) {
            const uint64_t o1 = 2ull * ((uint64_t)(4 * t - 3) * W1 + c1);
            if (!box) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        cp8(ring8 + so + l1_at<BOX>(j, k), b.band[0][k] + o1 + 2ull * j * W1, 8);
            }
            if (F == 1) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    cp8(ring8 + so + inv_x<BOX>() + 256 * j, b.ll + o1 + 2ull * j * W1, 8);
            } else {
                const uint64_t o2 = 2ull * ((uint64_t)(2 * t - 1) * W2 + c2);
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        cp4(ring4 + so + inv_x<BOX>() + 128 * (3 * k + m), b.band[1][m] + o2 + 2ull * k * W2, 4);
                if (F == 2) {
#pragma unroll
                    for (int k = 0; k < 2; ++k)
                        cp4(ring4 + so + inv_l2ll<BOX>() + 128 * k, b.ll + o2 + 2ull * k * W2, 4);
                }
            }
        } else {
            const uint64_t off = 2ull * ((uint64_t)(4 * t - 3) * W1 + c1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = 4 * t - 3 + j;
                if (q >= 0 && q < (int)H1) {
                    const uint64_t o = off + 2ull * j * W1;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        cp8(ring8 + so + l1_at<BOX>(j, k), b.band[0][k] + o, 8);
                    if (F == 1)
                        cp8(ring8 + so + inv_x<BOX>() + 256 * j, b.ll + o, 8);
                }
            }
            if (F >= 2) {
                const uint64_t off2 = 2ull * ((uint64_t)(2 * t - 1) * W2 + c2);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int q = 2 * t - 1 + k;
                    if (q >= 0 && q < (int)H2) {
                        const uint64_t o = off2 + 2ull * k * W2;
#pragma unroll
                        for (int m = 0; m < 3; ++m)
                            cp4(ring4 + so + inv_x<BOX>() + 128 * (3 * k + m), b.band[1][m] + o, 4);
                        if (F == 2)
                            cp4(ring4 + so + inv_l2ll<BOX>() + 128 * k, b.ll + o, 4);
                    }
                }
            }
        }
        if (F == 3 && (inside || t < (int)(b.H >> 3))) {
            // one int16 per lane: copy the aligned word that holds it (band
            // bases are 4-byte aligned, so the word stays inside the band)
            const uint64_t e = (uint64_t)t * (b.W >> 3) + ((uint32_t)ln.c0 >> 3);
            const uint64_t off = 2ull * (e & ~1ull);
            const uint32_t bytes = (e & 1ull) ? 4u : 2u;
#pragma unroll
            for (int m = 0; m < 3; ++m)
                cp4(ring4 + so + inv_l3<BOX>() + 128 * m, b.band[2][m] + off, bytes);
            cp4(ring4 + so + inv_l3<BOX>() + 128 * 3, b.ll + off, bytes);
        }
    }
    cp_commit();
}

// eager column inverse of one coefficient row q of a level (words of the
// lane): xe = x[2q], xo = x[2q-1]; (xp, dp) = (x[2q-2], d[q-1]) carried.
// top: q == 0 (d[-1] = d[0]); bottom: q is one past the last row (x[2q] =
// x[2q-2], only the odd row is real).  SQ / DQ: s / d (and dp) come
// store-ready (a band read as one XOR) instead of biased; xe, xo are biased.
template <bool CHECK, bool SQ, bool DQ>
__device__ __forceinline__ void col_inv(uint32_t s, uint32_t d, bool top, bool bottom, uint32_t &xp,
                                        uint32_t &dp, uint32_t &xo, uint32_t &xe)
{
    if (CHECK && top)
        dp = d;
    const uint32_t q = DQ ? pq4q(dp, d) : pq4(dp, d);
    xe = (CHECK && bottom) ? xp : (SQ ? s - q - 0x20002000u : s - q + 0x20002000u); // undo Eq. 5.2
    xo = DQ ? dp + pavg(xp, xe) - kQ : dp + pavg(xp, xe) - kB2;                      // undo Eq. 5.1
    xp = xe;
    dp = d;
}

// 8 recovered bytes of row r at the lane's columns
__device__ __forceinline__ void store_bytes(const FuseBuf &b, const Lane &ln, int r, uint2 v)
{
    const uint64_t g = (uint64_t)r * b.W + (uint64_t)ln.c0;
    if (g + 8 <= b.n) {
        __stcs(reinterpret_cast<uint2 *>(b.out + g), v);
    } else {
        for (int i = 0; i < 8 && g + (uint64_t)i < b.n; ++i)
            b.out[g + i] = (uint8_t)((i < 4 ? v.x : v.y) >> (8 * (i & 3)));
    }
}

struct InvState {
    uint32_t x1[4], d1[4]; // level 1: x[2q-2] and d[q-1] (store-ready) of each word
    uint32_t x2[2], d2[2]; // level 2 (d2 store-ready)
    uint32_t x3, d3;
};

template <bool CHECK, bool PK, bool CIPH, int FL, bool BOX>
__device__ __forceinline__ void inv_iter(const FuseBuf &b, const Lane &ln, int t, uint32_t s8,
                                         uint32_t s4, bool store, bool whole, InvState &S, const Ks &K)
{
    const int W = (int)b.W, H = (int)b.H;
    const int F = FL ? FL : (int)b.F;
    const int W3 = W >> 3, H1 = H >> 1, H2 = H >> 2, H3 = H >> 3;
    const uint32_t llb = b.ll_final ? 0x00800080u : 0u; // LL_L - 128 -> LL_L
    const bool ciph = CIPH && b.cipher != 0; // LL_F is the private fragment, deciphered here

    // level 3: row t -> LL_2 rows 2t-1, 2t
    uint32_t z[2];
    if (F == 3) {
        const uint64_t e3 = (uint64_t)t * (uint64_t)W3 + (uint64_t)(ln.c0 >> 3);
        const uint32_t sh = 16u * (uint32_t)(e3 & 1ull);
        const uint32_t hl = (lds4(s4 + inv_l3<BOX>()) >> sh) & 0xffffu;
        const uint32_t lh = (lds4(s4 + inv_l3<BOX>() + 128) >> sh) & 0xffffu;
        const uint32_t hh = (lds4(s4 + inv_l3<BOX>() + 256) >> sh) & 0xffffu;
        uint32_t ll = (lds4(s4 + inv_l3<BOX>() + 384) >> sh) & 0xffffu;
        if (ciph)
            ll ^= lds2(ks_at(K, (uint64_t)t, e3));
        const uint32_t s = b.ll_final ? in16(ll | (hl << 16)) + 0x80u
                                      : (ll | (in16(hl << 16) & 0xffff0000u));
        const uint32_t d = in16(lh | (hh << 16));
        uint32_t xo, xe;
        col_inv<CHECK, false, false>(s, d, t == 0, t == H3, S.x3, S.d3, xo, xe);
        z[0] = unlift2(xo, ln.first, ln.last);
        z[1] = unlift2(xe, ln.first, ln.last);
    }

    // level 2: rows 2t-1+k -> LL_1 rows 4t-3+2k, 4t-2+2k
    uint32_t y[4][2];
    if (F >= 2) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int q2 = 2 * t - 1 + k;
            const uint32_t hl = q_i16(lds4(s4 + inv_x<BOX>() + 128 * (3 * k))); // store-ready
            const uint32_t lh = q_i16(lds4(s4 + inv_x<BOX>() + 128 * (3 * k + 1)));
            const uint32_t hh = q_i16(lds4(s4 + inv_x<BOX>() + 128 * (3 * k + 2)));
            uint32_t ll;
            if (F == 3) {
                ll = z[k];
            } else if (b.ll_final) {
                uint32_t c = lds4(s4 + inv_l2ll<BOX>() + 128 * k);
                if (ciph)
                    c ^= lds4(ks_at(K, (uint64_t)q2,
                                    (uint64_t)q2 * (uint64_t)(W >> 2) + (uint64_t)(ln.c0 >> 2)));
                ll = in16(c) + llb;
            } else {
                ll = lds4(s4 + inv_l2ll<BOX>() + 128 * k);
            }
            uint32_t oL, eL, oH, eH;
            col_inv<CHECK, false, true>(ll, lh, q2 == 0, q2 == H2, S.x2[0], S.d2[0], oL, eL);
            col_inv<CHECK, true, true>(hl, hh, q2 == 0, q2 == H2, S.x2[1], S.d2[1], oH, eH);
            unlift4(oL, oH, ln.sR, ln.sL, y[2 * k][0], y[2 * k][1]);
            unlift4(eL, eH, ln.sR, ln.sL, y[2 * k + 1][0], y[2 * k + 1][1]);
        }
    }

    // level 1: rows 4t-3+j -> level-0 rows 8t-7+2j, 8t-6+2j
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int q = 4 * t - 3 + j;
        const uint2 hl = lds8(s8 + l1_at<BOX>(j, 0));
        const uint2 lh = lds8(s8 + l1_at<BOX>(j, 1));
        const uint2 hh = lds8(s8 + l1_at<BOX>(j, 2));
        uint32_t s[4], d[4];
        if (F == 1) {
            uint2 ll = lds8(s8 + inv_x<BOX>() + 256 * j);
            if (ciph) {
                const uint2 k = lds8(ks_at(K, (uint64_t)q, (uint64_t)q * (uint64_t)(W >> 1) + (uint64_t)(ln.c0 >> 1)));
                ll.x ^= k.x;
                ll.y ^= k.y;
            }
            s[0] = b.ll_final ? in16(ll.x) + llb : ll.x;
            s[1] = b.ll_final ? in16(ll.y) + llb : ll.y;
        } else {
            s[0] = y[j][0];
            s[1] = y[j][1];
        }
        // the bands store-ready (one XOR each), LL biased
        s[2] = q_i16(hl.x);
        s[3] = q_i16(hl.y);
        d[0] = q_i16(lh.x);
        d[1] = q_i16(lh.y);
        d[2] = q_i16(hh.x);
        d[3] = q_i16(hh.y);
        uint32_t xo[4], xe[4];
#pragma unroll
        for (int m = 0; m < 2; ++m)
            col_inv<CHECK, false, true>(s[m], d[m], q == 0, q == H1, S.x1[m], S.d1[m], xo[m], xe[m]);
#pragma unroll
        for (int m = 2; m < 4; ++m)
            col_inv<CHECK, true, true>(s[m], d[m], q == 0, q == H1, S.x1[m], S.d1[m], xo[m], xe[m]);
        const int r = 2 * q - 1;
        if (PK) {
            // packed samples out (the LL_3 scratch a second pass hands down)
            const uint4 po = unlift8p(xo, ln.sR, ln.sL);
            const uint4 pe = unlift8p(xe, ln.sR, ln.sL);
            uint8_t *p = b.out + 2 * ((uint64_t)r * b.W + (uint64_t)ln.c0);
            pst16b(store && (!CHECK || (r >= 0 && r < H)), p, po);
            pst16b(store && (!CHECK || (r + 1 >= 0 && r + 1 < H)), p + 2ull * b.W, pe);
            continue;
        }
        const uint2 vo = unlift8(xo, ln.sR, ln.sL);
        const uint2 ve = unlift8(xe, ln.sR, ln.sL);
        if (!CHECK) { // both rows are whole rows of data (the caller sends others to CHECK)
            uint8_t *p = b.out + (uint64_t)r * b.W + (uint64_t)ln.c0;
            pst8b(store, p, vo);
            pst8b(store, p + b.W, ve);
        } else {
            if (store && (!CHECK || (r >= 0 && r < H)))
                store_bytes(b, ln, r, vo);
            if (store && (!CHECK || (r + 1 >= 0 && r + 1 < H)))
                store_bytes(b, ln, r + 1, ve);
        }
    }
}

// The warm-up iteration of an inverse unit away from the matrix's top and
// bottom (t >= 1, before the last two): only the column state of every level
// for the unit's first stored rows -- no row inverse of level 1, nothing
// stored.  Each level needs just the even sample x[2q] of its last
// coefficient row in the iteration, whose d[q-1] is the row before it,
// loaded in the same iteration (level 3: the d preloaded at the unit's
// start); level 2 hands down its row-inversed even row, LL_1 row 4t.
template <bool CIPH, int FL, bool BOX>
__device__ __forceinline__ void inv_warm(const FuseBuf &b, const Lane &ln, int t, uint32_t s8, uint32_t s4,
                                         InvState &S, const Ks &K)
{
    const int F = FL ? FL : (int)b.F;
    const uint32_t llb = b.ll_final ? 0x00800080u : 0u;
    const bool ciph = CIPH && b.cipher != 0;
    uint32_t y3[2] = {0u, 0u};
    uint32_t z1 = 0u;
    if (F == 3) { // level-3 row t
        const uint64_t e3 = (uint64_t)t * (uint64_t)(b.W >> 3) + (uint64_t)(ln.c0 >> 3);
        const uint32_t sh = 16u * (uint32_t)(e3 & 1ull);
        const uint32_t hl = (lds4(s4 + inv_l3<BOX>()) >> sh) & 0xffffu;
        const uint32_t lh = (lds4(s4 + inv_l3<BOX>() + 128) >> sh) & 0xffffu;
        const uint32_t hh = (lds4(s4 + inv_l3<BOX>() + 256) >> sh) & 0xffffu;
        uint32_t ll = (lds4(s4 + inv_l3<BOX>() + 384) >> sh) & 0xffffu;
        if (ciph)
            ll ^= lds2(ks_at(K, (uint64_t)t, e3));
        const uint32_t s = b.ll_final ? in16(ll | (hl << 16)) + 0x80u
                                      : (ll | (in16(hl << 16) & 0xffff0000u));
        const uint32_t d = in16(lh | (hh << 16));
        S.x3 = s - pq4(S.d3, d) + 0x20002000u; // undo Eq. 5.2
        S.d3 = d;
        z1 = unlift2(S.x3, ln.first, ln.last);
    }
    if (F >= 2) { // level-2 row 2t; d[-1] from row 2t-1
        const uint32_t lh0 = q_i16(lds4(s4 + inv_x<BOX>() + 128 * 1));
        const uint32_t hh0 = q_i16(lds4(s4 + inv_x<BOX>() + 128 * 2));
        const uint32_t hl1 = q_i16(lds4(s4 + inv_x<BOX>() + 128 * 3));
        const uint32_t lh1 = q_i16(lds4(s4 + inv_x<BOX>() + 128 * 4));
        const uint32_t hh1 = q_i16(lds4(s4 + inv_x<BOX>() + 128 * 5));
        uint32_t ll;
        if (F == 3) {
            ll = z1;
        } else if (b.ll_final) {
            uint32_t c = lds4(s4 + inv_l2ll<BOX>() + 128);
            if (ciph)
                c ^= lds4(ks_at(K, (uint64_t)(2 * t),
                                (uint64_t)(2 * t) * (uint64_t)(b.W >> 2) + (uint64_t)(ln.c0 >> 2)));
            ll = in16(c) + llb;
        } else {
            ll = lds4(s4 + inv_l2ll<BOX>() + 128);
        }
        const uint32_t eL = ll - pq4q(lh0, lh1) + 0x20002000u;
        const uint32_t eH = hl1 - pq4q(hh0, hh1) - 0x20002000u;
        S.x2[0] = eL;
        S.d2[0] = lh1;
        S.x2[1] = eH;
        S.d2[1] = hh1;
        unlift4(eL, eH, ln.sR, ln.sL, y3[0], y3[1]);
    }
    // level-1 row 4t (pair j = 3); d[-1] from row 4t-1 (j = 2)
    const uint2 lh2 = lds8(s8 + l1_at<BOX>(2, 1)), hh2 = lds8(s8 + l1_at<BOX>(2, 2));
    const uint2 hl3 = lds8(s8 + l1_at<BOX>(3, 0)), lh3 = lds8(s8 + l1_at<BOX>(3, 1)), hh3 = lds8(s8 + l1_at<BOX>(3, 2));
    uint32_t s[4];
    if (F == 1) {
        uint2 ll = lds8(s8 + inv_x<BOX>() + 256 * 3);
        if (ciph) {
            const uint2 k = lds8(ks_at(K, (uint64_t)(4 * t),
                                       (uint64_t)(4 * t) * (uint64_t)(b.W >> 1) + (uint64_t)(ln.c0 >> 1)));
            ll.x ^= k.x;
            ll.y ^= k.y;
        }
        s[0] = b.ll_final ? in16(ll.x) + llb : ll.x;
        s[1] = b.ll_final ? in16(ll.y) + llb : ll.y;
    } else {
        s[0] = y3[0];
        s[1] = y3[1];
    }
    s[2] = q_i16(hl3.x);
    s[3] = q_i16(hl3.y);
    const uint32_t d[4] = {q_i16(lh3.x), q_i16(lh3.y), q_i16(hh3.x), q_i16(hh3.y)};
    const uint32_t dp[4] = {q_i16(lh2.x), q_i16(lh2.y), q_i16(hh2.x), q_i16(hh2.y)};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t u = s[m] - pq4q(dp[m], d[m]);
        S.x1[m] = m < 2 ? u + 0x20002000u : u - 0x20002000u;
        S.d1[m] = d[m];
    }
}

// tm: the level-1 box loads (tm.map nullptr: none); tph: the phase bit of
// each stage barrier (kept across the warp's units).  False: a box load did
// not arrive within the spin limit (error word set); the warp stops.
template <bool PK, bool CIPH, int FL, bool BOX>
__device__ __forceinline__ bool inv_unit(const FuseBuf &b, uint32_t sx, uint32_t sy, uint32_t ring_lane8,
                                         uint32_t ring_lane4, int lane, uint32_t ks_ring, const uint32_t *tel,
                                         const AesKeys &keys, const Tma &tm, uint32_t &tph, int *err)
{
    const Lane ln = make_lane(b, sx, lane);
    const int F = FL ? FL : (int)b.F;
    const int t_begin = (int)(sy * b.seg_iters);
    const int t_end = min(t_begin + (int)b.seg_iters, (int)b.iters);
    // one iteration rebuilds the column state of every level above the
    // unit's first row, given d of level-3 row t_begin - 2 (three levels),
    // which is loaded here instead of running a second iteration
    const int t_first = max(t_begin - 1, 0);
    const int t_fast_end = (int)b.iters - 2;
    // LL rows iteration t reads: R t - R + 1 .. R t (the warm-up iteration
    // only the last of them)
    const int R = 8 >> F;
    Ks K = {};
    if (CIPH && b.cipher) {
        const bool warm = t_first >= 1 && t_first < t_fast_end && t_first < t_begin;
        K = ks_init(b, sx, lane, ks_ring, warm ? R * t_first : R * t_first - R + 1);
    }

#pragma unroll
    for (int k = 0; k < kInvDepth - 1; ++k)
        inv_issue<FL, BOX>(b, ln, t_first + k, t_end, ring_lane8, ring_lane4, tm);

    InvState S; // zeros, in each word's form
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        S.x1[k] = kB2;
        S.d1[k] = kQ;
    }
    S.x2[0] = S.x2[1] = S.x3 = S.d3 = kB2;
    S.d2[0] = S.d2[1] = kQ;
    if (F == 3 && t_begin >= 2 && ln.loads) {
        const uint64_t e = (uint64_t)(t_begin - 2) * (b.W >> 3) + ((uint32_t)ln.c0 >> 3);
        const uint32_t lh = __ldg(reinterpret_cast<const unsigned short *>(b.band[2][1]) + e);
        const uint32_t hh = __ldg(reinterpret_cast<const unsigned short *>(b.band[2][2]) + e);
        S.d3 = in16(lh | (hh << 16));
    }

    for (int t = t_first; t < t_end; ++t) {
        inv_issue<FL, BOX>(b, ln, t + kInvDepth - 1, t_end, ring_lane8, ring_lane4, tm);
        if (CIPH && b.cipher)
            ks_fill(K, (uint32_t)((uint64_t)(R * t + 1) - K.r_first) * K.nb, tel, keys, b.nonce, lane);
        cp_wait<kInvDepth - 1>();
        if (BOX && tm.map != nullptr && inv_inside<FL>(b, t)) {
            const uint32_t st = (uint32_t)(t % kInvDepth);
            const uint32_t bar = tm.bar + 8u * st, par = (tph >> st) & 1u;
            if (!box_wait(bar, par, kTmaSpinLimit)) {
                if (err != nullptr && tm.leader)
                    atomicCAS(err, 0, kErrTmaWait);
                cp_wait<0>();
                return false;
            }
            tph ^= 1u << st;
        }
        const uint32_t so = (uint32_t)(t % kInvDepth) * inv_stage<BOX>();
        const bool store = ln.own && t >= t_begin;
        const bool whole = 8 * t < (int)b.full_rows; // rows 8t-7 .. 8t hold only data
        // the unchecked iteration stores whole rows only; an iteration over
        // the last, partial row of the data takes the checked one
        if (t >= 1 && t < t_fast_end && (PK || whole || t < t_begin)) {
            if (t < t_begin)
                inv_warm<CIPH, FL, BOX>(b, ln, t, ring_lane8 + so, ring_lane4 + so, S, K);
            else
                inv_iter<false, PK, CIPH, FL, BOX>(b, ln, t, ring_lane8 + so, ring_lane4 + so, store, whole, S, K);
        } else {
            inv_iter<true, PK, CIPH, FL, BOX>(b, ln, t, ring_lane8 + so, ring_lane4 + so, store, whole, S, K);
        }
    }
    cp_wait<0>();
    return true;
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

// shared memory of a block: every warp's stage ring, then (launches that
// encipher) the lane-replicated AES table and every warp's keystream ring,
// then (launches with level-1 box loads, BOX) two stage barriers a warp
template <bool FWD, bool PK, bool BOX = false>
__host__ __device__ constexpr uint32_t stage_ring_bytes()
{
    return FWD ? fwd_depth<PK>() * fwd_stage<PK>() : kInvDepth * inv_stage<BOX>();
}

// CIPH: the launch enciphers some buffer's LL (table and keystream rings);
// the others leave that shared memory to L1
template <bool FWD, bool PK, bool CIPH>
__host__ __device__ constexpr size_t bar_offset(bool box)
{
    return (size_t)cta_warps<FWD, PK, CIPH>() * (box ? stage_ring_bytes<FWD, PK, true>() : stage_ring_bytes<FWD, PK>()) +
           (CIPH ? (size_t)kTableBytes + (size_t)cta_warps<FWD, PK, CIPH>() * kKsBytes : 0);
}
template <bool FWD, bool PK, bool CIPH>
__host__ __device__ constexpr size_t smem_bytes(bool box)
{
    return bar_offset<FWD, PK, CIPH>(box) + (box ? (size_t)16 * cta_warps<FWD, PK, CIPH>() : 0);
}
// the most a launch of the kernel takes (the attribute and the occupancy)
template <bool FWD, bool PK, bool CIPH>
__host__ __device__ constexpr size_t smem_max()
{
    return smem_bytes<FWD, PK, CIPH>(!FWD && !PK);
}

template <bool FWD, bool PK, bool CIPH>
__global__ void __launch_bounds__(32 * cta_warps<FWD, PK, CIPH>(), 16 / cta_warps<FWD, PK, CIPH>())
    fuse_kernel(const __grid_constant__ FuseWork w)
{
    extern __shared__ __align__(128) uint8_t smem[];
    // the next kernel (the CTR pass after a protect) may start its
    // data-independent part now; it waits for this grid before reading
    grid_release();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = cta_warps<FWD, PK, CIPH>();
    // the launch's level-1 box loads (a lone buffer's first inverse pass)
    // take the larger box-layout rings
    const bool box = !FWD && !PK && w.l1_tma != 0;
    // a launch whose shared memory is smaller than this layout records an
    // inconsistent descriptor (code 2) and does nothing
    uint32_t dyn_smem;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
    if (dyn_smem < (uint32_t)smem_bytes<FWD, PK, CIPH>(box)) {
        if (threadIdx.x == 0 && w.err != nullptr)
            atomicCAS(w.err, 0, 2);
        return;
    }
    const uint32_t rstride = box ? stage_ring_bytes<FWD, PK, true>() : stage_ring_bytes<FWD, PK>();
    const uint32_t kStages = (uint32_t)kWarps * rstride;
    uint32_t *te = reinterpret_cast<uint32_t *>(smem + kStages);
    if (CIPH) { // some buffer of the launch enciphers its LL here
        aes::build_table(te, w.aes_t0);
        __syncthreads();
    }
    const uint32_t ring = smem_addr(smem) + (uint32_t)warp * rstride;
    const uint32_t ks_ring = smem_addr(smem) + kStages + (uint32_t)kTableBytes + (uint32_t)warp * kKsBytes;
    const uint32_t *tel = te + lane;
    // the level-1 box loads of a lone buffer's first inverse pass: the warp's
    // two stage barriers after the rings (the boxes need a 128-byte aligned
    // ring; otherwise the lanes copy their own bytes)
    Tma tm = {};
    uint32_t tph = 0;
    if (box) {
        tm.bar = smem_addr(smem) + (uint32_t)bar_offset<FWD, PK, CIPH>(true) + 16u * (uint32_t)warp;
        tm.ring = ring;
        tm.leader = lane == 0;
        if (lane == 0) {
            mbar_init(tm.bar);
            mbar_init(tm.bar + 8);
            mbar_init_fence();
        }
        __syncwarp();
        if ((ring & 127u) == 0)
            tm.map = w.l1_map;
    }
    const uint64_t G = (uint64_t)gridDim.x * kWarps;
    const uint64_t u_end = w.unit_lo + w.total_units;
    const uint64_t u0 = w.spread ? (uint64_t)warp * gridDim.x + blockIdx.x : (uint64_t)blockIdx.x * kWarps + warp;
    for (uint64_t u = w.unit_lo + u0; u < u_end; u += G) {
        uint64_t local;
        const FuseBuf *bp = unit_buf(w, u, local);
        const FuseBuf b = *bp;
        const uint32_t sy = (uint32_t)(local / b.strips), sx = (uint32_t)(local % b.strips);
        // the inverse takes the levels a buffer fuses (1..3) as a template
        // argument, chosen once per unit: as a runtime value its tests and
        // the shuffles under them cost branches and reconvergence points in
        // every iteration.  The forward reads them from the descriptor
        // (FL = 0 reads b.F): specialised, it needed more registers and ran
        // slower
        if (FWD) {
            fwd_unit<PK, CIPH, 0>(b, sx, sy, ring + (PK ? 16u : 8u) * lane, lane, ks_ring, tel, w.keys);
        } else {
            const uint32_t r8 = ring + 8u * lane, r4 = ring + 4u * lane;
            // the box starts 4 level-1 columns left of lane 0's first (the
            // strip's halo lane), on a 16-byte boundary with one lane of halo
            Tma tu = tm;
            if (tu.map != nullptr) {
                const int c00 = (int)sx * 8 * (31 - (int)b.halo) - 8 * (int)b.halo;
                tu.x0 = (c00 >> 1) - 4;
                if ((tu.x0 & 7) != 0)
                    tu.map = nullptr;
            }
            bool ok = true;
            if (tu.map == nullptr) {
                if (b.F == 1)
                    inv_unit<PK, CIPH, 1, false>(b, sx, sy, r8, r4, lane, ks_ring, tel, w.keys, tu, tph, w.err);
                else if (b.F == 2)
                    inv_unit<PK, CIPH, 2, false>(b, sx, sy, r8, r4, lane, ks_ring, tel, w.keys, tu, tph, w.err);
                else
                    inv_unit<PK, CIPH, 3, false>(b, sx, sy, r8, r4, lane, ks_ring, tel, w.keys, tu, tph, w.err);
            } else if (!PK) {
                if (b.F == 1)
                    ok = inv_unit<PK, CIPH, 1, true>(b, sx, sy, r8, r4, lane, ks_ring, tel, w.keys, tu, tph, w.err);
                else if (b.F == 2)
                    ok = inv_unit<PK, CIPH, 2, true>(b, sx, sy, r8, r4, lane, ks_ring, tel, w.keys, tu, tph, w.err);
                else
                    ok = inv_unit<PK, CIPH, 3, true>(b, sx, sy, r8, r4, lane, ks_ring, tel, w.keys, tu, tph, w.err);
            }
            if (!ok)
                return;
        }
    }
}

template <bool FWD, bool PK, bool CIPH>
cudaError_t set_attr()
{
    static std::atomic<uint64_t> done{0};
    return smem_attr_once((const void *)fuse_kernel<FWD, PK, CIPH>, (int)smem_max<FWD, PK, CIPH>(), done);
}

template <bool FWD, bool PK, bool CIPH>
cudaError_t launch(const FuseWork &w, uint32_t grid, cudaStream_t stream)
{
    cudaError_t e = set_attr<FWD, PK, CIPH>();
    if (e != cudaSuccess)
        return e;
    // an ordinary launch (its loads go through L1, so it starts only once
    // the kernel before it has finished)
    fuse_kernel<FWD, PK, CIPH><<<grid, 32 * cta_warps<FWD, PK, CIPH>(), smem_bytes<FWD, PK, CIPH>(!FWD && !PK && w.l1_tma != 0), stream>>>(w);
    return cudaGetLastError();
}

template <bool FWD, bool PK>
cudaError_t launch(const FuseWork &w, uint32_t grid, cudaStream_t stream)
{
    return w.cipher ? launch<FWD, PK, true>(w, grid, stream) : launch<FWD, PK, false>(w, grid, stream);
}

// the CTAs of a launch an SM holds, and its warps per CTA
template <bool FWD, bool PK, bool CIPH>
cudaError_t shape(int *ctas_per_sm, int *warps_per_cta)
{
    cudaError_t e = set_attr<FWD, PK, CIPH>();
    if (e != cudaSuccess)
        return e;
    *warps_per_cta = cta_warps<FWD, PK, CIPH>();
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, (const void *)fuse_kernel<FWD, PK, CIPH>,
                                                         32 * cta_warps<FWD, PK, CIPH>(),
                                                         smem_max<FWD, PK, CIPH>());
}

} // namespace fuse
cudaError_t launch_fuse(bool fwd, bool packed, const FuseWork &w, uint32_t grid, cudaStream_t stream)
{
    if (fwd)
        return packed ? fuse::launch<true, true>(w, grid, stream) : fuse::launch<true, false>(w, grid, stream);
    return packed ? fuse::launch<false, true>(w, grid, stream) : fuse::launch<false, false>(w, grid, stream);
}

// A stage barrier armed for 16 bytes that no copy delivers, waited on with
// the box loads' bounded wait: lets a test check that such a wait that runs
// out sets the error word (7) and returns.
__global__ void box_stall_probe_kernel(uint32_t limit, int *err)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = fuse::smem_addr(&bar);
    if (threadIdx.x == 0) {
        fuse::mbar_init(a);
        fuse::mbar_init_fence();
        fuse::mbar_expect(a, 16);
    }
    __syncwarp();
    if (!fuse::box_wait(a, 0, limit) && threadIdx.x == 0)
        atomicCAS(err, 0, fuse::kErrTmaWait);
}

cudaError_t launch_box_stall_probe(uint32_t limit, int *err, cudaStream_t stream)
{
    box_stall_probe_kernel<<<1, 32, 0, stream>>>(limit, err);
    return cudaGetLastError();
}

cudaError_t fuse_shape(bool fwd, bool packed, bool cipher, int *ctas_per_sm, int *warps_per_cta)
{
    if (fwd) {
        if (packed)
            return cipher ? fuse::shape<true, true, true>(ctas_per_sm, warps_per_cta)
                          : fuse::shape<true, true, false>(ctas_per_sm, warps_per_cta);
        return cipher ? fuse::shape<true, false, true>(ctas_per_sm, warps_per_cta)
                      : fuse::shape<true, false, false>(ctas_per_sm, warps_per_cta);
    }
    if (packed)
        return cipher ? fuse::shape<false, true, true>(ctas_per_sm, warps_per_cta)
                      : fuse::shape<false, true, false>(ctas_per_sm, warps_per_cta);
    return cipher ? fuse::shape<false, false, true>(ctas_per_sm, warps_per_cta)
                  : fuse::shape<false, false, false>(ctas_per_sm, warps_per_cta);
}

} // namespace frag
