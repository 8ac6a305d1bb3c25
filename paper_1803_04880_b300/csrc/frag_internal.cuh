// frag_internal.cuh -- shared definitions of the CUDA library (kernels + C ABI).
//
// Nothing here is shared with the oracle: the AES tables are derived by this
// library's own host code (log/antilog tables over GF(2^8)), and the lifting
// is written for the in-place tile layout the kernels use.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda.h> // CUtensorMap (the type only; the library calls the runtime API)
#include <cuda_runtime.h>

namespace frag {

// One buffer of a tile-kernel launch (the allocation-free protect): `in` is
// read, priv / pub are written.
struct Job {
    const uint8_t *in;
    uint8_t *priv;
    uint8_t *pub;
    uint64_t n;       // bytes of the original buffer
    uint64_t nonce;   // AES-CTR nonce (high 64 bits of the counter block)
    uint32_t W;       // matrix width
    uint32_t H;       // padded rows (multiple of 2^L)
    uint32_t L;       // levels (1..kTileMaxLevels)
    uint32_t tile;    // owned tile side: tile_side(L)
    uint32_t tiles_x;
    uint32_t tiles_y;
};

// Job kinds of the dependency-ordered launch.
constexpr uint8_t kJobLevel = 0;  // one LeGall 5/3 level of one buffer
constexpr uint8_t kJobCipher = 1; // AES-128-CTR over the private fragment (LL_L)

// One job of one buffer in the dependency-ordered launch.
// Level job, forward: the level-(l-1) image `src` (bytes at l = 1, else packed
// LL pairs) gives the level-l bands and LL_l (packed pairs in scratch, or
// LL_L - 128 as int16 in the private fragment at the last level).  Inverse:
// LL_l (`ll_in`: packed pairs, or LL_L - 128 as int16 at the top level) and
// the bands give LL_{l-1} (packed pairs) or the bytes (`out`, l = 1).
// Cipher job: Ws x Hs is LL_L; forward XORs the keystream into `ll` in place,
// inverse writes `ll_in` XOR keystream to `out` (the plaintext scratch).
// Segment sy covers rows [sy * seg_pairs, (sy + 1) * seg_pairs) of the job's
// output (LL_l pair rows for a level job, LL_L rows for a cipher job); each
// segment has `strips` units (tiles of kTileStrips warp strips for a level
// job, kCipherBlocks AES blocks for a cipher job).
struct __align__(16) LevelJob {
    const uint8_t *src;
    uint8_t *hl, *lh, *hh; // band bases of level l
    uint8_t *ll;           // forward output
    const uint8_t *ll_in;  // inverse input
    uint8_t *out;          // inverse output
    uint64_t n;            // bytes of the buffer (level-1 source / output)
    uint64_t nonce;
    uint32_t Ws, Hs;       // level-(l-1) image (cipher job: LL_L)
    uint32_t strips;       // units per segment
    uint32_t wstrips;      // 240-column warp strips of the image (level job)
    uint32_t segs, seg_pairs;
    uint32_t done_off; // first completion counter of this job's segments
    int32_t dep;       // job whose output this job reads (-1: none)
    // the fields of job `dep` a unit's dependency check needs, copied here so
    // that the check reads one descriptor
    uint32_t dep_done_off, dep_segs, dep_units, dep_seg_pairs, dep_Ws;
    uint8_t dep_kind;
    uint8_t kind, src_bytes, final_level, top_level, out_bytes;
    uint8_t publish; // another job of the launch reads this one's output
    uint8_t bulk;    // bases and pitches allow whole-row bulk copies and vector stores
};
static_assert(sizeof(LevelJob) % 16 == 0, "job descriptors are copied in 16-byte pieces");

struct DagUnit {
    uint32_t job, sx, sy, pad; // 16 bytes: one vector load
};

// jobs of one buffer in one launch: up to 8 levels and the cipher units
constexpr int kMaxInlineJobs = 10;

struct DagWork {
    // one buffer: its jobs inline, units implied (wavefront rounds); many
    // buffers: a job array and an explicit dependency-ordered unit list
    LevelJob inline_jobs[kMaxInlineJobs];
    uint32_t n_inline;    // > 0: implicit units over inline_jobs
    uint32_t lag;         // rounds between consecutive levels (implicit mode)
    const LevelJob *jobs;
    const DagUnit *units; // dependency-ordered
    uint64_t total_units;
    unsigned long long *queue;
    unsigned *done;       // completed strips per (job, segment)
    const uint32_t *aes_tables;
    const uint32_t *round_keys;
    int *err;
    uint32_t spin_limit;
};

// A tile-kernel launch: its jobs, their tiles and the work queue.
struct Work {
    const Job *jobs;            // device array of jobs
    const uint64_t *tile_start; // exclusive prefix of tiles per job (njobs + 1 entries)
    uint32_t njobs;
    uint64_t total_tiles;
    unsigned long long *queue;  // device work-queue head (zero at launch)
    const uint32_t *aes_tables; // 4 x 256 T-table words + 256 S-box words, device
    const uint32_t *round_keys; // 44 big-endian round-key words, device
    int *err;                   // device error word
};

constexpr int kThreads = 512;
constexpr int kAesWords = 4 * 256 + 256;

// Byte offset of band b (0 = HL, 1 = LH, 2 = HH) of level l (1..L) inside the
// public fragment: levels are stored coarsest first, three bands each.
__host__ __device__ inline uint64_t band_offset(uint32_t H, uint32_t W, uint32_t L, uint32_t l,
                                                uint32_t b)
{
    uint64_t off = 0;
    for (uint32_t k = L; k > l; --k)
        off += 6ull * (uint64_t)(H >> k) * (uint64_t)(W >> k);
    return off + 2ull * b * (uint64_t)(H >> l) * (uint64_t)(W >> l);
}

// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes) on the current
// device once per kernel and device: `done` is that kernel's mask of devices
// already set (devices 0..63; any other is set on every call).  A launch of
// a small buffer is host-bound (about 1 us a call of the attribute set out
// of 15-20 us a call), so the launches skip the repeat.  The attribute lasts
// as long as the device's context: the library is not for use across a
// cudaDeviceReset (its device state, AES tables and pool are cached too).
inline cudaError_t smem_attr_once(const void *fn, int bytes, std::atomic<uint64_t> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit))
        return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit)
        done.fetch_or(bit, std::memory_order_release);
    return e;
}

// host helpers (frag_api.cu)
const uint32_t *host_aes_words();                             // kAesWords words
void host_expand_key(const uint8_t key[16], uint32_t rk[44]); // FIPS-197 key schedule

// streaming level kernels (stream_kernels.cu)
cudaError_t launch_dag(bool fwd, const DagWork &w, uint32_t grid, cudaStream_t stream);
cudaError_t dag_occupancy(bool fwd, int *blocks_per_sm);
cudaError_t launch_stall_probe(const unsigned *ctr, uint32_t spin_limit, int *err,
                               cudaStream_t stream);
// fused kernels (fused_kernels.cu): the box loads' bounded wait on a barrier
// nothing completes
cudaError_t launch_box_stall_probe(uint32_t limit, int *err, cudaStream_t stream);
constexpr int kStripCols = 240;          // level-(l-1) columns owned by one warp strip
constexpr uint32_t kTileStrips = 4;      // warp strips (consumer warps) of one tile unit
constexpr uint32_t kCipherBlocks = 512;  // AES blocks of one cipher unit

// AES-128-CTR in a launch of its own (cipher_kernels.cu), for buffers whose
// private fragment is large: levels <= kSeparateCipherMaxLevels
constexpr uint32_t kSeparateCipherMaxLevels = 2;

// AES-128 round keys as a launch carries them in its parameters: rounds 0..9
// as big-endian words, the same rotated left by 8 bits (the form the
// two-table rounds XOR in), and the last round's with its bytes in stream
// order
struct __align__(16) AesKeys {
    uint4 k[10];
    uint4 kr[10];
    uint4 last_le;
};

// blocks [first_block, first_block + nblocks) of one fragment of `bytes`
// bytes: out = in XOR keystream(nonce)
struct CtrChunk {
    const uint8_t *in;
    uint8_t *out;
    uint64_t nonce;
    uint64_t first_block;
    uint64_t bytes;
    uint64_t nblocks; // this chunk's blocks (a lone fragment: from first_block on)
};

// A launch over one fragment (`single`, blocks first_block .. + nblocks) or
// a list of fragments (one descriptor each, all of its blocks).  Work goes
// by warp turns of `turn_blocks` blocks (a multiple of 32, one block a lane
// a step); a list's turns are numbered fragment by fragment, turn_start[f]
// the first of fragment f (nfrags + 1 entries), so no turn spans two.
struct CtrWork {
    const CtrChunk *frags;      // device array (nullptr: one fragment, `single`)
    const uint64_t *turn_start; // device array, with frags
    uint64_t nfrags, nturns;
    CtrChunk single;
    uint64_t turn_blocks;
    const uint32_t *aes_tables; // table 0 is the first 256 words
    AesKeys keys;
};

cudaError_t launch_ctr(const CtrWork &w, uint32_t grid, cudaStream_t stream);
cudaError_t ctr_occupancy(int *blocks_per_sm);

// The bitsliced AES-128-CTR of a whole buffer (aes_bs.cuh): the comparator
// form measured against the table form above.  Warp chunks of 1,024 counter
// blocks; the sliced key schedule (11 x 128 words, 0x63 folded into rounds
// 1..10) travels in the kernel parameter.
struct BsCtrWork {
    const uint8_t *in;
    uint8_t *out;
    uint64_t bytes;
    uint64_t nonce;
    uint64_t nchunks; // chunks of 1,024 blocks
    uint32_t w[11][128];
};
cudaError_t launch_ctr_bs(const BsCtrWork &w, cudaStream_t stream);
constexpr uint32_t kCtrTurn = 32;       // blocks of a warp turn at least (one a lane)
constexpr int kCtrThreads = 1024;       // one CTA an SM (the two-table AES in shared memory)

// Programmatic dependent launch: a kernel launched with
// launch_after_previous() may start while the kernel before it on the stream
// is still running; it calls grid_wait() before touching anything that
// kernel writes, and grid_release() lets the next kernel start early in turn.
__device__ __forceinline__ void grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Fused levels (fused_kernels.cu): up to kFuseMaxLevels levels of a buffer
// in one pass down its rows, no intermediate LL in memory.  A unit is one
// warp strip (8 (31 - halo) level-0 columns) by seg_iters iterations of 8
// level-0 rows; forward iteration t reads rows 8t-1 .. 8t+6, inverse
// iteration t writes rows 8t-7 .. 8t.
constexpr uint32_t kFuseMaxLevels = 3;
// resident warps of a fused launch an SM holds, whatever its CTA shape
constexpr int kFuseWarpsPerSm = 16;


struct __align__(16) FuseBuf {
    const uint8_t *src;   // forward: the n bytes
    uint8_t *out;         // inverse: the n recovered bytes
    uint8_t *band[3][3];  // [l - 1][HL, LH, HH] of level l = 1..F (int16 LE)
    uint8_t *ll;          // LL_F: forward output, inverse input
    uint64_t n;
    uint64_t unit0;       // first unit of this buffer in the launch
    uint32_t W, H;        // level-0 matrix
    uint32_t F;           // levels fused (1..kFuseMaxLevels)
    uint32_t ll_final;    // LL_F is LL_L - 128 as int16 (else biased 16-bit scratch)
    uint32_t halo;        // lanes left of the owned ones
    uint32_t strips;      // warp strips across W
    uint32_t iters;       // iterations covering the matrix
    uint32_t seg_iters;   // iterations per unit
    uint32_t segs;        // units per strip
    uint32_t full_rows;   // leading rows made only of data bytes (n / W)
    uint32_t vec;         // block mode: every access may use its vector width
    uint32_t packed;      // block mode: the packed three fragments pk instead of int16 bands
    uint32_t keyed;       // packed: B and C protected by the keyed hashes (sha2.cuh)
    uint32_t cipher;      // LL_F is the private fragment, enciphered (protect) or
                          // deciphered (recover) with AES-128-CTR inside the fused kernel
    uint8_t *pk[3];       // packed: A (private, plaintext), B, C (pack_bits.cuh)
    uint64_t nonce;       // the buffer's nonce (AES-CTR counter blocks, hash input)
};
static_assert(sizeof(FuseBuf) % 16 == 0, "fused buffer descriptors are copied in 16-byte pieces");

struct FuseWork {
    const FuseBuf *bufs; // device array (nbufs > 1), ordered by unit0
    FuseBuf single;      // nbufs == 1
    uint32_t nbufs;
    uint32_t cipher;     // some buffer of the launch has `cipher` set
    uint64_t unit_lo;    // the launch runs units unit_lo .. unit_lo + total_units - 1
    uint64_t total_units;
    int *err;            // device error word (block mode, packed: 5 = a value outside its width;
                         // the inverse's TMA loads: 7 = a box that did not arrive in time)
    const uint32_t *key_words; // device: the 4 big-endian AES key words (keyed packed launches)
    const uint32_t *aes_t0;    // device: AES table 0 (256 words), when `cipher`
    AesKeys keys;              // round keys, when `cipher`
    // the inverse's first pass over a lone buffer (nbufs == 1): TMA maps of
    // the buffer's three level-1 bands (uint16, rows of W/2, boxes of 4 rows x
    // 136 values) when l1_tma != 0, else per-lane copies
    uint32_t l1_tma;
    // units to warps: 0 = unit u to warp u % W of CTA u / W (W warps a CTA:
    // a CTA's warps take neighbouring strips of the same rows, which a full
    // launch reads faster); 1 = unit u to CTA u % grid (a launch with fewer
    // units than warps then spreads them over every SM instead of filling a
    // few)
    uint32_t spread;
    CUtensorMap l1_map[3];
};

// packed: the samples are 16-bit values (v + 0x4000) instead of bytes --
// a second pass over LL_3 (levels 4 and 5) reads them (forward) or writes them
// (inverse)
cudaError_t launch_fuse(bool fwd, bool packed, const FuseWork &w, uint32_t grid, cudaStream_t stream);
// a fused launch's CTAs an SM holds and warps per CTA (cipher: some buffer
// of the launch enciphers its LL in the kernel); every shape keeps 16 warps
// an SM
cudaError_t fuse_shape(bool fwd, bool packed, bool cipher, int *ctas_per_sm, int *warps_per_cta);

// Block mode (block_kernels.cu): every 8 x 8 block transformed on its own.
// The same descriptors: strips = ceil(W / 256) (32 blocks a warp), iters =
// block rows, F = levels (<= 3), ll = LL_L - 128 (int16).
constexpr uint32_t kBlockSide = 8;
// packed: every buffer of the launch stores the packed three fragments;
// keyed: some of them are keyed (FuseBuf::keyed), w.key_words is set
cudaError_t launch_blocks(bool fwd, bool packed, bool keyed, const FuseWork &w, uint32_t grid,
                          cudaStream_t stream);
cudaError_t block_occupancy(bool fwd, bool packed, bool keyed, int *blocks_per_sm);

// the tile kernel (tile_kernels.cu, fast_tiles.cuh): 1 to 5 levels, one
// square tile of a buffer and its halo in shared memory per CTA
constexpr uint32_t kTileMaxLevels = 5;
__host__ __device__ constexpr uint32_t tile_side(uint32_t L) { return L <= 3 ? 256 : (L == 4 ? 240 : 160); }
size_t tile_smem_bytes(uint32_t L); // dynamic shared memory of an L-level job's tiles
cudaError_t launch_tiles(const Work &w, uint32_t grid, size_t smem, cudaStream_t stream);
cudaError_t tile_occupancy(size_t smem, int *blocks_per_sm);

} // namespace frag
