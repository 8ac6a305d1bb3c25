// frag_api.cu -- host implementation of the C ABI declared in include/frag.h.
//
// Plans and keys are small host objects; keys keep their expanded round keys
// resident on each device that uses them, and every device gets one copy of
// the AES tables and a device error word.  All work is enqueued on the
// caller's stream; nothing here falls back to the CPU.
#include "aes_tt.cuh"
#include "aes_bs.cuh"
#include "frag.h"
#include "frag_internal.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

using frag::Job;

struct frag_plan_s {
    uint32_t width;
    uint32_t levels;
    uint32_t seg_rows;    // streaming path: level-0 rows per unit (0: adaptive)
    uint32_t max_ctas;    // streaming path: grid cap (0: all resident CTAs)
    uint32_t path;        // frag_path: which kernels run the levels
    uint32_t block;       // block mode: side of the blocks (0: whole matrix)
    uint32_t packed;      // the thesis's packed three fragments (8 x 8 blocks, two levels)
    uint32_t keyed;       // packed: the public fragments protected by the keyed hashes
};

struct frag_key_s {
    uint32_t rk[44]; // big-endian round-key words
    std::mutex mu;
    std::map<int, uint32_t *> on_device;
};


namespace {

constexpr uint32_t kMaxLevels = 8;

thread_local char g_err[512] = "";

frag_status fail(frag_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

frag_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(FRAG_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// AES tables, derived with log / antilog tables of GF(2^8) (generator 3)
// ---------------------------------------------------------------------------
struct AesHost {
    uint8_t sbox[256];
    uint32_t words[frag::kAesWords]; // T0..T3 (256 each) then the S-box as words
};

uint8_t gf_double(uint8_t a) { return (uint8_t)((a << 1) ^ ((a >> 7) * 0x1b)); }

const AesHost &aes_host()
{
    static AesHost h;
    static std::once_flag once;
    std::call_once(once, [] {
        uint8_t alog[256], lg[256] = {0};
        uint8_t p = 1;
        for (int i = 0; i < 255; ++i) { // powers of the generator x + 1
            alog[i] = p;
            lg[p] = (uint8_t)i;
            p = (uint8_t)(p ^ gf_double(p));
        }
        for (int a = 0; a < 256; ++a) {
            const uint8_t inv = a == 0 ? 0 : alog[(255 - lg[a]) % 255];
            // affine map, bit by bit: b_i ^= b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i
            uint8_t s = 0;
            for (int i = 0; i < 8; ++i) {
                int bit = (inv >> i) & 1;
                for (int k = 4; k <= 7; ++k)
                    bit ^= (inv >> ((i + k) % 8)) & 1;
                bit ^= (0x63 >> i) & 1;
                s |= (uint8_t)(bit << i);
            }
            h.sbox[a] = s;
        }
        for (int a = 0; a < 256; ++a) {
            const uint32_t s = h.sbox[a], s2 = gf_double((uint8_t)s), s3 = s2 ^ s;
            const uint32_t t0 = (s2 << 24) | (s << 16) | (s << 8) | s3;
            for (int i = 0; i < 4; ++i)
                h.words[i * 256 + a] = i == 0 ? t0 : ((t0 >> (8 * i)) | (t0 << (32 - 8 * i)));
            h.words[4 * 256 + a] = s;
        }
    });
    return h;
}

void expand_key(const uint8_t key[16], uint32_t rk[44])
{
    const AesHost &h = aes_host();
    for (int i = 0; i < 4; ++i)
        rk[i] = ((uint32_t)key[4 * i] << 24) | ((uint32_t)key[4 * i + 1] << 16) |
                ((uint32_t)key[4 * i + 2] << 8) | key[4 * i + 3];
    uint8_t rcon = 1;
    for (int i = 4; i < 44; ++i) {
        uint32_t t = rk[i - 1];
        if (i % 4 == 0) {
            t = (t << 8) | (t >> 24); // RotWord
            t = ((uint32_t)h.sbox[t >> 24] << 24) | ((uint32_t)h.sbox[(t >> 16) & 255] << 16) |
                ((uint32_t)h.sbox[(t >> 8) & 255] << 8) | h.sbox[t & 255];
            t ^= (uint32_t)rcon << 24;
            rcon = gf_double(rcon);
        }
        rk[i] = rk[i - 4] ^ t;
    }
}

// ---------------------------------------------------------------------------
// Per-device state
// ---------------------------------------------------------------------------
struct DeviceState {
    bool ready = false;
    uint32_t *tables = nullptr;
    int *err = nullptr;
    cudaMemPool_t pool = nullptr; // the calls' stream-ordered scratch
    int sms = 0;
    size_t smem_set[2] = {0, 0};
    std::map<size_t, int> occ[2];
};

std::mutex g_mu;
std::vector<DeviceState> g_devices;
// scratch the pool keeps between calls (one wave of a batch)
constexpr uint64_t kPoolKeepBytes = 8ull << 30;

frag_status device_state(DeviceState **out, int *dev_out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_mu);
    if ((int)g_devices.size() <= dev)
        g_devices.resize(dev + 1);
    DeviceState &d = g_devices[dev];
    if (!d.ready) {
        if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute");
        if ((e = cudaMalloc(&d.tables, sizeof(uint32_t) * frag::kAesWords)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(aes tables)");
        if ((e = cudaMemcpy(d.tables, aes_host().words, sizeof(uint32_t) * frag::kAesWords,
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy(aes tables)");
        if ((e = cudaMalloc(&d.err, sizeof(int))) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(error word)");
        if ((e = cudaMemset(d.err, 0, sizeof(int))) != cudaSuccess)
            return cuda_fail(e, "cudaMemset(error word)");
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if ((e = cudaMemPoolCreate(&d.pool, &props)) != cudaSuccess)
            return cuda_fail(e, "cudaMemPoolCreate");
        uint64_t keep = kPoolKeepBytes;
        if ((e = cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
            return cuda_fail(e, "cudaMemPoolSetAttribute");
        d.ready = true;
    }
    *out = &d;
    if (dev_out)
        *dev_out = dev;
    return FRAG_OK;
}

// stream-ordered scratch from the library's pool on the current device:
// freed memory stays pooled up to kPoolKeepBytes, so a call does not map
// device pages again after the previous one released them
cudaError_t pool_malloc(void **p, size_t n, cudaStream_t s)
{
    DeviceState *d = nullptr;
    if (device_state(&d, nullptr) != FRAG_OK)
        return cudaErrorInitializationError;
    return cudaMallocFromPoolAsync(p, n, d->pool, s);
}

frag_status key_on_device(frag_key key, int dev, const uint32_t **out)
{
    std::lock_guard<std::mutex> lock(key->mu);
    auto it = key->on_device.find(dev);
    if (it != key->on_device.end()) {
        *out = it->second;
        return FRAG_OK;
    }
    uint32_t *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(key->rk));
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(round keys)");
    if ((e = cudaMemcpy(p, key->rk, sizeof(key->rk), cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(p);
        return cuda_fail(e, "cudaMemcpy(round keys)");
    }
    key->on_device[dev] = p;
    *out = p;
    return FRAG_OK;
}

frag_status check_plan(frag_plan plan)
{
    if (plan == nullptr)
        return fail(FRAG_EINVAL, "plan is NULL");
    return FRAG_OK;
}

// H: ceil(n / W) rounded up to a multiple of 2^L, or of the block side
uint64_t rows_for(uint64_t n, uint32_t W, uint32_t L, uint32_t block = 0)
{
    const uint64_t step = std::max<uint64_t>(1ull << L, block);
    const uint64_t rows = (n + W - 1) / W;
    return (rows + step - 1) / step * step;
}

// a tile-kernel job for the allocation-free call (its buffers set by the caller)
frag_status fill_job(frag_plan plan, uint64_t nonce, uint64_t n, Job &j)
{
    if (plan->block)
        return fail(FRAG_EUNSUPPORTED, "the allocation-free call does not take block plans");
    if (plan->levels > frag::kTileMaxLevels)
        return fail(FRAG_EUNSUPPORTED, "the allocation-free call takes at most %u levels, got %u",
                    frag::kTileMaxLevels, plan->levels);
    const uint64_t H = rows_for(n, plan->width, plan->levels);
    if (H > 0xFFFFFFFFull || H * (uint64_t)plan->width / plan->width != H)
        return fail(FRAG_EINVAL, "buffer of %llu bytes is too tall for width %u",
                    (unsigned long long)n, plan->width);
    std::memset(&j, 0, sizeof(j));
    j.n = n;
    j.nonce = nonce;
    j.W = plan->width;
    j.H = (uint32_t)H;
    j.L = plan->levels;
    j.tile = frag::tile_side(j.L);
    j.tiles_x = (j.W + j.tile - 1) / j.tile;
    j.tiles_y = (j.H + j.tile - 1) / j.tile;
    return FRAG_OK;
}

// ---------------------------------------------------------------------------
// Streaming path: all levels of all buffers of a call in one launch of the
// dependency-ordered kernel; LL between levels in scratch
// ---------------------------------------------------------------------------
using frag::DagUnit;
using frag::DagWork;
using frag::LevelJob;

constexpr uint64_t kScratchBudget = 8ull << 30; // scratch of one wave of a batch
constexpr uint32_t kMinLag = 3;                 // rounds between consecutive levels, at least
constexpr uint32_t kSpinLimit = 1u << 22;       // polls of a dependency before giving up

uint64_t align256(uint64_t v) { return (v + 255) / 256 * 256; }

uint64_t ll_bytes(uint32_t H, uint32_t W, uint32_t l) { return 2ull * (H >> l) * (uint64_t)(W >> l); }

// the packed three fragments of an H x W matrix of 8 x 8 blocks: A (40 bits a
// block), B (124 bits a block, every block row starting on a byte), C (480)
void packed_sizes(uint64_t H, uint32_t W, uint64_t *a, uint64_t *b, uint64_t *c, uint64_t *brow = nullptr)
{
    const uint64_t nbx = W / frag::kBlockSide, nby = H / frag::kBlockSide;
    const uint64_t row = (124 * nbx + 7) / 8;
    *a = 5 * nbx * nby;
    *b = nby * row;
    *c = 60 * nbx * nby;
    if (brow)
        *brow = row;
}

// first and last level whose LL band goes through scratch: the fused kernel
// keeps LL_1 .. LL_{F-1} on chip and hands LL_F over in scratch when levels
// remain above it
uint32_t scratch_lo(uint32_t F) { return F > 1 ? F : 1; }
// kc: the fused kernel deciphers LL_L as it loads it (no plaintext copy)
uint32_t scratch_hi(bool fwd, uint32_t L, bool kc = false) { return fwd || kc ? L - 1 : L; }

// scratch of one buffer: LL_lo .. LL_{L-1}, each in its own region (the jobs
// of one buffer run concurrently, so no region can be reused), and for the
// inverse the deciphered LL_L unless the fused kernel deciphers it on chip;
// off[l] is the offset of LL_l
uint64_t scratch_bytes(bool fwd, uint32_t H, uint32_t W, uint32_t L, uint32_t F, uint64_t *off,
                       bool kc = false)
{
    uint64_t total = 0;
    for (uint32_t l = scratch_lo(F); l <= scratch_hi(fwd, L, kc); ++l) {
        if (off)
            off[l] = total;
        total += align256(ll_bytes(H, W, l));
    }
    return total;
}

struct Buf {
    uint32_t W, L, H;
    uint32_t F;        // levels 1..F run in fused passes (0: none): F1 + F2
    uint32_t F1, F2;   // levels of the first pass (bytes) and the second (packed LL_3)
    uint32_t block;    // block mode (every level in the block kernel)
    uint32_t packed;   // block mode with the packed three fragments
    uint32_t keyed;    // packed: B and C protected by the keyed hashes
    uint32_t kc;       // the fused pass of level L enciphers / deciphers LL_L on chip
    uint32_t R0;       // level-0 rows per work segment
    uint32_t R0_plan;  // the plan's choice (0: adaptive)
    uint64_t n, nonce;
    const uint8_t *in;
    uint8_t *priv, *pub;
    const uint8_t *priv_in, *pub_in;
    uint8_t *out;
    uint8_t *scr[frag::kMaxInlineJobs + 1]; // scr[l]: LL_l (1 <= l < L; l = L: deciphered LL_L)
};

// Level-0 rows per work segment, the same at every level: a power of two
// >= 2^L, so every level has the same number of segments.  64 rows unless the
// first level would then have fewer than two units per resident CTA; then
// down to 16 (each segment re-reads three rows above it).  A plan may fix it.
uint32_t seg_rows0(uint32_t L, uint64_t l1_units_at_64, uint64_t resident_ctas,
                   uint32_t plan_rows = 0)
{
    if (plan_rows) {
        uint32_t r = plan_rows;
        while (r < (1u << L))
            r <<= 1;
        return r;
    }
    uint32_t r = 64;
    uint64_t u = l1_units_at_64;
    while (r > 16 && u < 2 * resident_ctas) {
        r >>= 1;
        u <<= 1;
    }
    while (r < (1u << L))
        r <<= 1;
    return r;
}

uint32_t warp_strips(uint32_t Ws) { return (Ws + frag::kStripCols - 1) / frag::kStripCols; }
uint32_t tiles(uint32_t Ws) { return (warp_strips(Ws) + frag::kTileStrips - 1) / frag::kTileStrips; }

uint64_t l1_units_at_64(const Buf &b) { return (uint64_t)tiles(b.W) * ((b.H + 63) / 64); }

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

LevelJob level_job(bool fwd, const Buf &b, uint32_t l, uint32_t R0)
{
    LevelJob j;
    std::memset(&j, 0, sizeof(j));
    j.Ws = b.W >> (l - 1);
    j.Hs = b.H >> (l - 1);
    uint8_t *pub = fwd ? b.pub : const_cast<uint8_t *>(b.pub_in);
    j.hl = pub + frag::band_offset(b.H, b.W, b.L, l, 0);
    j.lh = pub + frag::band_offset(b.H, b.W, b.L, l, 1);
    j.hh = pub + frag::band_offset(b.H, b.W, b.L, l, 2);
    if (fwd) {
        j.src = l == 1 ? b.in : b.scr[l - 1];
        j.src_bytes = l == 1;
        j.final_level = l == b.L;
        j.ll = l == b.L ? b.priv : b.scr[l];
    } else {
        j.top_level = l == b.L;
        j.ll_in = b.scr[l];
        j.out_bytes = l == 1;
        j.out = l == 1 ? b.out : b.scr[l - 1];
    }
    j.n = b.n;
    j.nonce = b.nonce;
    j.wstrips = warp_strips(j.Ws);
    j.strips = tiles(j.Ws);
    // whole rows move by 16-byte bulk copies and results leave as 8- or
    // 16-byte vector stores when every base and pitch allows it
    const uint32_t Wl = j.Ws / 2;
    if (fwd)
        j.bulk = aligned(j.src, 16) && (j.src_bytes ? j.Ws % 16 == 0 : j.Ws % 8 == 0) &&
                 Wl % 4 == 0 && aligned(j.hl, 8) && aligned(j.lh, 8) && aligned(j.hh, 8) &&
                 aligned(j.ll, 8);
    else
        j.bulk = Wl % 8 == 0 && aligned(j.ll_in, 16) && aligned(j.lh, 16) && aligned(j.hl, 16) &&
                 aligned(j.hh, 16) && aligned(j.out, j.out_bytes ? 8 : 16);
    j.seg_pairs = R0 >> l;
    j.segs = ((j.Hs / 2) + j.seg_pairs - 1) / j.seg_pairs;
    j.dep = -1;
    j.kind = frag::kJobLevel;
    return j;
}

// AES-128-CTR over the private fragment (LL_L): forward in place, inverse into
// the plaintext scratch; segments of R0 >> L rows of LL_L, as at the last level
LevelJob cipher_job(bool fwd, const Buf &b, uint32_t R0)
{
    LevelJob j;
    std::memset(&j, 0, sizeof(j));
    j.kind = frag::kJobCipher;
    j.Ws = b.W >> b.L;
    j.Hs = b.H >> b.L;
    if (fwd) {
        j.ll = b.priv;
    } else {
        j.ll_in = b.priv_in;
        j.out = b.scr[b.L];
    }
    j.n = b.n;
    j.nonce = b.nonce;
    j.seg_pairs = R0 >> b.L;
    j.segs = (j.Hs + j.seg_pairs - 1) / j.seg_pairs;
    // blocks starting in one segment's rows, at most
    const uint64_t blocks = (uint64_t)j.seg_pairs * 2ull * j.Ws / 16 + 2;
    j.strips = (uint32_t)((blocks + frag::kCipherBlocks - 1) / frag::kCipherBlocks);
    j.dep = -1;
    return j;
}

// a buffer whose private fragment is large (few levels), or whose levels all
// run in the fused kernel, is enciphered by the separate CTR launch rather
// than by cipher units inside the dependency-ordered launch
bool separate_cipher(const Buf &b)
{
    return b.L <= frag::kSeparateCipherMaxLevels || b.F == b.L;
}

uint32_t buffer_njobs(const Buf &b) { return (b.L - b.F) + (separate_cipher(b) ? 0 : 1); }

// the private fragment goes through the separate CTR launch: enciphered
// neither by the fused kernel nor by cipher units of the level kernel
bool ctr_pass(const Buf &b) { return separate_cipher(b) && !b.kc; }

// the jobs of one buffer in the dependency-ordered launch, in processing
// order (forward: levels F+1..L, then the cipher; inverse: the cipher, then
// levels L..F+1); each reads what the previous one writes

void buffer_jobs(bool fwd, const Buf &b, uint32_t first_job, uint32_t *counters,
                 std::vector<LevelJob> &jobs)
{
    const uint32_t R0 = b.R0;
    const bool sep = separate_cipher(b);
    const uint32_t njobs = buffer_njobs(b);
    for (uint32_t m = 0; m < njobs; ++m) {
        LevelJob j;
        if (fwd)
            j = m < b.L - b.F ? level_job(true, b, b.F + 1 + m, R0) : cipher_job(true, b, R0);
        else if (sep)
            j = level_job(false, b, b.L - m, R0);
        else
            j = m == 0 ? cipher_job(false, b, R0) : level_job(false, b, b.L + 1 - m, R0);
        j.dep = m ? (int32_t)(first_job + m - 1) : -1;
        j.publish = m + 1 < njobs; // the last job's output is read by nothing in the launch
        j.done_off = *counters;
        *counters += j.segs;
        if (m) {
            const LevelJob &p = jobs.back();
            j.dep_done_off = p.done_off;
            j.dep_segs = p.segs;
            j.dep_units = p.strips;
            j.dep_seg_pairs = p.seg_pairs;
            j.dep_Ws = p.Ws;
            j.dep_kind = p.kind;
        }
        jobs.push_back(j);
    }
}

// Rounds between consecutive levels of a lone buffer: a level's segment is
// queued only after about 1.5 times the resident warps' worth of earlier
// units, so it rarely waits for its producers (small images end up level by
// level; tall ones stream with the coarse levels behind the fine ones).
uint32_t buffer_lag(const std::vector<LevelJob> &jobs, uint32_t first_job, uint32_t njobs,
                    uint64_t resident_ctas)
{
    uint64_t per_round = 0;
    for (uint32_t m = 0; m < njobs; ++m)
        per_round += jobs[first_job + m].strips;
    const uint64_t lag = (3 * resident_ctas / 2 + per_round - 1) / std::max<uint64_t>(1, per_round);
    return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(kMinLag, lag), 1u << 24);
}

// units of a wave of buffers, job by job (job m of every buffer before job
// m + 1 of any), each job's units in row-segment order
void wave_units(const std::vector<LevelJob> &jobs, const std::vector<uint32_t> &first,
                const std::vector<uint32_t> &njobs, std::vector<DagUnit> &units)
{
    uint32_t maxj = 0;
    for (uint32_t k : njobs)
        maxj = std::max(maxj, k);
    for (uint32_t m = 0; m < maxj; ++m)
        for (size_t b = 0; b < first.size(); ++b) {
            if (m >= njobs[b])
                continue;
            const LevelJob &j = jobs[first[b] + m];
            for (uint32_t sy = 0; sy < j.segs; ++sy)
                for (uint32_t sx = 0; sx < j.strips; ++sx)
                    units.push_back(DagUnit{first[b] + m, sx, sy, 0});
        }
}

frag_status dag_grid(DeviceState &d, bool fwd, uint64_t units, uint32_t *grid)
{
    int occ = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = d.occ[fwd].find(7777);
        if (it != d.occ[fwd].end())
            occ = it->second;
    }
    if (occ == 0) {
        cudaError_t e = frag::dag_occupancy(fwd, &occ);
        if (e != cudaSuccess)
            return cuda_fail(e, "occupancy query");
        if (occ <= 0)
            occ = 1;
        std::lock_guard<std::mutex> lock(g_mu);
        d.occ[fwd][7777] = occ;
    }
    // one unit at a time per CTA
    *grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)d.sms * occ, units));
    return FRAG_OK;
}

// the private fragment of a buffer as one CTR fragment: protect enciphers it
// in place after the transform; recover deciphers it into the scratch the
// top level reads, before the transform
frag::CtrChunk ctr_fragment(bool fwd, const Buf &b)
{
    frag::CtrChunk c;
    std::memset(&c, 0, sizeof(c));
    c.in = fwd ? b.priv : b.priv_in;
    c.out = fwd ? b.priv : b.scr[b.L];
    c.nonce = b.nonce;
    c.bytes = ll_bytes(b.H, b.W, b.L);
    if (b.packed) { // A: 5 bytes a block (fits the LL_2 scratch, 8 bytes a block)
        uint64_t sb, sc;
        packed_sizes(b.H, b.W, &c.bytes, &sb, &sc);
    }
    c.nblocks = (c.bytes + 15) / 16;
    return c;
}

// A CTR launch over a fragment list (frags, device; turn_start, device,
// nfrags + 1 entries; nturns warp turns of turn_blocks blocks) or over one
// fragment (single: blocks first_block .. + nblocks, turns sized here).
struct CtrList {
    const frag::CtrChunk *frags = nullptr;
    const uint64_t *turn_start = nullptr;
    uint64_t nfrags = 0, nturns = 0, turn_blocks = 0;
};

frag_status ctr_launch(DeviceState &d, const frag::AesKeys &keys, const CtrList *list,
                       const frag::CtrChunk *single, cudaStream_t s)
{
    int occ = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = d.occ[0].find(8888);
        if (it != d.occ[0].end())
            occ = it->second;
    }
    if (occ == 0) {
        cudaError_t e = frag::ctr_occupancy(&occ);
        if (e != cudaSuccess)
            return cuda_fail(e, "occupancy query");
        occ = std::max(occ, 1);
        std::lock_guard<std::mutex> lock(g_mu);
        d.occ[0][8888] = occ;
    }
    frag::CtrWork w;
    std::memset(&w, 0, sizeof(w));
    w.aes_tables = d.tables;
    w.keys = keys;
    const uint64_t slots = (uint64_t)d.sms * occ;
    uint64_t work = 0;
    if (list) {
        w.frags = list->frags;
        w.turn_start = list->turn_start;
        w.nfrags = list->nfrags;
        w.nturns = list->nturns;
        w.turn_blocks = list->turn_blocks;
        work = list->nturns;
    } else {
        // a lone fragment spread over every resident warp, whole warp turns
        w.single = *single;
        const uint64_t warps = slots * (frag::kCtrThreads / 32);
        const uint64_t per = (single->nblocks + warps - 1) / warps;
        w.turn_blocks = std::max<uint64_t>(frag::kCtrTurn, (per + 31) / 32 * 32);
        work = (single->nblocks + w.turn_blocks - 1) / w.turn_blocks;
    }
    if (work == 0)
        return FRAG_OK;
    // every SM takes a share of the turns (the kernel interleaves them over
    // its CTAs), even when the turns would fill fewer full CTAs
    const uint32_t grid = (uint32_t)std::min<uint64_t>(slots, work);
    cudaError_t e = frag::launch_ctr(w, grid, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "cipher launch");
    return FRAG_OK;
}

// ---------------------------------------------------------------------------
// Fused path: levels 1..F of a buffer in one pass down its rows
// ---------------------------------------------------------------------------
constexpr uint32_t kFuseMinSegIters = 8; // iterations per unit at least (adaptive choice)
#ifndef FRAG_FUSE_TINY_SEG
#define FRAG_FUSE_TINY_SEG 1
#endif
constexpr uint32_t kFuseTinySegIters = FRAG_FUSE_TINY_SEG;

// levels a fused pass over levels lo+1 .. lo+F can take (0: none): its
// input width (W >> lo) a multiple of 8 and every band and the LL output it
// writes with vector stores aligned
uint32_t pass_levels(bool fwd, const Buf &b, uint32_t lo)
{
    if ((b.W >> lo) % 8 != 0 || b.L <= lo)
        return 0;
    const uint32_t F = std::min(b.L - lo, frag::kFuseMaxLevels);
    const uint8_t *pub = fwd ? b.pub : b.pub_in;
    for (uint32_t l = 1; l <= F; ++l)
        for (uint32_t k = 0; k < 3; ++k)
            if (!aligned(pub + frag::band_offset(b.H, b.W, b.L, lo + l, k), l == 1 ? 8 : 4))
                return 0;
    if (fwd && lo + F == b.L && !aligned(b.priv, F == 1 ? 8 : 4))
        return 0; // LL_L goes straight to the private fragment
    return F;
}

// how buffer b splits over the fused passes: the first (bytes in / out)
// takes levels 1 .. F1 (up to 3), a second over the packed LL_3 scratch
// levels 4 .. 3 + F2 (up to level 6); the level kernel takes the rest
// (levels 7 and 8, or every level of a buffer neither pass takes)
void fused_split(bool fwd, Buf &b, uint32_t path)
{
    b.F1 = b.F2 = 0;
    b.kc = 0;
    if (b.block)
        b.F1 = b.L; // every level in the block kernel (no scratch but LL_L on recover)
    else if (path != FRAG_PATH_LEVELS && (fwd ? aligned(b.in, 8) : aligned(b.out, 8)))
        b.F1 = pass_levels(fwd, b, 0);
    if (!b.block && b.F1 == frag::kFuseMaxLevels)
        b.F2 = pass_levels(fwd, b, b.F1);
    b.F = b.F1 + b.F2;
    // on request, the pass that reaches level L enciphers LL_L before
    // storing it, or deciphers it right after loading it from the private
    // fragment (whose words it then reads with the same vector width as the
    // bands)
    if (!b.block && b.F == b.L && path == FRAG_PATH_FUSED_CIPHER) {
        const uint32_t last = b.F2 ? b.F2 : b.F1;
        b.kc = aligned(fwd ? (const void *)b.priv : (const void *)b.priv_in, last == 1 ? 8 : 4);
    }
}

// cuTensorMapEncodeTiled from the driver (looked up once; nullptr if the
// driver has none)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// The TMA maps of the three level-1 bands an inverse first pass over f reads
// (2D uint16: W/2 values a row, H/2 rows; boxes of 4 rows x 136 values, zeros
// outside) into w, with w.l1_tma = 1; left off (per-lane copies) unless the
// pass fuses one or two levels, the row pitch and the band bases are 16-byte
// aligned and a band is at least a box wide and tall.  The 256 MiB buffer at
// width 8192: 2 levels 157.5 -> 150.0 us a recover with the boxes, 3 levels
// 164.8 -> 167.2 us (so three-level passes keep the per-lane copies)
void set_l1_maps(frag::FuseWork &w, const frag::FuseBuf &f)
{
    w.l1_tma = 0;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    const uint64_t W1 = f.W >> 1, H1 = f.H >> 1;
    if (enc == nullptr || f.F < 1 || f.F > 2 || (f.W % 16) != 0 || W1 < 136 || H1 < 4)
        return;
    for (int k = 0; k < 3; ++k)
        if (!aligned(f.band[0][k], 16))
            return;
    const cuuint64_t dims[2] = {W1, H1};
    const cuuint64_t strides[1] = {2 * W1};
    const cuuint32_t box[2] = {136, 4};
    const cuuint32_t estr[2] = {1, 1};
    for (int k = 0; k < 3; ++k)
        if (enc(&w.l1_map[k], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, f.band[0][k], dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
    w.l1_tma = 1;
}

// descriptor of buffer b for a fused pass (schedule fields left 0): pass 1
// works on the bytes, pass 2 on the packed LL_{F1} scratch (levels
// F1+1 .. F1+F2)
frag::FuseBuf fuse_buf(bool fwd, const Buf &b, int pass = 1)
{
    frag::FuseBuf f;
    std::memset(&f, 0, sizeof(f));
    const uint32_t lo = pass == 1 ? 0 : b.F1, F = pass == 1 ? b.F1 : b.F2, top = lo + F;
    uint8_t *pub = fwd ? b.pub : const_cast<uint8_t *>(b.pub_in);
    for (uint32_t l = 1; l <= F; ++l)
        for (uint32_t k = 0; k < 3; ++k)
            f.band[l - 1][k] = pub + frag::band_offset(b.H, b.W, b.L, lo + l, k);
    // LL_top: the private fragment (protect, last level; recover, last level
    // deciphered on chip), the deciphered copy (recover, last level, after
    // the CTR launch) or the scratch the levels above read / write
    f.cipher = b.kc && top == b.L;
    f.nonce = b.nonce;
    f.ll = (fwd && top == b.L) ? b.priv : f.cipher ? const_cast<uint8_t *>(b.priv_in) : b.scr[top];
    f.ll_final = top == b.L;
    f.W = b.W >> lo;
    f.H = b.H >> lo;
    if (pass == 1) {
        f.src = b.in;
        f.out = b.out;
        f.n = b.n;
        f.full_rows = (uint32_t)std::min<uint64_t>(b.n / b.W, b.H);
    } else {
        f.src = b.scr[lo];
        f.out = b.scr[lo];
        f.n = (uint64_t)f.H * f.W;
        f.full_rows = f.H;
    }
    f.F = F;
    f.halo = (fwd && F == 3) ? 2 : 1;
    f.strips = (f.W + 8 * (31 - f.halo) - 1) / (8 * (31 - f.halo));
    f.iters = fwd ? f.H / 8 + 1 : (f.H + 6) / 8 + 1;
    return f;
}

// units of each buffer: one segment height for a launch, chosen so that the
// units about fill the resident warps once (or from the plan's seg_rows);
// returns the launch's units
// a batch's launch: units of at most this many iterations, so that the
// warps of many buffers of very different heights share the work evenly
// (10,000 buffers of 4 KiB .. 64 MiB: one unit a strip took 71 ms to
// protect, units of 32 iterations 60.5 ms, of 16 or 8 iterations 62.5 ms)
constexpr uint32_t kFuseBatchSegIters = 32;

uint64_t fuse_schedule(frag::FuseBuf *f, size_t nbufs, uint64_t warps, uint32_t plan_rows, bool batch = false,
                       bool tiny = true)
{
    uint32_t seg = 0;
    if (plan_rows) {
        seg = std::max(1u, plan_rows / 8);
    } else {
        uint64_t work = 0;
        for (size_t i = 0; i < nbufs; ++i)
            work += (uint64_t)f[i].strips * f[i].iters;
        uint64_t per = (work + warps - 1) / std::max<uint64_t>(1, warps);
        if (batch && nbufs > 1) // one buffer's units are all alike
            per = std::min<uint64_t>(per, kFuseBatchSegIters);
        // a launch too small to give each resident warp one iteration is
        // latency-bound: shorter units shorten its longest chain (the
        // 256 x 256 buffer at one level: units of 8 / 4 / 2 / 1 iterations,
        // protect p50 17.5 / 15.5 / 12.9 / 11.2 us); `tiny` false keeps the
        // longer units (a band of the host forms, which overlaps copies)
        const uint32_t lo = tiny && work <= warps ? kFuseTinySegIters : kFuseMinSegIters;
        seg = (uint32_t)std::min<uint64_t>(1u << 20, std::max<uint64_t>(lo, per));
    }
    uint64_t units = 0;
    for (size_t i = 0; i < nbufs; ++i) {
        f[i].seg_iters = seg;
        f[i].segs = (f[i].iters + seg - 1) / seg;
        f[i].unit0 = units;
        units += (uint64_t)f[i].strips * f[i].segs;
    }
    return units;
}

// shape of a fused launch (CTAs an SM holds, warps per CTA), cached per device
frag_status fuse_shape(DeviceState &d, bool fwd, bool packed, bool cipher, int *ctas, int *warps)
{
    const size_t tag = 9990 + (packed ? 2 : 0) + (cipher ? 1 : 0);
    int v = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = d.occ[fwd].find(tag);
        if (it != d.occ[fwd].end())
            v = it->second;
    }
    if (v == 0) {
        int occ = 0, wpc = 0;
        cudaError_t e = frag::fuse_shape(fwd, packed, cipher, &occ, &wpc);
        if (e != cudaSuccess)
            return cuda_fail(e, "occupancy query");
        v = std::max(occ, 1) * 1000 + wpc;
        std::lock_guard<std::mutex> lock(g_mu);
        d.occ[fwd][tag] = v;
    }
    *ctas = v / 1000;
    *warps = v % 1000;
    return FRAG_OK;
}

// warps a fused launch keeps resident on the device; a plan's grid cap
// counts them in groups of 4 (the level kernel's consumer warps per CTA)
frag_status fuse_slots(DeviceState &d, bool fwd, bool packed, uint32_t max_ctas, uint64_t *slots)
{
    int ctas = 0, wpc = 0;
    frag_status st = fuse_shape(d, fwd, packed, false, &ctas, &wpc);
    if (st != FRAG_OK)
        return st;
    *slots = (uint64_t)d.sms * ctas * wpc;
    if (max_ctas)
        *slots = std::min<uint64_t>(*slots, 4ull * max_ctas);
    return FRAG_OK;
}

// slots: the resident warps fuse_slots gave
frag_status fuse_launch(DeviceState &d, bool fwd, bool packed, frag::FuseWork &w, uint64_t slots,
                        cudaStream_t s)
{
    if (w.total_units == 0)
        return FRAG_OK;
    w.aes_t0 = d.tables; // table 0: the first 256 words
    int ctas = 0, wpc = 0;
    frag_status st = fuse_shape(d, fwd, packed, w.cipher != 0, &ctas, &wpc);
    if (st != FRAG_OK)
        return st;
    const uint64_t cap = std::min<uint64_t>((uint64_t)d.sms * ctas, (slots + wpc - 1) / wpc);
    // at most half as many units as the launch's warps: one CTA a unit
    // first, spread over the SMs (8 / 16 MiB at 3 levels, protect 30.7 /
    // 31.6 -> 21.5 / 24.6 us); a fuller launch keeps a CTA's warps on
    // neighbouring strips of the same rows (spread, 32 / 48 / 64 MiB lost
    // 1 us a protect, the 256 MiB buffer's went from 154.8 to 171.7 us)
    w.spread = 2 * w.total_units <= cap * (uint64_t)wpc;
    const uint64_t need = w.spread ? w.total_units : (w.total_units + wpc - 1) / wpc;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min(cap, need));
    cudaError_t e = frag::launch_fuse(fwd, packed, w, grid, s);
    if (e != cudaSuccess)
        return cuda_fail(e, fwd ? "fused protect launch" : "fused recover launch");
    return FRAG_OK;
}

// ---------------------------------------------------------------------------
// Block mode: every 8 x 8 block on its own, one lane a block
// ---------------------------------------------------------------------------
frag::FuseBuf block_buf(bool fwd, const Buf &b)
{
    frag::FuseBuf f = fuse_buf(fwd, b);
    f.halo = 0;
    f.strips = (b.W + 255) / 256; // 32 blocks of 8 columns a warp
    f.iters = b.H / frag::kBlockSide;
    f.seg_iters = 1;
    f.segs = f.iters;
    f.ll_final = 1;
    bool v = fwd ? aligned(b.in, 8) : aligned(b.out, 8);
    for (uint32_t l = 1; l <= b.L; ++l)
        for (uint32_t k = 0; k < 3; ++k)
            v = v && aligned(f.band[l - 1][k], l == 1 ? 8 : (l == 2 ? 4 : 2));
    v = v && aligned(f.ll, b.L == 1 ? 8 : (b.L == 2 ? 4 : 2));
    f.vec = v;
    return f;
}

// a packed buffer's descriptor: the block kernel writes (reads) the bit
// records; A is the private fragment (protect) or its deciphered copy in the
// LL_2 scratch (recover), the public fragment is B then C
frag::FuseBuf packed_buf(bool fwd, const Buf &b)
{
    frag::FuseBuf f = block_buf(fwd, b);
    uint64_t sa, sb, sc;
    packed_sizes(b.H, b.W, &sa, &sb, &sc);
    f.packed = 1;
    f.keyed = b.keyed;
    f.nonce = b.nonce;
    f.pk[0] = fwd ? b.priv : b.scr[b.L];
    f.pk[1] = fwd ? b.pub : const_cast<uint8_t *>(b.pub_in);
    f.pk[2] = f.pk[1] + sb;
    return f;
}

uint64_t block_units(frag::FuseBuf *f, size_t nbufs)
{
    uint64_t units = 0;
    for (size_t i = 0; i < nbufs; ++i) {
        f[i].unit0 = units;
        units += (uint64_t)f[i].strips * f[i].segs;
    }
    return units;
}

// keyed: some packed buffer is keyed; rk (device) holds the key's words
frag_status block_launch(DeviceState &d, bool fwd, frag::FuseWork &w, cudaStream_t s, bool packed = false,
                         bool keyed = false, const uint32_t *rk = nullptr)
{
    if (w.total_units == 0)
        return FRAG_OK;
    int occ = 0;
    const size_t tag = packed ? (keyed ? 6668 : 6667) : 6666;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = d.occ[fwd].find(tag);
        if (it != d.occ[fwd].end())
            occ = it->second;
    }
    if (occ == 0) {
        cudaError_t e = frag::block_occupancy(fwd, packed, keyed, &occ);
        if (e != cudaSuccess)
            return cuda_fail(e, "occupancy query");
        occ = std::max(occ, 1);
        std::lock_guard<std::mutex> lock(g_mu);
        d.occ[fwd][tag] = occ;
    }
    w.err = d.err;
    w.key_words = rk;
    const uint64_t need = (w.total_units + 3) / 4; // 4 warps a CTA
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)d.sms * occ, need));
    cudaError_t e = frag::launch_blocks(fwd, packed, keyed && rk != nullptr, w, grid, s);
    if (e != cudaSuccess)
        return cuda_fail(e, fwd ? "block protect launch" : "block recover launch");
    return FRAG_OK;
}

// One buffer in the thesis's packed storage: protect runs the block kernel,
// which writes the three fragments' bit records, then enciphers the private
// one in place; recover deciphers it into scratch and runs the block inverse
// on the records
frag_status run_packed(bool fwd, frag_plan plan, frag_key key, Buf b, cudaStream_t s)
{
    DeviceState *d = nullptr;
    int dev = 0;
    frag_status st = device_state(&d, &dev);
    if (st != FRAG_OK)
        return st;
    const uint32_t *rk = nullptr;
    if ((st = key_on_device(key, dev, &rk)) != FRAG_OK)
        return st;
    uint64_t sa = 0, sb = 0, sc = 0;
    packed_sizes(b.H, b.W, &sa, &sb, &sc);
    uint8_t *plainA = nullptr; // recover: the deciphered private fragment
    if (!fwd) {
        cudaError_t e = pool_malloc((void **)&plainA, align256(sa), s);
        if (e != cudaSuccess)
            return cuda_fail(e, "pool_malloc(private fragment)");
    }
    fused_split(fwd, b, plan->path);
    frag::FuseWork w;
    std::memset(&w, 0, sizeof(w));
    w.single = block_buf(fwd, b);
    w.single.packed = 1;
    w.single.keyed = b.keyed;
    w.single.nonce = b.nonce;
    w.single.pk[0] = fwd ? b.priv : plainA;
    w.single.pk[1] = fwd ? b.pub : const_cast<uint8_t *>(b.pub_in);
    w.single.pk[2] = w.single.pk[1] + sb;
    w.nbufs = 1;
    w.total_units = block_units(&w.single, 1);
    frag::CtrChunk c;
    std::memset(&c, 0, sizeof(c));
    c.in = fwd ? b.priv : b.priv_in;
    c.out = fwd ? b.priv : plainA;
    c.nonce = b.nonce;
    c.bytes = sa;
    c.nblocks = (sa + 15) / 16;
    if (fwd) {
        st = block_launch(*d, true, w, s, true, b.keyed != 0, rk);
        if (st == FRAG_OK)
            st = ctr_launch(*d, frag::aes::keys_from_words(key->rk), nullptr, &c, s);
    } else {
        st = ctr_launch(*d, frag::aes::keys_from_words(key->rk), nullptr, &c, s);
        if (st == FRAG_OK)
            st = block_launch(*d, false, w, s, true, b.keyed != 0, rk);
        cudaFreeAsync(plainA, s);
    }
    return st;
}

// One buffer: protect runs the fused levels, then the dependency-ordered
// launch for the levels above them (and the cipher units), then the CTR
// launch; recover runs them in the reverse order.
frag_status run_single(bool fwd, frag_plan plan, frag_key key, Buf b, cudaStream_t s)
{
    if (plan->packed)
        return run_packed(fwd, plan, key, b, s);
    DeviceState *d = nullptr;
    int dev = 0;
    frag_status st = device_state(&d, &dev);
    if (st != FRAG_OK)
        return st;
    const uint32_t *rk = nullptr;
    if ((st = key_on_device(key, dev, &rk)) != FRAG_OK)
        return st;
    fused_split(fwd, b, plan->path);
    if (b.block) {
        // block mode: the block kernel and the CTR pass (recover deciphers
        // LL_L into scratch first)
        uint64_t off[frag::kMaxInlineJobs + 1] = {0};
        const uint64_t sb = scratch_bytes(fwd, b.H, b.W, b.L, b.F1, off);
        uint8_t *mem = nullptr;
        if (sb) {
            cudaError_t e = pool_malloc((void **)&mem, sb, s);
            if (e != cudaSuccess)
                return cuda_fail(e, "pool_malloc(level scratch)");
            b.scr[b.L] = mem + off[b.L];
        }
        frag::FuseWork w;
        std::memset(&w, 0, sizeof(w));
        w.single = block_buf(fwd, b);
        w.nbufs = 1;
        w.total_units = block_units(&w.single, 1);
        const frag::CtrChunk frag_chunk = ctr_fragment(fwd, b);
        if (!fwd)
            st = ctr_launch(*d, frag::aes::keys_from_words(key->rk), nullptr, &frag_chunk, s);
        if (st == FRAG_OK)
            st = block_launch(*d, fwd, w, s);
        if (st == FRAG_OK && fwd)
            st = ctr_launch(*d, frag::aes::keys_from_words(key->rk), nullptr, &frag_chunk, s);
        if (mem)
            cudaFreeAsync(mem, s);
        return st;
    }
    const uint32_t njobs = buffer_njobs(b);
    if (njobs > (uint32_t)frag::kMaxInlineJobs)
        return fail(FRAG_EUNSUPPORTED, "more than %d levels", frag::kMaxInlineJobs - 1);
    // one stream-ordered allocation: [scratch][counters][queue head]
    uint64_t off[frag::kMaxInlineJobs + 1] = {0};
    const uint64_t sb = align256(scratch_bytes(fwd, b.H, b.W, b.L, b.F1, off, b.kc));
    uint32_t grid = 0;
    uint64_t cb = 0;
    if (njobs) {
        if ((st = dag_grid(*d, fwd, ~0ull, &grid)) != FRAG_OK)
            return st;
        if (plan->max_ctas)
            grid = std::min(grid, plan->max_ctas);
        b.R0 = seg_rows0(b.L, l1_units_at_64(b), grid, plan->seg_rows);
        const uint32_t NS = (b.H + b.R0 - 1) / b.R0;
        cb = align256(4ull * NS * njobs);
    }
    uint8_t *mem = nullptr;
    if (sb + cb) {
        cudaError_t e = pool_malloc((void **)&mem, sb + cb + 256, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "pool_malloc(level scratch)");
    }
    for (uint32_t l = scratch_lo(b.F1); l <= scratch_hi(fwd, b.L, b.kc); ++l)
        b.scr[l] = mem + off[l];
    // the fused passes: [0] over the bytes, [1] over the packed LL_3
    frag::FuseWork fw[2];
    std::memset(fw, 0, sizeof(fw));
    uint64_t fslots[2] = {0, 0};
    for (int p = 0; p < 2; ++p) {
        if ((p == 0 ? b.F1 : b.F2) == 0)
            continue;
        if ((st = fuse_slots(*d, fwd, p == 1, plan->max_ctas, &fslots[p])) != FRAG_OK) {
            cudaFreeAsync(mem, s);
            return st;
        }
        fw[p].single = fuse_buf(fwd, b, p + 1);
        fw[p].nbufs = 1;
        fw[p].total_units = fuse_schedule(&fw[p].single, 1, fslots[p], plan->seg_rows);
        if (fw[p].single.cipher) {
            fw[p].cipher = 1;
            fw[p].keys = frag::aes::keys_from_words(key->rk);
        }
        fw[p].err = d->err;
        if (!fwd && p == 0)
            set_l1_maps(fw[p], fw[p].single);
    }
    const bool sep = ctr_pass(b);
    const frag::CtrChunk frag_chunk = ctr_fragment(fwd, b);
    if (fwd && b.F1)
        st = fuse_launch(*d, true, false, fw[0], fslots[0], s);
    if (st == FRAG_OK && fwd && b.F2)
        st = fuse_launch(*d, true, true, fw[1], fslots[1], s);
    if (st == FRAG_OK && sep && !fwd)
        st = ctr_launch(*d, frag::aes::keys_from_words(key->rk), nullptr, &frag_chunk, s);
    if (st == FRAG_OK && njobs) {
        std::vector<LevelJob> jobs;
        uint32_t counters = 0;
        buffer_jobs(fwd, b, 0, &counters, jobs);
        DagWork w;
        std::memset(&w, 0, sizeof(w));
        uint64_t units = 0;
        for (uint32_t m = 0; m < njobs; ++m) {
            w.inline_jobs[m] = jobs[m];
            units += (uint64_t)jobs[m].strips * jobs[m].segs;
        }
        w.n_inline = njobs;
        w.lag = buffer_lag(jobs, 0, njobs, grid);
        w.total_units = units;
        w.done = (unsigned *)(mem + sb);
        w.queue = (unsigned long long *)(mem + sb + cb);
        w.aes_tables = d->tables;
        w.round_keys = rk;
        w.err = d->err;
        w.spin_limit = kSpinLimit;
        cudaError_t e = cudaMemsetAsync(mem + sb, 0, cb + 256, s);
        if (e != cudaSuccess)
            st = cuda_fail(e, "counter reset");
        if (st == FRAG_OK && (st = dag_grid(*d, fwd, units, &grid)) == FRAG_OK) {
            if (plan->max_ctas)
                grid = std::min(grid, plan->max_ctas);
            if ((e = frag::launch_dag(fwd, w, grid, s)) != cudaSuccess)
                st = cuda_fail(e, fwd ? "protect launch" : "recover launch");
        }
    }
    if (st == FRAG_OK && sep && fwd)
        st = ctr_launch(*d, frag::aes::keys_from_words(key->rk), nullptr, &frag_chunk, s);
    if (st == FRAG_OK && !fwd && b.F2)
        st = fuse_launch(*d, false, true, fw[1], fslots[1], s);
    if (st == FRAG_OK && !fwd && b.F1)
        st = fuse_launch(*d, false, false, fw[0], fslots[0], s);
    if (mem)
        cudaFreeAsync(mem, s);
    return st;
}

// ---------------------------------------------------------------------------
// Host-buffer forms pipelined by row bands
//
// A buffer whose levels all run in the first fused pass (L <= 3) is cut into
// bands of whole fused segments.  Band k's copies in, its kernels and its
// copies out run on three streams, so band k + 1 arrives over PCIe while
// band k is transformed and band k - 1 leaves.  What a band needs and makes
// follows from the fused kernel's row schedule: the forward's iteration t
// reads level-0 rows 8t-1 .. 8t+6 and writes level-l rows (8>>l) t - 1 ..
// (8>>l) t + (8>>l) - 2; the inverse's iteration t reads level-l rows up to
// (8>>l) t and writes level-0 rows 8t-7 .. 8t.  A band enciphers only the
// AES blocks whose bytes are all written by then (CTR is its own inverse, so
// no block may be done twice); recover deciphers, band by band, every block
// the band's rows touch into the plaintext scratch the inverse reads.
// ---------------------------------------------------------------------------
// bands of about FRAG_HOST_BAND_MB MiB, 8 to 64 of them: the first band's
// copy in and the last band's copy out overlap nothing, so finer bands
// shorten the pipeline's head and tail, but every copy also costs a few us
// of its own (pinned, one B300, protect + recover of 256 MiB at 2 levels:
// 8 / 16 / 32 / 64 bands 11.24 / 10.96 / 10.50 / 9.83 GB/s; of 1 GiB: 8 /
// 16 / 32 bands 11.69 / 11.82 / 11.86 GB/s).  FRAG_HOST_COPY2D moves a
// level's three band pieces in one strided copy instead of three
// (256 MiB: 11.40 against 11.20 GB/s; 1 GiB: 11.86 against 11.51)
#ifndef FRAG_HOST_BAND_MB
#define FRAG_HOST_BAND_MB 32
#endif
#ifndef FRAG_HOST_COPY2D
#define FRAG_HOST_COPY2D 1
#endif
constexpr uint64_t kHostBandBytes = (uint64_t)FRAG_HOST_BAND_MB << 20;
constexpr uint32_t kHostBandsMin = 8, kHostBandsMax = 64;
constexpr uint64_t kHostBandMin = 16ull << 20; // smaller buffers run in one piece

uint32_t host_bands(uint64_t n)
{
    return (uint32_t)std::min<uint64_t>(kHostBandsMax, std::max<uint64_t>(kHostBandsMin, (n + kHostBandBytes - 1) / kHostBandBytes));
}

struct Pipe {
    cudaStream_t in = nullptr, out = nullptr;
    std::vector<cudaEvent_t> ev;
    ~Pipe()
    {
        for (cudaEvent_t e : ev)
            cudaEventDestroy(e);
        if (in)
            cudaStreamDestroy(in);
        if (out)
            cudaStreamDestroy(out);
    }
    cudaError_t make(size_t events)
    {
        cudaError_t e = cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking);
        for (size_t i = 0; e == cudaSuccess && i < events; ++i) {
            cudaEvent_t v = nullptr;
            e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
            if (e == cudaSuccess)
                ev.push_back(v);
        }
        return e;
    }
};

cudaError_t copy_async(void *dst, const void *src, uint64_t bytes, cudaMemcpyKind kind, cudaStream_t s)
{
    return bytes ? cudaMemcpyAsync(dst, src, bytes, kind, s) : cudaSuccess;
}

// *done false: the buffer does not take the banded form (the caller runs
// the plain one).  mem: device scratch of n + pb + ub bytes (each part at
// a 256-byte boundary) and, for recover, the plaintext LL_L after them.
frag_status run_host_banded(bool fwd, frag_plan plan, frag_key key, uint64_t nonce, const uint8_t *h_a,
                            const uint8_t *h_b, uint8_t *h_c, uint8_t *h_d, uint64_t n, cudaStream_t s,
                            bool *done)
{
    *done = false;
    if (n < kHostBandMin || plan->block || plan->packed || plan->levels > 2 * frag::kFuseMaxLevels ||
        plan->path != FRAG_PATH_AUTO)
        return FRAG_OK;
    DeviceState *d = nullptr;
    int dev = 0;
    frag_status st = device_state(&d, &dev);
    if (st != FRAG_OK)
        return st;
    const uint32_t W = plan->width, L = plan->levels;
    const uint64_t H = rows_for(n, W, L);
    if (H > 0xFFFFFFFFull)
        return fail(FRAG_EINVAL, "buffer too tall for width %u", W);
    const uint64_t pb = ll_bytes(H, W, L), ub = 2ull * H * W - pb;
    const uint64_t a_n = align256(n), a_pb = align256(pb), a_ub = align256(ub);
    const uint64_t ll_scr = fwd ? 0 : a_pb;
    // 4..6 levels: LL_3 between the banded first pass and the second pass
    const uint64_t a_s3 = L > frag::kFuseMaxLevels ? align256(ll_bytes(H, W, frag::kFuseMaxLevels)) : 0;
    Buf b;
    std::memset(&b, 0, sizeof(b));
    b.W = W;
    b.L = L;
    b.H = (uint32_t)H;
    b.n = n;
    b.nonce = nonce;
    uint8_t *mem = nullptr;
    cudaError_t e = pool_malloc((void **)&mem, a_n + a_pb + a_ub + ll_scr + a_s3, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "pool_malloc(host-form buffers)");
    uint8_t *d_data = mem, *d_priv = mem + a_n, *d_pub = d_priv + a_pb;
    if (fwd) {
        b.in = d_data;
        b.priv = d_priv;
        b.pub = d_pub;
    } else {
        b.out = d_data;
        b.priv_in = d_priv;
        b.pub_in = d_pub;
        b.scr[L] = d_pub + a_ub;
    }
    if (a_s3)
        b.scr[frag::kFuseMaxLevels] = d_pub + a_ub + ll_scr;
    fused_split(fwd, b, plan->path);
    const uint32_t *rk = nullptr;
    // fw: the first fused pass, run band by band; fw2: the second (levels
    // 4..L over LL_3), one launch after the bands (protect) or before them
    // (recover)
    frag::FuseWork fw, fw2;
    std::memset(&fw, 0, sizeof(fw));
    std::memset(&fw2, 0, sizeof(fw2));
    uint64_t slots = 0, slots2 = 0;
    const bool two = b.F2 != 0;
    bool ok = b.F1 + b.F2 == L && (!two || b.F1 == frag::kFuseMaxLevels) && !b.kc;
    if (ok && two && (st = fuse_slots(*d, fwd, true, plan->max_ctas, &slots2)) == FRAG_OK) {
        fw2.single = fuse_buf(fwd, b, 2);
        fw2.nbufs = 1;
        fw2.total_units = fuse_schedule(&fw2.single, 1, slots2, plan->seg_rows);
        fw2.err = d->err;
    }
    if (ok && st == FRAG_OK && (st = key_on_device(key, dev, &rk)) == FRAG_OK &&
        (st = fuse_slots(*d, fwd, false, plan->max_ctas, &slots)) == FRAG_OK) {
        fw.single = fuse_buf(fwd, b, 1);
        fw.nbufs = 1;
        fw.err = d->err;
        // units for the band count times the resident warps, so that every
        // band's launch still fills the device
        fuse_schedule(&fw.single, 1, slots * host_bands(n), plan->seg_rows, false, false);
        ok = fw.single.segs >= 2;
    }
    if (st != FRAG_OK || !ok) {
        cudaFreeAsync(mem, s);
        return st;
    }
    *done = true;
    const frag::AesKeys keys = frag::aes::keys_from_words(key->rk);
    const uint32_t segs = fw.single.segs, strips = fw.single.strips, seg = fw.single.seg_iters;
    const uint32_t iters = fw.single.iters, K = std::min(host_bands(n), segs);
    Pipe p;
    if ((e = p.make(2 * K + 2)) != cudaSuccess) {
        cudaFreeAsync(mem, s);
        return cuda_fail(e, "host-form streams");
    }
    const uint32_t WL = W >> L, F1 = b.F1;
    uint64_t row0 = 0;                     // level-0 rows moved so far
    uint64_t lrow[frag::kFuseMaxLevels + 1] = {0, 0, 0, 0}; // level-l rows moved so far
    uint64_t blk0 = 0;                     // AES blocks handled so far
    const uint64_t nblk = (pb + 15) / 16;
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
    // the band pieces of level-l rows [r0, r1) of every detail band: in
    // (recover) or out (protect)
    auto band_rows = [&](uint32_t l, uint64_t r0, uint64_t r1, bool in, cudaStream_t cs) {
        const uint64_t rowb = 2ull * (W >> l);
        cudaError_t r = cudaSuccess;
#if FRAG_HOST_COPY2D
        // the three bands of a level lie one after another, so one strided
        // copy moves their rows [r0, r1)
        const uint64_t pitch = frag::band_offset(b.H, W, L, l, 1) - frag::band_offset(b.H, W, L, l, 0);
        if (pitch < (1ull << 31)) {
            const uint64_t off = frag::band_offset(b.H, W, L, l, 0) + rowb * r0, len = rowb * (r1 - r0);
            return in ? cudaMemcpy2DAsync(d_pub + off, pitch, h_b + off, pitch, len, 3, h2d, cs)
                      : cudaMemcpy2DAsync(h_d + off, pitch, d_pub + off, pitch, len, 3, d2h, cs);
        }
#endif
        for (uint32_t k = 0; k < 3 && r == cudaSuccess; ++k) {
            const uint64_t off = frag::band_offset(b.H, W, L, l, k) + rowb * r0, len = rowb * (r1 - r0);
            r = in ? copy_async(d_pub + off, h_b + off, len, h2d, cs) : copy_async(h_d + off, d_pub + off, len, d2h, cs);
        }
        return r;
    };
    auto whole_chunk = [&](const uint8_t *in, uint8_t *out) {
        frag::CtrChunk c;
        std::memset(&c, 0, sizeof(c));
        c.nonce = nonce;
        c.bytes = pb;
        c.in = in;
        c.out = out;
        c.nblocks = nblk;
        return c;
    };
    if (two && !fwd) {
        // the private fragment and the levels above 3 are small: in at once,
        // then the deciphering and the second pass make LL_3 before the
        // first band's kernels
        e = copy_async(d_priv, h_a, pb, h2d, p.in);
        for (uint32_t l = F1 + 1; l <= L && e == cudaSuccess; ++l)
            e = band_rows(l, 0, H >> l, true, p.in);
        if (e == cudaSuccess && (e = cudaEventRecord(p.ev[2 * K + 1], p.in)) == cudaSuccess)
            e = cudaStreamWaitEvent(s, p.ev[2 * K + 1], 0);
        if (e == cudaSuccess) {
            const frag::CtrChunk c = whole_chunk(d_priv, b.scr[L]);
            if ((st = ctr_launch(*d, keys, nullptr, &c, s)) == FRAG_OK)
                st = fuse_launch(*d, false, true, fw2, slots2, s);
        }
    }
    for (uint32_t k = 0; k < K && e == cudaSuccess && st == FRAG_OK; ++k) {
        const bool last = k + 1 == K;
        const uint64_t sy0 = (uint64_t)k * segs / K, sy1 = (uint64_t)(k + 1) * segs / K;
        const uint64_t t1 = last ? iters : std::min<uint64_t>(sy1 * seg, iters);
        cudaEvent_t ev_in = p.ev[2 * k], ev_comp = p.ev[2 * k + 1];
        frag::CtrChunk c;
        std::memset(&c, 0, sizeof(c));
        c.nonce = nonce;
        c.bytes = pb;
        if (fwd) {
            // in: level-0 rows the band's iterations read
            const uint64_t r1 = last ? H : std::min<uint64_t>(H, 8 * t1 + 8);
            const uint64_t lo = std::min(n, row0 * W), hi = std::min(n, r1 * W);
            e = copy_async(d_data + lo, h_a + lo, hi - lo, h2d, p.in);
            row0 = r1;
        } else {
            // in: coefficient rows the band's iterations read, and the
            // private blocks that cover its LL_L rows
            for (uint32_t l = 1; l <= F1 && e == cudaSuccess; ++l) {
                const uint64_t Hl = H >> l, r1 = last ? Hl : std::min<uint64_t>(Hl, (8u >> l) * t1 + 1);
                if (r1 > lrow[l])
                    e = band_rows(l, lrow[l], r1, true, p.in);
                lrow[l] = std::max(lrow[l], r1);
            }
            const uint64_t bhi = two ? 0 : last ? nblk : std::min<uint64_t>(nblk, (2ull * WL * lrow[L] + 15) / 16);
            if (e == cudaSuccess && bhi > blk0)
                e = copy_async(d_priv + 16 * blk0, h_a + 16 * blk0, std::min(pb, 16 * bhi) - 16 * blk0, h2d, p.in);
            if (bhi > blk0) {
                c.in = d_priv;
                c.out = b.scr[L];
                c.first_block = blk0;
                c.nblocks = bhi - blk0;
                blk0 = bhi;
            }
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_in, p.in);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s, ev_in, 0);
        if (e != cudaSuccess)
            break;
        fw.unit_lo = sy0 * strips;
        fw.total_units = (sy1 - sy0) * strips;
        if (!fwd && c.nblocks)
            st = ctr_launch(*d, keys, nullptr, &c, s);
        if (st == FRAG_OK)
            st = fuse_launch(*d, fwd, false, fw, slots, s);
        if (st == FRAG_OK && fwd && !two) {
            // encipher the blocks whose bytes are all written now
            const uint64_t Hl = H >> L, r1 = last ? Hl : std::min<uint64_t>(Hl, (8u >> L) * t1 - 1);
            const uint64_t bhi = last ? nblk : std::min<uint64_t>(nblk, 2ull * WL * r1 / 16);
            if (bhi > blk0) {
                c.in = d_priv;
                c.out = d_priv;
                c.first_block = blk0;
                c.nblocks = bhi - blk0;
                st = ctr_launch(*d, keys, nullptr, &c, s);
            }
        }
        if (st != FRAG_OK)
            break;
        if ((e = cudaEventRecord(ev_comp, s)) == cudaSuccess)
            e = cudaStreamWaitEvent(p.out, ev_comp, 0);
        if (e != cudaSuccess)
            break;
        if (fwd) {
            // out: the detail rows and the enciphered blocks the band finished
            for (uint32_t l = 1; l <= F1 && e == cudaSuccess; ++l) {
                const uint64_t Hl = H >> l, r1 = last ? Hl : std::min<uint64_t>(Hl, (8u >> l) * t1 - 1);
                if (r1 > lrow[l])
                    e = band_rows(l, lrow[l], r1, false, p.out);
                lrow[l] = std::max(lrow[l], r1);
            }
            const uint64_t Hl = H >> L, r1 = last ? Hl : std::min<uint64_t>(Hl, (8u >> L) * t1 - 1);
            const uint64_t bhi = two ? 0 : last ? nblk : std::min<uint64_t>(nblk, 2ull * WL * r1 / 16);
            if (e == cudaSuccess && bhi > blk0)
                e = copy_async(h_c + 16 * blk0, d_priv + 16 * blk0, std::min(pb, 16 * bhi) - 16 * blk0, d2h, p.out);
            blk0 = std::max(blk0, bhi);
        } else {
            // out: the level-0 rows the band wrote
            const uint64_t r1 = last ? H : std::min<uint64_t>(H, 8 * t1 - 7);
            const uint64_t lo = std::min(n, row0 * W), hi = std::min(n, r1 * W);
            e = copy_async(h_c + lo, d_data + lo, hi - lo, d2h, p.out);
            row0 = std::max(row0, r1);
        }
    }
    if (two && fwd && e == cudaSuccess && st == FRAG_OK) {
        // after the last band: the second pass over LL_3, the private
        // fragment enciphered whole, and the small rest copied out
        const frag::CtrChunk c = whole_chunk(d_priv, d_priv);
        if ((st = fuse_launch(*d, true, true, fw2, slots2, s)) == FRAG_OK &&
            (st = ctr_launch(*d, keys, nullptr, &c, s)) == FRAG_OK &&
            (e = cudaEventRecord(p.ev[2 * K + 1], s)) == cudaSuccess &&
            (e = cudaStreamWaitEvent(p.out, p.ev[2 * K + 1], 0)) == cudaSuccess) {
            for (uint32_t l = F1 + 1; l <= L && e == cudaSuccess; ++l)
                e = band_rows(l, 0, H >> l, false, p.out);
            if (e == cudaSuccess)
                e = copy_async(h_c, d_priv, pb, d2h, p.out);
        }
    }
    if (e == cudaSuccess && st == FRAG_OK && (e = cudaEventRecord(p.ev[2 * K], p.out)) == cudaSuccess)
        e = cudaStreamWaitEvent(s, p.ev[2 * K], 0);
    if (e != cudaSuccess || st != FRAG_OK) { // copies may still be in flight on the side streams
        cudaStreamSynchronize(p.in);
        cudaStreamSynchronize(p.out);
    }
    cudaFreeAsync(mem, s);
    // the copies read and write the caller's host buffers: nothing returns
    // before they are done
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaError_t e3 = cudaStreamSynchronize(p.out);
    if (st != FRAG_OK)
        return st;
    if (e != cudaSuccess)
        return cuda_fail(e, "host-form band copies");
    if (e2 != cudaSuccess)
        return cuda_fail(e2, "cudaStreamSynchronize");
    if (e3 != cudaSuccess)
        return cuda_fail(e3, "cudaStreamSynchronize");
    return FRAG_OK;
}

// ---------------------------------------------------------------------------
// Batches: buffers, most work first, cut into waves whose scratch fits a
// budget; one launch per wave over an explicit dependency-ordered unit list
// ---------------------------------------------------------------------------
struct DagWave {
    std::vector<LevelJob> jobs;
    std::vector<uint32_t> first, levels; // per buffer: first job, number of jobs
    std::vector<DagUnit> units;
    std::vector<frag::CtrChunk> chunks; // private fragments of the separate CTR launch
    std::vector<uint64_t> turn_start;   // their first warp turns (one more entry)
    uint64_t turn_blocks = 0;
    std::vector<frag::FuseBuf> fbufs;   // buffers of the first fused pass (levels 1..3)
    uint64_t fuse_units = 0;
    std::vector<uint32_t> fgroups;      // fbufs[fgroups[g] .. fgroups[g + 1]): one launch each
    std::vector<uint64_t> fgroup_units; // the units of each of those launches
    std::vector<frag::FuseBuf> fbufs2;  // buffers of the second fused pass (levels 4 to 6)
    uint64_t fuse_units2 = 0;
    std::vector<frag::FuseBuf> bbufs;   // buffers of the block launch
    uint64_t block_units = 0;
    std::vector<frag::FuseBuf> pbufs;   // buffers of the packed block launch
    uint64_t packed_units = 0;
    uint32_t counters = 0;
    size_t jobs_off = 0, units_off = 0, done_off = 0, queue_off = 0, chunks_off = 0, turns_off = 0, fbufs_off = 0,
           bbufs_off = 0, fbufs2_off = 0, pbufs_off = 0;
};

struct BatchPlan {
    bool fwd = true;
    uint64_t resident_ctas = 0; // CTAs one launch keeps resident
    uint64_t sms = 0;           // the device's SMs
    uint32_t max_ctas = 0;      // grid cap from the first item's plan (0: none)
    uint32_t fuse_rows = 0;     // fused segment rows from the first item's plan (0: adaptive)
    uint64_t fuse_slots = 0;    // fused warps one launch keeps resident
    uint64_t fuse_slots2 = 0;   // the same for the second (packed) pass
    std::vector<Buf> bufs;
    std::vector<uint64_t> scr_off;
    std::vector<uint32_t> wave_of;
    std::vector<DagWave> waves;
    uint64_t scratch = 0;
    size_t desc_bytes = 0;
};

frag_status plan_batch(bool fwd, const frag_item *pi, const frag_ritem *ri, uint32_t count,
                       BatchPlan &bp)
{
    bp.fwd = fwd;
    std::vector<std::pair<uint64_t, Buf>> v;
    for (uint32_t i = 0; i < count; ++i) {
        frag_plan plan = fwd ? pi[i].plan : ri[i].plan;
        if (plan == nullptr)
            return fail(FRAG_EINVAL, "item %u has no plan", i);
        const uint64_t n = fwd ? pi[i].nbytes : ri[i].nbytes;
        if (n == 0)
            continue;
        Buf b;
        std::memset(&b, 0, sizeof(b));
        b.W = plan->width;
        b.L = plan->levels;
        b.R0_plan = plan->seg_rows;
        b.block = plan->block;
        b.packed = plan->packed;
        b.keyed = plan->keyed;
        if (bp.bufs.empty() && v.empty()) {
            bp.max_ctas = plan->max_ctas; // the grid of a launch: the first item's plan
            bp.fuse_rows = plan->seg_rows;
        }
        const uint64_t H = rows_for(n, b.W, b.L, b.block);
        if (H > 0xFFFFFFFFull)
            return fail(FRAG_EINVAL, "item %u is too tall for width %u", i, b.W);
        b.H = (uint32_t)H;
        b.n = n;
        if (fwd) {
            b.nonce = pi[i].nonce;
            b.in = (const uint8_t *)pi[i].d_in;
            b.priv = (uint8_t *)pi[i].d_private;
            b.pub = (uint8_t *)pi[i].d_public;
            if (!b.in || !b.priv || !b.pub)
                return fail(FRAG_EINVAL, "item %u has a NULL buffer", i);
        } else {
            b.nonce = ri[i].nonce;
            b.priv_in = (const uint8_t *)ri[i].d_private;
            b.pub_in = (const uint8_t *)ri[i].d_public;
            b.out = (uint8_t *)ri[i].d_out;
            if (!b.priv_in || !b.pub_in || !b.out)
                return fail(FRAG_EINVAL, "item %u has a NULL buffer", i);
        }
        fused_split(fwd, b, plan->path);
        v.emplace_back(H * (uint64_t)b.W, b);
    }
    std::stable_sort(v.begin(), v.end(),
                     [](const std::pair<uint64_t, Buf> &a, const std::pair<uint64_t, Buf> &c) {
                         return a.first > c.first;
                     });
    uint64_t used = 0;
    uint32_t wave = 0;
    for (auto &p : v) {
        const uint64_t sb = align256(
            scratch_bytes(fwd, p.second.H, p.second.W, p.second.L, p.second.F1, nullptr, p.second.kc));
        if (used > 0 && used + sb > kScratchBudget) {
            ++wave;
            used = 0;
        }
        bp.bufs.push_back(p.second);
        bp.scr_off.push_back(used);
        bp.wave_of.push_back(wave);
        used += sb;
        bp.scratch = std::max(bp.scratch, used);
    }
    bp.waves.assign(bp.bufs.empty() ? 0 : wave + 1, DagWave());
    return FRAG_OK;
}

// The launches of a first fused pass over f[0..n): one per level count
// (true) when every count present has at least kFuseSplitRounds rounds of
// full units for the `slots` resident warps, else one launch.  Protect of
// 1, 2 and 3 levels at width 4096, one launch per count against one mixed
// launch, by rounds per count: 1.4 rounds 17 % slower (each launch ends in a
// part-filled round), 2.9 even, 4.3 3 % slower, 8.7 4 % faster, 17 and 52
// 7-8 % faster; C4 (10,000 buffers, about 118 rounds a count) 51.5 -> 45.4 ms.
constexpr uint64_t kFuseSplitRounds = 8;

bool fuse_split_by_levels(const frag::FuseBuf *f, size_t n, uint64_t slots)
{
    uint64_t work[frag::kFuseMaxLevels + 1] = {0};
    for (size_t i = 0; i < n; ++i)
        work[f[i].F] += (uint64_t)f[i].strips * f[i].iters;
    int kinds = 0;
    bool split = true;
    for (uint32_t F = 1; F <= frag::kFuseMaxLevels; ++F)
        if (work[F]) {
            ++kinds;
            split = split && work[F] >= kFuseSplitRounds * slots * kFuseBatchSegIters;
        }
    return kinds > 1 && split;
}

// a wave's first-pass launches (fgroups, fgroup_units) by that rule: a
// count's buffers keep their order (largest first), and each launch's units
// are scheduled on their own
void fuse_groups(DagWave &wv, uint64_t slots, uint32_t plan_rows)
{
    std::vector<frag::FuseBuf> &f = wv.fbufs;
    wv.fgroups.assign(1, 0);
    wv.fgroup_units.clear();
    wv.fuse_units = 0;
    if (f.empty())
        return;
    if (fuse_split_by_levels(f.data(), f.size(), slots)) {
        std::stable_sort(f.begin(), f.end(),
                         [](const frag::FuseBuf &a, const frag::FuseBuf &b) { return a.F > b.F; });
        for (size_t i = 1; i < f.size(); ++i)
            if (f[i].F != f[i - 1].F)
                wv.fgroups.push_back((uint32_t)i);
    }
    wv.fgroups.push_back((uint32_t)f.size());
    for (size_t g = 0; g + 1 < wv.fgroups.size(); ++g) {
        const uint64_t u = fuse_schedule(f.data() + wv.fgroups[g], wv.fgroups[g + 1] - wv.fgroups[g],
                                         slots, plan_rows, true);
        wv.fgroup_units.push_back(u);
        wv.fuse_units += u;
    }
}

// jobs and units of every wave, with scratch pointers from `scratch_base`;
// then the layout of the descriptors after the scratch
void fill_batch(BatchPlan &bp, uint8_t *scratch_base)
{
    // one segment height for the whole batch, from its first-level units
    uint64_t u64 = 0;
    for (const Buf &b : bp.bufs)
        u64 += l1_units_at_64(b);
    // CTR warp turns: kCtrTurn blocks (one a lane a step), doubled up to
    // 128x while the batch keeps more than 4 turns a resident warp of the CTR
    // launch, so a batch of small fragments still spreads over every SM;
    // the launch reads one descriptor per fragment and finds a turn's
    // fragment by binary search, so the host's work grows with the buffers,
    // not with the blocks
    uint64_t ctr_blocks = 0;
    for (const Buf &b : bp.bufs)
        if (ctr_pass(b))
            ctr_blocks += ctr_fragment(bp.fwd, b).nblocks;
    uint64_t turn = frag::kCtrTurn;
    const uint64_t per_warp = 4 * std::max<uint64_t>(1, bp.sms) * (frag::kCtrThreads / 32);
    while (turn < 128 * frag::kCtrTurn && ctr_blocks / (2 * turn) >= per_warp)
        turn *= 2;
    for (auto &wv : bp.waves) {
        wv.jobs.clear();
        wv.first.clear();
        wv.levels.clear();
        wv.units.clear();
        wv.chunks.clear();
        wv.turn_start.assign(1, 0);
        wv.turn_blocks = turn;
        wv.fbufs.clear();
        wv.fuse_units = 0;
        wv.bbufs.clear();
        wv.block_units = 0;
        wv.pbufs.clear();
        wv.packed_units = 0;
        wv.fbufs2.clear();
        wv.fuse_units2 = 0;
        wv.counters = 0;
    }
    for (size_t i = 0; i < bp.bufs.size(); ++i) {
        Buf &b = bp.bufs[i];
        uint64_t off[frag::kMaxInlineJobs + 1] = {0};
        b.R0 = seg_rows0(b.L, u64, bp.resident_ctas, b.R0_plan);
        scratch_bytes(bp.fwd, b.H, b.W, b.L, b.F1, off, b.kc);
        for (uint32_t l = scratch_lo(b.F1); l <= scratch_hi(bp.fwd, b.L, b.kc); ++l)
            b.scr[l] = scratch_base + bp.scr_off[i] + off[l];
        DagWave &wv = bp.waves[bp.wave_of[i]];
        const uint32_t first = (uint32_t)wv.jobs.size();
        buffer_jobs(bp.fwd, b, first, &wv.counters, wv.jobs);
        wv.first.push_back(first);
        wv.levels.push_back(buffer_njobs(b));
        if (b.block && b.packed)
            wv.pbufs.push_back(packed_buf(bp.fwd, b));
        else if (b.block)
            wv.bbufs.push_back(block_buf(bp.fwd, b));
        else if (b.F1)
            wv.fbufs.push_back(fuse_buf(bp.fwd, b, 1));
        if (b.F2)
            wv.fbufs2.push_back(fuse_buf(bp.fwd, b, 2));
        if (ctr_pass(b)) { // the private fragment, whole, and its turns
            const frag::CtrChunk whole = ctr_fragment(bp.fwd, b);
            wv.chunks.push_back(whole);
            wv.turn_start.push_back(wv.turn_start.back() + (whole.nblocks + turn - 1) / turn);
        }
    }
    for (auto &wv : bp.waves) {
        wave_units(wv.jobs, wv.first, wv.levels, wv.units);
        fuse_groups(wv, std::max<uint64_t>(1, bp.fuse_slots), bp.fuse_rows);
        wv.block_units = block_units(wv.bbufs.data(), wv.bbufs.size());
        wv.packed_units = block_units(wv.pbufs.data(), wv.pbufs.size());
        wv.fuse_units2 = fuse_schedule(wv.fbufs2.data(), wv.fbufs2.size(),
                                       std::max<uint64_t>(1, bp.fuse_slots2),
                                       bp.fuse_rows, true);
    }
    size_t off = align256(bp.scratch);
    for (auto &wv : bp.waves) {
        wv.jobs_off = off;
        off += align256(std::max<size_t>(1, wv.jobs.size()) * sizeof(LevelJob));
        wv.units_off = off;
        off += align256(std::max<size_t>(1, wv.units.size()) * sizeof(DagUnit));
        wv.done_off = off;
        off += align256(4ull * std::max(1u, wv.counters));
        wv.queue_off = off;
        off += 256;
        wv.chunks_off = off;
        off += align256(wv.chunks.size() * sizeof(frag::CtrChunk));
        wv.turns_off = off;
        off += align256(wv.turn_start.size() * sizeof(uint64_t));
        wv.fbufs_off = off;
        off += align256(wv.fbufs.size() * sizeof(frag::FuseBuf));
        wv.bbufs_off = off;
        off += align256(wv.bbufs.size() * sizeof(frag::FuseBuf));
        wv.fbufs2_off = off;
        off += align256(wv.fbufs2.size() * sizeof(frag::FuseBuf));
        wv.pbufs_off = off;
        off += align256(wv.pbufs.size() * sizeof(frag::FuseBuf));
    }
    bp.desc_bytes = off - align256(bp.scratch);
}

size_t batch_mem_bytes(const BatchPlan &bp) { return align256(bp.scratch) + bp.desc_bytes; }

frag_status upload_batch(const BatchPlan &bp, uint8_t *mem, cudaStream_t s, bool async)
{
    const size_t base = align256(bp.scratch);
    std::vector<uint8_t> host(bp.desc_bytes, 0);
    for (const auto &wv : bp.waves) {
        std::memcpy(host.data() + (wv.jobs_off - base), wv.jobs.data(), wv.jobs.size() * sizeof(LevelJob));
        std::memcpy(host.data() + (wv.units_off - base), wv.units.data(), wv.units.size() * sizeof(DagUnit));
        if (!wv.chunks.empty()) {
            std::memcpy(host.data() + (wv.chunks_off - base), wv.chunks.data(),
                        wv.chunks.size() * sizeof(frag::CtrChunk));
            std::memcpy(host.data() + (wv.turns_off - base), wv.turn_start.data(),
                        wv.turn_start.size() * sizeof(uint64_t));
        }
        if (!wv.fbufs.empty())
            std::memcpy(host.data() + (wv.fbufs_off - base), wv.fbufs.data(),
                        wv.fbufs.size() * sizeof(frag::FuseBuf));
        if (!wv.bbufs.empty())
            std::memcpy(host.data() + (wv.bbufs_off - base), wv.bbufs.data(),
                        wv.bbufs.size() * sizeof(frag::FuseBuf));
        if (!wv.fbufs2.empty())
            std::memcpy(host.data() + (wv.fbufs2_off - base), wv.fbufs2.data(),
                        wv.fbufs2.size() * sizeof(frag::FuseBuf));
        if (!wv.pbufs.empty())
            std::memcpy(host.data() + (wv.pbufs_off - base), wv.pbufs.data(),
                        wv.pbufs.size() * sizeof(frag::FuseBuf));
    }
    cudaError_t e = async ? cudaMemcpyAsync(mem + base, host.data(), host.size(), cudaMemcpyHostToDevice, s)
                          : cudaMemcpy(mem + base, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail(e, "batch descriptor upload");
    return FRAG_OK;
}

// event pair around one launch of a timed batch run
struct TimedLaunch {
    uint32_t kind;
    cudaEvent_t a, b;
};

struct LaunchTimer {
    std::vector<TimedLaunch> *out;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    void begin()
    {
        if (out && cudaEventCreate(&a) == cudaSuccess && cudaEventRecord(a, s) != cudaSuccess) {
            cudaEventDestroy(a);
            a = nullptr;
        }
    }
    void end(uint32_t kind)
    {
        if (!out || !a)
            return;
        cudaEvent_t b = nullptr;
        if (cudaEventCreate(&b) == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess)
            out->push_back(TimedLaunch{kind, a, b});
        else {
            cudaEventDestroy(a);
            if (b)
                cudaEventDestroy(b);
        }
        a = nullptr;
    }
};

// the fused launches of a wave: the first pass, one launch per group of
// fgroups (descriptors at fbufs_off), or the second pass, one launch
// (descriptors at fbufs2_off)
frag_status launch_wave_fused(const BatchPlan &bp, const DagWave &wv, uint8_t *mem, DeviceState &d,
                              cudaStream_t s, LaunchTimer &tm, const frag::AesKeys &keys, int pass = 1)
{
    const std::vector<frag::FuseBuf> &bufs = pass == 1 ? wv.fbufs : wv.fbufs2;
    if (bufs.empty())
        return FRAG_OK;
    const size_t groups = pass == 1 ? wv.fgroups.size() - 1 : 1;
    for (size_t g = 0; g < groups; ++g) {
        const size_t lo = pass == 1 ? wv.fgroups[g] : 0, hi = pass == 1 ? wv.fgroups[g + 1] : bufs.size();
        frag::FuseWork w;
        std::memset(&w, 0, sizeof(w));
        for (size_t i = lo; i < hi; ++i)
            w.cipher |= bufs[i].cipher;
        if (w.cipher)
            w.keys = keys;
        w.nbufs = (uint32_t)(hi - lo);
        w.bufs = (const frag::FuseBuf *)(mem + (pass == 1 ? wv.fbufs_off : wv.fbufs2_off)) + lo;
        w.err = d.err;
        if (w.nbufs == 1) {
            w.single = bufs[lo];
            if (!bp.fwd && pass == 1)
                set_l1_maps(w, w.single);
        }
        w.total_units = pass == 1 ? wv.fgroup_units[g] : wv.fuse_units2;
        tm.begin();
        frag_status st = fuse_launch(d, bp.fwd, pass == 2, w,
                                     std::max<uint64_t>(1, pass == 1 ? bp.fuse_slots : bp.fuse_slots2), s);
        tm.end(pass == 1 ? FRAG_KERNEL_FUSED : FRAG_KERNEL_FUSED_LOW);
        if (st != FRAG_OK)
            return st;
    }
    return FRAG_OK;
}

// the block launch of a wave (its buffers' descriptors at bbufs_off)
frag_status launch_wave_blocks(const BatchPlan &bp, const DagWave &wv, uint8_t *mem, DeviceState &d,
                               cudaStream_t s, LaunchTimer &tm, bool packed = false, const uint32_t *rk = nullptr)
{
    const std::vector<frag::FuseBuf> &bufs = packed ? wv.pbufs : wv.bbufs;
    if (bufs.empty())
        return FRAG_OK;
    frag::FuseWork w;
    std::memset(&w, 0, sizeof(w));
    w.nbufs = (uint32_t)bufs.size();
    w.bufs = (const frag::FuseBuf *)(mem + (packed ? wv.pbufs_off : wv.bbufs_off));
    if (w.nbufs == 1)
        w.single = bufs[0];
    w.total_units = packed ? wv.packed_units : wv.block_units;
    tm.begin();
    bool keyed = false;
    for (const auto &f : bufs)
        keyed = keyed || f.keyed;
    frag_status st = block_launch(d, bp.fwd, w, s, packed, keyed, rk);
    tm.end(FRAG_KERNEL_BLOCKS);
    return st;
}

// per wave, protect: fused levels, block mode, dependency-ordered levels
// above the fused ones, CTR; recover: CTR, dependency-ordered levels, block
// mode, fused levels
frag_status launch_batch(const BatchPlan &bp, uint8_t *mem, DeviceState &d, const uint32_t *rk,
                         const frag::AesKeys &keys, cudaStream_t s, std::vector<TimedLaunch> *timed = nullptr)
{
    LaunchTimer tm{timed, s};
    for (const auto &wv : bp.waves) {
        CtrList clist;
        clist.frags = (const frag::CtrChunk *)(mem + wv.chunks_off);
        clist.turn_start = (const uint64_t *)(mem + wv.turns_off);
        clist.nfrags = wv.chunks.size();
        clist.nturns = wv.turn_start.empty() ? 0 : wv.turn_start.back();
        clist.turn_blocks = wv.turn_blocks;
        frag_status st = FRAG_OK;
        if (bp.fwd && (st = launch_wave_fused(bp, wv, mem, d, s, tm, keys)) != FRAG_OK)
            return st;
        if (bp.fwd && (st = launch_wave_fused(bp, wv, mem, d, s, tm, keys, 2)) != FRAG_OK)
            return st;
        if (bp.fwd && (st = launch_wave_blocks(bp, wv, mem, d, s, tm)) != FRAG_OK)
            return st;
        if (bp.fwd && (st = launch_wave_blocks(bp, wv, mem, d, s, tm, true, rk)) != FRAG_OK)
            return st;
        if (!bp.fwd && !wv.chunks.empty()) { // decipher before the transform reads LL_L
            tm.begin();
            st = ctr_launch(d, keys, &clist, nullptr, s);
            tm.end(FRAG_KERNEL_CIPHER);
            if (st != FRAG_OK)
                return st;
        }
        if (!wv.units.empty()) {
            cudaError_t e = cudaMemsetAsync(mem + wv.done_off, 0, wv.queue_off + 256 - wv.done_off, s);
            if (e != cudaSuccess)
                return cuda_fail(e, "counter reset");
            DagWork w;
            std::memset(&w, 0, sizeof(w));
            w.jobs = (const LevelJob *)(mem + wv.jobs_off);
            w.units = (const DagUnit *)(mem + wv.units_off);
            w.total_units = wv.units.size();
            w.done = (unsigned *)(mem + wv.done_off);
            w.queue = (unsigned long long *)(mem + wv.queue_off);
            w.aes_tables = d.tables;
            w.round_keys = rk;
            w.err = d.err;
            w.spin_limit = kSpinLimit;
            uint32_t grid = 0;
            st = dag_grid(d, bp.fwd, w.total_units, &grid);
            if (bp.max_ctas)
                grid = std::min(grid, bp.max_ctas);
            if (st != FRAG_OK)
                return st;
            tm.begin();
            e = frag::launch_dag(bp.fwd, w, grid, s);
            tm.end(FRAG_KERNEL_LEVELS);
            if (e != cudaSuccess)
                return cuda_fail(e, "batch launch");
        }
        if (bp.fwd && !wv.chunks.empty()) { // encipher after the transform wrote LL_L
            tm.begin();
            st = ctr_launch(d, keys, &clist, nullptr, s);
            tm.end(FRAG_KERNEL_CIPHER);
            if (st != FRAG_OK)
                return st;
        }
        if (!bp.fwd && (st = launch_wave_blocks(bp, wv, mem, d, s, tm)) != FRAG_OK)
            return st;
        if (!bp.fwd && (st = launch_wave_blocks(bp, wv, mem, d, s, tm, true, rk)) != FRAG_OK)
            return st;
        if (!bp.fwd && (st = launch_wave_fused(bp, wv, mem, d, s, tm, keys, 2)) != FRAG_OK)
            return st;
        if (!bp.fwd && (st = launch_wave_fused(bp, wv, mem, d, s, tm, keys)) != FRAG_OK)
            return st;
    }
    return FRAG_OK;
}

// warps the fused launches of a batch keep resident
frag_status batch_fuse_slots(BatchPlan &bp, DeviceState &d)
{
    bool any = false, any2 = false;
    for (const Buf &b : bp.bufs) {
        any = any || (b.F1 != 0 && !b.block);
        any2 = any2 || b.F2 != 0;
    }
    frag_status st = FRAG_OK;
    if (any)
        st = fuse_slots(d, bp.fwd, false, bp.max_ctas, &bp.fuse_slots);
    if (st == FRAG_OK && any2)
        st = fuse_slots(d, bp.fwd, true, bp.max_ctas, &bp.fuse_slots2);
    return st;
}

frag_status run_batch_once(bool fwd, const frag_item *pi, const frag_ritem *ri, uint32_t count,
                           frag_key key, cudaStream_t s)
{
    if (key == nullptr)
        return fail(FRAG_EINVAL, "key is NULL");
    if (count == 0)
        return FRAG_OK;
    if ((fwd ? (const void *)pi : (const void *)ri) == nullptr)
        return fail(FRAG_EINVAL, "items is NULL");
    BatchPlan bp;
    frag_status st = plan_batch(fwd, pi, ri, count, bp);
    if (st != FRAG_OK || bp.bufs.empty())
        return st;
    DeviceState *d = nullptr;
    int dev = 0;
    if ((st = device_state(&d, &dev)) != FRAG_OK)
        return st;
    const uint32_t *rk = nullptr;
    if ((st = key_on_device(key, dev, &rk)) != FRAG_OK)
        return st;
    uint32_t grid = 0;
    if ((st = dag_grid(*d, fwd, ~0ull, &grid)) != FRAG_OK)
        return st;
    bp.resident_ctas = bp.max_ctas ? std::min(grid, bp.max_ctas) : grid;
    bp.sms = (uint64_t)d->sms;
    if ((st = batch_fuse_slots(bp, *d)) != FRAG_OK)
        return st;
    BatchPlan sizing = bp; // the layout does not depend on the scratch base
    fill_batch(sizing, nullptr);
    uint8_t *mem = nullptr;
    cudaError_t e = pool_malloc((void **)&mem, batch_mem_bytes(sizing), s);
    if (e != cudaSuccess)
        return cuda_fail(e, "pool_malloc(batch)");
    fill_batch(bp, mem);
    st = upload_batch(bp, mem, s, true);
    if (st == FRAG_OK)
        st = launch_batch(bp, mem, *d, rk, frag::aes::keys_from_words(key->rk), s);
    cudaFreeAsync(mem, s); // released once the launches have completed
    return st;
}

} // namespace

struct frag_batch_s {
    int device = 0;
    BatchPlan bp;
    uint8_t *mem = nullptr; // [scratch][descriptors, counters, queue heads]
    bool timing = false;
    std::vector<TimedLaunch> timed; // event pairs of timed runs not yet read
};

namespace {

frag_status create_batch(bool fwd, const frag_item *pi, const frag_ritem *ri, uint32_t count,
                         frag_batch *out)
{
    if (out == nullptr)
        return fail(FRAG_EINVAL, "out is NULL");
    *out = nullptr;
    if ((fwd ? (const void *)pi : (const void *)ri) == nullptr && count != 0)
        return fail(FRAG_EINVAL, "items is NULL");
    frag_batch bt = new (std::nothrow) frag_batch_s();
    if (bt == nullptr)
        return fail(FRAG_ENOMEM, "out of host memory");
    frag_status st = plan_batch(fwd, pi, ri, count, bt->bp);
    DeviceState *d = nullptr;
    if (st == FRAG_OK)
        st = device_state(&d, &bt->device);
    uint32_t grid = 0;
    if (st == FRAG_OK && (st = dag_grid(*d, fwd, ~0ull, &grid)) == FRAG_OK) {
        bt->bp.resident_ctas = bt->bp.max_ctas ? std::min(grid, bt->bp.max_ctas) : grid;
        bt->bp.sms = (uint64_t)d->sms;
    }
    if (st == FRAG_OK)
        st = batch_fuse_slots(bt->bp, *d);
    if (st == FRAG_OK && !bt->bp.bufs.empty()) {
        BatchPlan sizing = bt->bp;
        fill_batch(sizing, nullptr);
        cudaError_t e = cudaMalloc((void **)&bt->mem, batch_mem_bytes(sizing));
        if (e != cudaSuccess) {
            bt->mem = nullptr;
            st = cuda_fail(e, "cudaMalloc(batch)");
        } else {
            fill_batch(bt->bp, bt->mem);
            st = upload_batch(bt->bp, bt->mem, nullptr, false);
        }
    }
    if (st != FRAG_OK) {
        if (bt->mem)
            cudaFree(bt->mem);
        delete bt;
        return st;
    }
    *out = bt;
    return FRAG_OK;
}

} // namespace

// Accessors for other translation units of this library (no new behaviour).
namespace frag {
const uint32_t *host_aes_words() { return aes_host().words; }
void host_expand_key(const uint8_t key[16], uint32_t rk[44]) { expand_key(key, rk); }
frag_status plan_job(frag_plan plan, uint64_t nonce, uint64_t n, Job &j)
{
    return fill_job(plan, nonce, n, j);
}
frag_status report(frag_status st, const char *msg) { return fail(st, "%s", msg); }
frag_status report_cuda(cudaError_t e, const char *what) { return cuda_fail(e, what); }

// A protect item of the allocation-free call whose levels all run in the
// first fused pass (1..3 levels, under FRAG_PATH_AUTO's width and alignment
// conditions, whatever the plan's path): its fused descriptor (schedule
// fields 0) and the CTR chunk of its private fragment, the ones a batch
// builds for it; *cells = H * W, the batch's ordering key.  False: the
// item is not one (the tile kernel takes it).
bool noalloc_fused_item(frag_plan plan, const frag_item &it, FuseBuf &f, CtrChunk &c,
                        uint64_t *cells)
{
    if (plan->block || plan->packed || plan->levels > kFuseMaxLevels || it.nbytes == 0)
        return false;
    const uint64_t H = rows_for(it.nbytes, plan->width, plan->levels);
    if (H > 0xFFFFFFFFull)
        return false;
    Buf b;
    std::memset(&b, 0, sizeof(b));
    b.W = plan->width;
    b.L = plan->levels;
    b.H = (uint32_t)H;
    b.n = it.nbytes;
    b.nonce = it.nonce;
    b.in = (const uint8_t *)it.d_in;
    b.priv = (uint8_t *)it.d_private;
    b.pub = (uint8_t *)it.d_public;
    fused_split(true, b, FRAG_PATH_AUTO);
    if (b.F1 != b.L || b.F2 != 0 || !ctr_pass(b))
        return false;
    f = fuse_buf(true, b, 1);
    c = ctr_fragment(true, b);
    *cells = H * (uint64_t)b.W;
    return true;
}

// a batch's schedule of one fused protect launch over f[0..n) for `slots`
// resident warps (plan_rows: the level-0 rows of a unit, 0 = adaptive);
// returns the launch's units
uint64_t noalloc_fuse_schedule(FuseBuf *f, size_t n, uint64_t slots, uint32_t plan_rows)
{
    return fuse_schedule(f, n, std::max<uint64_t>(1, slots), plan_rows, true);
}

// a batch's choice for the fused protect of f[0..n): one launch per level
// count (true) or one launch
bool noalloc_split_fused(const FuseBuf *f, size_t n, uint64_t slots)
{
    return fuse_split_by_levels(f, n, std::max<uint64_t>(1, slots));
}
} // namespace frag

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int frag_abi_version(void) { return FRAG_ABI_VERSION; }

frag_status frag_get_error(char *buf, size_t len)
{
    if (buf == nullptr || len == 0)
        return FRAG_EINVAL;
    std::snprintf(buf, len, "%s", g_err);
    return FRAG_OK;
}

frag_status frag_plan_create(frag_plan *out, uint32_t width, uint32_t levels, frag_filter filter)
{
    if (out == nullptr)
        return fail(FRAG_EINVAL, "out is NULL");
    *out = nullptr;
    if (filter != FRAG_FILTER_LEGALL53)
        return fail(FRAG_EUNSUPPORTED, "unknown filter %d", (int)filter);
    if (levels == 0 || levels > kMaxLevels)
        return fail(FRAG_EINVAL, "levels must be 1..%u, got %u", kMaxLevels, levels);
    if (width == 0 || (width % (1u << levels)) != 0)
        return fail(FRAG_EINVAL, "width %u is not a positive multiple of 2^%u", width, levels);
    frag_plan p = new (std::nothrow) frag_plan_s();
    if (p == nullptr)
        return fail(FRAG_ENOMEM, "out of host memory");
    p->width = width;
    p->levels = levels;
    *out = p;
    return FRAG_OK;
}

frag_status frag_plan_destroy(frag_plan plan)
{
    delete plan;
    return FRAG_OK;
}

frag_status frag_plan_sizes(frag_plan plan, uint64_t nbytes, uint32_t *height,
                            uint64_t *private_bytes, uint64_t *public_bytes)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    const uint64_t H = rows_for(nbytes, plan->width, plan->levels, plan->block);
    if (H > 0xFFFFFFFFull)
        return fail(FRAG_EINVAL, "buffer too tall for width %u", plan->width);
    const uint64_t pb = 2 * (H >> plan->levels) * (uint64_t)(plan->width >> plan->levels);
    if (height)
        *height = (uint32_t)H;
    if (plan->packed) {
        uint64_t a, b, c;
        packed_sizes(H, plan->width, &a, &b, &c);
        if (private_bytes)
            *private_bytes = a;
        if (public_bytes)
            *public_bytes = b + c;
        return FRAG_OK;
    }
    if (private_bytes)
        *private_bytes = pb;
    if (public_bytes)
        *public_bytes = 2 * H * (uint64_t)plan->width - pb;
    return FRAG_OK;
}

frag_status frag_plan_fragment_sizes(frag_plan plan, uint64_t nbytes, uint64_t sizes[3])
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (sizes == nullptr)
        return fail(FRAG_EINVAL, "sizes is NULL");
    uint32_t H = 0;
    uint64_t pb = 0, ub = 0;
    if ((st = frag_plan_sizes(plan, nbytes, &H, &pb, &ub)) != FRAG_OK)
        return st;
    if (plan->packed) {
        packed_sizes(H, plan->width, &sizes[0], &sizes[1], &sizes[2]);
        return FRAG_OK;
    }
    // the detail bands of level L lead the public fragment
    const uint64_t first = 3 * ll_bytes(H, plan->width, plan->levels);
    sizes[0] = pb;
    sizes[1] = first;
    sizes[2] = ub - first;
    return FRAG_OK;
}

frag_status frag_plan_set_schedule(frag_plan plan, uint32_t seg_rows, uint32_t ctas)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (seg_rows && (seg_rows < 16 || seg_rows > 256 || (seg_rows & (seg_rows - 1))))
        return fail(FRAG_EINVAL, "seg_rows %u must be 0 or a power of two in 16..256", seg_rows);
    plan->seg_rows = seg_rows;
    plan->max_ctas = ctas;
    return FRAG_OK;
}

frag_status frag_plan_get_schedule(frag_plan plan, uint32_t *seg_rows, uint32_t *ctas)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (seg_rows)
        *seg_rows = plan->seg_rows;
    if (ctas)
        *ctas = plan->max_ctas;
    return FRAG_OK;
}

frag_status frag_plan_set_block(frag_plan plan, uint32_t block)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (block != 0) {
        if (block < (1u << plan->levels) || plan->width % block != 0)
            return fail(FRAG_EINVAL, "block %u must be >= 2^levels and divide the width %u", block,
                        plan->width);
        if (block != frag::kBlockSide || plan->levels > 3)
            return fail(FRAG_EUNSUPPORTED, "the block mode runs 8 x 8 blocks with up to 3 levels");
    }
    if (plan->packed && block != frag::kBlockSide)
        return fail(FRAG_EINVAL, "the plan stores packed fragments: clear that first");
    plan->block = block;
    return FRAG_OK;
}

frag_status frag_plan_set_packed(frag_plan plan, uint32_t packed)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (packed && (plan->block != frag::kBlockSide || plan->levels != 2))
        return fail(FRAG_EUNSUPPORTED, "packed fragments are the thesis's storage of 8 x 8 blocks at two "
                                       "levels (frag_plan_set_block(plan, 8) on a 2-level plan first)");
    if (!packed && plan->keyed)
        return fail(FRAG_EINVAL, "the plan protects its public fragments: clear that first");
    plan->packed = packed ? 1u : 0u;
    return FRAG_OK;
}

frag_status frag_plan_set_protect_public(frag_plan plan, uint32_t on)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (on && !plan->packed)
        return fail(FRAG_EUNSUPPORTED, "the keyed protection of the public fragments works on the packed "
                                       "fragments (frag_plan_set_packed(plan, 1) first)");
    plan->keyed = on ? 1u : 0u;
    return FRAG_OK;
}

frag_status frag_plan_get_protect_public(frag_plan plan, uint32_t *on)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (on == nullptr)
        return fail(FRAG_EINVAL, "on is NULL");
    *on = plan->keyed;
    return FRAG_OK;
}

frag_status frag_plan_get_packed(frag_plan plan, uint32_t *packed)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (packed == nullptr)
        return fail(FRAG_EINVAL, "packed is NULL");
    *packed = plan->packed;
    return FRAG_OK;
}

frag_status frag_plan_get_block(frag_plan plan, uint32_t *block)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (block == nullptr)
        return fail(FRAG_EINVAL, "block is NULL");
    *block = plan->block;
    return FRAG_OK;
}

frag_status frag_plan_set_path(frag_plan plan, frag_path path)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (path != FRAG_PATH_AUTO && path != FRAG_PATH_LEVELS && path != FRAG_PATH_FUSED_CIPHER)
        return fail(FRAG_EINVAL, "unknown path %d", (int)path);
    plan->path = (uint32_t)path;
    return FRAG_OK;
}

frag_status frag_plan_get_path(frag_plan plan, frag_path *path)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (path == nullptr)
        return fail(FRAG_EINVAL, "path is NULL");
    *path = (frag_path)plan->path;
    return FRAG_OK;
}

frag_status frag_key_create(frag_key *out, const uint8_t key[16])
{
    if (out == nullptr || key == nullptr)
        return fail(FRAG_EINVAL, "NULL argument");
    *out = nullptr;
    frag_key k = new (std::nothrow) frag_key_s();
    if (k == nullptr)
        return fail(FRAG_ENOMEM, "out of host memory");
    expand_key(key, k->rk);
    int dev = 0;
    DeviceState *d = nullptr;
    const uint32_t *rk = nullptr;
    frag_status st = device_state(&d, &dev);
    if (st == FRAG_OK)
        st = key_on_device(k, dev, &rk);
    if (st != FRAG_OK) {
        delete k;
        return st;
    }
    *out = k;
    return FRAG_OK;
}

frag_status frag_key_destroy(frag_key key)
{
    if (key == nullptr)
        return FRAG_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : key->on_device) {
        cudaSetDevice(kv.first);
        cudaFree(kv.second);
    }
    cudaSetDevice(cur);
    delete key;
    return FRAG_OK;
}

frag_status frag_protect(frag_plan plan, frag_key key, uint64_t nonce, const void *d_in,
                         uint64_t nbytes, void *d_private, void *d_public, frag_stream stream)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (key == nullptr)
        return fail(FRAG_EINVAL, "key is NULL");
    if (nbytes == 0)
        return FRAG_OK;
    if (d_in == nullptr || d_private == nullptr || d_public == nullptr)
        return fail(FRAG_EINVAL, "NULL buffer");
    const uint64_t H = rows_for(nbytes, plan->width, plan->levels, plan->block);
    if (H > 0xFFFFFFFFull)
        return fail(FRAG_EINVAL, "buffer too tall for width %u", plan->width);
    Buf b;
    std::memset(&b, 0, sizeof(b));
    b.W = plan->width;
    b.L = plan->levels;
    b.block = plan->block;
    b.packed = plan->packed;
    b.keyed = plan->keyed;
    b.H = (uint32_t)H;
    b.n = nbytes;
    b.nonce = nonce;
    b.in = (const uint8_t *)d_in;
    b.priv = (uint8_t *)d_private;
    b.pub = (uint8_t *)d_public;
    return run_single(true, plan, key, b, (cudaStream_t)stream);
}

frag_status frag_aes128_ctr(frag_key key, uint64_t nonce, const void *d_in, void *d_out, uint64_t nbytes,
                            frag_stream stream)
{
    if (key == nullptr)
        return fail(FRAG_EINVAL, "key is NULL");
    if (nbytes == 0)
        return FRAG_OK;
    if (d_in == nullptr || d_out == nullptr)
        return fail(FRAG_EINVAL, "NULL buffer");
    DeviceState *d = nullptr;
    int dev = 0;
    frag_status st = device_state(&d, &dev);
    if (st != FRAG_OK)
        return st;
    const uint32_t *rk = nullptr;
    if ((st = key_on_device(key, dev, &rk)) != FRAG_OK)
        return st;
    // the whole buffer as one fragment of the CTR pass
    frag::CtrChunk c;
    std::memset(&c, 0, sizeof(c));
    c.in = (const uint8_t *)d_in;
    c.out = (uint8_t *)d_out;
    c.nonce = nonce;
    c.bytes = nbytes;
    c.nblocks = (nbytes + 15) / 16;
    return ctr_launch(*d, frag::aes::keys_from_words(key->rk), nullptr, &c, (cudaStream_t)stream);
}

frag_status frag_aes128_ctr_bitsliced(frag_key key, uint64_t nonce, const void *d_in, void *d_out,
                                      uint64_t nbytes, frag_stream stream)
{
    if (key == nullptr)
        return fail(FRAG_EINVAL, "key is NULL");
    if (nbytes == 0)
        return FRAG_OK;
    if (d_in == nullptr || d_out == nullptr)
        return fail(FRAG_EINVAL, "NULL buffer");
    DeviceState *d = nullptr;
    int dev = 0;
    frag_status st = device_state(&d, &dev);
    if (st != FRAG_OK)
        return st;
    // the key schedule sliced into bit planes: word b of byte p of round r is
    // all-ones when bit b of that byte is set; 0x63 (the S-box's affine
    // constant, which the circuit leaves out) folded into rounds 1..10
    static_assert(sizeof(frag::BsCtrWork) < 32000, "the sliced key schedule travels in the kernel parameter");
    frag::BsCtrWork w;
    std::memset(&w, 0, sizeof(w));
    w.in = (const uint8_t *)d_in;
    w.out = (uint8_t *)d_out;
    w.bytes = nbytes;
    w.nonce = nonce;
    const uint64_t nblocks = (nbytes + 15) / 16;
    w.nchunks = (nblocks + frag::bs::kChunkBlocks - 1) / frag::bs::kChunkBlocks;
    for (int r = 0; r < 11; ++r)
        for (int p = 0; p < 16; ++p) {
            const uint32_t byte = ((key->rk[4 * r + p / 4] >> (24 - 8 * (p % 4))) & 0xffu) ^ (r ? 0x63u : 0u);
            for (int b = 0; b < 8; ++b)
                w.w[r][8 * p + b] = ((byte >> b) & 1u) ? 0xffffffffu : 0u;
        }
    const cudaError_t e = frag::launch_ctr_bs(w, (cudaStream_t)stream);
    return e == cudaSuccess ? FRAG_OK : cuda_fail(e, "bitsliced CTR launch");
}

frag_status frag_recover(frag_plan plan, frag_key key, uint64_t nonce, const void *d_private,
                         const void *d_public, uint64_t nbytes, void *d_out, frag_stream stream)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (key == nullptr)
        return fail(FRAG_EINVAL, "key is NULL");
    if (nbytes == 0)
        return FRAG_OK;
    if (d_private == nullptr || d_public == nullptr || d_out == nullptr)
        return fail(FRAG_EINVAL, "NULL buffer");
    const uint64_t H = rows_for(nbytes, plan->width, plan->levels, plan->block);
    if (H > 0xFFFFFFFFull)
        return fail(FRAG_EINVAL, "buffer too tall for width %u", plan->width);
    Buf b;
    std::memset(&b, 0, sizeof(b));
    b.W = plan->width;
    b.L = plan->levels;
    b.block = plan->block;
    b.packed = plan->packed;
    b.keyed = plan->keyed;
    b.H = (uint32_t)H;
    b.n = nbytes;
    b.nonce = nonce;
    b.priv_in = (const uint8_t *)d_private;
    b.pub_in = (const uint8_t *)d_public;
    b.out = (uint8_t *)d_out;
    return run_single(false, plan, key, b, (cudaStream_t)stream);
}

frag_status frag_protect_host(frag_plan plan, frag_key key, uint64_t nonce, const void *h_in,
                              uint64_t nbytes, void *h_private, void *h_public,
                              frag_stream stream)
{
    uint64_t pb = 0, ub = 0;
    frag_status st = frag_plan_sizes(plan, nbytes, nullptr, &pb, &ub);
    if (st != FRAG_OK || nbytes == 0)
        return st;
    if (key == nullptr || h_in == nullptr || h_private == nullptr || h_public == nullptr)
        return fail(FRAG_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    bool banded = false;
    st = run_host_banded(true, plan, key, nonce, (const uint8_t *)h_in, nullptr, (uint8_t *)h_private,
                         (uint8_t *)h_public, nbytes, s, &banded);
    if (st != FRAG_OK || banded)
        return st;
    uint8_t *mem = nullptr;
    cudaError_t e = pool_malloc((void **)&mem, nbytes + pb + ub + 512, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "pool_malloc(host-form buffers)");
    uint8_t *d_in = mem, *d_priv = mem + ((nbytes + 255) / 256 * 256);
    uint8_t *d_pub = d_priv + ((pb + 255) / 256 * 256);
    e = cudaMemcpyAsync(d_in, h_in, nbytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        st = frag_protect(plan, key, nonce, d_in, nbytes, d_priv, d_pub, stream);
        if (st == FRAG_OK) {
            e = cudaMemcpyAsync(h_private, d_priv, pb, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_public, d_pub, ub, cudaMemcpyDeviceToHost, s);
        }
    }
    cudaFreeAsync(mem, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (st != FRAG_OK)
        return st;
    if (e != cudaSuccess)
        return cuda_fail(e, "host protect copies");
    if (e2 != cudaSuccess)
        return cuda_fail(e2, "cudaStreamSynchronize");
    return FRAG_OK;
}

frag_status frag_recover_host(frag_plan plan, frag_key key, uint64_t nonce, const void *h_private,
                              const void *h_public, uint64_t nbytes, void *h_out,
                              frag_stream stream)
{
    uint64_t pb = 0, ub = 0;
    frag_status st = frag_plan_sizes(plan, nbytes, nullptr, &pb, &ub);
    if (st != FRAG_OK || nbytes == 0)
        return st;
    if (key == nullptr || h_out == nullptr || h_private == nullptr || h_public == nullptr)
        return fail(FRAG_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    bool banded = false;
    st = run_host_banded(false, plan, key, nonce, (const uint8_t *)h_private, (const uint8_t *)h_public,
                         (uint8_t *)h_out, nullptr, nbytes, s, &banded);
    if (st != FRAG_OK || banded)
        return st;
    uint8_t *mem = nullptr;
    cudaError_t e = pool_malloc((void **)&mem, nbytes + pb + ub + 512, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "pool_malloc(host-form buffers)");
    uint8_t *d_out = mem, *d_priv = mem + ((nbytes + 255) / 256 * 256);
    uint8_t *d_pub = d_priv + ((pb + 255) / 256 * 256);
    e = cudaMemcpyAsync(d_priv, h_private, pb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pub, h_public, ub, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        st = frag_recover(plan, key, nonce, d_priv, d_pub, nbytes, d_out, stream);
        if (st == FRAG_OK)
            e = cudaMemcpyAsync(h_out, d_out, nbytes, cudaMemcpyDeviceToHost, s);
    }
    cudaFreeAsync(mem, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (st != FRAG_OK)
        return st;
    if (e != cudaSuccess)
        return cuda_fail(e, "host recover copies");
    if (e2 != cudaSuccess)
        return cuda_fail(e2, "cudaStreamSynchronize");
    return FRAG_OK;
}

frag_status frag_protect_batch(const frag_item *items, uint32_t count, frag_key key,
                               frag_stream stream)
{
    return run_batch_once(true, items, nullptr, count, key, (cudaStream_t)stream);
}

frag_status frag_recover_batch(const frag_ritem *items, uint32_t count, frag_key key,
                               frag_stream stream)
{
    return run_batch_once(false, nullptr, items, count, key, (cudaStream_t)stream);
}

frag_status frag_batch_create_protect(frag_batch *out, const frag_item *items, uint32_t count)
{
    return create_batch(true, items, nullptr, count, out);
}

frag_status frag_batch_create_recover(frag_batch *out, const frag_ritem *items, uint32_t count)
{
    return create_batch(false, nullptr, items, count, out);
}

frag_status frag_batch_run(frag_batch batch, frag_key key, frag_stream stream)
{
    if (batch == nullptr || key == nullptr)
        return fail(FRAG_EINVAL, "NULL argument");
    if (batch->bp.bufs.empty())
        return FRAG_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev != batch->device)
        return fail(FRAG_EINVAL, "batch was created on device %d, current is %d", batch->device,
                    dev);
    DeviceState *d = nullptr;
    frag_status st = device_state(&d, nullptr);
    if (st != FRAG_OK)
        return st;
    const uint32_t *rk = nullptr;
    if ((st = key_on_device(key, dev, &rk)) != FRAG_OK)
        return st;
    return launch_batch(batch->bp, batch->mem, *d, rk, frag::aes::keys_from_words(key->rk),
                        (cudaStream_t)stream, batch->timing ? &batch->timed : nullptr);
}

frag_status frag_batch_set_timing(frag_batch batch, int enable)
{
    if (batch == nullptr)
        return fail(FRAG_EINVAL, "batch is NULL");
    batch->timing = enable != 0;
    return FRAG_OK;
}

frag_status frag_batch_launch_times(frag_batch batch, double *ms, uint32_t *launches)
{
    if (batch == nullptr)
        return fail(FRAG_EINVAL, "batch is NULL");
    double t[FRAG_KERNEL_KINDS] = {0};
    uint32_t n[FRAG_KERNEL_KINDS] = {0};
    frag_status st = FRAG_OK;
    for (const TimedLaunch &x : batch->timed) {
        float v = 0.f;
        cudaError_t e = cudaEventSynchronize(x.b);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&v, x.a, x.b);
        if (e != cudaSuccess && st == FRAG_OK)
            st = cuda_fail(e, "launch timing");
        if (x.kind < FRAG_KERNEL_KINDS) {
            t[x.kind] += v;
            n[x.kind] += 1;
        }
        cudaEventDestroy(x.a);
        cudaEventDestroy(x.b);
    }
    batch->timed.clear();
    for (int k = 0; k < FRAG_KERNEL_KINDS; ++k) {
        if (ms)
            ms[k] = t[k];
        if (launches)
            launches[k] = n[k];
    }
    return st;
}

frag_status frag_batch_info(frag_batch batch, uint32_t *launches, uint64_t *scratch_bytes)
{
    if (batch == nullptr)
        return fail(FRAG_EINVAL, "batch is NULL");
    uint32_t n = 0;
    for (const auto &wv : batch->bp.waves)
        n += (wv.units.empty() ? 0 : 1) + (wv.chunks.empty() ? 0 : 1) +
             (wv.fbufs.empty() ? 0 : (uint32_t)wv.fgroups.size() - 1) + (wv.bbufs.empty() ? 0 : 1) +
             (wv.fbufs2.empty() ? 0 : 1) + (wv.pbufs.empty() ? 0 : 1);
    if (launches)
        *launches = n;
    if (scratch_bytes)
        *scratch_bytes = batch->mem ? batch_mem_bytes(batch->bp) : 0;
    return FRAG_OK;
}

frag_status frag_batch_destroy(frag_batch batch)
{
    if (batch == nullptr)
        return FRAG_OK;
    for (const TimedLaunch &x : batch->timed) {
        cudaEventDestroy(x.a);
        cudaEventDestroy(x.b);
    }
    if (batch->mem)
        cudaFree(batch->mem);
    delete batch;
    return FRAG_OK;
}

frag_status frag_sync_status(frag_stream stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamSynchronize");
    DeviceState *d = nullptr;
    frag_status st = device_state(&d, nullptr);
    if (st != FRAG_OK)
        return st;
    int word = 0;
    if ((e = cudaMemcpy(&word, d->err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "read error word");
    if (word == 0)
        return FRAG_OK;
    cudaMemset(d->err, 0, sizeof(int));
    if (word == 3)
        return fail(FRAG_ETIMEOUT, "a bounded wait for another unit's output ran out");
    if (word == 4)
        return fail(FRAG_ETIMEOUT, "a bounded wait for a shared-memory stage ran out");
    if (word == 5)
        return fail(FRAG_EDEVICE, "a coefficient did not fit its width in the packed fragments");
    if (word == 7)
        return fail(FRAG_ETIMEOUT, "a bounded wait for a TMA box load ran out");
    return fail(FRAG_EDEVICE, "kernel reported inconsistent work descriptor (code %d)", word);
}

frag_status frag_check_wait_timeout(uint32_t polls, frag_stream stream)
{
    if (polls == 0)
        return fail(FRAG_EINVAL, "polls must be positive");
    DeviceState *d = nullptr;
    frag_status st = device_state(&d, nullptr);
    if (st != FRAG_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *ctr = nullptr;
    cudaError_t e = pool_malloc((void **)&ctr, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return cuda_fail(e, "pool_malloc(counter)");
    if ((e = cudaMemsetAsync(ctr, 0, sizeof(unsigned), s)) != cudaSuccess)
        st = cuda_fail(e, "counter reset");
    else if ((e = frag::launch_stall_probe(ctr, polls, d->err, s)) != cudaSuccess)
        st = cuda_fail(e, "wait probe launch");
    cudaFreeAsync(ctr, s);
    return st;
}

frag_status frag_check_box_wait_timeout(uint32_t polls, frag_stream stream)
{
    if (polls == 0)
        return fail(FRAG_EINVAL, "polls must be positive");
    DeviceState *d = nullptr;
    frag_status st = device_state(&d, nullptr);
    if (st != FRAG_OK)
        return st;
    cudaError_t e = frag::launch_box_stall_probe(polls, d->err, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "box wait probe launch");
    return FRAG_OK;
}

} // extern "C"
