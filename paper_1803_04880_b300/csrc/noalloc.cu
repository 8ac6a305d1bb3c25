// noalloc.cu -- batched protect that allocates no memory.
//
// Some callers cannot call cudaMalloc: a plug-in whose host process owns all
// device memory through its own pool (a framework's caching allocator, or a
// reservation made once at start-up), or a latency-critical path that must not
// take the implicit synchronisation and unbounded latency of a driver
// allocation.  For them frag_protect_batch_noalloc runs, for every item whose
// levels all fit the first fused pass (1..3 levels, aligned buffers), the
// same two launches as frag_protect_batch (the fused pass, then the CTR pass
// over the private fragments), and for the rest (4 or 5 levels, or buffers
// the fused pass does not take) the shared-memory tile kernel, which keeps
// every level of a tile on chip and so needs no level scratch.  Everything
// those launches read besides the caller's buffers (AES tables, round keys,
// the error word, the descriptors, the tile prefix and the queue head) lives
// in one file-scope static device array of fixed size, and the host-side
// staging lives in static host arrays.  Neither this file nor the calls it
// makes allocate host heap or device memory.
#include "aes_tt.cuh"
#include "frag.h"
#include "frag_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

namespace frag {
frag_status plan_job(frag_plan plan, uint64_t nonce, uint64_t n, Job &j);
frag_status report(frag_status st, const char *msg);
frag_status report_cuda(cudaError_t e, const char *what);
bool noalloc_fused_item(frag_plan plan, const frag_item &it, FuseBuf &f, CtrChunk &c,
                        uint64_t *cells);
uint64_t noalloc_fuse_schedule(FuseBuf *f, size_t n, uint64_t slots, uint32_t plan_rows);
bool noalloc_split_fused(const FuseBuf *f, size_t n, uint64_t slots);
} // namespace frag

namespace {

using frag::Job;
using frag::Work;

constexpr uint32_t kMaxItems = FRAG_NOALLOC_MAX_ITEMS;
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// layout of the static scratch, in bytes
constexpr size_t kOffHead = 0;                                   // queue head (8 B), error word (4 B)
constexpr size_t kOffTables = 256;                               // AES T-tables + S-box words
constexpr size_t kOffKeys = kOffTables + align256(sizeof(uint32_t) * frag::kAesWords);
constexpr size_t kOffStart = kOffKeys + 256;                     // 44 round-key words
constexpr size_t kOffJobs = kOffStart + align256(sizeof(uint64_t) * (kMaxItems + 1));
constexpr size_t kOffFuse = kOffJobs + align256(sizeof(Job) * kMaxItems); // fused descriptors
constexpr size_t kOffChunks = kOffFuse + align256(sizeof(frag::FuseBuf) * kMaxItems);
constexpr size_t kOffTurns = kOffChunks + align256(sizeof(frag::CtrChunk) * kMaxItems);
constexpr size_t kScratchBytes = kOffTurns + align256(sizeof(uint64_t) * (kMaxItems + 1));
static_assert(kScratchBytes <= 512 * 1024, "scratch must stay modest");

// The scratch.  Every GPU that loads the library holds it until the process
// exits.  In host code its name is only a host-side stand-in for the symbol:
// the device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool ready;
    unsigned char *base; // device address of g_noalloc_scratch on this device
    int sms;
    bool shaped;         // the launch shapes below are known
    int fuse_ctas;       // fused protect launch: CTAs an SM holds
    int fuse_warps;      //   and warps a CTA
    int ctr_ctas;        // CTR launch: CTAs an SM holds
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_mu; // guards g_setup and the host staging below

// host staging (static: filled under g_mu, copied to the device per call)
Job h_jobs[kMaxItems];
uint64_t h_start[kMaxItems + 1];
uint64_t h_cost[kMaxItems];
uint32_t h_order[kMaxItems];
Job h_sorted[kMaxItems];
uint32_t h_rk[44];
frag::FuseBuf h_fuse[kMaxItems], h_fuse_sorted[kMaxItems];
frag::CtrChunk h_chunk[kMaxItems], h_chunk_sorted[kMaxItems];
uint64_t h_turns[kMaxItems + 1];
uint64_t h_fcost[kMaxItems];
uint32_t h_forder[kMaxItems];
uint32_t h_group[frag::kFuseMaxLevels + 1];      // fused launches: h_fuse_sorted[h_group[g] ..
uint64_t h_group_units[frag::kFuseMaxLevels];    //   h_group[g + 1]) and their units

// Once per device, with that device current: look up the scratch's device
// address, copy the AES tables into it and zero the queue head and error
// word (synchronously).
frag_status setup_device(int dev, DeviceSetup **out)
{
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        unsigned char *base = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&base, g_noalloc_scratch);
        if (e != cudaSuccess)
            return frag::report_cuda(e, "cudaGetSymbolAddress(no-alloc scratch)");
        if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) !=
            cudaSuccess)
            return frag::report_cuda(e, "cudaDeviceGetAttribute");
        if ((e = cudaMemcpy(base + kOffTables, frag::host_aes_words(),
                            sizeof(uint32_t) * frag::kAesWords, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return frag::report_cuda(e, "copy of AES tables into the no-alloc scratch");
        if ((e = cudaMemset(base + kOffHead, 0, 256)) != cudaSuccess)
            return frag::report_cuda(e, "clearing the no-alloc scratch");
        d.base = base;
        d.ready = true;
    }
    *out = &d;
    return FRAG_OK;
}

// Once per device: the occupancy of the fused protect and CTR launches
// (queries that allocate nothing).
frag_status device_shapes(DeviceSetup &d)
{
    if (d.shaped)
        return FRAG_OK;
    cudaError_t e = frag::fuse_shape(true, false, false, &d.fuse_ctas, &d.fuse_warps);
    if (e == cudaSuccess)
        e = frag::ctr_occupancy(&d.ctr_ctas);
    if (e != cudaSuccess)
        return frag::report_cuda(e, "frag_protect_batch_noalloc: occupancy query");
    d.fuse_ctas = std::max(d.fuse_ctas, 1);
    d.fuse_warps = std::max(d.fuse_warps, 1);
    d.ctr_ctas = std::max(d.ctr_ctas, 1);
    d.shaped = true;
    return FRAG_OK;
}

} // namespace

extern "C" frag_status frag_protect_batch_noalloc(const frag_item *items, uint32_t count,
                                                  const uint8_t key[16], frag_stream stream)
{
    if (key == nullptr)
        return frag::report(FRAG_EINVAL, "frag_protect_batch_noalloc: key is NULL");
    if (count > kMaxItems) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "frag_protect_batch_noalloc: %u items exceed the static scratch limit of "
                      "%u items per call",
                      count, kMaxItems);
        return frag::report(FRAG_EINVAL, msg);
    }
    if (count == 0)
        return FRAG_OK;
    if (items == nullptr)
        return frag::report(FRAG_EINVAL, "frag_protect_batch_noalloc: items is NULL");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return frag::report_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return frag::report(FRAG_EUNSUPPORTED, "frag_protect_batch_noalloc: device index too high");

    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSetup *d = nullptr;
    frag_status st = setup_device(dev, &d);
    if (st != FRAG_OK)
        return st;

    // the items the fused pass takes whole, and tile jobs for the rest
    uint32_t nj = 0, nf = 0;
    size_t smem = 0;
    for (uint32_t i = 0; i < count; ++i) {
        if (items[i].plan == nullptr)
            return frag::report(FRAG_EINVAL, "frag_protect_batch_noalloc: an item has no plan");
        if (items[i].nbytes == 0)
            continue;
        if (!items[i].d_in || !items[i].d_private || !items[i].d_public)
            return frag::report(FRAG_EINVAL, "frag_protect_batch_noalloc: NULL buffer");
        if (frag::noalloc_fused_item(items[i].plan, items[i], h_fuse[nf], h_chunk[nf],
                                     &h_fcost[nf])) {
            h_forder[nf] = nf;
            ++nf;
            continue;
        }
        Job &j = h_jobs[nj];
        if ((st = frag::plan_job(items[i].plan, items[i].nonce, items[i].nbytes, j)) != FRAG_OK)
            return st;
        j.in = (const uint8_t *)items[i].d_in;
        j.priv = (uint8_t *)items[i].d_private;
        j.pub = (uint8_t *)items[i].d_public;
        h_cost[nj] = (uint64_t)j.tiles_x * j.tiles_y * (uint64_t)j.tile * j.tile;
        h_order[nj] = nj;
        smem = std::max(smem, frag::tile_smem_bytes(j.L));
        ++nj;
    }
    if (nj + nf == 0)
        return FRAG_OK;
    if ((st = device_shapes(*d)) != FRAG_OK)
        return st;
    // both lists most costly first (the order rule of frag_protect_batch),
    // sorted in place (no temporary buffer); ties keep the caller's order
    std::sort(h_order, h_order + nj, [](uint32_t a, uint32_t b) {
        return h_cost[a] != h_cost[b] ? h_cost[a] > h_cost[b] : a < b;
    });
    // the fused items in one launch, or (as a batch decides) one launch per
    // level count, each count's items together
    const uint64_t fslots = (uint64_t)d->sms * d->fuse_ctas * d->fuse_warps;
    const bool split = nf > 1 && frag::noalloc_split_fused(h_fuse, nf, fslots);
    std::sort(h_forder, h_forder + nf, [split](uint32_t a, uint32_t b) {
        if (split && h_fuse[a].F != h_fuse[b].F)
            return h_fuse[a].F > h_fuse[b].F;
        return h_fcost[a] != h_fcost[b] ? h_fcost[a] > h_fcost[b] : a < b;
    });
    h_start[0] = 0;
    for (uint32_t k = 0; k < nj; ++k) {
        h_sorted[k] = h_jobs[h_order[k]];
        h_start[k + 1] = h_start[k] + (uint64_t)h_sorted[k].tiles_x * h_sorted[k].tiles_y;
    }
    // the fused launches' units and the CTR launch's warp turns, as a batch
    // schedules them: units for the resident warps of each fused launch;
    // turns of kCtrTurn blocks, doubled (up to 128x) while the fragments keep
    // more than 4 turns a resident warp of the CTR launch
    uint64_t turn = frag::kCtrTurn;
    uint32_t ngroups = 0;
    if (nf) {
        uint64_t ctr_blocks = 0;
        h_group[0] = 0;
        for (uint32_t k = 0; k < nf; ++k) {
            h_fuse_sorted[k] = h_fuse[h_forder[k]];
            h_chunk_sorted[k] = h_chunk[h_forder[k]];
            ctr_blocks += h_chunk_sorted[k].nblocks;
            if (k > 0 && h_fuse_sorted[k].F != h_fuse_sorted[k - 1].F && split)
                h_group[++ngroups] = k;
        }
        h_group[++ngroups] = nf;
        for (uint32_t g = 0; g < ngroups; ++g)
            h_group_units[g] = frag::noalloc_fuse_schedule(h_fuse_sorted + h_group[g],
                                                           h_group[g + 1] - h_group[g], fslots, 0);
        const uint64_t per_warp = 4ull * d->sms * (frag::kCtrThreads / 32);
        while (turn < 128 * frag::kCtrTurn && ctr_blocks / (2 * turn) >= per_warp)
            turn *= 2;
        h_turns[0] = 0;
        for (uint32_t k = 0; k < nf; ++k)
            h_turns[k + 1] = h_turns[k] + (h_chunk_sorted[k].nblocks + turn - 1) / turn;
    }
    frag::host_expand_key(key, h_rk);

    // The scratch keeps whatever the previous call left there; what must
    // start at zero (the queue head) is cleared on the stream.  The error
    // word is not: it keeps the first nonzero code any call's kernel set
    // until frag_noalloc_sync_status reads and clears it.  Copies from these
    // pageable host arrays return once the source has been staged.
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = d->base;
    e = cudaMemcpyAsync(base + kOffKeys, h_rk, sizeof(h_rk), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nj)
        e = cudaMemcpyAsync(base + kOffStart, h_start, sizeof(uint64_t) * (nj + 1),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nj)
        e = cudaMemcpyAsync(base + kOffJobs, h_sorted, sizeof(Job) * nj, cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess && nf)
        e = cudaMemcpyAsync(base + kOffFuse, h_fuse_sorted, sizeof(frag::FuseBuf) * nf,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nf)
        e = cudaMemcpyAsync(base + kOffChunks, h_chunk_sorted, sizeof(frag::CtrChunk) * nf,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nf)
        e = cudaMemcpyAsync(base + kOffTurns, h_turns, sizeof(uint64_t) * (nf + 1),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nj)
        e = cudaMemsetAsync(base + kOffHead, 0, 8, s);
    if (e != cudaSuccess)
        return frag::report_cuda(e, "frag_protect_batch_noalloc: staging descriptors");
    int *err = (int *)(base + kOffHead + 8);
    const uint32_t *tables = (const uint32_t *)(base + kOffTables);

    if (nf) {
        // the fused pass over the bytes (a launch per group), then the CTR
        // pass enciphering every private fragment in place
        for (uint32_t g = 0; g < ngroups; ++g) {
            const uint32_t lo = h_group[g], cnt = h_group[g + 1] - lo;
            const uint64_t units = h_group_units[g];
            frag::FuseWork fw;
            std::memset(&fw, 0, sizeof(fw));
            fw.bufs = (const frag::FuseBuf *)(base + kOffFuse) + lo;
            if (cnt == 1)
                fw.single = h_fuse_sorted[lo];
            fw.nbufs = cnt;
            fw.total_units = units;
            fw.err = err;
            fw.aes_t0 = tables;
            // at most half as many units as warps: spread over the SMs, as
            // the other calls do
            const uint64_t cap = (uint64_t)d->sms * d->fuse_ctas;
            fw.spread = 2 * units <= cap * d->fuse_warps;
            const uint64_t need = fw.spread ? units : (units + d->fuse_warps - 1) / d->fuse_warps;
            const uint32_t fgrid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(cap, need));
            if (units && (e = frag::launch_fuse(true, false, fw, fgrid, s)) != cudaSuccess)
                return frag::report_cuda(e, "frag_protect_batch_noalloc: fused launch");
        }
        frag::CtrWork cw;
        std::memset(&cw, 0, sizeof(cw));
        cw.frags = (const frag::CtrChunk *)(base + kOffChunks);
        cw.turn_start = (const uint64_t *)(base + kOffTurns);
        cw.nfrags = nf;
        cw.nturns = h_turns[nf];
        cw.turn_blocks = turn;
        cw.aes_tables = tables;
        cw.keys = frag::aes::keys_from_words(h_rk);
        const uint32_t cgrid =
            (uint32_t)std::min<uint64_t>((uint64_t)d->sms * d->ctr_ctas, cw.nturns);
        if (cgrid && (e = frag::launch_ctr(cw, cgrid, s)) != cudaSuccess)
            return frag::report_cuda(e, "frag_protect_batch_noalloc: cipher launch");
    }
    if (nj == 0)
        return FRAG_OK;

    Work w;
    std::memset(&w, 0, sizeof(w));
    w.jobs = (const Job *)(base + kOffJobs);
    w.tile_start = (const uint64_t *)(base + kOffStart);
    w.njobs = nj;
    w.total_tiles = h_start[nj];
    w.queue = (unsigned long long *)(base + kOffHead);
    w.err = err;
    w.aes_tables = tables;
    w.round_keys = (const uint32_t *)(base + kOffKeys);

    int occ = 0;
    if ((e = frag::tile_occupancy(smem, &occ)) != cudaSuccess)
        return frag::report_cuda(e, "frag_protect_batch_noalloc: occupancy query");
    if (occ <= 0)
        return frag::report(FRAG_EUNSUPPORTED, "frag_protect_batch_noalloc: tile too large");
    const uint32_t grid =
        (uint32_t)std::min<uint64_t>((uint64_t)d->sms * (uint64_t)occ, w.total_tiles);
    if ((e = frag::launch_tiles(w, grid, smem, s)) != cudaSuccess)
        return frag::report_cuda(e, "frag_protect_batch_noalloc: launch");
    return FRAG_OK;
}

extern "C" frag_status frag_noalloc_sync_status(frag_stream stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess)
        return frag::report_cuda(e, "frag_noalloc_sync_status: cudaStreamSynchronize");
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess)
        return frag::report_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return frag::report(FRAG_EUNSUPPORTED, "frag_noalloc_sync_status: device index too high");
    std::lock_guard<std::mutex> lock(g_mu);
    const DeviceSetup &d = g_setup[dev];
    if (!d.ready) // no call has run on this device
        return FRAG_OK;
    // a synchronous read into a static host word, then a synchronous clear:
    // neither allocates
    static int h_word;
    if ((e = cudaMemcpy(&h_word, d.base + kOffHead + 8, sizeof(int), cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
        return frag::report_cuda(e, "frag_noalloc_sync_status: reading the error word");
    const int word = h_word;
    if (word == 0)
        return FRAG_OK;
    if ((e = cudaMemset(d.base + kOffHead + 8, 0, sizeof(int))) != cudaSuccess)
        return frag::report_cuda(e, "frag_noalloc_sync_status: clearing the error word");
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "frag_protect_batch_noalloc: the tile kernel reported an inconsistent work "
                  "descriptor (code %d)",
                  word);
    return frag::report(FRAG_EDEVICE, msg);
}
