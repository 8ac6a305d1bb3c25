// frag_api.cu -- host implementation of the C ABI declared in include/frag.h.
//
// Plans and keys are small host objects; keys keep their expanded round keys
// resident on each device that uses them, and every device gets one copy of
// the AES tables and a device error word.  All work is enqueued on the
// caller's stream; nothing here falls back to the CPU.
#include "frag.h"
#include "frag_internal.cuh"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

using frag::Job;
using frag::Work;

struct frag_plan_s {
    uint32_t width;
    uint32_t levels;
    uint32_t tile_w;
    uint32_t tile_h;
    uint32_t ctas_per_sm;
};

struct frag_key_s {
    uint32_t rk[44]; // big-endian round-key words
    std::mutex mu;
    std::map<int, uint32_t *> on_device;
};

struct frag_batch_s {
    int device;
    bool fwd;
    Work work;
    uint32_t grid;
    size_t smem;
    void *d_mem; // jobs | tile_start | queue head
};

namespace {

constexpr uint32_t kMaxLevels = 8;
constexpr uint32_t kMaxFusedLevels = 5; // one tile window in shared memory
constexpr uint32_t kDefaultTile = 64;

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
    int sms = 0;
    size_t smem_set[2] = {0, 0};
    std::map<size_t, int> occ[2];
};

std::mutex g_mu;
std::vector<DeviceState> g_devices;

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
        d.ready = true;
    }
    *out = &d;
    if (dev_out)
        *dev_out = dev;
    return FRAG_OK;
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

// occupancy-sized persistent grid for a launch that needs `smem` bytes
frag_status launch_shape(DeviceState &d, bool fwd, size_t smem, uint32_t ctas_per_sm,
                         uint64_t total_tiles, uint32_t *grid)
{
    int occ = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = d.occ[fwd].find(smem);
        if (it != d.occ[fwd].end())
            occ = it->second;
    }
    if (occ == 0) {
        cudaError_t e = frag::tile_occupancy(fwd, smem, &occ);
        if (e != cudaSuccess)
            return cuda_fail(e, "occupancy query");
        if (occ <= 0)
            return fail(FRAG_EUNSUPPORTED, "tile window of %zu bytes does not fit on an SM", smem);
        std::lock_guard<std::mutex> lock(g_mu);
        d.occ[fwd][smem] = occ;
    }
    if (ctas_per_sm != 0 && (int)ctas_per_sm < occ)
        occ = (int)ctas_per_sm;
    const uint64_t slots = (uint64_t)d.sms * (uint64_t)occ;
    *grid = (uint32_t)std::min<uint64_t>(slots, total_tiles);
    return FRAG_OK;
}

frag_status check_plan(frag_plan plan)
{
    if (plan == nullptr)
        return fail(FRAG_EINVAL, "plan is NULL");
    return FRAG_OK;
}

uint64_t rows_for(uint64_t n, uint32_t W, uint32_t L)
{
    const uint64_t step = 1ull << L;
    const uint64_t rows = (n + W - 1) / W;
    return (rows + step - 1) / step * step;
}

frag_status fill_job(frag_plan plan, uint64_t nonce, uint64_t n, Job &j)
{
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
    if (plan->levels <= frag::kFastMaxLevels) {
        j.path = 1;
        j.tile_w = frag::kFastTile;
        j.tile_h = frag::kFastTile;
    } else {
        j.path = 0;
        j.tile_w = plan->tile_w;
        j.tile_h = plan->tile_h;
    }
    j.tiles_x = (j.W + j.tile_w - 1) / j.tile_w;
    j.tiles_y = (j.H + j.tile_h - 1) / j.tile_h;
    return FRAG_OK;
}

size_t job_smem(const Job &j, bool fwd) { return frag::job_smem_bytes(j, fwd); }

void base_work(Work &w, DeviceState &d, const uint32_t *rk)
{
    std::memset(&w, 0, sizeof(w));
    w.aes_tables = d.tables;
    w.round_keys = rk;
    w.err = d.err;
}

frag_status launch_single(bool fwd, frag_plan plan, frag_key key, const Job &j, cudaStream_t s)
{
    DeviceState *d = nullptr;
    int dev = 0;
    frag_status st = device_state(&d, &dev);
    if (st != FRAG_OK)
        return st;
    const uint32_t *rk = nullptr;
    if ((st = key_on_device(key, dev, &rk)) != FRAG_OK)
        return st;
    Work w;
    base_work(w, *d, rk);
    w.single = j;
    w.total_tiles = (uint64_t)j.tiles_x * j.tiles_y;
    const size_t smem = job_smem(j, fwd);
    uint32_t grid = 0;
    if ((st = launch_shape(*d, fwd, smem, plan->ctas_per_sm, w.total_tiles, &grid)) != FRAG_OK)
        return st;
    cudaError_t e = frag::launch_tiles(fwd, w, grid, smem, s);
    if (e != cudaSuccess)
        return cuda_fail(e, fwd ? "protect launch" : "recover launch");
    return FRAG_OK;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
struct BatchHost {
    std::vector<Job> jobs;
    std::vector<uint64_t> tile_start;
    size_t smem = 0;
    uint32_t min_ctas = 0;
};

// Order items from the most to the least costly (tiles x window area), so the
// queue hands out the long jobs first and the short ones fill the tail.
frag_status build_batch(bool fwd, const frag_item *pi, const frag_ritem *ri, uint32_t count,
                        BatchHost &b)
{
    std::vector<std::pair<uint64_t, Job>> v;
    v.reserve(count);
    for (uint32_t i = 0; i < count; ++i) {
        frag_plan plan = fwd ? pi[i].plan : ri[i].plan;
        if (plan == nullptr)
            return fail(FRAG_EINVAL, "item %u has no plan", i);
        const uint64_t n = fwd ? pi[i].nbytes : ri[i].nbytes;
        if (n == 0)
            continue;
        Job j;
        frag_status st = fill_job(plan, fwd ? pi[i].nonce : ri[i].nonce, n, j);
        if (st != FRAG_OK)
            return st;
        if (fwd) {
            j.in = (const uint8_t *)pi[i].d_in;
            j.priv = (uint8_t *)pi[i].d_private;
            j.pub = (uint8_t *)pi[i].d_public;
            if (!j.in || !j.priv || !j.pub)
                return fail(FRAG_EINVAL, "item %u has a NULL buffer", i);
        } else {
            j.priv_in = (const uint8_t *)ri[i].d_private;
            j.pub_in = (const uint8_t *)ri[i].d_public;
            j.out = (uint8_t *)ri[i].d_out;
            if (!j.priv_in || !j.pub_in || !j.out)
                return fail(FRAG_EINVAL, "item %u has a NULL buffer", i);
        }
        const uint64_t tiles = (uint64_t)j.tiles_x * j.tiles_y;
        const uint64_t cost = tiles * (uint64_t)j.tile_w * j.tile_h;
        v.emplace_back(cost, j);
        b.smem = std::max(b.smem, job_smem(j, fwd));
        const uint32_t c = plan->ctas_per_sm;
        if (c != 0)
            b.min_ctas = b.min_ctas == 0 ? c : std::min(b.min_ctas, c);
    }
    std::stable_sort(v.begin(), v.end(),
                     [](const std::pair<uint64_t, Job> &a, const std::pair<uint64_t, Job> &c) {
                         return a.first > c.first;
                     });
    b.jobs.clear();
    b.tile_start.assign(1, 0);
    for (auto &p : v) {
        b.jobs.push_back(p.second);
        b.tile_start.push_back(b.tile_start.back() + (uint64_t)p.second.tiles_x * p.second.tiles_y);
    }
    return FRAG_OK;
}

size_t batch_bytes(const BatchHost &b, size_t *off_start, size_t *off_queue)
{
    const size_t jb = (b.jobs.size() * sizeof(Job) + 255) / 256 * 256;
    const size_t sb = (b.tile_start.size() * sizeof(uint64_t) + 255) / 256 * 256;
    *off_start = jb;
    *off_queue = jb + sb;
    return jb + sb + 256;
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
    BatchHost b;
    frag_status st = build_batch(fwd, pi, ri, count, b);
    if (st != FRAG_OK)
        return st;
    if (b.jobs.empty())
        return FRAG_OK;
    DeviceState *d = nullptr;
    int dev = 0;
    if ((st = device_state(&d, &dev)) != FRAG_OK)
        return st;
    const uint32_t *rk = nullptr;
    if ((st = key_on_device(key, dev, &rk)) != FRAG_OK)
        return st;
    size_t off_start = 0, off_queue = 0;
    const size_t bytes = batch_bytes(b, &off_start, &off_queue);
    uint8_t *mem = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&mem, bytes, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync(batch queue)");
    // pageable sources: each copy returns once its source has been staged
    e = cudaMemcpyAsync(mem, b.jobs.data(), b.jobs.size() * sizeof(Job), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mem + off_start, b.tile_start.data(),
                            b.tile_start.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(mem + off_queue, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(mem, s);
        return cuda_fail(e, "batch queue upload");
    }
    Work w;
    base_work(w, *d, rk);
    w.jobs = (const Job *)mem;
    w.tile_start = (const uint64_t *)(mem + off_start);
    w.njobs = (uint32_t)b.jobs.size();
    w.total_tiles = b.tile_start.back();
    w.queue = (unsigned long long *)(mem + off_queue);
    const size_t smem = b.smem;
    uint32_t grid = 0;
    st = launch_shape(*d, fwd, smem, b.min_ctas, w.total_tiles, &grid);
    if (st == FRAG_OK) {
        e = frag::launch_tiles(fwd, w, grid, smem, s);
        if (e != cudaSuccess)
            st = cuda_fail(e, "batch launch");
    }
    cudaFreeAsync(mem, s); // released once the launch has completed
    return st;
}

frag_status create_batch(bool fwd, const frag_item *pi, const frag_ritem *ri, uint32_t count,
                         frag_batch *out)
{
    if (out == nullptr)
        return fail(FRAG_EINVAL, "out is NULL");
    *out = nullptr;
    if ((fwd ? (const void *)pi : (const void *)ri) == nullptr && count != 0)
        return fail(FRAG_EINVAL, "items is NULL");
    BatchHost b;
    frag_status st = build_batch(fwd, pi, ri, count, b);
    if (st != FRAG_OK)
        return st;
    DeviceState *d = nullptr;
    int dev = 0;
    if ((st = device_state(&d, &dev)) != FRAG_OK)
        return st;
    frag_batch bt = new (std::nothrow) frag_batch_s();
    if (bt == nullptr)
        return fail(FRAG_ENOMEM, "out of host memory");
    bt->device = dev;
    bt->fwd = fwd;
    base_work(bt->work, *d, nullptr);
    if (!b.jobs.empty()) {
        size_t off_start = 0, off_queue = 0;
        const size_t bytes = batch_bytes(b, &off_start, &off_queue);
        cudaError_t e = cudaMalloc(&bt->d_mem, bytes);
        if (e != cudaSuccess) {
            delete bt;
            return cuda_fail(e, "cudaMalloc(batch queue)");
        }
        uint8_t *mem = (uint8_t *)bt->d_mem;
        e = cudaMemcpy(mem, b.jobs.data(), b.jobs.size() * sizeof(Job), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(mem + off_start, b.tile_start.data(),
                           b.tile_start.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(bt->d_mem);
            delete bt;
            return cuda_fail(e, "batch queue upload");
        }
        bt->work.jobs = (const Job *)mem;
        bt->work.tile_start = (const uint64_t *)(mem + off_start);
        bt->work.njobs = (uint32_t)b.jobs.size();
        bt->work.total_tiles = b.tile_start.back();
        bt->work.queue = (unsigned long long *)(mem + off_queue);
        bt->smem = b.smem;
        if ((st = launch_shape(*d, fwd, bt->smem, b.min_ctas, bt->work.total_tiles, &bt->grid)) !=
            FRAG_OK) {
            cudaFree(bt->d_mem);
            delete bt;
            return st;
        }
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
    if (levels > kMaxFusedLevels)
        return fail(FRAG_EUNSUPPORTED, "levels above %u are not implemented", kMaxFusedLevels);
    frag_plan p = new (std::nothrow) frag_plan_s();
    if (p == nullptr)
        return fail(FRAG_ENOMEM, "out of host memory");
    p->width = width;
    p->levels = levels;
    p->tile_w = std::max(kDefaultTile, 1u << levels);
    p->tile_h = std::max(kDefaultTile, 1u << levels);
    p->ctas_per_sm = 0;
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
    const uint64_t H = rows_for(nbytes, plan->width, plan->levels);
    if (H > 0xFFFFFFFFull)
        return fail(FRAG_EINVAL, "buffer too tall for width %u", plan->width);
    const uint64_t pb = 2 * (H >> plan->levels) * (uint64_t)(plan->width >> plan->levels);
    if (height)
        *height = (uint32_t)H;
    if (private_bytes)
        *private_bytes = pb;
    if (public_bytes)
        *public_bytes = 2 * H * (uint64_t)plan->width - pb;
    return FRAG_OK;
}

frag_status frag_plan_set_tiling(frag_plan plan, uint32_t tile_w, uint32_t tile_h,
                                 uint32_t ctas_per_sm)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    const uint32_t step = std::max(16u, 1u << plan->levels);
    tile_w = tile_w ? tile_w : std::max(kDefaultTile, 1u << plan->levels);
    tile_h = tile_h ? tile_h : std::max(kDefaultTile, 1u << plan->levels);
    if (tile_w % step || tile_h % step || tile_w > 256 || tile_h > 256)
        return fail(FRAG_EINVAL, "tile %ux%u must be multiples of %u, at most 256", tile_w, tile_h,
                    step);
    const size_t smem = std::max(frag::tile_smem_bytes(tile_w, tile_h, plan->levels, true),
                                 frag::tile_smem_bytes(tile_w, tile_h, plan->levels, false));
    if (smem > 227 * 1024)
        return fail(FRAG_EINVAL, "tile %ux%u needs %zu bytes of shared memory", tile_w, tile_h,
                    smem);
    plan->tile_w = tile_w;
    plan->tile_h = tile_h;
    plan->ctas_per_sm = ctas_per_sm;
    return FRAG_OK;
}

frag_status frag_plan_get_tiling(frag_plan plan, uint32_t *tile_w, uint32_t *tile_h,
                                 uint32_t *ctas_per_sm)
{
    frag_status st = check_plan(plan);
    if (st != FRAG_OK)
        return st;
    if (tile_w)
        *tile_w = plan->tile_w;
    if (tile_h)
        *tile_h = plan->tile_h;
    if (ctas_per_sm)
        *ctas_per_sm = plan->ctas_per_sm;
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
    Job j;
    if ((st = fill_job(plan, nonce, nbytes, j)) != FRAG_OK)
        return st;
    j.in = (const uint8_t *)d_in;
    j.priv = (uint8_t *)d_private;
    j.pub = (uint8_t *)d_public;
    return launch_single(true, plan, key, j, (cudaStream_t)stream);
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
    Job j;
    if ((st = fill_job(plan, nonce, nbytes, j)) != FRAG_OK)
        return st;
    j.priv_in = (const uint8_t *)d_private;
    j.pub_in = (const uint8_t *)d_public;
    j.out = (uint8_t *)d_out;
    return launch_single(false, plan, key, j, (cudaStream_t)stream);
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
    uint8_t *mem = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&mem, nbytes + pb + ub + 512, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync");
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
    uint8_t *mem = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&mem, nbytes + pb + ub + 512, s);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync");
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
    if (batch->work.total_tiles == 0)
        return FRAG_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev != batch->device)
        return fail(FRAG_EINVAL, "batch was created on device %d, current is %d", batch->device,
                    dev);
    const uint32_t *rk = nullptr;
    frag_status st = key_on_device(key, dev, &rk);
    if (st != FRAG_OK)
        return st;
    Work w = batch->work;
    w.round_keys = rk;
    cudaStream_t s = (cudaStream_t)stream;
    if ((e = cudaMemsetAsync(w.queue, 0, sizeof(unsigned long long), s)) != cudaSuccess)
        return cuda_fail(e, "queue reset");
    if ((e = frag::launch_tiles(batch->fwd, w, batch->grid, batch->smem, s)) != cudaSuccess)
        return cuda_fail(e, "batch launch");
    return FRAG_OK;
}

frag_status frag_batch_destroy(frag_batch batch)
{
    if (batch == nullptr)
        return FRAG_OK;
    if (batch->d_mem)
        cudaFree(batch->d_mem);
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
        return fail(FRAG_ETIMEOUT, "a bounded device wait ran out");
    return fail(FRAG_EDEVICE, "kernel reported inconsistent work descriptor (code %d)", word);
}

} // extern "C"
