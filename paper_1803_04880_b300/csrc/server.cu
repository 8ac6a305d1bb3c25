// server.cu -- the serving loop: protect / recover requests admitted by device
// memory and launched in batched groups while earlier groups still run
// (continuous batching).  The thesis has no counterpart; it is the deployment
// form of the batched calls.
//
// Submitting only records the caller's stream position (an event) and queues
// the request under a lock.  A scheduler thread takes waiting requests in
// arrival order while their memory (outputs plus the library's level scratch)
// fits the budget and a group slot is free, allocates their outputs from the
// library's pool on the slot's stream, makes that stream wait for every
// request's submit event, and launches the group as one frag_protect_batch
// and one frag_recover_batch.  A host function enqueued after the group's
// launches marks its requests done and frees the budget, so nothing polls
// for completions.  Results equal those of lone calls: the transform is exact
// integer arithmetic and each buffer's work is independent of the others in
// a launch.
#include "frag.h"

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

namespace frag {
frag_status report(frag_status st, const char *msg);
frag_status report_cuda(cudaError_t e, const char *what);
} // namespace frag

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    bool fwd = true;
    frag_plan plan = nullptr;
    uint64_t nonce = 0, nbytes = 0;
    const void *in = nullptr;                      // protect: the bytes
    const void *priv_in = nullptr, *pub_in = nullptr; // recover: the fragments
    void *priv = nullptr, *pub = nullptr;          // protect: allocated at launch
    void *out = nullptr;                           // recover: allocated at launch
    uint64_t pb = 0, ub = 0, need = 0;
    cudaEvent_t ready = nullptr;                   // the caller's stream at submit
    bool done = false, released = false;
    frag_status status = FRAG_OK;
    double t_submit = 0, t_launch = 0, t_done = 0;
};

struct Server;

struct Group {
    Server *srv = nullptr;
    std::vector<std::shared_ptr<Request>> reqs;
    uint32_t slot = 0;
    uint64_t need = 0;
};

struct Server {
    int device = 0;
    frag_key key = nullptr;
    uint64_t budget = 0, used = 0;
    uint32_t max_groups = 2, max_items = 2048;
    std::vector<cudaStream_t> streams;
    std::vector<bool> busy;
    // the requests' outputs: a pool of the server's own that keeps freed
    // memory mapped (a pool that trims at synchronisations would map
    // gigabytes again for every burst of large requests)
    cudaMemPool_t pool = nullptr;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_id = 1, launches = 0;
    uint32_t inflight = 0;
    int hold = 0;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv;      // scheduler: work to admit, a slot freed, stop
    std::condition_variable cv_done; // waiters: a request finished
    std::thread thread;
    std::vector<cudaEvent_t> spare_events;

    // a spare submit event, or nullptr (the caller creates one outside the lock)
    cudaEvent_t take_event()
    {
        if (spare_events.empty())
            return nullptr;
        cudaEvent_t e = spare_events.back();
        spare_events.pop_back();
        return e;
    }

    // outputs plus the level scratch the library allocates (at most about
    // two thirds of the padded matrix, as packed pairs) and descriptors
    static uint64_t need_of(bool fwd, uint64_t n, uint64_t pb, uint64_t ub)
    {
        return (fwd ? pb + ub : n) + (pb + ub) / 3 + (1u << 16);
    }

    void loop();
    void launch(std::unique_ptr<Group> g);
};

// stream-ordered host function at the end of a group: its requests are done
void CUDART_CB group_done(void *p)
{
    Group *g = static_cast<Group *>(p);
    Server *s = g->srv;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        const double t = now_s();
        for (auto &r : g->reqs) {
            r->done = true;
            r->t_done = t;
        }
        s->used -= g->need;
        s->busy[g->slot] = false;
        --s->inflight;
    }
    s->cv.notify_one();
    s->cv_done.notify_all();
    delete g;
}

void Server::launch(std::unique_ptr<Group> g)
{
    cudaStream_t st = streams[g->slot];
    const double t = now_s();
    std::vector<frag_item> pi;
    std::vector<frag_ritem> ri;
    frag_status status = FRAG_OK;
    for (auto &r : g->reqs) {
        r->t_launch = t;
        cudaError_t e = cudaStreamWaitEvent(st, r->ready, 0);
        if (r->fwd) {
            if (e == cudaSuccess)
                e = cudaMallocFromPoolAsync(&r->priv, r->pb ? r->pb : 1, pool, st);
            if (e == cudaSuccess)
                e = cudaMallocFromPoolAsync(&r->pub, r->ub ? r->ub : 1, pool, st);
            pi.push_back(frag_item{r->plan, r->nonce, r->nbytes, r->in, r->priv, r->pub});
        } else {
            if (e == cudaSuccess)
                e = cudaMallocFromPoolAsync(&r->out, r->nbytes ? r->nbytes : 1, pool, st);
            ri.push_back(frag_ritem{r->plan, r->nonce, r->nbytes, r->priv_in, r->pub_in, r->out});
        }
        if (e != cudaSuccess && status == FRAG_OK)
            status = frag::report_cuda(e, "frag_server: output allocation");
    }
    uint32_t n_launch = 0;
    if (status == FRAG_OK && !pi.empty()) {
        status = frag_protect_batch(pi.data(), (uint32_t)pi.size(), key, (frag_stream)st);
        ++n_launch;
    }
    if (status == FRAG_OK && !ri.empty()) {
        status = frag_recover_batch(ri.data(), (uint32_t)ri.size(), key, (frag_stream)st);
        ++n_launch;
    }
    {
        std::lock_guard<std::mutex> lock(mu);
        launches += n_launch;
        for (auto &r : g->reqs) {
            r->status = status;
            spare_events.push_back(r->ready);
            r->ready = nullptr;
        }
    }
    Group *gp = g.release();
    if (cudaLaunchHostFunc(st, group_done, gp) != cudaSuccess) {
        // no callback will come: finish the group here once the stream is idle
        cudaStreamSynchronize(st);
        group_done(gp);
    }
}

void Server::loop()
{
    cudaSetDevice(device);
    for (;;) {
        std::unique_ptr<Group> g;
        {
            std::unique_lock<std::mutex> lock(mu);
            cv.wait(lock, [&] {
                return (stop && pending.empty()) || (!pending.empty() && !hold && inflight < max_groups);
            });
            if (pending.empty()) { // stopping, nothing left to admit
                cv.wait(lock, [&] { return inflight == 0; });
                return;
            }
            g.reset(new Group());
            g->srv = this;
            uint64_t u = used;
            while (!pending.empty() && g->reqs.size() < max_items) {
                auto &r = pending.front();
                if (u + r->need > budget && (!g->reqs.empty() || inflight > 0))
                    break; // wait for memory (a request alone always goes, so nothing starves)
                u += r->need;
                g->need += r->need;
                g->reqs.push_back(r);
                pending.pop_front();
            }
            if (g->reqs.empty()) { // the head waits for memory: sleep until a group ends
                g.reset();
                const uint32_t before = inflight;
                cv.wait(lock, [&] { return inflight < before || stop; });
                continue;
            }
            uint32_t slot = 0;
            while (busy[slot])
                ++slot;
            busy[slot] = true;
            g->slot = slot;
            used = u;
            ++inflight;
        }
        launch(std::move(g));
    }
}

} // namespace

struct frag_server_s : Server {
};

namespace {
frag_status submit(frag_server s, std::shared_ptr<Request> r, frag_stream ready, uint64_t *id)
{
    uint64_t pb = 0, ub = 0;
    frag_status st = frag_plan_sizes(r->plan, r->nbytes, nullptr, &pb, &ub);
    if (st != FRAG_OK)
        return st;
    r->pb = pb;
    r->ub = ub;
    r->need = Server::need_of(r->fwd, r->nbytes, pb, ub);
    r->t_submit = now_s();
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->stop)
        return frag::report(FRAG_EINVAL, "frag_server: the server is stopping");
    r->ready = s->take_event();
    lock.unlock();
    cudaError_t e = cudaSuccess;
    if (r->ready == nullptr)
        e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventRecord(r->ready, (cudaStream_t)ready);
    if (e != cudaSuccess)
        return frag::report_cuda(e, "frag_server: submit event");
    lock.lock();
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->pending.push_back(r);
    *id = r->id;
    lock.unlock();
    s->cv.notify_one();
    return FRAG_OK;
}
} // namespace

extern "C" {

frag_status frag_server_create(frag_server *out, frag_key key, uint64_t memory_budget, uint32_t max_groups,
                               uint32_t max_items)
{
    if (out == nullptr || key == nullptr)
        return frag::report(FRAG_EINVAL, "frag_server_create: NULL argument");
    *out = nullptr;
    if (max_groups == 0 || max_groups > 16 || max_items == 0)
        return frag::report(FRAG_EINVAL, "frag_server_create: max_groups must be 1..16, max_items positive");
    frag_server s = new (std::nothrow) frag_server_s();
    if (s == nullptr)
        return frag::report(FRAG_ENOMEM, "out of host memory");
    cudaError_t e = cudaGetDevice(&s->device);
    s->key = key;
    s->max_groups = max_groups;
    s->max_items = max_items;
    s->budget = memory_budget;
    if (e == cudaSuccess && memory_budget == 0) { // free memory now, less 4 GiB
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        s->budget = fr > (4ull << 30) ? fr - (4ull << 30) : fr / 2;
    }
    if (e == cudaSuccess) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        e = cudaMemPoolCreate(&s->pool, &props);
        uint64_t keep = ~0ull;
        if (e == cudaSuccess)
            e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (uint32_t i = 0; e == cudaSuccess && i < max_groups; ++i) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            s->streams.push_back(st);
            s->busy.push_back(false);
        }
    }
    if (e != cudaSuccess) {
        for (cudaStream_t st : s->streams)
            cudaStreamDestroy(st);
        if (s->pool)
            cudaMemPoolDestroy(s->pool);
        delete s;
        return frag::report_cuda(e, "frag_server_create");
    }
    s->thread = std::thread([s] { s->loop(); });
    *out = s;
    return FRAG_OK;
}

frag_status frag_server_stop(frag_server s)
{
    if (s == nullptr)
        return frag::report(FRAG_EINVAL, "frag_server_stop: server is NULL");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->hold = 0;
    }
    s->cv.notify_all();
    if (s->thread.joinable())
        s->thread.join();
    for (cudaStream_t st : s->streams)
        cudaStreamSynchronize(st);
    return FRAG_OK;
}

frag_status frag_server_destroy(frag_server s)
{
    if (s == nullptr)
        return FRAG_OK;
    frag_server_stop(s);
    // outputs the caller did not release go back to the pool
    for (auto &kv : s->all) {
        Request &r = *kv.second;
        for (void *p : {r.priv, r.pub, r.out})
            if (p && !r.released)
                cudaFreeAsync(p, s->streams[0]);
    }
    cudaStreamSynchronize(s->streams[0]);
    for (cudaEvent_t e : s->spare_events)
        cudaEventDestroy(e);
    for (cudaStream_t st : s->streams)
        cudaStreamDestroy(st);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return FRAG_OK;
}

frag_status frag_server_submit_protect(frag_server s, frag_plan plan, uint64_t nonce, const void *d_in,
                                       uint64_t nbytes, frag_stream ready, uint64_t *id)
{
    if (s == nullptr || plan == nullptr || id == nullptr || (d_in == nullptr && nbytes))
        return frag::report(FRAG_EINVAL, "frag_server_submit_protect: NULL argument");
    auto r = std::make_shared<Request>();
    r->fwd = true;
    r->plan = plan;
    r->nonce = nonce;
    r->nbytes = nbytes;
    r->in = d_in;
    return submit(s, r, ready, id);
}

frag_status frag_server_submit_recover(frag_server s, frag_plan plan, uint64_t nonce, const void *d_private,
                                       const void *d_public, uint64_t nbytes, frag_stream ready, uint64_t *id)
{
    if (s == nullptr || plan == nullptr || id == nullptr || ((d_private == nullptr || d_public == nullptr) && nbytes))
        return frag::report(FRAG_EINVAL, "frag_server_submit_recover: NULL argument");
    auto r = std::make_shared<Request>();
    r->fwd = false;
    r->plan = plan;
    r->nonce = nonce;
    r->nbytes = nbytes;
    r->priv_in = d_private;
    r->pub_in = d_public;
    return submit(s, r, ready, id);
}

frag_status frag_server_wait(frag_server s, uint64_t id, double timeout_s, frag_request_info *info)
{
    if (s == nullptr)
        return frag::report(FRAG_EINVAL, "frag_server_wait: server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end())
        return frag::report(FRAG_EINVAL, "frag_server_wait: unknown request");
    std::shared_ptr<Request> r = it->second;
    if (timeout_s < 0) {
        s->cv_done.wait(lock, [&] { return r->done; });
    } else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [&] { return r->done; })) {
        return frag::report(FRAG_ETIMEOUT, "frag_server_wait: the request is not done yet");
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->done = 1;
        info->status = (int32_t)r->status;
        info->d_private = r->fwd ? r->priv : nullptr;
        info->d_public = r->fwd ? r->pub : nullptr;
        info->private_bytes = r->pb;
        info->public_bytes = r->ub;
        info->d_out = r->fwd ? nullptr : r->out;
        info->nbytes = r->nbytes;
        info->t_submit = r->t_submit;
        info->t_launch = r->t_launch;
        info->t_done = r->t_done;
    }
    return r->status;
}

frag_status frag_server_release(frag_server s, uint64_t id, frag_stream after)
{
    if (s == nullptr)
        return frag::report(FRAG_EINVAL, "frag_server_release: server is NULL");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->all.find(id);
        if (it == s->all.end())
            return frag::report(FRAG_EINVAL, "frag_server_release: unknown request");
        r = it->second;
        if (!r->done)
            return frag::report(FRAG_EINVAL, "frag_server_release: the request is not done");
        s->all.erase(it);
    }
    cudaError_t e = cudaSuccess;
    for (void *p : {r->priv, r->pub, r->out})
        if (p && e == cudaSuccess)
            e = cudaFreeAsync(p, (cudaStream_t)after);
    r->released = true;
    return e == cudaSuccess ? FRAG_OK : frag::report_cuda(e, "frag_server_release");
}

frag_status frag_server_hold(frag_server s, int hold)
{
    if (s == nullptr)
        return frag::report(FRAG_EINVAL, "frag_server_hold: server is NULL");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->hold += hold ? 1 : -1;
        if (s->hold < 0)
            s->hold = 0;
    }
    s->cv.notify_one();
    return FRAG_OK;
}

frag_status frag_server_stats(frag_server s, uint64_t *launches, uint64_t *used_bytes, uint32_t *pending,
                              uint32_t *in_flight)
{
    if (s == nullptr)
        return frag::report(FRAG_EINVAL, "frag_server_stats: server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    if (launches)
        *launches = s->launches;
    if (used_bytes)
        *used_bytes = s->used;
    if (pending)
        *pending = (uint32_t)s->pending.size();
    if (in_flight)
        *in_flight = s->inflight;
    return FRAG_OK;
}

frag_status frag_server_check(frag_server s)
{
    if (s == nullptr)
        return frag::report(FRAG_EINVAL, "frag_server_check: server is NULL");
    for (cudaStream_t st : s->streams) {
        frag_status r = frag_sync_status((frag_stream)st);
        if (r != FRAG_OK)
            return r;
    }
    return FRAG_OK;
}

} // extern "C"
