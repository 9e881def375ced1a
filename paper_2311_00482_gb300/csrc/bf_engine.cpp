// Serving engine behind bf_submit / bf_poll: continuous batching on one GPU.
//
// bf_submit admits a request only if a slot (device RF buffer, staging pairs,
// images, output, pinned host staging) can be had within the engine's device
// memory budget; otherwise it returns BF_EAGAIN and the caller retries.  The
// RF is copied host -> pinned staging -> device on a copy stream before the
// call returns.  A scheduler thread launches everything admitted so far as
// one batch (one ingest per frame, one beamform launch per precision /
// combiner variant, one envelope and one log launch) on the next of several
// streams whenever fewer than `max_inflight` batches are on the GPU, so
// requests that arrive while others run are admitted and launched as memory
// and slots free up and their work overlaps on the device.  bf_poll waits for
// the request's batch, copies the result out and releases the slot.
//
// Host data moves by DMA where it can: RF in pinned (page-locked) host
// memory goes straight to the device slot, results go straight into a pinned
// or device destination; pageable buffers pass through the slot's pinned
// staging, copied on the host by a few helper threads at once.  A batch's job
// lists, status word and events are recycled through a pool, so a launch
// allocates nothing once the engine is warm.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <string>
#include <thread>

#include "bf_engine.h"
#include "bf_ptr.h"

namespace bfi {

namespace {

constexpr int kStreams = 4;

// Host memcpy split across helper threads (the caller takes chunks too): one
// core copies well below the host memory bandwidth, and the RF in and the
// images out of a serving loop are megabytes per frame.
class CopyPool {
public:
    static CopyPool &get()
    {
        static CopyPool *pool = new CopyPool();  // process lifetime, like the engines
        return *pool;
    }

    void copy(void *dst, const void *src, size_t n)
    {
        if (n < kMinSplit || helpers_ == 0) {
            std::memcpy(dst, src, n);
            return;
        }
        Job j;
        j.dst = static_cast<char *>(dst);
        j.src = static_cast<const char *>(src);
        j.n = n;
        j.nchunks = (int)((n + kChunk - 1) / kChunk);
        {
            std::lock_guard<std::mutex> lk(mu_);
            q_.push_back(&j);
        }
        cv_.notify_all();
        work(&j);
        std::unique_lock<std::mutex> lk(mu_);
        auto it = std::find(q_.begin(), q_.end(), &j);
        if (it != q_.end())
            q_.erase(it);
        // every chunk is claimed; wait for helpers still copying theirs
        done_.wait(lk, [&] { return j.users == 0; });
    }

private:
    static constexpr size_t kChunk = (size_t)256 << 10;
    static constexpr size_t kMinSplit = (size_t)512 << 10;
    struct Job {
        char *dst = nullptr;
        const char *src = nullptr;
        size_t n = 0;
        int nchunks = 0;
        std::atomic<int> next{0};
        int users = 0;  // helpers inside work(), guarded by mu_
    };

    CopyPool()
    {
        const unsigned hw = std::thread::hardware_concurrency();
        helpers_ = (int)std::min<unsigned>(7u, hw > 2 ? hw / 2 : 0u);
        for (int i = 0; i < helpers_; ++i)
            std::thread([this] { loop(); }).detach();
    }

    static void work(Job *j)
    {
        for (;;) {
            const int c = j->next.fetch_add(1, std::memory_order_relaxed);
            if (c >= j->nchunks)
                return;
            const size_t o = (size_t)c * kChunk;
            std::memcpy(j->dst + o, j->src + o, std::min(kChunk, j->n - o));
        }
    }

    void loop()
    {
        for (;;) {
            Job *j = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return !q_.empty(); });
                j = q_.front();
                if (j->next.load(std::memory_order_relaxed) >= j->nchunks) {
                    q_.pop_front();
                    continue;
                }
                ++j->users;
            }
            work(j);
            {
                std::lock_guard<std::mutex> lk(mu_);
                --j->users;
            }
            done_.notify_all();
        }
    }

    int helpers_ = 0;
    std::mutex mu_;
    std::condition_variable cv_, done_;
    std::deque<Job *> q_;
};

// Streams of the batched transfers (bf_submit_many, bf_poll_many): copies
// spread over them run on several copy engines at once.
constexpr int kXferStreams = 4;

// How a caller's buffer moves (see copy_route); write: the copy writes it.
CopyRoute route_of(const void *p, bool write)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return CopyRoute::kStaged;
    }
    bool host_alloc = false;
    if (a.type == cudaMemoryTypeHost && write) {
        unsigned flags = 0;
        host_alloc = cudaHostGetFlags(&flags, const_cast<void *>(p)) == cudaSuccess;
        if (!host_alloc)
            cudaGetLastError();
    }
    return copy_route(a.type, host_alloc, write);
}

// Page-locked host buffer that grows on demand (contents not kept).
struct PinnedBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~PinnedBuf()
    {
        if (p)
            cudaFreeHost(p);
    }
    bool ensure(size_t n)
    {
        if (n <= bytes && p)
            return true;
        if (p)
            cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        if (cudaMallocHost(&p, n) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        bytes = n;
        return true;
    }
};

struct Slot {
    DevMem rf, out;
    FrameScratch scratch;
    PinnedBuf pin_in, pin_out;
    cudaEvent_t h2d = nullptr;
    ~Slot()
    {
        if (h2d)
            cudaEventDestroy(h2d);
    }
    size_t device_bytes() const
    {
        return rf.bytes + out.bytes + scratch.pairs.bytes + scratch.y.bytes + scratch.env.bytes +
               scratch.maxbits.bytes + scratch.map.bytes;
    }
};

// Device job lists, status word and events of one launched batch.
struct BatchRes {
    DeviceLaunch dl;
    // results the batch delivers itself (direct routes), in request order: host
    // destinations that are contiguous leave in one transfer
    DevMem arena;
    cudaEvent_t start = nullptr, done = nullptr;
    int *err_host = nullptr;  // pinned copy of the status word, written after the last kernel
    bool clean = true;        // false: the launch failed part-way, do not reuse
    ~BatchRes()
    {
        if (start)
            cudaEventDestroy(start);
        if (done)
            cudaEventDestroy(done);
        if (err_host)
            cudaFreeHost(err_host);
    }
    int init()
    {
        if (!start && cudaEventCreate(&start) != cudaSuccess)
            return fail(BF_ECUDA, "cudaEventCreate");
        if (!done && cudaEventCreate(&done) != cudaSuccess)
            return fail(BF_ECUDA, "cudaEventCreate");
        if (!err_host && cudaMallocHost((void **)&err_host, 64) != cudaSuccess)
            return fail(BF_ENOMEM, "cudaMallocHost (status word)");
        *err_host = 0;
        return BF_OK;
    }
};

struct ResPool {
    std::mutex mu;
    std::vector<std::unique_ptr<BatchRes>> free;
    std::unique_ptr<BatchRes> take()
    {
        std::lock_guard<std::mutex> lk(mu);
        if (free.empty())
            return std::make_unique<BatchRes>();
        std::unique_ptr<BatchRes> r = std::move(free.back());
        free.pop_back();
        return r;
    }
    void give(std::unique_ptr<BatchRes> r)
    {
        std::lock_guard<std::mutex> lk(mu);
        free.push_back(std::move(r));
    }
};

// A launched batch; its resources go back to the pool once the last request
// riding in it has been released (its kernels have finished by then).
struct Batch {
    int id = 0, frames = 0;
    std::unique_ptr<BatchRes> res;
    ResPool *pool = nullptr;
    ~Batch()
    {
        if (res && pool && res->clean && cudaEventQuery(res->done) == cudaSuccess)
            pool->give(std::move(res));
    }
};

}  // namespace

// One event for the RF copies bf_submit_many queued on one transfer stream:
// every request among them waits on it (one record and one wait per stream
// instead of one per frame).  Destroyed with the last request that holds it.
struct CopyEvent {
    cudaEvent_t e = nullptr;
    ~CopyEvent()
    {
        if (e)
            cudaEventDestroy(e);
    }
};

struct Request {
    uint64_t ticket = 0;
    bf_handle *h = nullptr;
    std::unique_ptr<Slot> slot;
    // the RF copy's completion: the shared event of bf_submit_many's copies on
    // the request's stream, or (null) the slot's own event
    std::shared_ptr<CopyEvent> copied;
    FramePrep fp;
    size_t out_bytes = 0;
    // destination given at submission (bf_submit_many_into): the batch itself
    // copies the result there (or, for a staged route, into the slot's pinned
    // staging, which the poll copies on); null otherwise
    float *dest = nullptr;
    bool dest_staged = false;
    // nonzero: the destinations of this request's bf_submit_many_into call lie in
    // one allocation (BF_DEST_ONE_BUFFER), so neighbours may share a transfer
    uint64_t dest_group = 0;
    std::shared_ptr<Batch> batch;
    int state = 0;  // 0 queued, 1 launched, 2 failed to launch
    int rc = BF_OK;
    std::string err;
};

namespace {

class Engine {
public:
    explicit Engine(int dev) : device_(dev)
    {
        cudaSetDevice(dev);
        for (auto &s : streams_)
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&copy_, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&d2h_, cudaStreamNonBlocking);
        for (int i = 0; i < kXferStreams; ++i) {
            cudaStreamCreateWithFlags(&xin_[i], cudaStreamNonBlocking);
            cudaStreamCreateWithFlags(&xout_[i], cudaStreamNonBlocking);
        }
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget_ = tot / 2;
        if (const char *s = std::getenv("BF_MEM_BUDGET_MB"))
            budget_ = (size_t)std::strtoull(s, nullptr, 10) << 20;
        cudaEventCreate(&epoch_);
        cudaEventRecord(epoch_, streams_[0]);
        worker_ = std::thread([this] { loop(); });
        worker_.detach();  // lives for the process
    }

    // A request whose RF copy bf_submit_many issues with the call's others.
    struct Deferred {
        std::shared_ptr<Request> req;
        const void *src;
        size_t bytes;
    };
    // defer (bf_submit_many): a device or pinned source is not copied here; the
    // request gets its ticket but is queued by flush() once its copy is
    // enqueued.  Other sources are copied (and queued) at once.
    // dest (optional): where the batch delivers the result (see Request::dest).
    int submit(bf_handle *h, const int16_t *rf, int ns, const double *angles, int na,
               uint32_t flags, uint64_t *ticket, bool wait_copy = true,
               std::vector<Deferred> *defer = nullptr, float *dest = nullptr,
               uint64_t dest_group = 0, const CopyRoute *dest_route = nullptr);
    // a fresh id for the destinations of one bf_submit_many_into call
    uint64_t next_dest_group() { return next_group_.fetch_add(1) + 1; }
    int flush(std::vector<Deferred> &defer);
    int poll(bf_handle *h, uint64_t ticket, float *out, size_t out_bytes, int64_t timeout_us);
    int poll_many(bf_handle *h, int n, const uint64_t *tickets, float *const *outs, size_t out_bytes,
                  int64_t timeout_us);
    // the caller's sources of every submission so far have been copied
    int wait_copies()
    {
        cudaSetDevice(device_);
        cudaError_t e = cudaStreamSynchronize(copy_);
        for (int i = 0; i < kXferStreams && e == cudaSuccess; ++i)
            e = cudaStreamSynchronize(xin_[i]);
        return e == cudaSuccess ? BF_OK : cuda_fail(e, "copying the requests' RF");
    }
    int batch_of(bf_handle *h, uint64_t ticket, int *id, int *frames);
    int times_of(bf_handle *h, uint64_t ticket, double *start_ms, double *end_ms);
    void pause(bool p)
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            paused_ = p;
        }
        cv_work_.notify_one();
    }
    // A multi-frame submission in progress: the scheduler forms no batch from
    // what is pending (unless a full batch is) until it ends, so that the
    // call's frames ride together instead of in fragments.
    void hold(bool on)
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            holding_ += on ? 1 : -1;
        }
        if (!on)
            cv_work_.notify_one();
    }
    void configure(int max_batch, int max_inflight, size_t budget)
    {
        std::lock_guard<std::mutex> lk(mu_);
        if (max_batch > 0)
            max_batch_ = max_batch;
        if (max_inflight > 0)
            max_inflight_ = max_inflight;
        if (budget > 0)
            budget_ = budget;
    }

private:
    void loop();
    void launch(std::vector<std::shared_ptr<Request>> &reqs);
    std::unique_ptr<Slot> take_slot();
    void put_free(std::unique_ptr<Slot> s);  // under mu_

    int device_;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_launched_;
    std::deque<std::shared_ptr<Request>> pending_;
    std::deque<std::shared_ptr<Batch>> inflight_;
    std::vector<std::unique_ptr<Slot>> free_;
    std::vector<size_t> free_bytes_;  // device bytes of free_[i]
    size_t used_ = 0, budget_ = 0;
    int live_ = 0;
    int max_batch_ = 64, max_inflight_ = 3, max_live_ = 512;
    bool paused_ = false;
    int holding_ = 0;  // submit_many calls in progress
    cudaEvent_t epoch_ = nullptr;
    uint64_t next_ticket_ = 1;
    std::atomic<uint64_t> next_group_{0};
    int next_batch_ = 0;
    cudaStream_t streams_[kStreams]{};
    cudaStream_t copy_ = nullptr, d2h_ = nullptr;
    cudaStream_t xin_[kXferStreams] = {}, xout_[kXferStreams] = {};
    std::thread worker_;
    ResPool res_pool_;
};

std::unique_ptr<Slot> Engine::take_slot()
{
    if (free_.empty())
        return std::make_unique<Slot>();
    // the largest free slot (the least growth); sizes kept beside the list so
    // that the choice reads one contiguous array
    const size_t i = (size_t)(std::max_element(free_bytes_.begin(), free_bytes_.end()) -
                              free_bytes_.begin());
    std::unique_ptr<Slot> s = std::move(free_[i]);
    free_[i] = std::move(free_.back());
    free_.pop_back();
    free_bytes_[i] = free_bytes_.back();
    free_bytes_.pop_back();
    return s;
}

void Engine::put_free(std::unique_ptr<Slot> s)
{
    free_bytes_.push_back(s->device_bytes());
    free_.push_back(std::move(s));
}

int Engine::submit(bf_handle *h, const int16_t *rf, int ns, const double *angles, int na,
                   uint32_t flags, uint64_t *ticket, bool wait_copy, std::vector<Deferred> *defer,
                   float *dest, uint64_t dest_group, const CopyRoute *dest_route)
{
    int rc = check_frame_args(h, ns, angles, na, flags);
    if (rc)
        return rc;
    if (fault_injected("submit"))
        return fail(BF_EAGAIN, "injected admission refusal (BF_FAULT=submit)");
    const size_t rf_bytes = (size_t)na * h->g.ne * ns * sizeof(int16_t);
    const size_t out_bytes = frame_out_bytes(h, flags);
    auto req = std::make_shared<Request>();
    req->h = h;
    req->out_bytes = out_bytes;
    req->dest = dest;
    // (dest_route: the route of the call's one destination buffer, found once)
    req->dest_staged =
        dest && (dest_route ? *dest_route : route_of(dest, true)) != CopyRoute::kDirect;
    req->dest_group = dest ? dest_group : 0;
    {
        std::lock_guard<std::mutex> lk(mu_);
        if (live_ >= max_live_)
            return fail(BF_EAGAIN, "%d requests in flight", live_);
        req->slot = take_slot();
        live_ += 1;
    }
    Slot &s = *req->slot;
    const size_t before = s.device_bytes();
    // admission by device memory: the slot may have to grow
    const int prec = frame_prec(flags);
    Plan *plan = nullptr;
    rc = handle_plan(h, ns, angles, na, flags, &plan);
    // staged pairs: room for the frames of a multi-frame job this frame may lead
    const int cap = plan ? job_frames_cap(plan, flags, kMaxFramesPerJob) : 1;
    size_t need = rf_bytes + out_bytes +
                  (size_t)cap * na * h->g.ne * (plan ? plan->nsp : 0) * pair_bytes(prec);
    if ((flags & BF_OUT_MASK) != BF_OUT_RF)
        need += out_bytes * ((flags & BF_OUT_MASK) == BF_OUT_LOGDB ? 2 : 1);
    auto give_back = [&](int code) {
        std::lock_guard<std::mutex> lk(mu_);
        used_ -= before;
        used_ += s.device_bytes();
        put_free(std::move(req->slot));
        live_ -= 1;
        return code;
    };
    if (rc)
        return give_back(rc);
    {
        std::lock_guard<std::mutex> lk(mu_);
        const size_t grow = need > before ? need - before : 0;
        if (grow && used_ + grow > budget_) {
            put_free(std::move(req->slot));
            live_ -= 1;
            return fail(BF_EAGAIN, "device memory budget reached (%zu of %zu bytes in use)", used_,
                        budget_);
        }
        if (grow) {
            size_t fr = 0, tot = 0;
            cudaSetDevice(device_);
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess || fr < grow + ((size_t)256 << 20)) {
                put_free(std::move(req->slot));
                live_ -= 1;
                return fail(BF_EAGAIN, "not enough free device memory for a request (%zu needed)",
                            grow);
            }
        }
        used_ += grow;  // reserved; corrected after allocation
    }
    cudaSetDevice(device_);
    rc = s.rf.ensure(rf_bytes);
    if (!rc)
        rc = s.out.ensure(out_bytes);
    if (!rc && req->dest_staged && !s.pin_out.ensure(out_bytes))
        rc = fail(BF_ENOMEM, "page-locked staging of %zu bytes", out_bytes);
    if (!rc && !s.h2d && cudaEventCreateWithFlags(&s.h2d, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(BF_ECUDA, "cudaEventCreate");
    if (!rc)
        rc = prepare_frame(h, (const int16_t *)s.rf.p, ns, angles, na, flags, (float *)s.out.p,
                           s.scratch, req->fp, -1, kMaxFramesPerJob);
    if (rc) {
        std::lock_guard<std::mutex> lk(mu_);
        const size_t grow = need > before ? need - before : 0;
        used_ -= grow;
        used_ -= before;
        used_ += s.device_bytes();
        put_free(std::move(req->slot));
        live_ -= 1;
        return rc;
    }
    // RF into the slot: device and pinned host data by DMA straight from the
    // caller's buffer (waited for: the caller may reuse it on return),
    // pageable host data through the slot's pinned staging.
    cudaError_t e;
    const CopyRoute route = route_of(rf, false);
    const bool inject = fault_injected("copy");
    if (defer && !inject && route == CopyRoute::kDirect) {
        // copied with the call's other frames: registered now, queued by flush()
        {
            std::lock_guard<std::mutex> lk(mu_);
            const size_t grow = need > before ? need - before : 0;
            used_ -= grow;
            used_ -= before;
            used_ += s.device_bytes();
            req->ticket = next_ticket_++;
        }
        {
            std::lock_guard<std::mutex> lk(h->mu);
            h->tickets[req->ticket] = req;
        }
        defer->push_back(Deferred{req, rf, rf_bytes});
        *ticket = req->ticket;
        return BF_OK;
    }
    if (inject) {
        e = cudaErrorUnknown;  // stands for a failed copy; no CUDA call is made
    } else if (route == CopyRoute::kDirect) {
        e = cudaMemcpyAsync(s.rf.p, rf, rf_bytes, cudaMemcpyDefault, copy_);
    } else if (!s.pin_in.ensure(rf_bytes)) {
        e = cudaErrorMemoryAllocation;
    } else {
        CopyPool::get().copy(s.pin_in.p, rf, rf_bytes);
        e = cudaMemcpyAsync(s.rf.p, s.pin_in.p, rf_bytes, cudaMemcpyHostToDevice, copy_);
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(s.h2d, copy_);
    if (e == cudaSuccess && route == CopyRoute::kDirect && wait_copy)
        e = cudaEventSynchronize(s.h2d);
    {
        std::lock_guard<std::mutex> lk(mu_);
        const size_t grow = need > before ? need - before : 0;
        used_ -= grow;
        used_ -= before;
        used_ += s.device_bytes();
        if (e != cudaSuccess) {
            put_free(std::move(req->slot));
            live_ -= 1;
            return inject ? fail(BF_ECUDA, "injected RF copy failure (BF_FAULT=copy)")
                          : cuda_fail(e, "copying the request's RF");
        }
        req->ticket = next_ticket_++;
        pending_.push_back(req);
    }
    {
        std::lock_guard<std::mutex> lk(h->mu);
        h->tickets[req->ticket] = req;
    }
    *ticket = req->ticket;
    cv_work_.notify_one();
    return BF_OK;
}

int Engine::flush(std::vector<Deferred> &defer)
{
    if (defer.empty())
        return BF_OK;
    cudaSetDevice(device_);
    cudaError_t e = cudaSuccess;
    // one DMA per frame, spread over the transfer streams; one event per stream
    // after its copies, shared by the requests copied there
    const int nst = (int)std::min<size_t>(defer.size(), kXferStreams);
    std::shared_ptr<CopyEvent> ev[kXferStreams];
    for (int j = 0; j < nst && e == cudaSuccess; ++j) {
        ev[j] = std::make_shared<CopyEvent>();
        e = cudaEventCreateWithFlags(&ev[j]->e, cudaEventDisableTiming);
    }
    for (size_t i = 0; i < defer.size() && e == cudaSuccess; ++i) {
        Deferred &d = defer[i];
        e = cudaMemcpyAsync(d.req->slot->rf.p, d.src, d.bytes, cudaMemcpyDefault, xin_[i % nst]);
        d.req->copied = ev[i % nst];
    }
    for (int j = 0; j < nst && e == cudaSuccess; ++j)
        e = cudaEventRecord(ev[j]->e, xin_[j]);
    std::string msg;
    int rc = BF_OK;
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "RF copy");
        msg = bf_last_error();
    }
    {
        std::lock_guard<std::mutex> lk(mu_);
        for (auto &d : defer) {
            if (rc) {  // never launched: bf_poll reports the failure and releases it
                d.req->state = 2;
                d.req->rc = rc;
                d.req->err = msg;
            } else {
                pending_.push_back(d.req);
            }
        }
    }
    defer.clear();
    cv_work_.notify_one();
    return rc;
}

void Engine::launch(std::vector<std::shared_ptr<Request>> &reqs)
{
    auto b = std::make_shared<Batch>();
    b->id = next_batch_++;
    b->frames = (int)reqs.size();
    b->pool = &res_pool_;
    b->res = res_pool_.take();
    BatchRes &R = *b->res;
    cudaStream_t st = streams_[b->id % kStreams];
    std::vector<FramePrep> frames;
    frames.reserve(reqs.size());
    std::vector<cudaEvent_t> waited;  // each copy event once (many requests share one)
    for (auto &r : reqs) {
        frames.push_back(r->fp);
        const cudaEvent_t ev = r->copied ? r->copied->e : r->slot->h2d;
        if (std::find(waited.begin(), waited.end(), ev) == waited.end()) {
            cudaStreamWaitEvent(st, ev, 0);
            waited.push_back(ev);
        }
    }
    int rc = R.init();
    // results that leave with the batch by DMA: written into the batch's arena
    // (256-byte aligned, in request order) instead of the slots
    std::vector<size_t> aoff(reqs.size(), SIZE_MAX);
    size_t abytes = 0;
    for (size_t i = 0; i < reqs.size(); ++i) {
        const Request &q = *reqs[i];
        if (!q.dest || q.dest_staged)
            continue;
        aoff[i] = abytes;
        abytes += (q.out_bytes + 255) & ~(size_t)255;
    }
    if (!rc && abytes)
        rc = R.arena.ensure(abytes);
    for (size_t i = 0; i < reqs.size() && !rc; ++i) {
        if (aoff[i] == SIZE_MAX)
            continue;
        FramePrep &f = frames[i];
        float *to = (float *)((char *)R.arena.p + aoff[i]);
        if (f.y == f.out)
            f.y = to;
        if (f.env == f.out)
            f.env = to;
        f.out = to;
    }
    HostLaunch hl;
    build_launch(frames, hl);
    if (!rc)
        rc = upload_maps(frames, st, true);
    for (size_t i = 0; i < reqs.size(); ++i)
        reqs[i]->fp.map_dirty = false;
    if (!rc)
        rc = R.dl.upload(hl, st, true);
    if (!rc && cudaMemsetAsync(R.dl.err.p, 0, sizeof(int), st) != cudaSuccess)
        rc = fail(BF_ECUDA, "cudaMemsetAsync");
    if (!rc)
        cudaEventRecord(R.start, st);
    if (!rc)
        rc = enqueue(frames, hl, R.dl, st);
    // results with a destination leave with the batch (a copy engine moves them
    // while the next batch's kernels run): from the arena, one transfer per run
    // of destinations contiguous on both sides; staged routes from the slot
    // into its pinned staging
    const char *run_src = nullptr;
    char *run_dst = nullptr;
    size_t run_bytes = 0;
    uint64_t run_group = 0;
    auto flush_run = [&]() {
        if (run_bytes && !rc &&
            cudaMemcpyAsync(run_dst, run_src, run_bytes, cudaMemcpyDefault, st) != cudaSuccess)
            rc = fail(BF_ECUDA, "cudaMemcpyAsync (results to their destinations)");
        run_bytes = 0;
    };
    for (size_t i = 0; i < reqs.size() && !rc; ++i) {
        Request &q = *reqs[i];
        if (!q.dest)
            continue;
        if (q.dest_staged) {
            if (cudaMemcpyAsync(q.slot->pin_out.p, q.slot->out.p, q.out_bytes, cudaMemcpyDefault,
                                st) != cudaSuccess)
                rc = fail(BF_ECUDA, "cudaMemcpyAsync (result to its staging)");
            continue;
        }
        const char *src = (const char *)R.arena.p + aoff[i];
        char *dst = (char *)q.dest;
        if (run_bytes && q.dest_group && q.dest_group == run_group &&
            src == run_src + run_bytes && dst == run_dst + run_bytes) {
            run_bytes += q.out_bytes;
            continue;
        }
        flush_run();
        run_src = src;
        run_dst = dst;
        run_bytes = q.out_bytes;
        run_group = q.dest_group;
    }
    flush_run();
    // the status word travels back with the batch: polls read it without a sync
    if (!rc && cudaMemcpyAsync(R.err_host, R.dl.err.p, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                   cudaSuccess)
        rc = fail(BF_ECUDA, "cudaMemcpyAsync (status word)");
    if (!rc && cudaEventRecord(R.done, st) != cudaSuccess)
        rc = fail(BF_ECUDA, "cudaEventRecord");
    if (rc)
        R.clean = false;
    std::string msg = rc ? std::string(bf_last_error()) : std::string();
    std::lock_guard<std::mutex> lk(mu_);
    for (auto &r : reqs) {
        r->batch = b;
        r->state = rc ? 2 : 1;
        r->rc = rc;
        r->err = msg;
    }
    if (!rc)
        inflight_.push_back(b);
}

void Engine::loop()
{
    cudaSetDevice(device_);
    for (;;) {
        std::vector<std::shared_ptr<Request>> take;
        {
            std::unique_lock<std::mutex> lk(mu_);
            cv_work_.wait(lk, [&] {
                return !pending_.empty() && !paused_ &&
                       (holding_ == 0 || (int)pending_.size() >= max_batch_);
            });
            while (!inflight_.empty() &&
                   cudaEventQuery(inflight_.front()->res->done) != cudaErrorNotReady)
                inflight_.pop_front();
            if ((int)inflight_.size() >= max_inflight_) {
                std::shared_ptr<Batch> oldest = inflight_.front();
                lk.unlock();
                cudaEventSynchronize(oldest->res->done);
                continue;
            }
            while (!pending_.empty() && (int)take.size() < max_batch_) {
                take.push_back(pending_.front());
                pending_.pop_front();
            }
        }
        launch(take);
        cv_launched_.notify_all();
    }
}

int Engine::poll(bf_handle *h, uint64_t ticket, float *out, size_t out_bytes, int64_t timeout_us)
{
    std::shared_ptr<Request> req;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        auto it = h->tickets.find(ticket);
        if (it == h->tickets.end())
            return fail(BF_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
        req = it->second;
    }
    if (out && out_bytes < req->out_bytes)
        return fail(BF_EINVAL, "output buffer too small (%zu < %zu bytes)", out_bytes, req->out_bytes);
    using clk = std::chrono::steady_clock;
    const auto deadline = clk::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
    // launched yet?
    {
        std::unique_lock<std::mutex> lk(mu_);
        while (req->state == 0) {
            if (timeout_us == 0)
                return BF_PENDING;
            if (timeout_us < 0)
                cv_launched_.wait(lk);
            else if (cv_launched_.wait_until(lk, deadline) == std::cv_status::timeout &&
                     req->state == 0)
                return fail(BF_ETIMEDOUT, "ticket %llu not launched within the timeout",
                            (unsigned long long)ticket);
        }
    }
    int rc = req->rc ? fail(req->rc, "%s", req->err.c_str()) : BF_OK;
    if (!rc) {
        // spin (yielding) for the first half millisecond, then sleep between queries
        const auto spin_until = clk::now() + std::chrono::microseconds(500);
        for (;;) {
            cudaError_t q = cudaEventQuery(req->batch->res->done);
            if (q == cudaSuccess)
                break;
            if (q != cudaErrorNotReady) {
                rc = cuda_fail(q, "batch execution");
                break;
            }
            if (timeout_us == 0)
                return BF_PENDING;
            const auto now = clk::now();
            if (timeout_us > 0 && now >= deadline)
                return fail(BF_ETIMEDOUT, "ticket %llu not finished within the timeout",
                            (unsigned long long)ticket);
            if (now < spin_until)
                std::this_thread::yield();
            else
                std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    cudaSetDevice(device_);
    if (!rc) {
        const int v = *(volatile int *)req->batch->res->err_host;
        if (v & kErrTimeout)
            rc = fail(BF_ETIMEDOUT, "a bounded device wait gave up (status 0x%x)", v);
        else if (v)
            rc = fail(BF_ECUDA, "device-side check failed (status 0x%x)", v);
    }
    if (!rc && req->dest) {  // delivered by the batch (staged: from pinned staging)
        if (req->dest_staged)
            CopyPool::get().copy(req->dest, req->slot->pin_out.p, req->out_bytes);
    } else if (!rc && out) {
        Slot &s = *req->slot;
        cudaError_t e;
        if (route_of(out, true) == CopyRoute::kDirect) {
            e = cudaMemcpyAsync(out, s.out.p, req->out_bytes, cudaMemcpyDefault, d2h_);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(d2h_);
        } else if (!s.pin_out.ensure(req->out_bytes)) {
            e = cudaErrorMemoryAllocation;
        } else {
            e = cudaMemcpyAsync(s.pin_out.p, s.out.p, req->out_bytes, cudaMemcpyDeviceToHost, d2h_);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(d2h_);
            if (e == cudaSuccess)
                CopyPool::get().copy(out, s.pin_out.p, req->out_bytes);
        }
        if (e != cudaSuccess)
            rc = cuda_fail(e, "copying the result");
    }
    {
        std::lock_guard<std::mutex> lk(h->mu);
        h->tickets.erase(ticket);
    }
    {
        std::lock_guard<std::mutex> lk(mu_);
        put_free(std::move(req->slot));
        live_ -= 1;
    }
    return rc;
}

// Many tickets at once: wait for all their batches, copy every result with
// one synchronisation at the end, release every ticket.  Nothing is released
// when a wait times out (BF_ETIMEDOUT) or a ticket is unknown.
int Engine::poll_many(bf_handle *h, int n, const uint64_t *tickets, float *const *outs,
                      size_t out_bytes, int64_t timeout_us)
{
    std::vector<std::shared_ptr<Request>> reqs((size_t)n);
    {
        std::lock_guard<std::mutex> lk(h->mu);
        for (int k = 0; k < n; ++k) {
            auto it = h->tickets.find(tickets[k]);
            if (it == h->tickets.end())
                return fail(BF_ENOTFOUND, "unknown ticket %llu", (unsigned long long)tickets[k]);
            reqs[k] = it->second;
            if (!reqs[k]->dest && outs && outs[k] && out_bytes < reqs[k]->out_bytes)
                return fail(BF_EINVAL, "output buffer too small (%zu < %zu bytes)", out_bytes,
                            reqs[k]->out_bytes);
        }
    }
    using clk = std::chrono::steady_clock;
    const auto deadline = clk::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
    const Batch *finished = nullptr;  // the last batch seen complete (tickets share batches)
    for (auto &req : reqs) {  // launched and finished?
        {
            std::unique_lock<std::mutex> lk(mu_);
            while (req->state == 0) {
                if (timeout_us == 0)
                    return BF_PENDING;
                if (timeout_us < 0)
                    cv_launched_.wait(lk);
                else if (cv_launched_.wait_until(lk, deadline) == std::cv_status::timeout &&
                         req->state == 0)
                    return fail(BF_ETIMEDOUT, "a ticket was not launched within the timeout");
            }
        }
        if (req->rc || req->batch.get() == finished)
            continue;
        const auto spin_until = clk::now() + std::chrono::microseconds(500);
        for (;;) {
            cudaError_t q = cudaEventQuery(req->batch->res->done);
            if (q == cudaSuccess || q != cudaErrorNotReady)
                break;
            if (timeout_us == 0)
                return BF_PENDING;
            const auto now = clk::now();
            if (timeout_us > 0 && now >= deadline)
                return fail(BF_ETIMEDOUT, "a ticket did not finish within the timeout");
            if (now < spin_until)
                std::this_thread::yield();
            else
                std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        finished = req->batch.get();
    }
    cudaSetDevice(device_);
    int rc = BF_OK;
    std::vector<int> staged;
    // device and pinned destinations: one DMA per image, spread over the
    // transfer streams (copy engines run beside the next batch's kernels);
    // the rest through the slots' pinned staging
    int direct = 0;
    std::vector<int> staged_dest;  // results the batch left in pinned staging
    const Batch *checked = nullptr;  // the last batch whose completion was confirmed
    for (int k = 0; k < n; ++k) {
        Request &r = *reqs[k];
        int rk = r.rc ? fail(r.rc, "%s", r.err.c_str()) : BF_OK;
        if (!rk && r.batch.get() != checked) {
            cudaError_t q = cudaEventQuery(r.batch->res->done);
            if (q != cudaSuccess)
                rk = cuda_fail(q, "batch execution");
            else
                checked = r.batch.get();
        }
        if (!rk) {
            const int v = *(volatile int *)r.batch->res->err_host;
            if (v)
                rk = fail(v & kErrTimeout ? BF_ETIMEDOUT : BF_ECUDA,
                          "device-side failure in a batch (status 0x%x)", v);
        }
        float *out = r.dest ? nullptr : (outs ? outs[k] : nullptr);
        if (!rk && r.dest && r.dest_staged)  // delivered by the batch into pinned staging
            staged_dest.push_back(k);
        if (!rk && out) {
            Slot &s = *r.slot;
            cudaError_t e = cudaSuccess;
            if (route_of(out, true) == CopyRoute::kDirect) {
                e = cudaMemcpyAsync(out, s.out.p, r.out_bytes, cudaMemcpyDefault,
                                    xout_[direct++ % kXferStreams]);
            } else if (!s.pin_out.ensure(r.out_bytes)) {
                e = cudaErrorMemoryAllocation;
            } else {
                e = cudaMemcpyAsync(s.pin_out.p, s.out.p, r.out_bytes, cudaMemcpyDeviceToHost, d2h_);
                staged.push_back(k);
            }
            if (e != cudaSuccess)
                rk = cuda_fail(e, "copying a result");
        }
        if (rk && !rc)
            rc = rk;
    }
    cudaError_t e = cudaStreamSynchronize(d2h_);
    for (int i = 0; i < kXferStreams && e == cudaSuccess; ++i)
        e = cudaStreamSynchronize(xout_[i]);
    if (e != cudaSuccess && !rc)
        rc = cuda_fail(e, "copying the results");
    if (e == cudaSuccess) {
        for (int k : staged)
            CopyPool::get().copy(outs[k], reqs[k]->slot->pin_out.p, reqs[k]->out_bytes);
        for (int k : staged_dest)
            CopyPool::get().copy(reqs[k]->dest, reqs[k]->slot->pin_out.p, reqs[k]->out_bytes);
    }
    {
        std::lock_guard<std::mutex> lk(h->mu);
        for (int k = 0; k < n; ++k)
            h->tickets.erase(tickets[k]);
    }
    {
        std::lock_guard<std::mutex> lk(mu_);
        for (auto &req : reqs) {
            put_free(std::move(req->slot));
            live_ -= 1;
        }
    }
    return rc;
}

int Engine::batch_of(bf_handle *h, uint64_t ticket, int *id, int *frames)
{
    std::shared_ptr<Request> req;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        auto it = h->tickets.find(ticket);
        if (it == h->tickets.end())
            return fail(BF_ENOTFOUND, "unknown ticket");
        req = it->second;
    }
    std::lock_guard<std::mutex> lk(mu_);
    if (req->state == 0)
        return BF_PENDING;
    *id = req->batch->id;
    *frames = req->batch->frames;
    return BF_OK;
}

int Engine::times_of(bf_handle *h, uint64_t ticket, double *start_ms, double *end_ms)
{
    std::shared_ptr<Request> req;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        auto it = h->tickets.find(ticket);
        if (it == h->tickets.end())
            return fail(BF_ENOTFOUND, "unknown ticket");
        req = it->second;
    }
    std::shared_ptr<Batch> b;
    {
        std::lock_guard<std::mutex> lk(mu_);
        if (req->state != 1)
            return BF_PENDING;
        b = req->batch;
    }
    cudaError_t e = cudaEventQuery(b->res->done);
    if (e == cudaErrorNotReady)
        return BF_PENDING;
    float t0 = 0.f, t1 = 0.f;
    e = cudaEventElapsedTime(&t0, epoch_, b->res->start);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&t1, epoch_, b->res->done);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaEventElapsedTime");
    *start_ms = t0;
    *end_ms = t1;
    return BF_OK;
}

std::mutex g_engines_mu;
std::map<int, Engine *> g_engines;

Engine *engine_for(int dev)
{
    std::lock_guard<std::mutex> lk(g_engines_mu);
    auto it = g_engines.find(dev);
    if (it != g_engines.end())
        return it->second;
    Engine *e = new Engine(dev);  // process lifetime
    g_engines[dev] = e;
    return e;
}

}  // namespace

void engine_forget(bf_handle *) {}

}  // namespace bfi

using namespace bfi;

extern "C" {

BF_API int bf_submit(bf_handle *h, const int16_t *rf, int32_t n_samples, const double *angles_rad,
                     int32_t n_angles, uint32_t flags, uint64_t *ticket_out)
{
    if (!h || !rf || !ticket_out)
        return fail(BF_EINVAL, "null argument");
    cudaSetDevice(h->device);
    return engine_for(h->device)->submit(h, rf, n_samples, angles_rad, n_angles, flags, ticket_out);
}

BF_API int bf_poll(bf_handle *h, uint64_t ticket, float *out, size_t out_bytes, int64_t timeout_us)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    return engine_for(h->device)->poll(h, ticket, out, out_bytes, timeout_us);
}

static int submit_many(bf_handle *h, int32_t n, const int16_t *const *rf, int32_t n_samples,
                       const double *angles_rad, int32_t n_angles, uint32_t flags,
                       float *const *outs, size_t out_bytes, uint64_t *tickets_out,
                       int32_t *n_submitted, bool one_buffer = false)
{
    if (!h || !rf || !tickets_out || n < 0)
        return fail(BF_EINVAL, "null argument");
    if (n_submitted)
        *n_submitted = 0;
    if (outs) {
        const size_t need = frame_out_bytes(h, flags);
        for (int k = 0; k < n; ++k) {
            if (!outs[k])
                return fail(BF_EINVAL, "null destination %d", k);
            if (out_bytes < need)
                return fail(BF_EINVAL, "destination too small (%zu < %zu bytes)", out_bytes, need);
        }
    }
    cudaSetDevice(h->device);
    Engine *eng = engine_for(h->device);
    struct Hold {  // the call's frames form their batches together
        Engine *e;
        explicit Hold(Engine *x) : e(x) { e->hold(true); }
        ~Hold() { e->hold(false); }
    };
    int rc = BF_OK, k = 0;
    const uint64_t group = outs && one_buffer ? eng->next_dest_group() : 0;
    // one allocation holds every destination: one route for all of them
    CopyRoute one_route = CopyRoute::kStaged;
    if (group)
        one_route = route_of(outs[0], true);
    {
        Hold hold(eng);  // released once every frame is admitted (copies may still run)
        std::vector<Engine::Deferred> defer;  // device and pinned sources: DMA per frame
        for (; k < n; ++k) {
            if (!rf[k]) {
                rc = fail(BF_EINVAL, "null record pointer %d", k);
                break;
            }
            rc = eng->submit(h, rf[k], n_samples, angles_rad, n_angles, flags, tickets_out + k,
                             false, &defer, outs ? outs[k] : nullptr, group,
                             group ? &one_route : nullptr);
            if (rc)
                break;
        }
        const int rf_copy = eng->flush(defer);
        if (!rc)
            rc = rf_copy;
    }
    if (n_submitted)
        *n_submitted = k;
    const int rw = eng->wait_copies();  // every submitted source copied before returning
    return rc ? rc : rw;
}

BF_API int bf_submit_many(bf_handle *h, int32_t n, const int16_t *const *rf, int32_t n_samples,
                          const double *angles_rad, int32_t n_angles, uint32_t mode_and_flags,
                          uint64_t *tickets_out, int32_t *n_submitted)
{
    return submit_many(h, n, rf, n_samples, angles_rad, n_angles, mode_and_flags, nullptr, 0,
                       tickets_out, n_submitted);
}

BF_API int bf_submit_many_into(bf_handle *h, int32_t n, const int16_t *const *rf,
                               int32_t n_samples, const double *angles_rad, int32_t n_angles,
                               uint32_t mode_and_flags, float *const *outs, size_t out_bytes,
                               uint64_t *tickets_out, int32_t *n_submitted)
{
    if (!outs)
        return fail(BF_EINVAL, "null destinations");
    const bool one_buffer = (mode_and_flags & BF_DEST_ONE_BUFFER) != 0;
    return submit_many(h, n, rf, n_samples, angles_rad, n_angles,
                       mode_and_flags & ~(uint32_t)BF_DEST_ONE_BUFFER, outs, out_bytes, tickets_out,
                       n_submitted, one_buffer);
}

BF_API int bf_poll_many(bf_handle *h, int32_t n, const uint64_t *tickets, float *const *outs,
                        size_t out_bytes, int64_t timeout_us)
{
    if (!h || !tickets || n < 0)
        return fail(BF_EINVAL, "null argument");
    if (n == 0)
        return BF_OK;
    return engine_for(h->device)->poll_many(h, n, tickets, outs, out_bytes, timeout_us);
}

BF_API int bf_ticket_batch(bf_handle *h, uint64_t ticket, int32_t *batch_id, int32_t *batch_frames)
{
    if (!h || !batch_id || !batch_frames)
        return fail(BF_EINVAL, "null argument");
    return engine_for(h->device)->batch_of(h, ticket, batch_id, batch_frames);
}

BF_API int bf_ticket_times(bf_handle *h, uint64_t ticket, double *start_ms, double *end_ms)
{
    if (!h || !start_ms || !end_ms)
        return fail(BF_EINVAL, "null argument");
    cudaSetDevice(h->device);
    return engine_for(h->device)->times_of(h, ticket, start_ms, end_ms);
}

BF_API int bf_engine_pause(int32_t paused)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return fail(BF_ECUDA, "no CUDA device");
    engine_for(dev)->pause(paused != 0);
    return BF_OK;
}

BF_API int bf_engine_configure(int32_t max_batch, int32_t max_inflight, uint64_t memory_budget_bytes)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return fail(BF_ECUDA, "no CUDA device");
    engine_for(dev)->configure(max_batch, max_inflight, (size_t)memory_budget_bytes);
    return BF_OK;
}

}  // extern "C"
