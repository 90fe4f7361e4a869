// iwpp_server.cu -- a continuous-batching request server on one GPU.
//
// Requests (a reconstruction or a distance transform on host images) are
// queued by iwpp_server_submit and served by one worker thread:
//   * admission: a request is admitted when the device memory it needs
//     fits the server's HBM budget next to everything else the server holds:
//     the images of the requests in flight (stream-ordered allocations from
//     the server's own memory pool, which keeps freed blocks cached for the
//     next requests) and the resident workspace of every stream's context,
//     grown to what the batch needs (tile queue, tile states, spill queues);
//   * the pool never makes one stream wait for another to reuse a block
//     (no internal dependencies): a stream reuses its own freed blocks, or
//     blocks whose free has completed, and otherwise takes new memory, so
//     the streams' batches overlap instead of queueing behind each other's
//     frees;
//   * batching: the admitted requests form one batch, run as ONE persistent
//     launch (iwpp_run_jobs_async) on one of the server's streams; each
//     stream has its own resident context (tile queue, flags, spill space);
//   * continuous: while batches run on some streams, newly arrived requests
//     are admitted and launched on the others as soon as memory and a
//     stream are free, so their work overlaps on the device;
//   * completion: host-to-device copies, the launch, device-to-host copies
//     and the readback of the batch's status are ordered on the batch's
//     stream; an event marks the end.
//     The worker polls the events, releases the memory, and records each
//     request's status and latency (submit to completion), which
//     iwpp_server_poll / iwpp_server_wait hand out once (then the ticket is
//     retired and its record dropped).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "../../include/iwpp.h"
#include "iwpp_internal.h"
#include "iwpp_status.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    iwpp_request req;
    size_t bytes;          // device memory the request needs
    Clock::time_point t0;  // submit time
};

struct Done {
    int status;
    double latency_ms;
};

struct Slot {  // one stream with its resident context
    cudaStream_t stream = nullptr;
    iwpp_ctx *ctx = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Request> batch;
    std::vector<void *> allocs;
    size_t bytes = 0;      // request images of the batch in flight
    size_t ctx_bytes = 0;  // device memory the slot's context holds (resident)
};

size_t elem(int dtype) { return dtype == IWPP_I32 ? 4 : 1; }

// Device bytes of a request's three buffers, each rounded up to 2 MiB so that
// the count never falls below what the memory pool hands out for them.
size_t request_bytes(const iwpp_request &r) {
    const size_t px = (size_t)r.h * r.w;
    auto round = [](size_t n) { return (n + ((size_t)2 << 20) - 1) / ((size_t)2 << 20) * ((size_t)2 << 20); };
    if (r.op == IWPP_OP_RECON) return 3 * round(px * elem(r.dtype));
    return round(px) + 2 * round(4 * px);
}

}  // namespace

struct iwpp_server {
    int device = 0;
    size_t budget = 0;
    int max_batch = 64;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::map<uint64_t, Done> done;  // finished, not yet handed out
    std::set<uint64_t> live;        // submitted, not yet handed out
    uint64_t next_ticket = 1;
    size_t in_use = 0;              // request images in flight
    size_t ws_total = 0;            // resident context memory of all slots
    size_t peak_in_use = 0;         // peak of in_use + ws_total
    cudaMemPool_t pool = nullptr;
    uint64_t batches = 0, completed = 0, submitted = 0;
    bool stop = false;
    std::thread worker;
    char err[256] = {0};

    void run();
    bool launch(Slot &s, std::vector<Request> &&batch);
    void finish(Slot &s);
};

bool iwpp_server::launch(Slot &s, std::vector<Request> &&batch) {
    cudaStream_t st = s.stream;
    std::vector<iwpp_job> jobs(batch.size());
    bool ok = true;
    for (size_t i = 0; i < batch.size() && ok; ++i) {
        const iwpp_request &r = batch[i].req;
        const size_t px = (size_t)r.h * r.w;
        iwpp_job &j = jobs[i];
        memset(&j, 0, sizeof j);
        j.op = r.op;
        j.conn = r.conn;
        j.flags = r.flags;
        auto dev_alloc = [&](size_t n) -> void * {
            void *p = nullptr;
            if (cudaMallocFromPoolAsync(&p, std::max<size_t>(n, 1), pool, st) != cudaSuccess) {
                ok = false;
                return nullptr;
            }
            s.allocs.push_back(p);
            return p;
        };
        if (r.op == IWPP_OP_RECON) {
            const size_t n = px * elem(r.dtype);
            void *m = dev_alloc(n), *k = dev_alloc(n), *o = dev_alloc(n);
            if (!ok) break;
            ok = cudaMemcpyAsync(m, r.marker, n, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                 cudaMemcpyAsync(k, r.mask, n, cudaMemcpyHostToDevice, st) == cudaSuccess;
            j.a = iwpp_image{m, r.h, r.w, r.w, r.dtype};
            j.b = iwpp_image{k, r.h, r.w, r.w, r.dtype};
            j.out = iwpp_image{o, r.h, r.w, r.w, r.dtype};
        } else {
            void *b = dev_alloc(px), *sq = dev_alloc(4 * px), *nn = dev_alloc(4 * px);
            if (!ok) break;
            ok = cudaMemcpyAsync(b, r.marker, px, cudaMemcpyHostToDevice, st) == cudaSuccess;
            j.a = iwpp_image{b, r.h, r.w, r.w, IWPP_U8};
            j.sqdist = (int32_t *)sq;
            j.nearest = (int32_t *)nn;
        }
    }
    if (ok) ok = iwpp_run_jobs_async(s.ctx, (int)jobs.size(), jobs.data(), st) == IWPP_OK;
    for (size_t i = 0; i < batch.size() && ok; ++i) {
        const iwpp_request &r = batch[i].req;
        const size_t px = (size_t)r.h * r.w;
        if (r.op == IWPP_OP_RECON)
            ok = cudaMemcpyAsync(r.out, jobs[i].out.data, px * elem(r.dtype), cudaMemcpyDeviceToHost, st) ==
                 cudaSuccess;
        else
            ok = cudaMemcpyAsync(r.sqdist, jobs[i].sqdist, 4 * px, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                 cudaMemcpyAsync(r.nearest, jobs[i].nearest, 4 * px, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    }
    // the batch's status follows its own copies on its stream, so reading
    // it needs no later copy (which would queue behind other streams'
    // transfers and hold up this thread)
    if (ok) ok = iwpp::status_readback(s.ctx, st) == IWPP_OK;
    for (void *p : s.allocs) cudaFreeAsync(p, st);  // stream-ordered: after the copies
    s.allocs.clear();
    if (ok) ok = cudaEventRecord(s.done, st) == cudaSuccess;
    s.batch = std::move(batch);
    s.busy = true;
    return ok;
}

void iwpp_server::finish(Slot &s) {
    // the stream is idle: the batch's status has arrived
    const int rc = iwpp::status_result(s.ctx, s.stream);
    const Clock::time_point t1 = Clock::now();
    std::lock_guard<std::mutex> lock(mu);
    for (Request &r : s.batch) {
        done[r.ticket] = Done{rc, std::chrono::duration<double, std::milli>(t1 - r.t0).count()};
        ++completed;
    }
    in_use -= s.bytes;
    s.bytes = 0;
    s.batch.clear();
    s.busy = false;
    cv_done.notify_all();
}

void iwpp_server::run() {
    cudaSetDevice(device);
    while (true) {
        // 1. retire finished batches
        for (Slot &s : slots)
            if (s.busy && cudaEventQuery(s.done) != cudaErrorNotReady) finish(s);
        // 2. admit and launch on free streams
        std::unique_lock<std::mutex> lock(mu);
        if (stop && pending.empty() && std::none_of(slots.begin(), slots.end(), [](const Slot &s) { return s.busy; }))
            break;
        for (Slot &s : slots) {
            if (s.busy || pending.empty()) continue;
            std::vector<Request> batch;
            std::vector<int> op, dt, hh, ww;
            size_t bytes = 0, ctx_after = s.ctx_bytes;
            const size_t others_ws = ws_total - s.ctx_bytes;
            while (!pending.empty() && (int)batch.size() < max_batch) {
                const Request &r = pending.front();
                // the slot context's memory once it has run the batch with r
                op.push_back(r.req.op);
                dt.push_back(r.req.op == IWPP_OP_RECON ? r.req.dtype : IWPP_U8);
                hh.push_back(r.req.h);
                ww.push_back(r.req.w);
                size_t after = 0, alone = 0;
                const bool sized =
                    iwpp::ctx_device_bytes_after(s.ctx, (int)op.size(), op.data(), dt.data(), hh.data(), ww.data(),
                                                 &after) == IWPP_OK &&
                    iwpp::ctx_device_bytes_after(s.ctx, 1, &op.back(), &dt.back(), &hh.back(), &ww.back(),
                                                 &alone) == IWPP_OK;
                if (!sized || others_ws + alone + r.bytes > budget) {
                    // can never fit, even alone on this stream: fail it
                    done[r.ticket] = Done{sized ? IWPP_ENOMEM : IWPP_ECUDA, 0.0};
                    ++completed;
                    pending.pop_front();
                    op.pop_back(); dt.pop_back(); hh.pop_back(); ww.pop_back();
                    cv_done.notify_all();
                    continue;
                }
                if (in_use + bytes + r.bytes + others_ws + after > budget) {
                    op.pop_back(); dt.pop_back(); hh.pop_back(); ww.pop_back();
                    break;
                }
                bytes += r.bytes;
                ctx_after = after;
                batch.push_back(r);
                pending.pop_front();
            }
            if (batch.empty()) break;  // memory exhausted: wait for completions
            in_use += bytes;
            ws_total += ctx_after - s.ctx_bytes;  // reserved before the context grows
            s.ctx_bytes = ctx_after;
            peak_in_use = std::max(peak_in_use, in_use + ws_total);
            ++batches;
            s.bytes = bytes;
            lock.unlock();
            const bool ok = launch(s, std::move(batch));
            lock.lock();
            {   // what the context really holds now (never more than reserved)
                const size_t real = iwpp::ctx_device_bytes(s.ctx);
                if (real > s.ctx_bytes) {
                    ws_total += real - s.ctx_bytes;
                    s.ctx_bytes = real;
                    peak_in_use = std::max(peak_in_use, in_use + ws_total);
                }
            }
            if (!ok) {
                const Clock::time_point t1 = Clock::now();
                for (Request &r : s.batch) {
                    done[r.ticket] = Done{IWPP_ECUDA, std::chrono::duration<double, std::milli>(t1 - r.t0).count()};
                    ++completed;
                }
                in_use -= s.bytes;
                s.bytes = 0;
                s.batch.clear();
                s.busy = false;
                cv_done.notify_all();
            }
        }
        // 3. sleep briefly: new arrivals or completions wake us up
        const bool any_busy = std::any_of(slots.begin(), slots.end(), [](const Slot &s) { return s.busy; });
        if (any_busy)
            cv_work.wait_for(lock, std::chrono::microseconds(20));
        else
            cv_work.wait_for(lock, std::chrono::milliseconds(2), [&] { return stop || !pending.empty(); });
    }
}

extern "C" {

int iwpp_server_create(iwpp_server **out, int device, size_t hbm_budget_bytes, int streams, int max_batch) {
    if (!out || streams < 1 || streams > 16 || max_batch < 1 || hbm_budget_bytes == 0) return IWPP_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return IWPP_ECUDA;
    iwpp_server *s = new iwpp_server();
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->max_batch = max_batch;
    s->slots.resize(streams);
    // the server's pool: freed memory stays cached up to the budget
    // (admission, not the allocator, bounds the footprint), and no reuse
    // across streams through inserted dependencies
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        s->pool = nullptr;
        iwpp_server_destroy(s);
        return IWPP_ECUDA;
    }
    uint64_t thr = hbm_budget_bytes;
    int no = 0;
    if (cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no) != cudaSuccess) {
        iwpp_server_destroy(s);
        return IWPP_ECUDA;
    }
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            iwpp_ctx_create(&sl.ctx, device, 0) != IWPP_OK) {
            iwpp_server_destroy(s);
            return IWPP_ECUDA;
        }
        sl.ctx_bytes = iwpp::ctx_device_bytes(sl.ctx);
        s->ws_total += sl.ctx_bytes;
    }
    if (s->ws_total > hbm_budget_bytes) {
        iwpp_server_destroy(s);
        return IWPP_ENOMEM;
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return IWPP_OK;
}

int iwpp_server_submit(iwpp_server *s, const iwpp_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return IWPP_EINVAL;
    const iwpp_request &r = *req;
    if (r.h < 1 || r.w < 1 || !r.marker) return IWPP_EINVAL;
    if (r.op == IWPP_OP_RECON) {
        if (!r.mask || !r.out || (r.conn != 4 && r.conn != 8) || (r.dtype != IWPP_U8 && r.dtype != IWPP_I32))
            return IWPP_EINVAL;
    } else if (r.op == IWPP_OP_EDT) {
        if (!r.sqdist || !r.nearest || (r.flags & ~3) || r.h > 32768 || r.w > 32768) return IWPP_EINVAL;
    } else {
        return IWPP_EINVAL;
    }
    Request q{0, r, request_bytes(r), Clock::now()};
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return IWPP_EINVAL;
        q.ticket = s->next_ticket++;
        s->live.insert(q.ticket);
        s->pending.push_back(q);
        ++s->submitted;
    }
    s->cv_work.notify_one();
    *ticket = q.ticket;
    return IWPP_OK;
}

int iwpp_server_poll(iwpp_server *s, uint64_t ticket, int *status) {
    if (!s) return IWPP_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->live.count(ticket)) return IWPP_EINVAL;  // unknown or already handed out
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return 0;
    if (status) *status = it->second.status;
    s->done.erase(it);
    s->live.erase(ticket);
    return 1;
}

int iwpp_server_wait(iwpp_server *s, uint64_t ticket, int *status, double *latency_ms) {
    if (!s) return IWPP_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    if (!s->live.count(ticket)) return IWPP_EINVAL;  // unknown or already handed out
    s->cv_done.wait(lock, [&] { return s->done.count(ticket) != 0; });
    const Done d = s->done[ticket];
    s->done.erase(ticket);
    s->live.erase(ticket);
    if (status) *status = d.status;
    if (latency_ms) *latency_ms = d.latency_ms;
    return IWPP_OK;
}

int iwpp_server_stats(iwpp_server *s, iwpp_server_stats_t *out) {
    if (!s || !out) return IWPP_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->batches = s->batches;
    out->pending = s->pending.size();
    out->bytes_in_use = s->in_use + s->ws_total;
    out->peak_bytes_in_use = s->peak_in_use;
    out->workspace_bytes = s->ws_total;
    out->records = s->done.size();
    out->pool_used_high = 0;
    if (s->pool) {
        uint64_t v = 0;
        if (cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrUsedMemHigh, &v) == cudaSuccess) out->pool_used_high = v;
    }
    return IWPP_OK;
}

int iwpp_server_destroy(iwpp_server *s) {
    if (!s) return IWPP_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ctx) iwpp_ctx_destroy(sl.ctx);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return IWPP_OK;
}

}  // extern "C"
