// serve.cu -- continuous-batching precoding server on top of the plan API.
//
// Requests (one channel each, already on the device) are submitted from any
// host thread and get a ticket.  A scheduler thread owns the context: while
// fewer than max_inflight batches are on the GPU it takes the waiting
// requests of the oldest one's cost class (K class; K = 256 split by
// M >= 4 K), so that a cheap request never waits inside a batch held up by
// a slow one (up to max_batch) -- the 256-user classes holding at most all
// but one of the slots, which stays for the cheap ones -- checks the arena for room (admission by free
// device memory; otherwise it waits for a batch to retire), builds a ragged
// plan and launches it on its own stream, so requests that arrive while
// other batches run are admitted as soon as a slot and memory free up and
// their work overlaps on the device.  A host callback after each batch
// records the completion time; the scheduler retires finished batches,
// releases their plans (stream-ordered), and publishes per-request status
// and latency.  Waits are bounded; no call blocks forever.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/jacpcg.h"

struct jacpcg_server;

namespace {

using clk = std::chrono::steady_clock;

double now_us() {
    return std::chrono::duration<double, std::micro>(clk::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket;
    jacpcg_instance inst;
    double t_submit;
};

struct Batch {
    jacpcg_server *srv = nullptr;
    std::vector<uint64_t> tickets;
    jacpcg_plan *plan = nullptr;
    int32_t *status_dev = nullptr;   // device, one per request
    int32_t *status_host = nullptr;  // pinned
    int slot = -1;
    int cls = 0;                     // cost class of its requests
    std::atomic<int> done{0};
    double t_done = 0.0;
};

struct Result {
    int state = 0;          // 0 queued / running, 1 done
    jacpcg_status status = JACPCG_OK;
    double latency_us = 0.0;
    double t_submit = 0.0;
};

}  // namespace

struct jacpcg_server {
    jacpcg_ctx *ctx = nullptr;
    jacpcg_server_config cfg{};
    std::vector<cudaStream_t> streams;
    std::vector<int32_t *> status_dev;    // per slot, max_batch entries
    std::vector<int32_t *> status_host;   // per slot, pinned
    std::vector<void *> plain_ws;         // per slot, workspace of the plain comparator
    size_t plain_ws_bytes = 0;
    std::vector<bool> slot_busy;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue[4];         // waiting requests per cost class (FIFO: class 0 only)
    size_t n_pending = 0;
    std::unordered_map<uint64_t, Result> results;
    std::vector<Batch *> inflight;
    int slow_inflight = 0;                // in-flight batches of the 256-user classes
    uint64_t next_ticket = 1;
    bool stop = false;
    bool failed = false;
    std::thread worker;
    // stats
    uint64_t n_done = 0, n_batches = 0;
    double sum_batch = 0.0;
};

namespace {

void CUDART_CB on_batch_done(void *arg) {
    Batch *b = static_cast<Batch *>(arg);
    b->t_done = now_us();
    b->done.store(1, std::memory_order_release);
    b->srv->cv_work.notify_one();   // wake the scheduler (no CUDA call here)
}

// Retire finished batches (called with the lock held).
void reap(jacpcg_server *s) {
    for (size_t i = 0; i < s->inflight.size();) {
        Batch *b = s->inflight[i];
        if (!b->done.load(std::memory_order_acquire)) {
            ++i;
            continue;
        }
        for (size_t k = 0; k < b->tickets.size(); ++k) {
            auto it = s->results.find(b->tickets[k]);
            if (it == s->results.end()) continue;
            it->second.state = 1;
            it->second.status = static_cast<jacpcg_status>(b->status_host[k]);
            it->second.latency_us = b->t_done - it->second.t_submit;
        }
        s->n_done += b->tickets.size();
        if (b->plan) jacpcg_plan_destroy(b->plan);
        s->slot_busy[b->slot] = false;
        if (b->cls >= 2) --s->slow_inflight;
        delete b;
        s->inflight.erase(s->inflight.begin() + i);
        s->cv_done.notify_all();
    }
}

void fail_all(jacpcg_server *s, std::vector<Request> &reqs) {
    for (auto &r : reqs) {
        auto it = s->results.find(r.ticket);
        if (it != s->results.end()) {
            it->second.state = 1;
            it->second.status = JACPCG_ECUDA;
        }
    }
    s->failed = true;
    s->cv_done.notify_all();
}

// Cost class of a request (JACPCG_BATCH_COST_CLASS): the K class, with the
// 256 class split by M >= 4 K.
int cost_class(const jacpcg_instance &q) {
    const int K = q.K;
    if (K <= 64) return 0;
    if (K <= 128) return 1;
    return q.M >= 4 * K ? 2 : 3;
}

void scheduler(jacpcg_server *s) {
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        reap(s);
        if (s->stop && s->n_pending == 0 && s->inflight.empty()) break;
        int slot = -1;
        for (size_t k = 0; k < s->slot_busy.size(); ++k)
            if (!s->slot_busy[k]) {
                slot = (int)k;
                break;
            }
        if (s->n_pending == 0 || slot < 0 || s->failed) {
            // nothing to launch now: sleep briefly (callbacks do not notify the lock)
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
            continue;
        }
        // the class of the oldest waiting request (tickets grow with arrival); under
        // cost classes the 256-user classes (batches of milliseconds) may hold at
        // most max_inflight - 1 slots, so one stays for the cheap classes
        const bool reserve = s->cfg.batch_policy == JACPCG_BATCH_COST_CLASS && s->cfg.max_inflight >= 2 &&
                             s->slow_inflight >= s->cfg.max_inflight - 1;
        int cls = -1;
        for (int c = 0; c < 4; ++c)
            if (!s->queue[c].empty() && !(reserve && c >= 2) &&
                (cls < 0 || s->queue[c].front().ticket < s->queue[cls].front().ticket))
                cls = c;
        if (cls < 0) {   // only slow requests wait and their share of the slots is taken
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
            continue;
        }
        std::deque<Request> &q = s->queue[cls];
        // take up to max_batch of its requests, shrinking until the arena admits them
        size_t take = std::min<size_t>(q.size(), (size_t)s->cfg.max_batch);
        std::vector<jacpcg_instance> insts;
        size_t need = 0, have = 0;
        while (take > 0) {
            insts.clear();
            for (size_t k = 0; k < take; ++k) insts.push_back(q[k].inst);
            if (jacpcg_plan_bytes(s->ctx, insts.data(), (int)take, &need) != JACPCG_OK) {
                need = SIZE_MAX;
                break;
            }
            jacpcg_arena_free_bytes(s->ctx, &have);
            if (need <= have) break;
            if (!s->inflight.empty()) {   // wait for memory to come back
                take = 0;
                break;
            }
            take /= 2;
        }
        if (take == 0) {
            if (need == SIZE_MAX || s->inflight.empty()) {   // cannot ever fit: reject the head
                std::vector<Request> bad{q.front()};
                q.pop_front();
                --s->n_pending;
                auto it = s->results.find(bad[0].ticket);
                if (it != s->results.end()) {
                    it->second.state = 1;
                    it->second.status = need == SIZE_MAX ? JACPCG_EINVAL : JACPCG_ENOMEM;
                }
                s->cv_done.notify_all();
            } else {
                s->cv_work.wait_for(lk, std::chrono::microseconds(20));
            }
            continue;
        }
        std::vector<Request> reqs(q.begin(), q.begin() + take);
        q.erase(q.begin(), q.begin() + take);
        s->n_pending -= take;
        Batch *b = new (std::nothrow) Batch();
        if (!b) {
            fail_all(s, reqs);
            continue;
        }
        b->srv = s;
        b->slot = slot;
        b->cls = cls;
        b->status_dev = s->status_dev[slot];
        b->status_host = s->status_host[slot];
        for (auto &r : reqs) b->tickets.push_back(r.ticket);
        const cudaStream_t st = s->streams[slot];
        s->slot_busy[slot] = true;
        lk.unlock();   // the context is touched only by this thread; submitters may proceed
        jacpcg_status e;
        if (s->cfg.plain) {
            e = jacpcg_precode_plain(insts.data(), (int)take, s->cfg.plain_variant, s->plain_ws[slot],
                                     s->plain_ws_bytes, b->status_dev, nullptr, nullptr, nullptr, st);
        } else {
            e = jacpcg_plan_create(s->ctx, insts.data(), (int)take, b->status_dev, nullptr, nullptr,
                                   nullptr, 0, &b->plan);
            if (e == JACPCG_OK) e = jacpcg_plan_execute(b->plan, st);
        }
        if (e == JACPCG_OK &&
            (cudaMemcpyAsync(b->status_host, b->status_dev, take * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaLaunchHostFunc(st, on_batch_done, b) != cudaSuccess))
            e = JACPCG_ECUDA;
        lk.lock();
        if (e != JACPCG_OK) {
            s->slot_busy[slot] = false;
            if (b->plan) jacpcg_plan_destroy(b->plan);
            delete b;
            fail_all(s, reqs);
            continue;
        }
        s->inflight.push_back(b);
        if (cls >= 2) ++s->slow_inflight;
        s->n_batches += 1;
        s->sum_batch += (double)take;
    }
}

}  // namespace

extern "C" {

jacpcg_status jacpcg_server_create(jacpcg_ctx *ctx, const jacpcg_server_config *cfg,
                                   jacpcg_server **out) {
    if (!ctx || !cfg || !out || cfg->max_batch < 1 || cfg->max_inflight < 1 || cfg->max_inflight > 64 ||
        (cfg->batch_policy != JACPCG_BATCH_COST_CLASS && cfg->batch_policy != JACPCG_BATCH_FIFO))
        return JACPCG_EINVAL;
    jacpcg_server *s = new (std::nothrow) jacpcg_server();
    if (!s) return JACPCG_ENOMEM;
    s->ctx = ctx;
    s->cfg = *cfg;
    const int nslot = cfg->max_inflight;
    s->streams.assign(nslot, nullptr);
    s->status_dev.assign(nslot, nullptr);
    s->status_host.assign(nslot, nullptr);
    s->slot_busy.assign(nslot, false);
    s->plain_ws.assign(nslot, nullptr);
    s->plain_ws_bytes = 5 * 256 * 256 * 8 + 16 * 256 + 256;
    bool ok = true;
    for (int k = 0; k < nslot && ok; ++k) {
        ok = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaMalloc(reinterpret_cast<void **>(&s->status_dev[k]), sizeof(int32_t) * cfg->max_batch) ==
                 cudaSuccess &&
             cudaHostAlloc(reinterpret_cast<void **>(&s->status_host[k]), sizeof(int32_t) * cfg->max_batch,
                           cudaHostAllocDefault) == cudaSuccess &&
             (!cfg->plain || cudaMalloc(&s->plain_ws[k], s->plain_ws_bytes) == cudaSuccess);
    }
    if (!ok) {
        (void)cudaGetLastError();
        jacpcg_server_destroy(s);
        return JACPCG_ENOMEM;
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return JACPCG_OK;
}

jacpcg_status jacpcg_submit(jacpcg_server *s, const jacpcg_instance *inst, uint64_t *ticket) {
    if (!s || !inst || !ticket) return JACPCG_EINVAL;
    size_t one = 0;
    if (jacpcg_plan_bytes(s->ctx, inst, 1, &one) != JACPCG_OK) return JACPCG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed) return JACPCG_ECUDA;
    if (s->stop) return JACPCG_EBUSY;
    if (s->cfg.max_queue > 0 && s->n_pending >= (size_t)s->cfg.max_queue) return JACPCG_EBUSY;
    Request r{s->next_ticket++, *inst, now_us()};
    Result res;
    res.t_submit = r.t_submit;
    s->results.emplace(r.ticket, res);
    s->queue[s->cfg.batch_policy == JACPCG_BATCH_COST_CLASS ? cost_class(r.inst) : 0].push_back(r);
    ++s->n_pending;
    *ticket = r.ticket;
    s->cv_work.notify_one();
    return JACPCG_OK;
}

jacpcg_status jacpcg_poll(jacpcg_server *s, uint64_t ticket, jacpcg_status *result,
                          double *latency_us, int blocking) {
    if (!s || !result) return JACPCG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return JACPCG_EINVAL;
    if (blocking) {
        const auto limit = clk::now() + std::chrono::seconds(60);
        while (it->second.state == 0) {
            if (s->cv_done.wait_until(lk, limit) == std::cv_status::timeout && it->second.state == 0)
                return JACPCG_ETIMEOUT;
            it = s->results.find(ticket);
            if (it == s->results.end()) return JACPCG_EINVAL;
        }
    }
    if (it->second.state == 0) return JACPCG_EBUSY;
    *result = it->second.status;
    if (latency_us) *latency_us = it->second.latency_us;
    s->results.erase(it);
    return JACPCG_OK;
}

jacpcg_status jacpcg_server_replay(jacpcg_server *s, const jacpcg_instance *pool, int n_pool,
                                   const int *which, const double *arrival_us, int n_req,
                                   double *latency_us, int32_t *status) {
    if (!s || !pool || !which || !arrival_us || n_pool < 1 || n_req < 0) return JACPCG_EINVAL;
    for (int i = 0; i < n_req; ++i)
        if (which[i] < 0 || which[i] >= n_pool) return JACPCG_EINVAL;
    std::vector<uint64_t> tickets(n_req, 0);
    std::vector<jacpcg_status> sub(n_req, JACPCG_OK);
    const double t0 = now_us();
    for (int i = 0; i < n_req; ++i) {
        while (now_us() - t0 < arrival_us[i]) {
        }
        sub[i] = jacpcg_submit(s, &pool[which[i]], &tickets[i]);
    }
    jacpcg_status worst = JACPCG_OK;
    for (int i = 0; i < n_req; ++i) {
        jacpcg_status r = sub[i];
        double lat = -1.0;
        if (r == JACPCG_OK) {
            jacpcg_status pst = jacpcg_poll(s, tickets[i], &r, &lat, 1);
            if (pst != JACPCG_OK) r = pst;
        }
        if (latency_us) latency_us[i] = lat;
        if (status) status[i] = r;
        if (r == JACPCG_ECUDA || r == JACPCG_ETIMEOUT) worst = r;
    }
    return worst;
}

jacpcg_status jacpcg_server_stats(jacpcg_server *s, uint64_t *n_done, uint64_t *n_batches,
                                  double *mean_batch) {
    if (!s) return JACPCG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (n_done) *n_done = s->n_done;
    if (n_batches) *n_batches = s->n_batches;
    if (mean_batch) *mean_batch = s->n_batches ? s->sum_batch / (double)s->n_batches : 0.0;
    return JACPCG_OK;
}

jacpcg_status jacpcg_server_destroy(jacpcg_server *s) {
    if (!s) return JACPCG_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto st : s->streams)
        if (st) cudaStreamSynchronize(st);
    for (size_t k = 0; k < s->streams.size(); ++k) {
        if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
        if (s->status_dev[k]) cudaFree(s->status_dev[k]);
        if (s->status_host[k]) cudaFreeHost(s->status_host[k]);
        if (s->plain_ws[k]) cudaFree(s->plain_ws[k]);
    }
    (void)cudaGetLastError();
    delete s;
    return JACPCG_OK;
}

}  // extern "C"
