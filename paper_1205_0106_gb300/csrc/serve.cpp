// Serving loop: continuous batching of pricing requests on one GPU.
//
// A host scheduler thread owns the context while serving runs.  Requests are
// queued by amc_serve_submit (thread-safe, non-blocking).  The device memory
// budget is split into `slots` sub-arenas, each with its own CUDA stream;
// whenever a slot is free the scheduler admits the oldest pending requests
// that share a launch group and fit the slot's memory and the co-resident
// CTA capacity, and launches their path generation, sweep and finalize on
// the slot's stream.  Several slots run at once, so requests that arrive
// while others are on the GPU overlap with them on the device.  Completion
// is detected with a CUDA event per batch; results are copied to pinned
// host memory and handed out by amc_serve_poll / amc_serve_drain with the
// request's latency (submit to completion, host monotonic clock).
// Each option keeps its own CTA group and reduction order, so its result
// is bit-identical whether it is served alone or among others.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx.h"
#include "trace.h"

namespace amc {

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    amc_option opt;
    SweepPlan plan;
    GroupKey key;
    size_t bytes = 0;
    double t_submit = 0.0, t_done = 0.0;
    amc_result res;
    bool done = false;
    bool returned = false;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    SubArena ar;
    double *res_host = nullptr;          // pinned, max_batch * AMC_RES_DOUBLES
    std::vector<uint64_t> tickets;
    bool busy = false;
};

}  // namespace

struct Server {
    amc_ctx *c = nullptr;
    amc_serve_config cfg;
    std::thread th;
    std::mutex mu;                       // pending queue and request table
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<Slot> slots;
    uint64_t next_ticket = 1;
    bool stopping = false;
    int error = AMC_OK;
    amc_serve_stats stats;

    void loop();
    bool launch_into(Slot &sl, std::unique_lock<std::mutex> &lk);
    bool collect(Slot &sl);
};

// Admit and launch one batch into a free slot: the oldest pending request
// fixes the group; later pending requests of the same group are added while
// they fit (bytes, CTAs, batch size).  Called with `mu` held; drops it
// around the launch.
bool Server::launch_into(Slot &sl, std::unique_lock<std::mutex> &lk) {
    if (pending.empty()) return false;
    TraceRange trace_range("amc serve batch");
    const Request &head = reqs[pending.front()];
    const GroupKey key = head.key;
    const int cap = group_cta_cap(c, head.plan);
    std::vector<uint64_t> take;
    size_t bytes = 4096;
    int ctas = 0;
    for (auto it = pending.begin(); it != pending.end() && (int)take.size() < cfg.max_batch;) {
        const Request &r = reqs[*it];
        if (r.key == key && bytes + r.bytes <= sl.ar.size && ctas + r.plan.ctas <= cap) {
            bytes += r.bytes;
            ctas += r.plan.ctas;
            take.push_back(*it);
            it = pending.erase(it);
        } else {
            ++it;
        }
    }
    if (take.empty()) return false;
    std::vector<amc_option> opts(take.size());
    std::vector<SweepPlan> plans(take.size());
    for (size_t k = 0; k < take.size(); ++k) {
        opts[k] = reqs[take[k]].opt;
        plans[k] = reqs[take[k]].plan;
    }
    lk.unlock();
    std::vector<const amc_option *> ptrs(take.size());
    for (size_t k = 0; k < take.size(); ++k) ptrs[k] = &opts[k];
    sl.ar.top = 0;
    double *res_dev = nullptr;
    int rc;
    {
        std::lock_guard<std::mutex> g(c->mu);
        rc = launch_group(c, ptrs.data(), plans.data(), (int)take.size(), cfg.prec, false, sl.ar, sl.st, &res_dev);
    }
    if (rc == AMC_OK &&
        cudaMemcpyAsync(sl.res_host, res_dev, sizeof(double) * AMC_RES_DOUBLES * take.size(), cudaMemcpyDeviceToHost,
                        sl.st) != cudaSuccess)
        rc = AMC_ECUDA;
    if (rc == AMC_OK && cudaEventRecord(sl.ev, sl.st) != cudaSuccess) rc = AMC_ECUDA;
    lk.lock();
    if (rc != AMC_OK) {
        for (uint64_t t : take) {           // fail these requests
            Request &r = reqs[t];
            memset(&r.res, 0, sizeof(r.res));
            r.res.status = rc;
            r.done = true;
            r.t_done = now_s();
        }
        error = rc;
        cv.notify_all();
        return false;
    }
    sl.tickets = take;
    sl.busy = true;
    stats.batches += 1;
    stats.launched += (int64_t)take.size();
    return true;
}

// If the slot's batch has finished, publish its results.  `mu` held.
bool Server::collect(Slot &sl) {
    if (!sl.busy) return false;
    const cudaError_t q = cudaEventQuery(sl.ev);
    if (q == cudaErrorNotReady) return false;
    const double t = now_s();
    for (size_t k = 0; k < sl.tickets.size(); ++k) {
        Request &r = reqs[sl.tickets[k]];
        if (q == cudaSuccess) {
            result_from(sl.res_host + k * AMC_RES_DOUBLES, &r.res);
        } else {
            memset(&r.res, 0, sizeof(r.res));
            r.res.status = AMC_ECUDA;
        }
        r.done = true;
        r.t_done = t;
    }
    stats.completed += (int64_t)sl.tickets.size();
    sl.tickets.clear();
    sl.busy = false;
    cv.notify_all();
    return true;
}

void Server::loop() {
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progress = false;
        for (Slot &sl : slots) progress |= collect(sl);
        for (Slot &sl : slots)
            if (!sl.busy && !pending.empty()) progress |= launch_into(sl, lk);
        bool busy = false;
        for (Slot &sl : slots) busy |= sl.busy;
        if (stopping && pending.empty() && !busy) break;
        if (!progress) {
            // wait for a submission, or poll the in-flight batches again soon
            cv.wait_for(lk, std::chrono::microseconds(busy ? 20 : 2000));
        }
    }
}

}  // namespace amc

using namespace amc;

extern "C" {

int amc_serve_start(amc_ctx *c, const amc_serve_config *cfg) {
    if (!c || !cfg || cfg->slots < 1 || cfg->slots > 8 || cfg->max_batch < 1 || cfg->max_batch > 4096 ||
        (cfg->prec != AMC_FP64 && cfg->prec != AMC_MIXED))
        return AMC_EINVAL;
    if (c->server) return AMC_EBUSY;
    if (cudaSetDevice(c->device) != cudaSuccess) return AMC_ECUDA;
    const size_t per = cfg->slot_bytes ? cfg->slot_bytes : (c->arena_bytes / cfg->slots) / 4096 * 4096;
    if (per * cfg->slots > c->arena_bytes || per < (1u << 20)) return AMC_ENOMEM;
    Server *s = new Server();
    s->c = c;
    s->cfg = *cfg;
    s->cfg.slot_bytes = per;
    memset(&s->stats, 0, sizeof(s->stats));
    s->slots.resize(cfg->slots);
    int rc = AMC_OK;
    for (int k = 0; k < cfg->slots && rc == AMC_OK; ++k) {
        Slot &sl = s->slots[k];
        sl.ar.base = c->arena + (size_t)k * per;
        sl.ar.size = per;
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.res_host, sizeof(double) * AMC_RES_DOUBLES * cfg->max_batch) != cudaSuccess)
            rc = AMC_ECUDA;
        // the slots reuse the arena: after any device-form batch still in flight
        for (int h = 1; h < 3 && rc == AMC_OK; ++h)
            if (cudaStreamWaitEvent(sl.st, c->bev[h], 0) != cudaSuccess) rc = AMC_ECUDA;
    }
    if (rc != AMC_OK) {
        for (Slot &sl : s->slots) {
            if (sl.st) cudaStreamDestroy(sl.st);
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.res_host) cudaFreeHost(sl.res_host);
        }
        delete s;
        return rc;
    }
    c->server = s;
    s->th = std::thread([s] { s->loop(); });
    return AMC_OK;
}

int amc_serve_submit(amc_ctx *c, const amc_option *opt, uint64_t *ticket) {
    if (!c || !opt || !ticket) return AMC_EINVAL;
    Server *s = c->server;
    if (!s) return AMC_EINVAL;
    int rc = host_validate(opt);
    if (rc != AMC_OK) return rc;
    Request r;
    r.opt = *opt;
    rc = host_plan_sweep(opt->n_paths, c->sm_count, s->cfg.prec, opt->rule, &r.plan, c->max_cluster);
    if (rc != AMC_OK) return rc;
    r.key = group_key(*opt, r.plan);
    r.bytes = option_bytes(*opt, r.plan, s->cfg.prec);
    if (r.bytes + 4096 > s->cfg.slot_bytes || r.plan.ctas > group_cta_cap(c, r.plan)) return AMC_EBUSY;
    r.t_submit = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return AMC_EBUSY;
    if ((int64_t)s->pending.size() >= s->cfg.max_pending) {
        s->stats.rejected += 1;
        return AMC_EBUSY;
    }
    const uint64_t t = s->next_ticket++;
    s->reqs.emplace(t, r);
    s->pending.push_back(t);
    s->stats.submitted += 1;
    *ticket = t;
    s->cv.notify_all();
    return AMC_OK;
}

int amc_serve_poll(amc_ctx *c, uint64_t ticket, amc_result *out, double *latency_s) {
    if (!c || !out) return AMC_EINVAL;
    Server *s = c->server;
    if (!s) return AMC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return AMC_ENOTFOUND;
    if (!it->second.done) return AMC_PENDING;
    *out = it->second.res;
    if (latency_s) *latency_s = it->second.t_done - it->second.t_submit;
    s->reqs.erase(it);
    return AMC_OK;
}

int amc_serve_drain(amc_ctx *c, uint64_t *tickets, amc_result *out, double *latency_s, int cap, int *n_out) {
    if (!c || !tickets || !out || !n_out || cap < 0) return AMC_EINVAL;
    Server *s = c->server;
    if (!s) return AMC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    for (auto it = s->reqs.begin(); it != s->reqs.end() && n < cap;) {
        if (it->second.done) {
            tickets[n] = it->first;
            out[n] = it->second.res;
            if (latency_s) latency_s[n] = it->second.t_done - it->second.t_submit;
            ++n;
            it = s->reqs.erase(it);
        } else {
            ++it;
        }
    }
    *n_out = n;
    return AMC_OK;
}

int amc_serve_cancel(amc_ctx *c, uint64_t ticket) {
    if (!c) return AMC_EINVAL;
    Server *s = c->server;
    if (!s) return AMC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return AMC_ENOTFOUND;
    auto q = std::find(s->pending.begin(), s->pending.end(), ticket);
    if (q == s->pending.end()) return AMC_EBUSY;   // in a batch on the GPU, or finished
    s->pending.erase(q);
    Request &r = it->second;
    memset(&r.res, 0, sizeof(r.res));
    r.res.status = AMC_ECANCELED;
    r.done = true;
    r.t_done = now_s();
    s->stats.cancelled += 1;
    s->cv.notify_all();
    return AMC_OK;
}

int amc_serve_stats_get(amc_ctx *c, amc_serve_stats *out) {
    if (!c || !out) return AMC_EINVAL;
    Server *s = c->server;
    if (!s) return AMC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->pending = (int64_t)s->pending.size();
    return AMC_OK;
}

int amc_serve_stop(amc_ctx *c) {
    if (!c) return AMC_EINVAL;
    Server *s = c->server;
    if (!s) return AMC_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cv.notify_all();
    }
    s->th.join();
    for (Slot &sl : s->slots) {
        cudaStreamSynchronize(sl.st);
        cudaStreamDestroy(sl.st);
        cudaEventDestroy(sl.ev);
        cudaFreeHost(sl.res_host);
    }
    const int err = s->error;
    c->server = nullptr;
    delete s;
    return err;
}

}  // extern "C"
