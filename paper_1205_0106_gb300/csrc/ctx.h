// The amc_ctx structure and the batch-launch helpers shared by the C-ABI
// runtime (runtime.cu) and the serving loop (serve.cpp).  Internal.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace amc {

struct DevBridge {
    NodeF *nf = nullptr;
    NodeD *nd = nullptr;
    int nslots = 0;
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bump allocator over a fixed region of device memory.
struct SubArena {
    char *base = nullptr;
    size_t size = 0, top = 0;
    int alloc(size_t bytes, void **p) {
        const size_t off = align_up(top, 256);
        if (off + bytes > size) return AMC_ENOMEM;
        *p = base + off;
        top = off + bytes;
        return AMC_OK;
    }
};

struct Server;   // serve.cpp

}  // namespace amc

struct amc_ctx {
    int device = 0;
    int sm_count = 0;
    int max_cluster = 0;                             // largest cluster sweep the device holds (0: none)
    cudaStream_t stream = nullptr;
    cudaStream_t bstream[2] = {nullptr, nullptr};   // batch waves, double-buffered
    double *bres_host[2] = {nullptr, nullptr};       // pinned wave results
    int batch_cap = 4096;                            // options per wave
    // path arena (bump allocation, reset by each host-level call)
    char *arena = nullptr;
    size_t arena_bytes = 0, arena_top = 0;
    // tables
    uint32_t *V = nullptr;                           // [AMC_MAX_STEPS][32]
    std::unordered_map<int, amc::DevBridge> bridges;  // by n_steps
    // single-option scratch (step-level calls); the job itself travels by
    // value in the kernel arguments
    amc::KArgs args;
    uint32_t *shift1 = nullptr;
    void *part1 = nullptr;
    uint32_t *arrive1 = nullptr;
    double *fin1 = nullptr;
    double *res1 = nullptr;
    int32_t *status1 = nullptr;
    double *finv = nullptr;                          // per-CTA sums of the boundary valuation (grown on demand)
    int64_t finv_ctas = 0;
    double *dualw = nullptr;                         // per-path L_1, V and inner steps of the dual upper bound (grown on demand)
    int64_t dualw_n = 0;
    double *streamw = nullptr;                       // streaming LSM sweep: cash flows, partials, coefficients (grown on demand)
    int64_t streamw_n = 0;
    uint64_t *xch1 = nullptr;                        // exchange units of the mixed LSM sweep
    uint32_t epoch = 0;                              // launch tag of those units
    int gcap = 0;
    double *res_host = nullptr;                      // pinned
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t bev[3] = {nullptr, nullptr, nullptr};  // ordering of the batch streams with a caller's stream
    double timeout_s = 2.0;
    uint32_t poll_ns = 0;                            // exchange poll back-off, ns (AMC_POLL_NS overrides)
    int inject_kind = 0;
    int64_t inject_arg = 0;
    // opt-in profiling of path generation and sweep launches (events)
    struct Prof {
        bool on = false;
        std::vector<cudaEvent_t> pool;                // free events
        struct Rec { cudaEvent_t a, b; int kind; int64_t units; };
        std::vector<Rec> recs;                        // kind 0: path generation, 1: sweep
    } prof;
    std::mutex mu;                                   // launches and tables
    amc::Server *server = nullptr;                   // running serving loop, if any
};

namespace amc {

// Options that can share one launch have the same group key.
struct GroupKey {
    int kind, type, chunks;
    bool lsm;
    int cubic;                      // cluster sweep: p = 4 (its own kernel variant)
    bool operator==(const GroupKey &o) const {
        return kind == o.kind && type == o.type && chunks == o.chunks && lsm == o.lsm && cubic == o.cubic;
    }
};
GroupKey group_key(const amc_option &o, const SweepPlan &pl);
// CTAs one launch of this group may use (co-resident capacity).
int group_cta_cap(amc_ctx *c, const SweepPlan &pl);
// Device bytes one option of a group needs (paths and sweep scratch).
size_t option_bytes(const amc_option &o, const SweepPlan &pl, int prec);
// Device-side inputs and outputs of a batch (the _device calls): spot and
// volatility overrides and result arrays indexed by input position, any of
// them null.  `idx` gives the input position of each option of the wave.
struct DeviceIO {
    const double *S0 = nullptr, *sigma = nullptr;
    double *res = nullptr, *price = nullptr, *delta = nullptr, *vega = nullptr;
    const int32_t *idx = nullptr;      // host, one per option of the wave
};
// Launch path generation, sweep and finalize for n options of one group on
// stream st, memory from ar; results (AMC_RES_DOUBLES per option, wave
// order) in *res_dev, and scattered to io's arrays when io is given.
// Asynchronous.  Caller holds c->mu.
int launch_group(amc_ctx *c, const amc_option *const *opts, const SweepPlan *plans, int n, int prec, bool greeks,
                 SubArena &ar, cudaStream_t st, double **res_dev, const DeviceIO *io = nullptr);
int result_from(const double *r, amc_result *out);
// Profiling (no-op unless enabled): an event before a launch, and after it
// the record of its kind and work units (path-steps).  Caller holds c->mu.
cudaEvent_t prof_begin(amc_ctx *c, cudaStream_t st);
void prof_end(amc_ctx *c, cudaEvent_t a, int kind, int64_t units, cudaStream_t st);

}  // namespace amc
