// C ABI runtime of the amc library: contexts, the device arena, option
// validation, job packing and the launch sequence of the hot path
// (path generation -> sweep -> finalize) and of the second pass, the dual
// bound and the no-path-array pricing.  Everything that computes runs in the
// kernels of pathgen.cu, sweep_v2.cu, sweep.cu, sweep_stream.cu, value.cu
// and dual.cu; this file only plans and launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace amc;

#include "ctx.h"
#include "trace.h"

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? AMC_OK : AMC_ECUDA; }

#define AMC_TRY_CUDA(x)                         \
    do {                                        \
        cudaError_t _e = (x);                   \
        if (_e != cudaSuccess) return AMC_ECUDA; \
    } while (0)
#define AMC_TRY(x)                 \
    do {                           \
        int _r = (x);              \
        if (_r != AMC_OK) return _r; \
    } while (0)

int get_bridge(amc_ctx *c, int m, DevBridge **out) {
    auto it = c->bridges.find(m);
    if (it != c->bridges.end()) {
        *out = &it->second;
        return AMC_OK;
    }
    BridgePlan plan;
    AMC_TRY(host_bridge_plan(m, &plan));
    DevBridge b;
    b.nslots = plan.nslots;
    AMC_TRY_CUDA(cudaMalloc(&b.nf, sizeof(NodeF) * m));
    AMC_TRY_CUDA(cudaMalloc(&b.nd, sizeof(NodeD) * m));
    AMC_TRY_CUDA(cudaMemcpy(b.nf, plan.nf.data(), sizeof(NodeF) * m, cudaMemcpyHostToDevice));
    AMC_TRY_CUDA(cudaMemcpy(b.nd, plan.nd.data(), sizeof(NodeD) * m, cudaMemcpyHostToDevice));
    c->bridges[m] = b;
    *out = &c->bridges[m];
    return AMC_OK;
}

int arena_alloc(amc_ctx *c, size_t bytes, void **p) {
    if (c->inject_kind == 2) {
        c->inject_kind = 0;
        return AMC_ENOMEM;
    }
    size_t off = align_up(c->arena_top, 256);
    if (off + bytes > c->arena_bytes) return AMC_ENOMEM;
    *p = c->arena + off;
    c->arena_top = off + bytes;
    return AMC_OK;
}

// Option fields shared by every job; device pointers are filled by callers.
void fill_job_common(const amc_option *o, Job *J) {
    memset(J, 0, sizeof(*J));
    J->S0 = o->S0; J->K = o->K; J->r = o->r; J->sigma = o->sigma; J->T = o->T;
    J->m = o->n_steps;
    J->p = o->rule == AMC_RULE_LSM ? o->basis : 1;
    J->type = o->type;
    J->rule = o->rule;
    J->N = o->n_paths;
    J->dt = o->T / o->n_steps;
    J->disc = exp(-o->r * J->dt);
    J->invK = 1.0 / o->K;
}

uint64_t timeout_ns(const amc_ctx *c) { return (uint64_t)(c->timeout_s * 1e9); }

// Next launch tag of the mixed LSM sweep's exchange units.  The
// single-option buffer xch1 only ever holds units, and tags never repeat
// within 2^22 launches; when the counter wraps it is cleared first.  The
// batch and serving launches take their units from the arena, whose bytes
// held other data before, so launch_group clears them on the launch stream
// before every launch instead.  A test can make the next launch reuse an
// earlier launch's tag (amc_ctx_inject kind 4; batch and serving launches
// only, whose units are cleared per launch: xch1 relies on unique tags).
uint32_t next_epoch(amc_ctx *c, bool from_arena) {
    if (from_arena && c->inject_kind == 4) {
        c->inject_kind = 0;
        c->epoch = (uint32_t)c->inject_arg;
        return c->epoch;
    }
    c->epoch = (c->epoch + 1) & ((1u << kEpochBits) - 1u);
    if (c->epoch == 0) {
        cudaDeviceSynchronize();
        cudaMemset(c->xch1, 0, sizeof(uint64_t) * v2_xch_units(AMC_MAX_STEPS, kV2MaxCtas));
        c->epoch = 1;
    }
    return c->epoch;
}

// Launch the sweep of the packed jobs in `a` (same precision, same plan
// kind and chunk count, same rule class) and their finalize.
int launch_sweeps(amc_ctx *c, KArgs &a, const SweepPlan &pl, int total_ctas, bool lsm, bool fp64, bool greeks,
                  cudaStream_t st, bool from_arena = false, int64_t units = 0) {
    a.timeout_ns = timeout_ns(c);
    cudaEvent_t pe = prof_begin(c, st);
    cudaError_t e;
    if (pl.kind == 3) {
        e = launch_sweep_cl(a, pl.ctas, total_ctas / pl.ctas, st);
    } else if (pl.kind == 2) {
        a.epoch = next_epoch(c, from_arena);
        a.poll_ns = c->poll_ns;
        e = launch_sweep_lsm_v2(a, total_ctas, greeks, st);
    } else if (lsm) {
        e = launch_sweep_lsm(a, total_ctas, pl.chunks, fp64, greeks, st);
    } else {
        e = launch_sweep_pathwise(a, total_ctas, pl.chunks, fp64, greeks, st);
    }
    AMC_TRY_CUDA(e);
    prof_end(c, pe, 1, units, st);
    AMC_TRY_CUDA(launch_finalize(a, st));
    return AMC_OK;
}

// Context scratch of `count` doubles, grown on demand (a cudaFree and a
// cudaMalloc, which synchronise the device once); *have tracks the size in
// units of `per` doubles.
int grow_scratch(double **buf, int64_t *have, int64_t need, size_t per) {
    if (need <= *have) return AMC_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc(buf, sizeof(double) * per * (size_t)need) != cudaSuccess) return AMC_ENOMEM;
    *have = need;
    return AMC_OK;
}

// AMC_MIXED16 only where the caller allows it (the LSM sweeps and path
// generation into a caller array).
int check_prec(int prec, bool h16_ok = false) {
    if (prec == AMC_FP64 || prec == AMC_MIXED) return AMC_OK;
    return (prec == AMC_MIXED16 && h16_ok) ? AMC_OK : AMC_EINVAL;
}
size_t elem_bytes(int prec) { return prec == AMC_FP64 ? 8 : (prec == AMC_MIXED16 ? 2 : 4); }

// Caller path storage: rows must start on 16-byte boundaries for the
// vector loads and stores, so S must be 16-byte aligned and ld a multiple
// of 32 elements (amc_path_ld rounds to that).
int check_storage(const void *S, int64_t ld, int64_t n_paths) {
    if (!S || ld < host_ld(n_paths) || ld % 32 != 0 || ((uintptr_t)S & 15u) != 0) return AMC_EINVAL;
    return AMC_OK;
}

int do_generate(amc_ctx *c, const amc_option *o, int prec, void *S, int64_t ld, cudaStream_t st) {
    AMC_TRY(host_validate(o));
    AMC_TRY(check_prec(prec, true));
    AMC_TRY(check_storage(S, ld, o->n_paths));
    DevBridge *b;
    AMC_TRY(get_bridge(c, o->n_steps, &b));
    KArgs &a = c->args;
    memset(&a, 0, sizeof(KArgs));
    Job &J = a.one;
    fill_job_common(o, &J);
    host_shifts(o->seed, o->n_steps, a.shift_one);
    J.nodes = prec == AMC_FP64 ? (const void *)b->nd : (const void *)b->nf;
    J.nslots = b->nslots;
    J.S = S;
    J.ld = ld;
    J.tile_begin = 0;
    J.n_tiles = (o->n_paths + kTilePoints - 1) / kTilePoints;
    a.jobs = nullptr;
    a.n_jobs = 1;
    a.max_m = o->n_steps;
    a.max_slots = b->nslots;
    a.total = J.n_tiles;
    a.V = c->V;
    a.h16 = prec == AMC_MIXED16 ? 1 : 0;
    cudaEvent_t pe = prof_begin(c, st);
    AMC_TRY_CUDA(launch_pathgen(a, prec == AMC_FP64, c->sm_count, st));
    prof_end(c, pe, 0, o->n_paths * (int64_t)o->n_steps, st);
    return AMC_OK;
}

// Paths from the paper's LCG-permuted unshifted points (one launch).
int do_generate_permuted(amc_ctx *c, const amc_option *o, int prec, void *S, int64_t ld, cudaStream_t st) {
    AMC_TRY(host_validate(o));
    AMC_TRY(check_prec(prec));
    AMC_TRY(check_storage(S, ld, o->n_paths));
    DevBridge *b;
    AMC_TRY(get_bridge(c, o->n_steps, &b));
    static thread_local PermArgs a;
    memset(&a, 0, sizeof(PermArgs));
    Job &J = a.one;
    fill_job_common(o, &J);
    J.nodes = prec == AMC_FP64 ? (const void *)b->nd : (const void *)b->nf;
    J.nslots = b->nslots;
    J.S = S;
    J.ld = ld;
    uint64_t M = 1;
    host_lcg_params(o->seed, o->n_steps, o->n_paths, a.a, a.c, &M);
    while ((1ull << a.log2M) < M) ++a.log2M;
    a.V = c->V;
    a.max_slots = b->nslots;
    a.total = (o->n_paths + kTilePoints - 1) / kTilePoints;
    AMC_TRY_CUDA(launch_pathgen_permuted(a, prec == AMC_FP64, c->sm_count, st));
    return AMC_OK;
}

// LSM sweep of an option too large for the register-resident sweeps: one
// streaming pass and one solve per date, scratch in context memory.
int do_sweep_stream(amc_ctx *c, const amc_option *o, int prec, const void *S, int64_t ld, double *res,
                    cudaStream_t st, double *coef) {
    const bool fp64 = prec == AMC_FP64;
    StreamArgs sa;
    memset(&sa, 0, sizeof(sa));
    Job &J = sa.one;
    fill_job_common(o, &J);
    J.S = const_cast<void *>(S);
    J.ld = ld;
    J.res = res;
    J.status = c->status1;
    J.coef = coef;
    sa.h16 = prec == AMC_MIXED16 ? 1 : 0;
    const int64_t grid = stream_grid(c->sm_count, fp64, o->type == AMC_PUT, sa.h16 != 0);
    // cash flows [ld] (up to 8 bytes each), partials [grid][kNV], coefficients
    // [AMC_MAX_STEPS][4], then degenerate flags and count (int32, in doubles)
    const int64_t n_flags = (AMC_MAX_STEPS + 2) / 2;
    AMC_TRY(grow_scratch(&c->streamw, &c->streamw_n, ld + grid * kNV + (int64_t)AMC_MAX_STEPS * 4 + n_flags, 1));
    sa.cf = c->streamw;
    sa.part = c->streamw + ld;
    sa.beta = sa.part + grid * kNV;
    sa.deg = reinterpret_cast<int32_t *>(sa.beta + (int64_t)AMC_MAX_STEPS * 4);
    sa.ndeg = sa.deg + AMC_MAX_STEPS;
    sa.grid = (int32_t)grid;
    AMC_TRY(grow_scratch(&c->finv, &c->finv_ctas, grid, 4));
    J.fin = c->finv;
    J.n_cta = (int)grid;
    AMC_TRY_CUDA(cudaMemsetAsync(sa.deg, 0, sizeof(int32_t) * (AMC_MAX_STEPS + 1), st));
    AMC_TRY_CUDA(cudaMemsetAsync(c->status1, 0, sizeof(int32_t), st));
    AMC_TRY_CUDA(launch_lsm_stream(sa, fp64, st));
    KArgs &a = c->args;
    memset(&a, 0, sizeof(KArgs));
    a.one = J;
    a.n_jobs = 1;
    AMC_TRY_CUDA(launch_finalize(a, st));
    return AMC_OK;
}

int do_sweep(amc_ctx *c, const amc_option *o, int prec, const void *S, int64_t ld, bool greeks, double *res,
             cudaStream_t st, double *coef = nullptr) {
    AMC_TRY(host_validate(o));
    AMC_TRY(check_prec(prec, o->rule == AMC_RULE_LSM && !greeks));
    AMC_TRY(check_storage(S, ld, o->n_paths));
    if (!res || ((uintptr_t)res & 7u) != 0) return AMC_EINVAL;
    if (greeks && o->rule == AMC_RULE_PAPER_UB) return AMC_EINVAL;
    if (c->inject_kind == 3 && o->rule == AMC_RULE_LSM && !greeks) {
        c->inject_kind = 0;
        return do_sweep_stream(c, o, prec, S, ld, res, st, coef);
    }
    SweepPlan pl;
    bool big = false;                                 // too many paths for the co-resident plans
    if (host_plan_sweep(o->n_paths, c->sm_count, prec, o->rule, &pl, greeks ? 0 : c->max_cluster) != AMC_OK ||
        pl.ctas > c->gcap) {
        if (greeks) return AMC_EINVAL;                // frozen-boundary Greeks: register-resident sizes only
        if (o->rule == AMC_RULE_LSM) return do_sweep_stream(c, o, prec, S, ld, res, st, coef);
        // the pathwise rules need no co-resident CTAs: any grid, 8 paths per thread
        pl.kind = 1;
        pl.chunks = 2;
        pl.ctas = (int)((o->n_paths + (int64_t)kSweepThreads * 8 - 1) / ((int64_t)kSweepThreads * 8));
        big = true;
    }
    KArgs &a = c->args;
    memset(&a, 0, sizeof(KArgs));
    Job &J = a.one;
    fill_job_common(o, &J);
    J.S = const_cast<void *>(S);
    J.ld = ld;
    J.cta_begin = 0;
    J.n_cta = pl.ctas;
    J.chunks = pl.chunks;
    J.greeks = greeks ? 1 : 0;
    J.part = c->part1;
    J.arrive = c->arrive1;
    J.fin = c->fin1;
    if (big) {
        AMC_TRY(grow_scratch(&c->finv, &c->finv_ctas, pl.ctas, 4));
        J.fin = c->finv;
    }
    J.res = res;
    J.status = c->status1;
    J.xch = c->xch1;
    J.coef = coef;
    if (c->inject_kind == 1) {
        J.inject_date = (int32_t)c->inject_arg;
        c->inject_kind = 0;
    }
    a.jobs = nullptr;
    a.n_jobs = 1;
    a.max_m = o->n_steps;
    a.V = c->V;
    a.h16 = prec == AMC_MIXED16 ? 1 : 0;
    if (a.h16 && pl.kind < 2) return AMC_EINVAL;      // the binary16 format is read by the mixed LSM sweeps only
    if (pl.kind == 1 && o->rule == AMC_RULE_LSM)
        AMC_TRY_CUDA(cudaMemsetAsync(c->arrive1, 0, sizeof(uint32_t) * o->n_steps, st));
    AMC_TRY_CUDA(cudaMemsetAsync(c->status1, 0, sizeof(int32_t), st));
    return launch_sweeps(c, a, pl, pl.ctas, o->rule == AMC_RULE_LSM, prec == AMC_FP64, greeks, st, false,
                         o->n_paths * (int64_t)o->n_steps);
}


// Valuation of caller paths with a given boundary (one streaming launch and
// its finalize; the grid covers 8 paths per thread, at most gcap CTAs).
int do_value(amc_ctx *c, const amc_option *o, int prec, const void *S, int64_t ld, const double *coef, double *res,
             cudaStream_t st) {
    AMC_TRY(host_validate(o));
    AMC_TRY(check_prec(prec));
    AMC_TRY(check_storage(S, ld, o->n_paths));
    if (o->rule != AMC_RULE_LSM || !coef || ((uintptr_t)coef & 7u) != 0 || !res || ((uintptr_t)res & 7u) != 0)
        return AMC_EINVAL;
    KArgs &a = c->args;
    memset(&a, 0, sizeof(KArgs));
    Job &J = a.one;
    fill_job_common(o, &J);
    J.S = const_cast<void *>(S);
    J.ld = ld;
    J.coef = const_cast<double *>(coef);
    const int64_t ctas = value_ctas(o->n_paths);
    AMC_TRY(grow_scratch(&c->finv, &c->finv_ctas, ctas, 4));
    J.n_cta = (int)ctas;
    J.fin = c->finv;
    J.res = res;
    J.status = c->status1;
    a.n_jobs = 1;
    a.max_m = o->n_steps;
    a.timeout_ns = timeout_ns(c);
    AMC_TRY_CUDA(cudaMemsetAsync(c->status1, 0, sizeof(int32_t), st));
    AMC_TRY_CUDA(launch_value_boundary(a, J.n_cta, prec == AMC_FP64, st));
    AMC_TRY_CUDA(launch_finalize(a, st));
    return AMC_OK;
}

// Steps 1-4 without a path array: path generation values every path as it
// is formed (the paper's rule, the European estimator, or a fitted
// boundary's valuation), then the fixed-order finalize.
int do_fused(amc_ctx *c, const amc_option *o, int prec, const double *coef, double *res, cudaStream_t st) {
    AMC_TRY(host_validate(o));
    AMC_TRY(check_prec(prec));
    const bool lsm = o->rule == AMC_RULE_LSM;
    if (!res || ((uintptr_t)res & 7u) != 0 || (lsm != (coef != nullptr)) || ((uintptr_t)coef & 7u) != 0)
        return AMC_EINVAL;
    DevBridge *b;
    AMC_TRY(get_bridge(c, o->n_steps, &b));
    KArgs &a = c->args;
    memset(&a, 0, sizeof(KArgs));
    Job &J = a.one;
    fill_job_common(o, &J);
    host_shifts(o->seed, o->n_steps, a.shift_one);
    J.nodes = prec == AMC_FP64 ? (const void *)b->nd : (const void *)b->nf;
    J.nslots = b->nslots;
    J.n_tiles = (o->n_paths + kTilePoints - 1) / kTilePoints;
    J.coef = const_cast<double *>(coef);
    J.res = res;
    J.status = c->status1;
    a.n_jobs = 1;
    a.max_m = o->n_steps;
    a.max_slots = b->nslots;
    a.total = J.n_tiles;
    a.V = c->V;
    const int mode = lsm ? kBoundary : (o->rule == AMC_RULE_PAPER_UB ? kPaperRule : kEuropean);
    int64_t grid = 0;
    AMC_TRY_CUDA(pathgen_fused_grid(a, mode, prec == AMC_FP64, c->sm_count, &grid));
    AMC_TRY(grow_scratch(&c->finv, &c->finv_ctas, grid, 4));
    J.fin = c->finv;
    J.n_cta = (int)grid;
    AMC_TRY_CUDA(cudaMemsetAsync(c->status1, 0, sizeof(int32_t), st));
    AMC_TRY_CUDA(launch_pathgen_fused(a, mode, prec == AMC_FP64, grid, st));
    AMC_TRY_CUDA(launch_finalize(a, st));
    return AMC_OK;
}

int do_dual(amc_ctx *c, const amc_option *o, int prec, const void *S, int64_t ld, const double *coef, int64_t n_in,
            uint64_t seed_in, double *res, double *U, cudaStream_t st) {
    AMC_TRY(host_validate(o));
    AMC_TRY(check_prec(prec));
    AMC_TRY(check_storage(S, ld, o->n_paths));
    if (o->rule != AMC_RULE_LSM || !coef || ((uintptr_t)coef & 7u) != 0 || !res || ((uintptr_t)res & 7u) != 0 ||
        ((uintptr_t)U & 7u) != 0 || n_in < 1 || n_in > AMC_DUAL_MAX_INNER || o->n_paths > INT32_MAX)
        return AMC_EINVAL;
    const double m = o->n_steps;
    if ((double)o->n_paths * (double)n_in * m * (m - 1.0) * 0.5 > (double)AMC_DUAL_MAX_WORK) return AMC_EINVAL;
    DualArgs a;
    memset(&a, 0, sizeof(a));
    Job &J = a.one;
    fill_job_common(o, &J);
    J.S = const_cast<void *>(S);
    J.ld = ld;
    J.coef = const_cast<double *>(coef);
    J.res = res;
    J.status = c->status1;
    AMC_TRY(grow_scratch(&c->dualw, &c->dualw_n, o->n_paths, 3));
    a.n_in = n_in;
    a.seed_in = seed_in;
    a.L1 = c->dualw;
    a.V = c->dualw + o->n_paths;
    a.W = c->dualw + 2 * o->n_paths;
    a.U = U;
    AMC_TRY_CUDA(cudaMemsetAsync(c->status1, 0, sizeof(int32_t), st));
    AMC_TRY_CUDA(launch_dual_upper(a, prec == AMC_FP64, st));
    return AMC_OK;
}

amc_option make_option(double S0, double K, double r, double sigma, double T, int n_steps, int64_t n_paths,
                       int basis, int type, uint64_t seed, int rule) {
    amc_option o;
    memset(&o, 0, sizeof(o));
    o.S0 = S0; o.K = K; o.r = r; o.sigma = sigma; o.T = T;
    o.n_steps = n_steps; o.basis = basis; o.n_paths = n_paths;
    o.type = type; o.rule = rule; o.seed = seed;
    return o;
}

// ------------------------------------------------------------- batches
// A wave: options whose paths fit half the arena and whose sweep CTAs fit
// one co-resident launch; within a wave the options share the group key
// (plan kind, put/call for the mixed LSM kernel, chunk count, rule class).
// Within a group the options are ordered by date count, so a wave's CTAs
// finish together.  Waves alternate between two streams and two halves of
// the arena: the next wave is prepared and launched while the previous one
// is still on the GPU.  Every option keeps its own CTA group and reduction
// order, so its result does not depend on the wave it lands in.
// Host form (out != nullptr): per wave, results copied to pinned memory and
// handed out in input order; blocking.  Device form (dev != nullptr):
// results scattered on the device into the caller's arrays, spot and
// volatility optionally taken from device memory, the waves ordered after
// the work already queued on user_st and user_st after them; no host
// synchronisation.
int run_batch(amc_ctx *c, const amc_option *opts, int n, int prec, bool greeks, amc_result *out,
              const DeviceIO *dev = nullptr, cudaStream_t user_st = nullptr) {
    AMC_TRY(check_prec(prec, !greeks));
    for (int i = 0; i < n; ++i) {
        amc_option o = opts[i];
        if (dev && dev->S0) o.S0 = 1.0;             // checked on the device
        if (dev && dev->sigma) o.sigma = 0.2;
        AMC_TRY(host_validate(&o));
        if (greeks && opts[i].rule == AMC_RULE_PAPER_UB) return AMC_EINVAL;
        if (prec == AMC_MIXED16 && opts[i].rule != AMC_RULE_LSM) return AMC_EINVAL;
    }
    struct Item {
        int idx;
        SweepPlan pl;
        GroupKey key;
    };
    std::vector<Item> items;
    for (int i = 0; i < n; ++i) {
        Item it;
        it.idx = i;
        AMC_TRY(host_plan_sweep(opts[i].n_paths, c->sm_count, prec, opts[i].rule, &it.pl,
                                greeks ? 0 : c->max_cluster));
        it.key = group_key(opts[i], it.pl);
        items.push_back(it);
    }
    std::stable_sort(items.begin(), items.end(), [&](const Item &a, const Item &b) {
        if (a.key.kind != b.key.kind) return a.key.kind < b.key.kind;
        if (a.key.type != b.key.type) return a.key.type < b.key.type;
        if (a.key.chunks != b.key.chunks) return a.key.chunks < b.key.chunks;
        if (a.key.lsm != b.key.lsm) return a.key.lsm && !b.key.lsm;
        if (a.key.cubic != b.key.cubic) return a.key.cubic < b.key.cubic;
        return opts[a.idx].n_steps > opts[b.idx].n_steps;
    });
    if (out)
        for (int i = 0; i < n; ++i) memset(&out[i], 0, sizeof(amc_result));
    if (c->inject_kind == 2) {
        c->inject_kind = 0;
        return AMC_ENOMEM;
    }
    if (dev) {                                                // after the caller's queued work
        AMC_TRY_CUDA(cudaEventRecord(c->bev[0], user_st));
        for (int h = 0; h < 2; ++h) AMC_TRY_CUDA(cudaStreamWaitEvent(c->bstream[h], c->bev[0], 0));
    }
    struct Half {
        cudaStream_t st;
        SubArena ar;
        std::vector<int32_t> widx;
        double *res_host = nullptr;
        bool busy = false;
    };
    Half half[2];
    const size_t hb = c->arena_bytes / 2 / 4096 * 4096;
    for (int h = 0; h < 2; ++h) {
        // with profiling on, the waves run one after another on one stream,
        // so that every launch's measured time is its own
        half[h].st = c->prof.on ? c->bstream[0] : c->bstream[h];
        half[h].ar.base = c->arena + h * hb;
        half[h].ar.size = hb;
    }
    int status = AMC_OK;
    auto finish = [&](Half &H) -> int {
        if (!H.busy) return AMC_OK;
        H.busy = false;
        if (dev) return AMC_OK;                               // stream-ordered: nothing to collect
        if (cudaStreamSynchronize(H.st) != cudaSuccess) return AMC_ECUDA;
        int ws = AMC_OK;
        for (size_t k = 0; k < H.widx.size(); ++k) {
            int s2 = result_from(H.res_host + k * AMC_RES_DOUBLES, &out[H.widx[k]]);
            if (s2 != AMC_OK) ws = s2;
        }
        return ws;
    };
    size_t pos = 0;
    int cur = 0;
    while (pos < items.size() && status == AMC_OK) {
        Half &H = half[cur];
        int rc = finish(H);                                   // this half's previous wave
        if (rc != AMC_OK) { status = rc; break; }
        const GroupKey key = items[pos].key;
        const int cap = group_cta_cap(c, items[pos].pl);
        std::vector<const amc_option *> wopts;
        std::vector<SweepPlan> wplans;
        H.widx.clear();
        size_t bytes = 4096 + (dev ? 256 + sizeof(int32_t) * c->batch_cap : 0);   // + input positions (device form)
        int ctas = 0;
        while (pos < items.size() && items[pos].key == key && (int)wopts.size() < c->batch_cap) {
            const amc_option &o = opts[items[pos].idx];
            const size_t need = option_bytes(o, items[pos].pl, prec);
            if (!wopts.empty() && (bytes + need > H.ar.size || ctas + items[pos].pl.ctas > cap)) break;
            if (bytes + need > H.ar.size) { status = AMC_ENOMEM; break; }
            wopts.push_back(&o);
            wplans.push_back(items[pos].pl);
            H.widx.push_back(items[pos].idx);
            bytes += need;
            ctas += items[pos].pl.ctas;
            ++pos;
        }
        if (status != AMC_OK) break;
        H.ar.top = 0;
        double *res_dev = nullptr;
        DeviceIO wio;
        if (dev) {
            wio = *dev;
            wio.idx = H.widx.data();
        }
        rc = launch_group(c, wopts.data(), wplans.data(), (int)wopts.size(), prec, greeks, H.ar, H.st, &res_dev,
                          dev ? &wio : nullptr);
        if (rc != AMC_OK) { status = rc; break; }
        if (!dev) {
            H.res_host = c->bres_host[cur];
            if (cudaMemcpyAsync(H.res_host, res_dev, sizeof(double) * AMC_RES_DOUBLES * wopts.size(),
                                cudaMemcpyDeviceToHost, H.st) != cudaSuccess) {
                status = AMC_ECUDA;
                break;
            }
        }
        H.busy = true;
        cur ^= 1;
    }
    for (int h = 0; h < 2; ++h) {
        int rc = finish(half[h]);
        if (status == AMC_OK) status = rc;
    }
    if (dev) {
        // the caller's stream after every wave; so is the context's own
        // stream, whose calls reuse the arena (the serving slots wait on
        // the same events when serving starts)
        for (int h = 0; h < 2; ++h) {
            if (cudaEventRecord(c->bev[1 + h], c->bstream[h]) != cudaSuccess ||
                cudaStreamWaitEvent(user_st, c->bev[1 + h], 0) != cudaSuccess ||
                cudaStreamWaitEvent(c->stream, c->bev[1 + h], 0) != cudaSuccess)
                return AMC_ECUDA;
        }
    }
    return status;
}

}  // namespace

namespace amc {

int result_from(const double *r, amc_result *out) {
    memset(out, 0, sizeof(*out));
    out->price = r[0];
    out->std_err = r[1];
    out->delta = r[2];
    out->vega = r[3];
    out->degenerate_dates = (int32_t)r[4];
    out->status = (int32_t)r[5];
    return out->status;
}

cudaEvent_t prof_begin(amc_ctx *c, cudaStream_t st) {
    if (!c->prof.on) return nullptr;
    cudaEvent_t e = nullptr;
    if (!c->prof.pool.empty()) {
        e = c->prof.pool.back();
        c->prof.pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    if (cudaEventRecord(e, st) != cudaSuccess) {
        c->prof.pool.push_back(e);
        return nullptr;
    }
    return e;
}

void prof_end(amc_ctx *c, cudaEvent_t a, int kind, int64_t units, cudaStream_t st) {
    if (!a) return;
    cudaEvent_t b = prof_begin(c, st);
    if (!b) {
        c->prof.pool.push_back(a);
        return;
    }
    c->prof.recs.push_back({a, b, kind, units});
}

GroupKey group_key(const amc_option &o, const SweepPlan &pl) {
    GroupKey k;
    k.kind = pl.kind;
    k.type = pl.kind >= 2 ? o.type : 0;
    k.chunks = pl.kind == 3 ? pl.ctas : pl.chunks;    // one cluster size per cluster launch
    k.lsm = o.rule == AMC_RULE_LSM;
    k.cubic = (pl.kind == 3 && o.basis == 4) ? 1 : 0;
    return k;
}

int group_cta_cap(amc_ctx *c, const SweepPlan &pl) {
    if (pl.kind == 3) return 1 << 30;                 // clusters run independently: no co-residency cap
    return pl.kind == 2 ? std::min(c->sm_count, kV2MaxCtas) : sweep_ctas_per_sm(pl.chunks) * c->sm_count;
}

size_t option_bytes(const amc_option &o, const SweepPlan &pl, int prec) {
    const size_t esz = elem_bytes(prec);
    size_t need = align_up((size_t)o.n_steps * host_ld(o.n_paths) * esz, 256);            // paths
    need += pl.kind == 3 ? 0                                                              // on-chip exchange
            : pl.kind == 2 ? align_up(v2_xch_units(o.n_steps, pl.ctas) * 8, 256)          // exchange units
                           : align_up((size_t)o.n_steps * pl.ctas * kNV * 8, 256);        // partials
    need += 2 * align_up((size_t)o.n_steps * 4, 256);                                      // arrive + shifts
    need += align_up((size_t)pl.ctas * 32, 256) + align_up(sizeof(Job), 256) + 256;       // fin, job, result
    return need;
}

int launch_group(amc_ctx *c, const amc_option *const *opts, const SweepPlan *plans, int nw, int prec, bool greeks,
                 SubArena &ar, cudaStream_t st, double **res_out, const DeviceIO *io) {
    const bool fp64 = prec == AMC_FP64;
    const size_t esz = elem_bytes(prec);
    const SweepPlan plan0 = plans[0];
    const bool lsm = opts[0]->rule == AMC_RULE_LSM;
    std::vector<Job> jobs(nw);
    Job *jobs_dev;
    int32_t *status_dev;
    double *res_dev;
    uint32_t *arrive_all;
    AMC_TRY(ar.alloc(sizeof(Job) * nw, (void **)&jobs_dev));
    AMC_TRY(ar.alloc(sizeof(int32_t), (void **)&status_dev));
    AMC_TRY(ar.alloc(sizeof(double) * AMC_RES_DOUBLES * nw, (void **)&res_dev));
    size_t arrive_words = 0;
    for (int k = 0; k < nw; ++k) arrive_words += opts[k]->n_steps;
    AMC_TRY(ar.alloc(sizeof(uint32_t) * arrive_words, (void **)&arrive_all));
    std::vector<uint32_t> shifts;
    std::vector<size_t> shift_off(nw);
    for (int k = 0; k < nw; ++k) {
        shift_off[k] = shifts.size();
        shifts.resize(shifts.size() + opts[k]->n_steps);
        host_shifts(opts[k]->seed, opts[k]->n_steps, shifts.data() + shift_off[k]);
    }
    uint32_t *shift_dev;
    AMC_TRY(ar.alloc(sizeof(uint32_t) * shifts.size(), (void **)&shift_dev));
    // Exchange units of the mixed LSM sweep: one block for the wave, cleared
    // below on the launch stream.  The arena bytes held earlier requests'
    // paths and partial sums, and a stale word whose high half happened to
    // equal this launch's tag would pass for a posted unit.
    uint64_t *xch_all = nullptr;
    size_t xch_words = 0;
    if (plan0.kind == 2) {
        for (int k = 0; k < nw; ++k) xch_words += v2_xch_units(opts[k]->n_steps, plans[k].ctas);
        AMC_TRY(ar.alloc(sizeof(uint64_t) * xch_words, (void **)&xch_all));
    }
    int64_t tiles = 0;
    int cta = 0, max_slots = 1, max_m = 1;
    size_t arr_off = 0, xch_off = 0;
    for (int k = 0; k < nw; ++k) {
        const amc_option &o = *opts[k];
        Job &J = jobs[k];
        fill_job_common(&o, &J);
        DevBridge *b;
        AMC_TRY(get_bridge(c, o.n_steps, &b));
        J.shift = shift_dev + shift_off[k];
        J.nodes = fp64 ? (const void *)b->nd : (const void *)b->nf;
        J.nslots = b->nslots;
        max_slots = std::max(max_slots, b->nslots);
        max_m = std::max(max_m, o.n_steps);
        J.ld = host_ld(o.n_paths);
        AMC_TRY(ar.alloc((size_t)o.n_steps * J.ld * esz, &J.S));
        J.tile_begin = tiles;
        J.n_tiles = (o.n_paths + kTilePoints - 1) / kTilePoints;
        tiles += J.n_tiles;
        J.cta_begin = cta;
        J.n_cta = plans[k].ctas;
        J.chunks = plan0.chunks;
        cta += J.n_cta;
        J.greeks = greeks ? 1 : 0;
        if (plan0.kind == 2) {
            J.xch = xch_all + xch_off;
            xch_off += v2_xch_units(o.n_steps, J.n_cta);
        } else if (plan0.kind == 1) {
            AMC_TRY(ar.alloc((size_t)o.n_steps * J.n_cta * kNV * 8, &J.part));
        }
        J.arrive = arrive_all + arr_off;
        arr_off += o.n_steps;
        AMC_TRY(ar.alloc((size_t)J.n_cta * 4 * sizeof(double), &J.fin));
        J.res = res_dev + (size_t)k * AMC_RES_DOUBLES;
        J.status = status_dev;
    }
    AMC_TRY_CUDA(cudaMemcpyAsync(shift_dev, shifts.data(), sizeof(uint32_t) * shifts.size(), cudaMemcpyHostToDevice,
                                 st));
    AMC_TRY_CUDA(cudaMemcpyAsync(jobs_dev, jobs.data(), sizeof(Job) * nw, cudaMemcpyHostToDevice, st));
    int32_t *idx_dev = nullptr;
    if (io) {
        AMC_TRY(ar.alloc(sizeof(int32_t) * nw, (void **)&idx_dev));
        AMC_TRY_CUDA(cudaMemcpyAsync(idx_dev, io->idx, sizeof(int32_t) * nw, cudaMemcpyHostToDevice, st));
        AMC_TRY_CUDA(launch_patch_inputs(jobs_dev, nw, idx_dev, io->S0, io->sigma, st));
    }
    AMC_TRY_CUDA(cudaMemsetAsync(arrive_all, 0, sizeof(uint32_t) * arrive_words, st));
    AMC_TRY_CUDA(cudaMemsetAsync(status_dev, 0, sizeof(int32_t), st));
    if (xch_words) AMC_TRY_CUDA(cudaMemsetAsync(xch_all, 0, sizeof(uint64_t) * xch_words, st));
    KArgs a;
    memset(&a, 0, sizeof(KArgs));
    a.jobs = jobs_dev;
    a.n_jobs = nw;
    a.max_m = max_m;
    a.max_slots = max_slots;
    a.jobs_type = opts[0]->type;
    a.jobs_p = opts[0]->basis;
    a.total = tiles;
    a.V = c->V;
    a.h16 = prec == AMC_MIXED16 ? 1 : 0;
    if (a.h16 && plan0.kind < 2) return AMC_EINVAL;
    int64_t units = 0;
    for (int k = 0; k < nw; ++k) units += opts[k]->n_paths * (int64_t)opts[k]->n_steps;
    cudaEvent_t pe = prof_begin(c, st);
    AMC_TRY_CUDA(launch_pathgen(a, fp64, c->sm_count, st));
    prof_end(c, pe, 0, units, st);
    AMC_TRY(launch_sweeps(c, a, plan0, cta, lsm, fp64, greeks, st, true, units));
    if (io) AMC_TRY_CUDA(launch_scatter_results(res_dev, nw, idx_dev, io->res, io->price, io->delta, io->vega, st));
    *res_out = res_dev;
    return AMC_OK;
}

}  // namespace amc

// =================================================================== C ABI
extern "C" {

const char *amc_strerror(int code) {
    switch (code) {
        case AMC_OK: return "ok";
        case AMC_EINVAL: return "invalid argument";
        case AMC_ENOMEM: return "out of arena or device memory";
        case AMC_ECUDA: return "CUDA runtime error";
        case AMC_ETIMEOUT: return "device wait timed out";
        case AMC_EBUSY: return "admission refused";
        case AMC_PENDING: return "pending";
        case AMC_ENOTFOUND: return "unknown ticket";
        case AMC_ECANCELED: return "request cancelled";
        default: return "unknown error";
    }
}

int amc_version(void) { return 1; }

int amc_validate_option(const amc_option *opt) { return host_validate(opt); }
int64_t amc_path_ld(int64_t n_paths) { return n_paths < 1 ? 0 : host_ld(n_paths); }
size_t amc_path_bytes(int n_steps, int64_t n_paths, int prec) {
    if (n_steps < 1 || n_paths < 1) return 0;
    return (size_t)n_steps * host_ld(n_paths) * elem_bytes(prec);
}
int amc_digital_shifts(uint64_t seed, int n_dims, uint32_t *out) {
    if (n_dims < 0 || (n_dims > 0 && !out)) return AMC_EINVAL;
    host_shifts(seed, n_dims, out);
    return AMC_OK;
}
int amc_sobol_directions(int n_dims, uint32_t *out) {
    if (!out) return AMC_EINVAL;
    return host_directions(n_dims, out);
}
int amc_bridge_schedule(int n_steps, int32_t *date, int32_t *left, int32_t *right) {
    if (!date || !left || !right) return AMC_EINVAL;
    return host_bridge_bfs(n_steps, date, left, right);
}
int amc_bridge_plan(int n_steps, int32_t *coord, int32_t *date, int32_t *sl, int32_t *sr, int32_t *so, double *wl,
                    double *wr, double *sdu, int32_t *n_slots) {
    if (!coord || !date || !sl || !sr || !so || !wl || !wr || !sdu || !n_slots) return AMC_EINVAL;
    if (n_steps < 1 || n_steps > AMC_MAX_STEPS) return AMC_EINVAL;
    BridgePlan plan;
    AMC_TRY(host_bridge_plan(n_steps, &plan));
    for (int k = 0; k < n_steps; ++k) {
        const NodeD &n = plan.nd[k];
        coord[k] = n.coord;
        date[k] = n.date;
        sl[k] = n.sl;
        sr[k] = n.sr;
        so[k] = n.so;
        wl[k] = n.wl;
        wr[k] = n.wr;
        sdu[k] = n.sdu;
    }
    *n_slots = plan.nslots;
    return AMC_OK;
}
int amc_plan_sweep(int64_t n_paths, int sm_count, int prec, int rule, int32_t *ctas, int32_t *paths_per_thread) {
    SweepPlan p;
    int rc = host_plan_sweep(n_paths, sm_count, prec, rule, &p);
    if (rc != AMC_OK) return rc;
    if (ctas) *ctas = p.ctas;
    if (paths_per_thread) *paths_per_thread = p.kind == 3 ? kClPPT : (p.kind == 2 ? kV2PPT : 4 * p.chunks);
    return AMC_OK;
}

int amc_ctx_create(int device, size_t arena_bytes, amc_ctx **out) {
    if (!out) return AMC_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return AMC_ECUDA;
    AMC_TRY_CUDA(cudaSetDevice(device));
    amc_ctx *c = new amc_ctx();
    c->device = device;
    int rc = AMC_OK;
    do {
        if (const char *e = getenv("AMC_POLL_NS")) c->poll_ns = (uint32_t)strtoul(e, nullptr, 10);
        if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            rc = AMC_ECUDA;
            break;
        }
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c->bstream[0], cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c->bstream[1], cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&c->bres_host[0], sizeof(double) * AMC_RES_DOUBLES * c->batch_cap) != cudaSuccess ||
            cudaMallocHost(&c->bres_host[1], sizeof(double) * AMC_RES_DOUBLES * c->batch_cap) != cudaSuccess) {
            rc = AMC_ECUDA;
            break;
        }
        std::vector<uint32_t> V((size_t)AMC_MAX_STEPS * 32);
        if (host_directions(AMC_MAX_STEPS, V.data()) != AMC_OK) { rc = AMC_EINVAL; break; }
        if (cudaMalloc(&c->V, V.size() * 4) != cudaSuccess ||
            cudaMemcpy(c->V, V.data(), V.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = AMC_ECUDA;
            break;
        }
        c->gcap = 4 * c->sm_count;
        if (sweep_cl_max_cluster(&c->max_cluster) != cudaSuccess) c->max_cluster = 0;
        cudaGetLastError();
        size_t part_bytes = (size_t)AMC_MAX_STEPS * c->gcap * kNV * 8;
        if (cudaMalloc(&c->shift1, 4 * AMC_MAX_STEPS) != cudaSuccess ||
            cudaMalloc(&c->part1, part_bytes) != cudaSuccess ||
            cudaMalloc(&c->arrive1, 4 * AMC_MAX_STEPS) != cudaSuccess ||
            cudaMalloc(&c->fin1, sizeof(double) * 4 * c->gcap) != cudaSuccess ||
            cudaMalloc(&c->res1, sizeof(double) * AMC_RES_DOUBLES) != cudaSuccess ||
            cudaMalloc(&c->status1, sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&c->xch1, sizeof(uint64_t) * v2_xch_units(AMC_MAX_STEPS, kV2MaxCtas)) != cudaSuccess ||
            cudaMemset(c->xch1, 0, sizeof(uint64_t) * v2_xch_units(AMC_MAX_STEPS, kV2MaxCtas)) != cudaSuccess ||
            cudaMallocHost(&c->res_host, sizeof(double) * AMC_RES_DOUBLES) != cudaSuccess) {
            rc = AMC_ENOMEM;
            break;
        }
        for (int k = 0; k < 3; ++k)
            if (cudaEventCreate(&c->ev[k]) != cudaSuccess ||
                cudaEventCreateWithFlags(&c->bev[k], cudaEventDisableTiming) != cudaSuccess)
                rc = AMC_ECUDA;
        if (rc != AMC_OK) break;
        if (arena_bytes == 0) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { rc = AMC_ECUDA; break; }
            arena_bytes = (size_t)(fr * 0.6) / 4096 * 4096;
        }
        if (cudaMalloc(&c->arena, arena_bytes) != cudaSuccess) { rc = AMC_ENOMEM; break; }
        if (cudaMemset(c->arena, 0, arena_bytes) != cudaSuccess) { rc = AMC_ECUDA; break; }
        c->arena_bytes = arena_bytes;
    } while (0);
    if (rc != AMC_OK) {
        amc_ctx_destroy(c);
        return rc;
    }
    *out = c;
    return AMC_OK;
}

int amc_ctx_destroy(amc_ctx *c) {
    if (!c) return AMC_EINVAL;
    if (c->server) amc_serve_stop(c);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &kv : c->bridges) {
        cudaFree(kv.second.nf);
        cudaFree(kv.second.nd);
    }
    cudaFree(c->V);
    cudaFree(c->shift1);
    cudaFree(c->part1);
    cudaFree(c->arrive1);
    cudaFree(c->fin1);
    cudaFree(c->finv);
    cudaFree(c->dualw);
    cudaFree(c->streamw);
    cudaFree(c->res1);
    cudaFree(c->status1);
    cudaFree(c->xch1);
    cudaFree(c->arena);
    if (c->res_host) cudaFreeHost(c->res_host);
    for (int k = 0; k < 3; ++k) {
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
        if (c->bev[k]) cudaEventDestroy(c->bev[k]);
    }
    for (auto &r : c->prof.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    for (int h = 0; h < 2; ++h) {
        if (c->bstream[h]) cudaStreamDestroy(c->bstream[h]);
        if (c->bres_host[h]) cudaFreeHost(c->bres_host[h]);
    }
    delete c;
    return AMC_OK;
}

int amc_ctx_set_timeout(amc_ctx *c, double seconds) {
    if (!c || !(seconds > 0.0) || seconds > 3600.0) return AMC_EINVAL;
    c->timeout_s = seconds;
    return AMC_OK;
}

int amc_ctx_inject(amc_ctx *c, int kind, int64_t arg) {
    if (!c || kind < 0 || kind > 4) return AMC_EINVAL;
    if (kind == 4 && (arg < 1 || arg >= (int64_t)(1u << kEpochBits))) return AMC_EINVAL;
    c->inject_kind = kind;
    c->inject_arg = arg;
    return AMC_OK;
}

int amc_ctx_set_profiling(amc_ctx *c, int enable) {
    if (!c) return AMC_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    c->prof.on = enable != 0;
    return AMC_OK;
}

int amc_ctx_profile(amc_ctx *c, double *gen_ms, double *sweep_ms, int64_t *gen_launches, int64_t *sweep_launches,
                    int64_t *gen_units, int64_t *sweep_units) {
    if (!c) return AMC_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    if (cudaSetDevice(c->device) != cudaSuccess) return AMC_ECUDA;
    double ms[2] = {0.0, 0.0};
    int64_t n[2] = {0, 0}, u[2] = {0, 0};
    int rc = AMC_OK;
    for (auto &r : c->prof.recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            rc = AMC_ECUDA;
        ms[r.kind] += t;
        n[r.kind] += 1;
        u[r.kind] += r.units;
        c->prof.pool.push_back(r.a);
        c->prof.pool.push_back(r.b);
    }
    c->prof.recs.clear();
    if (gen_ms) *gen_ms = ms[0];
    if (sweep_ms) *sweep_ms = ms[1];
    if (gen_launches) *gen_launches = n[0];
    if (sweep_launches) *sweep_launches = n[1];
    if (gen_units) *gen_units = u[0];
    if (sweep_units) *sweep_units = u[1];
    return rc;
}

int amc_ctx_memory(amc_ctx *c, size_t *free_bytes, size_t *total_bytes) {
    if (!c) return AMC_EINVAL;
    if (free_bytes) *free_bytes = c->arena_bytes - c->arena_top;
    if (total_bytes) *total_bytes = c->arena_bytes;
    return AMC_OK;
}

int amc_sobol(amc_ctx *c, int n_dims, int64_t n_points, uint64_t seed, uint32_t *x_dev, int64_t ld, void *stream) {
    if (c && c->server) return AMC_EBUSY;
    if (!c || !x_dev || n_dims < 1 || n_dims > AMC_MAX_STEPS || n_points < 0 || n_points > AMC_MAX_PATHS ||
        ld < n_points)
        return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<uint32_t> sh(n_dims);
    host_shifts(seed, n_dims, sh.data());
    AMC_TRY_CUDA(cudaMemcpyAsync(c->shift1, sh.data(), 4 * n_dims, cudaMemcpyHostToDevice, st));
    return cuda_rc(launch_sobol(c->V, n_dims, n_points, c->shift1, x_dev, ld, st));
}

int amc_generate_paths(amc_ctx *c, const amc_option *opt, int prec, void *S_dev, int64_t ld, void *stream) {
    TraceRange trace_range("amc_generate_paths");
    if (c && c->server) return AMC_EBUSY;
    if (!c) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_generate(c, opt, prec, S_dev, ld, (cudaStream_t)stream);
}

int amc_generate_paths_permuted(amc_ctx *c, const amc_option *opt, int prec, void *S_dev, int64_t ld, void *stream) {
    if (c && c->server) return AMC_EBUSY;
    if (!c || !opt) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_generate_permuted(c, opt, prec, S_dev, ld, (cudaStream_t)stream);
}

int amc_lcg_params(uint64_t seed, int n_dims, int64_t n_points, uint32_t *a, uint32_t *c, uint64_t *M) {
    if (n_dims < 1 || n_dims > AMC_MAX_STEPS || n_points < 1 || n_points > AMC_MAX_PATHS || !a || !c || !M)
        return AMC_EINVAL;
    host_lcg_params(seed, n_dims, n_points, a, c, M);
    return AMC_OK;
}

int amc_sweep(amc_ctx *c, const amc_option *opt, int prec, const void *S_dev, int64_t ld, int with_greeks,
              double *res_dev, void *stream) {
    TraceRange trace_range("amc_sweep");
    if (c && c->server) return AMC_EBUSY;
    if (!c) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_sweep(c, opt, prec, S_dev, ld, with_greeks != 0, res_dev, (cudaStream_t)stream);
}

int amc_price_device(amc_ctx *c, const amc_option *opt, int prec, void *S_dev, int64_t ld, double *res_dev,
                     void *stream) {
    TraceRange trace_range("amc_price_device");
    if (c && c->server) return AMC_EBUSY;
    if (!c) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    AMC_TRY(do_generate(c, opt, prec, S_dev, ld, (cudaStream_t)stream));
    return do_sweep(c, opt, prec, S_dev, ld, false, res_dev, (cudaStream_t)stream);
}

int amc_fit_boundary(amc_ctx *c, const amc_option *opt, int prec, const void *S_dev, int64_t ld, double *coef_dev,
                     double *res_dev, void *stream) {
    TraceRange trace_range("amc_fit_boundary");
    if (c && c->server) return AMC_EBUSY;
    if (!c || !opt || opt->rule != AMC_RULE_LSM || !coef_dev || ((uintptr_t)coef_dev & 7u) != 0) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_sweep(c, opt, prec, S_dev, ld, false, res_dev, (cudaStream_t)stream, coef_dev);
}

int amc_value_boundary(amc_ctx *c, const amc_option *opt, int prec, const void *S_dev, int64_t ld,
                       const double *coef_dev, double *res_dev, void *stream) {
    TraceRange trace_range("amc_value_boundary");
    if (c && c->server) return AMC_EBUSY;
    if (!c || !opt) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_value(c, opt, prec, S_dev, ld, coef_dev, res_dev, (cudaStream_t)stream);
}

int amc_price_oos(amc_ctx *c, const amc_option *opt, uint64_t value_seed, int prec, amc_result *fit,
                  amc_result *value) {
    TraceRange trace_range("amc_price_oos");
    if (c && c->server) return AMC_EBUSY;
    if (!c || !opt || !value || opt->rule != AMC_RULE_LSM) return AMC_EINVAL;
    AMC_TRY(host_validate(opt));
    AMC_TRY(check_prec(prec));
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    c->arena_top = 0;
    const int64_t ld = host_ld(opt->n_paths);
    void *S;
    double *coef, *res2;
    AMC_TRY(arena_alloc(c, (size_t)opt->n_steps * ld * (prec == AMC_FP64 ? 8 : 4), &S));
    AMC_TRY(arena_alloc(c, sizeof(double) * kCoefStride * opt->n_steps, (void **)&coef));
    AMC_TRY(arena_alloc(c, sizeof(double) * 2 * AMC_RES_DOUBLES, (void **)&res2));
    cudaStream_t st = c->stream;
    amc_option ov = *opt;
    ov.seed = value_seed;
    AMC_TRY(do_generate(c, opt, prec, S, ld, st));
    AMC_TRY(do_sweep(c, opt, prec, S, ld, false, res2, st, coef));
    AMC_TRY(do_generate(c, &ov, prec, S, ld, st));
    AMC_TRY(do_value(c, &ov, prec, S, ld, coef, res2 + AMC_RES_DOUBLES, st));
    double h[2 * AMC_RES_DOUBLES];
    AMC_TRY_CUDA(cudaMemcpyAsync(h, res2, sizeof(h), cudaMemcpyDeviceToHost, st));
    AMC_TRY_CUDA(cudaStreamSynchronize(st));
    int s1 = AMC_OK;
    if (fit) s1 = result_from(h, fit);
    else if ((int32_t)h[5] != 0) s1 = (int32_t)h[5];
    int s2 = result_from(h + AMC_RES_DOUBLES, value);
    return s1 != AMC_OK ? s1 : s2;
}

int amc_price_fused(amc_ctx *c, const amc_option *opt, int prec, const double *coef_dev, double *res_dev,
                    void *stream) {
    TraceRange trace_range("amc_price_fused");
    if (c && c->server) return AMC_EBUSY;
    if (!c || !opt) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_fused(c, opt, prec, coef_dev, res_dev, (cudaStream_t)stream);
}

int amc_dual_upper(amc_ctx *c, const amc_option *opt, int prec, const void *S_dev, int64_t ld, const double *coef_dev,
                   int64_t n_inner, uint64_t inner_seed, double *res_dev, double *U_dev, void *stream) {
    TraceRange trace_range("amc_dual_upper");
    if (c && c->server) return AMC_EBUSY;
    if (!c || !opt) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_dual(c, opt, prec, S_dev, ld, coef_dev, n_inner, inner_seed, res_dev, U_dev, (cudaStream_t)stream);
}

int amc_price_dual(amc_ctx *c, const amc_option *opt, uint64_t outer_seed, int64_t n_outer, int64_t n_inner,
                   uint64_t inner_seed, int prec, amc_result *fit, amc_result *lower, amc_result *upper) {
    TraceRange trace_range("amc_price_dual");
    if (c && c->server) return AMC_EBUSY;
    if (!c || !opt || !upper || opt->rule != AMC_RULE_LSM) return AMC_EINVAL;
    amc_option ov = *opt;
    ov.seed = outer_seed;
    ov.n_paths = n_outer;
    AMC_TRY(host_validate(opt));
    AMC_TRY(host_validate(&ov));
    AMC_TRY(check_prec(prec));
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    c->arena_top = 0;
    const size_t es = prec == AMC_FP64 ? 8 : 4;
    const int64_t ld = host_ld(opt->n_paths), ldo = host_ld(n_outer);
    const size_t bytes = (size_t)opt->n_steps * es * (size_t)(ld > ldo ? ld : ldo);
    void *S;
    double *coef, *res3;
    AMC_TRY(arena_alloc(c, bytes, &S));               // fitting paths, then (stream-ordered) the outer paths
    AMC_TRY(arena_alloc(c, sizeof(double) * kCoefStride * opt->n_steps, (void **)&coef));
    AMC_TRY(arena_alloc(c, sizeof(double) * 3 * AMC_RES_DOUBLES, (void **)&res3));
    cudaStream_t st = c->stream;
    AMC_TRY(do_generate(c, opt, prec, S, ld, st));
    AMC_TRY(do_sweep(c, opt, prec, S, ld, false, res3, st, coef));
    AMC_TRY(do_generate(c, &ov, prec, S, ldo, st));
    AMC_TRY(do_value(c, &ov, prec, S, ldo, coef, res3 + AMC_RES_DOUBLES, st));
    AMC_TRY(do_dual(c, &ov, prec, S, ldo, coef, n_inner, inner_seed, res3 + 2 * AMC_RES_DOUBLES, nullptr, st));
    double h[3 * AMC_RES_DOUBLES];
    AMC_TRY_CUDA(cudaMemcpyAsync(h, res3, sizeof(h), cudaMemcpyDeviceToHost, st));
    AMC_TRY_CUDA(cudaStreamSynchronize(st));
    amc_result tmp;
    const int s1 = result_from(h, fit ? fit : &tmp);
    const int s2 = result_from(h + AMC_RES_DOUBLES, lower ? lower : &tmp);
    const int s3 = result_from(h + 2 * AMC_RES_DOUBLES, upper);
    return s1 != AMC_OK ? s1 : (s2 != AMC_OK ? s2 : s3);
}

int amc_price_american(amc_ctx *c, double S0, double K, double r, double sigma, double T, int n_steps,
                       int64_t n_paths, int basis, int type, uint64_t seed, int rule, int prec, amc_result *out) {
    TraceRange trace_range("amc_price_american");
    if (c && c->server) return AMC_EBUSY;
    if (!c || !out) return AMC_EINVAL;
    amc_option o = make_option(S0, K, r, sigma, T, n_steps, n_paths, basis, type, seed, rule);
    AMC_TRY(host_validate(&o));
    AMC_TRY(check_prec(prec, rule == AMC_RULE_LSM));
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    c->arena_top = 0;
    const int64_t ld = host_ld(n_paths);
    void *S;
    AMC_TRY(arena_alloc(c, (size_t)n_steps * ld * elem_bytes(prec), &S));
    cudaStream_t st = c->stream;
    AMC_TRY_CUDA(cudaEventRecord(c->ev[0], st));
    AMC_TRY(do_generate(c, &o, prec, S, ld, st));
    AMC_TRY_CUDA(cudaEventRecord(c->ev[1], st));
    AMC_TRY(do_sweep(c, &o, prec, S, ld, false, c->res1, st));
    AMC_TRY_CUDA(cudaEventRecord(c->ev[2], st));
    AMC_TRY_CUDA(cudaMemcpyAsync(c->res_host, c->res1, sizeof(double) * AMC_RES_DOUBLES, cudaMemcpyDeviceToHost, st));
    AMC_TRY_CUDA(cudaStreamSynchronize(st));
    int s = result_from(c->res_host, out);
    cudaEventElapsedTime(&out->ms_gen, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&out->ms_sweep, c->ev[1], c->ev[2]);
    return s;
}

int amc_price_batch(amc_ctx *c, const amc_option *opts, int n, int prec, amc_result *out) {
    TraceRange trace_range("amc_price_batch");
    if (c && c->server) return AMC_EBUSY;
    if (!c || n < 0 || (n > 0 && (!opts || !out))) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return run_batch(c, opts, n, prec, false, out);
}

int amc_price_batch_device(amc_ctx *c, const amc_option *opts, int n, int prec, double *res_dev, void *stream) {
    TraceRange trace_range("amc_price_batch_device");
    if (c && c->server) return AMC_EBUSY;
    if (!c || n < 0 || (n > 0 && (!opts || !res_dev)) || ((uintptr_t)res_dev & 7u) != 0) return AMC_EINVAL;
    if (n == 0) return AMC_OK;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    DeviceIO io;
    io.res = res_dev;
    return run_batch(c, opts, n, prec, false, nullptr, &io, (cudaStream_t)stream);
}

int amc_greeks_device(amc_ctx *c, const amc_option *opts, int n, int prec, const double *S0_dev,
                      const double *sigma_dev, double *price_dev, double *delta_dev, double *vega_dev, double *res_dev,
                      void *stream) {
    TraceRange trace_range("amc_greeks_device");
    if (c && c->server) return AMC_EBUSY;
    if (!c || n < 0) return AMC_EINVAL;
    const void *ptrs[] = {S0_dev, sigma_dev, price_dev, delta_dev, vega_dev, res_dev};
    for (const void *q : ptrs)
        if (((uintptr_t)q & 7u) != 0) return AMC_EINVAL;
    if (n > 0 && (!opts || !price_dev || !delta_dev || !vega_dev)) return AMC_EINVAL;
    if (n == 0) return AMC_OK;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    DeviceIO io;
    io.S0 = S0_dev;
    io.sigma = sigma_dev;
    io.res = res_dev;
    io.price = price_dev;
    io.delta = delta_dev;
    io.vega = vega_dev;
    return run_batch(c, opts, n, prec, true, nullptr, &io, (cudaStream_t)stream);
}

int amc_greeks(amc_ctx *c, const amc_option *opts, int n, int prec, double *price, double *delta, double *vega) {
    TraceRange trace_range("amc_greeks");
    if (c && c->server) return AMC_EBUSY;
    if (!c || n < 0 || (n > 0 && (!opts || !price || !delta || !vega))) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    std::vector<amc_result> res(n);
    int rc = run_batch(c, opts, n, prec, true, res.data());
    for (int i = 0; i < n; ++i) {
        price[i] = res[i].price;
        delta[i] = res[i].delta;
        vega[i] = res[i].vega;
    }
    return rc;
}

}  // extern "C"
