// C ABI runtime of the amc library: contexts, the device arena, option
// validation, job packing and the launch sequence of the hot path
// (path generation -> sweep -> finalize).  Everything that computes runs in
// the kernels of pathgen.cu and sweep.cu; this file only plans and launches.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace amc;

namespace {

struct DevBridge {
    NodeF *nf = nullptr;
    NodeD *nd = nullptr;
    int nslots = 0;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct amc_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    // path arena (bump allocation, reset by each host-level call)
    char *arena = nullptr;
    size_t arena_bytes = 0, arena_top = 0;
    // tables
    uint32_t *V = nullptr;                      // [AMC_MAX_STEPS][32]
    std::unordered_map<int, DevBridge> bridges;  // by n_steps
    // single-option scratch (step-level calls); the job itself travels by
    // value in the kernel arguments
    KArgs args;
    uint32_t *shift1 = nullptr;
    void *part1 = nullptr;
    uint32_t *arrive1 = nullptr;
    double *fin1 = nullptr;
    double *res1 = nullptr;
    int32_t *status1 = nullptr;
    uint64_t *xch1 = nullptr;                   // exchange units of the mixed LSM sweep
    uint32_t epoch = 0;                         // launch tag of those units
    int gcap = 0;
    double *res_host = nullptr;                 // pinned
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    double timeout_s = 2.0;
    int inject_kind = 0;
    int64_t inject_arg = 0;
    std::mutex mu;
};

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

// Next launch tag of the mixed LSM sweep's exchange units.  Tags never
// repeat within 2^22 launches; when the counter wraps, every buffer that
// can hold units (the context scratch and the arena) is cleared first.
uint32_t next_epoch(amc_ctx *c) {
    c->epoch = (c->epoch + 1) & ((1u << kEpochBits) - 1u);
    if (c->epoch == 0) {
        cudaDeviceSynchronize();
        cudaMemset(c->xch1, 0, sizeof(uint64_t) * v2_xch_units(AMC_MAX_STEPS, kV2MaxCtas));
        cudaMemset(c->arena, 0, c->arena_bytes);
        c->epoch = 1;
    }
    return c->epoch;
}

// Launch the sweep of the packed jobs in `a` (same precision, same plan
// kind and chunk count, same rule class) and their finalize.
int launch_sweeps(amc_ctx *c, KArgs &a, const SweepPlan &pl, int total_ctas, bool lsm, bool fp64, bool greeks,
                  cudaStream_t st) {
    a.timeout_ns = timeout_ns(c);
    cudaError_t e;
    if (pl.kind == 2) {
        a.epoch = next_epoch(c);
        e = launch_sweep_lsm_v2(a, total_ctas, greeks, st);
    } else if (lsm) {
        e = launch_sweep_lsm(a, total_ctas, pl.chunks, fp64, greeks, st);
    } else {
        e = launch_sweep_pathwise(a, total_ctas, pl.chunks, fp64, greeks, st);
    }
    AMC_TRY_CUDA(e);
    AMC_TRY_CUDA(launch_finalize(a, st));
    return AMC_OK;
}

int check_prec(int prec) { return (prec == AMC_FP64 || prec == AMC_MIXED) ? AMC_OK : AMC_EINVAL; }

// Caller path storage: rows must start on 16-byte boundaries for the
// vector loads and stores, so S must be 16-byte aligned and ld a multiple
// of 32 elements (amc_path_ld rounds to that).
int check_storage(const void *S, int64_t ld, int64_t n_paths) {
    if (!S || ld < host_ld(n_paths) || ld % 32 != 0 || ((uintptr_t)S & 15u) != 0) return AMC_EINVAL;
    return AMC_OK;
}

int do_generate(amc_ctx *c, const amc_option *o, int prec, void *S, int64_t ld, cudaStream_t st) {
    AMC_TRY(host_validate(o));
    AMC_TRY(check_prec(prec));
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
    AMC_TRY_CUDA(launch_pathgen(a, prec == AMC_FP64, c->sm_count, st));
    return AMC_OK;
}

int do_sweep(amc_ctx *c, const amc_option *o, int prec, const void *S, int64_t ld, bool greeks, double *res,
             cudaStream_t st) {
    AMC_TRY(host_validate(o));
    AMC_TRY(check_prec(prec));
    AMC_TRY(check_storage(S, ld, o->n_paths));
    if (!res || ((uintptr_t)res & 7u) != 0) return AMC_EINVAL;
    if (greeks && o->rule == AMC_RULE_PAPER_UB) return AMC_EINVAL;
    SweepPlan pl;
    AMC_TRY(host_plan_sweep(o->n_paths, c->sm_count, prec, o->rule, &pl));
    if (pl.ctas > c->gcap) return AMC_EINVAL;
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
    J.res = res;
    J.status = c->status1;
    J.xch = c->xch1;
    if (c->inject_kind == 1) {
        J.inject_date = (int32_t)c->inject_arg;
        c->inject_kind = 0;
    }
    a.jobs = nullptr;
    a.n_jobs = 1;
    a.max_m = o->n_steps;
    a.V = c->V;
    if (pl.kind == 1 && o->rule == AMC_RULE_LSM)
        AMC_TRY_CUDA(cudaMemsetAsync(c->arrive1, 0, sizeof(uint32_t) * o->n_steps, st));
    AMC_TRY_CUDA(cudaMemsetAsync(c->status1, 0, sizeof(int32_t), st));
    return launch_sweeps(c, a, pl, pl.ctas, o->rule == AMC_RULE_LSM, prec == AMC_FP64, greeks, st);
}

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
// A wave: options whose paths fit the arena and whose sweep CTAs fit one
// co-resident launch; within a wave the options share the chunk count, the
// rule class and the precision.
int run_batch(amc_ctx *c, const amc_option *opts, int n, int prec, bool greeks, amc_result *out) {
    AMC_TRY(check_prec(prec));
    for (int i = 0; i < n; ++i) {
        AMC_TRY(host_validate(&opts[i]));
        if (greeks && opts[i].rule == AMC_RULE_PAPER_UB) return AMC_EINVAL;
    }
    const bool fp64 = prec == AMC_FP64;
    const size_t esz = fp64 ? 8 : 4;
    struct Item {
        int idx;
        SweepPlan pl;
        bool lsm;
    };
    std::vector<Item> items;
    for (int i = 0; i < n; ++i) {
        Item it;
        it.idx = i;
        AMC_TRY(host_plan_sweep(opts[i].n_paths, c->sm_count, prec, opts[i].rule, &it.pl));
        it.lsm = opts[i].rule == AMC_RULE_LSM;
        items.push_back(it);
    }
    // group by (plan kind, chunks, rule class), keeping input order within a group
    // (the mixed LSM kernel is also specialised on put / call)
    auto tkey = [&](const Item &it) { return it.pl.kind == 2 ? opts[it.idx].type : 0; };
    std::stable_sort(items.begin(), items.end(), [&](const Item &a, const Item &b) {
        if (a.pl.kind != b.pl.kind) return a.pl.kind < b.pl.kind;
        if (tkey(a) != tkey(b)) return tkey(a) < tkey(b);
        if (a.pl.chunks != b.pl.chunks) return a.pl.chunks < b.pl.chunks;
        return a.lsm && !b.lsm;
    });
    for (int i = 0; i < n; ++i) memset(&out[i], 0, sizeof(amc_result));
    size_t pos = 0;
    cudaStream_t st = c->stream;
    while (pos < items.size()) {
        const SweepPlan plan0 = items[pos].pl;
        const int chunks = plan0.chunks;
        const bool lsm = items[pos].lsm;
        const int cap = plan0.kind == 2 ? std::min(c->sm_count, kV2MaxCtas)
                                        : sweep_ctas_per_sm(chunks) * c->sm_count;
        c->arena_top = 0;
        // per-wave fixed scratch sized for the worst case of this wave
        std::vector<Item> wave;
        size_t bytes = 0;
        int ctas = 0, max_m = 1;
        size_t budget = c->arena_bytes;
        const int type0 = tkey(items[pos]);
        while (pos < items.size() && items[pos].pl.kind == plan0.kind && items[pos].pl.chunks == chunks &&
               items[pos].lsm == lsm && tkey(items[pos]) == type0) {
            const amc_option &o = opts[items[pos].idx];
            size_t need = align_up((size_t)o.n_steps * host_ld(o.n_paths) * esz, 256);
            need += align_up((size_t)o.n_steps * items[pos].pl.ctas * kNV * 8, 256);   // partials
            need += align_up(v2_xch_units(o.n_steps, items[pos].pl.ctas) * 8, 256);    // exchange units
            need += align_up((size_t)o.n_steps * 4, 256) * 2;                          // arrive + shifts
            need += align_up((size_t)items[pos].pl.ctas * 32, 256) + 256 + sizeof(Job) + 256;
            if (!wave.empty() && (bytes + need > budget || ctas + items[pos].pl.ctas > cap)) break;
            if (need > budget) return AMC_ENOMEM;
            wave.push_back(items[pos]);
            bytes += need;
            ctas += items[pos].pl.ctas;
            max_m = std::max(max_m, o.n_steps);
            ++pos;
        }
        const int nw = (int)wave.size();
        std::vector<Job> jobs(nw);
        Job *jobs_dev;
        int32_t *status_dev;
        double *res_dev;
        uint32_t *arrive_all;
        AMC_TRY(arena_alloc(c, sizeof(Job) * nw, (void **)&jobs_dev));
        AMC_TRY(arena_alloc(c, sizeof(int32_t), (void **)&status_dev));
        AMC_TRY(arena_alloc(c, sizeof(double) * AMC_RES_DOUBLES * nw, (void **)&res_dev));
        size_t arrive_words = 0;
        for (auto &it : wave) arrive_words += opts[it.idx].n_steps;
        AMC_TRY(arena_alloc(c, sizeof(uint32_t) * arrive_words, (void **)&arrive_all));
        std::vector<uint32_t> shifts;
        std::vector<size_t> shift_off(nw);
        for (int k = 0; k < nw; ++k) {
            const amc_option &o = opts[wave[k].idx];
            shift_off[k] = shifts.size();
            shifts.resize(shifts.size() + o.n_steps);
            host_shifts(o.seed, o.n_steps, shifts.data() + shift_off[k]);
        }
        uint32_t *shift_dev;
        AMC_TRY(arena_alloc(c, sizeof(uint32_t) * shifts.size(), (void **)&shift_dev));
        int64_t tiles = 0;
        int cta = 0, max_slots = 1;
        size_t arr_off = 0;
        for (int k = 0; k < nw; ++k) {
            const amc_option &o = opts[wave[k].idx];
            Job &J = jobs[k];
            fill_job_common(&o, &J);
            DevBridge *b;
            AMC_TRY(get_bridge(c, o.n_steps, &b));
            J.shift = shift_dev + shift_off[k];
            J.nodes = fp64 ? (const void *)b->nd : (const void *)b->nf;
            J.nslots = b->nslots;
            max_slots = std::max(max_slots, b->nslots);
            J.ld = host_ld(o.n_paths);
            AMC_TRY(arena_alloc(c, (size_t)o.n_steps * J.ld * esz, &J.S));
            J.tile_begin = tiles;
            J.n_tiles = (o.n_paths + kTilePoints - 1) / kTilePoints;
            tiles += J.n_tiles;
            J.cta_begin = cta;
            J.n_cta = wave[k].pl.ctas;
            J.chunks = chunks;
            cta += J.n_cta;
            J.greeks = greeks ? 1 : 0;
            if (plan0.kind == 2) {
                AMC_TRY(arena_alloc(c, v2_xch_units(o.n_steps, J.n_cta) * 8, (void **)&J.xch));
            } else {
                AMC_TRY(arena_alloc(c, (size_t)o.n_steps * J.n_cta * kNV * 8, &J.part));
            }
            J.arrive = arrive_all + arr_off;
            arr_off += o.n_steps;
            AMC_TRY(arena_alloc(c, (size_t)J.n_cta * 4 * sizeof(double), &J.fin));
            J.res = res_dev + (size_t)k * AMC_RES_DOUBLES;
            J.status = status_dev;
        }
        AMC_TRY_CUDA(cudaMemcpyAsync(shift_dev, shifts.data(), sizeof(uint32_t) * shifts.size(),
                                     cudaMemcpyHostToDevice, st));
        AMC_TRY_CUDA(cudaMemcpyAsync(jobs_dev, jobs.data(), sizeof(Job) * nw, cudaMemcpyHostToDevice, st));
        AMC_TRY_CUDA(cudaMemsetAsync(arrive_all, 0, sizeof(uint32_t) * arrive_words, st));
        AMC_TRY_CUDA(cudaMemsetAsync(status_dev, 0, sizeof(int32_t), st));
        KArgs &a = c->args;
        memset(&a, 0, sizeof(KArgs));
        a.jobs = jobs_dev;
        a.n_jobs = nw;
        a.max_m = max_m;
        a.max_slots = max_slots;
        a.jobs_type = opts[wave[0].idx].type;
        a.total = tiles;
        a.V = c->V;
        AMC_TRY_CUDA(launch_pathgen(a, fp64, c->sm_count, st));
        AMC_TRY(launch_sweeps(c, a, plan0, cta, lsm, fp64, greeks, st));
        std::vector<double> res((size_t)nw * AMC_RES_DOUBLES);
        AMC_TRY_CUDA(cudaMemcpyAsync(res.data(), res_dev, sizeof(double) * res.size(), cudaMemcpyDeviceToHost, st));
        AMC_TRY_CUDA(cudaStreamSynchronize(st));
        int wave_status = AMC_OK;
        for (int k = 0; k < nw; ++k) {
            int s = result_from(&res[(size_t)k * AMC_RES_DOUBLES], &out[wave[k].idx]);
            if (s != AMC_OK) wave_status = s;
        }
        if (wave_status != AMC_OK) return wave_status;
    }
    return AMC_OK;
}

}  // namespace

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
        default: return "unknown error";
    }
}

int amc_version(void) { return 1; }

int amc_validate_option(const amc_option *opt) { return host_validate(opt); }
int64_t amc_path_ld(int64_t n_paths) { return n_paths < 1 ? 0 : host_ld(n_paths); }
size_t amc_path_bytes(int n_steps, int64_t n_paths, int prec) {
    if (n_steps < 1 || n_paths < 1) return 0;
    return (size_t)n_steps * host_ld(n_paths) * (prec == AMC_FP64 ? 8 : 4);
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
int amc_plan_sweep(int64_t n_paths, int sm_count, int prec, int rule, int32_t *ctas, int32_t *paths_per_thread) {
    SweepPlan p;
    int rc = host_plan_sweep(n_paths, sm_count, prec, rule, &p);
    if (rc != AMC_OK) return rc;
    if (ctas) *ctas = p.ctas;
    if (paths_per_thread) *paths_per_thread = p.kind == 2 ? kV2PPT : 4 * p.chunks;
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
        if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            rc = AMC_ECUDA;
            break;
        }
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = AMC_ECUDA; break; }
        std::vector<uint32_t> V((size_t)AMC_MAX_STEPS * 32);
        if (host_directions(AMC_MAX_STEPS, V.data()) != AMC_OK) { rc = AMC_EINVAL; break; }
        if (cudaMalloc(&c->V, V.size() * 4) != cudaSuccess ||
            cudaMemcpy(c->V, V.data(), V.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = AMC_ECUDA;
            break;
        }
        c->gcap = 4 * c->sm_count;
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
            if (cudaEventCreate(&c->ev[k]) != cudaSuccess) rc = AMC_ECUDA;
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
    cudaFree(c->res1);
    cudaFree(c->status1);
    cudaFree(c->xch1);
    cudaFree(c->arena);
    if (c->res_host) cudaFreeHost(c->res_host);
    for (int k = 0; k < 3; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return AMC_OK;
}

int amc_ctx_set_timeout(amc_ctx *c, double seconds) {
    if (!c || !(seconds > 0.0) || seconds > 3600.0) return AMC_EINVAL;
    c->timeout_s = seconds;
    return AMC_OK;
}

int amc_ctx_inject(amc_ctx *c, int kind, int64_t arg) {
    if (!c || kind < 0 || kind > 2) return AMC_EINVAL;
    c->inject_kind = kind;
    c->inject_arg = arg;
    return AMC_OK;
}

int amc_ctx_memory(amc_ctx *c, size_t *free_bytes, size_t *total_bytes) {
    if (!c) return AMC_EINVAL;
    if (free_bytes) *free_bytes = c->arena_bytes - c->arena_top;
    if (total_bytes) *total_bytes = c->arena_bytes;
    return AMC_OK;
}

int amc_sobol(amc_ctx *c, int n_dims, int64_t n_points, uint64_t seed, uint32_t *x_dev, int64_t ld, void *stream) {
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
    if (!c) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_generate(c, opt, prec, S_dev, ld, (cudaStream_t)stream);
}

int amc_sweep(amc_ctx *c, const amc_option *opt, int prec, const void *S_dev, int64_t ld, int with_greeks,
              double *res_dev, void *stream) {
    if (!c) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return do_sweep(c, opt, prec, S_dev, ld, with_greeks != 0, res_dev, (cudaStream_t)stream);
}

int amc_price_device(amc_ctx *c, const amc_option *opt, int prec, void *S_dev, int64_t ld, double *res_dev,
                     void *stream) {
    if (!c) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    AMC_TRY(do_generate(c, opt, prec, S_dev, ld, (cudaStream_t)stream));
    return do_sweep(c, opt, prec, S_dev, ld, false, res_dev, (cudaStream_t)stream);
}

int amc_price_american(amc_ctx *c, double S0, double K, double r, double sigma, double T, int n_steps,
                       int64_t n_paths, int basis, int type, uint64_t seed, int rule, int prec, amc_result *out) {
    if (!c || !out) return AMC_EINVAL;
    amc_option o = make_option(S0, K, r, sigma, T, n_steps, n_paths, basis, type, seed, rule);
    AMC_TRY(host_validate(&o));
    AMC_TRY(check_prec(prec));
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    c->arena_top = 0;
    const int64_t ld = host_ld(n_paths);
    void *S;
    AMC_TRY(arena_alloc(c, (size_t)n_steps * ld * (prec == AMC_FP64 ? 8 : 4), &S));
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
    if (!c || n < 0 || (n > 0 && (!opts || !out))) return AMC_EINVAL;
    AMC_TRY_CUDA(cudaSetDevice(c->device));
    return run_batch(c, opts, n, prec, false, out);
}

int amc_greeks(amc_ctx *c, const amc_option *opts, int n, int prec, double *price, double *delta, double *vega) {
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
