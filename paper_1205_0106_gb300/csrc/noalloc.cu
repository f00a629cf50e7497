// amc_sweep_noalloc: the backward sweep with its scratch memory in a
// file-scope device array instead of a context, for callers that must not
// allocate device memory.  Nothing here calls cudaMalloc, cudaFree or any
// other allocating routine; the kernels are the same ones amc_sweep
// launches, only their scratch pointers differ.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "internal.h"

using namespace amc;

namespace {

// Scratch of every amc_sweep_noalloc call on a device: status word, arrival
// counters, per-CTA final sums and per-date cross-CTA partials.  Each GPU
// that loads the library holds these bytes until the process exits (with
// lazy module loading, from the first call on that device on).
constexpr size_t kNoallocBytes = size_t(16) << 20;
constexpr size_t kOffStatus = 0;
constexpr size_t kOffArrive = 256;                                  // AMC_MAX_STEPS u32
constexpr size_t kOffFin = kOffArrive + 4 * AMC_MAX_STEPS;          // [G][4] double
constexpr size_t kMaxFinCtas = 2048;
constexpr size_t kOffData = kOffFin + 32 * kMaxFinCtas;             // partials [m][G][kNV] or exchange units
static_assert(kOffData == 67840, "fixed overhead stated in amc.h");
constexpr uint64_t kWaitNs = 2000000000ull;                         // device-wait limit, stated in amc.h

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_dev[kMaxDevices];   // device address of g_noalloc_scratch, per device
int g_sm_count[kMaxDevices];
int g_max_cluster[kMaxDevices];              // largest cluster sweep the device holds, per device
uint32_t g_epoch[kMaxDevices];               // launch tags of the exchange units, per device

// Once per device, with that device current: look up the array's device
// address (the host-side name is only a stand-in) and the SM count.
int setup_device(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_dev[dev]) return AMC_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return AMC_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return AMC_ECUDA;
    g_sm_count[dev] = sms;
    if (sweep_cl_max_cluster(&g_max_cluster[dev]) != cudaSuccess) g_max_cluster[dev] = 0;
    cudaGetLastError();
    g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    return AMC_OK;
}

}  // namespace

extern "C" size_t amc_sweep_noalloc_capacity(void) { return kNoallocBytes; }

extern "C" int amc_sweep_noalloc(const amc_option *opt, int prec, const void *S_dev, int64_t ld,
                                 int with_greeks, double *res_dev, void *stream) {
    int rc = host_validate(opt);
    if (rc != AMC_OK) return rc;
    if (prec != AMC_FP64 && prec != AMC_MIXED) return AMC_EINVAL;
    if (!S_dev || ld < host_ld(opt->n_paths) || ld % 32 != 0 || ((uintptr_t)S_dev & 15u) != 0) return AMC_EINVAL;
    if (!res_dev || ((uintptr_t)res_dev & 7u) != 0) return AMC_EINVAL;
    if (with_greeks && opt->rule == AMC_RULE_PAPER_UB) return AMC_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AMC_ECUDA;
    rc = setup_device(dev);
    if (rc != AMC_OK) return rc;
    SweepPlan pl;
    rc = host_plan_sweep(opt->n_paths, g_sm_count[dev], prec, opt->rule, &pl, with_greeks ? 0 : g_max_cluster[dev]);
    if (rc != AMC_OK) return rc;
    const size_t data_bytes = pl.kind == 3 ? 0
                              : pl.kind == 2 ? v2_xch_units(opt->n_steps, pl.ctas) * 8
                                             : (size_t)opt->n_steps * pl.ctas * kNV * 8;
    if ((size_t)pl.ctas > kMaxFinCtas || kOffData + data_bytes > kNoallocBytes) return AMC_EINVAL;

    unsigned char *base = g_scratch_dev[dev];
    cudaStream_t st = (cudaStream_t)stream;
    KArgs a;
    memset(&a, 0, sizeof(a));
    Job &J = a.one;
    J.S0 = opt->S0; J.K = opt->K; J.r = opt->r; J.sigma = opt->sigma; J.T = opt->T;
    J.m = opt->n_steps;
    J.p = opt->rule == AMC_RULE_LSM ? opt->basis : 1;
    J.type = opt->type;
    J.rule = opt->rule;
    J.N = opt->n_paths;
    J.dt = opt->T / opt->n_steps;
    J.disc = exp(-opt->r * J.dt);
    J.invK = 1.0 / opt->K;
    J.S = const_cast<void *>(S_dev);
    J.ld = ld;
    J.cta_begin = 0;
    J.n_cta = pl.ctas;
    J.chunks = pl.chunks;
    J.greeks = with_greeks ? 1 : 0;
    J.status = reinterpret_cast<int32_t *>(base + kOffStatus);
    J.arrive = reinterpret_cast<uint32_t *>(base + kOffArrive);
    J.fin = base + kOffFin;
    J.part = base + kOffData;
    J.xch = reinterpret_cast<uint64_t *>(base + kOffData);
    J.res = res_dev;
    a.jobs = nullptr;
    a.n_jobs = 1;
    a.max_m = opt->n_steps;
    a.timeout_ns = kWaitNs;
    // The array keeps the previous call's contents: clear what must start at
    // zero (status, arrival counters).  The data region holds the FP64 and
    // pathwise sweeps' double partials as well as the mixed sweep's tagged
    // exchange units, and a stale double whose high word happened to equal
    // this call's tag would pass for a posted unit: a mixed call clears the
    // units it will poll first.
    if (cudaMemsetAsync(base, 0, kOffFin, st) != cudaSuccess) return AMC_ECUDA;
    if (pl.kind == 2) {
        if (cudaMemsetAsync(base + kOffData, 0, data_bytes, st) != cudaSuccess) return AMC_ECUDA;
        std::lock_guard<std::mutex> lk(g_mu);
        g_epoch[dev] = (g_epoch[dev] + 1) & ((1u << kEpochBits) - 1u);
        if (g_epoch[dev] == 0) g_epoch[dev] = 1;
        a.epoch = g_epoch[dev];
        a.poll_ns = 0;
    }
    const bool fp64 = prec == AMC_FP64;
    a.timeout_ns = kWaitNs;
    cudaError_t e = pl.kind == 3 ? launch_sweep_cl(a, pl.ctas, 1, st)
                    : pl.kind == 2 ? launch_sweep_lsm_v2(a, pl.ctas, with_greeks != 0, st)
                    : opt->rule == AMC_RULE_LSM
                        ? launch_sweep_lsm(a, pl.ctas, pl.chunks, fp64, with_greeks != 0, st)
                        : launch_sweep_pathwise(a, pl.ctas, pl.chunks, fp64, with_greeks != 0, st);
    if (e != cudaSuccess) return AMC_ECUDA;
    if (launch_finalize(a, st) != cudaSuccess) return AMC_ECUDA;
    return AMC_OK;
}
