// Internal declarations of the amc library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/amc.h"

namespace amc {

// Brownian-bridge node, in the depth-first evaluation order used by the
// path-generation kernel.  `coord` is the Sobol' dimension that the
// breadth-first numbering gives this node; `sl`/`sr`/`so` are slots of the
// per-path stack (slot d holds the latest node of depth d).
// W(t_date) = wl W(t_l) + wr W(t_r) + sdu sqrt(dt) z; a node with t_l = 0
// has wl = 0 and sl = sr (W(0) = 0 has no slot), the root wl = wr = 0.
struct NodeF {
    int32_t coord, date;
    int16_t sl, sr, so, pad;
    float wl, wr, sdu, pad2;
};
struct NodeD {
    int32_t coord, date;
    int16_t sl, sr, so, pad;
    double wl, wr, sdu;
};
static_assert(sizeof(NodeF) == 32, "NodeF layout");
static_assert(sizeof(NodeD) == 40, "NodeD layout");

constexpr int kMaxSlots = 12;       // depth <= 10 for m <= 512: 11 slots

struct BridgePlan {
    int m = 0;
    int nslots = 0;                 // stack slots (the tree's depth + 1)
    std::vector<NodeF> nf;          // depth-first order
    std::vector<NodeD> nd;
};

// Host tables (tables.cpp).
int host_directions(int n_dims, uint32_t *V);
void host_shifts(uint64_t seed, int n_dims, uint32_t *out);
void host_lcg_params(uint64_t seed, int n_dims, int64_t n_points, uint32_t *a, uint32_t *c, uint64_t *M);
int host_bridge_bfs(int m, int32_t *date, int32_t *left, int32_t *right);
int host_bridge_plan(int m, BridgePlan *plan);
int host_validate(const amc_option *o);
int64_t host_ld(int64_t n_paths);

// Sweep launch plan: threads per CTA, 4-path chunks per thread, CTAs.
constexpr int kSweepThreads = 256;
// CTAs per SM that the LSM kernel's launch bounds guarantee for a given
// number of 4-path chunks per thread (registers hold the per-path state).
constexpr int sweep_ctas_per_sm(int chunks) { return chunks <= 2 ? 4 : (chunks == 4 ? 2 : 1); }
// kind 1: generic sweep kernels (sweep.cu: FP64 LSM and the pathwise
// rules), `chunks` 4-path chunks per thread, 256 threads per CTA;
// kind 2: mixed-precision LSM kernel (sweep_v2.cu), 7680 paths per CTA,
// exchange through L2, all CTAs co-resident;
// kind 3: mixed-precision LSM kernel of one cluster per option
// (sweep_cl.cu), 16384 paths per CTA, `ctas` = the cluster size (up to
// max_cluster), exchange through distributed shared memory.  Frozen-
// boundary Greeks use kind 2 (plan_for_greeks).
struct SweepPlan {
    int kind;
    int chunks;
    int ctas;                       // CTAs for this option
};
constexpr int kClThreads = 1024;
constexpr int kClPPT = 16;
constexpr int kClPathsPerCta = kClThreads * kClPPT;   // 16384
constexpr int kClMaxCluster = 16;
int host_plan_sweep(int64_t n_paths, int sm_count, int prec, int rule, SweepPlan *p,
                    int max_cluster = kClMaxCluster);
// The plan of the Greeks variant: kind 3 has none, so such options take the
// kind-2 plan (AMC_EINVAL where that does not fit).
int plan_for_greeks(int64_t n_paths, int sm_count, SweepPlan *p);
constexpr int kV2MaxCtas = 160;

// ----------------------------------------------------------- device jobs
// One option as the kernels see it.  All pointers are device pointers.
struct Job {
    double S0, K, r, sigma, T;
    double dt, disc, invK;          // T/m, e^{-r dt}, 1/K
    int32_t m, p, type, rule;
    int64_t N, ld;
    const uint32_t *shift;          // [m]
    const void *nodes;              // NodeF[m] or NodeD[m], depth-first order
    int32_t nslots;
    int32_t greeks;                 // also accumulate delta and vega
    void *S;                        // Real S[m][ld]
    int64_t tile_begin;             // path-generation tiles: prefix over jobs
    int64_t n_tiles;
    int32_t cta_begin, n_cta;       // sweep CTA group
    int32_t chunks;                 // 4-path chunks per thread
    int32_t inject_date;            // test fault injection (0 = off)
    int32_t bad;                    // nonzero: a device-side input of this job failed validation
    void *part;                     // cross-CTA partial sums [m][n_cta][kNV] (double-float or double)
    uint32_t *arrive;               // [m] arrival counters (zeroed before launch)
    void *fin;                      // [n_cta][4] final per-CTA sums
    double *res;                    // [AMC_RES_DOUBLES]
    int32_t *status;                // shared error word of the launch
    double *coef;                   // exercise boundary [m][kCoefStride] written by an LSM sweep / read by valuation, or null
    uint64_t *xch;                  // tagged exchange units [m+2][kXV][n_cta] (mixed LSM sweep)
};

constexpr int kCoefStride = AMC_COEF_STRIDE;   // c_0..c_3 (units of K, basis y^k), degenerate flag
constexpr int kValueThreads = 256;             // boundary valuation: threads per CTA, 8 paths per thread
constexpr int kNV = 12;             // cross-CTA values per date: 2p-1 moments + p RHS (p <= 4)

// Mixed-precision LSM sweep (sweep_v2.cu): 2 solver warps + 30 path warps,
// 8 paths per path thread, a ring of 5 date slices in shared memory.
constexpr int kV2Threads = 1024;
constexpr int kV2Workers = 960;
constexpr int kV2PPT = 8;
constexpr int kV2PathsPerCta = kV2Workers * kV2PPT;   // 7680
constexpr int kV2Slots = 5;
constexpr int kXV = 11;             // exchanged values per date: 7 moment slots + 4 RHS slots
constexpr uint32_t kEpochBits = 22; // tag = epoch << 10 | exchange index
inline int v2_ctas(int64_t n_paths) { return (int)((n_paths + kV2PathsPerCta - 1) / kV2PathsPerCta); }
inline size_t v2_xch_units(int m, int ctas) { return (size_t)(m + 2) * kXV * ctas; }
constexpr int kPathgenThreads = 128;
constexpr int kPathgenQ = 4;        // consecutive points per thread per tile
constexpr int kTilePoints = kPathgenThreads * kPathgenQ;

// Kernel arguments, passed by value (__grid_constant__): either a device
// array of jobs (batches) or one job held inline together with its digital
// shifts, so a single-option call needs no host-to-device copy at all.
struct KArgs {
    const Job *jobs;                // device array, or nullptr: use `one`
    int32_t n_jobs;
    int32_t max_m;
    int32_t max_slots;              // largest bridge stack over the jobs (path generation)
    int32_t jobs_type;              // AMC_PUT / AMC_CALL shared by all jobs of a mixed LSM launch
    int32_t h16;                    // path arrays hold binary16 moneyness (AMC_MIXED16)
    int32_t jobs_p;                 // basis size shared by all jobs of a cluster-sweep launch
    int64_t total;                  // path-generation tiles over all jobs
    const uint32_t *V;              // direction numbers [AMC_MAX_STEPS][32]
    uint64_t timeout_ns;
    uint32_t epoch;                 // launch tag of the mixed LSM sweep's exchange units
    uint32_t poll_ns;               // back-off between exchange polls (mixed LSM sweep)
    Job one;
    uint32_t shift_one[AMC_MAX_STEPS];
};

// Kernel launchers (pathgen.cu, sweep.cu).  Return a cudaError_t.
cudaError_t launch_sobol(const uint32_t *V, int n_dims, int64_t n_points, const uint32_t *shift,
                         uint32_t *x, int64_t ld, cudaStream_t st);
cudaError_t launch_pathgen(const KArgs &a, bool fp64, int sm_count, cudaStream_t st);
// Path generation that values each path as it is formed and stores nothing
// (pathgen.cu): the rules that need no regression across paths, and the
// valuation of a fitted boundary.  One option (a.one); per-CTA sums into
// a.one.fin[grid][4] for launch_finalize.
// kStore16 (FP32 only) stores the moneyness y = S/K - 1 in binary16
// instead of S (AMC_MIXED16).
enum { kStore = 0, kPaperRule = 1, kEuropean = 2, kBoundary = 3, kStore16 = 4 };
cudaError_t pathgen_fused_grid(const KArgs &a, int mode, bool fp64, int sm_count, int64_t *grid);
cudaError_t launch_pathgen_fused(const KArgs &a, int mode, bool fp64, int64_t grid, cudaStream_t st);
cudaError_t launch_sweep_lsm(const KArgs &a, int total_ctas, int chunks, bool fp64, bool greeks,
                             cudaStream_t st);
cudaError_t launch_sweep_pathwise(const KArgs &a, int total_ctas, int chunks, bool fp64, bool greeks,
                                  cudaStream_t st);
cudaError_t launch_finalize(const KArgs &a, cudaStream_t st);
// Device-side inputs and outputs of a batch wave (sweep.cu): the spot and
// volatility of job k replaced by S0[idx[k]] and sigma[idx[k]] (either may
// be null) before path generation, a job whose value is not finite and
// positive marked bad; after finalize the wave's result blocks res_wave
// [n][AMC_RES_DOUBLES] scattered to res[idx[k]] (full blocks) and to
// price/delta/vega[idx[k]] (any of the four may be null).
cudaError_t launch_patch_inputs(Job *jobs, int n, const int32_t *idx, const double *S0, const double *sigma,
                                cudaStream_t st);
cudaError_t launch_scatter_results(const double *res_wave, int n, const int32_t *idx, double *res, double *price,
                                   double *delta, double *vega, cudaStream_t st);
cudaError_t launch_sweep_lsm_v2(const KArgs &a, int total_ctas, bool greeks, cudaStream_t st);
// Cluster sweep (sweep_cl.cu): n_clusters options of `cluster` CTAs each
// (a.jobs[k] on CTAs k*cluster ..), or a.one on one cluster.
cudaError_t launch_sweep_cl(const KArgs &a, int cluster, int n_clusters, cudaStream_t st);
// Largest cluster the current device can hold at once (0: none).
cudaError_t sweep_cl_max_cluster(int *out);
size_t sweep_cl_smem();
cudaError_t launch_value_boundary(const KArgs &a, int ctas, bool fp64, cudaStream_t st);

// Path generation from the LCG-permuted unshifted points (one option).
struct PermArgs {
    Job one;
    const uint32_t *V;              // direction numbers [AMC_MAX_STEPS][32]
    int64_t total;                  // tiles of kTilePoints points
    int32_t max_slots;
    uint32_t log2M;                 // modulus M = 2^log2M >= N
    uint32_t a[AMC_MAX_STEPS], c[AMC_MAX_STEPS];
};
cudaError_t launch_pathgen_permuted(const PermArgs &a, bool fp64, int sm_count, cudaStream_t st);
int64_t value_ctas(int64_t n_paths);            // CTAs of the boundary valuation (one 2048-path slice each)

size_t pathgen_smem_bytes(int max_m, int nslots, bool fp64);

// Launch facts computed once (launch.cpp): raise a kernel's dynamic
// shared-memory limit to at least `smem`; its co-resident CTAs per SM.
cudaError_t ensure_smem(const void *f, size_t smem);
cudaError_t ctas_per_sm(const void *f, int threads, size_t smem, int *out);

// Streaming LSM sweep for options whose per-path state does not fit on chip
// (sweep_stream.cu): the option, its paths S [m][ld], result block, status
// and optional boundary output in `one`; scratch in device memory.
struct StreamArgs {
    Job one;
    void *cf;                       // [ld] cash flows (units of K), Real
    double *part;                   // [grid][kNV] per-CTA partial sums of the current date
    double *beta;                   // [m][4] coefficients (units of K) of dates 1..m
    int32_t *deg;                   // [m] degenerate flags
    int32_t *ndeg;                  // degenerate dates so far
    int32_t grid;                   // CTAs of every pass
    int32_t h16;                    // S holds binary16 moneyness (AMC_MIXED16)
};
constexpr int kStreamThreads = 256;
int64_t stream_grid(int sm_count, bool fp64, bool put, bool h16 = false);
cudaError_t launch_lsm_stream(const StreamArgs &a, bool fp64, cudaStream_t st);

// Dual upper bound of a fitted boundary (dual.cu): the option, its outer
// paths S [m][ld], boundary coef, result block and status word in `one`.
struct DualArgs {
    Job one;
    int64_t n_in;                   // inner paths per outer path and date
    uint64_t seed_in;               // counter-based SplitMix64 seed of the inner normals
    double *L1;                     // [N] L_1 per outer path (scratch)
    double *V;                      // [N] max_j (Z_j - M_j - L0) per outer path (scratch)
    double *W;                      // [N] inner steps simulated per outer path (scratch)
    double *U;                      // [N] U = L0 + V per outer path, or null
};
constexpr int kDualThreads = 256;           // inner simulations: up to 8 warps per outer path
constexpr int kDualFinalThreads = 1024;
size_t dual_smem(int m, bool fp64);
cudaError_t launch_dual_upper(const DualArgs &a, bool fp64, cudaStream_t st);

}  // namespace amc
