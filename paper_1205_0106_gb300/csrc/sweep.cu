// Backward early-exercise sweep (step 4 of the hot path) for sm_103a.
//
// LSM (Longstaff-Schwartz, ref. [12]; the backward induction of §V): one
// persistent cooperative launch; each CTA group owns one option and each
// thread owns 4*C paths whose cash flow CF (and, for Greeks, the stopping
// date and price) stay in registers for the whole sweep.  Per exercise date
// j = m-1..1:
//   read S[j-1][own paths] once (float4, streaming), CF *= e^{-r dt};
//   per-thread plain sums over the own paths of the in-the-money moments
//   M_k = sum y^k (k < 2p-1) and right-hand sides R_k = sum y^k CF (k < p),
//   y = S/K - 1, then a warp shuffle tree, then double-float (FP32 pairs;
//   doubles in FP64) across warps and the group's CTAs in a fixed order;
//   every CTA of the group reads all CTA partials once the date's arrival
//   counter is complete and reduces them the same way, so all CTAs obtain
//   bit-identical totals, solve the equilibrated normal equations in FP64
//   and apply the same exercise rule: CF = h(S) where h(S) > phi(x).beta.
// Every wait is bounded by a time limit read from %globaltimer; on expiry
// the CTA records AMC_ETIMEOUT in the launch's status word and returns, and
// the other CTAs see the status and return too.
//
// Pathwise rules (no cross-path reduction per date): the paper's Eqs. 10-11
// (Black-Scholes value over the last interval, then V = max(h, e^{-r dt} V)
// back to t = 0) and the European value of Eqs. 6-8.
//
// Final sums (price, second moment, delta, vega) per CTA, then one
// finalize CTA per option adds them in a fixed order in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <math_constants.h>

#include "devutil.cuh"
#include "internal.h"
#include "lsm_solve.cuh"

namespace amc {

namespace {

struct dfl {
    float hi, lo;
};

// Compensated addition of two double-float values (Knuth's TwoSum on the
// high words, low words folded in, then renormalised).  The _rn intrinsics
// keep the compiler from contracting or reassociating the error terms.
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, s))};
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void red_release_add(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_volatile_int(const int32_t *p) { return *(volatile const int32_t *)p; }

// 4 consecutive path values of one date row.
__device__ __forceinline__ void load4(const float *row, int64_t i, float *o) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(row + i));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double *row, int64_t i, double *o) {
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(row + i));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(row + i + 2));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

using dev::bs_value;
using dev::payoff;

__device__ __forceinline__ int find_job_by_cta(const Job *__restrict__ jobs, int n_jobs, int cta) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].cta_begin <= cta) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool FP64>
struct SW;
template <>
struct SW<false> {
    using Real = float;
};
template <>
struct SW<true> {
    using Real = double;
};

// Cross-CTA partial: one 8-byte word per value (double-float or double).
__device__ __forceinline__ void store_part(void *part, int64_t idx, dfl v) {
    reinterpret_cast<float2 *>(part)[idx] = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ void store_part(void *part, int64_t idx, double v) {
    reinterpret_cast<double *>(part)[idx] = v;
}
__device__ __forceinline__ dfl load_part_df(const void *part, int64_t idx) {
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(part) + idx);
    return {v.x, v.y};
}
__device__ __forceinline__ double load_part_d(const void *part, int64_t idx) {
    return __ldcg(reinterpret_cast<const double *>(part) + idx);
}

constexpr int kWarps = kSweepThreads / 32;

// Block sum of the per-thread values v[k] whose bit k is set in `mask`:
// warp shuffle tree in the working precision, then the warp partials in
// fixed order in double-float (mixed) or double.  Result in thread k.
template <bool FP64, int NVAL>
__device__ __forceinline__ void block_sum(typename SW<FP64>::Real (&v)[NVAL], void *s_warp, uint32_t mask,
                                          dfl *out_df, double *out_d) {
    using Real = typename SW<FP64>::Real;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NVAL; ++k) {
        if ((mask >> k) & 1) {
#pragma unroll
            for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
        }
    }
    Real *sw = reinterpret_cast<Real *>(s_warp);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NVAL; ++k)
            if ((mask >> k) & 1) sw[w * NVAL + k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < NVAL && ((mask >> threadIdx.x) & 1)) {
        const int k = threadIdx.x;
        if (FP64) {
            double a = 0.0;
            for (int q = 0; q < kWarps; ++q) a += (double)sw[q * NVAL + k];
            *out_d = a;
        } else {
            dfl a = {0.f, 0.f};
            for (int q = 0; q < kWarps; ++q) a = df_add(a, dfl{(float)sw[q * NVAL + k], 0.f});
            *out_df = a;
        }
    }
}

template <bool FP64, int C, bool GREEKS>
__global__ void __launch_bounds__(kSweepThreads, sweep_ctas_per_sm(C))
sweep_lsm_kernel(const __grid_constant__ KArgs a) {
    using Real = typename SW<FP64>::Real;
    constexpr int P = 4 * C;
    __shared__ __align__(16) unsigned char s_warp[kWarps * kNV * sizeof(Real)];
    __shared__ double s_tot[kNV];
    __shared__ double s_beta[4];
    __shared__ int s_flag;

    const int jb = a.jobs ? find_job_by_cta(a.jobs, a.n_jobs, blockIdx.x) : 0;
    const Job &J = a.jobs ? a.jobs[jb] : a.one;
    const uint64_t timeout_ns = a.timeout_ns;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int lc = blockIdx.x - J.cta_begin, G = J.n_cta;
    const int m = J.m, p = J.p, nmom = 2 * p - 1;
    const uint32_t vmask = ((1u << nmom) - 1u) | (((1u << p) - 1u) << 7);   // used value slots
    const bool put = J.type == AMC_PUT;
    const Real K = (Real)J.K, invK = (Real)J.invK, disc = (Real)J.disc;
    const Real *__restrict__ S = reinterpret_cast<const Real *>(J.S);
    const int64_t N = J.N, ld = J.ld;
    const int64_t gt = (int64_t)lc * kSweepThreads + tid, TT = (int64_t)G * kSweepThreads;
    void *part = J.part;
    int32_t *status = J.status;
    uint32_t *const arrive = J.arrive;
    const int inject_date = (lc == 0 && jb == 0) ? J.inject_date : 0;

    Real cf[P];
    int tau[GREEKS ? P : 1];
    Real st[GREEKS ? P : 1];
    {
        const Real *row = S + (int64_t)(m - 1) * ld;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int64_t i0 = 4 * (gt + c * TT);
            Real s[4] = {Real(0), Real(0), Real(0), Real(0)};
            if (i0 < N) load4(row, i0, s);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool valid = i0 + e < N;
                cf[4 * c + e] = valid ? payoff(put, s[e], K) : Real(0);
                if (GREEKS) { tau[4 * c + e] = m; st[4 * c + e] = s[e]; }
            }
        }
    }
    int degenerate = 0;
    if (J.coef && lc == 0 && tid < kCoefStride)             // maturity: no exercise decision
        J.coef[(size_t)(m - 1) * kCoefStride + tid] = tid == 4 ? 1.0 : 0.0;
    for (int j = m - 1; j >= 1; --j) {
        const Real *row = S + (int64_t)(j - 1) * ld;
        Real s[P];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int64_t i0 = 4 * (gt + c * TT);
            if (i0 < N) load4(row, i0, s + 4 * c);
            else { s[4 * c] = s[4 * c + 1] = s[4 * c + 2] = s[4 * c + 3] = Real(0); }
        }
        Real th[kNV - 1];
#pragma unroll
        for (int k = 0; k < kNV - 1; ++k) th[k] = Real(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int q = 4 * c + e;
                const bool valid = 4 * (gt + c * TT) + e < N;
                cf[q] *= disc;
                const Real h = payoff(put, s[q], K);
                if (valid && h > Real(0)) {
                    const Real y = s[q] * invK - Real(1);
                    Real yp = Real(1);
#pragma unroll
                    for (int k = 0; k < 7; ++k) {
                        if (k < nmom) th[k] += yp;
                        if (k < p) th[7 + k] += yp * cf[q];
                        yp *= y;
                    }
                }
            }
        }
        // fixed slots: moments 0..6 (first nmom used), RHS 7..10 (first p used)
        dfl mydf;
        double myd;
        block_sum<FP64, kNV - 1>(th, s_warp, vmask, &mydf, &myd);
        if (tid < kNV - 1 && ((vmask >> tid) & 1)) {
            const int64_t idx = ((int64_t)(j - 1) * G + lc) * kNV + tid;
            if (FP64) store_part(part, idx, myd); else store_part(part, idx, mydf);
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) {
            // arrive (release: this CTA's partials are visible first), then
            // poll with relaxed loads and take one acquire fence at the end
            int flag = 0;
            uint32_t *arr = arrive + (j - 1);
            if (inject_date != j) red_release_add(arr, 1u);
            const uint64_t t0 = globaltimer();
            while (ld_relaxed(arr) < (uint32_t)G) {
                if (ld_volatile_int(status) != 0) { flag = 1; break; }
                if (globaltimer() - t0 > timeout_ns) {
                    atomicCAS(status, 0, AMC_ETIMEOUT);
                    flag = 1;
                    break;
                }
            }
            fence_acq_rel_gpu();
            s_flag = flag;
        }
        __syncthreads();
        if (s_flag) return;
        // every CTA reduces all partials of this date in the same fixed order
        for (int v = wid; v < kNV - 1; v += kWarps) {
            if (!((vmask >> v) & 1)) continue;
            const int64_t base = (int64_t)(j - 1) * G * kNV + v;
            if (FP64) {
                double a = 0.0;
                for (int c = lane; c < G; c += 32) a += load_part_d(part, base + (int64_t)c * kNV);
#pragma unroll
                for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
                if (lane == 0) s_tot[v] = a;
            } else {
                dfl a = {0.f, 0.f};
                for (int c = lane; c < G; c += 32) a = df_add(a, load_part_df(part, base + (int64_t)c * kNV));
#pragma unroll
                for (int off = 16; off; off >>= 1) {
                    dfl o;
                    o.hi = __shfl_xor_sync(0xffffffffu, a.hi, off);
                    o.lo = __shfl_xor_sync(0xffffffffu, a.lo, off);
                    a = df_add(a, o);
                }
                if (lane == 0) s_tot[v] = (double)a.hi + (double)a.lo;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double beta[4] = {0, 0, 0, 0};
            bool ok = s_tot[0] >= (double)p && solve_normal(p, s_tot, s_tot + 7, beta);
            for (int k = 0; k < 4; ++k) s_beta[k] = beta[k];
            s_flag = ok ? 0 : 2;
            if (J.coef && lc == 0) {                          // fitted boundary of date j (units of K)
                double *cj = J.coef + (size_t)(j - 1) * kCoefStride;
                for (int k = 0; k < 4; ++k) cj[k] = ok ? beta[k] * J.invK : 0.0;
                cj[4] = ok ? 0.0 : 1.0;
            }
        }
        __syncthreads();
        if (s_flag == 2) {
            ++degenerate;
            continue;
        }
        Real b[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = (Real)s_beta[k];
#pragma unroll
        for (int c = 0; c < C; ++c) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int q = 4 * c + e;
                const bool valid = 4 * (gt + c * TT) + e < N;
                const Real h = payoff(put, s[q], K);
                if (valid && h > Real(0)) {
                    const Real y = s[q] * invK - Real(1);
                    Real cont = b[3];
                    cont = cont * y + b[2];
                    cont = cont * y + b[1];
                    cont = cont * y + b[0];
                    if (h > cont) {
                        cf[q] = h;
                        if (GREEKS) { tau[q] = j; st[q] = s[q]; }
                    }
                }
            }
        }
    }
    // final per-CTA sums: CF, CF^2, delta, vega (discounting to 0 in finalize)
    Real fsum[4] = {Real(0), Real(0), Real(0), Real(0)};
    const Real S0 = (Real)J.S0, r = (Real)J.r, sig = (Real)J.sigma, dt = (Real)J.dt;
    const Real mu = r - Real(0.5) * sig * sig;
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = 4 * c + e;
            const bool valid = 4 * (gt + c * TT) + e < N;
            if (!valid) continue;
            fsum[0] += cf[q];
            fsum[1] += cf[q] * cf[q];
            if (GREEKS && cf[q] > Real(0)) {
                const Real t = (Real)tau[q] * dt;
                const Real dfac = exp(-r * t);
                const Real dh = put ? Real(-1) : Real(1);
                const Real Wt = (log(st[q] / S0) - mu * t) / sig;
                fsum[2] += dfac * dh * st[q] / S0;
                fsum[3] += dfac * dh * st[q] * (Wt - sig * t);
            }
        }
    }
    dfl fdf;
    double fd;
    block_sum<FP64, 4>(fsum, s_warp, 0xFu, &fdf, &fd);
    if (tid < 4) {
        double* fin = reinterpret_cast<double *>(J.fin);
        fin[(int64_t)lc * 4 + tid] = FP64 ? fd : (double)fdf.hi + (double)fdf.lo;
    }
    if (lc == 0 && tid == 0) J.res[4] = (double)degenerate;
}

template <bool FP64, int C, bool GREEKS>
__global__ void __launch_bounds__(kSweepThreads)
sweep_pathwise_kernel(const __grid_constant__ KArgs a) {
    using Real = typename SW<FP64>::Real;
    constexpr int P = 4 * C;
    __shared__ __align__(16) unsigned char s_warp[kWarps * kNV * sizeof(Real)];
    const int jb = a.jobs ? find_job_by_cta(a.jobs, a.n_jobs, blockIdx.x) : 0;
    const Job &J = a.jobs ? a.jobs[jb] : a.one;
    const int tid = threadIdx.x;
    const int lc = blockIdx.x - J.cta_begin, G = J.n_cta;
    const int m = J.m;
    const bool put = J.type == AMC_PUT;
    const Real K = (Real)J.K, disc = (Real)J.disc, S0 = (Real)J.S0, r = (Real)J.r;
    const Real sig = (Real)J.sigma, dt = (Real)J.dt, T = (Real)J.T;
    const Real *__restrict__ S = reinterpret_cast<const Real *>(J.S);
    const int64_t N = J.N, ld = J.ld;
    const int64_t gt = (int64_t)lc * kSweepThreads + tid, TT = (int64_t)G * kSweepThreads;
    Real V[P];
    Real fsum[4] = {Real(0), Real(0), Real(0), Real(0)};
    if (J.rule == AMC_RULE_EUROPEAN) {
        const Real dfT = exp(-r * T);
        const Real mu = r - Real(0.5) * sig * sig;
        const Real *row = S + (int64_t)(m - 1) * ld;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int64_t i0 = 4 * (gt + c * TT);
            Real s[4] = {Real(0), Real(0), Real(0), Real(0)};
            if (i0 < N) load4(row, i0, s);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (i0 + e >= N) continue;
                const Real h = payoff(put, s[e], K);
                const Real v = dfT * h;
                fsum[0] += v;
                fsum[1] += v * v;
                if (GREEKS && h > Real(0)) {
                    const Real dh = put ? Real(-1) : Real(1);
                    const Real Wt = (log(s[e] / S0) - mu * T) / sig;
                    fsum[2] += dfT * dh * s[e] / S0;
                    fsum[3] += dfT * dh * s[e] * (Wt - sig * T);
                }
            }
        }
    } else {
        // Eq. 10 over the last interval [t_{m-1}, t_m], then Eq. 11 back to t_0.
        {
            Real s[P];
            if (m >= 2) {
                const Real *row = S + (int64_t)(m - 2) * ld;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int64_t i0 = 4 * (gt + c * TT);
                    if (i0 < N) load4(row, i0, s + 4 * c);
                    else { s[4 * c] = s[4 * c + 1] = s[4 * c + 2] = s[4 * c + 3] = S0; }
                }
            } else {
#pragma unroll
                for (int q = 0; q < P; ++q) s[q] = S0;
            }
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const Real h = payoff(put, s[q], K);
                const Real c = bs_value(put, s[q], K, r, sig, dt);
                V[q] = h > c ? h : c;
            }
        }
#pragma unroll 4
        for (int j = m - 2; j >= 1; --j) {
            const Real *row = S + (int64_t)(j - 1) * ld;
            Real s[P];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int64_t i0 = 4 * (gt + c * TT);
                if (i0 < N) load4(row, i0, s + 4 * c);
                else { s[4 * c] = s[4 * c + 1] = s[4 * c + 2] = s[4 * c + 3] = S0; }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const Real h = payoff(put, s[q], K), cont = disc * V[q];
                V[q] = h > cont ? h : cont;
            }
        }
        if (m >= 2) {
            const Real h0 = payoff(put, S0, K);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const Real cont = disc * V[q];
                V[q] = h0 > cont ? h0 : cont;
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (4 * (gt + c * TT) + e >= N) continue;
                fsum[0] += V[4 * c + e];
                fsum[1] += V[4 * c + e] * V[4 * c + e];
            }
        }
    }
    dfl fdf;
    double fd;
    block_sum<FP64, 4>(fsum, s_warp, 0xFu, &fdf, &fd);
    if (tid < 4) {
        double* fin = reinterpret_cast<double *>(J.fin);
        fin[(int64_t)lc * 4 + tid] = FP64 ? fd : (double)fdf.hi + (double)fdf.lo;
    }
    if (lc == 0 && tid == 0) J.res[4] = 0.0;
}

// One CTA per option: fixed-order FP64 sum of the per-CTA final sums.
__global__ void __launch_bounds__(256) finalize_kernel(const __grid_constant__ KArgs a) {
    const Job &J = a.jobs ? a.jobs[blockIdx.x] : a.one;
    __shared__ double s[256][4];
    const int tid = threadIdx.x;
    double acc[4] = {0, 0, 0, 0};
    const double *fin = reinterpret_cast<const double *>(J.fin);
    for (int c = tid; c < J.n_cta; c += 256)
        for (int k = 0; k < 4; ++k) acc[k] += fin[(int64_t)c * 4 + k];
    for (int k = 0; k < 4; ++k) s[tid][k] = acc[k];
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (tid < w)
            for (int k = 0; k < 4; ++k) s[tid][k] += s[tid + w][k];
        __syncthreads();
    }
    if (tid == 0) {
        const double N = (double)J.N;
        const double scale = J.rule == AMC_RULE_LSM ? J.disc : 1.0;
        const double mean = s[0][0] / N;
        const double var = J.N > 1 ? (s[0][1] - N * mean * mean) / (N - 1.0) : 0.0;
        double *res = J.res;
        res[0] = scale * mean;
        res[1] = var > 0.0 ? scale * sqrt(var / N) : 0.0;
        res[2] = s[0][2] / N;
        res[3] = s[0][3] / N;
        res[5] = (double)ld_volatile_int(J.status);
        if (J.bad) {                    // a device-side input failed validation: no price
            res[0] = res[1] = res[2] = res[3] = CUDART_NAN;
            res[5] = (double)AMC_EINVAL;
        }
    }
}

// Spot and volatility of each job of a wave from device memory (a caller's
// tensors), checked here since the host never sees them; a rejected value
// is replaced by a harmless one so that the wave runs as planned, and the
// job is marked bad (finalize then writes NaN and AMC_EINVAL).
__global__ void patch_inputs_kernel(Job *jobs, int n, const int32_t *idx, const double *S0, const double *sigma) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    Job &J = jobs[k];
    const int i = idx[k];
    int bad = 0;
    if (S0) {
        const double v = S0[i];
        const bool ok = isfinite(v) && v > 0.0;
        J.S0 = ok ? v : J.K;
        bad |= !ok;
    }
    if (sigma) {
        const double v = sigma[i];
        const bool ok = isfinite(v) && v > 0.0;
        J.sigma = ok ? v : 0.2;
        bad |= !ok;
    }
    J.bad = bad;
}

// A wave's result blocks (wave order) to the caller's arrays (input order).
__global__ void scatter_results_kernel(const double *res_wave, int n, const int32_t *idx, double *res, double *price,
                                       double *delta, double *vega) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double *r = res_wave + (size_t)k * AMC_RES_DOUBLES;
    const int i = idx[k];
    if (res)
        for (int q = 0; q < AMC_RES_DOUBLES; ++q) res[(size_t)i * AMC_RES_DOUBLES + q] = r[q];
    if (price) price[i] = r[0];
    if (delta) delta[i] = r[2];
    if (vega) vega[i] = r[3];
}

template <bool FP64, bool GREEKS>
cudaError_t launch_lsm_c(const KArgs &a, int total, int chunks, cudaStream_t st) {
    void *args[] = {(void *)&a};
    const void *f;
    switch (chunks) {
        case 1: f = (const void *)sweep_lsm_kernel<FP64, 1, GREEKS>; break;
        case 2: f = (const void *)sweep_lsm_kernel<FP64, 2, GREEKS>; break;
        case 4: f = (const void *)sweep_lsm_kernel<FP64, 4, GREEKS>; break;
        case 8: f = (const void *)sweep_lsm_kernel<FP64, 8, GREEKS>; break;
        default: return cudaErrorInvalidValue;
    }
    return cudaLaunchCooperativeKernel(f, dim3((unsigned)total), dim3(kSweepThreads), args, 0, st);
}

template <bool FP64, bool GREEKS>
cudaError_t launch_pw_c(const KArgs &a, int total, int chunks, cudaStream_t st) {
    switch (chunks) {
        case 1: sweep_pathwise_kernel<FP64, 1, GREEKS><<<total, kSweepThreads, 0, st>>>(a); break;
        case 2: sweep_pathwise_kernel<FP64, 2, GREEKS><<<total, kSweepThreads, 0, st>>>(a); break;
        case 4: sweep_pathwise_kernel<FP64, 4, GREEKS><<<total, kSweepThreads, 0, st>>>(a); break;
        case 8: sweep_pathwise_kernel<FP64, 8, GREEKS><<<total, kSweepThreads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_lsm(const KArgs &a, int total_ctas, int chunks, bool fp64, bool greeks, cudaStream_t st) {
    if (fp64) return greeks ? launch_lsm_c<true, true>(a, total_ctas, chunks, st)
                            : launch_lsm_c<true, false>(a, total_ctas, chunks, st);
    return greeks ? launch_lsm_c<false, true>(a, total_ctas, chunks, st)
                  : launch_lsm_c<false, false>(a, total_ctas, chunks, st);
}

cudaError_t launch_sweep_pathwise(const KArgs &a, int total_ctas, int chunks, bool fp64, bool greeks,
                                  cudaStream_t st) {
    if (fp64) return greeks ? launch_pw_c<true, true>(a, total_ctas, chunks, st)
                            : launch_pw_c<true, false>(a, total_ctas, chunks, st);
    return greeks ? launch_pw_c<false, true>(a, total_ctas, chunks, st)
                  : launch_pw_c<false, false>(a, total_ctas, chunks, st);
}

cudaError_t launch_finalize(const KArgs &a, cudaStream_t st) {
    const int n = a.jobs ? a.n_jobs : 1;
    if (n <= 0) return cudaSuccess;
    finalize_kernel<<<n, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_patch_inputs(Job *jobs, int n, const int32_t *idx, const double *S0, const double *sigma,
                                cudaStream_t st) {
    if (n <= 0 || (!S0 && !sigma)) return cudaSuccess;
    patch_inputs_kernel<<<(n + 127) / 128, 128, 0, st>>>(jobs, n, idx, S0, sigma);
    return cudaGetLastError();
}

cudaError_t launch_scatter_results(const double *res_wave, int n, const int32_t *idx, double *res, double *price,
                                   double *delta, double *vega, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    scatter_results_kernel<<<(n + 127) / 128, 128, 0, st>>>(res_wave, n, idx, res, price, delta, vega);
    return cudaGetLastError();
}

}  // namespace amc
