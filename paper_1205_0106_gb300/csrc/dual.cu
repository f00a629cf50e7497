// Dual upper bound of a fitted exercise boundary (the dual formulation of
// §IV, ref. [11]; the Andersen-Broadie martingale built from the boundary).
//
// For outer path i and exercise date t_j, Q_j(i) estimates the value at t_j
// of continuing under the boundary: n_in inner paths start from S_j(i),
// step by the exact GBM increment of Eq. 9, and stop at the first date
// d > j where the boundary exercises (always at d = m); Q_j is the mean of
// e^{-r (t_d - t_j)} h(S_d).  With D_j = e^{-r t_j}, Z_j = D_j h(S_j) and
// L_j = Z_j where the boundary exercises at t_j, D_j Q_j elsewhere (L_m = Z_m),
// the martingale M_j = sum_{l<=j} (L_l - D_{l-1} Q_{l-1}) (D_0 Q_0 = L0, the
// mean of L_1 over the outer paths) gives U(i) = max_j (Z_j - M_j), whose
// mean is an upper bound on the Bermudan value.
//
// Inner normals come from a counter-based generator: inner path k started
// at date j on outer path i owns the H = ceil(m/2) SplitMix64 outputs
// ((i m + j - 1) n_in + k) H + 1 .. + H of inner_seed; steps 2q-1 and 2q
// take the high and the low 32 bits of the q-th as uniforms (x + 1/2) 2^-32,
// mapped by the inverse normal.  A loop trip draws one output and takes up
// to two steps, so every lane calls the generator on every trip.
//
// dual_inner_kernel: one CTA per outer path.  Warps take dates in snake
// order (most work first) and run their inner paths as a queue shared
// by the warp's lanes (a lane whose path stops takes the next path at once,
// across the boundary between two dates); per-lane sums (FP32 in mixed precision) meet in an FP64
// warp tree, and paths go to lanes in an order fixed by the data, so Q_j does not depend on timing.  One
// thread then forms L_1 and V(i) = max_j (Z_j - (M_j + L0)), so that
// U(i) = L0 + V(i).
// dual_final_kernel: one CTA reduces L_1 to L0 and V to the mean and the
// standard error, in a fixed order, and adds up the inner steps taken.
#include <cuda_runtime.h>
#include <math.h>

#include "devutil.cuh"
#include "icdf.cuh"
#include "internal.h"

namespace amc {

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;   // SplitMix64 increment

// SplitMix64 output for the state z (already advanced).
__device__ __forceinline__ uint64_t splitmix_out(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <bool FP64>
struct DualReal;
template <>
struct DualReal<false> {
    using T = float;
};
template <>
struct DualReal<true> {
    using T = double;
};

// Shared memory of dual_inner_kernel for m dates: coefficients cf[m][4]
// (units of K, the kernel's precision), S_j as double, Q_j, the start of the
// inner walk (log(S_j/K) in FP32, S_j in FP64), degenerate flags, then
// (8-byte aligned) the CTA's count of inner steps.
template <bool FP64>
__host__ __device__ constexpr size_t dual_steps_offset(int m) {
    return ((size_t)m * (4 * sizeof(typename DualReal<FP64>::T) + 2 * sizeof(double) +
                         sizeof(typename DualReal<FP64>::T) + sizeof(int32_t)) + 7) & ~(size_t)7;
}
template <bool FP64>
__host__ __device__ constexpr size_t dual_smem_bytes(int m) {
    return dual_steps_offset<FP64>(m) + sizeof(unsigned long long);
}

// One step of an inner path: S (FP64) or log(S/K) (FP32) moves to date d by
// the normal zn; returns whether the path stops at d (the boundary
// exercises, or d = m) and h(S_d) / K in hk.
template <bool FP64, bool PUT>
__device__ __forceinline__ bool inner_step(typename DualReal<FP64>::T &x, typename DualReal<FP64>::T zn, int d, int m,
                                           typename DualReal<FP64>::T drift, typename DualReal<FP64>::T vol,
                                           double K, typename DualReal<FP64>::T invK,
                                           const typename DualReal<FP64>::T *__restrict__ cf,
                                           const int32_t *__restrict__ deg, typename DualReal<FP64>::T &hk) {
    bool stop = d >= m;
    if constexpr (FP64) {
        x = x * exp(drift + vol * zn);
        hk = (PUT ? K - x : x - K) * invK;
        if (!stop && hk > 0.0 && !deg[d - 1]) {
            const double y = x * invK - 1.0;
            const double *c = cf + 4 * (d - 1);
            stop = hk > fma(fma(fma(c[3], y, c[2]), y, c[1]), y, c[0]);
        }
    } else {
        x += fmaf(vol, zn, drift);                  // log(S_d / K)
        const float sk = expf(x);
        hk = PUT ? 1.f - sk : sk - 1.f;
        if (!stop && hk > 0.f && !deg[d - 1]) {
            const float y = sk - 1.f;
            const float4 c = reinterpret_cast<const float4 *>(cf)[d - 1];
            stop = hk > fmaf(fmaf(fmaf(c.w, y, c.z), y, c.y), y, c.x);
        }
    }
    return stop;
}

// Date of round r for warp w of W in snake order (1..W, 2W..W+1, 2W+1..),
// m once the dates 1..m-1 are used up.  Rounds hand out dates in
// decreasing work order, so the warps' totals stay close.
__device__ __forceinline__ int snake_date(int r, int w, int W, int m) {
    const int j = 1 + r * W + ((r & 1) ? W - 1 - w : w);
    return j < m ? j : m;
}

// Idle lanes a warp collects before it hands out paths again (or every
// lane is idle): the hand-out is a divergent stretch of code, so it runs
// for several lanes at once.
constexpr int kRefill = 4;

// The inner simulations of one warp.  The warp holds a window of two dates
// A and B (its next two dates in snake order) and hands their inner paths,
// A's n_in then B's n_in, to its idle lanes, a few lanes at a time, so a
// lane whose path stops soon takes the next path of the window.  A lane
// adds each stopped payoff to its sum for A or for B (FP32 sums of a few
// payoffs per lane under AMC_MIXED, FP64 under AMC_FP64); when every path
// of A has stopped, the lanes' sums for A are added in FP64 in a fixed tree
// into Q_A, B becomes A and the warp's next date becomes B.  Which lane
// runs a path does not change its value, and the warp's schedule is a
// function of its own dates' paths only, so Q (sums included) is the same
// on every run.
template <bool FP64, bool PUT>
__device__ __forceinline__ void warp_dates(const DualArgs &a, int64_t i, int lane, int warp, int n_warps,
                                           const typename DualReal<FP64>::T *__restrict__ cf,
                                           const int32_t *__restrict__ deg,
                                           const typename DualReal<FP64>::T *__restrict__ start,
                                           double *__restrict__ sQ, int64_t &steps) {
    using Real = typename DualReal<FP64>::T;
    const unsigned full = 0xffffffffu, lt = (1u << lane) - 1u;
    const Job &J = a.one;
    const int m = J.m;
    const int n_in = (int)a.n_in;
    const Real drift = (Real)((J.r - 0.5 * J.sigma * J.sigma) * J.dt);
    const Real vol = (Real)(J.sigma * sqrt(J.dt));
    const Real rdt = (Real)(J.r * J.dt);
    const Real invK = (Real)J.invK;
    const uint64_t H = ((uint64_t)m + 1ull) / 2ull;                       // outputs per inner path
    const uint64_t mG = H * kGolden;
    // SplitMix64 state of the first output of inner path k from date j:
    // seed + (((i m + j - 1) n_in + k) H + 1) golden = z0(j) + k H golden
    auto z0 = [&](int j) -> uint64_t {
        const uint64_t base = ((uint64_t)i * (uint64_t)m + (uint64_t)(j - 1)) * (uint64_t)n_in;
        return a.seed_in + (base * H + 1ull) * kGolden;
    };
    int round = 0;
    int jA = snake_date(round++, warp, n_warps, m), jB = snake_date(round++, warp, n_warps, m);
    int endA = jA < m ? n_in : 0, endB = endA + (jB < m ? n_in : 0), nxt = 0;   // window [0, endB)
    uint64_t zA = z0(jA), zB = z0(jB);
    bool active = false, inB = false;
    int jl = 0, s = 0;
    Real x = (Real)0, accA = (Real)0, accB = (Real)0;
    uint64_t z = 0;
    for (;;) {
        if (active) {
            // one generator output: the normals of the next two steps
            const uint64_t out = splitmix_out(z);
            z += kGolden;
            const uint32_t u1 = (uint32_t)(out >> 32), u2 = (uint32_t)out;
            Real zn1, zn2;
            if constexpr (FP64) {
                zn1 = normcdfinv(((double)u1 + 0.5) * 0x1p-32);
            } else {
                icdf_u32x2(u1, u2, zn1, zn2);
            }
            Real hk;
            ++s;
            bool stop = inner_step<FP64, PUT>(x, zn1, jl + s, m, drift, vol, J.K, invK, cf, deg, hk);
            if (!stop) {
                if constexpr (FP64) zn2 = normcdfinv(((double)u2 + 0.5) * 0x1p-32);
                ++s;
                stop = inner_step<FP64, PUT>(x, zn2, jl + s, m, drift, vol, J.K, invK, cf, deg, hk);
            }
            if (stop) {
                Real v = (Real)0;
                if (hk > (Real)0) {
                    if constexpr (FP64) v = hk * exp(-rdt * s);
                    else v = hk * expf(-rdt * (float)s);
                }
                if (inB) accB += v;
                else accA += v;
                steps += s;
                active = false;
            }
        }
        const unsigned busy = __ballot_sync(full, active);
        if (__popc(busy) > 32 - kRefill && busy != 0u) continue;
        if (nxt < endB) {
            if (!active) {
                const int it = nxt + __popc(~busy & lt);
                if (it < endB) {
                    active = true;
                    inB = it >= endA;
                    jl = inB ? jB : jA;
                    z = (inB ? zB : zA) + (uint64_t)(inB ? it - endA : it) * mG;
                    x = start[jl - 1];
                    s = 0;
                }
            }
            nxt = min(nxt + 32 - __popc(busy), endB);
        }
        if (nxt >= endA && !__any_sync(full, active && !inB)) {
            // every path of A has stopped
            if (jA < m) {
                double t = (double)accA;
#pragma unroll
                for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(full, t, off);
                if (lane == 0) sQ[jA - 1] = J.K * t / (double)n_in;
            }
            if (jB >= m) break;
            accA = accB;
            accB = (Real)0;
            inB = false;
            nxt -= endA;
            endA = endB - endA;
            jA = jB;
            zA = zB;
            jB = snake_date(round++, warp, n_warps, m);
            zB = z0(jB);
            endB = endA + (jB < m ? n_in : 0);
        }
    }
}

template <bool FP64, bool PUT>
__global__ void __launch_bounds__(kDualThreads) dual_inner_kernel(const __grid_constant__ DualArgs a) {
    using Real = typename DualReal<FP64>::T;
    const Job &J = a.one;
    const int m = J.m;
    const int64_t i = blockIdx.x;
    extern __shared__ __align__(16) unsigned char dsm[];
    Real *cf = reinterpret_cast<Real *>(dsm);                                // [m][4]
    double *sS = reinterpret_cast<double *>(dsm + (size_t)m * 4 * sizeof(Real));
    double *sQ = sS + m;                                                     // Q_j at [j-1]
    Real *start = reinterpret_cast<Real *>(sQ + m);
    int32_t *deg = reinterpret_cast<int32_t *>(start + m);
    unsigned long long *nsteps = reinterpret_cast<unsigned long long *>(dsm + dual_steps_offset<FP64>(m));
    const Real *S = reinterpret_cast<const Real *>(J.S);
    for (int d = threadIdx.x; d < m; d += blockDim.x) {
        const double *c = J.coef + (size_t)d * kCoefStride;
#pragma unroll
        for (int q = 0; q < 4; ++q) cf[4 * d + q] = (Real)c[q];
        deg[d] = c[4] != 0.0;
        const double s = (double)S[(int64_t)d * J.ld + i];
        sS[d] = s;
        sQ[d] = 0.0;
        start[d] = FP64 ? (Real)s : (Real)log(s * J.invK);
    }
    if (threadIdx.x == 0) *nsteps = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int64_t steps = 0;
    warp_dates<FP64, PUT>(a, i, lane, threadIdx.x >> 5, blockDim.x >> 5, cf, deg, start, sQ, steps);
#pragma unroll
    for (int off = 16; off; off >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, off);
    if (lane == 0) atomicAdd(nsteps, (unsigned long long)steps);
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double K = J.K, disc = J.disc;
    double Dj = 1.0, Mp = 0.0, prevDQ = 0.0, best = -INFINITY, L1 = 0.0;
    for (int d = 1; d <= m; ++d) {
        Dj *= disc;
        const double s = sS[d - 1];
        const double h = PUT ? K - s : s - K;
        const double Z = Dj * fmax(h, 0.0);
        double L, DQ = 0.0;
        if (d == m) {
            L = Z;
        } else {
            DQ = Dj * sQ[d - 1];
            bool stop = false;
            if (!deg[d - 1] && h > 0.0) {
                const double *c = J.coef + (size_t)(d - 1) * kCoefStride;
                const double y = s * J.invK - 1.0;
                stop = h > K * fma(fma(fma(c[3], y, c[2]), y, c[1]), y, c[0]);
            }
            L = stop ? Z : DQ;
        }
        if (d == 1) L1 = L;
        Mp += L - prevDQ;
        prevDQ = DQ;
        best = fmax(best, Z - Mp);
    }
    a.L1[i] = L1;
    a.V[i] = best;
    a.W[i] = (double)*nsteps;
}

// Fixed-order sum over the block (1024 threads).
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(kDualFinalThreads) dual_final_kernel(const __grid_constant__ DualArgs a) {
    __shared__ double red[kDualFinalThreads / 32];
    __shared__ double bc[2];
    const Job &J = a.one;
    const int64_t N = J.N;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += a.L1[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) bc[0] = s / (double)N;
    s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += a.V[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) bc[1] = s / (double)N;
    __syncthreads();
    const double L0 = bc[0], meanV = bc[1];
    s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = a.V[i];
        s += (v - meanV) * (v - meanV);
        if (a.U) a.U[i] = L0 + v;
    }
    s = block_sum(s, red);
    double w = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) w += a.W[i];
    w = block_sum(w, red);
    if (threadIdx.x == 0) {
        int ndeg = 0;
        for (int d = 0; d < J.m - 1; ++d) ndeg += J.coef[(size_t)d * kCoefStride + 4] != 0.0;
        J.res[0] = L0 + meanV;
        J.res[1] = N > 1 ? sqrt(s / (double)(N - 1)) / sqrt((double)N) : 0.0;
        J.res[2] = 0.0;
        J.res[3] = 0.0;
        J.res[4] = (double)ndeg;
        J.res[5] = (double)*J.status;
        J.res[6] = L0;
        J.res[7] = w;
    }
}

}  // namespace

size_t dual_smem(int m, bool fp64) { return fp64 ? dual_smem_bytes<true>(m) : dual_smem_bytes<false>(m); }

cudaError_t launch_dual_upper(const DualArgs &a, bool fp64, cudaStream_t st) {
    const Job &J = a.one;
    if (J.N <= 0) return cudaSuccess;
    const bool put = J.type == AMC_PUT;
    const void *f = fp64 ? (put ? (const void *)dual_inner_kernel<true, true> : (const void *)dual_inner_kernel<true, false>)
                         : (put ? (const void *)dual_inner_kernel<false, true>
                                : (const void *)dual_inner_kernel<false, false>);
    const int warps = J.m - 1 < kDualThreads / 32 ? (J.m - 1 > 0 ? J.m - 1 : 1) : kDualThreads / 32;
    void *args[] = {(void *)&a};
    cudaError_t e = cudaLaunchKernel(f, dim3((unsigned)J.N), dim3(32 * warps), args, dual_smem(J.m, fp64), st);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel((const void *)dual_final_kernel, dim3(1), dim3(kDualFinalThreads), args, 0, st);
}

}  // namespace amc
