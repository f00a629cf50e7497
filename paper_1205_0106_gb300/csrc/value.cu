// Valuation of paths with a given exercise boundary: the second
// Longstaff-Schwartz pass (ref. [12] values out of sample; the paper's
// backward induction of §V values in sample).  The boundary is the
// continuation value c_d(y) = sum_k coef[d-1][k] y^k (units of K, moneyness
// y = S/K - 1) of each exercise date d, as fitted by an LSM sweep; on paths
// independent of the fit the price is a low-biased estimator.
//
// No per-date reduction: each path's cash flow runs back from maturity on
// its own, CF <- CF e^{-r dt}, then CF = h if the date is not degenerate and
// h > c_d(y) in the money, so the kernel is one streaming read of the
// date-major path array (4 or 8 bytes per path-step), bound by HBM.  Each
// CTA owns a contiguous slice of 2048 paths; one thread streams the slice's
// row of every date, maturity first, into a ring of shared-memory stages by
// TMA bulk copies (cp.async.bulk + one mbarrier per stage), several dates
// ahead, so the bytes in flight do not depend on registers; thread t
// evaluates paths 4t..4t+3 and 1024+4t..1024+4t+3 of the slice.  The
// arithmetic of a date (moneyness, Horner, compare, discount) is the mixed
// sweep's, so on the fitting paths the decisions are the in-sample ones.
#include <cuda_runtime.h>
#include <math.h>

#include "devutil.cuh"
#include "internal.h"

namespace amc {

namespace {

using namespace dev;

template <bool FP64>
struct VR;
template <>
struct VR<false> {
    using Real = float;
    static constexpr int kStages = 5;       // 5 x 8 KB per CTA, 4 CTAs per SM
};
template <>
struct VR<true> {
    using Real = double;
    static constexpr int kStages = 4;       // 4 x 16 KB
};

constexpr int kVP = 8 * kValueThreads;      // paths per CTA slice

template <bool FP64>
struct VSmem {
    using Real = typename VR<FP64>::Real;
    Real S[VR<FP64>::kStages][kVP];
    uint64_t full[VR<FP64>::kStages];
    int pend[VR<FP64>::kStages];
    Real c[AMC_MAX_STEPS][4];
    unsigned char deg[AMC_MAX_STEPS];
    double red[kValueThreads / 32][2];
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

template <bool FP64, bool PUT>
__global__ void __launch_bounds__(kValueThreads) value_boundary_kernel(const __grid_constant__ KArgs a) {
    using Real = typename VR<FP64>::Real;
    constexpr int kSt = VR<FP64>::kStages;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    VSmem<FP64> &sm = *reinterpret_cast<VSmem<FP64> *>(smem_raw);
    const Job &J = a.one;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = J.m, p = J.p;
    const Real invK = (Real)J.invK, disc = (Real)J.disc;
    const Real *__restrict__ S = reinterpret_cast<const Real *>(J.S);
    const int64_t N = J.N, ld = J.ld;
    const int64_t base = (int64_t)blockIdx.x * kVP;
    const int64_t rem = ld - base;
    const uint32_t slice_bytes = (uint32_t)((rem < kVP ? rem : kVP) * (int64_t)sizeof(Real));   // multiple of 128
    const int nloc = (N - base) < kVP ? (int)(N - base) : kVP;
    const uint64_t timeout_ns = a.timeout_ns;

    if (tid == 0) {
        for (int s = 0; s < kSt; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&sm.full[s])) : "memory");
            sm.pend[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int d = tid; d < m; d += kValueThreads) {
        const double *c = J.coef + (size_t)d * kCoefStride;
#pragma unroll
        for (int k = 0; k < 4; ++k) sm.c[d][k] = k < p ? (Real)c[k] : Real(0);
        sm.deg[d] = (d == m - 1 || c[4] != 0.0) ? 1 : 0;
    }
    __syncthreads();
    // date d goes to stage (m - d) mod kSt, its fill number (m - d) / kSt
    auto issue = [&](int d) {                        // tid 0 only
        const int s = (m - d) % kSt;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&sm.full[s])),
                     "r"(slice_bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                saddr(sm.S[s])),
            "l"(S + (int64_t)(d - 1) * ld + base), "r"(slice_bytes), "r"(saddr(&sm.full[s]))
            : "memory");
        sm.pend[s] = d;
    };
    if (tid == 0)
        for (int d = m; d >= 1 && d > m - kSt; --d) issue(d);

    Real cf[8];
    bool stop = false;
    const uint64_t t0 = globaltimer();
    for (int d = m; d >= 1; --d) {
        const int s = (m - d) % kSt;
        const uint32_t parity = (uint32_t)((m - d) / kSt) & 1u;
        bool late = false;
        while (!mbar_test(&sm.full[s], parity)) {
            if (globaltimer() - t0 > timeout_ns) {
                late = true;
                break;
            }
        }
        if (!late) {
            Real x[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const Real *src = sm.S[s] + 4 * tid + h * 4 * kValueThreads;
                if (FP64) {
                    const double2 u = reinterpret_cast<const double2 *>(src)[0];
                    const double2 v = reinterpret_cast<const double2 *>(src)[1];
                    x[4 * h] = (Real)u.x; x[4 * h + 1] = (Real)u.y; x[4 * h + 2] = (Real)v.x; x[4 * h + 3] = (Real)v.y;
                } else {
                    const float4 u = *reinterpret_cast<const float4 *>(src);
                    x[4 * h] = (Real)u.x; x[4 * h + 1] = (Real)u.y; x[4 * h + 2] = (Real)u.z; x[4 * h + 3] = (Real)u.w;
                }
            }
            if (d == m) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const Real y = fma(x[e], invK, Real(-1));
                    const Real h = PUT ? -y : y;
                    const int idx = 4 * tid + (e & 3) + (e >> 2) * 4 * kValueThreads;
                    cf[e] = (idx < nloc && h > Real(0)) ? h : Real(0);
                }
            } else {
                const bool deg = sm.deg[d - 1];
                const Real c0 = sm.c[d - 1][0], c1 = sm.c[d - 1][1], c2 = sm.c[d - 1][2], c3 = sm.c[d - 1][3];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    cf[e] *= disc;
                    const Real y = fma(x[e], invK, Real(-1));
                    const Real cont = fma(fma(fma(c3, y, c2), y, c1), y, c0);
                    const Real h = PUT ? -y : y;
                    const bool ex = !deg && (PUT ? y < Real(0) : y > Real(0)) && h > cont;
                    cf[e] = ex ? h : cf[e];
                }
            }
        }
        // every thread is done with stage s (and learns of a wait that ran out)
        if (__syncthreads_or(late)) {
            stop = true;
            break;
        }
        if (tid == 0) {
            sm.pend[s] = 0;
            if (d - kSt >= 1) issue(d - kSt);
        }
    }
    if (stop) {
        if (tid == 0) {
            atomicCAS(J.status, 0, AMC_ETIMEOUT);
            // bounded wait for this CTA's own copies still in flight
            for (int s = 0; s < kSt; ++s) {
                const int d = sm.pend[s];
                if (d <= 0) continue;
                const uint32_t parity = (uint32_t)((m - d) / kSt) & 1u;
                const uint64_t t1 = globaltimer();
                while (!mbar_test(&sm.full[s], parity) && globaltimer() - t1 < timeout_ns) {
                }
            }
        }
        return;
    }
    Real t0s = Real(0), t1s = Real(0);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int idx = 4 * tid + (e & 3) + (e >> 2) * 4 * kValueThreads;
        if (idx < nloc) {
            t0s += cf[e];
            t1s += cf[e] * cf[e];
        }
    }
    double acc0 = (double)t0s, acc1 = (double)t1s;
    // fixed-order block sum; per-CTA sums in currency units for finalize
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, off);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, off);
    }
    if (lane == 0) {
        sm.red[warp][0] = acc0;
        sm.red[warp][1] = acc1;
    }
    __syncthreads();
    if (tid == 0) {
        double b0 = 0.0, b1 = 0.0;
        for (int w = 0; w < kValueThreads / 32; ++w) {
            b0 += sm.red[w][0];
            b1 += sm.red[w][1];
        }
        double *fin = reinterpret_cast<double *>(J.fin) + (int64_t)blockIdx.x * 4;
        fin[0] = J.K * b0;
        fin[1] = J.K * J.K * b1;
        fin[2] = 0.0;
        fin[3] = 0.0;
        if (blockIdx.x == 0) {
            int deg = 0;
            for (int d = 0; d < m - 1; ++d) deg += sm.deg[d];
            J.res[4] = (double)deg;
        }
    }
}

}  // namespace

int64_t value_ctas(int64_t n_paths) { return (n_paths + kVP - 1) / kVP; }

cudaError_t launch_value_boundary(const KArgs &a, int ctas, bool fp64, cudaStream_t st) {
    if (ctas <= 0) return cudaSuccess;
    const bool put = a.one.type == AMC_PUT;
    const void *f = fp64 ? (put ? (const void *)value_boundary_kernel<true, true>
                                : (const void *)value_boundary_kernel<true, false>)
                         : (put ? (const void *)value_boundary_kernel<false, true>
                                : (const void *)value_boundary_kernel<false, false>);
    const int smem = fp64 ? (int)sizeof(VSmem<true>) : (int)sizeof(VSmem<false>);
    cudaError_t e = ensure_smem(f, (size_t)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(f, dim3((unsigned)ctas), dim3(kValueThreads), args, (size_t)smem, st);
}

}  // namespace amc
