// Valuation of paths with a given exercise boundary: the second
// Longstaff-Schwartz pass (ref. [12] values out of sample; the paper's
// backward induction of §V values in sample).  The boundary is the
// continuation value c_d(y) = sum_k coef[d-1][k] y^k (units of K, moneyness
// y = S/K - 1) of each exercise date d, as fitted by an LSM sweep; on paths
// independent of the fit the price is a low-biased estimator.
//
// No per-date reduction: each path's cash flow runs back from maturity on
// its own, CF <- CF e^{-r dt}, then CF = h if the date is not degenerate and
// h > c_d(y) > -inf in the money, so the kernel is one streaming read of the
// date-major path array (4 or 8 bytes per path-step), bound by HBM.  Thread
// t owns the 4-path quads t and t + T (T threads in the grid, grid-stride
// beyond that), read with 16-byte evict-first loads; the coefficients sit in
// shared memory.  The arithmetic of a date (moneyness, Horner, compare,
// discount) is the mixed sweep's, so on the fitting paths the decisions are
// the in-sample ones.
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
};
template <>
struct VR<true> {
    using Real = double;
};

__device__ __forceinline__ void load_quad(const float *row, int64_t i0, float (&s)[4]) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(row + i0));
    s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
}
__device__ __forceinline__ void load_quad(const double *row, int64_t i0, double (&s)[4]) {
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(row + i0));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(row + i0) + 1);
    s[0] = a.x; s[1] = a.y; s[2] = b.x; s[3] = b.y;
}

template <bool FP64, bool PUT>
__global__ void __launch_bounds__(kValueThreads) value_boundary_kernel(const __grid_constant__ KArgs a) {
    using Real = typename VR<FP64>::Real;
    __shared__ Real s_c[AMC_MAX_STEPS][4];
    __shared__ unsigned char s_deg[AMC_MAX_STEPS];
    __shared__ double s_red[kValueThreads / 32][2];
    const Job &J = a.one;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = J.m, p = J.p;
    const Real invK = (Real)J.invK, disc = (Real)J.disc;
    const Real *__restrict__ S = reinterpret_cast<const Real *>(J.S);
    const int64_t N = J.N, ld = J.ld;
    for (int d = tid; d < m; d += kValueThreads) {
        const double *c = J.coef + (size_t)d * kCoefStride;
#pragma unroll
        for (int k = 0; k < 4; ++k) s_c[d][k] = k < p ? (Real)c[k] : Real(0);
        s_deg[d] = (d == m - 1 || c[4] != 0.0) ? 1 : 0;
    }
    __syncthreads();

    const int64_t T = (int64_t)gridDim.x * kValueThreads;
    double acc0 = 0.0, acc1 = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * kValueThreads + tid; 4 * q < N; q += 2 * T) {
        const int64_t i0 = 4 * q, i1 = 4 * (q + T);
        const bool has1 = i1 < N;                       // i1 < ld whenever i1 < N (ld is a multiple of 32)
        Real cf[8], s[8];
        {
            Real u[4], v[4] = {Real(0), Real(0), Real(0), Real(0)};
            const Real *row = S + (int64_t)(m - 1) * ld;
            load_quad(row, i0, u);
            if (has1) load_quad(row, i1, v);
#pragma unroll
            for (int e = 0; e < 4; ++e) { s[e] = u[e]; s[4 + e] = v[e]; }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const Real y = fma(s[e], invK, Real(-1));
            const Real h = PUT ? -y : y;
            const bool valid = (e < 4 ? i0 + e : i1 + e - 4) < N;
            cf[e] = (valid && h > Real(0)) ? h : Real(0);
        }
#pragma unroll 2
        for (int d = m - 1; d >= 1; --d) {
            const Real *row = S + (int64_t)(d - 1) * ld;
            Real u[4], v[4] = {Real(0), Real(0), Real(0), Real(0)};
            load_quad(row, i0, u);
            if (has1) load_quad(row, i1, v);
            const bool deg = s_deg[d - 1];
            const Real c0 = s_c[d - 1][0], c1 = s_c[d - 1][1], c2 = s_c[d - 1][2], c3 = s_c[d - 1][3];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                cf[e] *= disc;
                const Real y = fma(e < 4 ? u[e] : v[e - 4], invK, Real(-1));
                const Real cont = fma(fma(fma(c3, y, c2), y, c1), y, c0);
                const Real h = PUT ? -y : y;
                const bool ex = !deg && (PUT ? y < Real(0) : y > Real(0)) && h > cont;
                cf[e] = ex ? h : cf[e];
            }
        }
        Real t0 = Real(0), t1 = Real(0);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const bool valid = (e < 4 ? i0 + e : i1 + e - 4) < N;
            if (valid) {
                t0 += cf[e];
                t1 += cf[e] * cf[e];
            }
        }
        acc0 += (double)t0;
        acc1 += (double)t1;
    }
    // fixed-order block sum; per-CTA sums in currency units for finalize
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, off);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, off);
    }
    if (lane == 0) {
        s_red[warp][0] = acc0;
        s_red[warp][1] = acc1;
    }
    __syncthreads();
    if (tid == 0) {
        double b0 = 0.0, b1 = 0.0;
        for (int w = 0; w < kValueThreads / 32; ++w) {
            b0 += s_red[w][0];
            b1 += s_red[w][1];
        }
        double *fin = reinterpret_cast<double *>(J.fin) + (int64_t)blockIdx.x * 4;
        fin[0] = J.K * b0;
        fin[1] = J.K * J.K * b1;
        fin[2] = 0.0;
        fin[3] = 0.0;
        if (blockIdx.x == 0) {
            int deg = 0;
            for (int d = 0; d < m - 1; ++d) deg += s_deg[d];
            J.res[4] = (double)deg;
        }
    }
}

}  // namespace

cudaError_t launch_value_boundary(const KArgs &a, int ctas, bool fp64, cudaStream_t st) {
    if (ctas <= 0) return cudaSuccess;
    const bool put = a.one.type == AMC_PUT;
    if (fp64) {
        if (put) value_boundary_kernel<true, true><<<ctas, kValueThreads, 0, st>>>(a);
        else value_boundary_kernel<true, false><<<ctas, kValueThreads, 0, st>>>(a);
    } else {
        if (put) value_boundary_kernel<false, true><<<ctas, kValueThreads, 0, st>>>(a);
        else value_boundary_kernel<false, false><<<ctas, kValueThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace amc
