// FP64 solves of the Longstaff-Schwartz normal equations of one date: an
// equilibrated Cholesky solve (one thread; the register-resident FP64 sweep)
// and the inverse by cofactors over one warp (the mixed sweep's solver warps
// and the streaming sweep).
#pragma once

#include <cuda_runtime.h>

namespace amc {
namespace {

// Equilibrated Cholesky solve of G beta = R with G_kl = M_{k+l}: scale by
// D^{-1/2}, D = diag(G); any pivot <= 1e-12 (or a non-positive diagonal)
// makes the date degenerate (false).  FP64, straight-line for a fixed basis
// size; square roots and divisions are replaced by reciprocal square roots
// (sqrt(a) = a rsqrt(a)) because FP64 division and square root are long
// instruction sequences on this part and the solve sits on the per-date
// critical path.
template <int P>
__device__ __forceinline__ bool solve_normal_t(const double *M, const double *R, double *beta) {
    double sc[P], L[P][P], il[P], y[P], g[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const double d = M[2 * k];
        if (!(d > 0.0)) return false;
        sc[k] = rsqrt(d);
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
#pragma unroll
        for (int l = 0; l <= k; ++l) {
            double a = M[k + l] * sc[k] * sc[l];
#pragma unroll
            for (int q = 0; q < l; ++q) a -= L[k][q] * L[l][q];
            if (l == k) {
                if (!(a > 1e-12)) return false;
                il[k] = rsqrt(a);
                L[k][k] = a * il[k];
            } else {
                L[k][l] = a * il[l];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
        double a = R[k] * sc[k];
#pragma unroll
        for (int q = 0; q < k; ++q) a -= L[k][q] * y[q];
        y[k] = a * il[k];
    }
#pragma unroll
    for (int k = P - 1; k >= 0; --k) {
        double a = y[k];
#pragma unroll
        for (int q = k + 1; q < P; ++q) a -= L[q][k] * g[q];
        g[k] = a * il[k];
    }
#pragma unroll
    for (int k = 0; k < P; ++k) beta[k] = g[k] * sc[k];
    return true;
}

__device__ bool solve_normal(int p, const double *M, const double *R, double *beta) {
    switch (p) {
        case 1: return solve_normal_t<1>(M, R, beta);
        case 2: return solve_normal_t<2>(M, R, beta);
        case 3: return solve_normal_t<3>(M, R, beta);
        default: return solve_normal_t<4>(M, R, beta);
    }
}

// Solver warp: inverse of the p x p Gram matrix G_kl = M_{k+l} (identity
// beyond p) as the transposed cofactor matrix over the determinant, lane
// 4k+l computing cofactor (k, l); G is symmetric, so is its inverse.  The
// matrix is first scaled by exact powers of two, A = P G P, which changes
// no rounding.  Degenerate date test: the q-th Cholesky pivot of the
// equilibrated matrix D^{-1/2} G D^{-1/2} (D = diag G) equals
//   det(G_{q+1}) / (det(G_q) G_qq)
// with G_q the leading q x q block, so "pivot <= 1e-12" is decided from
// leading principal minors (lanes 16..18) without divisions or square
// roots.  Every FP64 chain here is a handful of operations deep, against
// a long sequential chain for a Cholesky factorisation.
__device__ __forceinline__ double det3(double a00, double a01, double a02, double a10, double a11, double a12,
                                       double a20, double a21, double a22) {
    return a00 * fma(a11, a22, -a12 * a21) - a01 * fma(a10, a22, -a12 * a20) + a02 * fma(a10, a21, -a11 * a20);
}

__device__ __forceinline__ double gram_inverse(const double *M, int p, int lane, double *sA, double *sP,
                                               bool &deg) {
    // (sA, sP: this solver warp's staging area)
    // power-of-two scale factors P_k ~ 1/sqrt(M_2k) (exact), scaled matrix in shared memory
    if (lane < 4) {
        int e = 0;
        if (lane < p && M[2 * lane] > 0.0) frexp(M[2 * lane], &e);
        sP[lane] = ldexp(1.0, -(e / 2));
    }
    __syncwarp();
    if (lane < 16) {
        const int r = lane >> 2, c = lane & 3;
        sA[lane] = (r < p && c < p) ? M[r + c] * sP[r] * sP[c] : (r == c ? 1.0 : 0.0);
    }
    __syncwarp();
    const int k = (lane >> 2) & 3, l = lane & 3;
    // cofactor (k, l): rows != k, cols != l
    const int r0 = k == 0 ? 1 : 0, r1 = k <= 1 ? 2 : 1, r2 = k <= 2 ? 3 : 2;
    const int c0 = l == 0 ? 1 : 0, c1 = l <= 1 ? 2 : 1, c2 = l <= 2 ? 3 : 2;
    const double minor = det3(sA[4 * r0 + c0], sA[4 * r0 + c1], sA[4 * r0 + c2], sA[4 * r1 + c0], sA[4 * r1 + c1],
                              sA[4 * r1 + c2], sA[4 * r2 + c0], sA[4 * r2 + c1], sA[4 * r2 + c2]);
    const double cof = ((k + l) & 1) ? -minor : minor;
    // det = sum_l A[0][l] C_0l (lanes 0..3), same value in every lane
    double t = lane < 4 ? sA[lane] * cof : 0.0;
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    const double det = __shfl_sync(0xffffffffu, t, 0);
    // leading principal minors det(A_1..A_3); det(A_4) = det
    const double d1 = sA[0];
    const double d2 = fma(sA[0], sA[5], -sA[1] * sA[4]);
    const double d3 = det3(sA[0], sA[1], sA[2], sA[4], sA[5], sA[6], sA[8], sA[9], sA[10]);
    bool bad = !(M[0] >= (double)p);
    if (p >= 1 && !(d1 > 1e-12 * sA[0])) bad = true;
    if (p >= 2 && !(d2 > 1e-12 * d1 * sA[5])) bad = true;
    if (p >= 3 && !(d3 > 1e-12 * d2 * sA[10])) bad = true;
    if (p >= 4 && !(det > 1e-12 * d3 * sA[15])) bad = true;
    deg = bad;
    // 1/det: single-precision seed, two Newton steps in FP64
    double rd = (double)__frcp_rn((float)det);
    rd = rd * fma(-det, rd, 2.0);
    rd = rd * fma(-det, rd, 2.0);
    return (k < p && l < p) ? cof * rd * sP[k] * sP[l] : 0.0;
}

}  // namespace
}  // namespace amc
