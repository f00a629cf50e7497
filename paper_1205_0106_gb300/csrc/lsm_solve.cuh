// FP64 solve of the Longstaff-Schwartz normal equations of one date, shared
// by the register-resident FP64 sweep and the streaming sweep.
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

}  // namespace
}  // namespace amc
