// FP32 inverse cumulative normal of a 32-bit uniform integer x, at the
// point u = (x + 1/2) 2^-32 (shared by path generation and the inner
// simulations of the dual upper bound).
#pragma once

#include <stdint.h>

#include "devutil.cuh"

namespace amc {
namespace {

// Inverse cumulative normal in FP32.  Two-region form of M. Giles
// (GPU Computing Gems, 2010) applied to the normal quantile, with this
// project's own coefficients (Chebyshev least-squares fit to the exact
// quantile, fit_icdf.py; worst relative error of the float evaluation
// 2.9e-7 over the whole 32-bit uniform grid):
//   y = u - 1/2 from the signed offset x - 2^31 (no rounding at 0 or 1),
//   |y| < 0.4983 (99.66 % of points): z = y A(w - 2.5), w = -log(1 - 4y^2),
//   otherwise: z = y B(sqrt(w) - 3), w = -log(4p(1-p)), p = min(u, 1-u)
//   taken from x or its complement so the tail keeps full precision.
// One logarithm per point and almost no divergence inside a warp, where the
// paper's Moro formula needs a division in the centre and two logarithms in
// the tails.
__device__ __forceinline__ float lg2_approx(float v) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float ex2_approx(float v) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Central region: straight-line code, valid when |u - 1/2| < 0.4983.
__device__ __forceinline__ float icdf_central(float y) {
    const float wc = fmaf(-0.693147181f, lg2_approx(fmaf(-4.f * y, y, 1.f)), -2.5f);
    float a = -2.471926130e-08f;
    a = fmaf(a, wc, 6.586265044e-08f);
    a = fmaf(a, wc, 1.316422299e-06f);
    a = fmaf(a, wc, -9.795854567e-06f);
    a = fmaf(a, wc, -1.402823636e-05f);
    a = fmaf(a, wc, 6.175783346e-04f);
    a = fmaf(a, wc, -3.543307772e-03f);
    a = fmaf(a, wc, -1.181544270e-02f);
    a = fmaf(a, wc, 6.976040602e-01f);
    a = fmaf(a, wc, 4.246626854e+00f);
    return y * a;
}
// The same for two points in packed f32x2 arithmetic (identical rounding).
__device__ __forceinline__ dev::f2 icdf_central2(dev::f2 y) {
    using namespace dev;
    const f2 t = f2_fma(f2_mul(y, f2_splat(-4.f)), y, f2_splat(1.f));
    const f2 l = f2_pack(lg2_approx(f2_lo(t)), lg2_approx(f2_hi(t)));
    const f2 wc = f2_fma(f2_splat(-0.693147181f), l, f2_splat(-2.5f));
    f2 a = f2_splat(-2.471926130e-08f);
    a = f2_fma(a, wc, f2_splat(6.586265044e-08f));
    a = f2_fma(a, wc, f2_splat(1.316422299e-06f));
    a = f2_fma(a, wc, f2_splat(-9.795854567e-06f));
    a = f2_fma(a, wc, f2_splat(-1.402823636e-05f));
    a = f2_fma(a, wc, f2_splat(6.175783346e-04f));
    a = f2_fma(a, wc, f2_splat(-3.543307772e-03f));
    a = f2_fma(a, wc, f2_splat(-1.181544270e-02f));
    a = f2_fma(a, wc, f2_splat(6.976040602e-01f));
    a = f2_fma(a, wc, f2_splat(4.246626854e+00f));
    return f2_mul(y, a);
}
// Tails: p = min(u, 1-u) from x or its complement.
__device__ __noinline__ float icdf_tail(uint32_t x, float y) {
    const uint32_t xs = (x & 0x80000000u) ? ~x : x;
    const float p = fmaf((float)xs, 0x1p-32f, 0x1p-33f);
    const float sc = sqrtf(-0.693147181f * lg2_approx(fmaf(-4.f * p, p, 4.f * p))) - 3.f;
    float b = 9.611179121e-05f;
    b = fmaf(b, sc, -3.932459513e-04f);
    b = fmaf(b, sc, -1.151860997e-04f);
    b = fmaf(b, sc, 3.614928108e-03f);
    b = fmaf(b, sc, -1.002847217e-02f);
    b = fmaf(b, sc, 1.631816290e-02f);
    b = fmaf(b, sc, -2.166599594e-02f);
    b = fmaf(b, sc, 2.668302692e-02f);
    b = fmaf(b, sc, 2.833170176e+00f);
    b = fmaf(b, sc, 8.012868881e+00f);
    return y * b;
}
__device__ __forceinline__ float icdf_y(uint32_t x) {            // u - 1/2 from the signed offset
    return fmaf((float)(int32_t)(x ^ 0x80000000u), 0x1p-32f, 0x1p-33f);
}
// z = Phi^-1((x + 1/2) 2^-32) for two integers at once: the central form
// in packed f32x2 arithmetic, then the tail for whichever lies outside it.
__device__ __forceinline__ void icdf_u32x2(uint32_t x0, uint32_t x1, float &z0, float &z1) {
    using namespace dev;
    const f2 y = f2_pack(icdf_y(x0), icdf_y(x1));
    const f2 zc = icdf_central2(y);
    z0 = f2_lo(zc);
    z1 = f2_hi(zc);
    if (!(fabsf(f2_lo(y)) < 0.4983f)) z0 = icdf_tail(x0, f2_lo(y));
    if (!(fabsf(f2_hi(y)) < 0.4983f)) z1 = icdf_tail(x1, f2_hi(y));
}

}  // namespace
}  // namespace amc
