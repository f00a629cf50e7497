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
// quantile, fit_icdf.py; A of degree 7, B of degree 9; worst relative error
// of the float polynomials 4.6e-7 over the whole 32-bit uniform grid, and
// 2.4e-6 with y itself in FP32: near the edge of the central region, where
// p = 1/2 - |y| is small, the 24-bit y carries p to about 3e-8 absolute):
//   y = u - 1/2 from the signed offset x - 2^31 (no rounding at 0 or 1),
//   |y| < kIcdfY0 (99.88 % of points): z = y A(w - 3), w = -log(1 - 4y^2),
//   otherwise: z = y B(sqrt(w) - 3), w = -log(4p(1-p)), p = min(u, 1-u)
//   taken from x or its complement so the tail keeps full precision.
// One logarithm per point and almost no divergence inside a warp, where the
// paper's Moro formula needs a division in the centre and two logarithms in
// the tails.  The central region ends at w = 6: in 128 points (one warp's
// share of a bridge node) a tail point then turns up 15 % of the time.
constexpr float kIcdfY0 = 4.993799031e-01f;     // largest float below 1/2 - p(w = 6)
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

// Central region: straight-line code, valid when |u - 1/2| < kIcdfY0.
__device__ __forceinline__ float icdf_central(float y) {
    const float wc = fmaf(-0.693147181f, lg2_approx(fmaf(-4.f * y, y, 1.f)), -3.f);
    float a = 9.548626849e-07f;
    a = fmaf(a, wc, -5.553251412e-06f);
    a = fmaf(a, wc, -3.383041985e-05f);
    a = fmaf(a, wc, 5.541322753e-04f);
    a = fmaf(a, wc, -2.370398026e-03f);
    a = fmaf(a, wc, -1.623339206e-02f);
    a = fmaf(a, wc, 6.834375858e-01f);
    a = fmaf(a, wc, 4.592071056e+00f);
    return y * a;
}
// The same for two points in packed f32x2 arithmetic (identical rounding).
__device__ __forceinline__ dev::f2 icdf_central2(dev::f2 y) {
    using namespace dev;
    const f2 t = f2_fma(f2_mul(y, f2_splat(-4.f)), y, f2_splat(1.f));
    const f2 l = f2_pack(lg2_approx(f2_lo(t)), lg2_approx(f2_hi(t)));
    const f2 wc = f2_fma(f2_splat(-0.693147181f), l, f2_splat(-3.f));
    f2 a = f2_splat(9.548626849e-07f);
    a = f2_fma(a, wc, f2_splat(-5.553251412e-06f));
    a = f2_fma(a, wc, f2_splat(-3.383041985e-05f));
    a = f2_fma(a, wc, f2_splat(5.541322753e-04f));
    a = f2_fma(a, wc, f2_splat(-2.370398026e-03f));
    a = f2_fma(a, wc, f2_splat(-1.623339206e-02f));
    a = f2_fma(a, wc, f2_splat(6.834375858e-01f));
    a = f2_fma(a, wc, f2_splat(4.592071056e+00f));
    return f2_mul(y, a);
}
// Tails: p = min(u, 1-u) from x or its complement.
__device__ __noinline__ float icdf_tail(uint32_t x, float y) {
    const uint32_t xs = (x & 0x80000000u) ? ~x : x;
    const float p = fmaf((float)xs, 0x1p-32f, 0x1p-33f);
    const float sc = sqrtf(-0.693147181f * lg2_approx(fmaf(-4.f * p, p, 4.f * p))) - 3.f;
    float b = 3.474594632e-05f;
    b = fmaf(b, sc, -7.568509318e-05f);
    b = fmaf(b, sc, -6.680240040e-04f);
    b = fmaf(b, sc, 3.875148715e-03f);
    b = fmaf(b, sc, -9.793787263e-03f);
    b = fmaf(b, sc, 1.609553955e-02f);
    b = fmaf(b, sc, -2.167562954e-02f);
    b = fmaf(b, sc, 2.671968937e-02f);
    b = fmaf(b, sc, 2.833168507e+00f);
    b = fmaf(b, sc, 8.012867928e+00f);
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
    if (!(fabsf(f2_lo(y)) < kIcdfY0)) z0 = icdf_tail(x0, f2_lo(y));
    if (!(fabsf(f2_hi(y)) < kIcdfY0)) z1 = icdf_tail(x1, f2_hi(y));
}

}  // namespace
}  // namespace amc
