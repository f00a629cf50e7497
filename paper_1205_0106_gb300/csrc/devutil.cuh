// Device helpers shared by the sweep, valuation and path-generation kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amc {
namespace dev {

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

__device__ __forceinline__ dfl df_shfl_xor(dfl a, int off) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}

// Fixed-order butterfly sum of one double-float per lane (same result in
// every lane).
__device__ __forceinline__ dfl df_warp_sum(dfl a) {
#pragma unroll
    for (int off = 16; off; off >>= 1) a = df_add(a, df_shfl_xor(a, off));
    return a;
}

// Two floats in one 64-bit register for the packed FP32 instructions of
// sm_100 and later: add/mul/fma.rn.f32x2 give the two round-to-nearest
// results of the scalar instructions, in one issue slot.
struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2 f2_splat(float x) { return f2_pack(x, x); }
__device__ __forceinline__ float f2_lo(f2 a) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
    return lo;
}
__device__ __forceinline__ float f2_hi(f2 a) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
    return hi;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile_int(const int32_t *p) { return *(volatile const int32_t *)p; }

template <typename Real>
__device__ __forceinline__ Real payoff(bool put, Real s, Real K) {
    const Real h = put ? K - s : s - K;
    return h > Real(0) ? h : Real(0);
}

__device__ __forceinline__ float ncdf(float x) { return normcdff(x); }
__device__ __forceinline__ double ncdf(double x) { return normcdf(x); }

// Black-Scholes value over time tau, Eqs. 1-5 (put through Eq. 5: N(-d2), N(-d1)).
template <typename Real>
__device__ __forceinline__ Real bs_value(bool put, Real S, Real K, Real r, Real sig, Real tau) {
    const Real sq = sig * sqrt(tau);
    const Real d1 = (log(S / K) + (r + Real(0.5) * sig * sig) * tau) / sq;
    const Real d2 = d1 - sq;
    const Real dfk = K * exp(-r * tau);
    return put ? dfk * ncdf(-d2) - S * ncdf(-d1) : S * ncdf(d1) - dfk * ncdf(d2);
}

}  // namespace dev
}  // namespace amc
