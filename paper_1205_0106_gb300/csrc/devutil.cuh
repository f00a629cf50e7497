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

// IEEE binary16 storage: two values in one 32-bit word, the element at the
// lower address in the low half.  Widening is exact; narrowing rounds to
// nearest even.
__device__ __forceinline__ float h_to_f(uint16_t h) {
    float f;
    asm("{.reg .b16 t;\n\tmov.b16 t, %1;\n\tcvt.f32.f16 %0, t;}" : "=f"(f) : "h"(h));
    return f;
}
__device__ __forceinline__ f2 h2_to_f2(uint32_t w) {
    float lo, hi;
    asm("{.reg .b16 a, b;\n\tmov.b32 {a, b}, %2;\n\tcvt.f32.f16 %0, a;\n\tcvt.f32.f16 %1, b;}"
        : "=f"(lo), "=f"(hi)
        : "r"(w));
    return f2_pack(lo, hi);
}
__device__ __forceinline__ uint32_t f_to_h2(float lo, float hi) {
    uint32_t w;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));   // first operand -> upper half
    return w;
}

// One date slice of the path array in shared memory, as the mixed LSM
// sweeps hold it: FP32 prices S, or binary16 moneyness y = S/K - 1.  The
// Gram pass of a date rewrites the slice in place as y for in-the-money
// paths and 0 otherwise; the raw_* reads come before that pass, the y*
// reads after it.  A binary16 slice takes the rewritten values exactly
// (each is a stored value or 0).
__device__ __forceinline__ float raw_y(const float *sl, int i, float invK) { return fmaf(sl[i], invK, -1.f); }
__device__ __forceinline__ float raw_y(const uint16_t *sl, int i, float) { return h_to_f(sl[i]); }
__device__ __forceinline__ f2 raw_y2(const float *sl, int i, float invK) {
    return f2_fma(*reinterpret_cast<const f2 *>(sl + i), f2_splat(invK), f2_splat(-1.f));
}
__device__ __forceinline__ f2 raw_y2(const uint16_t *sl, int i, float) {
    return h2_to_f2(*reinterpret_cast<const uint32_t *>(sl + i));
}
__device__ __forceinline__ float y_at(const float *sl, int i) { return sl[i]; }
__device__ __forceinline__ float y_at(const uint16_t *sl, int i) { return h_to_f(sl[i]); }
__device__ __forceinline__ f2 y2_at(const float *sl, int i) { return *reinterpret_cast<const f2 *>(sl + i); }
__device__ __forceinline__ f2 y2_at(const uint16_t *sl, int i) {
    return h2_to_f2(*reinterpret_cast<const uint32_t *>(sl + i));
}
__device__ __forceinline__ void put_y2(float *sl, int i, f2 v) { *reinterpret_cast<f2 *>(sl + i) = v; }
__device__ __forceinline__ void put_y2(uint16_t *sl, int i, f2 v) {
    *reinterpret_cast<uint32_t *>(sl + i) = f_to_h2(f2_lo(v), f2_hi(v));
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
