// Device helpers shared by the sweep kernels.
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

}  // namespace dev
}  // namespace amc
