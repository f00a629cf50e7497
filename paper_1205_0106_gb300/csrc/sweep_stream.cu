// Longstaff-Schwartz backward sweep (ref. [12], the backward induction of
// §V) for options whose per-path state does not fit on chip: the cash flows
// live in device memory and every exercise date is one streaming pass plus
// one small solve, so any path count runs (the register-resident sweeps
// need all their CTAs resident at once, which caps them near 1.2 M paths).
//
//   pass(j), j = m-1 .. 1 (grid-stride over groups of 4 consecutive paths,
//   16-byte row loads):
//     j = m-1: CF = h(S_m) / K; otherwise CF is read, and the paths that the
//       boundary of date j+1 exercises (not degenerate, in the money,
//       h > c_{j+1}(y)) take CF = h(S_{j+1}) / K;
//     CF <- e^{-r dt} CF, written back;
//     the in-the-money moments sum y^k (k = 0..2p-2) and right-hand sides
//       sum y^k CF (k < p) of date j, y = S_j / K - 1, per thread in
//       compensated FP32 (two sums per packed f32x2 register pair), then
//       double-float (FP32 pairs) through the warp
//       and CTA trees into the CTA's partial row (FP64 throughout under
//       AMC_FP64: this GPU's FP64 pipe is slow enough that a tree of
//       doubles would cost more than the pass's memory traffic);
//   solve(j) (one CTA): the partial rows added in a fixed order (double-
//     float, then FP64), the inverse of the Gram matrix by cofactors over
//     one warp, beta_j or the degenerate flag (fewer than p paths in the
//     money, or an equilibrated Cholesky pivot <= 1e-12, decided from the
//     leading principal minors), and the boundary row;
//   final pass: the exercise of date 1 (or CF = h(S_1) / K when m = 1), then
//     per-CTA FP64 sums of CF and CF^2 for finalize_kernel, which applies the
//     last e^{-r dt}.
// Traffic per path and date: S_j and S_{j+1} read, CF read and written
// (16 bytes in FP32; 12 when the path array holds binary16 moneyness).  Deterministic: fixed grid, fixed path ranges, fixed
// reduction order.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "devutil.cuh"
#include "internal.h"
#include "lsm_solve.cuh"

namespace amc {

namespace {

template <bool FP64>
struct ST;
template <>
struct ST<false> {
    using Real = float;
};
template <>
struct ST<true> {
    using Real = double;
};

// Plain cached loads: a pass touches rows S_j and S_{j+1} and the cash
// flows, and the previous pass touched two of the three, so at sizes whose
// working set fits the L2 (126 MB) those come from the L2.
__device__ __forceinline__ void ld4(const float *p, float *o) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double *o) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
// y = S/K - 1 of 4 consecutive paths from a row of the path array: FP32 or
// FP64 prices, or binary16 moneyness (AMC_MIXED16), widened exactly.
__device__ __forceinline__ void ldy4(const float *p, float invK, float *y) {
    ld4(p, y);
#pragma unroll
    for (int e = 0; e < 4; ++e) y[e] = fmaf(y[e], invK, -1.f);
}
__device__ __forceinline__ void ldy4(const double *p, double invK, double *y) {
    ld4(p, y);
#pragma unroll
    for (int e = 0; e < 4; ++e) y[e] = fma(y[e], invK, -1.0);
}
__device__ __forceinline__ void ldy4(const uint16_t *p, float, float *y) {
    const uint2 w = *reinterpret_cast<const uint2 *>(p);
    const dev::f2 a = dev::h2_to_f2(w.x), b = dev::h2_to_f2(w.y);
    y[0] = dev::f2_lo(a); y[1] = dev::f2_hi(a); y[2] = dev::f2_lo(b); y[3] = dev::f2_hi(b);
}
// Programmatic dependent launch: the passes and solves are launched so that
// the next kernel of the stream may start once every CTA of the current
// one has signalled (at its start), and each waits in griddepcontrol.wait,
// until the previous kernel has completed and its writes are visible,
// before it reads what that kernel wrote.  The wait is the hardware's own:
// it ends when the previous grid ends.  Launched without the attribute
// both instructions do nothing.
__device__ __forceinline__ void pdl_signal() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void st4(float *p, const float *v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double *v) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// Fixed-order FP64 sum of NV values over the CTA (kStreamThreads threads);
// thread 0 holds the totals.
template <int NV>
__device__ __forceinline__ void block_sum_d(double (&v)[NV], double (*red)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int w = 0; w < kStreamThreads / 32; ++w) t += red[w][k];
            v[k] = t;
        }
}

// Compensated accumulation (Kahan; FP32 adds that FMA contraction cannot
// merge).  In FP64 a plain sum.
template <bool FP64>
struct Acc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ dev::dfl get_df() const { return dev::df_add({s, 0.f}, {-c, 0.f}); }
};
template <>
struct Acc<true> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double get() const { return s; }
};

// Two of the compensated FP32 accumulators above in one packed register
// pair: add/sub.rn.f32x2 take the two lanes' round-to-nearest steps in one
// issue slot, the same steps in the same order as the scalar sum.  The
// totals are not always bit-identical to the scalar loop's: on a 2^22-path,
// 252-date put the price moves by 0.9e-6 K (the powers y^5 of paths within
// about 3e-8 of the strike are subnormal, the likely source).
__device__ __forceinline__ dev::f2 f2_sub(dev::f2 a, dev::f2 b) {
    dev::f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
struct Acc2 {
    dev::f2 s{0ull}, c{0ull};
    __device__ __forceinline__ void add(dev::f2 v) {
        const dev::f2 y = f2_sub(v, c);
        const dev::f2 t = dev::f2_add(s, y);
        c = f2_sub(f2_sub(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void unpack(Acc<false> &lo, Acc<false> &hi) const {
        lo.s = dev::f2_lo(s); lo.c = dev::f2_lo(c);
        hi.s = dev::f2_hi(s); hi.c = dev::f2_hi(c);
    }
};

// Per-thread sums of one pass, accumulator k = moment k (k < 7) or right-
// hand side k - 7.  FP64: one double each.  FP32: the 11 compensated sums
// as packed pairs (M0,M1) (M2,M3) (M4,M5) (R0,R1) (R2,R3) and M6 alone, the
// powers y^k formed one product at a time as in the scalar loop.  A pair
// with one slot the basis uses also fills the other (M1 for p = 1, M3 for
// p <= 2, M5 and R3 for p = 3); no solve reads those slots.
template <bool FP64>
struct PathSums {
    Acc<true> a[kNV];
    __device__ __forceinline__ void add_path(double y, double v, int p) {
        double pw = 1.0;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            if (k < 2 * p - 1) a[k].add(pw);
            if (k < p) a[7 + k].add(pw * v);
            pw *= y;
        }
    }
    __device__ __forceinline__ void add_final(double v) {
        a[0].add(v);
        a[1].add(v * v);
    }
    __device__ __forceinline__ void get(Acc<true> (&o)[kNV]) const {
#pragma unroll
        for (int k = 0; k < kNV; ++k) o[k] = a[k];
    }
};
template <>
struct PathSums<false> {
    Acc2 m01, m23, m45, r01, r23;
    Acc<false> m6;
    __device__ __forceinline__ void add_path(float y, float v, int p) {
        const float y2 = y * y, y3 = y2 * y;
        const dev::f2 p01 = dev::f2_pack(1.f, y), p23 = dev::f2_pack(y2, y3);
        const dev::f2 V = dev::f2_splat(v);
        m01.add(p01);
        r01.add(dev::f2_mul(p01, V));
        if (p >= 2) m23.add(p23);
        if (p >= 3) {
            const float y4 = y3 * y, y5 = y4 * y;
            m45.add(dev::f2_pack(y4, y5));
            r23.add(dev::f2_mul(p23, V));
            if (p >= 4) m6.add(y5 * y);
        }
    }
    __device__ __forceinline__ void add_final(float v) { m01.add(dev::f2_pack(v, v * v)); }
    __device__ __forceinline__ void get(Acc<false> (&o)[kNV]) const {
        m01.unpack(o[0], o[1]);
        m23.unpack(o[2], o[3]);
        m45.unpack(o[4], o[5]);
        o[6] = m6;
        r01.unpack(o[7], o[8]);
        r23.unpack(o[9], o[10]);
        o[11] = Acc<false>();
    }
};

// Per-CTA totals of the kNV accumulators.  FP32 path: double-float through
// the warp and the CTA (the FP64 pipe of this GPU is slow; a tree of
// doubles here costs more than the pass's memory traffic), thread k ending
// with total k; FP64 path: doubles, all totals in thread 0.  Fixed order in
// both.
struct DfRed {
    dev::dfl w[kStreamThreads / 32][kNV];
};
struct DRed {
    double w[kStreamThreads / 32][kNV];
};

// Fixed-order warp sums of 16 double-float values by a transposed
// butterfly: at offsets 16, 8, 4 and 2 each lane keeps half of its values
// (the upper half where the offset bit of its index is set) and adds the
// partner's copy of that half, so a lane exchanges 8 + 4 + 2 + 1 values
// instead of 5 per value; offset 1 is an ordinary butterfly step.  Lane l
// ends with the warp's sum of value (l >> 1) & 15.
__device__ __forceinline__ dev::dfl df_warp_sum16(dev::dfl (&v)[16], int lane) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const int off = 2 * h;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const dev::dfl send = up ? v[i] : v[i + h];
            const dev::dfl keep = up ? v[i + h] : v[i];
            v[i] = dev::df_add(keep, dev::df_shfl_xor(send, off));
        }
    }
    return dev::df_add(v[0], dev::df_shfl_xor(v[0], 1));
}

// CTA total of value k (k < kNV) in thread k from one double-float per
// value and thread: the warp sums above, then the warps' sums in warp order.
__device__ __forceinline__ dev::dfl cta_total_df(dev::dfl (&v)[16], DfRed &red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const dev::dfl s = df_warp_sum16(v, lane);
    const int k = lane >> 1;
    if ((lane & 1) == 0 && k < kNV) red.w[warp][k] = s;
    __syncthreads();
    dev::dfl t = {0.f, 0.f};
    if (threadIdx.x < kNV) {
        t = red.w[0][threadIdx.x];
        for (int w = 1; w < kStreamThreads / 32; ++w) t = dev::df_add(t, red.w[w][threadIdx.x]);
    }
    return t;
}
__device__ __forceinline__ void cta_totals(Acc<true> (&acc)[kNV], DRed &red, double (&tot)[kNV]) {
    double v[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) v[k] = acc[k].get();
    block_sum_d<kNV>(v, red.w);
#pragma unroll
    for (int k = 0; k < kNV; ++k) tot[k] = v[k];
}
__device__ __forceinline__ double to_d(dev::dfl x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ double to_d(double x) { return x; }


// One exercise date: j = 1 .. m-1 sums the moments of date j; j = 0 is the
// final pass (exercise of date 1, sums of CF).  H16: the path array holds
// binary16 moneyness (12 instead of 16 bytes per path and date).
template <bool FP64, bool PUT, bool H16>
__global__ void __launch_bounds__(kStreamThreads, (FP64 || H16) ? 3 : 4) lsm_stream_pass(const __grid_constant__ StreamArgs a, int j) {
    static_assert(!(FP64 && H16), "binary16 moneyness is an FP32-path format");
    using Real = typename ST<FP64>::Real;
    using Elem = typename std::conditional<H16, uint16_t, Real>::type;
    using Red = typename std::conditional<FP64, DRed, DfRed>::type;
    using Tot = typename std::conditional<FP64, double, dev::dfl>::type;
    __shared__ Red red;
    pdl_signal();
    pdl_wait();                                             // the cash flows, beta and flags of the last kernels
    const Job &J = a.one;
    const int m = J.m, p = J.p;
    const int64_t N = J.N, ld = J.ld;
    const Elem *__restrict__ S = reinterpret_cast<const Elem *>(J.S);
    Real *__restrict__ cf = reinterpret_cast<Real *>(a.cf);
    const Real invK = (Real)J.invK, disc = (Real)J.disc;
    // exercise boundary of date j+1 (row j), unless the pass starts at maturity
    const int ed = j + 1;                                   // date whose boundary this pass applies
    const bool init = (j == m - 1) || (m == 1);
    const bool exer = !init && ed <= m - 1 && !a.deg[ed - 1];
    Real c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    if (exer) {
        c0 = (Real)a.beta[(ed - 1) * 4 + 0];
        c1 = (Real)a.beta[(ed - 1) * 4 + 1];
        c2 = (Real)a.beta[(ed - 1) * 4 + 2];
        c3 = (Real)a.beta[(ed - 1) * 4 + 3];
    }
    PathSums<FP64> sums;
    const int64_t groups = (N + 3) / 4;
#pragma unroll 2
    for (int64_t g = (int64_t)blockIdx.x * kStreamThreads + threadIdx.x; g < groups;
         g += (int64_t)gridDim.x * kStreamThreads) {
        const int64_t i0 = 4 * g;
        Real v[4], ye[4], yj[4];
        if (j >= 1) ldy4(S + (int64_t)(j - 1) * ld + i0, invK, yj);   // date j, issued with the other rows
        if (init) {
            ldy4(S + (int64_t)(m - 1) * ld + i0, invK, ye);          // maturity
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const Real y = ye[e];
                const Real h = PUT ? -y : y;
                v[e] = h > Real(0) ? h : Real(0);
            }
        } else {
            ld4(cf + i0, v);
            if (exer) {
                ldy4(S + (int64_t)(ed - 1) * ld + i0, invK, ye);   // date j+1
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const Real y = ye[e];
                    const Real h = PUT ? -y : y;
                    const Real cont = fma(fma(fma(c3, y, c2), y, c1), y, c0);
                    if ((PUT ? y < Real(0) : y > Real(0)) && h > cont) v[e] = h;
                }
            }
        }
        if (j >= 1) {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] *= disc;
            st4(cf + i0, v);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (i0 + e >= N) continue;
                const Real y = yj[e];
                if (!(PUT ? y < Real(0) : y > Real(0))) continue;      // in the money, strictly
                sums.add_path(y, v[e], p);
            }
        } else {
            // final pass: the cash flow at t_1 (finalize applies the last discount)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (i0 + e >= N) continue;
                sums.add_final(v[e]);
            }
        }
    }
    Acc<FP64> acc[kNV];
    sums.get(acc);
    Tot *row = reinterpret_cast<Tot *>(a.part) + (int64_t)blockIdx.x * kNV;
    double *fin = reinterpret_cast<double *>(J.fin) + (int64_t)blockIdx.x * 4;
    if constexpr (FP64) {
        Tot tot[kNV];
        cta_totals(acc, red, tot);
        if (threadIdx.x == 0) {
            if (j >= 1) {
#pragma unroll
                for (int k = 0; k < kNV; ++k) row[k] = tot[k];
            } else {
                fin[0] = J.K * to_d(tot[0]);
                fin[1] = J.K * J.K * to_d(tot[1]);
                fin[2] = 0.0;
                fin[3] = 0.0;
                if (blockIdx.x == 0) J.res[4] = (double)*a.ndeg;
            }
        }
    } else {
        dev::dfl v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = k < kNV ? acc[k].get_df() : dev::dfl{0.f, 0.f};
        const dev::dfl t = cta_total_df(v, red);
        const int k = threadIdx.x;
        if (j >= 1) {
            if (k < kNV) row[k] = t;
        } else if (k < 4) {
            fin[k] = k == 0 ? J.K * to_d(t) : (k == 1 ? J.K * J.K * to_d(t) : 0.0);
            if (blockIdx.x == 0 && k == 0) J.res[4] = (double)*a.ndeg;
        }
    }
}

// Solve of date j from the partial rows: fixed-order sums (thread t adds
// rows t, t + kStreamThreads, ..; double-float, or FP64 under AMC_FP64), a
// fixed tree, then warp 0.
template <bool FP64>
__global__ void __launch_bounds__(kStreamThreads) lsm_stream_solve(const __grid_constant__ StreamArgs a, int j) {
    pdl_signal();
    pdl_wait();                                             // the pass's partial rows
    const Job &J = a.one;
    const int p = J.p;
    __shared__ double sM[kNV], sA[16], sP[4];
    if constexpr (FP64) {
        __shared__ double red[kStreamThreads / 32][kNV];
        double tot[kNV];
#pragma unroll
        for (int k = 0; k < kNV; ++k) tot[k] = 0.0;
        for (int c = threadIdx.x; c < a.grid; c += kStreamThreads) {
            const double *row = a.part + (int64_t)c * kNV;
#pragma unroll
            for (int k = 0; k < kNV; ++k) tot[k] += row[k];
        }
        block_sum_d<kNV>(tot, red);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < kNV; ++k) sM[k] = tot[k];
    } else {
        __shared__ DfRed red;
        dev::dfl t[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) t[k] = {0.f, 0.f};
        for (int c = threadIdx.x; c < a.grid; c += kStreamThreads) {
            const dev::dfl *row = reinterpret_cast<const dev::dfl *>(a.part) + (int64_t)c * kNV;
#pragma unroll
            for (int k = 0; k < kNV; ++k) t[k] = dev::df_add(t[k], row[k]);
        }
        const dev::dfl u = cta_total_df(t, red);
        if (threadIdx.x < kNV) sM[threadIdx.x] = to_d(u);
    }
    __syncthreads();
    // the inverse of the Gram matrix by cofactors over warp 0 (FP64 chains a
    // few operations deep: this GPU's FP64 latency makes a one-thread
    // Cholesky the longest step of a date), then beta_k = sum_l Ginv_kl R_l
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    bool degen = false;
    const double inv = gram_inverse(sM, p, lane, sA, sP, degen);
    double t = (lane < 16 && (lane & 3) < p) ? inv * sM[7 + (lane & 3)] : 0.0;   // R_l, l >= p: unread
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    double beta[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) beta[k] = __shfl_sync(0xffffffffu, t, 4 * k);
    if (lane != 0) return;
    const bool ok = !degen;
    a.deg[j - 1] = ok ? 0 : 1;
    if (!ok) *a.ndeg += 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) a.beta[(j - 1) * 4 + k] = ok ? beta[k] : 0.0;
    if (J.coef) {
        double *c = J.coef + (size_t)(j - 1) * kCoefStride;
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = ok ? beta[k] : 0.0;
        c[4] = ok ? 0.0 : 1.0;
        if (j == J.m - 1) {                                 // maturity: no exercise decision
            double *cm = J.coef + (size_t)(J.m - 1) * kCoefStride;
            cm[0] = cm[1] = cm[2] = cm[3] = 0.0;
            cm[4] = 1.0;
        }
    }
}

__global__ void lsm_stream_coef_m1(const __grid_constant__ StreamArgs a) {
    // m = 1: only the maturity row of the boundary
    if (threadIdx.x == 0 && a.one.coef) {
        double *cm = a.one.coef;
        cm[0] = cm[1] = cm[2] = cm[3] = 0.0;
        cm[4] = 1.0;
    }
}

}  // namespace

namespace {
using PassFn = void (*)(StreamArgs, int);
PassFn pass_fn(bool fp64, bool put, bool h16) {
    if (h16) return put ? lsm_stream_pass<false, true, true> : lsm_stream_pass<false, false, true>;
    return fp64 ? (put ? lsm_stream_pass<true, true, false> : lsm_stream_pass<true, false, false>)
                : (put ? lsm_stream_pass<false, true, false> : lsm_stream_pass<false, false, false>);
}
}  // namespace

// As many CTAs as fit on the SMs at once.
int64_t stream_grid(int sm_count, bool fp64, bool put, bool h16) {
    int per = 0;
    if (ctas_per_sm((const void *)pass_fn(fp64 && !h16, put, h16), kStreamThreads, 0, &per) != cudaSuccess || per < 1)
        per = 1;
    return (int64_t)per * sm_count;
}

cudaError_t launch_lsm_stream(const StreamArgs &a, bool fp64, cudaStream_t st) {
    const Job &J = a.one;
    if (fp64 && a.h16) return cudaErrorInvalidValue;
    const PassFn pass = pass_fn(fp64, J.type == AMC_PUT, a.h16 != 0);
    void (*solve)(StreamArgs, int) = fp64 ? lsm_stream_solve<true> : lsm_stream_solve<false>;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cp = {}, cs = {};
    cp.gridDim = dim3((unsigned)a.grid);
    cp.blockDim = dim3(kStreamThreads);
    cp.stream = st;
    cp.attrs = attr;
    cp.numAttrs = 1;
    cs = cp;
    cs.gridDim = dim3(1);
    cudaError_t e = cudaSuccess;
    if (J.m == 1) {
        lsm_stream_coef_m1<<<1, 32, 0, st>>>(a);
    } else {
        for (int j = J.m - 1; j >= 1 && e == cudaSuccess; --j) {
            e = cudaLaunchKernelEx(&cp, pass, a, j);
            if (e == cudaSuccess) e = cudaLaunchKernelEx(&cs, solve, a, j);
        }
    }
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cp, pass, a, 0);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace amc
