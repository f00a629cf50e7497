// Mixed-precision Longstaff-Schwartz sweep for sm_103a (ref. [12]; the
// backward induction of §V), built around the per-date latency chain.
//
// One CTA of 1024 threads per SM: warps 0 and 1 are solvers, warps 2..31
// own 8 paths per thread (7680 paths per CTA, a contiguous slice of every
// date row).  Per CTA:
//   - a ring of 5 date slices in shared memory, filled by TMA bulk copies
//     (cp.async.bulk + mbarrier) up to 5 dates ahead of use, so HBM latency
//     never sits on the critical path;
//   - the in-the-money Gram moments M_k = sum y^k (y = S/K - 1) depend on
//     the paths only, so they are summed from the ring and exchanged two
//     dates before they are needed; the solver warps (alternate dates) turn
//     each date's totals into the inverse Gram matrix in FP64 (16 cofactors
//     in parallel; the degenerate-date test on the equilibrated Cholesky
//     pivots is decided from leading principal minors) while the path warps
//     work on later dates;
//   - what is left on the critical path per date: the exercise update
//     h > phi(y).beta of the previous date, CF *= e^{-r dt} and the
//     right-hand sides R_k = sum y^k CF (packed f32x2 on path pairs), a
//     warp-shuffle + double-float block sum, the cross-CTA exchange (whose
//     latency the Gram pass of a later date fills), and beta = Ginv R in
//     double-float, formed by every path warp itself.
// Cross-CTA exchange: every CTA writes its partial of each value as one
// 64-bit unit (FP32 payload, 32-bit tag = launch epoch and exchange index)
// and every CTA polls all units of that value until every tag matches, then
// adds them in a fixed order in double-float: one L2 round trip, no counter,
// and bit-identical totals in all CTAs.  Every wait (ring slots, exchange,
// solver hand-off) is bounded by %globaltimer; on expiry the CTA records
// AMC_ETIMEOUT, the others see it, and each CTA waits (bounded) for its own
// copies in flight before it returns.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "devutil.cuh"
#include "internal.h"
#include "lsm_solve.cuh"

namespace amc {

namespace {

using namespace dev;

constexpr int kT = kV2Threads;
constexpr int kWorkers = kV2Workers;
constexpr int kPPT = kV2PPT;
constexpr int kPPC = kV2PathsPerCta;
constexpr int kSlots = kV2Slots;
constexpr int kMaxCtas = 160;               // exchange gather: 5 units per lane
constexpr unsigned kFull = 0xffffffffu;

constexpr int kSolvers = 2;                 // solver warps 0 and 1 take alternate dates
constexpr int kW0 = 32 * kSolvers;          // first path thread
constexpr int kXW0 = kSolvers;              // exchange warps kXW0 .. kXW0+10

// E: float (FP32 prices) or uint16_t (binary16 moneyness, AMC_MIXED16)
template <typename E>
struct SmemV2 {
    E S[kSlots][kPPC];
    uint64_t mbar[kSlots];
    float redG[2][32][7];           // warp sums of Gram moments (Gram warps), by exchange parity
    float redR[32][4];              // warp sums of right-hand sides (path warps)
    float red[32][4];               // final sums
    float tot_hi[kXV], tot_lo[kXV]; // exchange totals (double-float)
    double gtot[3][8];              // Gram totals by date mod 3
    double ginv[3][16];             // inverse Gram matrix (FP64) by date mod 3
    float ginv_hi[3][16], ginv_lo[3][16];  // the same as double-float for the path warps
    float betaw[32][4];             // per-warp copy of beta (Greeks variant: fewer registers)
    double sA[kSolvers][16];
    double sP[kSolvers][4];
    int gdeg[3];
    int pend[kSlots];
    volatile int gtot_date[3];      // date whose Gram totals are in gtot[b]
    volatile int ginv_date[3];      // date whose inverse is in ginv*[b]
    volatile int abort;
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_work() { asm volatile("bar.sync 1, %0;" ::"n"(kWorkers) : "memory"); }
// Barrier of the path warps that also ORs a flag over them: every path
// thread gets the same answer, so all leave the loop together.
__device__ __forceinline__ bool bar_work_any(bool flag) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)flag), "n"(kWorkers)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
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
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(b))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void st_unit(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_unit(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int find_job_by_cta(const Job *__restrict__ jobs, int n_jobs, int cta) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].cta_begin <= cta) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Warp sums by transposition: 8 values (7 used) over 32 lanes in 5 exchange
// steps; lane l ends with the full sum of value (l >> 2) & 7.  Fixed
// pattern, so the result does not depend on timing.
__device__ __forceinline__ float warp_sum8(const float (&v)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float u[4], t[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = b4 ? v[k] : v[k + 4];
        u[k] = (b4 ? v[k + 4] : v[k]) + __shfl_xor_sync(kFull, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = b3 ? u[k] : u[k + 2];
        t[k] = (b3 ? u[k + 2] : u[k]) + __shfl_xor_sync(kFull, send, 8);
    }
    float r = (b2 ? t[1] : t[0]) + __shfl_xor_sync(kFull, b2 ? t[0] : t[1], 4);
    r += __shfl_xor_sync(kFull, r, 2);
    r += __shfl_xor_sync(kFull, r, 1);
    return r;
}
// Same for 4 values: lane l ends with the sum of value (l >> 3) & 3.
__device__ __forceinline__ float warp_sum4(const float (&v)[4], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8;
    float u[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = b4 ? v[k] : v[k + 2];
        u[k] = (b4 ? v[k + 2] : v[k]) + __shfl_xor_sync(kFull, send, 16);
    }
    float r = (b3 ? u[1] : u[0]) + __shfl_xor_sync(kFull, b3 ? u[0] : u[1], 8);
    r += __shfl_xor_sync(kFull, r, 4);
    r += __shfl_xor_sync(kFull, r, 2);
    r += __shfl_xor_sync(kFull, r, 1);
    return r;
}

// Double-float product of a (Ginv entry) and b (total), a.hi*b.hi exact via FMA.
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float hi = __fadd_rn(p, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, p))};
}

template <bool GREEKS, bool PUT, bool H16>
__global__ void __launch_bounds__(kT, 1) sweep_lsm_v2_kernel(const __grid_constant__ KArgs a) {
    static_assert(!(GREEKS && H16), "the Greeks variant needs the prices: FP32 paths only");
    using E = typename std::conditional<H16, uint16_t, float>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemV2<E> &sm = *reinterpret_cast<SmemV2<E> *>(smem_raw);
    const int jb = a.jobs ? find_job_by_cta(a.jobs, a.n_jobs, blockIdx.x) : 0;
    const Job &J = a.jobs ? a.jobs[jb] : a.one;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lc = blockIdx.x - J.cta_begin, G = J.n_cta;
    const int m = J.m, p = J.p, nmom = 2 * p - 1;
    const float invK = (float)J.invK, disc = (float)J.disc;
    const E *__restrict__ S = reinterpret_cast<const E *>(J.S);
    const int64_t N = J.N, ld = J.ld;
    const int64_t base = (int64_t)lc * kPPC;
    const int64_t rem = ld - base;
    const uint32_t slice_bytes = (uint32_t)(rem < kPPC ? rem : kPPC) * (uint32_t)sizeof(E);
    const int nloc = (N - base) < kPPC ? (int)(N - base) : kPPC;      // own paths below N
    uint64_t *const xch = J.xch;
    int32_t *const status = J.status;
    const uint64_t timeout_ns = a.timeout_ns;
    const uint32_t tag_hi = a.epoch << 10;
    const int inject_date = (lc == 0 && jb == 0) ? J.inject_date : 0;
    const unsigned poll_ns = a.poll_ns;

    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&sm.mbar[s], 1);
            sm.pend[s] = 0;
        }
        for (int b = 0; b < 3; ++b) {
            sm.gtot_date[b] = 0;
            sm.ginv_date[b] = 0;
        }
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();

    // ----------------------------------------------------------- solver warps
    // Warp q handles the dates d = m-1-q, m-1-q-2, ...: it waits for the
    // date's Gram totals (double-float, from an exchange two dates earlier),
    // forms them in FP64 and inverts; the path warps pick the result up when
    // they reach that date.
    if (warp < kSolvers) {
        for (int d = m - 1 - warp; d >= 1; d -= kSolvers) {
            const int b = d % 3;
            bool bail = false;
            if (sm.gtot_date[b] != d) {
                const uint64_t t0 = globaltimer();
                while (sm.gtot_date[b] != d) {
                    if (sm.abort || ld_volatile_int(status) != 0 || globaltimer() - t0 > timeout_ns) {
                        bail = true;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            bail = __any_sync(kFull, bail);
            if (bail) {
                if (lane == 0) {
                    atomicCAS(status, 0, AMC_ETIMEOUT);
                    sm.abort = 1;
                }
                return;
            }
            __threadfence_block();
            bool deg;
            const double gi = gram_inverse(sm.gtot[b], p, lane, sm.sA[warp], sm.sP[warp], deg);
            if (lane < 16) {
                sm.ginv[b][lane] = gi;
                const float hi = (float)gi;
                sm.ginv_hi[b][lane] = hi;
                sm.ginv_lo[b][lane] = (float)(gi - (double)hi);
            }
            if (lane == 0) sm.gdeg[b] = deg ? 1 : 0;
            __syncwarp();
            __threadfence_block();
            if (lane == 0) sm.ginv_date[b] = d;
        }
        return;
    }

    // ------------------------------------------------------------ path warps
    // Per-path state is held in units of K: cash flow cf, and for Greeks the
    // stopping date and y = S/K - 1 at stopping.  The ring slots hold S (or
    // the binary16 y) as copied from HBM until the Gram pass of that date
    // rewrites them in place as y for in-the-money own paths and 0 otherwise;
    // later passes then need no payoff, moneyness or validity arithmetic
    // (ITM <=> y != 0).
    // Per date all 30 path warps run the exercise and right-hand-side pass
    // and, after the post, the Gram pass of a later date over their own 8
    // paths; warps kXW0..kXW0+10 also post and gather one exchanged value
    // each.
    const int w = tid - kW0;
    // path thread w owns the pairs 2w, 2w+1 (+ 2 * 960 i, i = 0..3) of the
    // CTA's slice: one 8-byte shared-memory access and packed f32x2
    // arithmetic per pair
    auto pidx = [&](int i) { return 2 * w + (i & 1) + (i >> 1) * (2 * kWorkers); };
    auto issue = [&](int d) {            // w == 0 only
        const int s = d % kSlots;
        fence_proxy_async();
        mbar_expect(&sm.mbar[s], slice_bytes);
        bulk_load(sm.S[s], S + (int64_t)(d - 1) * ld + base, slice_bytes, &sm.mbar[s]);
        sm.pend[s] = d;
    };
    // The bounded waits on the ring slots and the inverse read %globaltimer
    // only once they have to wait: the read takes hundreds of cycles, and
    // most of these waits find their condition already met.
    auto wait_slice = [&](int d) -> bool {
        const int s = d % kSlots;
        const uint32_t parity = (uint32_t)((m - d) / kSlots) & 1u;
        if (!mbar_test(&sm.mbar[s], parity)) {
            const uint64_t t0 = globaltimer();
            while (!mbar_test(&sm.mbar[s], parity)) {
                if (sm.abort || globaltimer() - t0 > timeout_ns) {
                    atomicCAS(status, 0, AMC_ETIMEOUT);
                    sm.abort = 1;
                    return false;
                }
            }
        }
        if (w == 0) sm.pend[s] = 0;
        return true;
    };
    // Gram pass of date d over the own paths: y in place, in-the-money
    // moments summed over the warp into sm.redG[buf][warp][k]
    auto gram_post = [&](int d, int buf) {
        // the in-the-money indicator I = sat(-y 2^100) (put) or sat(y 2^100)
        // (call) is exactly 1 for a nonzero FP32 y of the money's sign
        // (|y| >= 2^-48) and 0 otherwise, so y I is the in-place value and I
        // the count (multiplies instead of compares and selects).  Path
        // pairs: y I, y^2 and y^3 in packed f32x2, the moments summed path
        // by path in FP32 (the same sums as one path at a time); paths at or
        // beyond nloc (last CTA) take 0 by selects
        float g[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = 0.f;
        E *sl = sm.S[d % kSlots];
        const float big = PUT ? -0x1p100f : 0x1p100f;
        auto pair = [&](int idx, bool tail) {
            const f2 Yr = raw_y2(sl, idx, invK);
            float in[2] = {__saturatef(f2_lo(Yr) * big), __saturatef(f2_hi(Yr) * big)};
            f2 Y;
            if (tail) {
                const bool v0 = idx < nloc, v1 = idx + 1 < nloc;
                in[0] = v0 ? in[0] : 0.f;
                in[1] = v1 ? in[1] : 0.f;
                Y = f2_pack(v0 ? f2_lo(Yr) * in[0] : 0.f, v1 ? f2_hi(Yr) * in[1] : 0.f);
            } else {
                Y = f2_mul(Yr, f2_pack(in[0], in[1]));
            }
            put_y2(sl, idx, Y);
            const f2 YY = f2_mul(Y, Y), Y3 = f2_mul(YY, Y);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float y = h ? f2_hi(Y) : f2_lo(Y), yy = h ? f2_hi(YY) : f2_lo(YY), y3 = h ? f2_hi(Y3) : f2_lo(Y3);
                g[0] += in[h];
                g[1] += y;
                g[2] += yy;
                g[3] += y3;
                g[4] = fmaf(yy, yy, g[4]);
                g[5] = fmaf(yy, y3, g[5]);
                g[6] = fmaf(y3, y3, g[6]);
            }
        };
#pragma unroll
        for (int i = 0; i < kPPT; i += 2) pair(pidx(i), nloc < kPPC);
        fence_proxy_async();             // these generic writes precede a later TMA refill
        const float r = warp_sum8(g, lane);
        const int k = (lane >> 2) & 7;
        if ((lane & 3) == 0 && k < nmom) sm.redG[buf][warp][k] = r;
    };

    if (!GREEKS && J.coef && lc == 0 && warp == kXW0 && lane < kCoefStride)   // maturity: no exercise decision
        J.coef[(size_t)(m - 1) * kCoefStride + lane] = lane == 4 ? 1.0 : 0.0;
    if (w == 0)
        for (int d = m; d >= 1 && d > m - kSlots; --d) issue(d);

    float cf[kPPT];
    uint32_t tau2[GREEKS ? kPPT / 2 : 1];    // stopping dates, two 16-bit halves per word
    float yt[GREEKS ? kPPT : 1];
    int degenerate = 0;
    const bool ok = wait_slice(m);
    if (ok) {
        const E *sl = sm.S[m % kSlots];
#pragma unroll
        for (int i = 0; i < kPPT; ++i) {
            const int idx = pidx(i);
            const float y = raw_y(sl, idx, invK);
            const float h = PUT ? -y : y;
            cf[i] = (idx < nloc && h > 0.f) ? h : 0.f;
            if (GREEKS) {
                if ((i & 1) == 0) tau2[i >> 1] = (uint32_t)m * 0x10001u;
                yt[i] = y;
            }
        }
    }
    bool stop = bar_work_any(!ok || sm.abort);
    if (w == 0 && m - kSlots >= 1 && !stop) issue(m - kSlots);
    // Gram moments of date m-1, posted at the first exchange (index m+1)
    if (m >= 2 && !stop && wait_slice(m - 1)) gram_post(m - 1, (m + 1) & 1);

    // exercise at date d with the coefficients b0..b3
    // (packed f32x2 pairs; the Greeks variant, which also carries the
    // stopping date and moneyness per path, stays scalar for its registers)
    auto exercise = [&](int d, float b0, float b1, float b2, float b3) {
        const E *sl = sm.S[d % kSlots];
        if (GREEKS) {
#pragma unroll
            for (int i = 0; i < kPPT; ++i) {
                const float y = y_at(sl, pidx(i));
                const float cont = fmaf(fmaf(fmaf(b3, y, b2), y, b1), y, b0);
                const float h = PUT ? -y : y;
                const bool ex = (PUT ? y < 0.f : y > 0.f) && h > cont;
                cf[i] = ex ? h : cf[i];
                if (ex) tau2[i >> 1] = (i & 1) ? ((tau2[i >> 1] & 0xffffu) | ((uint32_t)d << 16))
                                               : ((tau2[i >> 1] & 0xffff0000u) | (uint32_t)d);
                yt[i] = ex ? y : yt[i];
            }
            return;
        }
        // with y in place (0 off the money), "in the money and h > c(y)" is
        // h > max(c(y), 0), h = -y (put) or y (call)
        const f2 B0 = f2_splat(b0), B1 = f2_splat(b1), B2 = f2_splat(b2), B3 = f2_splat(b3);
        const f2 SG = f2_splat(PUT ? -1.f : 1.f);
#pragma unroll
        for (int i = 0; i < kPPT; i += 2) {
            const f2 Y = y2_at(sl, pidx(i));
            const f2 C = f2_fma(f2_fma(f2_fma(B3, Y, B2), Y, B1), Y, B0);
            const f2 H = f2_mul(Y, SG);
            const float hl = f2_lo(H), hh = f2_hi(H);
            cf[i] = hl > fmaxf(f2_lo(C), 0.f) ? hl : cf[i];
            cf[i + 1] = hh > fmaxf(f2_hi(C), 0.f) ? hh : cf[i + 1];
        }
    };

    // coefficients of the latest exchange and their degenerate flag, formed
    // by every path warp itself from the shared totals and inverse
    float bet[GREEKS ? 1 : 4] = {};
    int deg_cur = 0;
    if (GREEKS && lane < 4) sm.betaw[warp][lane] = 0.f;
    auto beta_k = [&](int k) { return GREEKS ? sm.betaw[warp][k] : bet[GREEKS ? 0 : k]; };
    for (int j = m + 1; j >= 1 && !stop; --j) {
        const bool hasR = j <= m - 1;
        const bool hasG = j - 2 >= 1;
        if (hasR) {
            // exercise at j+1 (coefficients of the previous exchange), then
            // discount to t_j and sum the right-hand sides of date j
            if (j + 1 <= m - 1) {
                if (deg_cur) {
                    if (w == 0) ++degenerate;
                } else {
                    exercise(j + 1, beta_k(0), beta_k(1), beta_k(2), beta_k(3));
                }
            }
            float rr[4] = {0.f, 0.f, 0.f, 0.f};
            const E *sl = sm.S[j % kSlots];
            if (GREEKS) {
#pragma unroll
                for (int i = 0; i < kPPT; ++i) {
                    cf[i] *= disc;
                    const float y = y_at(sl, pidx(i));
                    const float c = y != 0.f ? cf[i] : 0.f;
                    const float yy = y * y;
                    rr[0] += c;
                    rr[1] = fmaf(c, y, rr[1]);
                    rr[2] = fmaf(c, yy, rr[2]);
                    rr[3] = fmaf(c, yy * y, rr[3]);
                }
            } else {
                const f2 z2 = f2_splat(0.f), DISC = f2_splat(disc);
                f2 R0 = z2, R1 = z2, R2 = z2, R3 = z2;
#pragma unroll
                for (int i = 0; i < kPPT; i += 2) {
                    const f2 Y = y2_at(sl, pidx(i));
                    const f2 C = f2_mul(f2_pack(cf[i], cf[i + 1]), DISC);
                    cf[i] = f2_lo(C);
                    cf[i + 1] = f2_hi(C);
                    const float big = PUT ? -0x1p100f : 0x1p100f;          // in-the-money indicator, as in the Gram pass
                    R0 = f2_fma(C, f2_pack(__saturatef(f2_lo(Y) * big), __saturatef(f2_hi(Y) * big)), R0);
                    const f2 YY = f2_mul(Y, Y);
                    R1 = f2_fma(C, Y, R1);                        // y = 0 off the money
                    R2 = f2_fma(C, YY, R2);
                    R3 = f2_fma(C, f2_mul(YY, Y), R3);
                }
                rr[0] = f2_lo(R0) + f2_hi(R0);
                rr[1] = f2_lo(R1) + f2_hi(R1);
                rr[2] = f2_lo(R2) + f2_hi(R2);
                rr[3] = f2_lo(R3) + f2_hi(R3);
            }
            const float r = warp_sum4(rr, lane);
            const int k = (lane >> 3) & 3;
            if ((lane & 7) == 0 && k < p) sm.redR[warp][k] = r;
        }
        const uint32_t mask = (hasG ? ((1u << nmom) - 1u) : 0u) | (hasR ? (((1u << p) - 1u) << 7) : 0u);
        stop = bar_work_any(sm.abort);                            // B1
        if (stop) break;
        if (w == 0 && j + 1 <= m - 1 && j + 1 - kSlots >= 1) issue(j + 1 - kSlots);   // slice j+1 consumed
        // cross-CTA exchange: warp kXW0+k owns value slot k; it posts the
        // CTA's partial (an FP32 butterfly over the path warps' sums: few
        // instructions, since the other warps start the Gram pass at the
        // same time), runs its share of the next Gram pass (which also
        // absorbs the other CTAs' lag), then gathers.  The right-hand sides
        // are gathered from this exchange; the Gram moments one exchange
        // later, from the units posted at the previous date, which are in
        // place by then, so the barrier after the gather waits only for the
        // right-hand sides (the solver warps still get one date to invert)
        const int xk = warp - kXW0;
        const bool xw = xk >= 0 && xk < kXV && ((mask >> xk) & 1u);
        uint64_t *xu = xch + ((size_t)j * kXV + (xw ? xk : 0)) * G;
        if (xw) {
            float pv = 0.f;
            if (xk < 7) pv = lane < 32 - kXW0 ? sm.redG[j & 1][kXW0 + lane][xk] : 0.f;
            else pv = lane < 32 - kXW0 ? sm.redR[kXW0 + lane][xk - 7] : 0.f;
#pragma unroll
            for (int off = 16; off; off >>= 1) pv += __shfl_xor_sync(kFull, pv, off);
            if (lane == 0 && inject_date != j)
                st_unit(xu + lc, ((uint64_t)(tag_hi | (uint32_t)j) << 32) | __float_as_uint(pv));
        }
        // Gram pass of date j-3, posted at the next exchange
        if (j - 3 >= 1 && !sm.abort && wait_slice(j - 3)) gram_post(j - 3, (j - 1) & 1);
        // the Gram moments of date j-1, posted at exchange j+1
        const bool gw = xk >= 0 && xk < nmom && j + 1 <= m + 1 && j - 1 >= 1;
        if (xw && xk >= 7 || gw) {
            const int jx = xk < 7 ? j + 1 : j;
            const uint32_t tag = tag_hi | (uint32_t)jx;
            uint64_t *xg = xch + ((size_t)jx * kXV + xk) * G;
            float vals[kMaxCtas / 32];
            // the clock is read before the first poll: its latency also delays
            // that poll, and polling earlier only adds loaded L2 round trips
            const uint64_t t0 = globaltimer();
            for (;;) {
                bool good = true;
#pragma unroll
                for (int q = 0; q < kMaxCtas / 32; ++q) {
                    const int c = lane + 32 * q;
                    if (c < G) {
                        const uint64_t u = ld_unit(xg + c);
                        if ((uint32_t)(u >> 32) != tag) good = false;
                        vals[q] = __uint_as_float((uint32_t)u);
                    }
                }
                if (__all_sync(kFull, good)) break;
                bool bail = sm.abort || ld_volatile_int(status) != 0 || globaltimer() - t0 > timeout_ns;
                if (__any_sync(kFull, bail)) {
                    if (lane == 0) {
                        atomicCAS(status, 0, AMC_ETIMEOUT);
                        sm.abort = 1;
                    }
                    break;
                }
                __nanosleep(poll_ns);    // back off: all CTAs poll the same lines
            }
            dfl acc = {0.f, 0.f};
#pragma unroll
            for (int q = 0; q < kMaxCtas / 32; ++q)
                if (lane + 32 * q < G) acc = df_add(acc, dfl{vals[q], 0.f});
            acc = df_warp_sum(acc);
            if (lane == 0) {
                sm.tot_hi[xk] = acc.hi;
                sm.tot_lo[xk] = acc.lo;
            }
        }
        stop = bar_work_any(sm.abort);                            // B2
        if (stop) break;
        if (j + 1 <= m + 1 && j - 1 >= 1 && warp == kXW0 + 1 && lane < 7) {   // Gram totals of date j-1 -> solver
            const int b = (j - 1) % 3;
            sm.gtot[b][lane] = (double)sm.tot_hi[lane] + (double)sm.tot_lo[lane];
            __syncwarp(0x7fu);
            __threadfence_block();
            if (lane == 0) sm.gtot_date[b] = j - 1;
        }
        if (hasR) {
            // beta_j = Ginv_j R_j in double-float, in every path warp: lane
            // 4k+l one product, two butterfly steps, then beta_k from lane 4k
            const int b = j % 3;
            bool bail = false;
            if (sm.ginv_date[b] != j) {
                const uint64_t t0 = globaltimer();
                while (sm.ginv_date[b] != j) {
                    if (sm.abort || globaltimer() - t0 > timeout_ns) {
                        bail = true;
                        break;
                    }
                }
            }
            if (__any_sync(kFull, bail)) {
                if (lane == 0) {
                    atomicCAS(status, 0, AMC_ETIMEOUT);
                    sm.abort = 1;
                }
            } else {
                __threadfence_block();
                const int bl = lane & 3;
                dfl t = {0.f, 0.f};
                if (lane < 16 && bl < p)
                    t = df_mul(dfl{sm.ginv_hi[b][lane & 15], sm.ginv_lo[b][lane & 15]},
                               dfl{sm.tot_hi[7 + bl], sm.tot_lo[7 + bl]});
                t = df_add(t, df_shfl_xor(t, 1));
                t = df_add(t, df_shfl_xor(t, 2));
                const float bk = __fadd_rn(t.hi, t.lo);
                if (!GREEKS && J.coef && lc == 0 && warp == kXW0) {   // fitted boundary of date j (units of K)
                    const float ck = __shfl_sync(kFull, bk, 4 * (lane & 3));
                    const int dg = sm.gdeg[b];
                    if (lane < 4) J.coef[(size_t)(j - 1) * kCoefStride + lane] = dg ? 0.0 : (double)ck;
                    if (lane == 4) J.coef[(size_t)(j - 1) * kCoefStride + 4] = dg ? 1.0 : 0.0;
                }
                if (GREEKS) {
                    if (lane < 16 && bl == 0) sm.betaw[warp][lane >> 2] = bk;
                    __syncwarp();
                } else {
#pragma unroll
                    for (int k = 0; k < (GREEKS ? 1 : 4); ++k) bet[k] = __shfl_sync(kFull, bk, 4 * k);
                }
                deg_cur = sm.gdeg[b];
            }
        }
    }
    // the last exercise date, t_1 (a failed wait for its coefficients shows in sm.abort)
    if (!stop) stop = bar_work_any(sm.abort);
    if (!stop && m >= 2) {
        if (deg_cur) {
            if (w == 0) ++degenerate;
        } else {
            exercise(1, beta_k(0), beta_k(1), beta_k(2), beta_k(3));
        }
    }

    if (stop) {
        // bounded wait for this CTA's own copies still in flight, then leave
        if (w == 0) {
            for (int s = 0; s < kSlots; ++s) {
                const int d = sm.pend[s];
                if (d <= 0) continue;
                const uint32_t parity = (uint32_t)((m - d) / kSlots) & 1u;
                const uint64_t t0 = globaltimer();
                while (!mbar_test(&sm.mbar[s], parity) && globaltimer() - t0 < timeout_ns) {
                }
            }
        }
        return;
    }

    // final per-CTA sums (units of K): CF, CF^2, delta, vega; discounting to
    // 0 happens in finalize
    float fs[4] = {0.f, 0.f, 0.f, 0.f};
    const float Kf = (float)J.K;
    const float S0 = (float)J.S0, r = (float)J.r, sig = (float)J.sigma, dt = (float)J.dt;
    const float mu = r - 0.5f * sig * sig;
#pragma unroll
    for (int i = 0; i < kPPT; ++i) {
        if (pidx(i) >= nloc) continue;
        fs[0] += cf[i];
        fs[1] += cf[i] * cf[i];
        if (GREEKS && cf[i] > 0.f) {
            const float St = Kf * (1.f + yt[i]);
            const float t = (float)((tau2[i >> 1] >> (16 * (i & 1))) & 0xffffu) * dt;
            const float dfac = expf(-r * t);
            const float dh = PUT ? -1.f : 1.f;
            const float Wt = (logf(St / S0) - mu * t) / sig;
            fs[2] += dfac * dh * St / S0;
            fs[3] += dfac * dh * St * (Wt - sig * t);
        }
    }
    {
        const float rsum = warp_sum4(fs, lane);
        const int k = (lane >> 3) & 3;
        if ((lane & 7) == 0) sm.red[warp][k] = rsum;
    }
    bar_work();
    if (warp >= kXW0 && warp < kXW0 + 4) {
        const int k = warp - kXW0;
        dfl part = {lane < 32 - kXW0 ? sm.red[kXW0 + lane][k] : 0.f, 0.f};
        part = df_warp_sum(part);
        const double scale = k == 0 ? J.K : (k == 1 ? J.K * J.K : 1.0);
        if (lane == 0)
            reinterpret_cast<double *>(J.fin)[(int64_t)lc * 4 + k] = scale * ((double)part.hi + (double)part.lo);
    }
    if (lc == 0 && w == 0) J.res[4] = (double)degenerate;
}

}  // namespace

cudaError_t launch_sweep_lsm_v2(const KArgs &a, int total_ctas, bool greeks, cudaStream_t st) {
    const bool put = (a.jobs ? a.jobs_type : a.one.type) == AMC_PUT;
    if (greeks && a.h16) return cudaErrorInvalidValue;
    const void *f;
    if (a.h16)
        f = put ? (const void *)sweep_lsm_v2_kernel<false, true, true> : (const void *)sweep_lsm_v2_kernel<false, false, true>;
    else if (greeks)
        f = put ? (const void *)sweep_lsm_v2_kernel<true, true, false> : (const void *)sweep_lsm_v2_kernel<true, false, false>;
    else
        f = put ? (const void *)sweep_lsm_v2_kernel<false, true, false> : (const void *)sweep_lsm_v2_kernel<false, false, false>;
    const int smem = (int)(a.h16 ? sizeof(SmemV2<uint16_t>) : sizeof(SmemV2<float>));
    cudaError_t e = ensure_smem(f, (size_t)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel(f, dim3((unsigned)total_ctas), dim3(kT), args, (size_t)smem, st);
}

}  // namespace amc
