// Mixed-precision Longstaff-Schwartz sweep of one option per thread-block
// cluster (ref. [12]; the backward induction of §V), for options of up to
// kClMaxCluster * kClPathsPerCta paths (2^18).
//
// The per-date regression needs every path of the option, so each date ends
// in a reduction across the option's CTAs.  Here those CTAs form one cluster
// and the reduction runs through distributed shared memory: every CTA sends
// its double-float partial of each value straight into every CTA's shared
// memory (st.async with an mbarrier transaction count), so a date's exchange
// is one on-chip round trip instead of a store to L2 and polling.  Clusters
// do not depend on one another, so the launch is an ordinary one: a batch
// of options streams through the GPU cluster by cluster.
//
// One CTA of 1024 threads per SM holds 16384 paths: warps 1..31 own 16
// paths per thread with the cash flow (units of K) in registers, plus one
// path each for the first 512 of them with its cash flow in shared memory;
// warp 0 owns none and solves.  The date slices of S stream through a ring
// of 3 slots in shared memory (64 KB each; 32 KB when the path array holds
// binary16 moneyness), filled by TMA bulk copies about one date ahead.  Per date d (from m-1 down to 1), path warps:
//   1. wait for beta_{d+1} (named barrier, published by the solver warp);
//      exercise at d+1, discount, right-hand sides R_d of date d over their
//      own paths (packed f32x2);
//   2. the CTA's double-float partials of R_d (warps 1..4) go to every CTA
//      of the cluster;
//   3. Gram pass of date d-1 over all paths (y = S/K - 1 in place for
//      in-the-money paths, 0 otherwise; the 7 Hankel moments), whose
//      partials (warps 5..11) go to every CTA as well.
// The solver warp waits for R_d from every CTA, forms beta_d = G_d^-1 R_d in
// double-float and publishes it; then it waits for the moments of date d-1
// and inverts G_{d-1} (cofactors, one Newton-Schulz step), which is off the
// critical path: the chain per date is the exercise and right-hand-side
// pass, one on-chip exchange and a 4x4 matrix-vector product.  Every CTA
// adds the peers' partials in CTA order, so all form the same totals.
// Every wait (ring slots, exchanges) is bounded by %globaltimer; on expiry
// the CTA records AMC_ETIMEOUT, stops, waits (bounded) for its own copies
// in flight, and every thread still meets the others at the closing cluster
// barrier, so no CTA leaves while a peer may write into its shared memory.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "devutil.cuh"
#include "internal.h"

namespace amc {

namespace {

using namespace dev;

constexpr int kT = kClThreads;                 // 1024
constexpr int kPPT = kClPPT;                   // 16 paths per thread
constexpr int kPPC = kClPathsPerCta;           // 16384
constexpr int kPairs = kPPC / 2;
constexpr int kSlots = 3;
constexpr int kMaxG = kClMaxCluster;           // 16
constexpr int kPathWarps = kT / 32 - 1;        // warps 1..31 hold paths; warp 0 solves
constexpr int kPathThreads = kPathWarps * 32;  // 992
constexpr int kRegPaths = kPathThreads * kPPT; // 15872 paths in registers
constexpr unsigned kFull = 0xffffffffu;
static_assert(kPPC - kRegPaths <= kPathThreads, "one shared-memory path per path thread at most");

// E: float (FP32 prices) or uint16_t (binary16 moneyness, AMC_MIXED16)
template <typename E>
struct SmemCl {
    E S[kSlots][kPPC];
    uint64_t mbar[kSlots];                     // ring slots (TMA)
    uint64_t xbarR[2];                         // exchange arrivals of the right-hand sides, by date mod 2
    uint64_t xbarM[3];                         // and of the Gram moments, by date mod 3
    float2 recvR[2][4][kMaxG];                 // per-source-CTA double-float partials
    float2 recvM[3][7][kMaxG];
    float redR[2][kPathWarps][4];              // warp partials, by date parity
    float redM[2][kPathWarps][8];
    float redF[kPathWarps][4];                 // final sums
    float cfx[kPPC - kRegPaths];               // cash flows of the paths held in shared memory
    float beta[2][4];                          // coefficients by date parity (FP32, as the path warps use them)
    int deg[2];
    int pend[kSlots];
    volatile int abort;
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Path warps only (named barrier 1): OR of a flag over them.
__device__ __forceinline__ bool bar_paths_any(bool flag) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)flag), "n"(kPathThreads)
        : "memory");
    return r != 0;
}
// Named barrier 2, producer-consumer: the solver warp arrives once per
// published beta (or abort), the path warps wait once per use.
__device__ __forceinline__ void bar_arrive_beta() { asm volatile("bar.arrive 2, %0;" ::"n"(kT) : "memory"); }
__device__ __forceinline__ void bar_sync_beta() { asm volatile("bar.sync 2, %0;" ::"n"(kT) : "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
// Wait test with cluster-scope acquire: makes the peers' st.async data (and
// this CTA's TMA data) visible to the waiting thread.
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
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
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t map_to(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
// One double-float partial into CTA `rank`'s receive slot, counted on its
// exchange mbarrier (8 bytes of transaction).
// FP32 butterfly sum of one value per lane, the same in every lane: a CTA's
// total of the path warps' partials before it is sent (on the path warps'
// critical path, where a double-float butterfly took about 300 cycles more;
// the CTAs' totals are then added in double-float)
__device__ __forceinline__ float f_warp_sum(float v) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}
__device__ __forceinline__ void send_df(uint32_t dst, uint32_t bar, float hi, float lo) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(dst),
                 "f"(hi), "f"(lo), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ------------------------------------------------------ double-float algebra
__device__ __forceinline__ dfl df_of(float x) { return {x, 0.f}; }
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
// a*b with the high product exact through an FMA.
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float hi = __fadd_rn(p, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, p))};
}
__device__ __forceinline__ dfl df_scale(dfl a, float pow2) { return {a.hi * pow2, a.lo * pow2}; }
__device__ __forceinline__ dfl df_det3(dfl a00, dfl a01, dfl a02, dfl a10, dfl a11, dfl a12, dfl a20, dfl a21,
                                       dfl a22) {
    const dfl t0 = df_sub(df_mul(a11, a22), df_mul(a12, a21));
    const dfl t1 = df_sub(df_mul(a10, a22), df_mul(a12, a20));
    const dfl t2 = df_sub(df_mul(a10, a21), df_mul(a11, a20));
    return df_add(df_sub(df_mul(a00, t0), df_mul(a01, t1)), df_mul(a02, t2));
}
__device__ __forceinline__ dfl ld_df(const float2 &v) { return {v.x, v.y}; }
__device__ __forceinline__ dfl df_shfl(dfl a, int src) {
    return {__shfl_sync(kFull, a.hi, src), __shfl_sync(kFull, a.lo, src)};
}

// Transposed warp sums (fixed pattern): 8 values -> lane l holds the sum of
// value (l >> 2) & 7; 4 values -> lane l holds value (l >> 3) & 3.
__device__ __forceinline__ float warp_sum8(const float (&v)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float u[4], t[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = (b4 ? v[k + 4] : v[k]) + __shfl_xor_sync(kFull, b4 ? v[k] : v[k + 4], 16);
#pragma unroll
    for (int k = 0; k < 2; ++k) t[k] = (b3 ? u[k + 2] : u[k]) + __shfl_xor_sync(kFull, b3 ? u[k] : u[k + 2], 8);
    float r = (b2 ? t[1] : t[0]) + __shfl_xor_sync(kFull, b2 ? t[0] : t[1], 4);
    r += __shfl_xor_sync(kFull, r, 2);
    r += __shfl_xor_sync(kFull, r, 1);
    return r;
}
__device__ __forceinline__ float warp_sum4(const float (&v)[4], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8;
    float u[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) u[k] = (b4 ? v[k + 2] : v[k]) + __shfl_xor_sync(kFull, b4 ? v[k] : v[k + 2], 16);
    float r = (b3 ? u[1] : u[0]) + __shfl_xor_sync(kFull, b3 ? u[0] : u[1], 8);
    r += __shfl_xor_sync(kFull, r, 4);
    r += __shfl_xor_sync(kFull, r, 2);
    r += __shfl_xor_sync(kFull, r, 1);
    return r;
}

// Solver warp: the inverse of the p x p Gram matrix G_kl = M_{k+l} of one
// date from its double-float totals (lane q < 7 holds M_q), identity beyond
// p.  The matrix is scaled by exact powers of two, A = P G P with
// P_k ~ 1/sqrt(M_2k); lane 4k+l forms cofactor (k, l) of A, and
// G^-1 = P (C / det) P (C symmetric).  One Newton-Schulz step
// X <- X (2I - G X) then squares the relative error of the double-float
// inverse.  Degenerate date (no exercise): M_0 < p, or a Cholesky pivot of
// the equilibrated matrix <= 1e-12; the q-th pivot equals
// det(A_{q+1}) / (det(A_q) A_qq), leading principal minors that do not
// depend on the diagonal scaling, decided on the high words.  Returns
// (G^-1)_kl in lane 4k+l (k, l < p; 0 elsewhere and in lanes >= 16).
// Totals of the 7 Gram moments over the G CTAs of the cluster from the
// received double-float partials rm[k][c]: lane 8c'+k adds sources c',
// c'+4, c'+8, c'+12, then a butterfly over c' (fixed order, the same in
// every CTA); lane k (k < 7) ends with moment k, lanes 7, 15, .. with 0.
__device__ __noinline__ dfl cl_moment_totals(const float2 (*rm)[kMaxG], int G, int lane) {
    const int k = lane & 7, c = lane >> 3;
    dfl acc = df_of(0.f);
    if (k < 7)
#pragma unroll
        for (int s = 0; s < kMaxG; s += 4)
            if (c + s < G) acc = df_add(acc, ld_df(rm[k][c + s]));
    acc = df_add(acc, df_shfl_xor(acc, 8));
    return df_add(acc, df_shfl_xor(acc, 16));
}

__device__ __noinline__ dfl cl_gram_inverse(dfl Mq, int p, int lane, bool &deg) {
    const int k = (lane >> 2) & 3, l = lane & 3;
    const dfl Mkl = df_shfl(Mq, (k + l) & 7);                 // M_{k+l} (k + l <= 6)
    float Pl = 1.f;
    {
        const dfl d = df_shfl(Mq, (2 * (lane & 3)) & 7);      // M_{2 l}
        if ((lane & 3) < p && d.hi > 0.f) {
            int e;
            frexpf(d.hi, &e);
            Pl = ldexpf(1.f, -(e / 2));
        }
    }
    const float Pk = __shfl_sync(kFull, Pl, k), Pc = __shfl_sync(kFull, Pl, l);
    const dfl Akl = (k < p && l < p) ? df_scale(Mkl, Pk * Pc) : df_of(k == l ? 1.f : 0.f);
    // lane 4r+c holds A_rc; every lane gathers the entries it needs by shuffles
    auto A = [&](int r, int c) { return df_shfl(Akl, 4 * r + c); };
    const int r0 = k == 0 ? 1 : 0, r1 = k <= 1 ? 2 : 1, r2 = k <= 2 ? 3 : 2;
    const int c0 = l == 0 ? 1 : 0, c1 = l <= 1 ? 2 : 1, c2 = l <= 2 ? 3 : 2;
    dfl cof = df_det3(A(r0, c0), A(r0, c1), A(r0, c2), A(r1, c0), A(r1, c1), A(r1, c2), A(r2, c0), A(r2, c1),
                      A(r2, c2));
    if ((k + l) & 1) cof = df_neg(cof);
    // det = sum_l A_0l C_0l (lanes 0..3), the same in every lane
    dfl t = lane < 4 ? df_mul(Akl, cof) : df_of(0.f);
    t = df_add(t, df_shfl_xor(t, 1));
    t = df_add(t, df_shfl_xor(t, 2));
    const dfl det = df_shfl(t, 0);
    const dfl d3 = df_shfl(cof, 15);                          // cofactor (3, 3) = det(A_3)
    const dfl a00 = A(0, 0), a01 = A(0, 1), a10 = A(1, 0), a11 = A(1, 1);
    const float a22 = A(2, 2).hi, a33 = A(3, 3).hi;
    const float d1 = a00.hi;
    const dfl d2 = df_sub(df_mul(a00, a11), df_mul(a01, a10));
    const dfl M0 = df_shfl(Mq, 0);
    bool bad = !(M0.hi >= (float)p);
    if (p >= 2 && !(d2.hi > 1e-12f * d1 * a11.hi)) bad = true;
    if (p >= 3 && !(d3.hi > 1e-12f * d2.hi * a22)) bad = true;
    if (p >= 4 && !(det.hi > 1e-12f * d3.hi * a33)) bad = true;
    if (!(det.hi != 0.f) || !isfinite(det.hi)) bad = true;
    deg = bad;
    if (bad) return df_of(0.f);
    dfl rd = df_of(__frcp_rn(det.hi));
#pragma unroll
    for (int it = 0; it < 2; ++it) rd = df_mul(rd, df_sub(df_of(2.f), df_mul(det, rd)));
    // X = G^-1 estimate; one Newton-Schulz step X (2I - G X) with G unscaled
    const bool in = lane < 16 && k < p && l < p;
    const dfl X = in ? df_scale(df_mul(cof, rd), Pk * Pc) : df_of(0.f);
    const dfl Gkl = in ? Mkl : df_of(0.f);
    // (G X)_kl = sum_q G_kq X_ql: the four products at once, then a pairwise
    // sum (a dependent chain of 2 additions instead of 4)
    auto matmul = [&](dfl P, dfl Q) {
        dfl t[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] = df_mul(df_shfl(P, 4 * k + q), df_shfl(Q, 4 * q + l));
        return df_add(df_add(t[0], t[1]), df_add(t[2], t[3]));
    };
    const dfl E = df_sub(df_of((k == l && k < p) ? 2.f : 0.f), matmul(Gkl, X));   // 2I - G X
    const dfl xn = matmul(X, E);
    return in ? xn : df_of(0.f);
}

// P4: the cubic basis (p = 4); otherwise p <= 3.  Every option of a launch
// has the same kind (batches are grouped by it).
template <bool PUT, bool H16, bool P4>
__global__ void __launch_bounds__(kT, 1) sweep_cl_kernel(const __grid_constant__ KArgs a) {
    using E = typename std::conditional<H16, uint16_t, float>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemCl<E> &sm = *reinterpret_cast<SmemCl<E> *>(smem_raw);
    const int G = (int)cluster_size(), lc = (int)cluster_rank();
    const int jb = a.jobs ? (int)(blockIdx.x / (unsigned)G) : 0;
    const Job &J = a.jobs ? a.jobs[jb] : a.one;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = J.m, p = J.p;
    if (P4 != (p == 4)) {            // the launch chose the other variant: every CTA of the cluster leaves here
        if (tid == 0 && lc == 0) atomicCAS(J.status, 0, AMC_EINVAL);
        return;
    }
    const float invK = (float)J.invK, disc = (float)J.disc;
    const E *__restrict__ S = reinterpret_cast<const E *>(J.S);
    const int64_t N = J.N, ld = J.ld;
    const int64_t base = (int64_t)lc * kPPC;
    const int64_t rem = ld - base;
    const uint32_t slice_bytes = (uint32_t)(rem < kPPC ? rem : kPPC) * (uint32_t)sizeof(E);
    const int nloc = (N - base) < kPPC ? (int)(N - base) : kPPC;
    int32_t *const status = J.status;
    const uint64_t timeout_ns = a.timeout_ns;
    const int inject_date = (lc == 0 && jb == 0) ? J.inject_date : 0;
    double *const coef = (J.coef && lc == 0) ? J.coef : nullptr;

    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&sm.mbar[s], 1);
            sm.pend[s] = 0;
        }
        for (int q = 0; q < 2; ++q) mbar_init(&sm.xbarR[q], 1);
        for (int q = 0; q < 3; ++q) mbar_init(&sm.xbarM[q], 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    // every CTA's barriers are initialised before any peer sends to them
    cluster_sync_all();

    auto fail = [&]() {
        atomicCAS(status, 0, AMC_ETIMEOUT);
        sm.abort = 1;
    };
    auto issue = [&](int d) {            // one thread
        const int s = d % kSlots;
        fence_proxy_async();
        mbar_expect(&sm.mbar[s], slice_bytes);
        bulk_load(sm.S[s], S + (int64_t)(d - 1) * ld + base, slice_bytes, &sm.mbar[s]);
        sm.pend[s] = d;
    };
    // bounded wait on an mbarrier phase; the abort flag, the peers' status
    // word (a global load) and the clock are checked every 32 polls only,
    // so that they do not delay noticing the phase, and %globaltimer (a read
    // of hundreds of cycles) only once the phase is found incomplete
    auto wait_bar = [&](uint64_t *b, uint32_t parity, bool peers) -> bool {
        if (mbar_test(b, parity)) return true;
        const uint64_t t0 = globaltimer();
        for (uint32_t n = 1;; ++n) {
            if (mbar_test(b, parity)) return true;
            if ((n & 31u) == 0 &&
                (sm.abort || (peers && ld_volatile_int(status) != 0) || globaltimer() - t0 > timeout_ns)) {
                fail();
                return false;
            }
        }
    };
    auto slot_parity = [&](int d) { return (uint32_t)((m - d) / kSlots) & 1u; };
    // exchange phases: the right-hand sides of date d use barrier d mod 2,
    // the Gram moments of date e barrier e mod 3; both start at date m-1.
    // Three Gram buffers: a peer can send the moments of date e-3 only after
    // this CTA's beta_e, for which the solver warp has read those of date e.
    auto r_parity = [&](int d) { return (uint32_t)((m - 1 - d) >> 1) & 1u; };
    auto m_parity = [&](int e) { return (uint32_t)((m - 1 - e) / 3) & 1u; };

    int degenerate = 0;
    if (warp == 0) {
        // ================================================= solver warp
        // beta of date m does not exist: no exercise at maturity
        if (lane == 0) sm.deg[m & 1] = 1;
        bar_arrive_beta();
        if (coef && lane < kCoefStride) coef[(size_t)(m - 1) * kCoefStride + lane] = lane == 4 ? 1.0 : 0.0;
        dfl ginv = df_of(0.f);
        bool gdeg = true;
        bool ok = true;
        // Gram totals of date m-1 (sent before the first date's exchange)
        if (m >= 2) {
            if (lane == 0) mbar_expect(&sm.xbarM[(m - 1) % 3], (uint32_t)(G * 7 * 8));
            ok = __all_sync(kFull, wait_bar(&sm.xbarM[(m - 1) % 3], m_parity(m - 1), true));
            if (ok) ginv = cl_gram_inverse(cl_moment_totals(sm.recvM[(m - 1) % 3], G, lane), p, lane, gdeg);
        }
        for (int d = m - 1; d >= 1 && ok; --d) {
            const int par = d & 1;
            // right-hand sides of date d from every CTA -> beta_d = G_d^-1 R_d
            if (lane == 0) mbar_expect(&sm.xbarR[par], (uint32_t)(G * 4 * 8));
            ok = __all_sync(kFull, wait_bar(&sm.xbarR[par], r_parity(d), true));
            if (ok) {
                // R_k in lane k: lane 4c'+k adds sources c' and c'+8, then a
                // butterfly over c' (fixed order, the same in every CTA)
                dfl acc = df_of(0.f);
                {
                    const int k4 = lane & 3, c = lane >> 2;
                    if (c < G) acc = ld_df(sm.recvR[par][k4][c]);
                    if (c + 8 < G) acc = df_add(acc, ld_df(sm.recvR[par][k4][c + 8]));
#pragma unroll
                    for (int off = 4; off < 32; off <<= 1) acc = df_add(acc, df_shfl_xor(acc, off));
                }
                const int k = (lane >> 2) & 3, l = lane & 3;
                dfl b = df_mul(ginv, df_shfl(acc, l));
                b = df_add(b, df_shfl_xor(b, 1));
                b = df_add(b, df_shfl_xor(b, 2));
                const float bk = (k < p && !gdeg) ? __fadd_rn(b.hi, b.lo) : 0.f;
                if (lane < 16 && l == 0) sm.beta[par][k] = bk;
                if (lane == 0) {
                    sm.deg[par] = gdeg ? 1 : 0;
                    degenerate += gdeg ? 1 : 0;
                }
                if (coef && lane < 16 && l == 0) coef[(size_t)(d - 1) * kCoefStride + k] = gdeg ? 0.0 : (double)bk;
                if (coef && lane == 0) coef[(size_t)(d - 1) * kCoefStride + 4] = gdeg ? 1.0 : 0.0;
            }
            __syncwarp();
            bar_arrive_beta();                                // beta_d (or the abort) to the path warps
            if (!ok || d == 1) break;
            // Gram totals of date d-1 -> its inverse, off the critical path
            if (lane == 0) mbar_expect(&sm.xbarM[(d - 1) % 3], (uint32_t)(G * 7 * 8));
            ok = __all_sync(kFull, wait_bar(&sm.xbarM[(d - 1) % 3], m_parity(d - 1), true));
            if (ok) ginv = cl_gram_inverse(cl_moment_totals(sm.recvM[(d - 1) % 3], G, lane), p, lane, gdeg);
        }
        if (!ok) {
            bar_arrive_beta();                                // path warps waiting for a beta see the abort
        }
    } else {
        // The cubic basis (P4: moments up to y^6, right-hand sides up to y^3 C)
        // or p <= 3 (y^4 and y^2 C at most) is a compile-time choice.
        auto path_warps = [&](auto Q) {
            // ================================================== path warps
            // thread t = tid - 32 owns register pairs t + 992 s (s = 0..7), and,
            // for t < 512, the one path 15872 + t whose cash flow is in shared memory
            const int t = tid - 32;
            auto pidx = [&](int i) { return 2 * (t + kPathThreads * (i >> 1)) + (i & 1); };
            const int xidx = kRegPaths + t;
            const bool has_x = t < kPPC - kRegPaths;
            if (t == 0)
                for (int d = m; d >= 1 && d > m - kSlots; --d) issue(d);
            float cf[kPPT];
            bool stop = !wait_bar(&sm.mbar[m % kSlots], slot_parity(m), false);
            if (!stop) {
                const E *sl = sm.S[m % kSlots];
#pragma unroll
                for (int i = 0; i < kPPT; ++i) {
                    const int idx = pidx(i);
                    const float y = raw_y(sl, idx, invK);
                    const float h = PUT ? -y : y;
                    cf[i] = (idx < nloc && h > 0.f) ? h : 0.f;
                }
                if (has_x) {
                    const float y = raw_y(sl, xidx, invK);
                    const float h = PUT ? -y : y;
                    sm.cfx[t] = (xidx < nloc && h > 0.f) ? h : 0.f;
                }
            }
            // Gram pass of date e over all paths of the CTA: y in place (0 off
            // the money), the 7 moments.  The in-the-money indicator is
            // I = sat(-y 2^100) for a put, sat(y 2^100) for a call: exactly 1 for
            // every y of the money's sign, since a nonzero FP32 y of
            // fma(S, fl(1/K), -1) has |y| >= 2^-48, and 0 otherwise; then y I is
            // the in-place value and I the count (multiplies on the FMA pipe
            // instead of compares and selects)
            auto gram = [&](int e) -> bool {
                if (!wait_bar(&sm.mbar[e % kSlots], slot_parity(e), false)) return false;
                E *sl = sm.S[e % kSlots];
                const f2 z2 = f2_splat(0.f);
                const float big = PUT ? -0x1p100f : 0x1p100f;
                f2 g0 = z2, g1 = z2, g2 = z2, g3 = z2, g4 = z2, g5 = z2, g6 = z2;
                // P4: the cubic basis (moments up to y^6); otherwise p <= 3 needs y^4 at most
                auto pair = [&](int idx, bool tail, auto P4) {
                    const f2 Yr = raw_y2(sl, idx, invK);
                    float ilo = __saturatef(f2_lo(Yr) * big), ihi = __saturatef(f2_hi(Yr) * big);
                    f2 Y;
                    if (tail) {
                        // the last CTA's slot holds no paths beyond nloc (nor copied
                        // bytes beyond the row's end): select, never multiply, there
                        const bool v0 = idx < nloc, v1 = idx + 1 < nloc;
                        ilo = v0 ? ilo : 0.f;
                        ihi = v1 ? ihi : 0.f;
                        Y = f2_pack(v0 ? f2_lo(Yr) * ilo : 0.f, v1 ? f2_hi(Yr) * ihi : 0.f);
                    } else {
                        Y = f2_mul(Yr, f2_pack(ilo, ihi));
                    }
                    const f2 I = f2_pack(ilo, ihi);
                    put_y2(sl, idx, Y);
                    g0 = f2_add(g0, I);
                    const f2 YY = f2_mul(Y, Y), Y3 = f2_mul(YY, Y);
                    g1 = f2_add(g1, Y);
                    g2 = f2_add(g2, YY);
                    g3 = f2_add(g3, Y3);
                    g4 = f2_fma(YY, YY, g4);
                    if constexpr (decltype(P4)::value) {
                        g5 = f2_fma(YY, Y3, g5);
                        g6 = f2_fma(Y3, Y3, g6);
                    }
                };
                // pairs t + 992 s: s = 0..7 for every path thread, s = 8 for t < 256
                constexpr int kFullRounds = kPairs / kPathThreads;           // 8
                auto all_pairs = [&](auto P4) {
                    if (nloc == kPPC) {
#pragma unroll
                        for (int s2 = 0; s2 < kFullRounds; ++s2) pair(2 * (t + kPathThreads * s2), false, P4);
                        if (t + kPathThreads * kFullRounds < kPairs)
                            pair(2 * (t + kPathThreads * kFullRounds), false, P4);
                    } else {
#pragma unroll 2
                        for (int q = t; q < kPairs; q += kPathThreads) pair(2 * q, true, P4);
                    }
                };
                all_pairs(Q);
                fence_proxy_async();         // these generic writes precede a later TMA refill
                const float g[8] = {f2_lo(g0) + f2_hi(g0), f2_lo(g1) + f2_hi(g1), f2_lo(g2) + f2_hi(g2),
                                    f2_lo(g3) + f2_hi(g3), f2_lo(g4) + f2_hi(g4), f2_lo(g5) + f2_hi(g5),
                                    f2_lo(g6) + f2_hi(g6), 0.f};
                const float r = warp_sum8(g, lane);
                const int k = (lane >> 2) & 7;
                if ((lane & 3) == 0 && k < 7) sm.redM[e & 1][warp - 1][k] = r;
                return true;
            };
            auto send_gram = [&](int e) {    // after the path-warp barrier that completes redM[e & 1]
                const int v = warp - 5;
                if (v >= 0 && v < 7) {
                    const dfl tot = df_of(f_warp_sum(lane < kPathWarps ? sm.redM[e & 1][lane][v] : 0.f));
                    if (lane < G && inject_date != e + 1) {
                        send_df(map_to(saddr(&sm.recvM[e % 3][v][lc]), (uint32_t)lane),
                                map_to(saddr(&sm.xbarM[e % 3]), (uint32_t)lane), tot.hi, tot.lo);
                    }
                }
            };
            if (!stop && m >= 2) stop = !gram(m - 1);
            stop = bar_paths_any(stop || sm.abort);
            if (!stop && m >= 2) send_gram(m - 1);

            for (int d = m - 1; d >= 1 && !stop; --d) {
                const int par = d & 1;
                bar_sync_beta();                                  // beta_{d+1} from the solver warp
                if (sm.abort) {
                    stop = true;
                    break;
                }
                // exercise at d+1, discount to t_d, right-hand sides of date d.
                // With y in place (0 off the money) the exercise test
                // "in the money and h > c(y)" is h > max(c(y), 0), h = -y (put)
                // or y (call); the in-the-money indicator of the date-d sums is
                // sat(-+y 2^100) as in the Gram pass
                {
                    const int pe = (d + 1) & 1;
                    const bool ex = d + 1 <= m - 1 && !sm.deg[pe];
                    const float b0 = sm.beta[pe][0], b1 = sm.beta[pe][1], b2 = sm.beta[pe][2], b3 = sm.beta[pe][3];
                    const f2 B0 = f2_splat(b0), B1 = f2_splat(b1), B2 = f2_splat(b2), B3 = f2_splat(b3);
                    const f2 DISC = f2_splat(disc), z2 = f2_splat(0.f), SG = f2_splat(PUT ? -1.f : 1.f);
                    const E *se = sm.S[(d + 1) % kSlots];
                    const E *sr = sm.S[d % kSlots];
                    f2 R0 = z2, R1 = z2, R2 = z2, R3 = z2;
                    // P4: the cubic basis; otherwise b3 = 0 and R3 is not used (p <= 3)
                    // EX: exercise at d+1 as well (a compile-time branch: each variant
                    // is one straight run of the 8 pairs)
                    auto ex_rhs = [&](auto P4, auto EX) {
                        constexpr bool Q4 = decltype(P4)::value;
#pragma unroll
                    for (int i = 0; i < kPPT; i += 2) {
                        const int idx = pidx(i);
                        if constexpr (decltype(EX)::value) {
                            const f2 Y = y2_at(se, idx);
                            const f2 C = Q4 ? f2_fma(f2_fma(f2_fma(B3, Y, B2), Y, B1), Y, B0)
                                            : f2_fma(f2_fma(B2, Y, B1), Y, B0);
                            const f2 H = f2_mul(Y, SG);
                            const float hl = f2_lo(H), hh = f2_hi(H);
                            cf[i] = hl > fmaxf(f2_lo(C), 0.f) ? hl : cf[i];
                            cf[i + 1] = hh > fmaxf(f2_hi(C), 0.f) ? hh : cf[i + 1];
                        }
                        const f2 Y = y2_at(sr, idx);
                        const f2 C = f2_mul(f2_pack(cf[i], cf[i + 1]), DISC);
                        cf[i] = f2_lo(C);
                        cf[i + 1] = f2_hi(C);
                        const float big = PUT ? -0x1p100f : 0x1p100f;
                        R0 = f2_fma(C, f2_pack(__saturatef(f2_lo(Y) * big), __saturatef(f2_hi(Y) * big)), R0);
                        const f2 YY = f2_mul(Y, Y);
                        R1 = f2_fma(C, Y, R1);                            // y = 0 off the money
                        R2 = f2_fma(C, YY, R2);
                        if (Q4) R3 = f2_fma(C, f2_mul(YY, Y), R3);
                    }
                    };
                    if (ex)
                        ex_rhs(Q, std::true_type{});
                    else
                        ex_rhs(Q, std::false_type{});
                    float rr[4] = {f2_lo(R0) + f2_hi(R0), f2_lo(R1) + f2_hi(R1), f2_lo(R2) + f2_hi(R2),
                                   f2_lo(R3) + f2_hi(R3)};
                    if (has_x) {                                          // the shared-memory path
                        float c = sm.cfx[t];
                        if (ex) {
                            const float y = y_at(se, xidx);
                            const float cont = fmaf(fmaf(fmaf(b3, y, b2), y, b1), y, b0);
                            const float h = PUT ? -y : y;
                            c = ((PUT ? y < 0.f : y > 0.f) && h > cont) ? h : c;
                        }
                        c *= disc;
                        sm.cfx[t] = c;
                        const float y = y_at(sr, xidx);
                        const float cc = y != 0.f ? c : 0.f, yy = y * y;
                        rr[0] += cc;
                        rr[1] = fmaf(c, y, rr[1]);
                        rr[2] = fmaf(c, yy, rr[2]);
                        rr[3] = fmaf(c, yy * y, rr[3]);
                    }
                    const float r = warp_sum4(rr, lane);
                    const int k = (lane >> 3) & 3;
                    if ((lane & 7) == 0) sm.redR[par][warp - 1][k] = k < p ? r : 0.f;
                }
                stop = bar_paths_any(sm.abort);                       // partials complete; slot d+1 free
                if (stop) break;
                if (t == 0 && d - 2 >= 1) issue(d - 2);                   // into the slot of date d+1
                {
                    const int v = warp - 1;                               // warps 1..4: right-hand side v
                    if (v < 4) {
                        const dfl tot = df_of(f_warp_sum(lane < kPathWarps ? sm.redR[par][lane][v] : 0.f));
                        if (lane < G && inject_date != d) {
                            send_df(map_to(saddr(&sm.recvR[par][v][lc]), (uint32_t)lane),
                                    map_to(saddr(&sm.xbarR[par]), (uint32_t)lane), tot.hi, tot.lo);
                        }
                    }
                }
                // Gram pass of date d-1 while the exchange and the solve run
                if (d - 1 >= 1) {
                    bool ok = gram(d - 1);
                    stop = bar_paths_any(!ok || sm.abort);
                    if (stop) break;
                    send_gram(d - 1);
                }
            }
            // the last exercise date, t_1
            if (!stop && m >= 2) {
                bar_sync_beta();
                if (sm.abort) {
                    stop = true;
                } else if (!sm.deg[1]) {
                    const float b0 = sm.beta[1][0], b1 = sm.beta[1][1], b2 = sm.beta[1][2], b3 = sm.beta[1][3];
                    const E *se = sm.S[1 % kSlots];
#pragma unroll
                    for (int i = 0; i < kPPT; ++i) {
                        const float y = y_at(se, pidx(i));
                        const float cont = fmaf(fmaf(fmaf(b3, y, b2), y, b1), y, b0);
                        const float h = PUT ? -y : y;
                        cf[i] = ((PUT ? y < 0.f : y > 0.f) && h > cont) ? h : cf[i];
                    }
                    if (has_x) {
                        const float y = y_at(se, xidx);
                        const float cont = fmaf(fmaf(fmaf(b3, y, b2), y, b1), y, b0);
                        const float h = PUT ? -y : y;
                        if ((PUT ? y < 0.f : y > 0.f) && h > cont) sm.cfx[t] = h;
                    }
                }
            }
            // final per-thread sums (units of K): CF, CF^2
            float fs[4] = {0.f, 0.f, 0.f, 0.f};
            if (!stop) {
#pragma unroll
                for (int i = 0; i < kPPT; ++i) {
                    if (pidx(i) >= nloc) continue;
                    fs[0] += cf[i];
                    fs[1] += cf[i] * cf[i];
                }
                if (has_x && xidx < nloc) {
                    const float c = sm.cfx[t];
                    fs[0] += c;
                    fs[1] += c * c;
                }
            }
            const float r = warp_sum4(fs, lane);
            const int k = (lane >> 3) & 3;
            if ((lane & 7) == 0) sm.redF[warp - 1][k] = r;
            if (stop && t == 0) {
                // bounded wait for this CTA's own copies still in flight
                for (int s = 0; s < kSlots; ++s) {
                    const int d = sm.pend[s];
                    if (d <= 0) continue;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_test(&sm.mbar[s], slot_parity(d)) && globaltimer() - t0 < timeout_ns) {
                    }
                }
            }
        };
        path_warps(std::integral_constant<bool, P4>{});
    }
    __syncthreads();
    if (!sm.abort) {
        if (warp < 2) {
            const dfl part = df_warp_sum(df_of(lane < kPathWarps ? sm.redF[lane][warp] : 0.f));
            const double scale = warp == 0 ? J.K : J.K * J.K;
            if (lane == 0) {
                double *fin = reinterpret_cast<double *>(J.fin) + (int64_t)lc * 4;
                fin[warp] = scale * ((double)part.hi + (double)part.lo);
                if (warp == 0) fin[2] = fin[3] = 0.0;
            }
        }
        if (lc == 0 && tid == 0) J.res[4] = (double)degenerate;
    } else if (tid == 0) {
        // a short grace period for peers' sends issued just before they
        // stopped (every send is awaited on the normal path)
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 20000u) {
        }
    }
    // no CTA leaves while a peer may still send into its shared memory
    cluster_sync_all();
}

}  // namespace

size_t sweep_cl_smem() { return sizeof(SmemCl<float>); }

cudaError_t launch_sweep_cl(const KArgs &a, int cluster, int n_clusters, cudaStream_t st) {
    if (cluster < 1 || cluster > kMaxG || n_clusters < 1) return cudaErrorInvalidValue;
    const bool put = (a.jobs ? a.jobs_type : a.one.type) == AMC_PUT;
    const bool p4 = (a.jobs ? a.jobs_p : a.one.p) == 4;
    void (*kern)(KArgs);
    if (p4)
        kern = a.h16 ? (put ? sweep_cl_kernel<true, true, true> : sweep_cl_kernel<false, true, true>)
                     : (put ? sweep_cl_kernel<true, false, true> : sweep_cl_kernel<false, false, true>);
    else
        kern = a.h16 ? (put ? sweep_cl_kernel<true, true, false> : sweep_cl_kernel<false, true, false>)
                     : (put ? sweep_cl_kernel<true, false, false> : sweep_cl_kernel<false, false, false>);
    const void *f = (const void *)kern;
    const size_t smem = a.h16 ? sizeof(SmemCl<uint16_t>) : sizeof(SmemCl<float>);
    cudaError_t e = ensure_smem(f, smem);
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(cluster * n_clusters));
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// Largest cluster of this kernel that the current device can hold at once
// (0 if none): a 16-CTA cluster needs 16 SMs of one GPC with room for a
// 1024-thread CTA and its ring.  Taken with the FP32 ring; the binary16
// ring is smaller, so the binary16 variants hold at least as many.
cudaError_t sweep_cl_max_cluster(int *out) {
    *out = 0;
    const void *f = (const void *)sweep_cl_kernel<true, false, true>;
    const size_t smem = sizeof(SmemCl<float>);
    cudaError_t e = ensure_smem(f, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)sweep_cl_kernel<false, false, true>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = ensure_smem((const void *)sweep_cl_kernel<false, false, true>, smem);
    if (e != cudaSuccess) return e;
    for (int g = kMaxG; g >= 1; --g) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)g);
        cfg.blockDim = dim3(kT);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)g;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, f, &cfg);
        if (e == cudaSuccess && n > 0) {
            *out = g;
            return cudaSuccess;
        }
    }
    return cudaSuccess;
}

}  // namespace amc
