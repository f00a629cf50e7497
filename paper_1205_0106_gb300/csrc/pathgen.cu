// Path generation (steps 1-3 of the hot path) for sm_103a:
//   Sobol' integers (Gray-code order, digital XOR shift)      §III.D
//   -> uniform (x + 1/2) 2^-32 -> N(0,1)                      §III.D
//   -> Brownian bridge (breadth-first coordinate order,       ref. [13]
//      evaluated depth-first with a per-path slot stack)
//   -> GBM in log space, S = S0 exp((r - sigma^2/2) t + sigma W)   Eq. 9
//   -> date-major store S[j-1][i].
//
// One CTA of kPathgenThreads threads owns a tile of 4 kPathgenThreads
// consecutive Sobol' points and thread t the 4 consecutive points
// tile + 4t + q (q = 0..3), so every date row is written with one 16-byte
// store per thread and the bridge stack is read and written as float4.  The Gray code is linear over GF(2) and the
// three index parts occupy disjoint bits, hence
//   x(tile + 4t + q) = x(tile) xor x(4t) xor x(q):
// x(tile) per dimension once per tile (shared memory), x(4t) from the
// direction numbers v_2..v_(kGB+1) selected by the thread's Gray bits, x(q) from
// v_1, v_2 (the same for all threads).
#include <cuda_runtime.h>
#include <math.h>

#include "devutil.cuh"
#include "icdf.cuh"
#include "internal.h"

namespace amc {

namespace {

__device__ __forceinline__ uint32_t sobol_direct(const uint32_t *__restrict__ V, int d, uint32_t i) {
    uint32_t g = i ^ (i >> 1), x = 0;
    while (g) {
        int b = __ffs(g) - 1;
        x ^= __ldg(V + d * 32 + b);
        g &= g - 1;
    }
    return x;
}


template <bool FP64>
struct PG;
template <>
struct PG<false> {
    using Real = float;
    using Node = NodeF;
};
template <>
struct PG<true> {
    using Real = double;
    using Node = NodeD;
};

template <typename Real>
struct alignas(4 * sizeof(Real)) R4 {
    Real v[4];
};

// A bridge node as pathgen_kernel reads it, expanded from NodeF/NodeD once
// per job: shared-memory offsets instead of indices, and the job's scale
// factors applied (the same products the node loop would form).  32 bytes
// in FP32; the node's direction numbers and tile integers sit in tables
// indexed by node, so the record holds no Sobol' dimension.
template <typename Real>
struct alignas(16) NodeX {
    uint16_t wl_o, wr_o, wo_o;    // byte offsets of the left, right and own stack slots
    uint16_t date;
    Real wl, wr, sd, drift;       // bridge weights, sdu sqrt(dt), the exponent's constant (node_points)
    int64_t row;                  // (date - 1) ld: element offset of the date's row
};
static_assert(sizeof(NodeX<float>) == 32 && sizeof(NodeX<double>) == 48, "node records");
static_assert(kMaxSlots * kPathgenThreads * sizeof(double) * 4 <= 65536 && AMC_MAX_STEPS < 65536,
              "slot offsets and dates fit 16 bits");

// Shared-memory layout of the path-generation kernel: every sub-buffer
// starts on a 32-byte boundary (uint4 and R4<double> accesses).  A kernel
// that values a fitted boundary on the fly also holds the boundary (four
// coefficients and a flag per date); one that takes the paper's rule holds
// two discounted-payoff constants per date.
struct PathgenSmem {
    unsigned nodes, v, v9, xb, W, coef, deg, total;
};
__host__ __device__ __forceinline__ unsigned al32(unsigned v) { return (v + 31u) & ~31u; }
__host__ __device__ __forceinline__ PathgenSmem pathgen_layout(int max_m, int nslots, bool fp64, int mode = 0) {
    const bool boundary = mode == 3;
    const unsigned per_date = boundary ? 4u : (mode == 1 ? 2u : 0u);
    PathgenSmem L;
    const unsigned node = fp64 ? (unsigned)sizeof(NodeX<double>) : (unsigned)sizeof(NodeX<float>);
    static_assert(sizeof(NodeX<double>) >= sizeof(NodeD) && sizeof(NodeX<float>) >= sizeof(NodeF), "node region");
    const unsigned real = fp64 ? 8u : 4u;
    L.nodes = 0;
    L.v = al32(L.nodes + node * (unsigned)max_m);
    L.v9 = al32(L.v + 32u * (unsigned)max_m);             // v_1..v_8 as two uint4 per dimension, then v_9
    L.xb = al32(L.v9 + 4u * (unsigned)max_m);
    L.W = al32(L.xb + 4u * (unsigned)max_m);
    L.coef = al32(L.W + real * 4u * kPathgenThreads * (unsigned)nslots);
    L.deg = al32(L.coef + real * per_date * (unsigned)max_m);
    L.total = L.deg + (boundary ? (unsigned)max_m : 0u);
    return L;
}

__device__ __forceinline__ int find_job_by_tile(const Job *__restrict__ jobs, int n_jobs, int64_t tile) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The 4 points of one bridge node: z = N^{-1}(u) of the Sobol' integers xq,
// W = wl W_left + wr W_right + sd z (ref. [13]), then Eq. 9 in log space:
// FP64: S = S0 exp(drift + sig W), drift = mu t_d; FP32: base 2 with the
// spot folded into the exponent, S = 2^(drift + sig W), drift = mu t_d /
// ln 2 + log2(S0), or (Y16) the moneyness y = 2^(drift + sig W) - 1 with
// drift = mu t_d / ln 2 + log2(S0 / K).  In FP32 xq holds the integers with
// the top bit flipped, so that as signed values they are x - 2^31 (the
// uniform's offset from 1/2).
template <bool FP64, bool Y16, typename Real>
__device__ __forceinline__ void node_points(const uint32_t (&xq)[4], Real wl, Real wr, Real sd, Real drift,
                                            Real sig, Real S0, const R4<Real> &Wl, const R4<Real> &Wr,
                                            R4<Real> &Wo, R4<Real> &So) {
    if (FP64) {
        Real z[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) z[q] = (Real)normcdfinv(((double)xq[q] + 0.5) * 0x1p-32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Real W = fma(sd, z[q], fma(wr, Wr.v[q], wl * Wl.v[q]));
            Wo.v[q] = W;
            So.v[q] = S0 * (Real)exp((double)fma(sig, W, drift));
        }
    } else {
        // points (0, 1) and (2, 3) as packed pairs: central-region
        // values straight-line, then the rare tails, then bridge and GBM
        using namespace dev;
        float z[4], yv[4];
        bool tail = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const f2 y = f2_fma(f2_pack((float)(int32_t)xq[2 * h], (float)(int32_t)xq[2 * h + 1]),
                                f2_splat(0x1p-32f), f2_splat(0x1p-33f));
            const f2 zc = icdf_central2(y);
            yv[2 * h] = f2_lo(y);
            yv[2 * h + 1] = f2_hi(y);
            z[2 * h] = f2_lo(zc);
            z[2 * h + 1] = f2_hi(zc);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) tail |= !(fabsf(yv[q]) < kIcdfY0);
        // about one node in seven has a tail point somewhere in the warp:
        // a warp-uniform branch around the rare per-point tails
        if (__any_sync(0xffffffffu, tail)) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (!(fabsf(yv[q]) < kIcdfY0)) z[q] = icdf_tail(xq[q] ^ 0x80000000u, yv[q]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const f2 W = f2_fma(f2_splat((float)sd), f2_pack(z[2 * h], z[2 * h + 1]),
                                f2_fma(f2_splat((float)wr), f2_pack((float)Wr.v[2 * h], (float)Wr.v[2 * h + 1]),
                                       f2_mul(f2_splat((float)wl),
                                              f2_pack((float)Wl.v[2 * h], (float)Wl.v[2 * h + 1]))));
            const f2 e = f2_fma(f2_splat((float)sig), W, f2_splat((float)drift));
            f2 Sv = f2_pack(ex2_approx(f2_lo(e)), ex2_approx(f2_hi(e)));
            if (Y16) Sv = f2_add(Sv, f2_splat(-1.f));
            Wo.v[2 * h] = (Real)f2_lo(W);
            Wo.v[2 * h + 1] = (Real)f2_hi(W);
            So.v[2 * h] = (Real)f2_lo(Sv);
            So.v[2 * h + 1] = (Real)f2_hi(Sv);
        }
    }
}

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }
constexpr int kGB = ilog2(kTilePoints) - 1;       // Gray bits 1..kGB of the thread's point offset 4t
static_assert((1 << ilog2(kTilePoints)) == kTilePoints && kGB + 1 <= 9, "tile of 2^k points, direction numbers v_1..v_9");

// MODE kStore writes the path array (steps 1-3); kStore16 writes it as
// binary16 moneyness y = S/K - 1 (8 bytes per thread and date).  The other
// modes value
// every path as its dates are formed and store nothing; they need no
// regression across paths, and their per-path value does not depend on the
// order in which the bridge forms the dates:
//   kPaperRule  Eqs. 10-11: the backward recursion V = max(h_j, e^{-r dt} V)
//               from V_{m-1} = max(h_{m-1}, BS over [t_{m-1}, t_m]) down to
//               t_0 (S_0 = S0) equals max_j e^{-r t_j} h_j, with the
//               Black-Scholes term taken at t_{m-1}; a running maximum;
//   kEuropean   Eqs. 6-8: e^{-rT} h(S_m);
//   kBoundary   a fitted boundary (continuation value over K, polynomial in
//               y = S/K - 1): the first date tau < m where it exercises (not
//               flagged, in the money, h > c(y), in the valuation kernel's
//               arithmetic), else tau = m; the value at t_1 is
//               e^{-r (t_tau - t_1)} h(S_tau) (finalize adds the last e^{-r dt}).
// Each CTA adds its paths' values and squares in FP64 into its own slot of
// J.fin, in a fixed order, for finalize_kernel.
template <bool FP64, int MODE>
__global__ void __launch_bounds__(kPathgenThreads) pathgen_kernel(const __grid_constant__ KArgs a) {
    using Real = typename PG<FP64>::Real;
    using Node = typename PG<FP64>::Node;
    constexpr bool STORE = MODE == kStore || MODE == kStore16;
    static_assert(!(FP64 && MODE == kStore16), "binary16 moneyness is an FP32-path format");
    extern __shared__ __align__(32) unsigned char smem[];
    const int max_m = a.max_m;
    const PathgenSmem L = pathgen_layout(max_m, a.max_slots, FP64, MODE);
    Real(*s_c)[4] = reinterpret_cast<Real(*)[4]>(smem + L.coef);             // [m][4] boundary (units of K)
    Real(*s_ab)[2] = reinterpret_cast<Real(*)[2]>(smem + L.coef);            // [m][2] paper rule: a_d, b_d
    unsigned char *s_deg = smem + L.deg;                                    // [m] no exercise at the date
    NodeX<Real> *s_nodes = reinterpret_cast<NodeX<Real> *>(smem + L.nodes);
    uint4 *s_v = reinterpret_cast<uint4 *>(smem + L.v);                    // [m][2]: v_1..v_8 of each node's dim
    uint32_t *s_v9 = reinterpret_cast<uint32_t *>(smem + L.v9);            // [m]: v_9 of each node's dim
    uint32_t *s_xb = reinterpret_cast<uint32_t *>(smem + L.xb);            // [m]: x(tile) xor shift, by node
    R4<Real> *s_W = reinterpret_cast<R4<Real> *>(smem + L.W);              // [slot][128]

    const uint32_t *__restrict__ V = a.V;
    const int tid = threadIdx.x;
    const uint32_t t4 = 4u * (uint32_t)tid;
    const uint32_t g4 = t4 ^ (t4 >> 1);                                   // Gray bits 1..kGB of 4t
    uint32_t gm[kGB];                                                     // all-ones where bit b+1 is set
#pragma unroll
    for (int b = 0; b < kGB; ++b) gm[b] = 0u - ((g4 >> (b + 1)) & 1u);
    // FP32: the integers' top bit flipped once here (x - 2^31 as signed values, node_points)
    const uint32_t flip = FP64 ? 0u : 0x80000000u;
    unsigned char *const Wt = reinterpret_cast<unsigned char *>(s_W + tid);   // this thread's slot 0
    {
        // every stack slot starts at 0: the root, and a node whose left end
        // point is W(0) = 0, read a slot with weight 0 (never before it is
        // written in that tile but for these reads), which must hold a
        // finite value
        R4<Real> zero;
#pragma unroll
        for (int q = 0; q < 4; ++q) zero.v[q] = Real(0);
        for (int sl = 0; sl < a.max_slots; ++sl) s_W[sl * kPathgenThreads + tid] = zero;
    }
    int cur = -1;
    int m = 0;
    double vs1 = 0.0, vs2 = 0.0;                                          // this thread's path values (fused modes)
    for (int64_t tile = blockIdx.x; tile < a.total; tile += gridDim.x) {
        const int jb = a.jobs ? find_job_by_tile(a.jobs, a.n_jobs, tile) : 0;
        const Job &J = a.jobs ? a.jobs[jb] : a.one;
        const uint32_t base = (uint32_t)((tile - J.tile_begin) * kTilePoints);
        const uint32_t *__restrict__ shift = a.jobs ? J.shift : a.shift_one;
        __syncthreads();                                                  // previous tile done with smem
        if (jb != cur) {
            m = J.m;
            const Node *gn = reinterpret_cast<const Node *>(J.nodes);
            const double mu = J.r - 0.5 * J.sigma * J.sigma;
            const Real sqdt = (Real)sqrt(J.dt);
            // exponent per node: FP32 in base 2 (ex2), FP64 in base e
            const Real mu_dt = (Real)(mu * J.dt);                              // FP64
            const double mu_dt2 = mu * J.dt * 1.4426950408889634;                 // FP32: base 2
            const double lS0 = log2(MODE == kStore16 ? J.S0 * J.invK : J.S0);
            constexpr int kSlotBytes = kPathgenThreads * (int)sizeof(R4<Real>);
            for (int i = tid; i < m; i += kPathgenThreads) {
                const Node g = gn[i];
                NodeX<Real> x;
                x.wl_o = (uint16_t)(g.sl * kSlotBytes);
                x.wr_o = (uint16_t)(g.sr * kSlotBytes);
                x.wo_o = (uint16_t)(g.so * kSlotBytes);
                x.date = (uint16_t)g.date;
                x.wl = (Real)g.wl;
                x.wr = (Real)g.wr;
                x.sd = (Real)g.sdu * sqdt;
                x.drift = FP64 ? mu_dt * (Real)g.date : (Real)(mu_dt2 * (double)g.date + lS0);
                x.row = (int64_t)(g.date - 1) * J.ld;
                s_nodes[i] = x;
                const uint4 *Vd = reinterpret_cast<const uint4 *>(V + g.coord * 32);
                s_v[2 * i] = __ldg(Vd);
                s_v[2 * i + 1] = __ldg(Vd + 1);
                s_v9[i] = __ldg(V + g.coord * 32 + 8);
            }
            if (MODE == kPaperRule) {
                // e^{-r t_d} h(S) = a_d + b_d S where h > 0 (put: a_d = e^{-r t_d} K, b_d = -e^{-r t_d})
                for (int d = tid; d < m; d += kPathgenThreads) {
                    const double df = exp(-J.r * J.dt * (double)(d + 1));
                    const bool put = J.type == AMC_PUT;
                    s_ab[d][0] = (Real)(put ? df * J.K : -df * J.K);
                    s_ab[d][1] = (Real)(put ? -df : df);
                }
            }
            if (MODE == kBoundary) {
                for (int d = tid; d < m; d += kPathgenThreads) {
                    const double *c = J.coef + (size_t)d * kCoefStride;
#pragma unroll
                    for (int k = 0; k < 4; ++k) s_c[d][k] = k < J.p ? (Real)c[k] : Real(0);
                    s_deg[d] = (d == m - 1 || c[4] != 0.0) ? 1 : 0;
                }
            }
            cur = jb;
        }
        {
            const Node *gn = reinterpret_cast<const Node *>(J.nodes);
            for (int k = tid; k < m; k += kPathgenThreads) {
                const int c = __ldg(&gn[k].coord);
                s_xb[k] = sobol_direct(V, c, base) ^ shift[c] ^ flip;
            }
        }
        __syncthreads();

        const int64_t ld = J.ld;
        const bool store = (int64_t)base + t4 < ld;                       // float4 stays inside the row
        Real *__restrict__ S = reinterpret_cast<Real *>(J.S) + base + t4;
        uint16_t *__restrict__ Sh = reinterpret_cast<uint16_t *>(J.S) + base + t4;
        const Real S0 = (Real)J.S0;                                      // FP64 (FP32: in the drift)
        const Real sig = FP64 ? (Real)J.sigma : (Real)(J.sigma * 1.4426950408889634);
        // fused modes: per-path state of the thread's 4 paths
        const bool put = J.type == AMC_PUT;
        const Real K = (Real)J.K, invK = (Real)J.invK, rr = (Real)J.r, vol = (Real)J.sigma;
        const Real rdt = (Real)(J.r * J.dt);
        Real acc[4];                // kPaperRule: running max; kEuropean: value; kBoundary: h(S_tau) / K
        int tau[4];                 // kBoundary: first exercise date (m: none)
        Real hm[4];                 // kBoundary: h(S_m) / K
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            tau[q] = m;
            hm[q] = Real(0);
            acc[q] = Real(0);
            if (MODE == kPaperRule) {
                const Real h0 = dev::payoff(put, (Real)J.S0, K);
                if (m == 1) {
                    const Real c0 = dev::bs_value(put, (Real)J.S0, K, rr, vol, (Real)J.T);
                    acc[q] = h0 > c0 ? h0 : c0;
                } else {
                    acc[q] = h0;
                }
            }
        }

        // FP32 store/paper-rule modes unrolled: later nodes' quantiles overlap earlier nodes' bridge and store
        // (0.442 -> 0.405 ms on 2^20 x 252); FP64 stays rolled (unrolled by 8: 69 -> 106 ms all-FP64 pricing)
#pragma unroll ((!FP64 && (STORE || MODE == kPaperRule)) ? 8 : 1)
        for (int n = 0; n < m; ++n) {
            const NodeX<Real> nd = s_nodes[n];
            const uint4 v0 = s_v[2 * n], v1 = s_v[2 * n + 1];
            const uint32_t vd[9] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, s_v9[n]};
            uint32_t x0 = s_xb[n];
#pragma unroll
            for (int b = 0; b < kGB; ++b) x0 ^= vd[b + 1] & gm[b];
            const uint32_t xq[4] = {x0, x0 ^ v0.x, x0 ^ v0.x ^ v0.y, x0 ^ v0.y};
            const R4<Real> Wl = *reinterpret_cast<const R4<Real> *>(Wt + nd.wl_o);
            const R4<Real> Wr = *reinterpret_cast<const R4<Real> *>(Wt + nd.wr_o);
            R4<Real> Wo, So;
            node_points<FP64, MODE == kStore16, Real>(xq, nd.wl, nd.wr, nd.sd, nd.drift, sig, S0, Wl, Wr, Wo, So);
            *reinterpret_cast<R4<Real> *>(Wt + nd.wo_o) = Wo;
            if (MODE == kStore16) {
                if (store) {
                    uint16_t *dst = Sh + nd.row;
                    *reinterpret_cast<uint2 *>(dst) = make_uint2(dev::f_to_h2((float)So.v[0], (float)So.v[1]),
                                                                 dev::f_to_h2((float)So.v[2], (float)So.v[3]));
                }
            } else if (MODE == kStore) {
                if (store) {
                    Real *dst = S + nd.row;
                    if (FP64) {                                           // two 16-byte stores
                        reinterpret_cast<double2 *>(dst)[0] = make_double2((double)So.v[0], (double)So.v[1]);
                        reinterpret_cast<double2 *>(dst)[1] = make_double2((double)So.v[2], (double)So.v[3]);
                    } else {
                        *reinterpret_cast<float4 *>(dst) = make_float4((float)So.v[0], (float)So.v[1],
                                                                       (float)So.v[2], (float)So.v[3]);
                    }
                }
            } else if (MODE == kPaperRule) {
                // running maximum of a_d + b_d S_d: where the payoff is 0 that
                // value is <= 0 <= h(S0), the maximum's first term, so it never wins
                const int d = nd.date;
                if (d < m - 1) {
                    const Real ad = s_ab[d - 1][0], bd = s_ab[d - 1][1];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] = fmax(acc[q], fma(bd, So.v[q], ad));
                } else if (d == m - 1) {
                    const Real dfd = exp(-rdt * (Real)d);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const Real h = dev::payoff(put, So.v[q], K);
                        const Real c = dev::bs_value(put, So.v[q], K, rr, vol, (Real)J.dt);
                        acc[q] = fmax(acc[q], dfd * (h > c ? h : c));
                    }
                }
            } else if (MODE == kEuropean) {
                if (nd.date == m) {
                    const Real dfT = exp(-rr * (Real)J.T);
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] = dfT * dev::payoff(put, So.v[q], K);
                }
            } else {                                                      // kBoundary
                const int d = nd.date;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const Real y = fma(So.v[q], invK, Real(-1));
                    const Real h = put ? -y : y;
                    if (d == m) {
                        hm[q] = h > Real(0) ? h : Real(0);
                    } else if (d < tau[q] && !s_deg[d - 1]) {
                        const Real cont = fma(fma(fma(s_c[d - 1][3], y, s_c[d - 1][2]), y, s_c[d - 1][1]), y,
                                              s_c[d - 1][0]);
                        if ((put ? y < Real(0) : y > Real(0)) && h > cont) {
                            tau[q] = d;
                            acc[q] = h;
                        }
                    }
                }
            }
        }
        if (!STORE) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if ((int64_t)base + t4 + q >= J.N) continue;
                Real v = acc[q];
                if (MODE == kBoundary) v = (tau[q] < m ? acc[q] : hm[q]) * exp(-rdt * (Real)(tau[q] - 1));
                vs1 += (double)v;
                vs2 += (double)v * (double)v;
            }
        }
    }
    if (!STORE) {
        // fixed-order CTA sum into this CTA's slot of J.fin (finalize_kernel)
        __shared__ double red[kPathgenThreads / 32][2];
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            vs1 += __shfl_xor_sync(0xffffffffu, vs1, off);
            vs2 += __shfl_xor_sync(0xffffffffu, vs2, off);
        }
        if ((tid & 31) == 0) {
            red[tid >> 5][0] = vs1;
            red[tid >> 5][1] = vs2;
        }
        __syncthreads();
        if (tid == 0) {
            const Job &J = a.one;
            double b1 = 0.0, b2 = 0.0;
            for (int w = 0; w < kPathgenThreads / 32; ++w) {
                b1 += red[w][0];
                b2 += red[w][1];
            }
            const double sc = MODE == kBoundary ? J.K : 1.0;                // kBoundary sums in units of K
            double *fin = reinterpret_cast<double *>(J.fin) + (int64_t)blockIdx.x * 4;
            fin[0] = sc * b1;
            fin[1] = sc * sc * b2;
            fin[2] = 0.0;
            fin[3] = 0.0;
            if (blockIdx.x == 0) {
                int nd = 0;
                if (MODE == kBoundary)
                    for (int d = 0; d < J.m - 1; ++d) nd += s_deg[d];
                J.res[4] = (double)nd;
            }
        }
    }
}

// Path generation from the paper's randomised points (§III.D, read as a
// permutation of each dimension's quasi-random array by a linear
// congruential generator): path i takes the unshifted Sobol' point pi_d(i)
// in dimension d, pi_d(i) = L_d(i) walked back into 0..N-1, L_d(x) =
// (a_d x + c_d) mod 2^log2M with a_d = 1 mod 4 and c_d odd (full period, so
// pi_d is a permutation).  Neighbouring paths no longer share Gray-code
// structure, so every point is formed on its own from the direction
// numbers; the bridge, GBM and stores are those of pathgen_kernel.
template <bool FP64>
__global__ void __launch_bounds__(kPathgenThreads) pathgen_perm_kernel(const __grid_constant__ PermArgs a) {
    using Real = typename PG<FP64>::Real;
    using Node = typename PG<FP64>::Node;
    extern __shared__ __align__(32) unsigned char smem[];
    const Job &J = a.one;
    const int m = J.m;
    const PathgenSmem L = pathgen_layout(m, a.max_slots, FP64);
    Node *s_nodes = reinterpret_cast<Node *>(smem + L.nodes);
    R4<Real> *s_W = reinterpret_cast<R4<Real> *>(smem + L.W);
    const uint32_t *__restrict__ V = a.V;
    const int tid = threadIdx.x;
    const uint64_t mask = (1ull << a.log2M) - 1ull;
    const uint64_t N = (uint64_t)J.N;
    const Node *gn = reinterpret_cast<const Node *>(J.nodes);
    for (int i = tid; i < m; i += kPathgenThreads) s_nodes[i] = gn[i];
    const int64_t ld = J.ld;
    const double mu = J.r - 0.5 * J.sigma * J.sigma;
    const Real sqdt = (Real)sqrt(J.dt);
    const Real S0 = (Real)J.S0;
    const Real mu_dt = (Real)(mu * J.dt);                                  // FP64
    const double mu_dt2 = mu * J.dt * 1.4426950408889634, lS0 = log2(J.S0);   // FP32: base 2, spot folded in
    const Real sig = FP64 ? (Real)J.sigma : (Real)(J.sigma * 1.4426950408889634);
    {
        // every stack slot starts at 0 (the reads with weight 0, pathgen_kernel)
        R4<Real> zero;
#pragma unroll
        for (int q = 0; q < 4; ++q) zero.v[q] = Real(0);
        for (int sl = 0; sl < a.max_slots; ++sl) s_W[sl * kPathgenThreads + tid] = zero;
    }
    for (int64_t tile = blockIdx.x; tile < a.total; tile += gridDim.x) {
        const uint64_t base = (uint64_t)tile * kTilePoints;
        __syncthreads();                                                  // previous tile done with smem
        const bool store = (int64_t)(base + 4u * tid) < ld;
        Real *__restrict__ S = reinterpret_cast<Real *>(J.S) + base + 4u * tid;
        for (int n = 0; n < m; ++n) {
            const Node nd = s_nodes[n];
            const uint32_t ad = a.a[nd.coord], cd = a.c[nd.coord];
            const uint32_t *__restrict__ Vd = V + nd.coord * 32;
            uint32_t xq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint64_t i = base + 4u * tid + q;
                uint64_t j = 0;
                if (i < N) {
                    j = ((uint64_t)ad * i + cd) & mask;
                    while (j >= N) j = ((uint64_t)ad * j + cd) & mask;
                }
                const uint32_t g = (uint32_t)(j ^ (j >> 1));
                uint32_t x = 0;
                for (uint32_t b = 0; b < a.log2M; ++b) x ^= __ldg(Vd + b) & (0u - ((g >> b) & 1u));
                xq[q] = FP64 ? x : x ^ 0x80000000u;              // FP32: top bit flipped (node_points)
            }
            const Real wl = (Real)nd.wl, wr = (Real)nd.wr, sd = (Real)nd.sdu * sqdt;
            const Real drift = FP64 ? mu_dt * (Real)nd.date : (Real)(mu_dt2 * (double)nd.date + lS0);
            const R4<Real> Wl = s_W[nd.sl * kPathgenThreads + tid];
            const R4<Real> Wr = s_W[nd.sr * kPathgenThreads + tid];
            R4<Real> Wo, So;
            node_points<FP64, false, Real>(xq, wl, wr, sd, drift, sig, S0, Wl, Wr, Wo, So);
            s_W[nd.so * kPathgenThreads + tid] = Wo;
            if (store) {
                Real *dst = S + (int64_t)(nd.date - 1) * ld;
                if (FP64) {
                    reinterpret_cast<double2 *>(dst)[0] = make_double2((double)So.v[0], (double)So.v[1]);
                    reinterpret_cast<double2 *>(dst)[1] = make_double2((double)So.v[2], (double)So.v[3]);
                } else {
                    *reinterpret_cast<float4 *>(dst) = make_float4((float)So.v[0], (float)So.v[1],
                                                                   (float)So.v[2], (float)So.v[3]);
                }
            }
        }
    }
}

__global__ void sobol_kernel(const uint32_t *__restrict__ V, int n_dims, int64_t n_points,
                             const uint32_t *__restrict__ shift, uint32_t *__restrict__ x, int64_t ld) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (i >= n_points || d >= n_dims) return;
    x[(int64_t)d * ld + i] = sobol_direct(V, d, (uint32_t)i) ^ __ldg(shift + d);
}

}  // namespace

size_t pathgen_smem_bytes(int max_m, int nslots, bool fp64) { return pathgen_layout(max_m, nslots, fp64).total; }

cudaError_t launch_sobol(const uint32_t *V, int n_dims, int64_t n_points, const uint32_t *shift,
                         uint32_t *x, int64_t ld, cudaStream_t st) {
    if (n_points <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n_points + 255) / 256), (unsigned)n_dims);
    sobol_kernel<<<grid, 256, 0, st>>>(V, n_dims, n_points, shift, x, ld);
    return cudaGetLastError();
}

cudaError_t launch_pathgen_permuted(const PermArgs &a, bool fp64, int sm_count, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    size_t smem = pathgen_smem_bytes(a.one.m, a.max_slots, fp64);
    auto kern = fp64 ? pathgen_perm_kernel<true> : pathgen_perm_kernel<false>;
    cudaError_t e = ensure_smem((const void *)kern, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = ctas_per_sm((const void *)kern, kPathgenThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * sm_count;
    if (grid > a.total) grid = a.total;
    kern<<<(unsigned)grid, kPathgenThreads, smem, st>>>(a);
    return cudaGetLastError();
}

namespace {

using PathgenFn = void (*)(KArgs);

PathgenFn pathgen_fn(int mode, bool fp64) {
    switch (mode) {
        case kPaperRule: return fp64 ? pathgen_kernel<true, kPaperRule> : pathgen_kernel<false, kPaperRule>;
        case kEuropean: return fp64 ? pathgen_kernel<true, kEuropean> : pathgen_kernel<false, kEuropean>;
        case kBoundary: return fp64 ? pathgen_kernel<true, kBoundary> : pathgen_kernel<false, kBoundary>;
        case kStore16: return pathgen_kernel<false, kStore16>;
        default: return fp64 ? pathgen_kernel<true, kStore> : pathgen_kernel<false, kStore>;
    }
}

// Persistent grid: as many CTAs as fit on the SMs, at most one per tile.
cudaError_t pathgen_setup(const KArgs &a, int mode, bool fp64, int sm_count, PathgenFn *kern, size_t *smem,
                          int64_t *grid) {
    *smem = pathgen_layout(a.max_m, a.max_slots, fp64, mode).total;
    *kern = pathgen_fn(mode, fp64);
    cudaError_t e = ensure_smem((const void *)*kern, *smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = ctas_per_sm((const void *)*kern, kPathgenThreads, *smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    *grid = (int64_t)per_sm * sm_count;
    if (*grid > a.total) *grid = a.total;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_pathgen(const KArgs &a, bool fp64, int sm_count, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    PathgenFn kern;
    size_t smem;
    int64_t grid;
    if (a.h16 && fp64) return cudaErrorInvalidValue;
    cudaError_t e = pathgen_setup(a, a.h16 ? kStore16 : kStore, fp64, sm_count, &kern, &smem, &grid);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, kPathgenThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t pathgen_fused_grid(const KArgs &a, int mode, bool fp64, int sm_count, int64_t *grid) {
    PathgenFn kern;
    size_t smem;
    *grid = 0;
    if (a.total <= 0) return cudaSuccess;
    return pathgen_setup(a, mode, fp64, sm_count, &kern, &smem, grid);
}

cudaError_t launch_pathgen_fused(const KArgs &a, int mode, bool fp64, int64_t grid, cudaStream_t st) {
    if (a.total <= 0 || grid <= 0 || a.jobs != nullptr || mode == kStore || mode == kStore16)
        return cudaErrorInvalidValue;
    PathgenFn kern;
    size_t smem;
    int64_t g;
    cudaError_t e = pathgen_setup(a, mode, fp64, 1, &kern, &smem, &g);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, kPathgenThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace amc
