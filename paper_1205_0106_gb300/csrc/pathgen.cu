// Path generation (steps 1-3 of the hot path) for sm_103a:
//   Sobol' integers (Gray-code order, digital XOR shift)      §III.D
//   -> uniform (x + 1/2) 2^-32 -> N(0,1)                      §III.D (Moro)
//   -> Brownian bridge (breadth-first coordinate order,       ref. [13]
//      evaluated depth-first with a per-path slot stack)
//   -> GBM in log space, S = S0 exp((r - sigma^2/2) t + sigma W)   Eq. 9
//   -> date-major store S[j-1][i], coalesced across the warp.
//
// One CTA of 128 threads owns a tile of 512 consecutive Sobol' points; thread
// t owns points tile + q*128 + t (q = 0..3).  Because the Gray code is
// linear over GF(2) and these index parts occupy disjoint bits,
//   x(tile + q*128 + t) = x(tile + q*128) xor x(t),
// so the per-CTA part is computed once per tile (shared memory) and the
// per-thread part needs only the low 7 direction numbers of a dimension.
#include <cuda_runtime.h>
#include <math.h>

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

// Inverse cumulative normal in FP32 after Moro (1995): a rational function
// of (u - 1/2)^2 for |u - 1/2| < 0.42 and a degree-8 polynomial in
// log(-log p), p = min(u, 1 - u), in the tails.  The uniform comes straight
// from the 32-bit integer: u - 1/2 = (x - 2^31 + 1/2) 2^-32 from the signed
// offset, and the tail probability from x or its complement, so neither
// rounds to 0 or 1 in single precision.
__device__ __forceinline__ float icdf_moro(uint32_t x) {
    const int32_t d = (int32_t)(x ^ 0x80000000u);           // x - 2^31
    const float y = fmaf((float)d, 0x1p-32f, 0x1p-33f);      // u - 1/2
    float z;
    if (fabsf(y) < 0.42f) {
        const float r = y * y;
        const float num = fmaf(fmaf(fmaf(-25.44106049637f, r, 41.39119773534f), r, -18.61500062529f), r,
                               2.50662823884f);
        const float den = fmaf(fmaf(fmaf(fmaf(3.13082909833f, r, -21.06224101826f), r, 23.08336743743f), r,
                                    -8.47351093090f), r, 1.0f);
        z = y * __fdividef(num, den);
    } else {
        const uint32_t xs = (x & 0x80000000u) ? ~x : x;
        const float p = fmaf((float)xs, 0x1p-32f, 0x1p-33f);
        const float t = __logf(-__logf(p));
        float c = fmaf(0.0000003960315187f, t, 0.0000002888167364f);
        c = fmaf(c, t, 0.0000321767881768f);
        c = fmaf(c, t, 0.0003951896511919f);
        c = fmaf(c, t, 0.0038405729373609f);
        c = fmaf(c, t, 0.0276438810333863f);
        c = fmaf(c, t, 0.1607979714918209f);
        c = fmaf(c, t, 0.9761690190917186f);
        c = fmaf(c, t, 0.3374754822726147f);
        z = y < 0.0f ? -c : c;
    }
    return z;
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

__device__ __forceinline__ int find_job_by_tile(const Job *__restrict__ jobs, int n_jobs, int64_t tile) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool FP64>
__global__ void __launch_bounds__(kPathgenThreads) pathgen_kernel(const __grid_constant__ KArgs a) {
    using Real = typename PG<FP64>::Real;
    using Node = typename PG<FP64>::Node;
    extern __shared__ __align__(16) unsigned char smem[];
    const int max_m = a.max_m;
    Node *s_nodes = reinterpret_cast<Node *>(smem);
    uint32_t *s_xq = reinterpret_cast<uint32_t *>(s_nodes + max_m);      // [Q][m]
    uint32_t *s_vt = s_xq + kPathgenQ * max_m;                            // [m][8] low direction numbers
    Real *s_W = reinterpret_cast<Real *>(s_vt + 8 * max_m);              // [slot][Q][128]

    const uint32_t *__restrict__ V = a.V;
    const int tid = threadIdx.x;
    const uint32_t gt = (uint32_t)tid ^ ((uint32_t)tid >> 1);            // Gray code of t (7 bits)
    int cur = -1;
    int m = 0, nslots = 0;
    for (int64_t tile = blockIdx.x; tile < a.total; tile += gridDim.x) {
        const int jb = a.jobs ? find_job_by_tile(a.jobs, a.n_jobs, tile) : 0;
        const Job &J = a.jobs ? a.jobs[jb] : a.one;
        const uint32_t base = (uint32_t)((tile - J.tile_begin) * kTilePoints);
        const uint32_t *__restrict__ shift = a.jobs ? J.shift : a.shift_one;
        __syncthreads();                                                  // previous tile done with smem
        if (jb != cur) {
            m = J.m;
            nslots = J.nslots;
            const Node *gn = reinterpret_cast<const Node *>(J.nodes);
            for (int i = tid; i < m; i += kPathgenThreads) s_nodes[i] = gn[i];
            for (int i = tid; i < m * 8; i += kPathgenThreads)
                s_vt[i] = (i & 7) < 7 ? __ldg(V + (i >> 3) * 32 + (i & 7)) : 0u;
            cur = jb;
        }
        for (int i = tid; i < kPathgenQ * m; i += kPathgenThreads) {
            const int q = i / m, k = i - q * m;
            s_xq[i] = sobol_direct(V, k, base + (uint32_t)q * kPathgenThreads) ^ shift[k];
        }
        const int zero = nslots - 1;
#pragma unroll
        for (int q = 0; q < kPathgenQ; ++q) s_W[(zero * kPathgenQ + q) * kPathgenThreads + tid] = Real(0);
        __syncthreads();

        const int64_t N = J.N, ld = J.ld;
        Real *__restrict__ S = reinterpret_cast<Real *>(J.S);
        const double mu = J.r - 0.5 * J.sigma * J.sigma;
        const Real sqdt = (Real)sqrt(J.dt);
        const Real S0 = (Real)J.S0;
        // exponent per node: FP32 in base 2 (ex2), FP64 in base e
        const Real mu_dt = FP64 ? (Real)(mu * J.dt) : (Real)(mu * J.dt * 1.4426950408889634);
        const Real sig = FP64 ? (Real)J.sigma : (Real)(J.sigma * 1.4426950408889634);

        for (int n = 0; n < m; ++n) {
            const Node nd = s_nodes[n];
            uint32_t xt = 0;
            const uint32_t *vt = s_vt + nd.coord * 8;
#pragma unroll
            for (int b = 0; b < 7; ++b)
                if ((gt >> b) & 1u) xt ^= vt[b];
            const Real wl = (Real)nd.wl, wr = (Real)nd.wr, sd = (Real)nd.sdu * sqdt;
            const Real drift = mu_dt * (Real)nd.date;
            Real *__restrict__ row = S + (int64_t)(nd.date - 1) * ld;
            const Real *Wl = s_W + (nd.sl * kPathgenQ) * kPathgenThreads + tid;
            const Real *Wr = s_W + (nd.sr * kPathgenQ) * kPathgenThreads + tid;
            Real *Wo = s_W + (nd.so * kPathgenQ) * kPathgenThreads + tid;
#pragma unroll
            for (int q = 0; q < kPathgenQ; ++q) {
                const uint32_t x = xt ^ s_xq[q * m + nd.coord];
                Real z;
                if (FP64) z = (Real)normcdfinv(((double)x + 0.5) * 0x1p-32);
                else z = (Real)icdf_moro(x);
                const Real W = wl * Wl[q * kPathgenThreads] + wr * Wr[q * kPathgenThreads] + sd * z;
                Wo[q * kPathgenThreads] = W;
                Real s;
                if (FP64) s = S0 * (Real)exp((double)(drift + sig * W));
                else s = S0 * exp2f((float)(drift + sig * W));
                const int64_t i = (int64_t)base + q * kPathgenThreads + tid;
                if (i < N) row[i] = s;
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

size_t pathgen_smem_bytes(int max_m, int nslots, bool fp64) {
    size_t node = fp64 ? sizeof(NodeD) : sizeof(NodeF);
    size_t real = fp64 ? 8 : 4;
    (void)nslots;
    return node * max_m + 4u * kPathgenQ * max_m + 4u * 8 * max_m +
           real * kMaxSlots * kPathgenQ * kPathgenThreads;
}

cudaError_t launch_sobol(const uint32_t *V, int n_dims, int64_t n_points, const uint32_t *shift,
                         uint32_t *x, int64_t ld, cudaStream_t st) {
    if (n_points <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n_points + 255) / 256), (unsigned)n_dims);
    sobol_kernel<<<grid, 256, 0, st>>>(V, n_dims, n_points, shift, x, ld);
    return cudaGetLastError();
}

cudaError_t launch_pathgen(const KArgs &a, bool fp64, int sm_count, cudaStream_t st) {
    const int64_t total_tiles = a.total;
    if (total_tiles <= 0) return cudaSuccess;
    size_t smem = pathgen_smem_bytes(a.max_m, kMaxSlots, fp64);
    auto kern = fp64 ? pathgen_kernel<true> : pathgen_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPathgenThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * sm_count;
    if (grid > total_tiles) grid = total_tiles;
    kern<<<(unsigned)grid, kPathgenThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace amc
