/*
 * FP64 CPU oracle for quasi-Monte Carlo American option pricing
 * (Cvetanoska & Stojanovski, "Using High Performance Computing and Monte
 * Carlo Simulation for Pricing American Options").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * executes this file; only the test-suite, the smoke check and the CPU
 * baseline leg and reference arm of the benchmark load it.  It shares no code, header, table
 * or constant generator with the CUDA path: the Sobol direction numbers are
 * expanded here from the raw Joe-Kuo (polynomial, initial numbers) data by
 * this file's own recurrence, the inverse normal is the root of Phi(z) = u
 * found by Halley iteration on libm's erfc, and every step is written out in
 * plain double precision, one path and one date at a time, in the order the
 * method states it.  Build: gcc -O2 -fopenmp (no -ffast-math).
 *
 * Passages followed (section / equation of the paper, plus the standard
 * definitions the paper relies on):
 *   points          §III.D  quasi-random points, mapped to N(0,1) by an
 *                           inverse cumulative normal;  Sobol' construction
 *                           with Joe-Kuo direction numbers, Gray-code order,
 *                           digital (XOR) shift from SplitMix64(seed).
 *   Brownian bridge ref. [13] (named, not described): breadth-first
 *                           bisection, left before right, floor midpoints.
 *   path update     Eq. 9   exact GBM step, evaluated in log space.
 *   exercise dates  §III.E, §V  t_j = j T/m, j = 1..m (Bermudan grid).
 *   LSM sweep       ref. [12] (Longstaff-Schwartz), §V backward induction.
 *   paper rule      Eqs. 10-11 with the Black-Scholes value of Eqs. 1-5 over
 *                           the last interval; average of Eq. 6.
 *   European        Eqs. 6-8.
 *   Black-Scholes   Eqs. 1-5 (Eq. 2 read with -d2, -d1 via Eq. 5).
 *
 * Parity pins (what fixes each function independently of this file) are
 * listed in the test-suite; every function below is pinned.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Threads the oracle's parallel loops use (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the threads of the oracle's parallel loops (no effect without OpenMP). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

#define ORC_PUT 0
#define ORC_CALL 1

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the digital shift of
 * dimension d is the high 32 bits of the d-th output (d = 0, 1, ...) of the
 * generator seeded with `seed`.                                             */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_digital_shifts(uint64_t seed, int m, uint32_t *shift)
{
    uint64_t state = seed;
    for (int d = 0; d < m; ++d)
        shift[d] = (uint32_t)(orc_splitmix64_next(&state) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Sobol' direction numbers (Bratley & Fox; Joe & Kuo 2008).
 * poly[d] is the primitive polynomial of dimension d written as an integer
 * whose bit s is the leading x^s term and whose bit 0 is the constant 1;
 * the bits in between are a_1..a_{s-1} (a_1 the coefficient of x^{s-1}).
 * vinit[d*stride + k] holds m_{k+1}, k = 0..s-1.  Dimension 0 is the van
 * der Corput sequence.  The output V[d*32 + b] is the 32-bit direction
 * number v_{b+1} = m_{b+1} * 2^(32-(b+1)).                                 */
int orc_sobol_directions(int m, const int64_t *poly, const int64_t *vinit,
                         int stride, uint32_t *V)
{
    for (int d = 0; d < m; ++d) {
        uint64_t mk[33];
        if (d == 0) {
            for (int k = 1; k <= 32; ++k) mk[k] = 1;
        } else {
            int64_t p = poly[d];
            int s = 0;
            while ((p >> (s + 1)) != 0) ++s;          /* degree */
            if (s < 1 || s > stride) return -1;
            for (int k = 1; k <= s && k <= 32; ++k) mk[k] = (uint64_t)vinit[d * stride + (k - 1)];
            for (int k = s + 1; k <= 32; ++k) {
                /* m_k = 2 a_1 m_{k-1} ^ 4 a_2 m_{k-2} ^ ... ^ 2^{s-1} a_{s-1} m_{k-s+1}
                 *       ^ 2^s m_{k-s} ^ m_{k-s}                                   */
                uint64_t v = mk[k - s] ^ (mk[k - s] << s);
                for (int q = 1; q <= s - 1; ++q) {
                    int a_q = (int)((p >> (s - q)) & 1);
                    if (a_q) v ^= mk[k - q] << q;
                }
                mk[k] = v;
            }
        }
        for (int k = 1; k <= 32; ++k) {
            if (mk[k] == 0 || (mk[k] & 1) == 0 || mk[k] >= (1ULL << k)) return -2;
            V[d * 32 + (k - 1)] = (uint32_t)(mk[k] << (32 - k));
        }
    }
    return 0;
}

/* Point i of dimension d by the definition: XOR of the direction numbers
 * selected by the bits of the Gray code of i.                               */
uint32_t orc_sobol_direct(const uint32_t *V, int d, uint64_t i)
{
    uint64_t g = i ^ (i >> 1);
    uint32_t x = 0;
    for (int b = 0; b < 32; ++b)
        if ((g >> b) & 1) x ^= V[d * 32 + b];
    return x;
}

/* Points i0..i0+n-1 of dims 0..m-1 (unshifted) in Gray-code order by the
 * recurrence x_i = x_{i-1} ^ v_{ctz(i)}, written to X[d*n + (i-i0)].        */
void orc_sobol_block(const uint32_t *V, int m, uint64_t i0, int64_t n, uint32_t *X)
{
    if (n <= 0) return;
    for (int d = 0; d < m; ++d) {
        uint32_t x = orc_sobol_direct(V, d, i0);
        X[(int64_t)d * n] = x;
        for (int64_t t = 1; t < n; ++t) {
            uint64_t i = i0 + (uint64_t)t;
            int c = 0;
            while (((i >> c) & 1) == 0) ++c;
            x ^= V[d * 32 + c];
            X[(int64_t)d * n + t] = x;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Standard normal distribution.  Phi by its erfc form; Phi^{-1}(u) as the
 * root of Phi(z) = u: a starting value from Abramowitz & Stegun 26.2.23
 * (|error| < 4.5e-4) refined by Halley's method, whose cubic convergence
 * takes it to the rounding level of erfc in two or three steps.  The lower
 * tail is solved directly and the upper tail by symmetry, so tail
 * probabilities keep full relative accuracy.                               */
double orc_norm_cdf(double x) { return 0.5 * erfc(-x * M_SQRT1_2); }

static double orc_norm_pdf(double x) { return exp(-0.5 * x * x) * 0.39894228040143267794; }

static double orc_lower_tail_icdf(double p) /* 0 < p <= 0.5 */
{
    double t = sqrt(-2.0 * log(p));
    double z = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                         (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    for (int it = 0; it < 4; ++it) {
        double e = (orc_norm_cdf(z) - p) / orc_norm_pdf(z);
        double dz = e / (1.0 + 0.5 * z * e);
        z -= dz;
        if (fabs(dz) <= 1e-17 * (1.0 + fabs(z))) break;
    }
    return z;
}

double orc_norm_icdf(double u)
{
    if (!(u > 0.0 && u < 1.0)) return u <= 0.0 ? -INFINITY : INFINITY;
    if (u <= 0.5) return orc_lower_tail_icdf(u);
    return -orc_lower_tail_icdf(1.0 - u);
}

/* Uniform of a 32-bit Sobol' integer: u = (x + 1/2) / 2^32, never 0 or 1. */
double orc_uniform(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

/* ------------------------------------------------------------------------ */
/* Brownian-bridge schedule.  Node 0 sets W(t_m) from coordinate 0; then the
 * intervals (l, r) are visited breadth-first, left before right, starting
 * from (0, m); an interval with r - l >= 2 gets node mid = floor((l+r)/2)
 * from the next coordinate.  Exactly m nodes for every m >= 1.
 * Outputs, per node k: date[k], left[k], right[k] (left = right = 0 marks
 * node 0, which is conditioned on W(0) = 0 only).                          */
int orc_bridge_schedule(int m, int *date, int *left, int *right)
{
    int *ql = (int *)malloc(sizeof(int) * (size_t)(2 * m + 2));
    int *qr = (int *)malloc(sizeof(int) * (size_t)(2 * m + 2));
    int head = 0, tail = 0, k = 0;
    if (!ql || !qr) { free(ql); free(qr); return -1; }
    date[0] = m; left[0] = 0; right[0] = 0; k = 1;
    ql[tail] = 0; qr[tail] = m; ++tail;
    while (head < tail) {
        int l = ql[head], r = qr[head]; ++head;
        if (r - l >= 2) {
            int mid = (l + r) / 2;
            date[k] = mid; left[k] = l; right[k] = r; ++k;
            ql[tail] = l; qr[tail] = mid; ++tail;
            ql[tail] = mid; qr[tail] = r; ++tail;
        }
    }
    free(ql); free(qr);
    return k == m ? 0 : -2;
}

/* Apply the bridge to one path: z[0..m-1] (coordinates) -> W[0..m]
 * (W[0] = 0, W[j] = W(t_j)), t_j = j*dt.                                   */
static void orc_bridge_apply(int m, double dt, const int *date, const int *left,
                             const int *right, const double *z, double *W)
{
    W[0] = 0.0;
    W[m] = sqrt(m * dt) * z[0];
    for (int k = 1; k < m; ++k) {
        double tl = left[k] * dt, tr = right[k] * dt, tm = date[k] * dt;
        W[date[k]] = ((tr - tm) * W[left[k]] + (tm - tl) * W[right[k]]) / (tr - tl) +
                     sqrt((tm - tl) * (tr - tm) / (tr - tl)) * z[k];
    }
}

/* The bridge as a linear map W = A z (A is m x m, row j-1 = date j): column
 * k is the bridge applied to the k-th unit coordinate vector.              */
int orc_bridge_matrix(int m, double T, double *A)
{
    int *date = (int *)malloc(sizeof(int) * (size_t)m);
    int *left = (int *)malloc(sizeof(int) * (size_t)m);
    int *right = (int *)malloc(sizeof(int) * (size_t)m);
    double *z = (double *)calloc((size_t)m, sizeof(double));
    double *W = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    int rc = -1;
    if (date && left && right && z && W && orc_bridge_schedule(m, date, left, right) == 0) {
        for (int k = 0; k < m; ++k) {
            z[k] = 1.0;
            orc_bridge_apply(m, T / m, date, left, right, z, W);
            for (int j = 1; j <= m; ++j) A[(j - 1) * m + k] = W[j];
            z[k] = 0.0;
        }
        rc = 0;
    }
    free(date); free(left); free(right); free(z); free(W);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Steps 1-3 for N paths: Sobol' integers (Gray order, point index = path
 * index, dimension = bridge coordinate), digital shift, uniform, inverse
 * normal, bridge, GBM in log space (Eq. 9 iterated from S_0 = S0):
 *   S_{i,j} = S0 exp((r - sigma^2/2) t_j + sigma W_i(t_j)).
 * Paths first..first+N-1 are generated; output S[(j-1)*N + (i-first)],
 * j = 1..m (date-major); optional W in the same layout.  Paths are
 * independent; OpenMP splits them in contiguous blocks, each starting its
 * Gray recurrence from the direct formula.                                 */
int orc_paths(double S0, double r, double sigma, double T, int m, int64_t N, int64_t first,
              const uint32_t *V, const uint32_t *shift, double *S, double *Wout)
{
    int *date = (int *)malloc(sizeof(int) * (size_t)m);
    int *left = (int *)malloc(sizeof(int) * (size_t)m);
    int *right = (int *)malloc(sizeof(int) * (size_t)m);
    int bad = 0;
    if (!date || !left || !right || orc_bridge_schedule(m, date, left, right) != 0) {
        free(date); free(left); free(right);
        return -1;
    }
    double dt = T / m;
    double mu = r - 0.5 * sigma * sigma;
    const int64_t BLK = 4096;
    int64_t nblk = (N + BLK - 1) / BLK;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t b = 0; b < nblk; ++b) {
        int64_t i0 = b * BLK, n = N - i0 < BLK ? N - i0 : BLK;
        uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m * n));
        double *z = (double *)malloc(sizeof(double) * (size_t)m);
        double *W = (double *)malloc(sizeof(double) * (size_t)(m + 1));
        if (!X || !z || !W) { bad |= 1; free(X); free(z); free(W); continue; }
        orc_sobol_block(V, m, (uint64_t)(first + i0), n, X);
        for (int64_t t = 0; t < n; ++t) {
            int64_t i = i0 + t;
            for (int k = 0; k < m; ++k)
                z[k] = orc_norm_icdf(orc_uniform(X[(int64_t)k * n + t] ^ shift[k]));
            orc_bridge_apply(m, dt, date, left, right, z, W);
            for (int j = 1; j <= m; ++j) {
                S[(int64_t)(j - 1) * N + i] = S0 * exp(mu * (j * dt) + sigma * W[j]);
                if (Wout) Wout[(int64_t)(j - 1) * N + i] = W[j];
            }
        }
        free(X); free(z); free(W);
    }
    free(date); free(left); free(right);
    return bad ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's randomisation (§III.D): each quasi-random array (dimension)
 * is permuted by a linear congruential generator.  Reading: path i takes
 * the unshifted Sobol' point pi_d(i) in dimension d, where
 *   pi_d(i) = L_d(i), repeated (L_d applied again) while the value is >= N,
 *   L_d(x) = (a_d x + c_d) mod M,  M = least power of two >= N,
 * with a_d = 1 mod 4 and c_d odd, so L_d has full period M (Hull-Dobell)
 * and walking its cycle back into 0..N-1 makes pi_d a permutation of them.
 * a_d = 4 (r_{2d} mod max(M/4, 1)) + 1 and c_d = (r_{2d+1} mod M) | 1 (mod M), with r_k
 * the k-th output of SplitMix64(seed).                                      */
uint64_t orc_lcg_modulus(int64_t N)
{
    uint64_t M = 1;
    while ((int64_t)M < N) M <<= 1;
    return M;
}

void orc_lcg_params(uint64_t seed, int m, int64_t N, uint64_t *a, uint64_t *c)
{
    uint64_t state = seed, M = orc_lcg_modulus(N);
    uint64_t q = M >= 4 ? M / 4 : 1;
    for (int d = 0; d < m; ++d) {
        uint64_t r0 = orc_splitmix64_next(&state), r1 = orc_splitmix64_next(&state);
        a[d] = (4 * (r0 % q) + 1) % M;
        c[d] = ((r1 % M) | 1) % M;
        if (M == 1) a[d] = c[d] = 0;
    }
}

uint64_t orc_lcg_perm(uint64_t a, uint64_t c, uint64_t M, int64_t N, uint64_t i)
{
    uint64_t x = (a * i + c) & (M - 1);
    while ((int64_t)x >= N) x = (a * x + c) & (M - 1);
    return x;
}

/* Paths as orc_paths, with the permuted unshifted points in place of the
 * digitally shifted ones (points 0..N-1 only).                             */
int orc_paths_permuted(double S0, double r, double sigma, double T, int m, int64_t N, const uint32_t *V,
                       const uint64_t *a, const uint64_t *c, double *S)
{
    int *date = (int *)malloc(sizeof(int) * (size_t)m);
    int *left = (int *)malloc(sizeof(int) * (size_t)m);
    int *right = (int *)malloc(sizeof(int) * (size_t)m);
    int bad = 0;
    if (!date || !left || !right || orc_bridge_schedule(m, date, left, right) != 0) {
        free(date); free(left); free(right);
        return -1;
    }
    const uint64_t M = orc_lcg_modulus(N);
    double dt = T / m;
    double mu = r - 0.5 * sigma * sigma;
#pragma omp parallel reduction(| : bad)
    {
        double *z = (double *)malloc(sizeof(double) * (size_t)m);
        double *W = (double *)malloc(sizeof(double) * (size_t)(m + 1));
        if (!z || !W) bad |= 1;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            if (!z || !W) continue;
            for (int k = 0; k < m; ++k) {
                uint64_t j = orc_lcg_perm(a[k], c[k], M, N, (uint64_t)i);
                z[k] = orc_norm_icdf(orc_uniform(orc_sobol_direct(V, k, j)));
            }
            orc_bridge_apply(m, dt, date, left, right, z, W);
            for (int j = 1; j <= m; ++j) S[(int64_t)(j - 1) * N + i] = S0 * exp(mu * (j * dt) + sigma * W[j]);
        }
        free(z); free(W);
    }
    free(date); free(left); free(right);
    return bad ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
static double orc_payoff(int type, double S, double K)
{
    double h = type == ORC_CALL ? S - K : K - S;
    return h > 0.0 ? h : 0.0;
}

/* Black-Scholes European value, Eqs. 1-5 (put with N(-d2), N(-d1)).       */
double orc_bs(int type, double S, double K, double r, double sigma, double T)
{
    double sq = sigma * sqrt(T);
    double d1 = (log(S / K) + (r + 0.5 * sigma * sigma) * T) / sq;
    double d2 = d1 - sq;
    double df = exp(-r * T);
    if (type == ORC_CALL) return S * orc_norm_cdf(d1) - K * df * orc_norm_cdf(d2);
    return K * df * orc_norm_cdf(-d2) - S * orc_norm_cdf(-d1);
}

/* ------------------------------------------------------------------------ */
/* Equilibrated Cholesky solve of the p x p normal equations G beta = b.
 * Equilibration: Gh = D^-1/2 G D^-1/2 with D = diag(G).  A pivot (diagonal
 * entry before its square root) <= 1e-12 marks the date as degenerate.
 * Returns 0 on success, 1 if degenerate.                                    */
int orc_solve_normal(int p, const double *G, const double *b, double *beta)
{
    double s[8], A[8][8], L[8][8], y[8], g[8];
    for (int k = 0; k < p; ++k) {
        if (!(G[k * p + k] > 0.0)) return 1;
        s[k] = 1.0 / sqrt(G[k * p + k]);
    }
    for (int k = 0; k < p; ++k)
        for (int l = 0; l < p; ++l) A[k][l] = G[k * p + l] * s[k] * s[l];
    for (int k = 0; k < p; ++k) {
        for (int l = 0; l <= k; ++l) {
            double acc = A[k][l];
            for (int q = 0; q < l; ++q) acc -= L[k][q] * L[l][q];
            if (l == k) {
                if (!(acc > 1e-12)) return 1;
                L[k][k] = sqrt(acc);
            } else {
                L[k][l] = acc / L[l][l];
            }
        }
    }
    for (int k = 0; k < p; ++k) {                 /* L y = D^-1/2 b */
        double acc = b[k] * s[k];
        for (int q = 0; q < k; ++q) acc -= L[k][q] * y[q];
        y[k] = acc / L[k][k];
    }
    for (int k = p - 1; k >= 0; --k) {            /* L^T g = y */
        double acc = y[k];
        for (int q = k + 1; q < p; ++q) acc -= L[q][k] * g[q];
        g[k] = acc / L[k][k];
    }
    for (int k = 0; k < p; ++k) beta[k] = g[k] * s[k];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Longstaff-Schwartz backward sweep (ref. [12]; backward induction of §V)
 * on the date-major paths S[(j-1)*N + i].  With the moneyness y = S/K - 1
 * and basis phi = (1, y, ..., y^{p-1}) (the same function space as
 * {1, S, ..., S^{p-1}}, so the same least-squares fit; centred so that the
 * in-the-money y lie in (-1, 0) for puts and (0, inf) for calls):
 *   CF_i = h(S_{i,m}), tau_i = m;
 *   for j = m-1 .. 1:
 *     CF_i <- CF_i e^{-r dt};
 *     I_j = { i : h(S_{i,j}) > 0 };
 *     G = sum_{I_j} phi phi^T,  b = sum_{I_j} phi CF_i   (plain FP64 sums,
 *         ascending path index);
 *     if |I_j| < p or a pivot <= 1e-12: no exercise at j (degenerate date);
 *     else beta_j = G^{-1} b and, for i in I_j, if h(S_{i,j}) > phi_i.beta_j
 *       then CF_i = h(S_{i,j}), tau_i = j;
 *   price = e^{-r dt} mean(CF),  std_err = e^{-r dt} sd(CF) / sqrt(N).
 * Outputs (all optional): beta[(j-1)*p + k] (zeros on degenerate dates and at
 * j = m), tau[i], cf[i] (CF at t_1, undiscounted to 0), n_itm[j-1],
 * deg[j-1] (1 on degenerate dates and at j = m, else 0).                   */
int orc_lsm(int type, double K, double r, double T, int m, int64_t N, int p,
            const double *S, double *out /* price, std_err, degenerate */,
            double *beta_out, int32_t *tau_out, double *cf_out, int64_t *nitm_out, int32_t *deg_out)
{
    double dt = T / m, disc = exp(-r * dt);
    double *CF = (double *)malloc(sizeof(double) * (size_t)N);
    int32_t *tau = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int degenerate = 0;
    if (!CF || !tau || p < 1 || p > 8) { free(CF); free(tau); return -1; }
    if (beta_out) memset(beta_out, 0, sizeof(double) * (size_t)(m * p));
    if (deg_out) for (int j = 0; j < m; ++j) deg_out[j] = 1;
    for (int64_t i = 0; i < N; ++i) {
        CF[i] = orc_payoff(type, S[(int64_t)(m - 1) * N + i], K);
        tau[i] = m;
    }
    if (nitm_out) {
        int64_t c = 0;
        for (int64_t i = 0; i < N; ++i) c += orc_payoff(type, S[(int64_t)(m - 1) * N + i], K) > 0.0;
        nitm_out[m - 1] = c;
    }
    for (int j = m - 1; j >= 1; --j) {
        const double *Sj = S + (int64_t)(j - 1) * N;
        double G[64], b[8], beta[8];
        int64_t nitm = 0;
        memset(G, 0, sizeof(G));
        memset(b, 0, sizeof(b));
        for (int64_t i = 0; i < N; ++i) CF[i] *= disc;
        for (int64_t i = 0; i < N; ++i) {
            double h = orc_payoff(type, Sj[i], K);
            if (!(h > 0.0)) continue;
            double y = Sj[i] / K - 1.0, phi[8];
            phi[0] = 1.0;
            for (int k = 1; k < p; ++k) phi[k] = phi[k - 1] * y;
            for (int k = 0; k < p; ++k) {
                for (int l = 0; l < p; ++l) G[k * p + l] += phi[k] * phi[l];
                b[k] += phi[k] * CF[i];
            }
            ++nitm;
        }
        if (nitm_out) nitm_out[j - 1] = nitm;
        if (nitm < p || orc_solve_normal(p, G, b, beta) != 0) {
            ++degenerate;
            continue;
        }
        if (beta_out)
            for (int k = 0; k < p; ++k) beta_out[(j - 1) * p + k] = beta[k];
        if (deg_out) deg_out[j - 1] = 0;
        for (int64_t i = 0; i < N; ++i) {
            double h = orc_payoff(type, Sj[i], K);
            if (!(h > 0.0)) continue;
            double y = Sj[i] / K - 1.0, c = 0.0, yk = 1.0;
            for (int k = 0; k < p; ++k) { c += beta[k] * yk; yk *= y; }
            if (h > c) { CF[i] = h; tau[i] = j; }
        }
    }
    double sum = 0.0, sum2 = 0.0;
    for (int64_t i = 0; i < N; ++i) sum += CF[i];
    double mean = sum / (double)N;
    for (int64_t i = 0; i < N; ++i) sum2 += (CF[i] - mean) * (CF[i] - mean);
    out[0] = disc * mean;
    out[1] = N > 1 ? disc * sqrt(sum2 / (double)(N - 1)) / sqrt((double)N) : 0.0;
    out[2] = (double)degenerate;
    if (tau_out) memcpy(tau_out, tau, sizeof(int32_t) * (size_t)N);
    if (cf_out) memcpy(cf_out, CF, sizeof(double) * (size_t)N);
    free(CF); free(tau);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Valuation with a given exercise boundary (a second Longstaff-Schwartz
 * pass; ref. [12] values out of sample, the paper in sample).  The
 * boundary is the continuation value c_j(y) = sum_k beta[(j-1)*p+k] y^k
 * (currency units, y = S/K - 1) of each date j with deg[j-1] == 0; dates
 * with deg[j-1] != 0 have no exercise.  On each path, the same recursion as
 * the in-sample sweep without its regression:
 *   CF = h(S_m), tau = m;
 *   for j = m-1 .. 1: CF <- CF e^{-r dt};
 *                     if deg[j-1] == 0 and h(S_j) > 0 and h(S_j) > c_j(y_j):
 *                         CF = h(S_j), tau = j;
 *   price = e^{-r dt} mean(CF),  std_err = e^{-r dt} sd(CF) / sqrt(N).
 * With the coefficients fitted on these same paths it repeats the in-sample
 * decisions; on paths independent of the fit it is a low-biased estimator
 * of the Bermudan value (any stopping rule is at most optimal).
 * Optional cf_out[(j-1)*N + i], j = 1..m: the cash flow of path i under this
 * boundary discounted to t_j, before the decision at t_j (for j = m, h(S_m)):
 * what the least-squares regression of date j (ref. [12]) is fitted to when
 * the decisions at the later dates are this boundary's.                    */
int orc_value_boundary(int type, double K, double r, double T, int m, int64_t N, int p, const double *S,
                       const double *beta, const int32_t *deg, double *out, int32_t *tau_out, double *cf_out)
{
    double dt = T / m, disc = exp(-r * dt);
    double *CF = (double *)malloc(sizeof(double) * (size_t)N);
    if (!CF || p < 1 || p > 8) { free(CF); return -1; }
    int degenerate = 0;
    for (int j = 1; j < m; ++j) degenerate += deg[j - 1] != 0;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double cf = orc_payoff(type, S[(int64_t)(m - 1) * N + i], K);
        int32_t tau = m;
        if (cf_out) cf_out[(int64_t)(m - 1) * N + i] = cf;
        for (int j = m - 1; j >= 1; --j) {
            cf *= disc;
            if (cf_out) cf_out[(int64_t)(j - 1) * N + i] = cf;
            if (deg[j - 1]) continue;
            double s = S[(int64_t)(j - 1) * N + i];
            double h = orc_payoff(type, s, K);
            if (!(h > 0.0)) continue;
            double y = s / K - 1.0, c = 0.0, yk = 1.0;
            for (int k = 0; k < p; ++k) { c += beta[(j - 1) * p + k] * yk; yk *= y; }
            if (h > c) { cf = h; tau = j; }
        }
        CF[i] = cf;
        if (tau_out) tau_out[i] = tau;
    }
    double sum = 0.0, sum2 = 0.0;
    for (int64_t i = 0; i < N; ++i) sum += CF[i];
    double mean = sum / (double)N;
    for (int64_t i = 0; i < N; ++i) sum2 += (CF[i] - mean) * (CF[i] - mean);
    out[0] = disc * mean;
    out[1] = N > 1 ? disc * sqrt(sum2 / (double)(N - 1)) / sqrt((double)N) : 0.0;
    out[2] = (double)degenerate;
    free(CF);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Dual upper bound of the Bermudan value for a given exercise boundary
 * (Andersen & Broadie's primal-dual method; the duality of Rogers and of
 * Haugh & Kogan that the paper's §IV lists among the methods for American
 * options).  The policy: at date j < m exercise if h(S_j) > 0, the date is
 * not degenerate and h(S_j) > c_j(y_j) (coefficients as in
 * orc_value_boundary); at maturity take h(S_m).  On outer path i (paths S,
 * discount factors to 0: D_j = e^{-r t_j}, Z_j = D_j h(S_j)):
 *   Q_j  = continuation value at t_j, discounted to t_j: the mean over
 *          n_in inner paths from S_j of the policy's payoff from t_{j+1} on,
 *          discounted to t_j (j = 1..m-1);
 *   L_j  = Z_j if the policy exercises at j, else D_j Q_j   (j = 1..m-1);
 *   L_m  = Z_m;
 *   M_0 = 0,  M_1 = L_1 - L0,  M_j = M_{j-1} + L_j - D_{j-1} Q_{j-1} (j >= 2),
 *   with L0 = mean over the outer paths of L_1 (an estimate of E_0 L_1);
 *   U_i = max_{j = 1..m} (Z_j - M_j);
 * upper = mean U_i, std_err = sd(U_i)/sqrt(N); out[2] = L0.
 * Inner path k from S_j: S <- S exp((r - sigma^2/2) dt + sigma sqrt(dt) z_s),
 * s = 1, 2, .. until the policy stops or t_m; the normals z are the quantile
 * of u = (x + 1/2) 2^-32, x the high 32 bits of output number
 *   c + 1 = (((i m + j - 1) n_in + k) m + s - 1) + 1
 * of SplitMix64(seed_in) (a counter-based stream: output n is the SplitMix64
 * mix of seed_in + n 0x9E3779B97F4A7C15).                                   */
static uint64_t orc_splitmix64_at(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Normal of inner step s (1-based) of inner path k from date j of outer
 * path i: the inner path owns H = ceil(m/2) consecutive SplitMix64 outputs,
 * numbers ((i m + j - 1) n_in + k) H + 1 .. + H; steps 2q-1 and 2q take the
 * high and the low 32 bits of its q-th output. */
double orc_dual_normal(uint64_t seed_in, int m, int64_t n_in, int64_t i, int j, int64_t k, int s)
{
    uint64_t H = ((uint64_t)m + 1u) / 2u;
    uint64_t n = (((uint64_t)i * (uint64_t)m + (uint64_t)(j - 1)) * (uint64_t)n_in + (uint64_t)k) * H
                 + (uint64_t)(s + 1) / 2u;
    uint64_t out = orc_splitmix64_at(seed_in, n);
    uint32_t x = (s & 1) ? (uint32_t)(out >> 32) : (uint32_t)out;
    return orc_norm_icdf(orc_uniform(x));
}

static int orc_policy_stops(int type, double K, int p, const double *beta, const int32_t *deg, int j, int m,
                            double S)
{
    if (j >= m) return 1;
    if (deg[j - 1]) return 0;
    double h = orc_payoff(type, S, K);
    if (!(h > 0.0)) return 0;
    double y = S / K - 1.0, c = 0.0, yk = 1.0;
    for (int q = 0; q < p; ++q) { c += beta[(j - 1) * p + q] * yk; yk *= y; }
    return h > c;
}

int orc_dual_upper(int type, double K, double r, double sigma, double T, int m, int64_t N, int p, const double *S,
                   const double *beta, const int32_t *deg, int64_t n_in, uint64_t seed_in, double *out, double *Ui)
{
    double dt = T / m, disc = exp(-r * dt), drift = (r - 0.5 * sigma * sigma) * dt, vol = sigma * sqrt(dt);
    double *Q = (double *)malloc(sizeof(double) * (size_t)(N * (m > 1 ? m - 1 : 1)));
    double *U = (double *)malloc(sizeof(double) * (size_t)N);
    if (!Q || !U || p < 1 || p > 8) { free(Q); free(U); return -1; }
    /* inner simulations: Q[i][j-1], discounted to t_j */
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < N; ++i) {
        for (int j = 1; j < m; ++j) {
            double acc = 0.0;
            for (int64_t k = 0; k < n_in; ++k) {
                double x = S[(int64_t)(j - 1) * N + i], v = 0.0, dk = 1.0;
                for (int s = 1; j + s <= m; ++s) {
                    x = x * exp(drift + vol * orc_dual_normal(seed_in, m, n_in, i, j, k, s));
                    dk *= disc;
                    if (orc_policy_stops(type, K, p, beta, deg, j + s, m, x)) { v = dk * orc_payoff(type, x, K); break; }
                }
                acc += v;
            }
            Q[i * (m - 1) + (j - 1)] = acc / (double)n_in;
        }
    }
    /* L0 = mean over the outer paths of L_1 */
    double L0 = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double S1 = S[i], L1;
        if (m == 1) L1 = disc * orc_payoff(type, S1, K);
        else L1 = orc_policy_stops(type, K, p, beta, deg, 1, m, S1) ? disc * orc_payoff(type, S1, K)
                                                                   : disc * Q[i * (m - 1)];
        L0 += L1;
    }
    L0 /= (double)N;
    double sum = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double Dj = 1.0, Mj = 0.0, best = -1e300, prevDQ = L0;
        for (int j = 1; j <= m; ++j) {
            Dj *= disc;
            double Sj = S[(int64_t)(j - 1) * N + i], Zj = Dj * orc_payoff(type, Sj, K), Lj, DQ = 0.0;
            if (j == m) Lj = Zj;
            else {
                DQ = Dj * Q[i * (m - 1) + (j - 1)];
                Lj = orc_policy_stops(type, K, p, beta, deg, j, m, Sj) ? Zj : DQ;
            }
            Mj += Lj - prevDQ;
            prevDQ = DQ;
            if (Zj - Mj > best) best = Zj - Mj;
        }
        U[i] = best;
        sum += best;
    }
    double mean = sum / (double)N, s2 = 0.0;
    for (int64_t i = 0; i < N; ++i) s2 += (U[i] - mean) * (U[i] - mean);
    out[0] = mean;
    out[1] = N > 1 ? sqrt(s2 / (double)(N - 1)) / sqrt((double)N) : 0.0;
    out[2] = L0;
    if (Ui) memcpy(Ui, U, sizeof(double) * (size_t)N);
    free(Q); free(U);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's own rule, Eqs. 10-11, written for calls and mirrored for
 * puts: on each path, V = max(h(S_{m-1}), BS(S_{m-1}, K, dt)) over the last
 * interval, then V = max(h(S_j), e^{-r dt} V) for j = m-2 .. 0 with
 * S_0 = S0; the price is the plain average of Eq. 6 (the stepwise discount
 * already brings V to t = 0).  For m = 1 this is max(h(S0), BS(S0, K, T)).  */
int orc_paper_ub(int type, double S0, double K, double r, double sigma, double T,
                 int m, int64_t N, const double *S, double *out)
{
    double dt = T / m, disc = exp(-r * dt), sum = 0.0, sum2 = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double Slast = m >= 2 ? S[(int64_t)(m - 2) * N + i] : S0;
        double h = orc_payoff(type, Slast, K), c = orc_bs(type, Slast, K, r, sigma, dt);
        double V = h > c ? h : c;
        for (int j = m - 2; j >= 0; --j) {
            double Sj = j >= 1 ? S[(int64_t)(j - 1) * N + i] : S0;
            double hj = orc_payoff(type, Sj, K), cont = disc * V;
            V = hj > cont ? hj : cont;
        }
        sum += V;
        sum2 += V * V;
    }
    double mean = sum / (double)N;
    double var = N > 1 ? (sum2 - (double)N * mean * mean) / (double)(N - 1) : 0.0;
    out[0] = mean;
    out[1] = var > 0.0 ? sqrt(var / (double)N) : 0.0;
    out[2] = 0.0;
    return 0;
}

/* European value by Eqs. 6-8: e^{-rT} times the mean payoff at t_m = T.     */
int orc_european(int type, double K, double r, double T, int m, int64_t N,
                 const double *S, double *out)
{
    double sum = 0.0, sum2 = 0.0, df = exp(-r * T);
    for (int64_t i = 0; i < N; ++i) {
        double h = orc_payoff(type, S[(int64_t)(m - 1) * N + i], K);
        sum += h;
        sum2 += h * h;
    }
    double mean = sum / (double)N;
    double var = N > 1 ? (sum2 - (double)N * mean * mean) / (double)(N - 1) : 0.0;
    out[0] = df * mean;
    out[1] = var > 0.0 ? df * sqrt(var / (double)N) : 0.0;
    out[2] = 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Frozen-boundary pathwise Greeks of the estimator e^{-r t_tau} h(S_tau):
 *   dS_tau/dS0 = S_tau / S0,   dS_tau/dsigma = S_tau (W_tau - sigma t_tau),
 * h'(S) = -1[S < K] (put), +1[S > K] (call).  tau[i] in 1..m; W in the
 * date-major layout of orc_paths.  out = (price, delta, vega).             */
int orc_pathwise_greeks(int type, double S0, double K, double r, double sigma,
                        double T, int m, int64_t N, const double *S, const double *W,
                        const int32_t *tau, double *out)
{
    double dt = T / m, sp = 0.0, sd = 0.0, sv = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        int j = tau[i];
        if (j < 1 || j > m) return -1;
        double St = S[(int64_t)(j - 1) * N + i], Wt = W[(int64_t)(j - 1) * N + i];
        double t = j * dt, df = exp(-r * t);
        double h = orc_payoff(type, St, K);
        if (!(h > 0.0)) continue;
        double dh = type == ORC_CALL ? 1.0 : -1.0;
        sp += df * h;
        sd += df * dh * St / S0;
        sv += df * dh * St * (Wt - sigma * t);
    }
    out[0] = sp / (double)N;
    out[1] = sd / (double)N;
    out[2] = sv / (double)N;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cox-Ross-Rubinstein binomial tree with n steps (n a multiple of m when
 * bermudan != 0).  Bermudan: exercise only at the steps that coincide with
 * t_1..t_m (not at t = 0).  American: exercise at every node including the
 * root.  u = e^{sigma sqrt(d)}, q = (e^{r d} - 1/u)/(u - 1/u).              */
double orc_crr(int type, double S0, double K, double r, double sigma, double T,
               int n, int m, int bermudan)
{
    double d = T / n, u = exp(sigma * sqrt(d)), dn = 1.0 / u;
    double q = (exp(r * d) - dn) / (u - dn), df = exp(-r * d);
    double *v = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!v || (bermudan && (m < 1 || n % m != 0))) { free(v); return NAN; }
    int every = bermudan ? n / m : 1;
    for (int k = 0; k <= n; ++k) v[k] = orc_payoff(type, S0 * pow(u, 2 * k - n), K);
    for (int s = n - 1; s >= 0; --s) {
        int can = bermudan ? (s > 0 && s % every == 0) : 1;
        for (int k = 0; k <= s; ++k) {
            double cont = df * (q * v[k + 1] + (1.0 - q) * v[k]);
            if (can) {
                double h = orc_payoff(type, S0 * pow(u, 2 * k - s), K);
                v[k] = h > cont ? h : cont;
            } else {
                v[k] = cont;
            }
        }
    }
    double res = v[0];
    free(v);
    return res;
}
