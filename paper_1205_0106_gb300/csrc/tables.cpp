// Host-side tables and plans: Sobol' direction numbers, digital shifts,
// Brownian-bridge schedule and its depth-first evaluation plan, option
// validation and the sweep launch plan.  Pure host code (no CUDA calls), so
// every function here is testable without a GPU through the C ABI.
#include <algorithm>
#include <math.h>
#include <string.h>

#include <deque>
#include <vector>

#include "internal.h"
#include "joe_kuo_raw.h"

namespace amc {

// Direction numbers (Bratley & Fox recurrence on the Joe & Kuo data).  For
// dimension d >= 1 with primitive polynomial of degree s and interior
// coefficients a_1..a_{s-1}, the odd integers m_k (k > s) follow
//   m_k = m_{k-s} xor 2^s m_{k-s} xor  xor_{q=1}^{s-1} 2^q a_q m_{k-q},
// and the 32-bit direction number is v_k = m_k << (32 - k).  Dimension 0 is
// van der Corput (all m_k = 1).  V[d*32 + b] = v_{b+1}.
int host_directions(int n_dims, uint32_t *V) {
    if (n_dims < 1 || n_dims > AMC_JK_DIMS) return AMC_EINVAL;
    for (int d = 0; d < n_dims; ++d) {
        uint64_t mk[32];
        if (d == 0) {
            for (int k = 0; k < 32; ++k) mk[k] = 1;
        } else {
            const uint32_t poly = amc_jk_poly[d];
            int s = 31 - __builtin_clz(poly);
            if (s < 1 || s > AMC_JK_WIDTH) return AMC_EINVAL;
            const uint32_t a = (poly >> 1) & ((1u << (s - 1)) - 1u);
            for (int k = 0; k < s; ++k) mk[k] = amc_jk_minit[d][k];
            for (int k = s; k < 32; ++k) {
                uint64_t v = mk[k - s] ^ (mk[k - s] << s);
                for (int q = 1; q < s; ++q)
                    if ((a >> (s - 1 - q)) & 1u) v ^= mk[k - q] << q;
                mk[k] = v;
            }
        }
        for (int b = 0; b < 32; ++b) V[d * 32 + b] = (uint32_t)(mk[b] << (31 - b));
    }
    return AMC_OK;
}

// Digital shift of dimension d: the high word of the d-th output of
// SplitMix64 (Steele, Lea & Flood 2014) started from `seed`.
// Parameters of the paper's LCG permutation of the quasi-random points
// (§III.D): modulus M = least power of two >= n_points, per dimension
// a_d = 4 (r_{2d} mod max(M/4, 1)) + 1 (a_d = 1 mod 4) and c_d = (r_{2d+1}
// mod M) | 1 (odd), r_k the SplitMix64 outputs of the seed: a full-period
// generator (Hull-Dobell), walked back into 0..n_points-1 by the kernel.
void host_lcg_params(uint64_t seed, int n_dims, int64_t n_points, uint32_t *a, uint32_t *c, uint64_t *M_out) {
    uint64_t M = 1;
    while ((int64_t)M < n_points) M <<= 1;
    const uint64_t q = M >= 4 ? M / 4 : 1;
    uint64_t x = seed;
    auto next = [&]() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int d = 0; d < n_dims; ++d) {
        const uint64_t r0 = next(), r1 = next();
        a[d] = M == 1 ? 0u : (uint32_t)((4 * (r0 % q) + 1) % M);
        c[d] = M == 1 ? 0u : (uint32_t)(((r1 % M) | 1u) % M);
    }
    *M_out = M;
}

void host_shifts(uint64_t seed, int n_dims, uint32_t *out) {
    uint64_t x = seed;
    for (int d = 0; d < n_dims; ++d) {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[d] = (uint32_t)(z >> 32);
    }
}

// Breadth-first bridge schedule in coordinate order: coordinate 0 fills
// t_m from W(0) = 0; then intervals are split at floor((l+r)/2),
// breadth-first, left before right, one coordinate per split.
int host_bridge_bfs(int m, int32_t *date, int32_t *left, int32_t *right) {
    if (m < 1 || m > AMC_MAX_STEPS) return AMC_EINVAL;
    int k = 0;
    date[k] = m; left[k] = 0; right[k] = 0; ++k;
    std::deque<std::pair<int, int>> q;
    q.emplace_back(0, m);
    while (!q.empty()) {
        auto iv = q.front();
        q.pop_front();
        if (iv.second - iv.first < 2) continue;
        int mid = (iv.first + iv.second) / 2;
        date[k] = mid; left[k] = iv.first; right[k] = iv.second; ++k;
        q.emplace_back(iv.first, mid);
        q.emplace_back(mid, iv.second);
    }
    return k == m ? AMC_OK : AMC_EINVAL;
}

// Depth-first evaluation plan of the same bridge.  A node only needs the W
// of its interval end points, which are its ancestors; with one stack slot
// per tree depth those are always resident, so a path needs depth+1 slots
// instead of m values of shared memory.  W(0) = 0 needs none: a node on
// [0, r] has no left term (wl = 0, and it reads its right end point's slot
// in place of a left one), and the root has no terms at all (wl = wr = 0,
// reading its own slot); the kernels start every slot at 0, so these reads
// with weight 0 always meet finite values.
int host_bridge_plan(int m, BridgePlan *plan) {
    std::vector<int32_t> date(m), left(m), right(m);
    int rc = host_bridge_bfs(m, date.data(), left.data(), right.data());
    if (rc != AMC_OK) return rc;
    std::vector<int> coord_of_date(m + 1, -1), slot_of_date(m + 1, -1);
    for (int k = 0; k < m; ++k) coord_of_date[date[k]] = k;
    plan->m = m;
    plan->nf.clear();
    plan->nd.clear();
    int maxdepth = 0;
    auto emit = [&](int d, int l, int r, int depth) {
        NodeD n{};
        n.coord = coord_of_date[d];
        n.date = d;
        n.so = (int16_t)depth;
        if (depth == 0) {                               // W(t_m) = sqrt(t_m) z_0
            n.sl = n.sr = 0;
            n.wl = n.wr = 0.0;
            n.sdu = sqrt((double)m);
        } else {                                        // r >= 1: an earlier node's date
            n.sr = (int16_t)slot_of_date[r];
            n.sl = (int16_t)(l == 0 ? n.sr : slot_of_date[l]);
            n.wl = l == 0 ? 0.0 : (double)(r - d) / (double)(r - l);   // W(0) = 0: no left term
            n.wr = (double)(d - l) / (double)(r - l);
            n.sdu = sqrt((double)(d - l) * (double)(r - d) / (double)(r - l));
        }
        slot_of_date[d] = depth;
        plan->nd.push_back(n);
    };
    // first pass: depth of the tree
    std::vector<std::pair<std::pair<int, int>, int>> st;
    st.push_back({{0, m}, 1});
    while (!st.empty()) {
        auto e = st.back();
        st.pop_back();
        int l = e.first.first, r = e.first.second;
        if (r - l < 2) continue;
        if (e.second > maxdepth) maxdepth = e.second;
        int mid = (l + r) / 2;
        st.push_back({{mid, r}, e.second + 1});
        st.push_back({{l, mid}, e.second + 1});
    }
    plan->nslots = maxdepth + 1;
    if (plan->nslots > kMaxSlots) return AMC_EINVAL;
    emit(m, 0, 0, 0);
    // second pass: depth-first, left subtree first
    st.push_back({{0, m}, 1});
    while (!st.empty()) {
        auto e = st.back();
        st.pop_back();
        int l = e.first.first, r = e.first.second;
        if (r - l < 2) continue;
        int mid = (l + r) / 2;
        emit(mid, l, r, e.second);
        st.push_back({{mid, r}, e.second + 1});
        st.push_back({{l, mid}, e.second + 1});
    }
    if ((int)plan->nd.size() != m) return AMC_EINVAL;
    for (const NodeD &n : plan->nd) {
        NodeF f{};
        f.coord = n.coord; f.date = n.date; f.sl = n.sl; f.sr = n.sr; f.so = n.so;
        f.wl = (float)n.wl; f.wr = (float)n.wr; f.sdu = (float)n.sdu;
        plan->nf.push_back(f);
    }
    return AMC_OK;
}

int host_validate(const amc_option *o) {
    if (!o) return AMC_EINVAL;
    auto pos = [](double v) { return isfinite(v) && v > 0.0; };
    if (!pos(o->S0) || !pos(o->K) || !pos(o->sigma) || !pos(o->T) || !isfinite(o->r)) return AMC_EINVAL;
    if (o->n_steps < 1 || o->n_steps > AMC_MAX_STEPS) return AMC_EINVAL;
    if (o->n_paths < 1 || o->n_paths > AMC_MAX_PATHS) return AMC_EINVAL;
    if (o->type != AMC_PUT && o->type != AMC_CALL) return AMC_EINVAL;
    if (o->rule != AMC_RULE_LSM && o->rule != AMC_RULE_PAPER_UB && o->rule != AMC_RULE_EUROPEAN)
        return AMC_EINVAL;
    if (o->rule == AMC_RULE_LSM && (o->basis < 1 || o->basis > 4)) return AMC_EINVAL;
    return AMC_OK;
}

int64_t host_ld(int64_t n_paths) { return (n_paths + 31) / 32 * 32; }

// Sweep launch plan of one option.  Mixed-precision LSM: one 1024-thread
// CTA per 7680 paths, at most one CTA per SM (co-resident).  Otherwise:
// CTAs of kSweepThreads threads, each thread owning `chunks` groups of 4
// consecutive paths, the fewest chunks per thread (1, 2, 4, 8) whose CTA
// count fits the co-resident capacity sweep_ctas_per_sm(chunks) * SMs.
// Depends on the path count, precision, rule and SM count only, so an
// option's reduction order is the same alone or batched.
int host_plan_sweep(int64_t n_paths, int sm_count, int prec, int rule, SweepPlan *p, int max_cluster) {
    if (n_paths < 1 || sm_count < 1) return AMC_EINVAL;
    const bool mixed_lsm = (prec == AMC_MIXED || prec == AMC_MIXED16) && rule == AMC_RULE_LSM;
    if (mixed_lsm && max_cluster >= 1 &&
        n_paths <= (int64_t)std::min(max_cluster, kClMaxCluster) * kClPathsPerCta) {
        p->kind = 3;                                  // one cluster per option
        p->chunks = kClPPT;
        p->ctas = (int)((n_paths + kClPathsPerCta - 1) / kClPathsPerCta);
        return AMC_OK;
    }
    if (mixed_lsm) {
        const int64_t g = (n_paths + kV2PathsPerCta - 1) / kV2PathsPerCta;
        if (g > sm_count || g > kV2MaxCtas) return AMC_EINVAL;   // per-path state must stay on chip
        p->kind = 2;
        p->chunks = kV2PPT;
        p->ctas = (int)g;
        return AMC_OK;
    }
    for (int c = 1; c <= 8; c *= 2) {
        const int64_t cap = (int64_t)sweep_ctas_per_sm(c) * sm_count;
        const int64_t per_cta = (int64_t)kSweepThreads * 4 * c;
        const int64_t g = (n_paths + per_cta - 1) / per_cta;
        if (g <= cap) {
            p->kind = 1;
            p->chunks = c;
            p->ctas = (int)g;
            return AMC_OK;
        }
    }
    return AMC_EINVAL;                                // too many paths to keep in registers
}

int plan_for_greeks(int64_t n_paths, int sm_count, SweepPlan *p) {
    return host_plan_sweep(n_paths, sm_count, AMC_MIXED, AMC_RULE_LSM, p, 0);
}

}  // namespace amc
