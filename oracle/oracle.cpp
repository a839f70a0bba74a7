// Plain CPU oracle of the cluster-preserving correction pass.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark load this library.  It shares no code, header,
// constant generator or helper with the CUDA path and never calls it.
//
// Every function follows one step of the method in the order the paper gives
// it (arXiv 2604.18801, Sec. 2.4 and Sec. 3, Algorithm 1, Eq. 1-3), written
// for a reader who checks it against the paper by eye: sequential loops,
// std::sort, a textbook union-find, Kruskal for the halo forest, and the
// projected Adam iteration in float64.  Nothing is blocked, fused or reordered
// beyond what the method states.
//
// Readings the paper leaves open (they are fixed here and mirrored by the
// CUDA path):
//  * Link tests use one canonical float32 formula on the original float32
//    coordinates: dx = xi - xj (float32), minimum image by one add/subtract
//    of the box length when |dx| > L/2 (periodic boxes only), then
//    d2 = (dx*dx + dy*dy) + dz*dz with every operation rounded to float32 and
//    no fused multiply-add.  A pair is linked iff d2 <= fl32(b*b) (Sec. 2.4,
//    "d <= b", ties linked).
//  * The vulnerability window (Sec. 3.1) is evaluated on the same d2 with
//    float32 bounds lo2 = fl32((b-2sqrt3 xi)^2 (1-2^-20)) (or -1 when
//    b <= 2 sqrt3 xi: no safe links) and hi2 = fl32((b+2sqrt3 xi)^2 (1+2^-20)).
//    Classes: safe d2 <= lo2; potentially broken lo2 < d2 <= b2;
//    potentially created b2 < d2 <= hi2.
//  * Edit quantization (Sec. 3.3): codes q in [0, 2^m-1] over [-2 xi, 2 xi]
//    with step s = 4 xi/(2^m-1), so the error is at most s/2 = 2 xi/(2^m-1),
//    the paper's eps_q.  The projection box is xi_box = xi - eps_q - u, where
//    u = ulp_f32(M + 2 xi) and M is the largest coordinate magnitude; the
//    tight margin is delta_t = 2 sqrt3 (eps_q + u) + b 2^-20.  With these the
//    decoded output stays within xi and keeps the untightened loss at zero.
//  * Learning rate and Adam epsilon are scaled to the error bound:
//    alpha = alpha_rel * xi, eps_adam = eps_rel * xi (Sec. 4.2 gives them in
//    unstated data units).
//  * Halo forest: the spanning forest kept is the unique minimum spanning
//    forest under the key (float32 bits of d2, i, j) (Sec. 3.2 leaves the
//    forest unspecified).
//  * The current pair offset and distance are evaluated symmetrically: the
//    offset is dp + (delta_i - delta_j) rounded once, and |r| adds the squared
//    components smallest first.  The quantizer lattice makes mirror-image pairs
//    common; their gradient terms then cancel exactly, as in exact arithmetic.
//    (Adam's normalised step turns a last-bit asymmetry into an O(xi) move.)
//  * When a pair's current distance is at most b * 2^-30 (coincident points:
//    the quantizer lattice makes them common, and rounding turns an exact
//    zero into noise), its gradient direction is the original separation.
//  * Stall reset (not in the paper).  The loss is non-convex (the false-link
//    term), and at large xi / b PGD can settle in a local minimum where a few
//    non-link pairs sit well inside b with an endpoint on the box.  The original
//    positions P satisfy every constraint (Sec. 3.3, convergence analysis), so:
//    the loss of each check is also measured in fixed point, as the sum over violated pairs of
//    llrint(v^2 / (xi^2 2^-24)); a check makes progress when that value is
//    below best - floor(best / 1024), and best is the lowest value since the
//    last reset (it starts at check 0).  After `patience` consecutive checks
//    without progress (stall_patience at first, doubled after every reset, so
//    that a slow tail of tiny violations is disturbed less and less often), the
//    next check resets every editable particle that is an endpoint of a
//    violated pair to its original position (delta = 0), provided the RMS
//    violation of the violated pairs exceeds xi / 1024 (the fixed-point loss is
//    above 16 units per violated pair; a slow tail of tiny violations is left
//    to Adam), and
//    clears its Adam moments instead of taking its Adam step; the other
//    particles take their step.  The check after a reset starts a new best.
//    stall_patience = 0 turns this off.
//  * Threads.  Built with OpenMP, the pair search splits the particles among
//    threads and sorts the pairs afterwards, the PGD computes each pair's terms
//    independently and then sums them in pair order, and the Adam update takes
//    each coordinate on its own: results are the same bits for any thread count.
//  * Counting a violation.  A pair with violation v > 0 takes its loss term and
//    gradient; it counts as violated (the count that stops the loop at eps_L = 0,
//    and the stall rule's count) only when v > b * 2^-40.  Pairs held from both
//    sides with an endpoint on the box can settle at v -> 0+, where whether v is
//    above zero depends on the last bits of the arithmetic; b * 2^-40 is far below
//    the b * 2^-20 slack of the margin dt, so the decoded guarantee is unchanged.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// Parameters of one correction problem (Algorithm 1 REQUIRE line plus Adam).
typedef struct {
    double b;            // linking length
    double xi;           // pointwise absolute error bound
    double box_lo[3];    // box (periodic boxes: [lo, hi) per axis)
    double box_hi[3];
    int32_t periodic;    // 1 = minimum-image distances in the box
    int32_t mode;        // 0 = VP, 1 = SC, 2 = HF
    int32_t m_bits;      // edit bit depth m
    int32_t t_max;       // maximum number of updates
    double alpha_rel;    // learning rate / xi
    double beta1, beta2; // Adam moments
    double eps_rel;      // Adam epsilon / xi
    double loss_tol;     // convergence threshold eps_L
    int32_t replay_iters;// >= 0: run exactly this many updates, ignoring the loss
    int32_t stall_patience; // checks without progress before a stall reset (0 = never)
} or_params;

// Derived constants (float32 link-test bounds and float64 PGD constants).
typedef struct {
    float b2, lo2, hi2, L[3];
    double w2, eps_q, u, xi_box, dt, thr_link, thr_non, alpha, eps_adam, M, tau;
} or_consts;

typedef struct {
    int64_t iters;        // updates performed (T)
    int64_t loss_evals;   // tight-loss evaluations
    int64_t viol0;        // violated active pairs before the first update
    int64_t viol_final;   // violated active pairs at the end
    double loss0;
    double loss_final;
    int64_t n_editable;
    int32_t converged;
    int32_t pad_;
} or_pgd_stats;

}  // extern "C"

namespace {

enum { CLS_FAR = 0, CLS_SAFE = 1, CLS_PB = 2, CLS_PC = 3 };

// ulp of a float32 number of magnitude x (x > 0): 2^(e-24) with x in [2^(e-1), 2^e).
double ulp_f32(double x) {
    int e = 0;
    std::frexp(x, &e);
    return std::ldexp(1.0, e - 24);
}

// Constants of Sec. 3.1 and Sec. 3.3 (see the readings in the file header).
or_consts make_consts(const or_params *p, const float *orig, const float *recon, int64_t n) {
    or_consts c;
    std::memset(&c, 0, sizeof(c));
    const double b = p->b, xi = p->xi;
    c.w2 = 2.0 * std::sqrt(3.0) * xi;            // largest change of a pair distance
    const double lo = b - c.w2, hi = b + c.w2;
    c.b2 = (float)(b * b);
    c.lo2 = lo > 0.0 ? (float)(lo * lo * (1.0 - std::ldexp(1.0, -20))) : -1.0f;
    c.hi2 = (float)(hi * hi * (1.0 + std::ldexp(1.0, -20)));
    for (int k = 0; k < 3; ++k) c.L[k] = (float)(p->box_hi[k] - p->box_lo[k]);
    double M = 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) {
        M = std::max(M, (double)std::fabs(orig[i]));
        if (recon) M = std::max(M, (double)std::fabs(recon[i]));
    }
    c.M = M;
    c.eps_q = 2.0 * xi / (std::ldexp(1.0, p->m_bits) - 1.0);   // Algorithm 1, first line
    c.u = ulp_f32(M + 2.0 * xi);
    c.xi_box = xi - c.eps_q - c.u;
    c.dt = 2.0 * std::sqrt(3.0) * (c.eps_q + c.u) + b * std::ldexp(1.0, -20);  // Eq. 3 margin
    c.thr_link = b - c.dt;
    c.thr_non = b + c.dt;
    c.tau = std::ldexp(b, -30);   // coincidence radius for the gradient direction
    c.alpha = p->alpha_rel * xi;
    c.eps_adam = p->eps_rel * xi;
    return c;
}

// Canonical float32 coordinate difference with the minimum image (one add or
// subtract of the box length; exact for |d| in (L/2, L) by Sterbenz).
inline float cdiff(float a, float b, int periodic, float L) {
    float d = a - b;
    if (periodic) {
        const float h = 0.5f * L;
        if (d > h) d = d - L;
        else if (d < -h) d = d + L;
    }
    return d;
}

inline float cdist2(const float *P, int64_t i, int64_t j, int periodic, const float *L) {
    float dx = cdiff(P[3 * i + 0], P[3 * j + 0], periodic, L[0]);
    float dy = cdiff(P[3 * i + 1], P[3 * j + 1], periodic, L[1]);
    float dz = cdiff(P[3 * i + 2], P[3 * j + 2], periodic, L[2]);
    float xx = dx * dx;
    float yy = dy * dy;
    float zz = dz * dz;
    float s = xx + yy;
    return s + zz;
}

inline int classify(float d2, const or_consts &c) {
    if (d2 <= c.lo2) return CLS_SAFE;
    if (d2 <= c.b2) return CLS_PB;
    if (d2 <= c.hi2) return CLS_PC;
    return CLS_FAR;
}

struct Pair {
    uint32_t i, j;
    uint8_t cls;
};

// All pairs (i < j) closer than the window's outer bound, found with a uniform
// grid of cells no smaller than that bound (Sec. 2.4 "cell linking", Sec. 3.3):
// a pair can only join particles in the same or adjacent cells.
std::vector<Pair> grid_pairs(const float *P, int64_t n, const or_params *p, const or_consts &c) {
    std::vector<Pair> out;
    const double reach = std::sqrt((double)c.hi2) * (1.0 + 1e-4);
    int nc[3];
    double lo[3], w[3];
    for (int k = 0; k < 3; ++k) {
        double ext;
        if (p->periodic) {
            lo[k] = p->box_lo[k];
            ext = p->box_hi[k] - p->box_lo[k];
        } else {
            double mn = 1e300, mx = -1e300;
            for (int64_t i = 0; i < n; ++i) {
                mn = std::min(mn, (double)P[3 * i + k]);
                mx = std::max(mx, (double)P[3 * i + k]);
            }
            lo[k] = mn;
            ext = mx - mn;
        }
        double f = std::floor(ext / reach);
        nc[k] = (int)std::max(1.0, std::min(f, 256.0));
        w[k] = ext > 0 ? ext / nc[k] : 1.0;
    }
    const bool all_pairs = p->periodic && (nc[0] < 3 || nc[1] < 3 || nc[2] < 3);
    if (all_pairs) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j) {
                int cls = classify(cdist2(P, i, j, p->periodic, c.L), c);
                if (cls != CLS_FAR) out.push_back({(uint32_t)i, (uint32_t)j, (uint8_t)cls});
            }
        return out;
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    std::vector<int64_t> cell(n);
    std::vector<int> cc(3 * n);
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            int q = (int)std::floor(((double)P[3 * i + k] - lo[k]) / w[k]);
            if (p->periodic) q = ((q % nc[k]) + nc[k]) % nc[k];   // image inside the box
            q = std::max(0, std::min(nc[k] - 1, q));
            cc[3 * i + k] = q;
        }
        cell[i] = ((int64_t)cc[3 * i + 2] * nc[1] + cc[3 * i + 1]) * nc[0] + cc[3 * i + 0];
    }
    // members of each cell, in increasing id
    std::vector<int64_t> start(ncell + 1, 0);
    for (int64_t i = 0; i < n; ++i) start[cell[i] + 1]++;
    for (int64_t k = 0; k < ncell; ++k) start[k + 1] += start[k];
    std::vector<int64_t> fill(start.begin(), start.end() - 1), member(n);
    for (int64_t i = 0; i < n; ++i) member[fill[cell[i]]++] = i;
    // particles are split among threads; every thread keeps its own list, and the
    // lists are joined and sorted below, so the result does not depend on the split
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    std::vector<std::vector<Pair>> part(nthr);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        std::vector<Pair> &mine = part[tid];
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    int q[3] = {cc[3 * i] + ox, cc[3 * i + 1] + oy, cc[3 * i + 2] + oz};
                    bool skip = false;
                    for (int k = 0; k < 3; ++k) {
                        if (q[k] < 0 || q[k] >= nc[k]) {
                            if (p->periodic) q[k] = (q[k] + nc[k]) % nc[k];
                            else skip = true;
                        }
                    }
                    if (skip) continue;
                    int64_t cj = ((int64_t)q[2] * nc[1] + q[1]) * nc[0] + q[0];
                    for (int64_t t = start[cj]; t < start[cj + 1]; ++t) {
                        int64_t j = member[t];
                        if (j <= i) continue;
                        int cls = classify(cdist2(P, i, j, p->periodic, c.L), c);
                        if (cls != CLS_FAR) mine.push_back({(uint32_t)i, (uint32_t)j, (uint8_t)cls});
                    }
                }
    }
    for (const std::vector<Pair> &q : part) out.insert(out.end(), q.begin(), q.end());
    std::sort(out.begin(), out.end(), [](const Pair &a, const Pair &b) {
        return a.i != b.i ? a.i < b.i : a.j < b.j;
    });
    return out;
}

// Textbook union-find whose root is the smallest id of its set.
struct DSU {
    std::vector<int64_t> par;
    explicit DSU(int64_t n) : par(n) { std::iota(par.begin(), par.end(), (int64_t)0); }
    int64_t find(int64_t x) {
        while (par[x] != x) {
            par[x] = par[par[x]];
            x = par[x];
        }
        return x;
    }
    bool unite(int64_t a, int64_t b) {
        a = find(a);
        b = find(b);
        if (a == b) return false;
        if (a < b) par[b] = a;
        else par[a] = b;
        return true;
    }
};

// Connected components of the links among the given classes; label = min id (Sec. 2.4).
std::vector<int32_t> components(const std::vector<Pair> &pairs, int64_t n, bool use_safe, bool use_pb) {
    DSU d(n);
    for (const Pair &q : pairs)
        if ((use_safe && q.cls == CLS_SAFE) || (use_pb && q.cls == CLS_PB)) d.unite(q.i, q.j);
    std::vector<int32_t> lab(n);
    for (int64_t i = 0; i < n; ++i) lab[i] = (int32_t)d.find(i);
    return lab;
}

inline uint32_t f32_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

struct Active {
    uint32_t i, j;
    uint8_t link;   // 1: originally linked (d2 <= b2)
};

// Constraint selection (Sec. 3.2): VP keeps V; SC keeps V pairs joining different
// safe components; HF keeps potentially created pairs joining different halos plus a
// spanning forest of potentially broken links among safe components (Kruskal on the
// key (d2 bits, i, j)).  Output sorted by (i, j).
std::vector<Active> select_pairs(const float *P, const std::vector<Pair> &pairs, int64_t n,
                                 int mode, const or_params *p, const or_consts &c) {
    std::vector<Active> A;
    if (mode == 0) {
        for (const Pair &q : pairs)
            if (q.cls == CLS_PB || q.cls == CLS_PC) A.push_back({q.i, q.j, (uint8_t)(q.cls == CLS_PB)});
        return A;
    }
    std::vector<int32_t> safe = components(pairs, n, true, false);
    if (mode == 1) {
        for (const Pair &q : pairs)
            if ((q.cls == CLS_PB || q.cls == CLS_PC) && safe[q.i] != safe[q.j])
                A.push_back({q.i, q.j, (uint8_t)(q.cls == CLS_PB)});
        return A;
    }
    std::vector<int32_t> halo = components(pairs, n, true, true);
    struct Cand {
        uint32_t key, i, j;
    };
    std::vector<Cand> cand;
    for (const Pair &q : pairs) {
        if (q.cls == CLS_PC && halo[q.i] != halo[q.j]) A.push_back({q.i, q.j, 0});
        if (q.cls == CLS_PB && safe[q.i] != safe[q.j]) {
            float d2 = cdist2(P, q.i, q.j, p->periodic, c.L);
            cand.push_back({f32_bits(d2), q.i, q.j});
        }
    }
    std::sort(cand.begin(), cand.end(), [](const Cand &a, const Cand &b) {
        if (a.key != b.key) return a.key < b.key;
        if (a.i != b.i) return a.i < b.i;
        return a.j < b.j;
    });
    DSU super(n);   // over safe-component roots (supernodes)
    for (const Cand &e : cand)
        if (super.unite(safe[e.i], safe[e.j])) A.push_back({e.i, e.j, 1});
    std::sort(A.begin(), A.end(), [](const Active &a, const Active &b) {
        return a.i != b.i ? a.i < b.i : a.j < b.j;
    });
    return A;
}

// Current offset of a pair along one axis, dp + (delta_i - delta_j), rounded once: the
// exact errors of the two additions (Knuth's TwoSum) are added back before the final
// rounding, so offsets of mirror-image pairs are exact negatives of each other.
double offset(double dp, double di, double dj) {
    const double s1 = di - dj, b1 = s1 - di, e1 = (di - (s1 - b1)) + (-dj - b1);
    const double s2 = s1 + dp, b2 = s2 - s1, e2 = (s1 - (s2 - b2)) + (dp - b2);
    return s2 + (e1 + e2);
}

// |r| with the squares added smallest first, so the result does not depend on the
// order of the axes (mirror-image pairs get the same distance to the last bit).
double norm3(const double r[3]) {
    double q[3] = {r[0] * r[0], r[1] * r[1], r[2] * r[2]};
    std::sort(q, q + 3);
    return std::sqrt((q[0] + q[1]) + q[2]);
}

// Projected gradient descent with Adam on the tightened loss (Algorithm 1, Eq. 3),
// in float64 on offsets delta = P_hat - P of the editable particles.  ab (may be NULL)
// gives each active pair its own linking length: several thresholds are supported by
// enforcing the union of their selected pairs (Sec. 1 and Sec. 5), each pair with the
// constraint and the margin of its own threshold.
void pgd(const float *orig, const float *recon, int64_t n, const std::vector<Active> &A,
         const or_params *p, const or_consts &c, float *corrected, double *delta_out,
         int32_t *editable_out, or_pgd_stats *st, const double *ab = nullptr) {
    std::memset(st, 0, sizeof(*st));
    // E = endpoints(A), ascending id (Algorithm 1).
    std::vector<int64_t> idx(n, -1);
    std::vector<int64_t> E;
    for (const Active &a : A) {
        idx[a.i] = 1;
        idx[a.j] = 1;
    }
    for (int64_t i = 0; i < n; ++i)
        if (idx[i] >= 0) {
            idx[i] = (int64_t)E.size();
            E.push_back(i);
        }
    const int64_t ne = (int64_t)E.size();
    st->n_editable = ne;
    if (editable_out)
        for (int64_t i = 0; i < n; ++i) editable_out[i] = idx[i] >= 0 ? 1 : 0;
    // Per pair: original separation (canonical float32, minimum image) and link flag.
    const int64_t na = (int64_t)A.size();
    std::vector<double> dp(3 * na);
    for (int64_t k = 0; k < na; ++k)
        for (int d = 0; d < 3; ++d)
            dp[3 * k + d] = (double)cdiff(orig[3 * A[k].i + d], orig[3 * A[k].j + d], p->periodic, c.L[d]);
    // Per pair: thresholds of Eq. 3 (b -/+ dt with the pair's b) and the coincidence radius.
    std::vector<double> thr_link(na, c.thr_link), thr_non(na, c.thr_non), tau(na, c.tau);
    std::vector<double> vtol(na, std::ldexp(p->b, -40));   // smallest violation that counts
    if (ab)
        for (int64_t k = 0; k < na; ++k) {
            const double dt = 2.0 * std::sqrt(3.0) * (c.eps_q + c.u) + ab[k] * std::ldexp(1.0, -20);
            thr_link[k] = ab[k] - dt;
            thr_non[k] = ab[k] + dt;
            tau[k] = std::ldexp(ab[k], -30);
            vtol[k] = std::ldexp(ab[k], -40);
        }
    // P_hat starts at the base reconstruction: delta0 = recon - orig (exact in float64).
    std::vector<double> delta(3 * ne), m(3 * ne, 0.0), v(3 * ne, 0.0), g(3 * ne);
    for (int64_t e = 0; e < ne; ++e)
        for (int d = 0; d < 3; ++d)
            delta[3 * e + d] = (double)recon[3 * E[e] + d] - (double)orig[3 * E[e] + d];

    // Tight loss of Eq. 3 and (optionally) its gradient with respect to delta.  Each
    // pair's violated amount and direction are computed on their own (on several
    // threads when built with OpenMP); the loss, the counts and the gradient then add
    // them in pair order, so the sums do not depend on the number of threads.
    const double inv_unit = 1.0 / (p->xi * p->xi * std::ldexp(1.0, -24));
    std::vector<uint8_t> hit(ne);   // editable particle is an endpoint of a violated pair
    std::vector<double> vamt(na), dir(3 * na);
    auto evaluate = [&](bool want_grad, double *loss, int64_t *viol, int64_t *lfx) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < na; ++k) {
            const int64_t a = idx[A[k].i], b = idx[A[k].j];
            double r[3];
            for (int d = 0; d < 3; ++d) r[d] = offset(dp[3 * k + d], delta[3 * a + d], delta[3 * b + d]);
            const double dh = norm3(r);
            // link: penalise d_hat > b - dt;  non-link: penalise d_hat < b + dt
            const double viol_amt = A[k].link ? dh - thr_link[k] : thr_non[k] - dh;
            vamt[k] = viol_amt;
            if (!(viol_amt > 0.0) || !want_grad) continue;
            double u[3];
            if (dh > tau[k]) {
                for (int d = 0; d < 3; ++d) u[d] = r[d] / dh;
            } else {
                const double n0 = std::sqrt(dp[3 * k] * dp[3 * k] + dp[3 * k + 1] * dp[3 * k + 1] +
                                            dp[3 * k + 2] * dp[3 * k + 2]);
                for (int d = 0; d < 3; ++d) u[d] = n0 > 0.0 ? dp[3 * k + d] / n0 : 0.0;
            }
            for (int d = 0; d < 3; ++d) dir[3 * k + d] = u[d];
        }
        double L = 0.0;
        int64_t nv = 0, fx = 0;
        std::fill(hit.begin(), hit.end(), 0);
        if (want_grad) std::fill(g.begin(), g.end(), 0.0);
        for (int64_t k = 0; k < na; ++k) {
            const double viol_amt = vamt[k];
            if (!(viol_amt > 0.0)) continue;
            const int64_t a = idx[A[k].i], b = idx[A[k].j];
            L += viol_amt * viol_amt;
            if (viol_amt > vtol[k]) nv += 1;
            fx += (int64_t)std::llrint(viol_amt * viol_amt * inv_unit);
            hit[a] = hit[b] = 1;
            if (!want_grad) continue;
            // d/d(delta_i) of (d_hat - thr)^2 is 2 (d_hat - thr) r/|r|; of (thr - d_hat)^2 it is the negative
            const double s = A[k].link ? 2.0 * viol_amt : -2.0 * viol_amt;
            for (int d = 0; d < 3; ++d) {
                g[3 * a + d] += s * dir[3 * k + d];
                g[3 * b + d] -= s * dir[3 * k + d];
            }
        }
        *loss = L;
        *viol = nv;
        *lfx = fx;
    };

    int64_t t = 0;        // updates done
    bool converged = false;
    double L = 0.0;
    int64_t nv = 0;
    double b1t = 1.0, b2t = 1.0;
    int64_t lfx = 0;          // fixed-point loss of the last check
    int64_t best = 0;         // lowest fixed-point loss that counted as progress
    int64_t since = 0;        // checks since then
    int64_t patience = p->stall_patience;   // doubles after every reset
    bool reset_now = false;   // this check resets the endpoints of violated pairs
    for (;;) {
        const bool replay = p->replay_iters >= 0;
        const bool last = replay ? (t == p->replay_iters) : (t == p->t_max);
        const bool need_grad = !last;
        evaluate(need_grad, &L, &nv, &lfx);
        st->loss_evals += 1;
        if (t == 0) {
            st->loss0 = L;
            st->viol0 = nv;
        }
        const bool conv_now = p->loss_tol > 0.0 ? (L <= p->loss_tol) : (nv == 0);
        if (!replay && conv_now) {
            converged = true;
            break;
        }
        if (last) break;
        // Adam step (Kingma & Ba) on every editable coordinate, then projection onto the box.
        t += 1;
        b1t *= p->beta1;
        b2t *= p->beta2;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < 3 * ne; ++q) {
            if (reset_now && hit[q / 3]) {
                delta[q] = 0.0;
                m[q] = 0.0;
                v[q] = 0.0;
                continue;
            }
            m[q] = p->beta1 * m[q] + (1.0 - p->beta1) * g[q];
            v[q] = p->beta2 * v[q] + (1.0 - p->beta2) * g[q] * g[q];
            const double mh = m[q] / (1.0 - b1t);
            const double vh = v[q] / (1.0 - b2t);
            double dq = delta[q] - c.alpha * mh / (std::sqrt(vh) + c.eps_adam);
            delta[q] = std::min(c.xi_box, std::max(-c.xi_box, dq));
        }
        // stall rule on the loss of the check just taken (t now counts its update)
        if (reset_now) {
            reset_now = false;
            best = INT64_MAX;
            since = 0;
        } else if (t == 1) {
            best = lfx;
        } else if (lfx < best - best / 1024) {
            best = lfx;
            since = 0;
        } else if (p->stall_patience > 0 && ++since >= patience && lfx > 16 * nv) {
            reset_now = true;
            since = 0;
            if (patience < (1 << 24)) patience *= 2;
        }
    }
    if (p->replay_iters >= 0) converged = p->loss_tol > 0.0 ? (L <= p->loss_tol) : (nv == 0);
    st->iters = t;
    st->converged = converged ? 1 : 0;
    st->loss_final = L;
    st->viol_final = nv;
    // Output: untouched particles keep the reconstruction; editable ones become orig + delta.
    for (int64_t i = 0; i < 3 * n; ++i) corrected[i] = recon[i];
    if (t > 0)
        for (int64_t e = 0; e < ne; ++e)
            for (int d = 0; d < 3; ++d)
                corrected[3 * E[e] + d] = (float)((double)orig[3 * E[e] + d] + delta[3 * e + d]);
    if (delta_out)
        for (int64_t e = 0; e < ne; ++e)
            for (int d = 0; d < 3; ++d) delta_out[3 * E[e] + d] = delta[3 * e + d];
}

void put_u32(uint8_t *o, uint32_t v) {
    for (int k = 0; k < 4; ++k) o[k] = (uint8_t)(v >> (8 * k));
}
void put_u64(uint8_t *o, uint64_t v) {
    for (int k = 0; k < 8; ++k) o[k] = (uint8_t)(v >> (8 * k));
}
uint32_t get_u32(const uint8_t *o) {
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) v |= (uint32_t)o[k] << (8 * k);
    return v;
}
uint64_t get_u64(const uint8_t *o) {
    uint64_t v = 0;
    for (int k = 0; k < 8; ++k) v |= (uint64_t)o[k] << (8 * k);
    return v;
}

const int HEADER = 64;

}  // namespace

extern "C" {

// Threads of the OpenMP build (1 without OpenMP); n <= 0 leaves the count as it is.
int32_t or_threads(int32_t n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return (int32_t)omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void or_constants(const or_params *p, const float *orig, const float *recon, int64_t n, or_consts *out) {
    *out = make_consts(p, orig, recon, n);
}

// Canonical float32 squared distance of one pair (exported for the tests).
float or_dist2(const float *P, int64_t i, int64_t j, const or_params *p) {
    float L[3];
    for (int k = 0; k < 3; ++k) L[k] = (float)(p->box_hi[k] - p->box_lo[k]);
    return cdist2(P, i, j, p->periodic, L);
}

// Class of each listed pair (0 far, 1 safe, 2 potentially broken, 3 potentially created),
// one by one, with the constants of the whole point set (Sec. 3.1).
void or_classify(const float *P, int64_t n, const or_params *p, const uint32_t *ai, const uint32_t *aj,
                 int64_t m, uint8_t *cls) {
    or_consts c = make_consts(p, P, nullptr, n);
    for (int64_t k = 0; k < m; ++k) cls[k] = (uint8_t)classify(cdist2(P, ai[k], aj[k], p->periodic, c.L), c);
}

// Every pair with a class (safe, potentially broken, potentially created), sorted by (i, j).
// brute != 0 checks all n(n-1)/2 pairs instead of using the grid.  Returns the count;
// the arrays are filled only when cap is large enough.
int64_t or_pairs(const float *P, int64_t n, const or_params *p, int32_t brute,
                 uint32_t *oi, uint32_t *oj, uint8_t *ocls, int64_t cap) {
    or_consts c = make_consts(p, P, nullptr, n);
    std::vector<Pair> pairs;
    if (brute) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j) {
                int cls = classify(cdist2(P, i, j, p->periodic, c.L), c);
                if (cls != CLS_FAR) pairs.push_back({(uint32_t)i, (uint32_t)j, (uint8_t)cls});
            }
    } else {
        pairs = grid_pairs(P, n, p, c);
    }
    const int64_t np = (int64_t)pairs.size();
    if (np <= cap && oi) {
        for (int64_t k = 0; k < np; ++k) {
            oi[k] = pairs[k].i;
            oj[k] = pairs[k].j;
            ocls[k] = pairs[k].cls;
        }
    }
    return np;
}

// Friends-of-friends labels (Sec. 2.4): components of the links d2 <= b2; label = smallest id.
// Also returns the safe-component labels when safe_out != NULL.  Returns the number of halos.
int64_t or_fof_labels(const float *P, int64_t n, const or_params *p, int32_t *labels, int32_t *safe_out) {
    or_consts c = make_consts(p, P, nullptr, n);
    std::vector<Pair> pairs = grid_pairs(P, n, p, c);
    std::vector<int32_t> lab = components(pairs, n, true, true);
    std::memcpy(labels, lab.data(), n * sizeof(int32_t));
    if (safe_out) {
        std::vector<int32_t> s = components(pairs, n, true, false);
        std::memcpy(safe_out, s.data(), n * sizeof(int32_t));
    }
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) nc += (lab[i] == i);
    return nc;
}

// Active pairs of the given mode (Sec. 3.2), sorted by (i, j), with the original link flag.
int64_t or_select(const float *P, int64_t n, const or_params *p, int32_t mode,
                  uint32_t *oi, uint32_t *oj, uint8_t *olink, int64_t cap, int64_t *n_vulnerable) {
    or_consts c = make_consts(p, P, nullptr, n);
    std::vector<Pair> pairs = grid_pairs(P, n, p, c);
    if (n_vulnerable) {
        int64_t nv = 0;
        for (const Pair &q : pairs) nv += (q.cls == CLS_PB || q.cls == CLS_PC);
        *n_vulnerable = nv;
    }
    std::vector<Active> A = select_pairs(P, pairs, n, mode, p, c);
    const int64_t na = (int64_t)A.size();
    if (na <= cap && oi)
        for (int64_t k = 0; k < na; ++k) {
            oi[k] = A[k].i;
            oj[k] = A[k].j;
            olink[k] = A[k].link;
        }
    return na;
}

// PGD on a given active set (Algorithm 1 loop) with a linking length per active pair
// (ab may be NULL: p->b for every pair); alink[k] is the pair's link flag at its own
// linking length.  delta_out (n*3 doubles, may be NULL) receives the float64 offsets of
// editable particles; editable_out (n ints, may be NULL) marks E.  Returns 0, or -1 when
// the box is empty (xi too small for float32 coordinates).
int32_t or_pgd_thr(const float *orig, const float *recon, int64_t n, const or_params *p,
                   const uint32_t *ai, const uint32_t *aj, const uint8_t *alink, const double *ab, int64_t na,
                   float *corrected, double *delta_out, int32_t *editable_out, or_pgd_stats *st) {
    or_consts c = make_consts(p, orig, recon, n);
    if (!(c.xi_box > 0.0)) return -1;
    std::vector<Active> A(na);
    for (int64_t k = 0; k < na; ++k) A[k] = {ai[k], aj[k], alink[k]};
    pgd(orig, recon, n, A, p, c, corrected, delta_out, editable_out, st, ab);
    return 0;
}

// The same with p->b for every pair.
int32_t or_pgd(const float *orig, const float *recon, int64_t n, const or_params *p,
               const uint32_t *ai, const uint32_t *aj, const uint8_t *alink, int64_t na,
               float *corrected, double *delta_out, int32_t *editable_out, or_pgd_stats *st) {
    return or_pgd_thr(orig, recon, n, p, ai, aj, alink, nullptr, na, corrected, delta_out, editable_out, st);
}

// Edit stream (Algorithm 1 last lines, Sec. 3.3): flags + m-bit codes; format v1:
//   bytes 0-3 "PCE1", u32 version=1, u64 n, u32 m, u32 mode, u32 periodic, u32 0,
//   f64 xi, u64 flagged, u64 flag_bytes, u64 code_bytes  (64-byte header, little endian)
//   then ceil(n/8) flag bytes (particle i -> byte i>>3, bit i&7)
//   then per flagged particle in ascending id: x, y, z codes of ceil(m/8) bytes each.
// Returns the stream size; writes only when cap suffices.
int64_t or_encode(const float *recon, const float *corrected, int64_t n, const or_params *p,
                  uint8_t *out, int64_t cap) {
    const int m = p->m_bits;
    const int cb = (m + 7) / 8;
    const double xi = p->xi;
    const double qmax = std::ldexp(1.0, m) - 1.0;
    const double s = 4.0 * xi / qmax;
    std::vector<int64_t> flagged;
    for (int64_t i = 0; i < n; ++i) {
        bool f = false;
        for (int d = 0; d < 3; ++d) f = f || ((double)corrected[3 * i + d] - (double)recon[3 * i + d] != 0.0);
        if (f) flagged.push_back(i);
    }
    const int64_t fb = (n + 7) / 8;
    const int64_t codeb = (int64_t)flagged.size() * 3 * cb;
    const int64_t total = HEADER + fb + codeb;
    if (!out || cap < total) return total;
    std::memset(out, 0, total);
    std::memcpy(out, "PCE1", 4);
    put_u32(out + 4, 1);
    put_u64(out + 8, (uint64_t)n);
    put_u32(out + 16, (uint32_t)m);
    put_u32(out + 20, (uint32_t)p->mode);
    put_u32(out + 24, (uint32_t)p->periodic);
    std::memcpy(out + 32, &xi, 8);
    put_u64(out + 40, (uint64_t)flagged.size());
    put_u64(out + 48, (uint64_t)fb);
    put_u64(out + 56, (uint64_t)codeb);
    uint8_t *flags = out + HEADER;
    uint8_t *codes = flags + fb;
    int64_t w = 0;
    for (int64_t i : flagged) {
        flags[i >> 3] |= (uint8_t)(1u << (i & 7));
        for (int d = 0; d < 3; ++d) {
            const double delta = (double)corrected[3 * i + d] - (double)recon[3 * i + d];
            double q = std::nearbyint((delta + 2.0 * xi) / s);   // round half to even
            q = std::min(qmax, std::max(0.0, q));
            const uint64_t qi = (uint64_t)q;
            for (int k = 0; k < cb; ++k) codes[w++] = (uint8_t)(qi >> (8 * k));
        }
    }
    return total;
}

// Decoder (Sec. 3.3 "Reconstruction"): final = fl32(recon + (-2 xi + q s)) for flagged
// particles, recon elsewhere.  Returns 0, or -1 on a malformed stream.
int32_t or_decode(const float *recon, int64_t n, const uint8_t *in, int64_t nbytes, float *out) {
    if (nbytes < HEADER || std::memcmp(in, "PCE1", 4) != 0 || get_u32(in + 4) != 1) return -1;
    if ((int64_t)get_u64(in + 8) != n) return -1;
    const int m = (int)get_u32(in + 16);
    if (m < 2 || m > 32) return -1;
    const int cb = (m + 7) / 8;
    double xi;
    std::memcpy(&xi, in + 32, 8);
    const int64_t nf = (int64_t)get_u64(in + 40);
    const int64_t fb = (int64_t)get_u64(in + 48);
    const int64_t codeb = (int64_t)get_u64(in + 56);
    if (fb != (n + 7) / 8 || codeb != nf * 3 * cb || nbytes < HEADER + fb + codeb) return -1;
    const double s = 4.0 * xi / (std::ldexp(1.0, m) - 1.0);
    const uint8_t *flags = in + HEADER;
    const uint8_t *codes = flags + fb;
    int64_t r = 0, seen = 0;
    for (int64_t i = 0; i < n; ++i) {
        const bool f = (flags[i >> 3] >> (i & 7)) & 1u;
        for (int d = 0; d < 3; ++d) out[3 * i + d] = recon[3 * i + d];
        if (!f) continue;
        if (++seen > nf) return -1;
        for (int d = 0; d < 3; ++d) {
            uint64_t q = 0;
            for (int k = 0; k < cb; ++k) q |= (uint64_t)codes[r++] << (8 * k);
            out[3 * i + d] = (float)((double)recon[3 * i + d] + (-2.0 * xi + (double)q * s));
        }
    }
    return seen == nf ? 0 : -1;
}

// Whole correction pass (pairs -> selection -> PGD), the CPU baseline.
int32_t or_correct(const float *orig, const float *recon, int64_t n, const or_params *p,
                   float *corrected, or_pgd_stats *st, int64_t *n_vulnerable, int64_t *n_active) {
    or_consts c = make_consts(p, orig, recon, n);
    if (!(c.xi_box > 0.0)) return -1;
    std::vector<Pair> pairs = grid_pairs(orig, n, p, c);
    int64_t nv = 0;
    for (const Pair &q : pairs) nv += (q.cls == CLS_PB || q.cls == CLS_PC);
    std::vector<Active> A = select_pairs(orig, pairs, n, p->mode, p, c);
    if (n_vulnerable) *n_vulnerable = nv;
    if (n_active) *n_active = (int64_t)A.size();
    pgd(orig, recon, n, A, p, c, corrected, nullptr, nullptr, st);
    return 0;
}

// Untightened loss of Eq. 1 over the given pairs, evaluated with the canonical float32
// link test on the given coordinates: counts pairs whose link state differs from the
// original link flag.
int64_t or_count_flips(const float *P, int64_t n, const or_params *p, const uint32_t *ai,
                       const uint32_t *aj, const uint8_t *alink, int64_t na) {
    or_consts c = make_consts(p, P, nullptr, n);
    int64_t bad = 0;
    for (int64_t k = 0; k < na; ++k) {
        const bool now = cdist2(P, ai[k], aj[k], p->periodic, c.L) <= c.b2;
        bad += (now != (alink[k] != 0));
    }
    return bad;
}

}  // extern "C"
