// Projected gradient descent on the tightened loss (Algorithm 1, Eq. 3,
// Sec. 3.3 "Gradient descent and projection", Adam as in Sec. 4.2).
//
// Layout.  The editable set E = endpoints(A) is numbered in cell order (dense
// index e), so neighbouring particles sit close in memory.  A is stored as a
// CSR by endpoint: row e lists every active partner k of e (col = k | link
// bit << 31; with several linking lengths, k | threshold index << 29 | link << 31),
// rows sorted by the partner's position.  State per editable
// particle, float4 each (w unused): original position PE (w = id bits); the
// offset delta = P_hat - P as a double-float (hi, lo) and its float32 rounding
// Q = fl(P + delta), both in two ping-pong buffers; the Adam moments m, v as
// double-floats; one activity byte.
//
// One iteration = k_pgd_iter (+ k_pgd_heavy when some rows have more than
// HEAVY partners).  Warps take work items (groups of 32 light rows, or one
// HEAVY-edge chunk of a heavy row) from a counter.  A float32 screen on Q
// certifies most pairs as satisfied; the others are evaluated in
// double-float, 32 at a time, and each row's gradient is a fixed-order sum
// (segmented shuffle scan within a batch, batches in edge order, chunks in
// chunk order), so no float atomics are used and the offsets are
// deterministic.  The loss (each pair counted once, in the row of its smaller
// dense index) is accumulated in fixed point and the violations are counted;
// the last block takes the stop decision of Algorithm 1.  The Adam step of
// the same launch is written to the other buffers, so when the check says
// "stop" the current buffer is the answer and nothing has to be undone.
#include <algorithm>
#include <cmath>

#include "df.cuh"
#include "pipeline.cuh"

namespace pc {

namespace {

#define GRID_STRIDE(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

inline int grid_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), (int64_t)num_sms() * 16));
}

constexpr int PGD_THREADS = 256;
constexpr int WARPS = PGD_THREADS / 32;
constexpr int PGD_BLOCKS_PER_SM = 4;   // resident CTAs of the persistent iteration grid

// Linking lengths of one problem: one, or up to MAX_THR enforced together (the union of
// their active pairs, Sec. 1 and Sec. 5); a CSR entry then carries its pair's index.
constexpr int MAX_THR = 4;

// act[e]: bit 0 = the row has had a gradient (or needs its first projection), bit 1 = the
// row is heavy (more than HEAVY partners: its edges are walked in chunks of HEAVY).
constexpr uint8_t ACT_ON = 1, ACT_HEAVY = 2;
constexpr uint32_t HEAVY = 256;

// Per-block PGD constants (one entry per block of the problem set).  The threshold arrays
// are indexed by the pair's linking length (entry 0 alone with one).
struct PgdConsts {
    int periodic;
    float L[3];
    float b2;
    float screen_link[MAX_THR];   // link pair certainly satisfied when float32 d2 < screen_link
    float screen_non[MAX_THR];    // non-link pair certainly satisfied when float32 d2 > screen_non
    float tau[MAX_THR];           // coincidence radius b * 2^-30 for the gradient direction
    df thr_link[MAX_THR], thr_non[MAX_THR];   // b -/+ delta_t of Eq. 3
    double vtol[MAX_THR];         // a violation counts (stop rule, stall rule) above b * 2^-40
    int interior_ok;              // periodic box whose interior rows never wrap (see ilo, ihi)
    float ilo[3], ihi[3];         // current position of an interior row, per axis
    df xi_box, alpha, eps_adam;
    df beta1, one_m_beta1, beta2, one_m_beta2;
    int t_max;
    int replay;
    double loss_tol;
    double beta1_d, beta2_d;
    double loss_unit;    // xi^2 2^-24: fixed-point unit of the loss
    double inv_loss_unit;
    int stall_patience;  // checks without progress of the fixed-point loss before a reset (0 = off)
    int pad;
};

// Per-block iteration state.
struct PgdBlk {
    int32_t t;          // updates done
    int32_t stop;
    int32_t final_buf;
    int32_t converged;
    unsigned long long viol, viol0;
    double loss, loss0;
    double b1p, b2p;    // beta^(t+1) for the update of the next launch
    df ibc1, ibc2;      // 1 / (1 - beta^(t+1))
    int32_t upd_t;      // check index of the last launch
    int32_t upd_on;     // 1 if that launch's update stands
    df upd_ibc1, upd_ibc2;
    int32_t reset;      // this launch resets the endpoints of violated pairs (stall rule)
    int32_t upd_reset;  // the value of reset for the launch just finished (heavy rows)
    unsigned long long best;        // lowest fixed-point loss that counted as progress
    int32_t since;                  // checks since then
    int32_t patience;               // checks without progress before the next reset (doubles per reset)
    int32_t resets;                 // checks that triggered a stall reset
    unsigned long long lfx, vacc;   // launch accumulators: loss (fixed point), violations,
    unsigned long long uacc, eacc;  // ... rows updated (Adam steps), pairs evaluated in double-float
    unsigned long long n_upd, n_eval;   // totals of the last two over the run
};

struct PgdGlobal {
    uint32_t ticket;
    int32_t all_stop;
    unsigned long long work;        // next work item of the launch
    int32_t active;                 // blocks still iterating after the last launch
    int32_t pad;
    unsigned long long n_items;     // work items of the blocks still iterating (problem sets)
};

// Work of one block of a problem set: its rows [row0, row0 + nrows) form ceil(nrows / 32)
// light items (groups of 32 rows that never straddle two blocks; the heavy rows among
// them have no light edges), followed by its heavy chunks [ch0, ch0 + nch).
struct BlkWork {
    uint32_t row0, nrows, ch0, nch;
};

// Items of the blocks still iterating, for the next launch: active block k is act_blk[k]
// and owns the work items [act_pref[k], act_pref[k + 1]).
struct WorkTab {
    const BlkWork *bw;
    uint32_t *act_blk;
    unsigned long long *act_pref;
};

// One warp: rebuild the table from the stop flags (blocks in ascending order).
__device__ void build_worktab(int nb, const PgdBlk *blk, const WorkTab wt, PgdGlobal *gs) {
    const int lane = threadIdx.x & 31;
    unsigned long long carry = 0;
    int cnt = 0;
    for (int base = 0; base < nb; base += 32) {
        const int b = base + lane;
        const bool a = b < nb && !blk[b].stop;
        unsigned long long it = 0;
        if (a) {
            const BlkWork w = wt.bw[b];
            it = (unsigned long long)((w.nrows + 31u) >> 5) + w.nch;
        }
        unsigned long long inc = it;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, a);
        if (a) {
            const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
            wt.act_blk[pos] = (uint32_t)b;
            wt.act_pref[pos] = carry + inc - it;
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
        cnt += __popc(bal);
    }
    if (lane == 0) {
        wt.act_pref[cnt] = carry;
        gs->n_items = carry;
        gs->active = cnt;
    }
}

__global__ void k_worktab_init(int nb, const PgdBlk *blk, const WorkTab wt, PgdGlobal *gs) {
    if (threadIdx.x < 32) build_worktab(nb, blk, wt, gs);
}

// Per-block row and chunk ranges (rows are in sorted-position order, so every block owns
// a contiguous range of rows, and chunks follow their rows).
__global__ void k_blk_work(const int64_t *__restrict__ row_off, const uint32_t *__restrict__ c0, int64_t ne,
                           int64_t n_chunks, int nb, BlkWork *__restrict__ bw) {
    GRID_STRIDE(b, nb) {
        const int64_t r0 = row_off[b], r1 = row_off[b + 1];
        const uint32_t h0 = r0 < ne ? c0[r0] : (uint32_t)n_chunks, h1 = r1 < ne ? c0[r1] : (uint32_t)n_chunks;
        bw[b] = BlkWork{(uint32_t)r0, (uint32_t)(r1 - r0), h0, h1 - h0};
    }
}

// ------------------------------------------------------------------ CSR build
__global__ void k_mark(const unsigned long long *__restrict__ A, int64_t m, uint32_t *__restrict__ mark) {
    GRID_STRIDE(r, m) {
        const unsigned long long pk = A[r];
        mark[pk >> 32] = 1u;
        mark[pk & 0xffffffffull] = 1u;
    }
}

__global__ void k_epos(const uint32_t *__restrict__ mark, const uint32_t *__restrict__ dense, int64_t n,
                       uint32_t *__restrict__ epos) {
    GRID_STRIDE(k, n) {
        if (mark[k]) epos[dense[k]] = (uint32_t)k;
    }
}

// Directed keys (row << nb | partner position) << tb | threshold index (tb = 0: one
// linking length; tb = 2: Athr gives each pair's index).
__global__ void k_dir_keys(const unsigned long long *__restrict__ A, const uint8_t *__restrict__ Athr, int64_t m,
                           const uint32_t *__restrict__ dense, int nb, int tb, unsigned long long *__restrict__ keys) {
    GRID_STRIDE(r, m) {
        const unsigned long long pk = A[r];
        const uint32_t ki = (uint32_t)(pk >> 32), kj = (uint32_t)(pk & 0xffffffffull);
        const unsigned long long t = tb ? (unsigned long long)Athr[r] : 0ull;
        keys[2 * r] = ((((unsigned long long)dense[ki] << nb) | kj) << tb) | t;
        keys[2 * r + 1] = ((((unsigned long long)dense[kj] << nb) | ki) << tb) | t;
    }
}

__global__ void k_row_bounds(const unsigned long long *__restrict__ keys, int64_t m, int nb, int64_t nrows,
                             unsigned long long *__restrict__ row_ptr) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= m; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = t == 0 ? -1 : (int64_t)(keys[t - 1] >> nb);
        const int64_t cur = t == m ? nrows : (int64_t)(keys[t] >> nb);   // nb: all bits below the row
        for (int64_t r = prev + 1; r <= cur; ++r) row_ptr[r] = (unsigned long long)t;
    }
}

__device__ __forceinline__ float3 canon_dp(const float4 p, const float4 q, int periodic, const float *L) {
    const bool per = periodic != 0;
    return make_float3(cdiff(p.x, q.x, per, L[0]), cdiff(p.y, q.y, per, L[1]), cdiff(p.z, q.z, per, L[2]));
}

__global__ void k_state_init(const uint32_t *__restrict__ epos, int64_t ne, const float4 *__restrict__ P4,
                             const float *__restrict__ orig, const float *__restrict__ recon,
                             const int64_t *__restrict__ off, int nblk, const PgdConsts *__restrict__ CB,
                             float4 *__restrict__ PE, uint32_t *__restrict__ rb, float4 *__restrict__ Dhi,
                             float4 *__restrict__ Dlo, float4 *__restrict__ Dhi1, float4 *__restrict__ Dlo1,
                             float4 *__restrict__ Q, float4 *__restrict__ Q1, float4 *__restrict__ Mhi,
                             float4 *__restrict__ Mlo, float4 *__restrict__ Vhi, float4 *__restrict__ Vlo,
                             uint8_t *__restrict__ act, unsigned long long *__restrict__ rows_per_block) {
    GRID_STRIDE(e, ne) {
        const uint32_t pos = epos[e];
        const int b = find_block(off, nblk, pos);
        rb[e] = (uint32_t)b;
        atomicAdd(rows_per_block + b, 1ull);
        const float4 p = P4[pos];
        PE[e] = p;
        const int64_t id = (int64_t)__float_as_uint(p.w);
        const float4 q = make_float4(recon[3 * id + 0], recon[3 * id + 1], recon[3 * id + 2], 0.f);   // orig + delta0
        Q[e] = q;
        Q1[e] = q;
        // delta0 = recon - orig, exactly, as a double-float; both offset buffers start there
        const df dx = two_sum(recon[3 * id + 0], -orig[3 * id + 0]);
        const df dy = two_sum(recon[3 * id + 1], -orig[3 * id + 1]);
        const df dz = two_sum(recon[3 * id + 2], -orig[3 * id + 2]);
        Dhi[e] = make_float4(dx.hi, dy.hi, dz.hi, 0.f);
        Dlo[e] = make_float4(dx.lo, dy.lo, dz.lo, 0.f);
        Dhi1[e] = make_float4(dx.hi, dy.hi, dz.hi, 0.f);
        Dlo1[e] = make_float4(dx.lo, dy.lo, dz.lo, 0.f);
        // a row must be updated from the first update on if the projection moves it
        const df xb = CB[b].xi_box, nl = df_neg(xb);
        const bool out = df_lt(xb, dx) || df_lt(dx, nl) || df_lt(xb, dy) || df_lt(dy, nl) || df_lt(xb, dz) ||
                         df_lt(dz, nl);
        act[e] = out ? ACT_ON : 0;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        Mhi[e] = z;
        Mlo[e] = z;
        Vhi[e] = z;
        Vlo[e] = z;
    }
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ df comp(const float4 &h, const float4 &l, int a) {
    return a == 0 ? df_make(h.x, l.x) : (a == 1 ? df_make(h.y, l.y) : df_make(h.z, l.z));
}

__device__ __forceinline__ df df_clamp(df x, df lim) {
    if (df_lt(lim, x)) return lim;
    const df nl = df_neg(lim);
    if (df_lt(x, nl)) return nl;
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum_u(unsigned long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ bool is_last(const PgdConsts &C, int t) {
    return C.replay >= 0 ? (t == C.replay) : (t == C.t_max);
}

// ------------------------------------------------------------------ pair evaluation
// r = dp + ((eh + el) - (kh + kl)) in double-float: the offset difference with one
// double-word add, then the original separation.  Every step is an odd function of its
// inputs under round-to-nearest, so r(k, e) = -r(e, k) exactly and mirror-image pairs
// give exactly opposite terms; an exact zero stays exactly zero.
__device__ __forceinline__ df exact_r(float dp, float eh, float el, float kh, float kl) {
    return df_add_f(df_add(df_make(eh, el), df_make(-kh, -kl)), dp);
}

// Violated amount of Eq. 3 for one active pair (row e, partner k) at the current
// offsets, in double-float, and the gradient term d/d(delta_e) of max(0, v)^2.
__device__ __forceinline__ bool eval_pair(const float4 pe, const float4 deh, const float4 del, int64_t e, uint32_t k,
                                          bool link, int ti, const float4 *__restrict__ PE, const float4 *Dh,
                                          const float4 *Dl, const PgdConsts &C, df g[3], double &lt, bool &counts) {
    const float4 pk = __ldg(PE + k);
    const float4 dkh = Dh[k], dkl = Dl[k];
    const float3 dp = canon_dp(pe, pk, C.periodic, C.L);
    const float dpa[3] = {dp.x, dp.y, dp.z};
    df r[3];
    r[0] = exact_r(dp.x, deh.x, del.x, dkh.x, dkl.x);
    r[1] = exact_r(dp.y, deh.y, del.y, dkh.y, dkl.y);
    r[2] = exact_r(dp.z, deh.z, del.z, dkh.z, dkl.z);
    // squares added smallest first: the distance does not depend on the order of the axes,
    // so mirror-image pairs (common on the quantizer lattice) cancel exactly
    df q0 = df_mul(r[0], r[0]), q1 = df_mul(r[1], r[1]), q2 = df_mul(r[2], r[2]);
    if (df_lt(q1, q0)) { const df x = q0; q0 = q1; q1 = x; }
    if (df_lt(q2, q1)) { const df x = q1; q1 = q2; q2 = x; }
    if (df_lt(q1, q0)) { const df x = q0; q0 = q1; q1 = x; }
    const df dh = df_sqrt(df_add(df_add(q0, q1), q2));
    const df v = link ? df_sub(dh, C.thr_link[ti]) : df_sub(C.thr_non[ti], dh);
    if (!df_gt0(v)) return false;
    const double vd = df_to_d(v);
    counts = vd > C.vtol[ti];
    lt = (int64_t)k > e ? vd * vd * C.inv_loss_unit : 0.0;   // in loss units
    // 2 v r / |r| (link) or -2 v r / |r| (non-link); coincident points use the original separation
    const df s = link ? df_add(v, v) : df_neg(df_add(v, v));
    if (dh.hi > C.tau[ti]) {
        const df c = df_div(s, dh);
#pragma unroll
        for (int a = 0; a < 3; ++a) g[a] = df_mul(c, r[a]);
    } else {
        const df n0 = df_sqrt(df_add(df_add(two_prod(dp.x, dp.x), two_prod(dp.y, dp.y)), two_prod(dp.z, dp.z)));
        const df c = n0.hi > 0.f ? df_div(s, n0) : df_make(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < 3; ++a) g[a] = df_mul_f(c, dpa[a]);
    }
    return true;
}

// A row that has never had a gradient (and needs no projection) has zero moments and an
// unchanged offset: Adam leaves it where it is, and both offset buffers already hold
// that value, so nothing is read or written for it.  A reset row (stall rule) returns
// to its original position with cleared moments instead of taking its step.
// The row's state as loaded: offset (hi, lo), original position, moments (hi, lo).
struct RowState {
    float4 dh, dl, pe, mh, ml, vh, vl;
};

__device__ __forceinline__ void adam_core(int64_t e, const df g[3], const RowState &S, bool was, uint8_t av,
                                          uint8_t *__restrict__ act, const df ibc1, const df ibc2, bool reset,
                                          const PgdConsts &C, float4 *Nh, float4 *Nl, float4 *__restrict__ Mhi,
                                          float4 *__restrict__ Mlo, float4 *__restrict__ Vhi,
                                          float4 *__restrict__ Vlo, float4 *Qn) {
    const bool gz = g[0].hi == 0.f && g[1].hi == 0.f && g[2].hi == 0.f;
    if (!was && gz && !reset) return;
    if (!was) act[e] = (uint8_t)(av | ACT_ON);
    if (reset) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f), pe = S.pe;
        Nh[e] = z4;
        Nl[e] = z4;
        Mhi[e] = z4;
        Mlo[e] = z4;
        Vhi[e] = z4;
        Vlo[e] = z4;
        Qn[e] = make_float4(pe.x, pe.y, pe.z, 0.f);
        return;
    }
    const float4 deh = S.dh, del = S.dl, pe = S.pe;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 mh4 = was ? S.mh : z4, ml4 = was ? S.ml : z4, vh4 = was ? S.vh : z4, vl4 = was ? S.vl : z4;
    df nd[3], nm[3], nv[3];
    float qo[3];
    const float pa[3] = {pe.x, pe.y, pe.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        df m = comp(mh4, ml4, a), vv = comp(vh4, vl4, a);
        m = df_add(df_mul(C.beta1, m), df_mul(C.one_m_beta1, g[a]));
        vv = df_add(df_mul(C.beta2, vv), df_mul(C.one_m_beta2, df_mul(g[a], g[a])));
        const df mhat = df_mul(m, ibc1);
        const df vhat = df_mul(vv, ibc2);
        const df den = df_add(df_sqrt(vhat), C.eps_adam);
        const df step = df_div(df_mul(C.alpha, mhat), den);
        nd[a] = df_clamp(df_sub(comp(deh, del, a), step), C.xi_box);
        nm[a] = m;
        nv[a] = vv;
        const df sp = two_sum(pa[a], nd[a].hi);
        qo[a] = __fadd_rn(sp.hi, __fadd_rn(sp.lo, nd[a].lo));
    }
    Nh[e] = make_float4(nd[0].hi, nd[1].hi, nd[2].hi, 0.f);
    Nl[e] = make_float4(nd[0].lo, nd[1].lo, nd[2].lo, 0.f);
    Mhi[e] = make_float4(nm[0].hi, nm[1].hi, nm[2].hi, 0.f);
    Mlo[e] = make_float4(nm[0].lo, nm[1].lo, nm[2].lo, 0.f);
    Vhi[e] = make_float4(nv[0].hi, nv[1].hi, nv[2].hi, 0.f);
    Vlo[e] = make_float4(nv[0].lo, nv[1].lo, nv[2].lo, 0.f);
    Qn[e] = make_float4(qo[0], qo[1], qo[2], 0.f);
}

// Adam on one row, loading its state from global memory.
__device__ __forceinline__ void adam_row(int64_t e, const df g[3], const float4 *Dh, const float4 *Dl,
                                         const float4 *__restrict__ PE, uint8_t *__restrict__ act, const df ibc1,
                                         const df ibc2, bool reset, const PgdConsts &C, float4 *Nh, float4 *Nl,
                                         float4 *__restrict__ Mhi, float4 *__restrict__ Mlo, float4 *__restrict__ Vhi,
                                         float4 *__restrict__ Vlo, float4 *Qn) {
    const bool gz = g[0].hi == 0.f && g[1].hi == 0.f && g[2].hi == 0.f;
    const uint8_t av = act[e];
    const bool was = (av & ACT_ON) != 0;
    if (!was && gz && !reset) return;
    RowState S;
    S.dh = Dh[e];
    S.dl = Dl[e];
    S.pe = PE[e];
    if (was) {
        S.mh = Mhi[e];
        S.ml = Mlo[e];
        S.vh = Vhi[e];
        S.vl = Vlo[e];
    }
    adam_core(e, g, S, was, av, act, ibc1, ibc2, reset, C, Nh, Nl, Mhi, Mlo, Vhi, Vlo, Qn);
}

// ------------------------------------------------------------------ stop decisions
// The tight loss is accumulated in fixed point: each violated pair adds llrint(v^2 / unit)
// with unit = xi^2 2^-24 (v <= 2 sqrt3 xi + delta_t, so a term is below 2^28 units and 2^35
// terms fit in 63 bits), and the violated pairs are counted: a pair counts when its
// violation exceeds b * 2^-40 (pairs held from both sides with an endpoint on the box can
// settle at v -> 0+, where the sign of v is decided by the last bits of the arithmetic;
// the margin's b * 2^-20 slack is far larger).  Integer sums do not depend on the order
// in which warps finish, so the result is deterministic although work items are handed
// out dynamically.  The block that finishes the launch last takes, for every block still
// iterating, the stop decision of Algorithm 1 for its check t (at eps_L = 0 the count
// decides).
__device__ void decide_blocks(const PgdConsts *__restrict__ CB, int nb, PgdBlk *blk, PgdGlobal *gs,
                              double *hist_loss, unsigned long long *hist_viol, const WorkTab *wt) {
    const int lane = threadIdx.x & 31;
    int active = 0;
    for (int b = lane; b < nb; b += 32) {
        PgdBlk &B = blk[b];
        if (B.stop) continue;
        const PgdConsts &C = CB[b];
        const int t = B.t;
        const bool last = is_last(C, t);
        const unsigned long long LF = atomicAdd(&B.lfx, 0ull), V = atomicAdd(&B.vacc, 0ull);
        const double L = (double)LF * C.loss_unit;
        if (hist_loss) {
            hist_loss[t] = L;
            hist_viol[t] = V;
        }
        if (t == 0) {
            B.loss0 = L;
            B.viol0 = V;
        }
        B.loss = L;
        B.viol = V;
        const bool replay = C.replay >= 0;
        const bool conv = C.loss_tol > 0.0 ? (L <= C.loss_tol) : (V == 0);
        B.upd_t = t;
        B.upd_ibc1 = B.ibc1;
        B.upd_ibc2 = B.ibc2;
        B.upd_reset = B.reset;
        if ((!replay && conv) || last) {
            B.stop = 1;
            B.final_buf = t & 1;
            B.converged = conv ? 1 : 0;
            B.upd_on = 0;
        } else {
            ++active;
            B.upd_on = 1;
            B.t = t + 1;
            const double b1 = B.b1p * C.beta1_d, b2 = B.b2p * C.beta2_d;
            B.b1p = b1;
            B.b2p = b2;
            const double i1 = 1.0 / (1.0 - b1), i2 = 1.0 / (1.0 - b2);
            df x, y;
            x.hi = (float)i1;
            x.lo = (float)(i1 - (double)x.hi);
            y.hi = (float)i2;
            y.lo = (float)(i2 - (double)y.hi);
            B.ibc1 = x;
            B.ibc2 = y;
            // stall rule on the loss of check t: progress is a fixed-point loss below
            // best - floor(best / 1024); `patience` checks without progress (stall_patience,
            // doubled after every reset) make the next launch reset the endpoints of its
            // violated pairs, provided their RMS violation exceeds xi / 1024 (LF > 16 V in
            // loss units): a slow tail of tiny violations is left to Adam
            if (B.reset) {
                B.reset = 0;
                B.best = ~0ull;
                B.since = 0;
            } else if (t == 0) {
                B.best = LF;
            } else if (LF < B.best - B.best / 1024) {
                B.best = LF;
                B.since = 0;
            } else if (C.stall_patience > 0 && ++B.since >= B.patience && LF > 16ull * V) {
                B.reset = 1;
                ++B.resets;
                B.since = 0;
                B.patience = B.patience < (1 << 24) ? 2 * B.patience : B.patience;
            }
        }
        B.lfx = 0;
        B.vacc = 0;
        B.n_upd += B.uacc;
        B.n_eval += B.eacc;
        B.uacc = 0;
        B.eacc = 0;
    }
    active = __reduce_add_sync(0xffffffffu, active);
    if (wt) {
        __syncwarp();
        __threadfence_block();
        build_worktab(nb, blk, *wt, gs);
    }
    if (lane == 0) {
        gs->active = active;
        if (active == 0) gs->all_stop = 1;
        gs->work = 0;
        gs->ticket = 0;
    }
    __threadfence();
}

struct BlockRed {
    unsigned long long lfx, viol, upd, ev;
    unsigned count;
};

// Warp partials -> block counters -> block 0's launch accumulators (single block), then
// the last block of the launch takes the decisions.
template <bool MULTI>
__device__ __forceinline__ void finish_iteration(BlockRed &br, unsigned long long lfx, unsigned long long viol,
                                                 unsigned long long upd, unsigned long long ev,
                                                 const PgdConsts *CB, int nb, PgdBlk *blk, PgdGlobal *gs,
                                                 double *hist_loss, unsigned long long *hist_viol,
                                                 const WorkTab &wt) {
    const int lane = threadIdx.x & 31;
    if (!MULTI) {
        lfx = warp_sum_u(lfx);
        viol = warp_sum_u(viol);
        upd = warp_sum_u(upd);
        ev = warp_sum_u(ev);
    }
    unsigned prev = 0;
    if (lane == 0) {
        if (!MULTI) {
            if (lfx) atomicAdd(&br.lfx, lfx);
            if (viol) atomicAdd(&br.viol, viol);
            if (upd) atomicAdd(&br.upd, upd);
            if (ev) atomicAdd(&br.ev, ev);
        }
        __threadfence_block();
        prev = atomicAdd(&br.count, 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != WARPS - 1) return;          // not the last warp of this block
    unsigned gprev = 0;
    if (lane == 0) {
        __threadfence_block();
        if (!MULTI) {
            const unsigned long long bl = atomicAdd(&br.lfx, 0ull), bv = atomicAdd(&br.viol, 0ull),
                                     bu = atomicAdd(&br.upd, 0ull), be = atomicAdd(&br.ev, 0ull);
            if (bl) atomicAdd(&blk[0].lfx, bl);
            if (bv) atomicAdd(&blk[0].vacc, bv);
            if (bu) atomicAdd(&blk[0].uacc, bu);
            if (be) atomicAdd(&blk[0].eacc, be);
        }
        __threadfence();
        gprev = atomicAdd(&gs->ticket, 1u);
    }
    gprev = __shfl_sync(0xffffffffu, gprev, 0);
    if (gprev != gridDim.x - 1) return;     // not the last block
    __threadfence();
    decide_blocks(CB, nb, blk, gs, hist_loss, hist_viol, MULTI ? &wt : nullptr);
}

// ------------------------------------------------------------------ iteration kernel
struct HeavyPlan {
    int64_t n_chunks;                          // heavy chunks (one warp each)
    const uint32_t *chunk_row;                 // row of each chunk
    const unsigned long long *chunk_start;     // first edge of each chunk in the edge array
    const uint32_t *chunk_len;                 // edges of each chunk (at most HEAVY)
    float4 *chunk_g;                           // per chunk: gradient partial (hi at 2c, lo at 2c+1)
};

// One edge array holds the light rows' edges, in row order, then the heavy rows' edges
// (chunks index into that second part).  A group of 32 light rows owns the contiguous
// range [ptr[r0], ptr[r0 + 32]) (heavy rows own no light edge), and each light edge
// carries the slot of its row within the group, so a warp maps an edge to its row with
// one byte load.  Offsets are 64-bit: a problem may have more than 2^32 directed edges.
struct LightPlan {
    const unsigned long long *ptr;   // per row: first light edge (ne + 1 entries)
    const uint32_t *col;             // partner | link << 31 (| threshold index << 29 with several)
    const uint8_t *slot;             // light edges: row - first row of its 32-row group
};

struct PgdBufs {
    float4 *Dh[2], *Dl[2], *Q[2];
    float4 *Mh, *Ml, *Vh, *Vl;
    uint8_t *act;
    // buffer i of a ping-pong pair, chosen without indexing the parameter array at run
    // time (which would copy it to local memory)
    __device__ __forceinline__ float4 *dh(int i) const { return i ? Dh[1] : Dh[0]; }
    __device__ __forceinline__ float4 *dl(int i) const { return i ? Dl[1] : Dl[0]; }
    __device__ __forceinline__ float4 *q(int i) const { return i ? Q[1] : Q[0]; }
};

// A row whose Adam step waits in its warp's queue: the row, its block and flags
// (block | buffer parity << 31 | had a gradient before << 30 | stall reset << 29) and
// its gradient as three double-floats.
struct AdamEnt {
    uint32_t e, meta;
    float g[6];
};

#ifndef PC_PGD_EPL
#define PC_PGD_EPL 4
#endif
constexpr int EPL = PC_PGD_EPL;   // edges per lane per trip of the edge walk
constexpr int QCAP = 256;  // uncertain pairs waiting for evaluation (a ring per warp; < 32 + EPL x 32)
constexpr int ACAP = 64;   // rows waiting for their Adam step (a ring per warp)

struct WarpTab {
    uint32_t qk[QCAP];               // queued pairs: partner
    uint8_t qs[QCAP];                // queued pairs: row slot | threshold index << 5 | link << 7
    float4 q[32];                    // the rows' rounded current positions
    unsigned own[32];                // per row slot: this batch's violated entries of that row
    float gt[6][32];                 // this batch's gradient terms (x hi, x lo, y hi, ...) by entry
    AdamEnt aq[ACAP];                // rows whose gradient is complete, waiting for Adam
};

// One PGD iteration for every block still iterating: check t_b and, unless it is the
// block's last check, the update t_b + 1.
//
// Work items are groups of 32 consecutive light rows (editable particles) or one chunk
// of HEAVY edges of a heavy row, handed out from a counter.  A warp walks the flat edge
// range of its item 128 edges at a time (4 per lane, strided by 32 so that loads stay
// coalesced and edge order is lane order within each 32-edge slice).  The float32 screen
// on the rounded current positions Q certifies most pairs as satisfied; one warp vote
// skips the queue when a whole trip is certified.  The others enter, in edge order, the
// warp's ring of uncertain pairs, which the 32 lanes evaluate 32 at a time in
// double-float; each row then adds its violated pairs one by one in edge order, so a
// row's gradient does not depend on how rows are grouped into warps, batches or blocks
// of the problem set.  A light row whose gradient is complete enters the warp's Adam
// ring; whenever 32 rows are waiting, the warp applies Adam to them with every lane
// busy (rows that need no update never enter, so the update runs on full warps).  A
// heavy warp writes its chunk partial and k_pgd_heavy adds the partials of a heavy row
// in chunk order.  MULTI = false is the single-block specialisation; with MULTI the
// items come from the table of blocks still iterating, so a block that has stopped
// costs nothing in later launches, and the rows of one item share a block.  MT: the
// problem has several linking lengths and each CSR entry carries the index of its pair's
// (single block only); the screen and the evaluation use that length's thresholds.
template <bool MULTI, bool MT>
__global__ void __launch_bounds__(PGD_THREADS, PGD_BLOCKS_PER_SM) k_pgd_iter(
    const float4 *__restrict__ PE, int64_t ne, PgdBufs Bf, HeavyPlan H, LightPlan LP,
    const PgdConsts *__restrict__ CB, int nb, PgdBlk *blk, PgdGlobal *gs, const WorkTab wt,
    double *__restrict__ hist_loss, unsigned long long *__restrict__ hist_viol) {
    __shared__ int s_stop, s_t, s_reset, s_nact;
    __shared__ unsigned long long s_items;
    __shared__ df s_ibc1, s_ibc2;
    __shared__ WarpTab tab[WARPS];
    __shared__ BlockRed br;
    if (threadIdx.x == 0) {
        s_stop = gs->all_stop;
        s_nact = gs->active;
        s_items = gs->n_items;
        s_t = blk[0].t;
        s_ibc1 = blk[0].ibc1;
        s_ibc2 = blk[0].ibc2;
        s_reset = blk[0].reset;
        br.count = 0;
        br.lfx = 0;
        br.viol = 0;
        br.upd = 0;
        br.ev = 0;
    }
    __syncthreads();
    if (s_stop) return;

    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << (threadIdx.x & 31)) - 1u;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpTab &T = tab[w];
    // this lane's share of the tight loss (fixed point), violations, rows updated and
    // pairs evaluated (single block: summed at the end of the launch)
    unsigned long long lfx = 0;
    unsigned viol = 0, nupd = 0, nev = 0;
    const int64_t n_light_warps = (ne + 31) / 32;
    const int64_t n_items = MULTI ? (int64_t)s_items : n_light_warps + H.n_chunks;
    int ahead = 0, an = 0;   // Adam ring: first entry, entries waiting

    // Adam on the first c rows of the ring (lane i takes row i).
    auto adam_flush = [&](int c) {
        if (lane < c) {
            const AdamEnt &A = T.aq[(ahead + lane) & (ACAP - 1)];
            const uint32_t e = A.e, meta = A.meta;
            const int b = MULTI ? (int)(meta & 0x1fffffffu) : 0;
            const int pa = (int)(meta >> 31);
            const bool was = ((meta >> 30) & 1u) != 0, rs = ((meta >> 29) & 1u) != 0;
            const df g[3] = {df_make(A.g[0], A.g[1]), df_make(A.g[2], A.g[3]), df_make(A.g[4], A.g[5])};
            RowState S;
            S.dh = Bf.dh(pa)[e];
            S.dl = Bf.dl(pa)[e];
            S.pe = PE[e];
            if (was) {
                S.mh = Bf.Mh[e];
                S.ml = Bf.Ml[e];
                S.vh = Bf.Vh[e];
                S.vl = Bf.Vl[e];
            }
            const df i1 = MULTI ? blk[b].ibc1 : s_ibc1, i2 = MULTI ? blk[b].ibc2 : s_ibc2;
            adam_core(e, g, S, was, was ? ACT_ON : (uint8_t)0, Bf.act, i1, i2, rs, CB[b], Bf.dh(pa ^ 1),
                      Bf.dl(pa ^ 1), Bf.Mh, Bf.Ml, Bf.Vh, Bf.Vl, Bf.q(pa ^ 1));
        }
        ahead = (ahead + c) & (ACAP - 1);
        an -= c;
        __syncwarp();
    };

    // One loop, one place where Adam runs: a full warp's worth of waiting rows goes first;
    // after the last item, whatever is left.
    bool done = false;
    // the next item is claimed one item ahead, so the claim's round trip overlaps a walk
    unsigned long long nitm = 0;
    if (lane == 0) nitm = atomicAdd(&gs->work, 1ull);
    for (;;) {
        if (an >= 32 || (done && an > 0)) {
            adam_flush(min(an, 32));
            continue;
        }
        if (done) break;
        const int64_t item = (int64_t)__shfl_sync(FULL, nitm, 0);
        if (lane == 0 && item < n_items) nitm = atomicAdd(&gs->work, 1ull);
        if (item >= n_items) {
            done = true;
            continue;
        }

        // the item's block: iteration, buffers and screen constants (one block per item)
        int b = 0, tb = s_t;
        bool bstop = false;
        int64_t r0 = 0, item_chunk = 0;
        int cnt = 0;
        bool heavy_warp;
        if (MULTI) {
            // active block of the item: largest k with act_pref[k] <= item
            int kk = 0;
            if (lane == 0) {
                int lo = 0, hi = s_nact - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (wt.act_pref[mid] <= (unsigned long long)item) lo = mid;
                    else hi = mid - 1;
                }
                kk = lo;
            }
            kk = __shfl_sync(FULL, kk, 0);
            b = (int)wt.act_blk[kk];
            const int64_t j = item - (int64_t)wt.act_pref[kk];
            const BlkWork bw = wt.bw[b];
            const int64_t nl = (bw.nrows + 31u) >> 5;
            heavy_warp = j >= nl;
            if (!heavy_warp) {
                r0 = (int64_t)bw.row0 + 32 * j;
                cnt = (int)min((int64_t)32, (int64_t)bw.nrows - 32 * j);
            } else {
                item_chunk = (int64_t)bw.ch0 + (j - nl);
            }
            tb = blk[b].t;
            bstop = blk[b].stop != 0;
        } else {
            heavy_warp = item >= n_light_warps;
            if (!heavy_warp) {
                r0 = item * 32;
                cnt = (int)min((int64_t)32, ne - r0);
            } else {
                item_chunk = item - n_light_warps;
            }
        }
        const int pa = tb & 1;

        // Edge range [ebase, ebase + VT) of the edge array: the light edges of the item's
        // rows (each with its row's slot), or one heavy chunk (slot 0).  rbase: the row of
        // slot 0.
        int64_t rbase = r0, chunk = -1;
        bool upd = false, was = false;   // the lane's row takes an update at this launch; had a gradient
        uint32_t VT = 0;
        unsigned long long ebase = 0;
        float4 qe = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!heavy_warp) {
            const bool have = lane < cnt;
            uint8_t av = 0;
            if (have) {
                const int64_t e = r0 + lane;
                av = Bf.act[e];
                qe = Bf.q(pa)[e];
                T.q[lane] = qe;
            }
            const bool own = have && !bstop && !(av & ACT_HEAVY);
            upd = own && !is_last(CB[b], tb);
            was = (av & ACT_ON) != 0;
            unsigned long long lb = 0, le = 0;
            if (lane == 0) {
                lb = LP.ptr[r0];
                le = LP.ptr[r0 + cnt];
            }
            ebase = __shfl_sync(FULL, lb, 0);
            VT = bstop ? 0u : (uint32_t)(__shfl_sync(FULL, le, 0) - ebase);
        } else {
            chunk = item_chunk;
            const uint32_t row = H.chunk_row[chunk];
            ebase = H.chunk_start[chunk];
            VT = bstop ? 0u : H.chunk_len[chunk];
            rbase = row;
            qe = Bf.q(pa)[row];
            if (lane == 0) T.q[0] = qe;
        }
        __syncwarp();
        const PgdConsts &Cl = CB[b];            // the item's block
        const float sl_link = Cl.screen_link[0], sl_non = Cl.screen_non[0];
        constexpr uint32_t PMASK = MT ? 0x1fffffffu : 0x7fffffffu;   // partner bits of a CSR entry
        // a warp whose rows all sit in the box's interior screens without the minimum image
        // (it never wraps there, so the screen's d2 is the same bit for bit)
        const bool row_lane = heavy_warp || lane < cnt;
        const bool in_ok = Cl.interior_ok != 0 &&
                           (!row_lane || (qe.x >= Cl.ilo[0] && qe.x <= Cl.ihi[0] && qe.y >= Cl.ilo[1] &&
                                          qe.y <= Cl.ihi[1] && qe.z >= Cl.ilo[2] && qe.z <= Cl.ihi[2]));
        const bool pp = Cl.periodic != 0 && !__all_sync(FULL, in_ok);
        const float L0 = Cl.L[0], L1 = Cl.L[1], L2 = Cl.L[2];
        const float4 *Qc = Bf.q(pa);
        const float4 *Dh = Bf.dh(pa), *Dl = Bf.dl(pa);

        df g[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};   // gradient of the lane's row
        bool rv = false;             // the lane's row has a violated pair
        int qh = 0, qn = 0;          // uncertain-pair ring: first entry, entries waiting

        // Evaluates the first min(qn, 32) queued pairs and adds each violated pair's term
        // to its row's gradient.
        auto batch = [&]() {
            const int c = min(qn, 32);
            const bool valid = lane < c;
            int s = 32;
            df gt[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};
            bool hit = false;
            if (valid) {
                const int pos = (qh + lane) & (QCAP - 1);
                const uint32_t k = T.qk[pos];
                const uint32_t qsv = T.qs[pos];
                s = (int)(qsv & 0x1fu);
                const int ti = MT ? (int)((qsv >> 5) & 3u) : 0;
                const bool link = (qsv >> 7) != 0;
                const int64_t er = rbase + s;
                double ltv = 0.0;
                bool counts = false;
                hit = eval_pair(PE[er], Dh[er], Dl[er], er, k, link, ti, PE, Dh, Dl, Cl, gt, ltv, counts);
                if (hit) {
                    lfx += (unsigned long long)llrint(ltv);
                    viol += ((int64_t)k > er && counts) ? 1u : 0u;
                }
                ++nev;
            }
            // Each row adds its violated pairs one by one in edge order (queue order is
            // edge order).  The row's owner is lane `slot` (light) or lane 0 (heavy: slot 0):
            // the entries of a slot are found with one match, and every owner walks its own
            // entries while the others walk theirs.
            if (hit) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    T.gt[2 * a][lane] = gt[a].hi;
                    T.gt[2 * a + 1][lane] = gt[a].lo;
                }
            }
            const unsigned hm = __ballot_sync(FULL, hit);
            T.own[lane] = 0u;
            const unsigned same = __match_any_sync(FULL, s);
            __syncwarp();
            if (hit) T.own[s] = same & hm;   // the entries of one slot all write the same mask
            __syncwarp();
            for (unsigned mine = T.own[lane]; mine; mine &= mine - 1) {
                const int i = __ffs(mine) - 1;
#pragma unroll
                for (int a = 0; a < 3; ++a) g[a] = df_add(g[a], df_make(T.gt[2 * a][i], T.gt[2 * a + 1][i]));
                rv = true;
            }
            qh = (qh + c) & (QCAP - 1);
            qn -= c;
            __syncwarp();
        };

        // float32 screen of one edge of row slot s against partner cv: true when the pair
        // may be violated (the double-float evaluation decides)
        auto screen = [&](bool ok, int s, uint32_t cv) -> bool {
            if (!ok) return false;
            const float4 qr = T.q[s];
            const float4 qk = Qc[cv & PMASK];
            const float d2 =
                cdist2(cdiff(qr.x, qk.x, pp, L0), cdiff(qr.y, qk.y, pp, L1), cdiff(qr.z, qk.z, pp, L2));
            if (MT) {
                const int ti = (cv >> 29) & 3;
                return (cv >> 31) ? !(d2 < Cl.screen_link[ti]) : !(d2 > Cl.screen_non[ti]);
            }
            return (cv >> 31) ? !(d2 < sl_link) : !(d2 > sl_non);
        };

        const uint32_t *__restrict__ ecol = LP.col + ebase;
        const uint8_t *__restrict__ eslot = LP.slot + ebase;
        // software pipeline: the columns and slots of the next trip are loaded before this
        // trip's partner positions are gathered, so each trip waits on one round trip
        uint32_t cvn[EPL];
        int sln[EPL];
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
            const uint32_t v = 32u * j + lane;
            cvn[j] = v < VT ? __ldcs(ecol + v) : 0u;
            sln[j] = (v < VT && !heavy_warp) ? (int)__ldcs(eslot + v) : 0;
        }
        for (uint32_t base = 0; base < VT; base += 32 * EPL) {
            uint32_t cv[EPL];
            int sl[EPL];
            bool nd[EPL];
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                nd[j] = base + 32u * j + lane < VT;
                cv[j] = cvn[j];
                sl[j] = sln[j];
                const uint32_t v = base + 32u * (EPL + j) + lane;
                cvn[j] = v < VT ? __ldcs(ecol + v) : 0u;
                sln[j] = (v < VT && !heavy_warp) ? (int)__ldcs(eslot + v) : 0;
            }
            bool any = false;
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                nd[j] = screen(nd[j], sl[j], cv[j]);
                any |= nd[j];
            }
            if (!__any_sync(FULL, any)) continue;
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                const unsigned bal = __ballot_sync(FULL, nd[j]);
                if (nd[j]) {
                    const int pos = (qh + qn + __popc(bal & lt_mask)) & (QCAP - 1);
                    T.qk[pos] = cv[j] & PMASK;
                    T.qs[pos] = (uint8_t)(sl[j] | (MT ? ((cv[j] >> 29) & 3u) << 5 : 0u) | ((cv[j] >> 31) ? 0x80 : 0));
                }
                qn += __popc(bal);
            }
            __syncwarp();
            while (qn >= 32) batch();
        }
        while (qn > 0) batch();

        if (!heavy_warp) {
            // rows whose update is due join the Adam ring; a full warp's worth is applied
            bool need = false, rs = false;
            if (upd) {
                rs = rv && (MULTI ? blk[b].reset != 0 : s_reset != 0);
                const bool gz = g[0].hi == 0.f && g[1].hi == 0.f && g[2].hi == 0.f;
                need = was || !gz || rs;
            }
            const unsigned bal = __ballot_sync(FULL, need);
            if (need) {
                AdamEnt &A = T.aq[(ahead + an + __popc(bal & lt_mask)) & (ACAP - 1)];
                A.e = (uint32_t)(r0 + lane);
                A.meta = (MULTI ? (uint32_t)b : 0u) | ((uint32_t)pa << 31) | ((uint32_t)was << 30) |
                         ((uint32_t)rs << 29);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    A.g[2 * a] = g[a].hi;
                    A.g[2 * a + 1] = g[a].lo;
                }
            }
            const int nn = __popc(bal);
            an += nn;
            if (!MULTI) nupd += (lane == 0) ? (unsigned)nn : 0u;
            __syncwarp();
            if (MULTI && lane == 0 && nn) atomicAdd(&blk[b].uacc, (unsigned long long)nn);
        } else if (lane == 0 && !bstop) {
            H.chunk_g[2 * chunk] = make_float4(g[0].hi, g[1].hi, g[2].hi, rv ? 1.f : 0.f);
            H.chunk_g[2 * chunk + 1] = make_float4(g[0].lo, g[1].lo, g[2].lo, 0.f);
        }
        if (MULTI) {
            // the item's loss, violations and evaluations belong to its block
            const unsigned long long il = warp_sum_u(lfx), iv = __reduce_add_sync(FULL, viol),
                                     ie = __reduce_add_sync(FULL, nev);
            if (lane == 0 && !bstop) {
                if (il) atomicAdd(&blk[b].lfx, il);
                if (iv) atomicAdd(&blk[b].vacc, iv);
                if (ie) atomicAdd(&blk[b].eacc, ie);
            }
            lfx = 0;
            viol = 0;
            nev = 0;
        }
        __syncwarp();
    }   // work items
    finish_iteration<MULTI>(br, lfx, viol, nupd, nev, CB, nb, blk, gs, hist_loss, hist_viol, wt);
}

// Heavy rows: sum the chunk partials in chunk order and apply Adam (same update as
// light rows), with the check index and step of the iteration launch just finished.
__global__ void k_pgd_heavy(const uint32_t *__restrict__ hrow, const uint32_t *__restrict__ hc0, int64_t nh,
                            const float4 *__restrict__ chunk_g, const float4 *__restrict__ PE,
                            const uint32_t *__restrict__ rb, PgdBufs Bf, const PgdConsts *__restrict__ CB,
                            PgdBlk *blk) {
    GRID_STRIDE(i, nh) {
        const uint32_t e = hrow[i];
        const int b = (int)rb[e];
        PgdBlk &B = blk[b];
        if (!B.upd_on) continue;
        const int pa = B.upd_t & 1;
        df g[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};
        bool rv = false;
        for (uint32_t c = hc0[i]; c < hc0[i + 1]; ++c) {
            const float4 h = chunk_g[2 * c], l = chunk_g[2 * c + 1];
            rv |= h.w != 0.f;
            g[0] = df_add(g[0], df_make(h.x, l.x));
            g[1] = df_add(g[1], df_make(h.y, l.y));
            g[2] = df_add(g[2], df_make(h.z, l.z));
        }
        const bool gz = g[0].hi == 0.f && g[1].hi == 0.f && g[2].hi == 0.f;
        const bool rs = rv && B.upd_reset != 0;
        if ((Bf.act[e] & ACT_ON) || !gz || rs) atomicAdd(&B.n_upd, 1ull);
        adam_row(e, g, Bf.dh(pa), Bf.dl(pa), PE, Bf.act, B.upd_ibc1, B.upd_ibc2, rs, CB[b], Bf.dh(pa ^ 1),
                 Bf.dl(pa ^ 1), Bf.Mh, Bf.Ml, Bf.Vh, Bf.Vl, Bf.q(pa ^ 1));
    }
}

// ------------------------------------------------------------------ edge plan
// Degrees from the CSR offsets: light degree (0 for a heavy row), heavy degree, chunk
// count and heavy flag of every row; the heavy bit also goes into act.
__global__ void k_degrees(const unsigned long long *__restrict__ row_ptr, int64_t ne,
                          unsigned long long *__restrict__ ldeg, unsigned long long *__restrict__ hdeg,
                          uint32_t *__restrict__ nchunk, uint32_t *__restrict__ isheavy, uint8_t *__restrict__ act) {
    GRID_STRIDE(e, ne) {
        const unsigned long long d = row_ptr[e + 1] - row_ptr[e];
        const bool h = d > HEAVY;
        ldeg[e] = h ? 0ull : d;
        hdeg[e] = h ? d : 0ull;
        nchunk[e] = h ? (uint32_t)((d + HEAVY - 1) / HEAVY) : 0u;
        isheavy[e] = h ? 1u : 0u;
        if (h) act[e] = (uint8_t)(act[e] | ACT_HEAVY);
    }
}

// Squared linking lengths of the thresholds of a multi-threshold problem (float32).
struct ThrB2 {
    float b2[MAX_THR];
};

// One CSR entry per directed edge t (sorted keys: row, partner position, threshold
// index): partner's dense index, threshold index and the link flag at the pair's own
// linking length, written to the row's place in the edge array (light rows: their
// group's range, with the row's slot; heavy rows: after every light edge).
__global__ void k_cols(const unsigned long long *__restrict__ keys, int64_t m, int nb, int tb, ThrB2 tb2,
                       const unsigned long long *__restrict__ row_ptr, const unsigned long long *__restrict__ lptr,
                       const unsigned long long *__restrict__ hptr, unsigned long long n_light,
                       const uint32_t *__restrict__ dense, const uint32_t *__restrict__ epos,
                       const uint32_t *__restrict__ rb, const int64_t *__restrict__ roff,
                       const float4 *__restrict__ P4, const BlockDev *__restrict__ bt, const int64_t *__restrict__ off,
                       int nblk, uint32_t *__restrict__ ecol, uint8_t *__restrict__ eslot) {
    const unsigned long long mask = (1ull << nb) - 1ull;
    GRID_STRIDE(t, m) {
        const unsigned long long k = keys[t];
        const uint32_t ti = (uint32_t)(k & ((1ull << tb) - 1ull));
        const uint32_t row = (uint32_t)(k >> (nb + tb)), nbp = (uint32_t)((k >> tb) & mask);
        const uint32_t pos = epos[row];
        const BlockDev &B = bt[find_block(off, nblk, pos)];
        const float4 p = P4[pos], q = P4[nbp];
        const float3 d = canon_dp(p, q, B.periodic, B.L);
        // the link flag at the pair's own linking length
        const float b2 = tb ? (ti == 0 ? tb2.b2[0] : ti == 1 ? tb2.b2[1] : ti == 2 ? tb2.b2[2] : tb2.b2[3]) : B.b2;
        const bool link = cdist2(d.x, d.y, d.z) <= b2;
        const uint32_t cv = dense[nbp] | (ti << 29) | (link ? 0x80000000u : 0u);
        const unsigned long long r_lo = row_ptr[row], j = (unsigned long long)t - r_lo;
        if (row_ptr[row + 1] - r_lo > HEAVY) {
            ecol[n_light + hptr[row] + j] = cv;
        } else {
            const unsigned long long dst = lptr[row] + j;
            const int64_t r0 = roff ? roff[rb[row]] : 0;
            ecol[dst] = cv;
            eslot[dst] = (uint8_t)(((int64_t)row - r0) & 31);
        }
    }
}

// Heavy rows: the chunks (row, first edge, length) and the per-row chunk ranges.
__global__ void k_heavy_fill(const unsigned long long *__restrict__ hdeg, const unsigned long long *__restrict__ hptr,
                             unsigned long long n_light, int64_t ne, const uint32_t *__restrict__ nchunk,
                             const uint32_t *__restrict__ c0, const uint32_t *__restrict__ isheavy,
                             const uint32_t *__restrict__ hpos, uint32_t *__restrict__ chunk_row,
                             unsigned long long *__restrict__ chunk_start, uint32_t *__restrict__ chunk_len,
                             uint32_t *__restrict__ hrow, uint32_t *__restrict__ hc0) {
    GRID_STRIDE(e, ne) {
        if (!isheavy[e]) continue;
        const uint32_t c = c0[e];
        const unsigned long long d = hdeg[e];
        for (uint32_t j = 0; j < nchunk[e]; ++j) {
            const unsigned long long s0 = (unsigned long long)j * HEAVY;
            chunk_row[c + j] = (uint32_t)e;
            chunk_start[c + j] = n_light + hptr[e] + s0;
            chunk_len[c + j] = (uint32_t)min((unsigned long long)HEAVY, d - s0);
        }
        hrow[hpos[e]] = (uint32_t)e;
        hc0[hpos[e]] = c;
    }
}

__global__ void k_copy_recon(const float *__restrict__ recon, float *__restrict__ out, int64_t m) {
    GRID_STRIDE(i, m) out[i] = recon[i];
}

// Corrected output: P + delta of the block's final buffer, rounded once; blocks that
// stopped at check 0 keep the reconstruction.
__global__ void k_output(const float4 *__restrict__ PE, const uint32_t *__restrict__ rb, int64_t e0, int64_t cnt,
                         PgdBufs Bf, const PgdBlk *__restrict__ blk, float *__restrict__ out) {
    GRID_STRIDE(i, cnt) {
        const int64_t e = e0 + i;
        const PgdBlk &B = blk[rb[e]];
        if (B.t == 0) continue;
        const int fb = B.final_buf;
        const float4 p = PE[e], h = Bf.dh(fb)[e], l = Bf.dl(fb)[e];
        const int64_t id = (int64_t)__float_as_uint(p.w);
        const float pa[3] = {p.x, p.y, p.z}, ha[3] = {h.x, h.y, h.z}, la[3] = {l.x, l.y, l.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const df s = two_sum(pa[a], ha[a]);
            out[3 * id + a] = __fadd_rn(s.hi, __fadd_rn(s.lo, la[a]));
        }
    }
}

__global__ void k_delta_out(const float4 *__restrict__ PE, const uint32_t *__restrict__ rb, int64_t ne, PgdBufs Bf,
                            const PgdBlk *__restrict__ blk, double *__restrict__ out) {
    GRID_STRIDE(e, ne) {
        const int fb = blk[rb[e]].final_buf;
        const float4 p = PE[e], h = Bf.dh(fb)[e], l = Bf.dl(fb)[e];
        const int64_t id = (int64_t)__float_as_uint(p.w);
        out[3 * id + 0] = (double)h.x + (double)l.x;
        out[3 * id + 1] = (double)h.y + (double)l.y;
        out[3 * id + 2] = (double)h.z + (double)l.z;
    }
}

float f32_down(double x) {
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}
float f32_up(double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}
double ulp32(double x) {
    int e = 0;
    std::frexp(std::fabs(x), &e);
    return std::ldexp(1.0, e - 24);
}

PgdConsts pgd_consts(const Consts &c, const pc_params *p) {
    PgdConsts K;
    memset(&K, 0, sizeof(K));
    K.periodic = c.periodic;
    for (int a = 0; a < 3; ++a) K.L[a] = c.L[a];
    K.b2 = c.b2;
    const double thrL = c.b - c.dt, thrN = c.b + c.dt;
    // screen bound: the float32 difference of the rounded current positions differs from the
    // exact offset by at most one ulp of the coordinates plus one ulp of |r| per axis
    const double R = c.b + 2.0 * std::sqrt(3.0) * c.xi + 4.0 * c.xi;
    const double B4 = 2.0 * std::sqrt(3.0) * (ulp32(c.M + 2.0 * c.xi) + ulp32(R));
    K.screen_link[0] = thrL - B4 > 0 ? f32_down((thrL - B4) * (thrL - B4) * (1.0 - std::ldexp(1.0, -20))) : -1.0f;
    K.screen_non[0] = f32_up((thrN + B4) * (thrN + B4) * (1.0 + std::ldexp(1.0, -20)));
    K.tau[0] = (float)std::ldexp(c.b, -30);
    K.thr_link[0] = df_split(thrL);
    K.thr_non[0] = df_split(thrN);
    K.vtol[0] = std::ldexp(c.b, -40);
    K.interior_ok = c.interior_ok;
    for (int a = 0; a < 3; ++a) {   // rounded toward the interior
        K.ilo[a] = f32_up(c.in_lo[a]);
        K.ihi[a] = f32_down(c.in_hi[a]);
    }
    for (int k = 1; k < MAX_THR; ++k) {
        K.vtol[k] = K.vtol[0];
        K.screen_link[k] = K.screen_link[0];
        K.screen_non[k] = K.screen_non[0];
        K.tau[k] = K.tau[0];
        K.thr_link[k] = K.thr_link[0];
        K.thr_non[k] = K.thr_non[0];
    }
    K.xi_box = df_split(c.xi_box_d);
    K.alpha = df_split(p->alpha_rel * c.xi);
    K.eps_adam = df_split(p->eps_rel * c.xi);
    K.beta1 = df_split(p->beta1);
    K.one_m_beta1 = df_split(1.0 - p->beta1);
    K.beta2 = df_split(p->beta2);
    K.one_m_beta2 = df_split(1.0 - p->beta2);
    K.t_max = p->t_max;
    K.replay = p->replay_iters;
    K.loss_tol = p->loss_tol;
    K.beta1_d = p->beta1;
    K.beta2_d = p->beta2;
    K.loss_unit = c.xi * c.xi * std::ldexp(1.0, -24);
    K.inv_loss_unit = 1.0 / K.loss_unit;
    K.stall_patience = p->stall_patience;
    return K;
}

// The thresholds of several linking lengths (constants of each, same xi, m and data).
void pgd_thresholds(PgdConsts &K, const std::vector<Consts> &ck, const pc_params *p) {
    for (size_t k = 0; k < ck.size(); ++k) {
        const PgdConsts one = pgd_consts(ck[k], p);
        K.screen_link[k] = one.screen_link[0];
        K.screen_non[k] = one.screen_non[0];
        K.tau[k] = one.tau[0];
        K.thr_link[k] = one.thr_link[0];
        K.thr_non[k] = one.thr_non[0];
        K.vtol[k] = one.vtol[0];
    }
}

}  // namespace

// ------------------------------------------------------------------ resumable solver
struct PgdSolver::Impl {
    cudaStream_t s = 0;
    int nb = 0;
    int64_t ne = 0, n_heavy = 0, max_checks = 0;
    int nblk = 1;
    double *hist_loss = nullptr;
    unsigned long long *hist_viol = nullptr;
    DBuf<PgdConsts> CB;
    DBuf<PgdBlk> blk;
    DBuf<PgdGlobal> gs;
    DBuf<uint32_t> rb, chunk_row, chunk_len, hrow, hc0, ecol;
    DBuf<unsigned long long> lptr, chunk_start;
    DBuf<uint8_t> eslot;
    LightPlan LP{};
    DBuf<float4> PE, Dh0, Dl0, Dh1, Dl1, Mh, Ml, Vh, Vl, Q0, Q1, chunk_g;
    DBuf<uint8_t> act;
    DBuf<BlkWork> bw;
    DBuf<uint32_t> act_blk;
    DBuf<unsigned long long> act_pref;
    WorkTab wt{};
    PgdBufs Bf;
    HeavyPlan HP;
    std::vector<int64_t> row_off;            // rows of block b: [row_off[b], row_off[b+1])
    // status copies
    uint8_t *pin = nullptr;                  // nb PgdBlk + one PgdGlobal, pinned
    cudaEvent_t ev = nullptr;
    bool posted = false;
    // graph of `graph_k` iteration launches
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_k = 0;
    int kernels_per_iter = 1;

    bool mt = false;                         // several linking lengths (single block)

    void launch_iter() {
        if (mt)
            k_pgd_iter<false, true><<<nblk, PGD_THREADS, 0, s>>>(PE.p, ne, Bf, HP, LP, CB.p, nb, blk.p, gs.p, wt,
                                                                 hist_loss, hist_viol);
        else if (nb == 1)
            k_pgd_iter<false, false><<<nblk, PGD_THREADS, 0, s>>>(PE.p, ne, Bf, HP, LP, CB.p, nb, blk.p, gs.p, wt,
                                                                  hist_loss, hist_viol);
        else
            k_pgd_iter<true, false><<<nblk, PGD_THREADS, 0, s>>>(PE.p, ne, Bf, HP, LP, CB.p, nb, blk.p, gs.p, wt,
                                                                 nullptr, nullptr);
        PC_CHECK_LAUNCH();
        if (n_heavy > 0) {
            k_pgd_heavy<<<grid_for(n_heavy), 256, 0, s>>>(hrow.p, hc0.p, n_heavy, chunk_g.p, PE.p, rb.p, Bf, CB.p,
                                                          blk.p);
            PC_CHECK_LAUNCH();
        }
    }
    ~Impl() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev) cudaEventDestroy(ev);
        if (pin) cudaFreeHost(pin);
    }
};

PgdSolver::PgdSolver(const Binned &B, const BlockSet &S, const std::vector<Consts> &cp, const float *orig,
                     const float *recon, const unsigned long long *A, int64_t nA, cudaStream_t s, HostScratch &hs,
                     double *hist_loss, unsigned long long *hist_viol, const ThrSet *thr)
    : im(new Impl()) {
    Impl &I = *im;
    I.s = s;
    const int nb = S.nb;
    I.nb = nb;
    I.mt = thr && thr->c.size() > 1;
    if (I.mt && (nb != 1 || thr->c.size() > (size_t)MAX_THR || !thr->Athr))
        fail(PC_EINVAL, "several linking lengths: one block and at most 4 lengths");
    I.hist_loss = hist_loss;
    I.hist_viol = hist_viol;
    const int64_t n = B.n;
    PC_CUDA(cudaEventCreateWithFlags(&I.ev, cudaEventDisableTiming));
    PC_CUDA(cudaMallocHost((void **)&I.pin, nb * sizeof(PgdBlk) + sizeof(PgdGlobal)));

    // ---- constants and iteration state per block
    std::vector<PgdConsts> hK(nb);
    std::vector<PgdBlk> hB(nb);
    for (int b = 0; b < nb; ++b) {
        const pc_params *p = &S.prm[b];
        hK[b] = pgd_consts(cp[b], p);
        if (I.mt) pgd_thresholds(hK[b], thr->c, p);
        PgdBlk &k = hB[b];
        memset(&k, 0, sizeof(k));
        k.b1p = p->beta1;
        k.b2p = p->beta2;
        k.ibc1 = df_split(1.0 / (1.0 - p->beta1));
        k.ibc2 = df_split(1.0 / (1.0 - p->beta2));
        k.patience = p->stall_patience;
        I.max_checks = std::max<int64_t>(I.max_checks, (p->replay_iters >= 0 ? p->replay_iters : p->t_max) + 1);
    }
    I.CB.alloc(nb, s);
    I.blk.alloc(nb, s);
    I.gs.alloc(1, s);
    {
        const size_t bytes = nb * (sizeof(PgdConsts) + sizeof(PgdBlk)) + sizeof(PgdGlobal);
        uint8_t *h = (uint8_t *)host_scratch(hs, bytes);
        memcpy(h, hK.data(), nb * sizeof(PgdConsts));
        memcpy(h + nb * sizeof(PgdConsts), hB.data(), nb * sizeof(PgdBlk));
        memset(h + nb * (sizeof(PgdConsts) + sizeof(PgdBlk)), 0, sizeof(PgdGlobal));
        PC_CUDA(cudaMemcpyAsync(I.CB.p, h, nb * sizeof(PgdConsts), cudaMemcpyHostToDevice, s));
        PC_CUDA(cudaMemcpyAsync(I.blk.p, h + nb * sizeof(PgdConsts), nb * sizeof(PgdBlk), cudaMemcpyHostToDevice, s));
        PC_CUDA(cudaMemcpyAsync(I.gs.p, h + nb * (sizeof(PgdConsts) + sizeof(PgdBlk)), sizeof(PgdGlobal),
                                cudaMemcpyHostToDevice, s));
        PC_CUDA(cudaStreamSynchronize(s));   // the staging area is reused below
    }
    I.row_off.assign(nb + 1, 0);
    if (nA == 0) return;

    // ---- E and CSR
    const int nbits = std::max(1, ceil_log2((uint64_t)n));
    DBuf<uint32_t> mark(n, s), dense(n, s), tot(1, s);
    PC_CUDA(cudaMemsetAsync(mark.p, 0, n * sizeof(uint32_t), s));
    k_mark<<<grid_for(nA), 256, 0, s>>>(A, nA, mark.p);
    PC_CHECK_LAUNCH();
    scan_exclusive_u32(mark.p, dense.p, n, tot.p, s);
    const int64_t ne = *(uint32_t *)read_back(hs, tot.p, sizeof(uint32_t), s);
    I.ne = ne;
    if (I.mt && ne >= ((int64_t)1 << 29)) fail(PC_EINVAL, "several linking lengths: at most 2^29 editable particles");
    const int tb = I.mt ? 2 : 0;   // threshold-index bits of the directed keys
    ThrB2 tb2;
    for (int k = 0; k < MAX_THR; ++k) tb2.b2[k] = I.mt && k < (int)thr->c.size() ? thr->c[k].b2 : 0.f;
    DBuf<uint32_t> epos(ne, s);
    k_epos<<<grid_for(n), 256, 0, s>>>(mark.p, dense.p, n, epos.p);
    PC_CHECK_LAUNCH();
    mark.release();
    // directed edges sorted by (row, partner position, threshold index); 64-bit offsets
    const int64_t m = 2 * nA;
    DBuf<unsigned long long> keys(m, s);
    k_dir_keys<<<grid_for(nA), 256, 0, s>>>(A, I.mt ? thr->Athr : nullptr, nA, dense.p, nbits, tb, keys.p);
    PC_CHECK_LAUNCH();
    radix_sort_u64((uint64_t *)keys.p, nullptr, m, nbits + tb + std::max(1, ceil_log2((uint64_t)ne)), s);
    DBuf<unsigned long long> row_ptr(ne + 1, s);
    k_row_bounds<<<grid_for(m + 1), 256, 0, s>>>(keys.p, m, nbits + tb, ne, row_ptr.p);
    PC_CHECK_LAUNCH();

    // ---- iteration state
    for (DBuf<float4> *d : {&I.PE, &I.Dh0, &I.Dl0, &I.Dh1, &I.Dl1, &I.Mh, &I.Ml, &I.Vh, &I.Vl, &I.Q0, &I.Q1})
        d->alloc(ne, s);
    I.act.alloc(ne, s);
    I.rb.alloc(ne, s);
    DBuf<unsigned long long> rows_pb(nb, s);
    PC_CUDA(cudaMemsetAsync(rows_pb.p, 0, nb * sizeof(unsigned long long), s));
    k_state_init<<<grid_for(ne), 256, 0, s>>>(epos.p, ne, B.P4.p, orig, recon, S.doff.p, nb, I.CB.p, I.PE.p, I.rb.p,
                                              I.Dh0.p, I.Dl0.p, I.Dh1.p, I.Dl1.p, I.Q0.p, I.Q1.p, I.Mh.p, I.Ml.p,
                                              I.Vh.p, I.Vl.p, I.act.p, rows_pb.p);
    PC_CHECK_LAUNCH();
    // rows per block -> row offsets (rows are in sorted-position order, blocks own contiguous ranges)
    const unsigned long long *rows =
        (const unsigned long long *)read_back(hs, rows_pb.p, nb * sizeof(unsigned long long), s);
    for (int b = 0; b < nb; ++b) I.row_off[b + 1] = I.row_off[b] + (int64_t)rows[b];
    PgdBufs &Bf = I.Bf;
    Bf.Dh[0] = I.Dh0.p;
    Bf.Dh[1] = I.Dh1.p;
    Bf.Dl[0] = I.Dl0.p;
    Bf.Dl[1] = I.Dl1.p;
    Bf.Q[0] = I.Q0.p;
    Bf.Q[1] = I.Q1.p;
    Bf.Mh = I.Mh.p;
    Bf.Ml = I.Ml.p;
    Bf.Vh = I.Vh.p;
    Bf.Vl = I.Vl.p;
    Bf.act = I.act.p;
    DBuf<int64_t> roff;
    if (nb > 1) {
        roff.alloc(nb + 1, s);
        PC_CUDA(cudaMemcpyAsync(roff.p, I.row_off.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }

    // ---- edge plan: light rows' edges in row order, then heavy rows' (chunks of HEAVY)
    DBuf<unsigned long long> ldeg(ne, s), hdeg(ne, s), hptr(ne + 1, s), tot64(2, s);
    DBuf<uint32_t> nchunk(ne, s), isheavy(ne, s), c0(ne, s), hpos(ne, s), tot2(2, s);
    k_degrees<<<grid_for(ne), 256, 0, s>>>(row_ptr.p, ne, ldeg.p, hdeg.p, nchunk.p, isheavy.p, I.act.p);
    PC_CHECK_LAUNCH();
    I.lptr.alloc(ne + 1, s);
    scan_exclusive_u64((const uint64_t *)ldeg.p, (uint64_t *)I.lptr.p, ne, (uint64_t *)(I.lptr.p + ne), s);
    scan_exclusive_u64((const uint64_t *)hdeg.p, (uint64_t *)hptr.p, ne, (uint64_t *)tot64.p, s);
    scan_exclusive_u32(nchunk.p, c0.p, ne, tot2.p, s);
    scan_exclusive_u32(isheavy.p, hpos.p, ne, tot2.p + 1, s);
    ldeg.release();
    uint32_t tots[2];
    memcpy(tots, read_back(hs, tot2.p, 2 * sizeof(uint32_t), s), sizeof(tots));
    const unsigned long long n_light = *(const unsigned long long *)read_back(hs, I.lptr.p + ne, 8, s);
    const int64_t n_chunks = tots[0];
    I.n_heavy = tots[1];
    I.ecol.alloc(std::max<int64_t>(1, m), s);
    I.eslot.alloc(std::max<unsigned long long>(1, n_light), s);
    k_cols<<<grid_for(m), 256, 0, s>>>(keys.p, m, nbits, tb, tb2, row_ptr.p, I.lptr.p, hptr.p, n_light, dense.p,
                                       epos.p, I.rb.p, roff.p, B.P4.p, S.dev.p, S.doff.p, nb, I.ecol.p, I.eslot.p);
    PC_CHECK_LAUNCH();
    keys.release();
    row_ptr.release();
    dense.release();
    epos.release();
    I.chunk_row.alloc(n_chunks, s);
    I.chunk_start.alloc(n_chunks, s);
    I.chunk_len.alloc(n_chunks, s);
    I.hrow.alloc(I.n_heavy, s);
    I.hc0.alloc(I.n_heavy + 1, s);
    I.chunk_g.alloc(2 * n_chunks, s);
    if (I.n_heavy > 0) {
        k_heavy_fill<<<grid_for(ne), 256, 0, s>>>(hdeg.p, hptr.p, n_light, ne, nchunk.p, c0.p, isheavy.p, hpos.p,
                                                  I.chunk_row.p, I.chunk_start.p, I.chunk_len.p, I.hrow.p, I.hc0.p);
        PC_CHECK_LAUNCH();
        PC_CUDA(cudaMemcpyAsync(I.hc0.p + I.n_heavy, tot2.p, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    I.kernels_per_iter = I.n_heavy > 0 ? 2 : 1;
    I.LP = LightPlan{I.lptr.p, I.ecol.p, I.eslot.p};
    if (nb > 1) {
        // work table of the blocks still iterating (all of them before the first launch)
        I.bw.alloc(nb, s);
        I.act_blk.alloc(nb, s);
        I.act_pref.alloc(nb + 1, s);
        k_blk_work<<<grid_for(nb), 256, 0, s>>>(roff.p, c0.p, ne, n_chunks, nb, I.bw.p);
        PC_CHECK_LAUNCH();
        I.wt = WorkTab{I.bw.p, I.act_blk.p, I.act_pref.p};
        k_worktab_init<<<1, 32, 0, s>>>(nb, I.blk.p, I.wt, I.gs.p);
        PC_CHECK_LAUNCH();
    }
    PC_CUDA(cudaStreamSynchronize(s));   // roff and the plan temporaries are released on return
    I.HP.n_chunks = n_chunks;
    I.HP.chunk_row = I.chunk_row.p;
    I.HP.chunk_start = I.chunk_start.p;
    I.HP.chunk_len = I.chunk_len.p;
    I.HP.chunk_g = I.chunk_g.p;
    const int64_t n_items = cdiv(ne, 32) + nb + n_chunks;
    I.nblk = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n_items, WARPS), (int64_t)num_sms() * PGD_BLOCKS_PER_SM));
}

PgdSolver::~PgdSolver() { delete im; }

bool PgdSolver::empty() const { return im->ne == 0; }
int64_t PgdSolver::max_launches() const { return im->max_checks + 1; }
int64_t PgdSolver::rows() const { return im->ne; }

void PgdSolver::capture(int k) {
    Impl &I = *im;
    if (I.ne == 0 || k < 1) return;
    if (I.exec) {
        cudaGraphExecDestroy(I.exec);
        I.exec = nullptr;
    }
    if (I.graph) {
        cudaGraphDestroy(I.graph);
        I.graph = nullptr;
    }
    // capture on a private stream (the legacy default stream cannot be captured); nothing
    // runs during capture, and the graph is replayed on the solver's stream
    cudaStream_t cs = nullptr;
    PC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const cudaStream_t run_s = I.s;
    I.s = cs;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        try {
            for (int j = 0; j < k; ++j) I.launch_iter();
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            I.s = run_s;
            cudaStreamDestroy(cs);
            throw;
        }
        e = cudaStreamEndCapture(cs, &I.graph);
    }
    I.s = run_s;
    cudaStreamDestroy(cs);
    PC_CUDA(e);
    PC_CUDA(cudaGraphInstantiate(&I.exec, I.graph, 0));
    add_launches(-(int64_t)k * I.kernels_per_iter);   // captured, not run
    I.graph_k = k;
}

int64_t PgdSolver::launch(int k) {
    Impl &I = *im;
    if (I.ne == 0) return 0;
    int64_t done = 0;
    if (I.exec) {
        for (; done + I.graph_k <= k || done == 0; done += I.graph_k) {
            PC_CUDA(cudaGraphLaunch(I.exec, I.s));
            add_launches((int64_t)I.graph_k * I.kernels_per_iter);
        }
    } else {
        for (; done < k; ++done) I.launch_iter();
    }
    launches += done;
    return done;
}

void PgdSolver::post_status() {
    Impl &I = *im;
    PC_CUDA(cudaMemcpyAsync(I.pin, I.blk.p, I.nb * sizeof(PgdBlk), cudaMemcpyDeviceToHost, I.s));
    PC_CUDA(cudaMemcpyAsync(I.pin + I.nb * sizeof(PgdBlk), I.gs.p, sizeof(PgdGlobal), cudaMemcpyDeviceToHost, I.s));
    PC_CUDA(cudaEventRecord(I.ev, I.s));
    I.posted = true;
}

bool PgdSolver::status_ready() const {
    if (!im->posted) return false;
    const cudaError_t e = cudaEventQuery(im->ev);
    if (e == cudaErrorNotReady) return false;
    PC_CUDA(e);
    return true;
}

void PgdSolver::wait_status() const {
    if (!im->posted) return;
    PC_CUDA(cudaEventSynchronize(im->ev));
}

bool PgdSolver::all_stopped() const {
    if (im->ne == 0) return true;
    return ((const PgdGlobal *)(im->pin + im->nb * sizeof(PgdBlk)))->all_stop != 0;
}

bool PgdSolver::block_stopped(int b) const {
    if (im->ne == 0) return true;
    return ((const PgdBlk *)im->pin)[b].stop != 0;
}

int64_t PgdSolver::active_rows() const {
    if (im->ne == 0) return 0;
    const PgdBlk *hb = (const PgdBlk *)im->pin;
    int64_t r = 0;
    for (int b = 0; b < im->nb; ++b)
        if (!hb[b].stop) r += im->row_off[b + 1] - im->row_off[b];
    return r;
}

void PgdSolver::output(float *corrected, int b) {
    Impl &I = *im;
    if (I.ne == 0) return;
    const int64_t e0 = b < 0 ? 0 : I.row_off[b], e1 = b < 0 ? I.ne : I.row_off[b + 1];
    if (e1 <= e0) return;
    k_output<<<grid_for(e1 - e0), 256, 0, I.s>>>(I.PE.p, I.rb.p, e0, e1 - e0, I.Bf, I.blk.p, corrected);
    PC_CHECK_LAUNCH();
}

void PgdSolver::delta_out(double *d) {
    Impl &I = *im;
    if (I.ne == 0) return;
    k_delta_out<<<grid_for(I.ne), 256, 0, I.s>>>(I.PE.p, I.rb.p, I.ne, I.Bf, I.blk.p, d);
    PC_CHECK_LAUNCH();
}

void PgdSolver::results(std::vector<PgdResult> &out) {
    Impl &I = *im;
    out.assign(I.nb, PgdResult());
    if (I.ne == 0) {
        for (auto &r : out) {
            r.converged = true;
            r.loss_evals = 1;
        }
        return;
    }
    post_status();
    wait_status();
    const PgdBlk *hb = (const PgdBlk *)I.pin;
    for (int b = 0; b < I.nb; ++b) {
        PgdResult &r = out[b];
        r.iters = hb[b].t;
        r.loss_evals = hb[b].t + 1;
        r.viol0 = (int64_t)hb[b].viol0;
        r.viol_final = (int64_t)hb[b].viol;
        r.loss0 = hb[b].loss0;
        r.loss_final = hb[b].loss;
        r.converged = hb[b].converged != 0;
        r.n_editable = I.row_off[b + 1] - I.row_off[b];
        r.resets = hb[b].resets;
        r.row_updates = (int64_t)hb[b].n_upd;
        r.pair_evals = (int64_t)hb[b].n_eval;
    }
}

void PgdSolver::block_result(int b, PgdResult &r) const {
    const Impl &I = *im;
    r = PgdResult();
    if (I.ne == 0) {
        r.converged = true;
        r.loss_evals = 1;
        return;
    }
    const PgdBlk &B = ((const PgdBlk *)I.pin)[b];
    r.iters = B.t;
    r.loss_evals = B.t + 1;
    r.viol0 = (int64_t)B.viol0;
    r.viol_final = (int64_t)B.viol;
    r.loss0 = B.loss0;
    r.loss_final = B.loss;
    r.converged = B.converged != 0;
    r.n_editable = I.row_off[b + 1] - I.row_off[b];
    r.resets = B.resets;
    r.row_updates = (int64_t)B.n_upd;
    r.pair_evals = (int64_t)B.n_eval;
}

PgdRun run_pgd(const Binned &B, const BlockSet &S, const std::vector<Consts> &cp, const float *orig,
               const float *recon, const unsigned long long *A, int64_t nA, float *corrected, cudaStream_t s,
               HostScratch &hs, double *delta_out, double *hist_loss, unsigned long long *hist_viol, int graph_k,
               const ThrSet *thr) {
    PgdRun run;
    const int64_t n = B.n;
    cudaEvent_t ev[4];
    for (auto &e : ev) PC_CUDA(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int k = 0; k < 4; ++k) cudaEventDestroy(e[k]);
        }
    } guard{ev};
    PC_CUDA(cudaEventRecord(ev[0], s));
    k_copy_recon<<<grid_for(3 * n), 256, 0, s>>>(recon, corrected, 3 * n);
    PC_CHECK_LAUNCH();
    if (delta_out) PC_CUDA(cudaMemsetAsync(delta_out, 0, 3 * n * sizeof(double), s));
    PgdSolver sol(B, S, cp, orig, recon, A, nA, s, hs, hist_loss, hist_viol, thr);
    PC_CUDA(cudaEventRecord(ev[1], s));
    if (sol.empty()) {
        // nothing to enforce anywhere: reconstructions stand, zero iterations
        if (hist_loss) PC_CUDA(cudaMemsetAsync(hist_loss, 0, sizeof(double), s));
        if (hist_viol) PC_CUDA(cudaMemsetAsync(hist_viol, 0, sizeof(unsigned long long), s));
    } else {
        if (graph_k > 0) sol.capture(graph_k);
        // iterations: launch in growing chunks, poll the device stop flags between chunks
        const int64_t max_launch = sol.max_launches();
        int64_t launched = 0;
        int chunk = graph_k > 0 ? graph_k : 4;
        for (;;) {
            launched += sol.launch(chunk);
            sol.post_status();
            sol.wait_status();
            if (sol.all_stopped()) break;
            if (launched >= max_launch) {
                set_error("PGD loop did not reach its stop decision");
                throw Fail{PC_ETIMEOUT};
            }
            // the next poll comes after at most 32 launches: launches past every block's stop
            // return at once, so a bounded overshoot costs little
            chunk = std::min(chunk * 2, 32);
        }
    }
    PC_CUDA(cudaEventRecord(ev[2], s));
    sol.output(corrected);
    if (delta_out) sol.delta_out(delta_out);
    PC_CUDA(cudaEventRecord(ev[3], s));
    sol.results(run.blocks);
    float ms[3] = {0, 0, 0};
    cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
    cudaEventElapsedTime(&ms[1], ev[1], ev[3]);
    cudaEventElapsedTime(&ms[2], ev[1], ev[2]);
    run.ms_csr = ms[0];
    run.ms = ms[1];
    run.ms_iter = ms[2];
    run.launches = sol.launches;
    return run;
}

}  // namespace pc
