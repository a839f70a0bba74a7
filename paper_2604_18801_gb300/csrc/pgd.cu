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
// One iteration = one launch of k_pgd_iter.  Warps take work items (a heavy
// row -- more than HEAVY partners -- or a group of 32 light rows) from a
// counter, heavy rows first and longest first.  A float32 screen on Q
// certifies most pairs as satisfied; the others are evaluated in
// double-float, 32 at a time, and each row's gradient is a fixed-order sum
// (its violated pairs in edge order), so no float atomics are used and the
// offsets are deterministic.  The loss (each pair counted once, in the row of
// its smaller dense index) is accumulated in fixed point and the violations
// are counted; the last block takes the stop decision of Algorithm 1.  The
// Adam step of the same launch is written to the other buffers, so when the
// check says "stop" the current buffer is the answer and nothing has to be
// undone.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <type_traits>

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
constexpr int PGD_BLOCKS_PER_SM = 3;   // resident CTAs of the persistent iteration grid

// Linking lengths of one problem: one, or up to MAX_THR enforced together (the union of
// their active pairs, Sec. 1 and Sec. 5); a CSR entry then carries its pair's index.
constexpr int MAX_THR = 4;

// act[e]: bit 0 = the row has had a gradient (or needs its first projection), bit 1 = the
// row is heavy (more than HEAVY partners: it is a work item of its own).
constexpr uint8_t ACT_ON = 1, ACT_HEAVY = 2;
constexpr uint32_t HEAVY = 256;
// A light work item is ITEM_GROUPS consecutive groups of 32 rows (of one block): its
// stream ranges and row positions load together, so their latency is paid once.
constexpr int ITEM_GROUPS = 4;
constexpr int ITEM_ROWS = 32 * ITEM_GROUPS;

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

// Work items are claimed from NQ counters, each owning a contiguous slice of the item
// space and each on a line of its own, so that claims do not queue on one address.
constexpr int NQ = 16;
struct alignas(128) QCounter {
    unsigned long long v;
    unsigned long long pad[15];
};

struct PgdGlobal {
    uint32_t ticket;
    int32_t all_stop;
    int32_t active;                 // blocks still iterating after the last launch
    int32_t pad;
    unsigned long long n_items;     // work items of the blocks still iterating (problem sets)
    unsigned long long work3;       // next claim of heavy rows of the update
    QCounter q1[NQ];                // the screen's items
    QCounter q2[NQ];                // the update's light items
};

// The next item of [0, n) for a warp (called by one lane): a warp starts on slice
// `slice` (its global warp index mod NQ) and moves on to the next slice when its own is
// used up; n when every slice is used up.
__device__ __forceinline__ int64_t claim_item(QCounter *q, int64_t n, int &slice, int &tried) {
    const int64_t R = (n + NQ - 1) / NQ;
    while (tried < NQ) {
        const int64_t lo = (int64_t)slice * R, hi = min(n, lo + R);
        if (lo < hi) {
            const unsigned long long v = atomicAdd(&q[slice].v, 1ull);
            if ((int64_t)v < hi - lo) return lo + (int64_t)v;
        }
        slice = slice + 1 == NQ ? 0 : slice + 1;
        ++tried;
    }
    return n;
}

// Work of one block of a problem set: its heavy rows, items [h0, h0 + nh) of the heavy
// list (longest first), then ceil(nrows / 32) light items over its rows [row0, row0 +
// nrows) (groups of 32 rows that never straddle two blocks; the heavy rows among them
// have no light edges).
struct BlkWork {
    uint32_t row0, nrows, h0, nh;
    uint32_t g0;   // the light group index of the block's first 32 rows
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
            it = (unsigned long long)((w.nrows + (uint32_t)ITEM_ROWS - 1u) / (uint32_t)ITEM_ROWS) + w.nh;
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

// Per-block row ranges and heavy-item ranges (rows are in sorted-position order, so every
// block owns a contiguous range of rows; heavy items are sorted by block first).
__global__ void k_blk_work(const int64_t *__restrict__ row_off, const uint32_t *__restrict__ h_off,
                           const uint32_t *__restrict__ gbase, int nb, BlkWork *__restrict__ bw) {
    GRID_STRIDE(b, nb) {
        const int64_t r0 = row_off[b], r1 = row_off[b + 1];
        bw[b] = BlkWork{(uint32_t)r0, (uint32_t)(r1 - r0), h_off[b], h_off[b + 1] - h_off[b], gbase[b]};
    }
}

// ------------------------------------------------------------------ CSR build
// The editable particles are numbered in an order that depends on the data alone, not on
// the tuned cell grid of the pair search: by block, then by the Morton code of the
// original position on a fixed lattice of 2^14 cells per axis over the block's box, ties
// by particle id.  Each row lists its partners in that order.  Summation orders, and so
// the results' bits, do not depend on the tuning knobs; neighbours stay close in memory.
struct MortonBox {
    double lo[3], scale[3];   // lattice cell of coordinate x: floor((x - lo) * scale), clamped
};

// Spreads the low 21 bits of x to every third bit.
__device__ __forceinline__ unsigned long long spread3(unsigned long long x) {
    x &= 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

constexpr int MORTON_BITS = 14;   // per axis

__global__ void k_mark_ids(const unsigned long long *__restrict__ A, int64_t m, const uint32_t *__restrict__ order,
                           uint32_t *__restrict__ mark) {
    GRID_STRIDE(r, m) {
        const unsigned long long pk = A[r];
        mark[order[pk >> 32]] = 1u;
        mark[order[pk & 0xffffffffull]] = 1u;
    }
}

// Key (block << 42 | Morton code) of every editable particle, in id order.
__global__ void k_edit_keys(const uint32_t *__restrict__ mark, const uint32_t *__restrict__ rank, int64_t n,
                            const float *__restrict__ orig, const int64_t *__restrict__ off, int nblk,
                            const MortonBox *__restrict__ mb, unsigned long long *__restrict__ key,
                            uint32_t *__restrict__ eid) {
    GRID_STRIDE(i, n) {
        if (!mark[i]) continue;
        const uint32_t r = rank[i];
        const int b = find_block(off, nblk, i);
        const MortonBox &M = mb[b];
        unsigned long long code = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double q = floor(((double)orig[3 * i + a] - M.lo[a]) * M.scale[a]);
            q = fmin(fmax(q, 0.0), (double)((1 << MORTON_BITS) - 1));
            code |= spread3((unsigned long long)q) << a;
        }
        key[r] = ((unsigned long long)b << (3 * MORTON_BITS)) | code;
        eid[r] = (uint32_t)i;
    }
}

// Row e of the numbering: its sorted position (epos) and the position -> row map.
__global__ void k_edit_maps(const uint32_t *__restrict__ eid, int64_t ne, const uint32_t *__restrict__ inv,
                            uint32_t *__restrict__ epos, uint32_t *__restrict__ dense) {
    GRID_STRIDE(e, ne) {
        const uint32_t pos = inv[eid[e]];
        epos[e] = pos;
        dense[pos] = (uint32_t)e;
    }
}

// Directed keys (row << nbe | partner row) << tb | threshold index (tb = 0: one linking
// length; tb = 2: Athr gives each pair's index).
__global__ void k_dir_keys(const unsigned long long *__restrict__ A, const uint8_t *__restrict__ Athr, int64_t m,
                           const uint32_t *__restrict__ dense, int nbe, int tb, unsigned long long *__restrict__ keys) {
    GRID_STRIDE(r, m) {
        const unsigned long long pk = A[r];
        const unsigned long long di = dense[pk >> 32], dj = dense[pk & 0xffffffffull];
        const unsigned long long t = tb ? (unsigned long long)Athr[r] : 0ull;
        keys[2 * r] = (((di << nbe) | dj) << tb) | t;
        keys[2 * r + 1] = (((dj << nbe) | di) << tb) | t;
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
        gs->work3 = 0;
        gs->ticket = 0;
    }
    if (lane < NQ) {
        gs->q1[lane].v = 0;
        gs->q2[lane].v = 0;
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
// A heavy row: its edges (one contiguous range of the edge array) and its row.
struct HeavyItem {
    unsigned long long start;
    uint32_t row, len;
    uint32_t ulo;   // rank of the first partner after the row (the screen walks [ulo, len))
    uint32_t pad;
};

struct HeavyPlan {
    int64_t n_heavy;                 // heavy rows (one work item each)
    const HeavyItem *item;           // by block, then longest first
};

// One edge array holds the light rows' edges, in row order, then the heavy rows' edges
// (each heavy row one contiguous range of that second part).  A group of 32 light rows owns the contiguous
// range [ptr[r0], ptr[r0 + 32]) (heavy rows own no light edge), and each light edge
// carries the slot of its row within the group, so a warp maps an edge to its row with
// one byte load.  Offsets are 64-bit: a problem may have more than 2^32 directed edges.
struct LightPlan {
    const unsigned long long *ptr;   // per row: first light edge (ne + 1 entries)
    const uint32_t *col;             // partner | link << 31 (| threshold index << 29 with several)
    // The screen's stream: each pair once, from the row that comes first.  Group g (32
    // light rows) owns [gup[g], gup[g + 1]): its rows' edges to later partners, sorted by
    // partner so that neighbouring lanes gather the same or nearby partners; the groups of
    // a work item are consecutive, so an item's stream is one range.  An entry is the CSR
    // entry (x) and the edge's place relative to the item's first light edge << 7 | the row
    // within the item (y), loaded together.
    const unsigned long long *gup;
    const uint2 *sst;
    // per edge to a later partner (by position in the edge array): the position of the
    // reverse edge in the partner's row
    const unsigned long long *erev;
    // A single problem's screen takes its light items in chunks of at most screen_chunk
    // stream entries (n_chunks of them, items in order; an item with no entries has none),
    // so that items in dense regions, whose streams are many times a warp's mean share,
    // do not leave a tail of one long walk.  Problem sets take whole items (chunk null).
    const struct ScreenChunk *chunk;
    int64_t n_chunks;
};

// One chunk of a light item's screen stream: entries [eb, eb + len) of the item `item`
// (rows [ITEM_ROWS * item, ...)); the entries keep their places relative to the item.
constexpr uint32_t SCREEN_CHUNK = 1024;   // default chunk length (pc_params.screen_chunk = 0)
struct ScreenChunk {
    unsigned long long eb;
    uint32_t len, item;
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

// ------------------------------------------------------------------ one iteration: two kernels
// Per iteration, k_pgd_screen walks every active pair with a float32 screen and lists the
// candidate rows of the update: every row that has an uncertain pair (one the screen
// could not certify as satisfied) or takes an Adam step (it has had a gradient, or needs
// its first projection).  k_pgd_update then evaluates, for each candidate row with an
// uncertain pair, that row's pairs in double-float (re-screening its edges, in edge
// order), sums its gradient in edge order, and applies Adam to every candidate row; the
// last block of the update takes the stop decisions of Algorithm 1.  The screen needs no
// double-float state, so it runs at high occupancy, and the update works on a compact list
// with every lane busy.

// Candidate entry: row | CAND_UNC when the row has an uncertain pair | CAND_HG when it is
// a heavy row whose gradient a warp has already summed (kept in the heavy-gradient table).
constexpr uint32_t CAND_UNC = 0x80000000u, CAND_HG = 0x40000000u;
constexpr int SCREEN_BLOCKS_PER_SM = 6;        // a single problem
constexpr int SCREEN_BLOCKS_PER_SM_MULTI = 4;  // a problem set (its item map needs more registers)
constexpr int KERNELS_PER_ITER = 2;   // screen, update
constexpr int QCAP = 128;   // uncertain pairs waiting for evaluation (a ring per warp; < 32 + 2 x 32)
constexpr int EPL = 2;      // edges per lane per trip of the screen's walk

// Edge range of one row: light rows own [ptr[e], ptr[e + 1]) of the light part, heavy rows
// the range of their heavy item.
__device__ __forceinline__ void row_edges(const LightPlan &LP, const HeavyPlan &H, const uint32_t *__restrict__ hmap,
                                          uint32_t e, bool heavy, unsigned long long &start, uint32_t &len) {
    if (heavy) {
        const HeavyItem hv = H.item[hmap[e]];
        start = hv.start;
        len = hv.len;
    } else {
        start = LP.ptr[e];
        len = (uint32_t)(LP.ptr[e + 1] - start);
    }
}

// float32 screen of one pair: true when it may be violated (the double-float evaluation
// decides).  qr: the row's rounded position; qk: the partner's; cv: the CSR entry.  PP:
// minimum image; with one linking length the thresholds come in registers (sl_link,
// sl_non), with several (MT) from the table by the entry's index.
template <bool MT, bool PP>
__device__ __forceinline__ bool screen_pair(const float4 qr, const float4 qk, uint32_t cv, const float L0,
                                            const float L1, const float L2, float sl_link, float sl_non,
                                            const PgdConsts &C) {
    const float d2 = cdist2(cdiff(qr.x, qk.x, PP, L0), cdiff(qr.y, qk.y, PP, L1), cdiff(qr.z, qk.z, PP, L2));
    if (MT) {
        const int ti = (int)((cv >> 29) & 3u);
        return (cv >> 31) ? !(d2 < C.screen_link[ti]) : !(d2 > C.screen_non[ti]);
    }
    return (cv >> 31) ? !(d2 < sl_link) : !(d2 > sl_non);
}

// Whether a warp whose rows are at rounded positions q (one per lane that holds a row)
// may skip the minimum image: every row lies in the periodic box's interior, where no
// active pair wraps (so the screen's d2 is the same bit for bit).
__device__ __forceinline__ bool interior(const PgdConsts &C, const float4 q) {
    return q.x >= C.ilo[0] && q.x <= C.ihi[0] && q.y >= C.ilo[1] && q.y <= C.ihi[1] && q.z >= C.ilo[2] && q.z <= C.ihi[2];
}
__device__ __forceinline__ bool needs_image(const PgdConsts &C, bool row_lane, const float4 q) {
    const bool in_ok = C.interior_ok != 0 && (!row_lane || interior(C, q));
    return C.periodic != 0 && !__all_sync(0xffffffffu, in_ok);
}

// Work item `item` of the screen's item space: a heavy row (H.item[hk]) or up to
// ITEM_GROUPS consecutive groups of 32 light rows (first group g, rows [r0, r0 + cnt)) of
// block b.  A problem set's items are those of its blocks still iterating (the work
// table), each block's heavy rows first; a single problem's items are every heavy row,
// then the light items.  Called by all lanes of a warp.
template <bool MULTI>
__device__ __forceinline__ void map_item(int64_t item, int64_t ne, const HeavyPlan &H, const WorkTab &wt, int nact,
                                         int &b, bool &heavy, int64_t &r0, int &cnt, int64_t &hk, int64_t &g) {
    const unsigned FULL = 0xffffffffu;
    b = 0;
    r0 = 0;
    cnt = 0;
    hk = 0;
    g = 0;
    if (MULTI) {
        int kk = 0;
        if ((threadIdx.x & 31) == 0) {   // active block of the item: largest k with act_pref[k] <= item
            int lo = 0, hi = nact - 1;
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
        heavy = j < (int64_t)bw.nh;
        if (!heavy) {
            const int64_t jl = j - (int64_t)bw.nh;
            r0 = (int64_t)bw.row0 + ITEM_ROWS * jl;
            cnt = (int)min((int64_t)ITEM_ROWS, (int64_t)bw.nrows - ITEM_ROWS * jl);
            g = (int64_t)bw.g0 + ITEM_GROUPS * jl;
        } else {
            hk = (int64_t)bw.h0 + j;
        }
    } else {
        heavy = item < H.n_heavy;
        if (!heavy) {
            const int64_t jl = item - H.n_heavy;
            g = ITEM_GROUPS * jl;
            r0 = ITEM_ROWS * jl;
            cnt = (int)min((int64_t)ITEM_ROWS, ne - r0);
        } else {
            hk = item;
        }
    }
}

// The screen.  Work items are heavy rows (more than HEAVY partners; longest first, so the
// longest walks start early) and light items of ITEM_ROWS consecutive rows (for a single
// problem, chunks of at most screen_chunk pairs of them), handed out from counters (the
// next item is claimed one item ahead).  Every pair is screened once, from the row that
// comes first: a warp walks its item's stream of edges to later partners 32 * EPL at a
// time (EPL per lane, strided by 32 so that loads stay coalesced; the next trip's entries
// load while this trip's partner positions are gathered).  The walk is bound by the
// latency of the partner gathers, so the kernel runs small trips at high occupancy
// (SCREEN_BLOCKS_PER_SM CTAs per SM) rather than long trips at low occupancy.  A pair the
// float32 screen cannot certify sets the bits of both its directed edges in the bit mask
// of the edge array and the flags of both rows; the update reads them.
template <bool MULTI, bool MT>
__global__ void __launch_bounds__(PGD_THREADS, MULTI ? SCREEN_BLOCKS_PER_SM_MULTI : SCREEN_BLOCKS_PER_SM) k_pgd_screen(
    int64_t ne, PgdBufs Bf, HeavyPlan H, LightPlan LP, const PgdConsts *__restrict__ CB,
    const PgdBlk *__restrict__ blk, PgdGlobal *gs, const WorkTab wt, uint32_t *__restrict__ ubits,
    uint8_t *__restrict__ uflag) {
    __shared__ int s_stop, s_t, s_nact;
    __shared__ unsigned long long s_items;
    __shared__ float4 sq[WARPS][ITEM_ROWS];   // the item's rows' rounded positions
    if (threadIdx.x == 0) {
        s_stop = gs->all_stop;
        s_nact = gs->active;
        s_items = gs->n_items;
        s_t = blk[0].t;
    }
    __syncthreads();
    if (s_stop) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr uint32_t PMASK = MT ? 0x1fffffffu : 0x7fffffffu;   // partner bits of a CSR entry
    const int64_t n_items = MULTI ? (int64_t)s_items : H.n_heavy + LP.n_chunks;
    int qslice = (int)((blockIdx.x * WARPS + w) % NQ), qtried = 0;
    long long nitm = 0;
    if (lane == 0) nitm = claim_item(gs->q1, n_items, qslice, qtried);
    for (;;) {
        const int64_t item = (int64_t)__shfl_sync(FULL, nitm, 0);
        if (item >= n_items) break;
        if (lane == 0) nitm = claim_item(gs->q1, n_items, qslice, qtried);
        int b, cnt;
        int64_t r0, hk, g;
        bool heavy_warp;
        ScreenChunk chk{0ull, 0u, 0u};   // a single problem's light chunk
        if (MULTI) {
            map_item<MULTI>(item, ne, H, wt, s_nact, b, heavy_warp, r0, cnt, hk, g);
        } else {
            b = 0;
            g = 0;
            heavy_warp = item < H.n_heavy;
            hk = item;
            r0 = 0;
            cnt = 0;
            if (!heavy_warp) {
                chk = LP.chunk[item - H.n_heavy];
                r0 = (int64_t)ITEM_ROWS * chk.item;
                cnt = (int)min((int64_t)ITEM_ROWS, ne - r0);
            }
        }
        const int tb = MULTI ? blk[b].t : s_t;
        const int pa = tb & 1;
        const PgdConsts &Cl = CB[b];
        const float L0 = Cl.L[0], L1 = Cl.L[1], L2 = Cl.L[2];
        const float4 *__restrict__ Qc = Bf.q(pa);
        const float slk = Cl.screen_link[0], sln_ = Cl.screen_non[0];
        // one stream [ebase, ebase + VT): a heavy row's edges to later partners (row rbase,
        // position at sqg[0]), or a light item's (rows rbase + (aux & 127), positions
        // sqg[aux & 127]); fbase + (aux >> 7) is a light edge's place in the edge array
        auto walk = [&](auto image, auto heavy, unsigned long long ebase, uint32_t VT, unsigned long long fbase,
                        int64_t rbase, const float4 *sqg) {
            constexpr bool PP = decltype(image)::value, HV = decltype(heavy)::value;
            const uint32_t *__restrict__ hcol = LP.col + ebase;   // heavy rows: the CSR entries
            const uint2 *__restrict__ lst = LP.sst + ebase;       // light items: entry and aux
            uint32_t cvn[EPL], axn[EPL];
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                const uint32_t v = 32u * j + lane;
                if (HV) {
                    cvn[j] = v < VT ? __ldcs(hcol + v) : 0u;
                    axn[j] = 0u;
                } else {
                    const uint2 x = v < VT ? __ldcs(lst + v) : make_uint2(0u, 0u);
                    cvn[j] = x.x;
                    axn[j] = x.y;
                }
            }
            for (uint32_t base = 0; base < VT; base += 32 * EPL) {
                uint32_t cv[EPL], ax[EPL];
                bool nd[EPL];
#pragma unroll
                for (int j = 0; j < EPL; ++j) {
                    nd[j] = base + 32u * j + lane < VT;
                    cv[j] = cvn[j];
                    ax[j] = axn[j];
                    const uint32_t v = base + 32u * (EPL + j) + lane;
                    if (HV) {
                        cvn[j] = v < VT ? __ldcs(hcol + v) : 0u;
                    } else {
                        const uint2 x = v < VT ? __ldcs(lst + v) : make_uint2(0u, 0u);
                        cvn[j] = x.x;
                        axn[j] = x.y;
                    }
                }
                unsigned um = 0u;
#pragma unroll
                for (int j = 0; j < EPL; ++j)
                    if (nd[j] && screen_pair<MT, PP>(sqg[ax[j] & 127u], Qc[cv[j] & PMASK], cv[j], L0, L1, L2, slk, sln_,
                                                     Cl))
                        um |= 1u << j;
                if (um) {
                    // the trip's uncertain pairs: every reverse-edge load first, then both
                    // directed edges' bits and both rows' flags
                    auto fwd = [&](int j) -> unsigned long long {
                        return HV ? ebase + base + 32u * j + lane : fbase + (ax[j] >> 7);
                    };
                    unsigned long long r[EPL];
#pragma unroll
                    for (int j = 0; j < EPL; ++j) r[j] = (um >> j) & 1u ? LP.erev[fwd(j)] : 0ull;
#pragma unroll
                    for (int j = 0; j < EPL; ++j)
                        if ((um >> j) & 1u) {
                            const unsigned long long f = fwd(j);
                            atomicOr(ubits + (f >> 5), 1u << (f & 31));
                            atomicOr(ubits + (r[j] >> 5), 1u << (r[j] & 31));
                            uflag[rbase + (ax[j] & 127u)] = 1;
                            uflag[cv[j] & PMASK] = 1;
                        }
                }
            }
        };
        if (heavy_warp) {
            const HeavyItem hv = H.item[hk];
            const float4 qe = Qc[hv.row];
            if (lane == 0) sq[w][0] = qe;
            __syncwarp();
            if (needs_image(Cl, true, qe))
                walk(std::true_type{}, std::true_type{}, hv.start + hv.ulo, hv.len - hv.ulo, 0ull, hv.row, sq[w]);
            else
                walk(std::false_type{}, std::true_type{}, hv.start + hv.ulo, hv.len - hv.ulo, 0ull, hv.row, sq[w]);
        } else {
            // the item's stream range (its groups' ranges are consecutive), first light edge
            // and row positions, loaded together; one walk over the whole range
            const int ngr = (cnt + 31) >> 5;
            unsigned long long eb = 0, ee = 0, fb = 0;
            if (lane == 0) {
                if (MULTI) {
                    eb = LP.gup[g];
                    ee = LP.gup[g + ngr];
                } else {
                    eb = chk.eb;
                    ee = chk.eb + chk.len;
                }
                fb = LP.ptr[r0];
            }
            eb = __shfl_sync(FULL, eb, 0);
            ee = __shfl_sync(FULL, ee, 0);
            fb = __shfl_sync(FULL, fb, 0);
            bool inner = true;   // every row of the item lies in the periodic box's interior
#pragma unroll
            for (int j = 0; j < ITEM_GROUPS; ++j)
                if (32 * j + lane < cnt) {
                    const float4 q = Qc[r0 + 32 * j + lane];
                    sq[w][32 * j + lane] = q;
                    inner = inner && interior(Cl, q);
                }
            __syncwarp();
            const bool pp = Cl.periodic != 0 && !__all_sync(FULL, Cl.interior_ok != 0 && inner);
            if (pp) walk(std::true_type{}, std::false_type{}, eb, (uint32_t)(ee - eb), fb, r0, sq[w]);
            else walk(std::false_type{}, std::false_type{}, eb, (uint32_t)(ee - eb), fb, r0, sq[w]);
        }
        __syncwarp();
    }
}

struct WarpTab {
    float4 st[7][32];                // the rows' Adam state (offset hi, lo, position, m hi, lo, v hi, lo)
    uint32_t qk[QCAP];               // queued pairs: partner
    uint8_t qs[QCAP];                // queued pairs: row slot | threshold index << 5 | link << 7
    uint32_t erow[32];               // the chunk's rows by slot
    int eb[32], epa[32];             // ... their blocks and buffer parities
    unsigned own[32];                // per row slot: this batch's violated entries of that row
    float gt[6][32];                 // this batch's gradient terms (x hi, x lo, y hi, ...) by entry
    uint32_t cb[64];                 // candidate rows waiting for a chunk (row | CAND_UNC), a ring
    unsigned pm[2][ITEM_GROUPS];     // the current light item's groups: candidate and flag masks
};

// 16-byte asynchronous copies from global to shared memory (not cached in L1).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The update: warps take first the heavy rows with an uncertain pair, one each, then the
// other candidate rows 32 at a time (slot i = lane i).  A row's uncertain pairs are the set
// bits of its edge range in the screen's bit mask: a heavy row's warp reads its words 32
// at a time, and each lane of a chunk reads its own row's words, one pair per round.  The
// pairs enter the warp's ring, in edge order within each row, tagged with their row's
// slot, and are evaluated in double-float 32 at a time; their bits are cleared as read.
// Each light row's owner lane then adds its violated pairs one by one in edge order (the
// same order for any grouping of rows, so a row's gradient does not depend on its chunk,
// batch or block); a heavy row's warp adds each batch of its pairs by a fixed tree first.
// Then every candidate row that is due takes its Adam step, lanes in parallel.
template <bool MULTI, bool MT>
__global__ void __launch_bounds__(PGD_THREADS, PGD_BLOCKS_PER_SM) k_pgd_update(
    int64_t ne, const float4 *__restrict__ PE, PgdBufs Bf, HeavyPlan H, LightPlan LP,
    const uint32_t *__restrict__ hmap, float4 *__restrict__ HG, const uint32_t *__restrict__ rb,
    uint32_t *__restrict__ ubits,
    uint8_t *__restrict__ uflag, const PgdConsts *__restrict__ CB, int nb, PgdBlk *blk, PgdGlobal *gs,
    const WorkTab wt, double *__restrict__ hist_loss, unsigned long long *__restrict__ hist_viol) {
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
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    WarpTab &T = tab[w];
    constexpr uint32_t PMASK = MT ? 0x1fffffffu : 0x7fffffffu;
    unsigned long long lfx = 0;       // this lane's share of the tight loss, fixed point (single block)
    unsigned viol = 0, nupd = 0, nev = 0;
    // Work comes in two phases.  First the heavy rows, 32 per claim (one per lane, strided): a row
    // with an uncertain pair is taken by the warp (kind 1: the warp reads its pairs); a row
    // that only steps joins the warp's ring of candidates.  Then the light items (up to
    // ITEM_ROWS rows): each lane looks at its rows' flags and Adam state, all loaded
    // together, and the candidates join the ring one group of 32 rows at a time.  Whenever
    // the ring holds 32 (or nothing is left to claim), 32 of them are processed as a chunk
    // (kind 2: each lane one row).  The flags are cleared as read.
    const int64_t n_light_items = MULTI ? (int64_t)s_items : (ne + ITEM_ROWS - 1) / ITEM_ROWS;
    int qslice = (int)((blockIdx.x * WARPS + w) % NQ), qtried = 0;
    bool heavy_done = false, light_done = false;
    int nc = 0, ch = 0;          // candidates in the ring and its head (warp-uniform)
    unsigned hmask = 0u;         // lanes whose heavy row (hrow) has an uncertain pair, not yet taken
    uint32_t hrow = 0u;
    int lpend = 0, lnum = 0;     // groups of the current light item not yet in the ring: [lpend, lnum)
    int64_t lr0 = 0;             // first row of the current light item
    for (;;) {
        int kind = 0;   // 1: heavy row, 2: chunk, 0: nothing left
        bool have = false;
        uint32_t ce = 0u;
        for (;;) {
            if (nc >= 32 || (heavy_done && hmask == 0u && light_done && lpend >= lnum && nc > 0)) {
                const int take = min(nc, 32);
                have = lane < take;
                ce = have ? T.cb[(ch + lane) & 63] : 0u;
                __syncwarp();
                ch = (ch + take) & 63;
                nc -= take;
                kind = 2;
                break;
            }
            if (hmask) {
                const int j = __ffs(hmask) - 1;
                hmask &= hmask - 1u;
                const uint32_t r = __shfl_sync(FULL, hrow, j);
                have = lane == 0;
                ce = have ? (r | CAND_UNC) : 0u;
                kind = 1;
                break;
            }
            if (lpend < lnum) {   // the next group of the current light item joins the ring
                const unsigned cm = T.pm[0][lpend], fm = T.pm[1][lpend];
                if ((cm >> lane) & 1u)
                    T.cb[(ch + nc + __popc(cm & lt_mask)) & 63] =
                        (uint32_t)(lr0 + 32 * lpend + lane) | (((fm >> lane) & 1u) ? CAND_UNC : 0u);
                __syncwarp();
                nc += __popc(cm);
                ++lpend;
                continue;
            }
            if (heavy_done && light_done) break;
            unsigned long long k = 0;
            if (!heavy_done) {
                // claim c holds the heavy items c + j * stride (heavy rows are longest first,
                // so every claim gets a like share of long and short rows)
                const int64_t stride = (H.n_heavy + 31) / 32;
                if (lane == 0) k = atomicAdd(&gs->work3, 1ull);
                k = __shfl_sync(FULL, k, 0);
                if ((int64_t)k >= stride) {
                    heavy_done = true;
                    continue;
                }
                const int64_t hk = (int64_t)k + stride * lane;
                bool f = false, steps = false;
                hrow = 0u;
                if (hk < H.n_heavy) {
                    hrow = H.item[hk].row;
                    const int rbk = MULTI ? (int)rb[hrow] : 0;
                    if (!MULTI || blk[rbk].stop == 0) {
                        f = uflag[hrow] != 0;
                        if (f) uflag[hrow] = 0;
                        steps = (Bf.act[hrow] & ACT_ON) && !is_last(CB[rbk], MULTI ? blk[rbk].t : s_t);
                    }
                }
                hmask = __ballot_sync(FULL, f);
                const unsigned sm = __ballot_sync(FULL, !f && steps);
                if (!f && steps) T.cb[(ch + nc + __popc(sm & lt_mask)) & 63] = hrow;
                __syncwarp();
                nc += __popc(sm);
                continue;
            }
            if (lane == 0) k = (unsigned long long)claim_item(gs->q2, n_light_items, qslice, qtried);
            k = __shfl_sync(FULL, k, 0);
            if ((int64_t)k >= n_light_items) {
                light_done = true;
                continue;
            }
            int ib, icnt;
            int64_t ir0, ihk, ig;
            bool ih;
            if (MULTI) {
                map_item<true>((int64_t)k, ne, H, wt, s_nact, ib, ih, ir0, icnt, ihk, ig);
                if (ih) continue;   // heavy rows come in the first phase
            } else {
                ib = 0;
                ir0 = (int64_t)k * ITEM_ROWS;
                icnt = (int)min((int64_t)ITEM_ROWS, ne - ir0);
            }
            const int tlast = is_last(CB[ib], MULTI ? blk[ib].t : s_t);
            uint8_t av[ITEM_GROUPS], fl[ITEM_GROUPS];
#pragma unroll
            for (int j = 0; j < ITEM_GROUPS; ++j) {
                const int64_t r = ir0 + 32 * j + lane;
                const bool in = 32 * j + lane < icnt;
                av[j] = in ? Bf.act[r] : (uint8_t)ACT_HEAVY;
                fl[j] = in ? uflag[r] : (uint8_t)0;
            }
#pragma unroll
            for (int j = 0; j < ITEM_GROUPS; ++j) {
                const bool light = !(av[j] & ACT_HEAVY);
                const bool f = light && fl[j] != 0;
                if (f) uflag[ir0 + 32 * j + lane] = 0;
                const bool c = f || (light && (av[j] & ACT_ON) && !tlast);
                const unsigned cm = __ballot_sync(FULL, c), fm = __ballot_sync(FULL, f);
                if (lane == 0) {
                    T.pm[0][j] = cm;
                    T.pm[1][j] = fm;
                }
            }
            __syncwarp();
            lr0 = ir0;
            lpend = 0;
            lnum = (icnt + 31) >> 5;
        }
        if (kind == 0) break;
        const uint32_t e = ce & ~(CAND_UNC | CAND_HG);
        const bool unc = have && (ce & CAND_UNC);
        const bool hg = have && (ce & CAND_HG);
        const int b = MULTI ? (have ? (int)rb[e] : 0) : 0;
        const int tb = MULTI ? blk[b].t : s_t;
        const int pa = tb & 1;
        const PgdConsts &C = CB[b];
        df g[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};   // gradient of the lane's row
        bool rv = false;                   // the lane's row has a violated pair
        uint8_t av = 0;
        if (have) av = Bf.act[e];
        if (hg) {   // a heavy row's gradient, summed by the warp that read its pairs
            const uint32_t hk = hmap[e];
            const float4 gh = HG[2 * hk], gl = HG[2 * hk + 1];
            g[0] = df_make(gh.x, gl.x);
            g[1] = df_make(gh.y, gl.y);
            g[2] = df_make(gh.z, gl.z);
            rv = gh.w != 0.f;
        }
        // the rows' Adam state travels to shared memory while the uncertain pairs are evaluated;
        // a heavy row read by the whole warp (kind 1) takes its Adam step later, in a chunk
        const bool due = have && kind == 2 && !is_last(C, tb);
        const bool was = (av & ACT_ON) != 0;
        if (due && (was || unc || hg)) {
            cp_async16(&T.st[0][lane], Bf.dh(pa) + e);
            cp_async16(&T.st[1][lane], Bf.dl(pa) + e);
            cp_async16(&T.st[2][lane], PE + e);
            if (was) {
                cp_async16(&T.st[3][lane], Bf.Mh + e);
                cp_async16(&T.st[4][lane], Bf.Ml + e);
                cp_async16(&T.st[5][lane], Bf.Vh + e);
                cp_async16(&T.st[6][lane], Bf.Vl + e);
            }
        }
        cp_async_commit();
        T.erow[lane] = e;
        T.eb[lane] = b;
        T.epa[lane] = pa;
        __syncwarp();

        int qh = 0, qn = 0;
        // evaluates the first min(qn, 32) queued pairs; their rows' owners add the violated ones
        auto batch = [&]() {
            const int c = min(qn, 32);
            int sq = 32;
            df gt[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};
            bool hit = false;
            unsigned long long ll = 0;
            unsigned lv = 0;
            int bs = -1;
            if (lane < c) {
                const int pos = (qh + lane) & (QCAP - 1);
                const uint32_t k = T.qk[pos];
                const uint32_t qsv = T.qs[pos];
                sq = (int)(qsv & 0x1fu);
                const int ti = MT ? (int)((qsv >> 5) & 3u) : 0;
                const uint32_t er = T.erow[sq];
                bs = T.eb[sq];
                const int ps = T.epa[sq];
                const float4 *Dh = Bf.dh(ps), *Dl = Bf.dl(ps);
                double ltv = 0.0;
                bool counts = false;
                hit = eval_pair(PE[er], Dh[er], Dl[er], er, k, (qsv >> 7) != 0, ti, PE, Dh, Dl, CB[bs], gt, ltv,
                                counts);
                if (hit) {
                    ll = (unsigned long long)llrint(ltv);
                    lv = (k > er && counts) ? 1u : 0u;
                }
            }
            if (MULTI) {   // the pairs' loss belongs to their rows' blocks
                if (ll) atomicAdd(&blk[bs].lfx, ll);
                if (lv) atomicAdd(&blk[bs].vacc, (unsigned long long)lv);
                const unsigned same = __match_any_sync(FULL, bs);
                const unsigned ge = __reduce_add_sync(same, lane < c ? 1u : 0u);
                if (bs >= 0 && lane == __ffs(same) - 1 && ge) atomicAdd(&blk[bs].eacc, (unsigned long long)ge);
            } else {
                lfx += ll;
                viol += lv;
                nev += lane < c ? 1u : 0u;
            }
            const unsigned hm = __ballot_sync(FULL, hit);
            if (kind == 1) {
                // one heavy row (slot 0): the batch holds entries [32k, 32k + 32) of the row's
                // re-screened pairs, added by a fixed tree over those positions (zeros where
                // a pair is not violated), then into the row's sum; the shape depends on the
                // row's data alone, so the sum is the same in every run
                df t[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) t[a] = hit ? gt[a] : df_make(0.f, 0.f);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        t[a] = df_add(t[a], df_make(__shfl_down_sync(FULL, t[a].hi, off),
                                                    __shfl_down_sync(FULL, t[a].lo, off)));
                if (lane == 0 && hm) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) g[a] = df_add(g[a], t[a]);
                    rv = true;
                }
            } else {
                if (hit) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        T.gt[2 * a][lane] = gt[a].hi;
                        T.gt[2 * a + 1][lane] = gt[a].lo;
                    }
                }
                T.own[lane] = 0u;
                const unsigned same_s = __match_any_sync(FULL, sq);
                __syncwarp();
                if (hit) T.own[sq] = same_s & hm;   // the entries of one slot all write the same mask
                __syncwarp();
                for (unsigned mine = T.own[lane]; mine; mine &= mine - 1) {
                    const int i = __ffs(mine) - 1;
#pragma unroll
                    for (int a = 0; a < 3; ++a) g[a] = df_add(g[a], df_make(T.gt[2 * a][i], T.gt[2 * a + 1][i]));
                    rv = true;
                }
            }
            qh = (qh + c) & (QCAP - 1);
            qn -= c;
            __syncwarp();
        };

        // queue one entry per lane that has one (edge order within each row)
        auto push = [&](bool has, uint32_t cv, int slot) {
            const unsigned bal = __ballot_sync(FULL, has);
            if (has) {
                const int pos = (qh + qn + __popc(bal & lt_mask)) & (QCAP - 1);
                T.qk[pos] = cv & PMASK;
                T.qs[pos] = (uint8_t)(slot | (MT ? ((cv >> 29) & 3u) << 5 : 0u) | ((cv >> 31) ? 0x80 : 0));
            }
            qn += __popc(bal);
            __syncwarp();
            while (qn >= 32) batch();
        };
        // the bits of edge-array word wi that belong to the edge range [es, es + len), read
        // and cleared (whole words of one row with a plain store; a word shared with the
        // neighbouring rows' edges clears only this row's bits)
        auto take_word = [&](unsigned long long wi, unsigned long long es, unsigned long long ee) -> uint32_t {
            uint32_t m = 0xffffffffu;
            if (wi == (es >> 5)) m &= 0xffffffffu << (es & 31);
            if (wi == ((ee - 1) >> 5)) m &= 0xffffffffu >> (31 - ((ee - 1) & 31));
            const uint32_t v = ubits[wi] & m;
            if (v) {
                if (m == 0xffffffffu) ubits[wi] = 0u;
                else atomicAnd(ubits + wi, ~m);
            }
            return v;
        };
        if (kind == 1) {
            // a heavy row: the warp reads its words 32 at a time; the set bits of each word,
            // in order, are its uncertain pairs in edge order
            const uint32_t er = __shfl_sync(FULL, e, 0);
            unsigned long long es;
            uint32_t len;
            row_edges(LP, H, hmap, er, true, es, len);
            const unsigned long long ee = es + len, w0 = es >> 5, w1 = (ee - 1) >> 5;
            for (unsigned long long wb = w0; wb <= w1; wb += 32) {
                const unsigned long long wi = wb + lane;
                const uint32_t word = wi <= w1 ? take_word(wi, es, ee) : 0u;
                for (unsigned nz = __ballot_sync(FULL, word != 0u); nz; nz &= nz - 1) {
                    const int j = __ffs(nz) - 1;
                    const uint32_t bits = __shfl_sync(FULL, word, j);
                    const bool has = (bits >> lane) & 1u;
                    push(has, has ? LP.col[(wb + j) * 32 + lane] : 0u, 0);
                }
            }
        } else {
            // light rows with an uncertain pair: each lane reads its own row's words and
            // queues one pair per round
            unsigned long long wcur = 0, wend = 0, es = 0, ee = 0;
            uint32_t cur = 0;
            bool pend = false;
            if (unc) {
                es = LP.ptr[e];
                ee = LP.ptr[e + 1];
                pend = ee > es;   // a flagged row always has an edge
            }
            if (pend) {
                wcur = es >> 5;
                wend = (ee - 1) >> 5;
                cur = take_word(wcur, es, ee);
            }
            while (__any_sync(FULL, pend)) {
                bool has = false;
                uint32_t cv = 0u;
                if (pend) {
                    while (cur == 0u && wcur < wend) cur = take_word(++wcur, es, ee);
                    if (cur) {
                        const int bit = __ffs(cur) - 1;
                        cur &= cur - 1u;
                        cv = LP.col[wcur * 32 + bit];
                        has = true;
                    }
                    pend = cur != 0u || wcur < wend;
                }
                push(has, cv, lane);
            }
        }
        while (qn > 0) batch();
        if (kind == 1) {
            // the heavy row's gradient goes to the table; the row joins the ring for Adam
            if (lane == 0) {
                const uint32_t hk = hmap[e];
                HG[2 * hk] = make_float4(g[0].hi, g[1].hi, g[2].hi, rv ? 1.f : 0.f);
                HG[2 * hk + 1] = make_float4(g[0].lo, g[1].lo, g[2].lo, 0.f);
                T.cb[(ch + nc) & 63] = e | CAND_HG;
            }
            __syncwarp();
            ++nc;
        }

        // Adam on every candidate row that is due (its block is not at its last check)
        cp_async_wait_all();
        if (due) {
            const bool rs = rv && (MULTI ? blk[b].reset != 0 : s_reset != 0);
            const bool gz = g[0].hi == 0.f && g[1].hi == 0.f && g[2].hi == 0.f;
            if (was || !gz || rs) {
                RowState S;
                S.dh = T.st[0][lane];
                S.dl = T.st[1][lane];
                S.pe = T.st[2][lane];
                if (was) {
                    S.mh = T.st[3][lane];
                    S.ml = T.st[4][lane];
                    S.vh = T.st[5][lane];
                    S.vl = T.st[6][lane];
                }
                const df i1 = MULTI ? blk[b].ibc1 : s_ibc1, i2 = MULTI ? blk[b].ibc2 : s_ibc2;
                adam_core(e, g, S, was, av, Bf.act, i1, i2, rs, C, Bf.dh(pa ^ 1), Bf.dl(pa ^ 1), Bf.Mh, Bf.Ml, Bf.Vh,
                          Bf.Vl, Bf.q(pa ^ 1));
                ++nupd;
            }
        }
        if (MULTI) {
            // the chunk's updates, by the rows' blocks
            const unsigned same = __match_any_sync(FULL, have ? b : -1);
            const unsigned su = __reduce_add_sync(same, nupd);
            if (have && lane == __ffs(same) - 1 && su) atomicAdd(&blk[b].uacc, (unsigned long long)su);
            nupd = 0;
        }
        __syncwarp();
    }
    finish_iteration<MULTI>(br, lfx, viol, nupd, nev, CB, nb, blk, gs, hist_loss, hist_viol, wt);
}

// ------------------------------------------------------------------ edge plan
// Degrees from the CSR offsets: light degree (0 for a heavy row), heavy degree and heavy
// flag of every row; the heavy bit also goes into act.
__global__ void k_degrees(const unsigned long long *__restrict__ row_ptr, int64_t ne,
                          unsigned long long *__restrict__ ldeg, unsigned long long *__restrict__ hdeg,
                          uint32_t *__restrict__ isheavy, uint8_t *__restrict__ act) {
    GRID_STRIDE(e, ne) {
        const unsigned long long d = row_ptr[e + 1] - row_ptr[e];
        const bool h = d > HEAVY;
        ldeg[e] = h ? 0ull : d;
        hdeg[e] = h ? d : 0ull;
        isheavy[e] = h ? 1u : 0u;
        if (h) act[e] = (uint8_t)(act[e] | ACT_HEAVY);
    }
}

// Squared linking lengths of the thresholds of a multi-threshold problem (float32).
struct ThrB2 {
    float b2[MAX_THR];
};

// Place in the edge array of the j-th edge of a row (light rows: their own range in row
// order; heavy rows: after every light edge).
__device__ __forceinline__ unsigned long long edge_place(const unsigned long long *__restrict__ row_ptr,
                                                         const unsigned long long *__restrict__ lptr,
                                                         const unsigned long long *__restrict__ hptr,
                                                         unsigned long long n_light, uint32_t row,
                                                         unsigned long long j) {
    return row_ptr[row + 1] - row_ptr[row] > HEAVY ? n_light + hptr[row] + j : lptr[row] + j;
}

// One CSR entry per directed edge t (sorted keys: row, partner row, threshold index):
// partner's row, threshold index and the link flag at the pair's own linking length,
// written to the row's place in the edge array (light rows with the row's slot in its
// group).  An edge to a later partner also records where its reverse edge lies (found by
// binary search in the partner's sorted keys).
__global__ void k_cols(const unsigned long long *__restrict__ keys, int64_t m, int nbe, int tb, ThrB2 tb2,
                       const unsigned long long *__restrict__ row_ptr, const unsigned long long *__restrict__ lptr,
                       const unsigned long long *__restrict__ hptr, unsigned long long n_light,
                       const uint32_t *__restrict__ epos, const uint32_t *__restrict__ rb,
                       const int64_t *__restrict__ roff, const float4 *__restrict__ P4,
                       const BlockDev *__restrict__ bt, const int64_t *__restrict__ off, int nblk,
                       uint32_t *__restrict__ ecol, uint8_t *__restrict__ eslot, unsigned long long *__restrict__ erev) {
    const unsigned long long mask = (1ull << nbe) - 1ull;
    GRID_STRIDE(t, m) {
        const unsigned long long k = keys[t];
        const uint32_t ti = (uint32_t)(k & ((1ull << tb) - 1ull));
        const uint32_t row = (uint32_t)(k >> (nbe + tb)), prow = (uint32_t)((k >> tb) & mask);
        const uint32_t pos = epos[row];
        const BlockDev &B = bt[find_block(off, nblk, pos)];
        const float4 p = P4[pos], q = P4[epos[prow]];
        const float3 d = canon_dp(p, q, B.periodic, B.L);
        // the link flag at the pair's own linking length
        const float b2 = tb ? (ti == 0 ? tb2.b2[0] : ti == 1 ? tb2.b2[1] : ti == 2 ? tb2.b2[2] : tb2.b2[3]) : B.b2;
        const bool link = cdist2(d.x, d.y, d.z) <= b2;
        const uint32_t cv = prow | (ti << 29) | (link ? 0x80000000u : 0u);
        const unsigned long long r_lo = row_ptr[row], j = (unsigned long long)t - r_lo;
        const unsigned long long dst = edge_place(row_ptr, lptr, hptr, n_light, row, j);
        ecol[dst] = cv;
        if (row_ptr[row + 1] - r_lo <= HEAVY) {
            const int64_t r0 = roff ? roff[rb[row]] : 0;
            eslot[dst] = (uint8_t)(((int64_t)row - r0) & 31);
        }
        if (prow > row) {
            const unsigned long long want = ((((unsigned long long)prow << nbe) | row) << tb) | ti;
            unsigned long long lo = row_ptr[prow], hi = row_ptr[prow + 1];
            while (lo < hi) {   // first key >= want in the partner's row (the reverse edge)
                const unsigned long long mid = (lo + hi) >> 1;
                if (keys[mid] < want) lo = mid + 1;
                else hi = mid;
            }
            // both directions of every pair are keys, so the search always finds it; were it
            // ever missing, the edge would name itself (every bit index stays in range)
            erev[dst] = lo < row_ptr[prow + 1] && keys[lo] == want
                            ? edge_place(row_ptr, lptr, hptr, n_light, prow, lo - row_ptr[prow])
                            : dst;
        }
    }
}

// The 32-row groups of light rows (groups start at the first row of each block; group g
// of block b is gbase[b] + its index in the block): first row and row count of each, and
// the number of edges of its rows to later partners (partners are sorted, so those form
// the end of each row's range).
template <uint32_t PMASK>
__global__ void k_groups(int64_t ne, const uint32_t *__restrict__ rb, const int64_t *__restrict__ roff,
                         const uint32_t *__restrict__ gbase, const unsigned long long *__restrict__ lptr,
                         const uint32_t *__restrict__ col, uint4 *__restrict__ grp,
                         unsigned long long *__restrict__ nup) {
    GRID_STRIDE(e, ne) {
        const int64_t r0 = roff ? roff[rb[e]] : 0, r1 = roff ? roff[rb[e] + 1] : ne;
        const int64_t g = (roff ? (int64_t)gbase[rb[e]] : 0) + (e - r0) / 32;
        if (((e - r0) & 31) == 0)   // first row, rows, first row of the group's work item
            grp[g] = make_uint4((uint32_t)e, (uint32_t)min((int64_t)32, r1 - e),
                                (uint32_t)(r0 + (e - r0) / ITEM_ROWS * ITEM_ROWS), 0u);
        unsigned long long lo = lptr[e], hi = lptr[e + 1];
        const unsigned long long end = hi;
        while (lo < hi) {   // first partner after row e
            const unsigned long long mid = (lo + hi) >> 1;
            if ((col[mid] & PMASK) <= (uint32_t)e) lo = mid + 1;
            else hi = mid;
        }
        if (end > lo) atomicAdd(nup + g, end - lo);
    }
}

// The screen's stream of each group: its rows' edges to later partners sorted by partner
// (then by place), one CTA per group, a bitonic sort in shared memory (a group holds at
// most 32 x HEAVY light edges, so a place fits 13 bits).
constexpr int GSORT_CAP = 32 * HEAVY;
template <uint32_t PMASK>
__global__ void __launch_bounds__(256) k_group_sort(const uint4 *__restrict__ grp, const unsigned long long *__restrict__ lptr,
                                                    const uint32_t *__restrict__ col, const uint8_t *__restrict__ slot,
                                                    const unsigned long long *__restrict__ gup,
                                                    uint2 *__restrict__ sst) {
    extern __shared__ unsigned long long sk[];
    __shared__ int s_n;
    const int64_t g = blockIdx.x;
    const unsigned long long u0 = gup[g], nu = gup[g + 1] - u0;
    if (nu == 0) return;
    const uint4 gr = grp[g];
    const unsigned long long a = lptr[gr.x], len = lptr[gr.x + gr.y] - a;
    const uint32_t off0 = (uint32_t)(a - lptr[gr.z]), row0 = gr.x - gr.z;   // within the work item
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < (int)len; i += blockDim.x) {
        const uint32_t p = col[a + i] & PMASK, row = gr.x + slot[a + i];
        if (p > row) sk[atomicAdd(&s_n, 1)] = ((unsigned long long)p << 13) | (unsigned long long)i;
    }
    __syncthreads();
    const int n = min(s_n, (int)nu);   // equal: both count the partners after each row
    int cap = 1;
    while (cap < n) cap <<= 1;
    for (int i = n + threadIdx.x; i < cap; i += blockDim.x) sk[i] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= cap; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < cap; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long x = sk[i], y = sk[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        sk[i] = y;
                        sk[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const uint32_t i = (uint32_t)(sk[j] & 8191ull);
        sst[u0 + j] = make_uint2(col[a + i], ((off0 + i) << 7) | (row0 + slot[a + i]));
    }
}

// Heavy rows, compacted: sort key (block << 32 | ~degree, so that each block's heavy rows
// come together, longest first), row, and the rows per block.
__global__ void k_heavy_keys(const unsigned long long *__restrict__ hdeg, const uint32_t *__restrict__ isheavy,
                             const uint32_t *__restrict__ hpos, const uint32_t *__restrict__ rb, int64_t ne,
                             unsigned long long *__restrict__ hkey, uint32_t *__restrict__ hrow,
                             uint32_t *__restrict__ per_block) {
    GRID_STRIDE(e, ne) {
        if (!isheavy[e]) continue;
        const uint32_t k = hpos[e], b = rb[e];
        hkey[k] = ((unsigned long long)b << 32) | (0xffffffffull - min(hdeg[e], 0xffffffffull));
        hrow[k] = (uint32_t)e;
        atomicAdd(per_block + b, 1u);
    }
}

// The heavy items in sorted order: edge range and row.
template <uint32_t PMASK>
__global__ void k_heavy_items(const uint32_t *__restrict__ hrow, int64_t nh, const unsigned long long *__restrict__ hptr,
                              const unsigned long long *__restrict__ hdeg, unsigned long long n_light,
                              const uint32_t *__restrict__ col, HeavyItem *__restrict__ item,
                              uint32_t *__restrict__ hmap) {
    GRID_STRIDE(k, nh) {
        const uint32_t e = hrow[k];
        const unsigned long long st = n_light + hptr[e];
        uint32_t lo = 0, hi = (uint32_t)hdeg[e];
        while (lo < hi) {   // first partner after row e
            const uint32_t mid = (lo + hi) >> 1;
            if ((col[st + mid] & PMASK) <= e) lo = mid + 1;
            else hi = mid;
        }
        item[k] = HeavyItem{st, e, (uint32_t)hdeg[e], lo, 0u};
        hmap[e] = (uint32_t)k;
    }
}

// The screen's light chunks of a single problem: item j covers groups [ITEM_GROUPS j,
// min(ng, ITEM_GROUPS (j + 1))) and so the stream range between their offsets.
__global__ void k_chunk_count(const unsigned long long *__restrict__ gup, int64_t ng, int64_t nli, uint32_t clen,
                              uint32_t *__restrict__ cnt) {
    GRID_STRIDE(j, nli) {
        const int64_t g = ITEM_GROUPS * j, g1 = min(ng, g + ITEM_GROUPS);
        const unsigned long long vt = gup[g1] - gup[g];
        cnt[j] = (uint32_t)((vt + clen - 1) / clen);
    }
}

__global__ void k_chunk_fill(const unsigned long long *__restrict__ gup, int64_t ng, int64_t nli, uint32_t clen,
                             const uint32_t *__restrict__ coff, ScreenChunk *__restrict__ ch) {
    GRID_STRIDE(j, nli) {
        const int64_t g = ITEM_GROUPS * j, g1 = min(ng, g + ITEM_GROUPS);
        const unsigned long long e1 = gup[g1];
        uint32_t c = coff[j];
        for (unsigned long long e = gup[g]; e < e1; e += clen, ++c) {
            ScreenChunk x;
            x.eb = e;
            x.len = (uint32_t)min((unsigned long long)clen, e1 - e);
            x.item = (uint32_t)j;
            ch[c] = x;
        }
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
    int64_t ne = 0, n_heavy = 0, max_checks = 0, n_items = 0;
    int nblk = 1;
    double *hist_loss = nullptr;
    unsigned long long *hist_viol = nullptr;
    DBuf<PgdConsts> CB;
    DBuf<PgdBlk> blk;
    DBuf<PgdGlobal> gs;
    DBuf<uint32_t> rb, ecol, hmap;
    DBuf<float4> hgrad;   // per heavy row: gradient hi (w: has a violated pair), lo
    DBuf<unsigned long long> lptr;
    DBuf<HeavyItem> hitem;
    DBuf<uint32_t> ubits;
    DBuf<uint2> sst;
    DBuf<unsigned long long> gup, erev;
    DBuf<ScreenChunk> chunk;
    int64_t n_chunks = 0;
    DBuf<uint8_t> uflag;
    LightPlan LP{};
    DBuf<float4> PE, Dh0, Dl0, Dh1, Dl1, Mh, Ml, Vh, Vl, Q0, Q1;
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

    bool mt = false;                         // several linking lengths (single block)

    void launch_iter() {
        const int g1 = (int)std::max<int64_t>(
            1, std::min<int64_t>(cdiv(n_items, WARPS),
                                 (int64_t)num_sms() * (nb > 1 ? SCREEN_BLOCKS_PER_SM_MULTI : SCREEN_BLOCKS_PER_SM)));
        if (mt) {
            k_pgd_screen<false, true><<<g1, PGD_THREADS, 0, s>>>(ne, Bf, HP, LP, CB.p, blk.p, gs.p, wt, ubits.p,
                                                                 uflag.p);
            PC_CHECK_LAUNCH();
            k_pgd_update<false, true><<<nblk, PGD_THREADS, 0, s>>>(ne, PE.p, Bf, HP, LP, hmap.p, hgrad.p, rb.p, ubits.p,
                                                                   uflag.p, CB.p, nb, blk.p, gs.p, wt, hist_loss,
                                                                   hist_viol);
        } else if (nb == 1) {
            k_pgd_screen<false, false><<<g1, PGD_THREADS, 0, s>>>(ne, Bf, HP, LP, CB.p, blk.p, gs.p, wt, ubits.p,
                                                                  uflag.p);
            PC_CHECK_LAUNCH();
            k_pgd_update<false, false><<<nblk, PGD_THREADS, 0, s>>>(ne, PE.p, Bf, HP, LP, hmap.p, hgrad.p, rb.p, ubits.p,
                                                                    uflag.p, CB.p, nb, blk.p, gs.p, wt, hist_loss,
                                                                    hist_viol);
        } else {
            k_pgd_screen<true, false><<<g1, PGD_THREADS, 0, s>>>(ne, Bf, HP, LP, CB.p, blk.p, gs.p, wt, ubits.p,
                                                                 uflag.p);
            PC_CHECK_LAUNCH();
            k_pgd_update<true, false><<<nblk, PGD_THREADS, 0, s>>>(ne, PE.p, Bf, HP, LP, hmap.p, hgrad.p, rb.p, ubits.p,
                                                                   uflag.p, CB.p, nb, blk.p, gs.p, wt, nullptr,
                                                                   nullptr);
        }
        PC_CHECK_LAUNCH();
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

    // ---- E (numbered canonically, see MortonBox) and CSR
    DBuf<uint32_t> mark(n, s), rank(n, s), tot(1, s);
    PC_CUDA(cudaMemsetAsync(mark.p, 0, n * sizeof(uint32_t), s));
    k_mark_ids<<<grid_for(nA), 256, 0, s>>>(A, nA, B.order.p, mark.p);
    PC_CHECK_LAUNCH();
    scan_exclusive_u32(mark.p, rank.p, n, tot.p, s);
    const int64_t ne = *(uint32_t *)read_back(hs, tot.p, sizeof(uint32_t), s);
    I.ne = ne;
    if (I.mt && ne >= ((int64_t)1 << 29)) fail(PC_EINVAL, "several linking lengths: at most 2^29 editable particles");
    if (ne >= ((int64_t)1 << 30)) fail(PC_EINVAL, "at most 2^30 editable particles");   // candidate entries carry 2 flag bits
    const int tb = I.mt ? 2 : 0;   // threshold-index bits of the directed keys
    ThrB2 tb2;
    for (int k = 0; k < MAX_THR; ++k) tb2.b2[k] = I.mt && k < (int)thr->c.size() ? thr->c[k].b2 : 0.f;
    DBuf<uint32_t> epos(ne, s), dense(n, s);
    {
        // lattice of each block's box: the periodic box, or the bounding box of the originals
        std::vector<MortonBox> hm(nb);
        for (int b = 0; b < nb; ++b) {
            for (int a = 0; a < 3; ++a) {
                const bool per = S.prm[b].periodic != 0;
                const double lo = per ? S.prm[b].box_lo[a] : (double)S.ins[b].lo[a];
                const double ext = per ? S.prm[b].box_hi[a] - S.prm[b].box_lo[a]
                                       : (double)S.ins[b].hi[a] - (double)S.ins[b].lo[a];
                hm[b].lo[a] = lo;
                hm[b].scale[a] = ext > 0.0 ? std::ldexp(1.0, MORTON_BITS) / ext : 0.0;
            }
        }
        DBuf<MortonBox> mb(nb, s);
        PC_CUDA(cudaMemcpyAsync(mb.p, hm.data(), nb * sizeof(MortonBox), cudaMemcpyHostToDevice, s));
        DBuf<unsigned long long> ekey(std::max<int64_t>(1, ne), s);
        DBuf<uint32_t> eid(std::max<int64_t>(1, ne), s), inv(n, s);
        k_edit_keys<<<grid_for(n), 256, 0, s>>>(mark.p, rank.p, n, orig, S.doff.p, nb, mb.p, ekey.p, eid.p);
        PC_CHECK_LAUNCH();
        radix_sort_u64((uint64_t *)ekey.p, eid.p, ne, 3 * MORTON_BITS + std::max(1, ceil_log2((uint64_t)nb)), s);
        inverse_order(B, inv.p, s);
        k_edit_maps<<<grid_for(ne), 256, 0, s>>>(eid.p, ne, inv.p, epos.p, dense.p);
        PC_CHECK_LAUNCH();
        PC_CUDA(cudaStreamSynchronize(s));   // hm lives on this stack frame
    }
    mark.release();
    rank.release();
    // directed edges sorted by (row, partner row, threshold index); 64-bit offsets
    const int nbe = std::max(1, ceil_log2((uint64_t)ne));
    const int64_t m = 2 * nA;
    DBuf<unsigned long long> keys(m, s);
    k_dir_keys<<<grid_for(nA), 256, 0, s>>>(A, I.mt ? thr->Athr : nullptr, nA, dense.p, nbe, tb, keys.p);
    PC_CHECK_LAUNCH();
    radix_sort_u64((uint64_t *)keys.p, nullptr, m, 2 * nbe + tb, s);
    DBuf<unsigned long long> row_ptr(ne + 1, s);
    k_row_bounds<<<grid_for(m + 1), 256, 0, s>>>(keys.p, m, nbe + tb, ne, row_ptr.p);
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

    // ---- edge plan: light rows' edges in row order, then heavy rows' (one item each)
    DBuf<unsigned long long> ldeg(ne, s), hdeg(ne, s), hptr(ne + 1, s), tot64(2, s);
    DBuf<uint32_t> isheavy(ne, s), hpos(ne, s), tot2(1, s);
    k_degrees<<<grid_for(ne), 256, 0, s>>>(row_ptr.p, ne, ldeg.p, hdeg.p, isheavy.p, I.act.p);
    PC_CHECK_LAUNCH();
    I.lptr.alloc(ne + 1, s);
    scan_exclusive_u64((const uint64_t *)ldeg.p, (uint64_t *)I.lptr.p, ne, (uint64_t *)(I.lptr.p + ne), s);
    scan_exclusive_u64((const uint64_t *)hdeg.p, (uint64_t *)hptr.p, ne, (uint64_t *)tot64.p, s);
    scan_exclusive_u32(isheavy.p, hpos.p, ne, tot2.p, s);
    ldeg.release();
    I.n_heavy = *(const uint32_t *)read_back(hs, tot2.p, sizeof(uint32_t), s);
    const unsigned long long n_light = *(const unsigned long long *)read_back(hs, I.lptr.p + ne, 8, s);
    I.ecol.alloc(std::max<int64_t>(1, m), s);
    I.erev.alloc(std::max<int64_t>(1, m), s);
    DBuf<uint8_t> eslot(std::max<unsigned long long>(1, n_light), s);
    k_cols<<<grid_for(m), 256, 0, s>>>(keys.p, m, nbe, tb, tb2, row_ptr.p, I.lptr.p, hptr.p, n_light, epos.p,
                                       I.rb.p, roff.p, B.P4.p, S.dev.p, S.doff.p, nb, I.ecol.p, eslot.p, I.erev.p);
    PC_CHECK_LAUNCH();
    keys.release();
    row_ptr.release();
    dense.release();
    epos.release();
    // light groups, numbered by block, and the screen's stream of each: its rows' edges to
    // later partners, sorted by partner
    std::vector<uint32_t> hgb(nb + 1, 0);
    for (int b = 0; b < nb; ++b) hgb[b + 1] = hgb[b] + (uint32_t)cdiv(I.row_off[b + 1] - I.row_off[b], 32);
    const int64_t ng = hgb[nb];
    DBuf<uint32_t> gbase(nb + 1, s);
    PC_CUDA(cudaMemcpyAsync(gbase.p, hgb.data(), (nb + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    DBuf<uint4> grp(std::max<int64_t>(1, ng), s);
    DBuf<unsigned long long> nup(std::max<int64_t>(1, ng), s);
    I.gup.alloc(ng + 1, s);
    PC_CUDA(cudaMemsetAsync(nup.p, 0, std::max<int64_t>(1, ng) * sizeof(unsigned long long), s));
    if (I.mt)
        k_groups<0x1fffffffu><<<grid_for(ne), 256, 0, s>>>(ne, I.rb.p, roff.p, gbase.p, I.lptr.p, I.ecol.p, grp.p,
                                                           nup.p);
    else
        k_groups<0x7fffffffu><<<grid_for(ne), 256, 0, s>>>(ne, I.rb.p, roff.p, gbase.p, I.lptr.p, I.ecol.p, grp.p,
                                                           nup.p);
    PC_CHECK_LAUNCH();
    scan_exclusive_u64((const uint64_t *)nup.p, (uint64_t *)I.gup.p, ng, (uint64_t *)(I.gup.p + ng), s);
    const unsigned long long n_up = *(const unsigned long long *)read_back(hs, I.gup.p + ng, 8, s);
    I.sst.alloc(std::max<unsigned long long>(1, n_up), s);
    if (n_up > 0) {
        const int smem = (int)(GSORT_CAP * sizeof(unsigned long long));
        if (I.mt) {
            PC_CUDA(cudaFuncSetAttribute(k_group_sort<0x1fffffffu>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            k_group_sort<0x1fffffffu><<<(unsigned)ng, 256, smem, s>>>(grp.p, I.lptr.p, I.ecol.p, eslot.p, I.gup.p,
                                                                      I.sst.p);
        } else {
            PC_CUDA(cudaFuncSetAttribute(k_group_sort<0x7fffffffu>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            k_group_sort<0x7fffffffu><<<(unsigned)ng, 256, smem, s>>>(grp.p, I.lptr.p, I.ecol.p, eslot.p, I.gup.p,
                                                                      I.sst.p);
        }
        PC_CHECK_LAUNCH();
    }
    eslot.release();
    if (nb == 1) {
        // a single problem's screen chunks (screen_chunk entries at most)
        const uint32_t clen = S.prm[0].screen_chunk > 0 ? (uint32_t)S.prm[0].screen_chunk : SCREEN_CHUNK;
        const int64_t nli = cdiv(ne, ITEM_ROWS);
        DBuf<uint32_t> ccnt(std::max<int64_t>(1, nli), s), coff(nli + 1, s);
        k_chunk_count<<<grid_for(nli), 256, 0, s>>>(I.gup.p, ng, nli, clen, ccnt.p);
        PC_CHECK_LAUNCH();
        scan_exclusive_u32(ccnt.p, coff.p, nli, coff.p + nli, s);
        I.n_chunks = *(const uint32_t *)read_back(hs, coff.p + nli, sizeof(uint32_t), s);
        I.chunk.alloc(std::max<int64_t>(1, I.n_chunks), s);
        k_chunk_fill<<<grid_for(nli), 256, 0, s>>>(I.gup.p, ng, nli, clen, coff.p, I.chunk.p);
        PC_CHECK_LAUNCH();
    }
    // the screen's bit mask over the edge array and the rows' flags (both cleared as read)
    I.ubits.alloc(std::max<int64_t>(1, cdiv(m, 32)), s);
    PC_CUDA(cudaMemsetAsync(I.ubits.p, 0, std::max<int64_t>(1, cdiv(m, 32)) * sizeof(uint32_t), s));
    I.uflag.alloc(ne, s);
    PC_CUDA(cudaMemsetAsync(I.uflag.p, 0, ne, s));
    // heavy rows: by block, longest first (long walks start early); per-block ranges
    DBuf<uint32_t> h_per_blk(nb, s), h_off(nb + 1, s);
    PC_CUDA(cudaMemsetAsync(h_per_blk.p, 0, nb * sizeof(uint32_t), s));
    I.hitem.alloc(std::max<int64_t>(1, I.n_heavy), s);
    I.hmap.alloc(ne, s);
    I.hgrad.alloc(2 * std::max<int64_t>(1, I.n_heavy), s);
    if (I.n_heavy > 0) {
        DBuf<unsigned long long> hkey(I.n_heavy, s);
        DBuf<uint32_t> hrow(I.n_heavy, s);
        k_heavy_keys<<<grid_for(ne), 256, 0, s>>>(hdeg.p, isheavy.p, hpos.p, I.rb.p, ne, hkey.p, hrow.p,
                                                  h_per_blk.p);
        PC_CHECK_LAUNCH();
        radix_sort_u64((uint64_t *)hkey.p, hrow.p, I.n_heavy, 32 + std::max(1, ceil_log2((uint64_t)nb)), s);
        if (I.mt)
            k_heavy_items<0x1fffffffu><<<grid_for(I.n_heavy), 256, 0, s>>>(hrow.p, I.n_heavy, hptr.p, hdeg.p, n_light,
                                                                           I.ecol.p, I.hitem.p, I.hmap.p);
        else
            k_heavy_items<0x7fffffffu><<<grid_for(I.n_heavy), 256, 0, s>>>(hrow.p, I.n_heavy, hptr.p, hdeg.p, n_light,
                                                                           I.ecol.p, I.hitem.p, I.hmap.p);
        PC_CHECK_LAUNCH();
    }
    scan_exclusive_u32(h_per_blk.p, h_off.p, nb, h_off.p + nb, s);
    I.LP = LightPlan{I.lptr.p, I.ecol.p, I.gup.p, I.sst.p, I.erev.p, nb == 1 ? I.chunk.p : nullptr, I.n_chunks};
    if (nb > 1) {
        // work table of the blocks still iterating (all of them before the first launch)
        I.bw.alloc(nb, s);
        I.act_blk.alloc(nb, s);
        I.act_pref.alloc(nb + 1, s);
        k_blk_work<<<grid_for(nb), 256, 0, s>>>(roff.p, h_off.p, gbase.p, nb, I.bw.p);
        PC_CHECK_LAUNCH();
        I.wt = WorkTab{I.bw.p, I.act_blk.p, I.act_pref.p};
        k_worktab_init<<<1, 32, 0, s>>>(nb, I.blk.p, I.wt, I.gs.p);
        PC_CHECK_LAUNCH();
    }
    PC_CUDA(cudaStreamSynchronize(s));   // roff and the plan temporaries are released on return
    I.HP.n_heavy = I.n_heavy;
    I.HP.item = I.hitem.p;
    I.n_items = nb == 1 ? I.n_chunks + I.n_heavy : cdiv(ne, ITEM_ROWS) + nb + I.n_heavy;
    I.nblk = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(ne, 32 * WARPS), (int64_t)num_sms() * PGD_BLOCKS_PER_SM));
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
    add_launches(-KERNELS_PER_ITER * (int64_t)k);   // captured, not run
    I.graph_k = k;
}

int64_t PgdSolver::launch(int k) {
    Impl &I = *im;
    if (I.ne == 0) return 0;
    int64_t done = 0;
    if (I.exec) {
        for (; done + I.graph_k <= k || done == 0; done += I.graph_k) {
            PC_CUDA(cudaGraphLaunch(I.exec, I.s));
            add_launches(KERNELS_PER_ITER * (int64_t)I.graph_k);
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
        // every block stops by its last check, so max_launches() launches always suffice;
        // PC_PGD_LAUNCH_LIMIT (a host-side test hook) lowers the limit to exercise the
        // PC_ETIMEOUT path: the host stops polling and fails, the launches already queued
        // run to completion on the stream
        int64_t max_launch = sol.max_launches();
        if (const char *lim = getenv("PC_PGD_LAUNCH_LIMIT")) {
            const long long v = atoll(lim);
            if (v > 0) max_launch = std::min<int64_t>(max_launch, v);
        }
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
