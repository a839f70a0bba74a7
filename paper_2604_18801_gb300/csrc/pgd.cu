// Projected gradient descent on the tightened loss (Algorithm 1, Eq. 3,
// Sec. 3.3 "Gradient descent and projection", Adam as in Sec. 4.1).
//
// Layout.  The editable set E = endpoints(A) is numbered in cell order (dense
// index e), so neighbouring particles sit close in memory.  A is stored as a
// CSR by endpoint: row e lists every active partner k of e (col = k | link
// bit << 31), rows sorted by the partner's position.  State per editable
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

struct PgdConsts {
    int periodic;
    float L[3];
    float b2;
    float screen_link;   // link pair certainly satisfied when float32 d2 < screen_link
    float screen_non;    // non-link pair certainly satisfied when float32 d2 > screen_non
    float tau;           // coincidence radius b * 2^-30 for the gradient direction
    df thr_link, thr_non, xi_box, alpha, eps_adam;
    df beta1, one_m_beta1, beta2, one_m_beta2;
    int t_max;
    int replay;
    double loss_tol;
    double beta1_d, beta2_d;
    double loss_unit;    // xi^2 2^-24: fixed-point unit of the loss
    double inv_loss_unit;
};

struct PgdState {
    int32_t t;          // updates done
    int32_t stop;
    int32_t final_buf;
    int32_t converged;
    uint32_t ticket;
    uint32_t pad;
    unsigned long long viol, viol0;
    double loss, loss0;
    double b1p, b2p;    // beta^(t+1) for the update of this launch
    df ibc1, ibc2;      // 1 / (1 - beta^(t+1))
    int32_t upd_t;      // check index of the last iteration launch
    int32_t upd_on;     // 1 if that launch's update stands (no stop decided)
    df upd_ibc1, upd_ibc2;
    unsigned long long lfx, vacc;   // launch accumulators: loss (fixed point), violations
    unsigned long long work;        // next work item of the launch
};

struct Partial {
    double loss;
    unsigned long long viol;
};

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

__global__ void k_dir_keys(const unsigned long long *__restrict__ A, int64_t m, const uint32_t *__restrict__ dense,
                           int nb, unsigned long long *__restrict__ keys) {
    GRID_STRIDE(r, m) {
        const unsigned long long pk = A[r];
        const uint32_t ki = (uint32_t)(pk >> 32), kj = (uint32_t)(pk & 0xffffffffull);
        keys[2 * r] = ((unsigned long long)dense[ki] << nb) | kj;
        keys[2 * r + 1] = ((unsigned long long)dense[kj] << nb) | ki;
    }
}

__global__ void k_row_bounds(const unsigned long long *__restrict__ keys, int64_t m, int nb, int64_t nrows,
                             uint32_t *__restrict__ row_ptr) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= m; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = t == 0 ? -1 : (int64_t)(keys[t - 1] >> nb);
        const int64_t cur = t == m ? nrows : (int64_t)(keys[t] >> nb);
        for (int64_t r = prev + 1; r <= cur; ++r) row_ptr[r] = (uint32_t)t;
    }
}

__device__ __forceinline__ float3 canon_dp(const float4 p, const float4 q, int periodic, const float *L) {
    const bool per = periodic != 0;
    return make_float3(cdiff(p.x, q.x, per, L[0]), cdiff(p.y, q.y, per, L[1]), cdiff(p.z, q.z, per, L[2]));
}

__global__ void k_cols(const unsigned long long *__restrict__ keys, int64_t m, int nb,
                       const uint32_t *__restrict__ dense, const uint32_t *__restrict__ epos,
                       const float4 *__restrict__ P4, PgdConsts pc_, uint32_t *__restrict__ col) {
    const unsigned long long mask = (1ull << nb) - 1ull;
    GRID_STRIDE(t, m) {
        const unsigned long long k = keys[t];
        const uint32_t row = (uint32_t)(k >> nb), nbp = (uint32_t)(k & mask);
        const float4 p = P4[epos[row]], q = P4[nbp];
        const float3 d = canon_dp(p, q, pc_.periodic, pc_.L);
        const bool link = cdist2(d.x, d.y, d.z) <= pc_.b2;
        col[t] = dense[nbp] | (link ? 0x80000000u : 0u);
    }
}

__global__ void k_state_init(const uint32_t *__restrict__ epos, int64_t ne, const float4 *__restrict__ P4,
                             const float *__restrict__ orig, const float *__restrict__ recon,
                             float4 *__restrict__ PE, float4 *__restrict__ Dhi, float4 *__restrict__ Dlo,
                             float4 *__restrict__ Mhi, float4 *__restrict__ Mlo, float4 *__restrict__ Vhi,
                             float4 *__restrict__ Vlo, float4 *__restrict__ Q, float4 *__restrict__ Dhi1,
                             float4 *__restrict__ Dlo1, float4 *__restrict__ Q1, uint8_t *__restrict__ act,
                             df xi_box) {
    GRID_STRIDE(e, ne) {
        const float4 p = P4[epos[e]];
        PE[e] = p;
        const int64_t id = (int64_t)__float_as_uint(p.w);
        const float4 q = make_float4(recon[3 * id + 0], recon[3 * id + 1], recon[3 * id + 2], 0.f);   // orig + delta0
        Q[e] = q;
        Q1[e] = q;
        // delta0 = recon - orig, exactly, as a double-float
        const df dx = two_sum(recon[3 * id + 0], -orig[3 * id + 0]);
        const df dy = two_sum(recon[3 * id + 1], -orig[3 * id + 1]);
        const df dz = two_sum(recon[3 * id + 2], -orig[3 * id + 2]);
        Dhi[e] = make_float4(dx.hi, dy.hi, dz.hi, 0.f);
        Dlo[e] = make_float4(dx.lo, dy.lo, dz.lo, 0.f);
        Dhi1[e] = make_float4(dx.hi, dy.hi, dz.hi, 0.f);
        Dlo1[e] = make_float4(dx.lo, dy.lo, dz.lo, 0.f);
        // a row must be updated from the first update on if the projection moves it
        const df nl = df_neg(xi_box);
        const bool out = df_lt(xi_box, dx) || df_lt(dx, nl) || df_lt(xi_box, dy) || df_lt(dy, nl) ||
                         df_lt(xi_box, dz) || df_lt(dz, nl);
        act[e] = out ? 1 : 0;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        Mhi[e] = z;
        Mlo[e] = z;
        Vhi[e] = z;
        Vlo[e] = z;
    }
}

// ------------------------------------------------------------------ iteration
__device__ __forceinline__ df comp(const float4 &h, const float4 &l, int a) {
    return a == 0 ? df_make(h.x, l.x) : (a == 1 ? df_make(h.y, l.y) : df_make(h.z, l.z));
}

__device__ __forceinline__ df df_clamp(df x, df lim) {
    if (df_lt(lim, x)) return lim;
    const df nl = df_neg(lim);
    if (df_lt(x, nl)) return nl;
    return x;
}

// ------------------------------------------------------------------ loss reduction
// The tight loss is accumulated in fixed point: each violated pair adds
// llrint(v^2 / unit) with unit = xi^2 2^-24 (v <= 2 sqrt3 xi + delta_t, so a term is
// below 2^28 units and 2^35 terms fit in 63 bits), and the violated pairs are counted.
// Integer sums do not depend on the order in which warps finish, so the result is
// deterministic although work items are handed out dynamically.  Warps add into
// their block's counters, the last warp of a block into the launch counters, and the
// last block takes the stop decision of Algorithm 1 for check t (at eps_L = 0 the
// count decides: the loss is zero exactly when no active pair is violated).
constexpr int WARPS = PGD_THREADS / 32;

struct BlockRed {
    unsigned long long lfx, viol;
    unsigned count;
};

__device__ __forceinline__ unsigned long long warp_sum_u(unsigned long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ void finish_iteration(BlockRed &br, unsigned long long lfx, unsigned long long viol, int t,
                                                 bool last, const PgdConsts &C, PgdState *st,
                                                 double *hist_loss, unsigned long long *hist_viol) {
    const int lane = threadIdx.x & 31;
    lfx = warp_sum_u(lfx);
    viol = warp_sum_u(viol);
    unsigned prev = 0;
    if (lane == 0) {
        if (lfx) atomicAdd(&br.lfx, lfx);
        if (viol) atomicAdd(&br.viol, viol);
        __threadfence_block();
        prev = atomicAdd(&br.count, 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != WARPS - 1) return;          // not the last warp of this block
    if (lane != 0) return;
    __threadfence_block();
    const unsigned long long bl = atomicAdd(&br.lfx, 0ull), bv = atomicAdd(&br.viol, 0ull);
    if (bl) atomicAdd(&st->lfx, bl);
    if (bv) atomicAdd(&st->vacc, bv);
    __threadfence();
    const unsigned gprev = atomicAdd(&st->ticket, 1u);
    if (gprev != gridDim.x - 1) return;     // not the last block
    __threadfence();
    const unsigned long long LF = atomicAdd(&st->lfx, 0ull), V = atomicAdd(&st->vacc, 0ull);
    const double L = (double)LF * C.loss_unit;
    if (hist_loss) {
        hist_loss[t] = L;
        hist_viol[t] = V;
    }
    if (t == 0) {
        st->loss0 = L;
        st->viol0 = V;
    }
    st->loss = L;
    st->viol = V;
    const bool replay = C.replay >= 0;
    const bool conv = C.loss_tol > 0.0 ? (L <= C.loss_tol) : (V == 0);
    st->upd_t = t;
    st->upd_ibc1 = st->ibc1;
    st->upd_ibc2 = st->ibc2;
    if ((!replay && conv) || last) {
        st->stop = 1;
        st->final_buf = t & 1;
        st->converged = conv ? 1 : 0;
        st->upd_on = 0;
    } else {
        st->upd_on = 1;
        st->t = t + 1;
        const double b1 = st->b1p * C.beta1_d, b2 = st->b2p * C.beta2_d;
        st->b1p = b1;
        st->b2p = b2;
        const double i1 = 1.0 / (1.0 - b1), i2 = 1.0 / (1.0 - b2);
        df x, y;
        x.hi = (float)i1;
        x.lo = (float)(i1 - (double)x.hi);
        y.hi = (float)i2;
        y.lo = (float)(i2 - (double)y.hi);
        st->ibc1 = x;
        st->ibc2 = y;
    }
    st->lfx = 0;
    st->vacc = 0;
    st->work = 0;
    st->ticket = 0;
    __threadfence();
}

// ------------------------------------------------------------------ pair evaluation
// r = dp + (eh + el) - (kh + kl) formed without rounding: Shewchuk's grow-expansion
// (each input added through a chain of TwoSums) gives a nonoverlapping expansion whose
// components sum to r exactly; the largest component plus the rounded sum of the rest
// is r to about 2^-48 relative, and an exact zero stays exactly zero.
__device__ __forceinline__ df exact_r(float dp, float eh, float el, float kh, float kl) {
    float h[5];
    h[0] = dp;
    int m = 1;
    const float in[4] = {eh, el, -kh, -kl};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float q = in[j];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < m) {
                const df t = two_sum(q, h[i]);
                h[i] = t.lo;
                q = t.hi;
            }
        }
        h[m] = q;
        ++m;
    }
    const float rest = __fadd_rn(h[3], __fadd_rn(h[2], __fadd_rn(h[1], h[0])));
    return fast_two_sum(h[4], rest);
}

// Violated amount of Eq. 3 for one active pair (row e, partner k) at the current
// offsets, in double-float, and the gradient term d/d(delta_e) of max(0, v)^2.
__device__ __forceinline__ bool eval_pair(const float4 pe, const float4 deh, const float4 del, int64_t e, uint32_t k,
                                          bool link, const float4 *__restrict__ PE, const float4 *Dh,
                                          const float4 *Dl, const PgdConsts &C, df g[3], double &lt) {
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
    const df v = link ? df_sub(dh, C.thr_link) : df_sub(C.thr_non, dh);
    if (!df_gt0(v)) return false;
    const double vd = df_to_d(v);
    lt = (int64_t)k > e ? vd * vd * C.inv_loss_unit : 0.0;   // in loss units
    // 2 v r / |r| (link) or -2 v r / |r| (non-link); coincident points use the original separation
    const df s = link ? df_add(v, v) : df_neg(df_add(v, v));
    if (dh.hi > C.tau) {
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

__device__ __forceinline__ float shfl_f(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }

struct WarpTab {
    int64_t row[32];                 // the warp's rows: dense index
    uint32_t qk[96];                 // queued pairs: partner
    uint8_t qs[96];                  // queued pairs: row slot | link << 7
    float seg[32][6];                // per-row segment sums of one batch
    uint32_t segmask;                // rows with a segment in the batch
};

// Adam step t+1 and projection onto [-xi_box, xi_box] for one row; writes the next
// offsets, the moments and the next rounded position.
// A row that has never had a gradient (and needs no projection) has zero moments and an
// unchanged offset: Adam leaves it where it is, and both offset buffers already hold
// that value, so nothing is read or written for it.
__device__ __forceinline__ void adam_row(int64_t e, const df g[3], const float4 *Dh, const float4 *Dl,
                                         const float4 *__restrict__ PE, uint8_t *__restrict__ act, const df ibc1,
                                         const df ibc2, const PgdConsts &C, float4 *Nh, float4 *Nl,
                                         float4 *__restrict__ Mhi, float4 *__restrict__ Mlo, float4 *__restrict__ Vhi,
                                         float4 *__restrict__ Vlo, float4 *Qn) {
    const bool gz = g[0].hi == 0.f && g[1].hi == 0.f && g[2].hi == 0.f;
    const bool was = act[e] != 0;
    if (!was && gz) return;
    if (!was) act[e] = 1;
    const float4 deh = Dh[e], del = Dl[e], pe = PE[e];
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 mh4 = was ? Mhi[e] : z4, ml4 = was ? Mlo[e] : z4, vh4 = was ? Vhi[e] : z4, vl4 = was ? Vlo[e] : z4;
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

// Rows with more than HEAVY partners are split into chunks of HEAVY edges.
constexpr uint32_t HEAVY = 256;

struct HeavyPlan {
    int64_t n_light_blocks;          // blocks of 8 warps x 32 light rows
    int64_t n_chunks;                // heavy chunks (one warp each)
    const uint32_t *chunk_row;       // row of each chunk
    const uint32_t *chunk_start;     // first edge of each chunk
    float4 *chunk_g;                 // per chunk: gradient partial (hi at 2c, lo at 2c+1)
};

// One PGD iteration: check t and, unless it is the last check, the update t+1.
//
// Light warps own 32 consecutive rows (editable particles) and walk the flat range of
// the light rows' CSR edges 32 at a time; heavy warps take one chunk of HEAVY edges of
// a heavy row.  The float32 screen on the rounded current positions Q certifies most
// pairs as satisfied; the others are appended, in edge order, to the warp queue.  Every
// 32 queued pairs are evaluated in double-float by the 32 lanes together, and a
// segmented scan (fixed shuffle tree) sums the terms of each row; the row's lane adds
// its batch sum.  Light lane i then applies Adam to its row; a heavy warp writes its
// chunk partial, and k_pgd_heavy adds the partials of a heavy row in chunk order.
__global__ void __launch_bounds__(PGD_THREADS, 4) k_pgd_iter(
    const uint32_t *__restrict__ row_ptr, const uint32_t *__restrict__ col, const float4 *__restrict__ PE, int64_t ne,
    float4 *Dhi0, float4 *Dlo0, float4 *Dhi1, float4 *Dlo1, float4 *Q0, float4 *Q1, float4 *__restrict__ Mhi,
    float4 *__restrict__ Mlo, float4 *__restrict__ Vhi, float4 *__restrict__ Vlo, uint8_t *__restrict__ act,
    HeavyPlan H, PgdConsts C,
    PgdState *st, double *__restrict__ hist_loss,
    unsigned long long *__restrict__ hist_viol) {
    __shared__ int s_stop, s_t;
    __shared__ df s_ibc1, s_ibc2;
    __shared__ WarpTab tab[WARPS];
    __shared__ BlockRed br;
    if (threadIdx.x == 0) {
        s_stop = st->stop;
        s_t = st->t;
        s_ibc1 = st->ibc1;
        s_ibc2 = st->ibc2;
        br.count = 0;
        br.lfx = 0;
        br.viol = 0;
    }
    __syncthreads();
    if (s_stop) return;
    const int t = s_t;
    const bool last = C.replay >= 0 ? (t == C.replay) : (t == C.t_max);
    const float4 *Dh = (t & 1) ? Dhi1 : Dhi0;
    const float4 *Dl = (t & 1) ? Dlo1 : Dlo0;
    const float4 *Qc = (t & 1) ? Q1 : Q0;
    float4 *Nh = (t & 1) ? Dhi0 : Dhi1;
    float4 *Nl = (t & 1) ? Dlo0 : Dlo1;
    float4 *Qn = (t & 1) ? Q0 : Q1;

    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpTab &T = tab[w];
    unsigned long long lfx = 0;     // this lane's share of the tight loss, fixed point
    unsigned long long viol = 0;
    // work items: 32-row groups of light rows, then chunks of heavy rows; the grid is
    // persistent (a few blocks per SM) and warps take items round-robin
    const int64_t n_light_warps = (ne + 31) / 32;
    const int64_t n_items = n_light_warps + H.n_chunks;
    for (;;) {
    unsigned long long itm = 0;
    if (lane == 0) itm = atomicAdd(&st->work, 1ull);
    const int64_t item = (int64_t)__shfl_sync(FULL, itm, 0);
    if (item >= n_items) break;
    const bool heavy_warp = item >= n_light_warps;

    // Virtual edge range [0, VT): light warps map v to (row slot, edge) through the
    // prefix vp of the light rows' degrees; a heavy warp maps v to edge start + v of slot 0.
    int64_t e = -1;              // row of this lane (light warps) / of slot 0 (heavy warps, lane 0)
    bool own = false;            // this lane applies Adam to row e
    uint32_t rp = 0, vp = 0, VT = 0, hstart = 0;
    int64_t chunk = -1;
    float4 qe = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!heavy_warp) {
        const int64_t r0 = item * 32;
        e = r0 + lane;
        const bool have = e < ne;
        uint32_t deg = 0;
        if (have) {
            rp = row_ptr[e];
            deg = row_ptr[e + 1] - rp;
            qe = Qc[e];
            T.row[lane] = e;
        }
        const uint32_t ld = deg <= HEAVY ? deg : 0u;
        own = have && deg <= HEAVY;
        // exclusive warp scan of the light degrees
        uint32_t inc = ld;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, off);
            if (lane >= off) inc += y;
        }
        vp = inc - ld;
        VT = __shfl_sync(FULL, inc, 31);
    } else {
        chunk = item - n_light_warps;
        if (chunk < H.n_chunks) {
            const uint32_t row = H.chunk_row[chunk];
            hstart = H.chunk_start[chunk];
            const uint32_t rend = row_ptr[row + 1];
            VT = min(HEAVY, rend - hstart);
            e = row;
            if (lane == 0) T.row[0] = row;
            qe = Qc[row];
        }
    }
    __syncwarp();

    df g[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};   // gradient of the lane's row
    int qn = 0;
    const bool per = C.periodic != 0;

    auto batch = [&](int cnt) {
        const bool valid = lane < cnt;
        int s = 32;
        df gt[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};
        if (valid) {
            const uint32_t k = T.qk[lane];
            s = T.qs[lane] & 0x7f;
            const bool link = (T.qs[lane] >> 7) != 0;
            const int64_t er = T.row[s];
            double lt = 0.0;
            if (eval_pair(PE[er], Dh[er], Dl[er], er, k, link, PE, Dh, Dl, C, gt, lt)) {
                lfx += (unsigned long long)llrint(lt);
                viol += (int64_t)k > er ? 1ull : 0ull;
            }
        }
        // segmented inclusive scan over lanes; entries are grouped by row in edge order
        const int sp = __shfl_up_sync(FULL, s, 1);
        const bool head = lane == 0 || sp != s;
        const unsigned hm = __ballot_sync(FULL, head);
        const int seg0 = 31 - __clz(hm & (0xffffffffu >> (31 - lane)));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            df y[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                y[a] = df_make(__shfl_up_sync(FULL, gt[a].hi, off), __shfl_up_sync(FULL, gt[a].lo, off));
            if (lane - off >= seg0) {
#pragma unroll
                for (int a = 0; a < 3; ++a) gt[a] = df_add(y[a], gt[a]);
            }
        }
        const int sn = __shfl_down_sync(FULL, s, 1);
        const bool tail = valid && (lane == cnt - 1 || sn != s);
        if (tail) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                T.seg[s][2 * a] = gt[a].hi;
                T.seg[s][2 * a + 1] = gt[a].lo;
            }
        }
        const unsigned tm = __ballot_sync(FULL, tail);
        unsigned mask = 0;
        for (unsigned b = tm; b; b &= b - 1) {
            const int src = __ffs(b) - 1;
            mask |= 1u << __shfl_sync(FULL, s, src);
        }
        __syncwarp();
        if (mask & (1u << lane)) {
#pragma unroll
            for (int a = 0; a < 3; ++a) g[a] = df_add(g[a], df_make(T.seg[lane][2 * a], T.seg[lane][2 * a + 1]));
        }
        __syncwarp();
    };

    // row slot and edge of virtual edge v (light: largest s with vp[s] <= v)
    auto locate = [&](uint32_t v, int &s, uint32_t &tt) {
        s = 0;
        tt = hstart + v;
        if (!heavy_warp) {
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t y = __shfl_sync(FULL, vp, (s + step) & 31);
                if (s + step < 32 && y <= v) s += step;
            }
            tt = __shfl_sync(FULL, rp, s) + (v - __shfl_sync(FULL, vp, s));
        }
    };
    auto enqueue = [&](bool need, uint32_t k, int s, bool link) {
        const unsigned bal = __ballot_sync(FULL, need);
        if (need) {
            const int pos = qn + __popc(bal & ((1u << lane) - 1u));
            T.qk[pos] = k;
            T.qs[pos] = (uint8_t)(s | (link ? 0x80 : 0));
        }
        qn += __popc(bal);
    };
    // two edges per lane per trip: both partner loads are in flight before either is used
    for (uint32_t base = 0; base < VT; base += 64) {
        const uint32_t v0 = base + lane, v1 = base + 32 + lane;
        int s0, s1;
        uint32_t t0, t1;
        locate(v0, s0, t0);
        locate(v1, s1, t1);
        const bool ok0 = v0 < VT, ok1 = v1 < VT;
        const uint32_t c0v = ok0 ? col[t0] : 0u, c1v = ok1 ? col[t1] : 0u;
        const uint32_t k0 = c0v & 0x7fffffffu, k1 = c1v & 0x7fffffffu;
        const float4 q0 = ok0 ? Qc[k0] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q1 = ok1 ? Qc[k1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float ax = shfl_f(qe.x, s0), ay = shfl_f(qe.y, s0), az = shfl_f(qe.z, s0);
        const float bx = shfl_f(qe.x, s1), by = shfl_f(qe.y, s1), bz = shfl_f(qe.z, s1);
        const bool l0 = (c0v >> 31) != 0u, l1 = (c1v >> 31) != 0u;
        const float d0 = cdist2(cdiff(ax, q0.x, per, C.L[0]), cdiff(ay, q0.y, per, C.L[1]), cdiff(az, q0.z, per, C.L[2]));
        const float d1 = cdist2(cdiff(bx, q1.x, per, C.L[0]), cdiff(by, q1.y, per, C.L[1]), cdiff(bz, q1.z, per, C.L[2]));
        const bool n0 = ok0 && (l0 ? !(d0 < C.screen_link) : !(d0 > C.screen_non));
        const bool n1 = ok1 && (l1 ? !(d1 < C.screen_link) : !(d1 > C.screen_non));
        enqueue(n0, k0, s0, l0);
        enqueue(n1, k1, s1, l1);
        __syncwarp();
        while (qn >= 32) {
            batch(32);
            uint32_t mk[2] = {0u, 0u};
            uint8_t ms[2] = {0, 0};
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (lane + 32 * h < qn - 32) {
                    mk[h] = T.qk[32 + lane + 32 * h];
                    ms[h] = T.qs[32 + lane + 32 * h];
                }
            __syncwarp();
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (lane + 32 * h < qn - 32) {
                    T.qk[lane + 32 * h] = mk[h];
                    T.qs[lane + 32 * h] = ms[h];
                }
            qn -= 32;
            __syncwarp();
        }
    }
    if (qn > 0) batch(qn);

    if (!heavy_warp) {
        if (own && !last) adam_row(e, g, Dh, Dl, PE, act, s_ibc1, s_ibc2, C, Nh, Nl, Mhi, Mlo, Vhi, Vlo, Qn);
    } else if (chunk >= 0 && chunk < H.n_chunks && lane == 0) {
        H.chunk_g[2 * chunk] = make_float4(g[0].hi, g[1].hi, g[2].hi, 0.f);
        H.chunk_g[2 * chunk + 1] = make_float4(g[0].lo, g[1].lo, g[2].lo, 0.f);
    }
    __syncwarp();
    }   // work items
    finish_iteration(br, lfx, viol, t, last, C, st, hist_loss, hist_viol);
}

// Heavy rows: sum the chunk partials in chunk order and apply Adam (same update as
// light rows).  Runs after k_pgd_iter of the same iteration, with the step and buffers
// that launch used (recorded in the state by its last block).
__global__ void k_pgd_heavy(const uint32_t *__restrict__ hrow, const uint32_t *__restrict__ hc0, int64_t nh,
                            const float4 *__restrict__ chunk_g, const float4 *__restrict__ PE, float4 *Dhi0,
                            float4 *Dlo0, float4 *Dhi1, float4 *Dlo1, float4 *Q0, float4 *Q1,
                            float4 *__restrict__ Mhi, float4 *__restrict__ Mlo, float4 *__restrict__ Vhi,
                            float4 *__restrict__ Vlo, uint8_t *__restrict__ act, PgdConsts C,
                            const PgdState *st) {
    if (!st->upd_on) return;
    const int t = st->upd_t;
    const df ibc1 = st->upd_ibc1, ibc2 = st->upd_ibc2;
    const float4 *Dh = (t & 1) ? Dhi1 : Dhi0;
    const float4 *Dl = (t & 1) ? Dlo1 : Dlo0;
    float4 *Nh = (t & 1) ? Dhi0 : Dhi1;
    float4 *Nl = (t & 1) ? Dlo0 : Dlo1;
    float4 *Qn = (t & 1) ? Q0 : Q1;
    GRID_STRIDE(i, nh) {
        const uint32_t e = hrow[i];
        df g[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};
        for (uint32_t c = hc0[i]; c < hc0[i + 1]; ++c) {
            const float4 h = chunk_g[2 * c], l = chunk_g[2 * c + 1];
            g[0] = df_add(g[0], df_make(h.x, l.x));
            g[1] = df_add(g[1], df_make(h.y, l.y));
            g[2] = df_add(g[2], df_make(h.z, l.z));
        }
        adam_row(e, g, Dh, Dl, PE, act, ibc1, ibc2, C, Nh, Nl, Mhi, Mlo, Vhi, Vlo, Qn);
    }
}

// CSR-side plan of the heavy rows: chunk counts, row list, chunk list.
__global__ void k_heavy_count(const uint32_t *__restrict__ row_ptr, int64_t ne, uint32_t *__restrict__ nchunk,
                              uint32_t *__restrict__ isheavy) {
    GRID_STRIDE(e, ne) {
        const uint32_t d = row_ptr[e + 1] - row_ptr[e];
        const bool h = d > HEAVY;
        nchunk[e] = h ? (d + HEAVY - 1) / HEAVY : 0u;
        isheavy[e] = h ? 1u : 0u;
    }
}

__global__ void k_heavy_fill(const uint32_t *__restrict__ row_ptr, int64_t ne, const uint32_t *__restrict__ nchunk,
                             const uint32_t *__restrict__ c0, const uint32_t *__restrict__ isheavy,
                             const uint32_t *__restrict__ hpos, uint32_t *__restrict__ chunk_row,
                             uint32_t *__restrict__ chunk_start, uint32_t *__restrict__ hrow,
                             uint32_t *__restrict__ hc0) {
    GRID_STRIDE(e, ne) {
        if (!isheavy[e]) continue;
        const uint32_t c = c0[e];
        for (uint32_t j = 0; j < nchunk[e]; ++j) {
            chunk_row[c + j] = (uint32_t)e;
            chunk_start[c + j] = row_ptr[e] + j * HEAVY;
        }
        hrow[hpos[e]] = (uint32_t)e;
        hc0[hpos[e]] = c;
    }
}

__global__ void k_copy_recon(const float *__restrict__ recon, float *__restrict__ out, int64_t m) {
    GRID_STRIDE(i, m) out[i] = recon[i];
}

__global__ void k_output(const float4 *__restrict__ PE, int64_t ne, const float4 *Dhi0, const float4 *Dlo0,
                         const float4 *Dhi1, const float4 *Dlo1, const PgdState *st, float *__restrict__ out) {
    const int fb = st->final_buf;
    if (st->t == 0) return;   // no update happened: the reconstruction stands
    const float4 *Dh = fb ? Dhi1 : Dhi0;
    const float4 *Dl = fb ? Dlo1 : Dlo0;
    GRID_STRIDE(e, ne) {
        const float4 p = PE[e], h = Dh[e], l = Dl[e];
        const int64_t id = (int64_t)__float_as_uint(p.w);
        const float pa[3] = {p.x, p.y, p.z}, ha[3] = {h.x, h.y, h.z}, la[3] = {l.x, l.y, l.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // round(p + hi + lo) to float32
            const df s = two_sum(pa[a], ha[a]);
            out[3 * id + a] = __fadd_rn(s.hi, __fadd_rn(s.lo, la[a]));
        }
    }
}

__global__ void k_delta_out(const float4 *__restrict__ PE, int64_t ne, const float4 *Dhi0, const float4 *Dlo0,
                            const float4 *Dhi1, const float4 *Dlo1, const PgdState *st, double *__restrict__ out) {
    const int fb = st->final_buf;
    const float4 *Dh = fb ? Dhi1 : Dhi0;
    const float4 *Dl = fb ? Dlo1 : Dlo0;
    GRID_STRIDE(e, ne) {
        const float4 p = PE[e], h = Dh[e], l = Dl[e];
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

}  // namespace

PgdResult run_pgd(const Binned &B, const Consts &c, const pc_params *p, const float *orig, const float *recon,
                  const unsigned long long *A, int64_t nA, float *corrected, cudaStream_t s, HostScratch &hs,
                  double *ms_csr, double *delta_out, double *hist_loss, unsigned long long *hist_viol) {
    PgdResult res;
    const int64_t n = B.n;
    cudaEvent_t e0, e1, e2;
    PC_CUDA(cudaEventCreate(&e0));
    PC_CUDA(cudaEventCreate(&e1));
    PC_CUDA(cudaEventCreate(&e2));
    PC_CUDA(cudaEventRecord(e0, s));
    k_copy_recon<<<grid_for(3 * n), 256, 0, s>>>(recon, corrected, 3 * n);
    PC_CHECK_LAUNCH();

    // ---- constants
    PgdConsts K;
    K.periodic = c.periodic;
    for (int a = 0; a < 3; ++a) K.L[a] = c.L[a];
    K.b2 = c.b2;
    const double thrL = c.b - c.dt, thrN = c.b + c.dt;
    // screen bound: the float32 difference of the rounded current positions differs from the
    // exact offset by at most one ulp of the coordinates plus one ulp of |r| per axis
    const double R = c.b + 2.0 * std::sqrt(3.0) * c.xi + 4.0 * c.xi;
    const double B4 = 2.0 * std::sqrt(3.0) * (ulp32(c.M + 2.0 * c.xi) + ulp32(R));
    K.screen_link = thrL - B4 > 0 ? f32_down((thrL - B4) * (thrL - B4) * (1.0 - std::ldexp(1.0, -20))) : -1.0f;
    K.screen_non = f32_up((thrN + B4) * (thrN + B4) * (1.0 + std::ldexp(1.0, -20)));
    K.tau = (float)std::ldexp(c.b, -30);
    K.thr_link = df_split(thrL);
    K.thr_non = df_split(thrN);
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

    if (nA == 0) {
        // nothing to enforce: the reconstruction stands, zero iterations
        res.converged = true;
        res.loss_evals = 1;
        if (delta_out) PC_CUDA(cudaMemsetAsync(delta_out, 0, 3 * n * sizeof(double), s));
        if (hist_loss) PC_CUDA(cudaMemsetAsync(hist_loss, 0, sizeof(double), s));
        if (hist_viol) PC_CUDA(cudaMemsetAsync(hist_viol, 0, sizeof(unsigned long long), s));
        PC_CUDA(cudaEventRecord(e1, s));
        PC_CUDA(cudaEventRecord(e2, s));
        PC_CUDA(cudaEventSynchronize(e2));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        if (ms_csr) *ms_csr = 0;
        return res;
    }

    // ---- E and CSR
    const int nb = std::max(1, ceil_log2((uint64_t)n));
    DBuf<uint32_t> mark(n, s), dense(n, s), tot(1, s);
    PC_CUDA(cudaMemsetAsync(mark.p, 0, n * sizeof(uint32_t), s));
    k_mark<<<grid_for(nA), 256, 0, s>>>(A, nA, mark.p);
    PC_CHECK_LAUNCH();
    scan_exclusive_u32(mark.p, dense.p, n, tot.p, s);
    const int64_t ne = *(uint32_t *)read_back(hs, tot.p, sizeof(uint32_t), s);
    res.n_editable = ne;
    DBuf<uint32_t> epos(ne, s);
    k_epos<<<grid_for(n), 256, 0, s>>>(mark.p, dense.p, n, epos.p);
    PC_CHECK_LAUNCH();
    mark.release();
    const int64_t m = 2 * nA;
    DBuf<unsigned long long> keys(m, s);
    k_dir_keys<<<grid_for(nA), 256, 0, s>>>(A, nA, dense.p, nb, keys.p);
    PC_CHECK_LAUNCH();
    radix_sort_u64((uint64_t *)keys.p, nullptr, m, nb + std::max(1, ceil_log2((uint64_t)ne)), s);
    DBuf<uint32_t> row_ptr(ne + 1, s), col(m, s);
    k_row_bounds<<<grid_for(m + 1), 256, 0, s>>>(keys.p, m, nb, ne, row_ptr.p);
    PC_CHECK_LAUNCH();
    k_cols<<<grid_for(m), 256, 0, s>>>(keys.p, m, nb, dense.p, epos.p, B.P4.p, K, col.p);
    PC_CHECK_LAUNCH();
    keys.release();
    dense.release();
    DBuf<float4> PE(ne, s), Dh0(ne, s), Dl0(ne, s), Dh1(ne, s), Dl1(ne, s), Mh(ne, s), Ml(ne, s), Vh(ne, s),
        Vl(ne, s), Q0(ne, s), Q1(ne, s);
    DBuf<uint8_t> act(ne, s);
    k_state_init<<<grid_for(ne), 256, 0, s>>>(epos.p, ne, B.P4.p, orig, recon, PE.p, Dh0.p, Dl0.p, Mh.p, Ml.p, Vh.p,
                                              Vl.p, Q0.p, Dh1.p, Dl1.p, Q1.p, act.p, K.xi_box);
    PC_CHECK_LAUNCH();
    epos.release();

    // ---- state
    // heavy rows (more than HEAVY partners) are split into chunks of HEAVY edges
    DBuf<uint32_t> nchunk(ne, s), isheavy(ne, s), c0(ne, s), hpos(ne, s), tot2(2, s);
    k_heavy_count<<<grid_for(ne), 256, 0, s>>>(row_ptr.p, ne, nchunk.p, isheavy.p);
    PC_CHECK_LAUNCH();
    scan_exclusive_u32(nchunk.p, c0.p, ne, tot2.p, s);
    scan_exclusive_u32(isheavy.p, hpos.p, ne, tot2.p + 1, s);
    uint32_t tots[2];
    memcpy(tots, read_back(hs, tot2.p, 2 * sizeof(uint32_t), s), sizeof(tots));
    const int64_t n_chunks = tots[0], n_heavy = tots[1];
    DBuf<uint32_t> chunk_row(n_chunks, s), chunk_start(n_chunks, s), hrow(n_heavy, s), hc0(n_heavy + 1, s);
    DBuf<float4> chunk_g(2 * n_chunks, s);
    if (n_heavy > 0) {
        k_heavy_fill<<<grid_for(ne), 256, 0, s>>>(row_ptr.p, ne, nchunk.p, c0.p, isheavy.p, hpos.p, chunk_row.p,
                                                  chunk_start.p, hrow.p, hc0.p);
        PC_CHECK_LAUNCH();
        PC_CUDA(cudaMemcpyAsync(hc0.p + n_heavy, tot2.p, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    nchunk.release();
    isheavy.release();
    c0.release();
    hpos.release();
    HeavyPlan HP;
    HP.n_light_blocks = cdiv(ne, PGD_THREADS);      // one row per lane, 32 rows per warp
    HP.n_chunks = n_chunks;
    HP.chunk_row = chunk_row.p;
    HP.chunk_start = chunk_start.p;
    HP.chunk_g = chunk_g.p;
    const int64_t n_items = cdiv(ne, 32) + n_chunks;
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n_items, WARPS), (int64_t)num_sms() * 4));

    DBuf<PgdState> st(1, s);
    const int64_t hist_n = (p->replay_iters >= 0 ? p->replay_iters : p->t_max) + 1;
    DBuf<double> hl_own(hist_loss ? 0 : hist_n, s);
    DBuf<unsigned long long> hv_own(hist_viol ? 0 : hist_n, s);
    double *hl_p = hist_loss ? hist_loss : hl_own.p;
    unsigned long long *hv_p = hist_viol ? hist_viol : hv_own.p;
    PgdState h0;
    memset(&h0, 0, sizeof(h0));
    h0.b1p = p->beta1;
    h0.b2p = p->beta2;
    h0.ibc1 = df_split(1.0 / (1.0 - p->beta1));
    h0.ibc2 = df_split(1.0 / (1.0 - p->beta2));
    PgdState *hs0 = (PgdState *)host_scratch(hs, sizeof(PgdState));
    *hs0 = h0;
    PC_CUDA(cudaMemcpyAsync(st.p, hs0, sizeof(PgdState), cudaMemcpyHostToDevice, s));
    PC_CUDA(cudaEventRecord(e1, s));

    auto launch_iter = [&]() {
        k_pgd_iter<<<nblk, PGD_THREADS, 0, s>>>(row_ptr.p, col.p, PE.p, ne, Dh0.p, Dl0.p, Dh1.p, Dl1.p, Q0.p, Q1.p, Mh.p,
                                                 Ml.p, Vh.p, Vl.p, act.p, HP, K, st.p, hl_p, hv_p);
        if (n_heavy > 0) {
            PC_CHECK_LAUNCH();
            k_pgd_heavy<<<grid_for(n_heavy), 256, 0, s>>>(hrow.p, hc0.p, n_heavy, chunk_g.p, PE.p, Dh0.p, Dl0.p, Dh1.p,
                                                          Dl1.p, Q0.p, Q1.p, Mh.p, Ml.p, Vh.p, Vl.p, act.p, K, st.p);
        }
    };

    // ---- iterations: launch in growing chunks, poll the device stop flag between chunks
    int64_t launched = 0;
    const int64_t max_launch = hist_n + 1;
    int chunk = 4;
    for (;;) {
        for (int k = 0; k < chunk && launched < max_launch; ++k, ++launched) {
            launch_iter();
            PC_CHECK_LAUNCH();
        }
        const PgdState *h = (const PgdState *)read_back(hs, st.p, sizeof(PgdState), s);
        if (h->stop) break;
        if (launched >= max_launch) {
            set_error("PGD loop did not reach its stop decision");
            throw Fail{PC_ETIMEOUT};
        }
        chunk = std::min(chunk * 2, 256);
    }
    cudaEvent_t e_it;
    PC_CUDA(cudaEventCreate(&e_it));
    PC_CUDA(cudaEventRecord(e_it, s));
    k_output<<<grid_for(ne), 256, 0, s>>>(PE.p, ne, Dh0.p, Dl0.p, Dh1.p, Dl1.p, st.p, corrected);
    PC_CHECK_LAUNCH();
    if (delta_out) {
        PC_CUDA(cudaMemsetAsync(delta_out, 0, 3 * n * sizeof(double), s));
        k_delta_out<<<grid_for(ne), 256, 0, s>>>(PE.p, ne, Dh0.p, Dl0.p, Dh1.p, Dl1.p, st.p, delta_out);
        PC_CHECK_LAUNCH();
    }
    PC_CUDA(cudaEventRecord(e2, s));
    const PgdState *h = (const PgdState *)read_back(hs, st.p, sizeof(PgdState), s);
    res.iters = h->t;
    res.loss_evals = h->t + 1;
    res.viol0 = (int64_t)h->viol0;
    res.viol_final = (int64_t)h->viol;
    res.loss0 = h->loss0;
    res.loss_final = h->loss;
    res.converged = h->converged != 0;
    float ms1 = 0, ms2 = 0, ms3 = 0;
    cudaEventElapsedTime(&ms1, e0, e1);
    cudaEventElapsedTime(&ms2, e1, e2);
    cudaEventElapsedTime(&ms3, e1, e_it);
    cudaEventDestroy(e_it);
    res.ms = ms2;
    res.ms_iter = ms3;
    res.launches = launched;
    if (ms_csr) *ms_csr = ms1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    return res;
}

}  // namespace pc
