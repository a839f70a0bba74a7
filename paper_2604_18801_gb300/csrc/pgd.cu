// Projected gradient descent on the tightened loss (Algorithm 1, Eq. 3,
// Sec. 3.3 "Gradient descent and projection", Adam as in Sec. 4.1).
//
// Layout.  The editable set E = endpoints(A) is numbered in cell order (dense
// index e), so neighbouring particles sit close in memory.  A is stored as a
// CSR by endpoint: row e lists every active partner k of e (col = k | link
// bit << 31), rows sorted by the partner's position.  State per editable
// particle, float4 each (w unused): original position PE (w = id bits),
// offset delta = P_hat - P as a double-float (hi, lo) in two ping-pong
// buffers, and the Adam moments m, v as double-floats.
//
// One launch per iteration.  Thread e evaluates all active pairs of row e at
// the current offsets: the gradient of row e is a fixed-order segment sum, so
// no float atomics are used and the result is deterministic.  A float32
// screen first discards pairs that are certainly not violated; the others are
// evaluated in double-float.  The loss (each pair counted once, in the row of
// its smaller dense index) and the violation count are reduced per block and
// the last block sums the block partials in a fixed order and takes the stop
// decision of Algorithm 1.  The Adam step of the same launch is written to the
// other offset buffer, so when the check says "stop" the current buffer is
// the answer and nothing has to be undone.
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
                             float4 *__restrict__ Vlo) {
    GRID_STRIDE(e, ne) {
        const float4 p = P4[epos[e]];
        PE[e] = p;
        const int64_t id = (int64_t)__float_as_uint(p.w);
        // delta0 = recon - orig, exactly, as a double-float
        const df dx = two_sum(recon[3 * id + 0], -orig[3 * id + 0]);
        const df dy = two_sum(recon[3 * id + 1], -orig[3 * id + 1]);
        const df dz = two_sum(recon[3 * id + 2], -orig[3 * id + 2]);
        Dhi[e] = make_float4(dx.hi, dy.hi, dz.hi, 0.f);
        Dlo[e] = make_float4(dx.lo, dy.lo, dz.lo, 0.f);
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

__device__ __forceinline__ df shfl_xor_df(df v, int off) {
    return df_make(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

// G lanes share one row: lane `sub` takes edges sub, sub+G, ...; the partial gradients are
// combined by an xor butterfly (df_add is commutative, so every lane of the group ends with
// the same bits).  Rows are assigned in order, G consecutive lanes per row.
template <int G>
__global__ void __launch_bounds__(PGD_THREADS) k_pgd_iter(
    const uint32_t *__restrict__ row_ptr, const uint32_t *__restrict__ col, const float4 *__restrict__ PE, int64_t ne,
    float4 *Dhi0, float4 *Dlo0, float4 *Dhi1, float4 *Dlo1, float4 *__restrict__ Mhi, float4 *__restrict__ Mlo,
    float4 *__restrict__ Vhi, float4 *__restrict__ Vlo, PgdConsts C, PgdState *st, Partial *__restrict__ partials,
    double *__restrict__ hist_loss, unsigned long long *__restrict__ hist_viol) {
    __shared__ int s_stop, s_t;
    __shared__ df s_ibc1, s_ibc2;
    if (threadIdx.x == 0) {
        s_stop = st->stop;
        s_t = st->t;
        s_ibc1 = st->ibc1;
        s_ibc2 = st->ibc2;
    }
    __syncthreads();
    if (s_stop) return;
    const int t = s_t;
    const bool last = C.replay >= 0 ? (t == C.replay) : (t == C.t_max);
    const float4 *Dh = (t & 1) ? Dhi1 : Dhi0;
    const float4 *Dl = (t & 1) ? Dlo1 : Dlo0;
    float4 *Nh = (t & 1) ? Dhi0 : Dhi1;
    float4 *Nl = (t & 1) ? Dlo0 : Dlo1;

    double loss = 0.0;
    unsigned long long viol = 0;
    const int sub = (int)(threadIdx.x % G);
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const bool have = e < ne;
    df g[3] = {df_make(0.f, 0.f), df_make(0.f, 0.f), df_make(0.f, 0.f)};
    float4 deh = make_float4(0.f, 0.f, 0.f, 0.f), del = deh;
    if (have) {
        const float4 pe = PE[e];
        deh = Dh[e];
        del = Dl[e];
        const uint32_t t0 = row_ptr[e], t1 = row_ptr[e + 1];
        for (uint32_t q = t0 + sub; q < t1; q += G) {
            const uint32_t cv = col[q];
            const uint32_t k = cv & 0x7fffffffu;
            const bool link = (cv >> 31) != 0u;
            const float4 pk = __ldg(PE + k);
            const float4 dkh = Dh[k];
            const float3 dp = canon_dp(pe, pk, C.periodic, C.L);
            // float32 screen
            const float rx = __fadd_rn(dp.x, __fsub_rn(deh.x, dkh.x));
            const float ry = __fadd_rn(dp.y, __fsub_rn(deh.y, dkh.y));
            const float rz = __fadd_rn(dp.z, __fsub_rn(deh.z, dkh.z));
            const float d2f = cdist2(rx, ry, rz);
            if (link ? (d2f < C.screen_link) : (d2f > C.screen_non)) continue;
            // double-float evaluation of the pair
            const float4 dkl = Dl[k];
            df r[3];
            const float dpa[3] = {dp.x, dp.y, dp.z};
#pragma unroll
            for (int a = 0; a < 3; ++a) r[a] = df_add_f(df_sub(comp(deh, del, a), comp(dkh, dkl, a)), dpa[a]);
            df d2 = df_mul(r[0], r[0]);
            d2 = df_add(d2, df_mul(r[1], r[1]));
            d2 = df_add(d2, df_mul(r[2], r[2]));
            const df dh = df_sqrt(d2);
            const df v = link ? df_sub(dh, C.thr_link) : df_sub(C.thr_non, dh);
            if (!df_gt0(v)) continue;
            if ((int64_t)k > e) {
                const double vd = df_to_d(v);
                loss += vd * vd;
                viol += 1;
            }
            df u[3];
            if (dh.hi > C.tau) {
#pragma unroll
                for (int a = 0; a < 3; ++a) u[a] = df_div(r[a], dh);
            } else {
                // coincident points (|r| <= b 2^-30): move along the original separation
                const df n0 = df_sqrt(df_add(df_add(two_prod(dp.x, dp.x), two_prod(dp.y, dp.y)), two_prod(dp.z, dp.z)));
#pragma unroll
                for (int a = 0; a < 3; ++a) u[a] = n0.hi > 0.f ? df_div(df_make(dpa[a], 0.f), n0) : df_make(0.f, 0.f);
            }
            const df s = link ? df_add(v, v) : df_neg(df_add(v, v));
#pragma unroll
            for (int a = 0; a < 3; ++a) g[a] = df_add(g[a], df_mul(s, u[a]));
        }
    }
    if (G > 1) {
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
            for (int a = 0; a < 3; ++a) g[a] = df_add(g[a], shfl_xor_df(g[a], off));
            loss += __shfl_xor_sync(0xffffffffu, loss, off);
            viol += __shfl_xor_sync(0xffffffffu, viol, off);
        }
        if (sub != 0) {
            loss = 0.0;
            viol = 0;
        }
    }
    if (have && sub == 0) {
        if (!last) {
            // Adam step t+1 and projection onto [-xi_box, xi_box]
            float4 mh4 = Mhi[e], ml4 = Mlo[e], vh4 = Vhi[e], vl4 = Vlo[e];
            df nd[3], nm[3], nv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                df m = comp(mh4, ml4, a), vv = comp(vh4, vl4, a);
                m = df_add(df_mul(C.beta1, m), df_mul(C.one_m_beta1, g[a]));
                vv = df_add(df_mul(C.beta2, vv), df_mul(C.one_m_beta2, df_mul(g[a], g[a])));
                const df mhat = df_mul(m, s_ibc1);
                const df vhat = df_mul(vv, s_ibc2);
                const df den = df_add(df_sqrt(vhat), C.eps_adam);
                const df step = df_div(df_mul(C.alpha, mhat), den);
                nd[a] = df_clamp(df_sub(comp(deh, del, a), step), C.xi_box);
                nm[a] = m;
                nv[a] = vv;
            }
            Nh[e] = make_float4(nd[0].hi, nd[1].hi, nd[2].hi, 0.f);
            Nl[e] = make_float4(nd[0].lo, nd[1].lo, nd[2].lo, 0.f);
            Mhi[e] = make_float4(nm[0].hi, nm[1].hi, nm[2].hi, 0.f);
            Mlo[e] = make_float4(nm[0].lo, nm[1].lo, nm[2].lo, 0.f);
            Vhi[e] = make_float4(nv[0].hi, nv[1].hi, nv[2].hi, 0.f);
            Vlo[e] = make_float4(nv[0].lo, nv[1].lo, nv[2].lo, 0.f);
        }
    }
    // block reduction in a fixed order
    __shared__ double sl[PGD_THREADS];
    __shared__ unsigned long long sv[PGD_THREADS];
    sl[threadIdx.x] = loss;
    sv[threadIdx.x] = viol;
    __syncthreads();
    for (int w = PGD_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sl[threadIdx.x] += sl[threadIdx.x + w];
            sv[threadIdx.x] += sv[threadIdx.x + w];
        }
        __syncthreads();
    }
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x].loss = sl[0];
        partials[blockIdx.x].viol = sv[0];
        __threadfence();
        const uint32_t prev = atomicAdd(&st->ticket, 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: fixed-order sum of the partials and the stop decision
    double L = 0.0;
    unsigned long long V = 0;
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += PGD_THREADS) {
        L += __ldcg(&partials[b].loss);
        V += __ldcg(&partials[b].viol);
    }
    sl[threadIdx.x] = L;
    sv[threadIdx.x] = V;
    __syncthreads();
    for (int w = PGD_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sl[threadIdx.x] += sl[threadIdx.x + w];
            sv[threadIdx.x] += sv[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        L = sl[0];
        V = sv[0];
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
        const bool conv = L <= C.loss_tol;
        if ((!replay && conv) || last) {
            st->stop = 1;
            st->final_buf = t & 1;
            st->converged = conv ? 1 : 0;
        } else {
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
        st->ticket = 0;
        __threadfence();
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
    // screen bound: float32 r differs from the exact r by at most a few ulps of |r| per axis
    const double R = c.b + 2.0 * std::sqrt(3.0) * c.xi + 4.0 * c.xi;
    const double B4 = 8.0 * ulp32(R);
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
        Vl(ne, s);
    k_state_init<<<grid_for(ne), 256, 0, s>>>(epos.p, ne, B.P4.p, orig, recon, PE.p, Dh0.p, Dl0.p, Mh.p, Ml.p, Vh.p,
                                              Vl.p);
    PC_CHECK_LAUNCH();
    epos.release();

    // ---- state
    // lanes per row: about half the mean row length, a power of two in [1, 32]
    const double mean_deg = (double)m / (double)ne;
    int G = 1;
    while (G < 32 && 2.0 * G <= mean_deg / 2.0) G *= 2;
    const int nblk = (int)cdiv(ne * G, PGD_THREADS);
    DBuf<Partial> partials(nblk, s);

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
#define PC_PGD_LAUNCH(GG)                                                                                          \
    k_pgd_iter<GG><<<nblk, PGD_THREADS, 0, s>>>(row_ptr.p, col.p, PE.p, ne, Dh0.p, Dl0.p, Dh1.p, Dl1.p, Mh.p, Ml.p, \
                                                Vh.p, Vl.p, K, st.p, partials.p, hl_p, hv_p)
        switch (G) {
            case 1: PC_PGD_LAUNCH(1); break;
            case 2: PC_PGD_LAUNCH(2); break;
            case 4: PC_PGD_LAUNCH(4); break;
            case 8: PC_PGD_LAUNCH(8); break;
            case 16: PC_PGD_LAUNCH(16); break;
            default: PC_PGD_LAUNCH(32); break;
        }
#undef PC_PGD_LAUNCH
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
    float ms1 = 0, ms2 = 0;
    cudaEventElapsedTime(&ms1, e0, e1);
    cudaEventElapsedTime(&ms2, e1, e2);
    res.ms = ms2;
    if (ms_csr) *ms_csr = ms1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    return res;
}

}  // namespace pc
