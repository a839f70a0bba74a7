// Constraint selection helpers: the halo-forest spanning forest and the
// canonical export of the active pairs.
//
// Sec. 3.2 (mode HF): safe components are contracted into supernodes; within
// each original halo only a spanning forest of the potentially broken links
// among supernodes is kept.  The paper leaves the forest unspecified (its GPU
// code keeps whichever link wins a union race); here the forest is the unique
// minimum spanning forest under the key (float32 bits of d2, i, j), found by
// Boruvka rounds: every supernode tree picks its minimum incident candidate
// link with a 64-bit atomicMin on (d2 bits << 32 | rank of (i, j)), the picked
// links are hooked with the lock-free union-find, and the rounds repeat until
// no link joins two trees.  With distinct keys every picked link belongs to
// the unique forest, so the result does not depend on thread timing.
#include <algorithm>

#include "pipeline.cuh"

namespace pc {

__device__ __forceinline__ uint32_t sel_root(uint32_t *par, uint32_t x) {
    for (int it = 0; it < (1 << 26); ++it) {
        const uint32_t p = __ldcg(par + x);
        if (p == x) return x;
        const uint32_t g = __ldcg(par + p);
        if (g == p) return p;
        __stcg(par + x, g);
        x = g;
    }
    return x;
}

namespace {

constexpr int RETRY_CAP = 1 << 22;

__device__ __forceinline__ void sel_union(uint32_t *par, uint32_t a, uint32_t b, uint32_t *err) {
    for (int it = 0; it < RETRY_CAP; ++it) {
        a = sel_root(par, a);
        b = sel_root(par, b);
        if (a == b) return;
        if (a > b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(par + b, b, a) == b) return;
    }
    atomicOr(err, ERR_UF_RETRY);
}

inline int grid_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), (int64_t)num_sms() * 16));
}

#define GRID_STRIDE(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ float pair_d2(const float4 p, const float4 q, const BlockDev &c) {
    const bool per = c.periodic != 0;
    return cdist2(cdiff(p.x, q.x, per, c.L[0]), cdiff(p.y, q.y, per, c.L[1]), cdiff(p.z, q.z, per, c.L[2]));
}

// (min id << nb | max id), value = index of the candidate
__global__ void k_id_keys(const unsigned long long *__restrict__ P, int64_t m, const float4 *__restrict__ P4, int nb,
                          unsigned long long *__restrict__ keys, uint32_t *__restrict__ vals) {
    GRID_STRIDE(r, m) {
        const unsigned long long pk = P[r];
        const uint32_t i = __float_as_uint(P4[pk >> 32].w), j = __float_as_uint(P4[pk & 0xffffffffull].w);
        const uint32_t a = min(i, j), b = max(i, j);
        keys[r] = ((unsigned long long)a << nb) | b;
        vals[r] = (uint32_t)r;
    }
}

// Per ranked candidate: msf key, supernode endpoints.
__global__ void k_forest_setup(const unsigned long long *__restrict__ C, const uint32_t *__restrict__ rank_to_c,
                               int64_t m, const float4 *__restrict__ P4, const uint32_t *__restrict__ safe_lab,
                               const BlockDev *__restrict__ bt, const int64_t *__restrict__ off, int nb,
                               unsigned long long *__restrict__ ekey, uint32_t *__restrict__ eu,
                               uint32_t *__restrict__ ev) {
    GRID_STRIDE(q, m) {
        const unsigned long long pk = C[rank_to_c[q]];
        const float4 p = P4[pk >> 32], r = P4[pk & 0xffffffffull];
        const float d2 = pair_d2(p, r, bt[find_block(off, nb, (int64_t)(pk >> 32))]);
        ekey[q] = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned long long)q;
        eu[q] = safe_lab[__float_as_uint(p.w)];
        ev[q] = safe_lab[__float_as_uint(r.w)];
    }
}

__global__ void k_bv_min(const unsigned long long *__restrict__ ekey, const uint32_t *__restrict__ eu,
                         const uint32_t *__restrict__ ev, int64_t m, uint32_t *sup, uint32_t *__restrict__ ru,
                         uint32_t *__restrict__ rv, unsigned long long *best) {
    GRID_STRIDE(q, m) {
        const uint32_t a = sel_root(sup, eu[q]), b = sel_root(sup, ev[q]);
        ru[q] = a;
        rv[q] = b;
        if (a != b) {
            atomicMin(best + a, ekey[q]);
            atomicMin(best + b, ekey[q]);
        }
    }
}

__global__ void k_bv_hook(const unsigned long long *__restrict__ ekey, const uint32_t *__restrict__ ru,
                          const uint32_t *__restrict__ rv, int64_t m, uint32_t *sup,
                          const unsigned long long *__restrict__ best, uint32_t *__restrict__ sel,
                          unsigned long long *picked, uint32_t *err) {
    GRID_STRIDE(q, m) {
        const uint32_t a = ru[q], b = rv[q];
        if (a == b) continue;
        const unsigned long long k = ekey[q];
        if (best[a] == k || best[b] == k) {
            sel[q] = 1u;
            sel_union(sup, a, b, err);
            atomicAdd(picked, 1ull);
        }
    }
}

__global__ void k_bv_reset(const uint32_t *__restrict__ ru, const uint32_t *__restrict__ rv, int64_t m,
                           unsigned long long *best) {
    GRID_STRIDE(q, m) {
        best[ru[q]] = ~0ull;
        best[rv[q]] = ~0ull;
    }
}

__global__ void k_forest_emit(const uint32_t *__restrict__ sel, const uint32_t *__restrict__ pos, int64_t m,
                              const unsigned long long *__restrict__ C, const uint32_t *__restrict__ rank_to_c,
                              unsigned long long *__restrict__ A, int64_t nA) {
    GRID_STRIDE(q, m) {
        if (sel[q]) A[nA + pos[q]] = C[rank_to_c[q]];
    }
}

__global__ void k_fill_u64(unsigned long long *p, unsigned long long v, int64_t n) {
    GRID_STRIDE(i, n) p[i] = v;
}

// export: id pair key + link flag
__global__ void k_export_keys(const unsigned long long *__restrict__ A, int64_t m, const float4 *__restrict__ P4,
                              const BlockDev *__restrict__ bt, const int64_t *__restrict__ off, int nblk, int nb,
                              unsigned long long *__restrict__ keys, uint32_t *__restrict__ link) {
    GRID_STRIDE(r, m) {
        const unsigned long long pk = A[r];
        const float4 p = P4[pk >> 32], q = P4[pk & 0xffffffffull];
        const uint32_t i = __float_as_uint(p.w), j = __float_as_uint(q.w);
        keys[r] = ((unsigned long long)min(i, j) << nb) | max(i, j);
        const BlockDev &c = bt[find_block(off, nblk, (int64_t)(pk >> 32))];
        link[r] = pair_d2(p, q, c) <= c.b2 ? 1u : 0u;
    }
}

__global__ void k_export_split(const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ link,
                               int64_t m, int nb, uint32_t *__restrict__ i_out, uint32_t *__restrict__ j_out,
                               uint8_t *__restrict__ l_out) {
    GRID_STRIDE(r, m) {
        const unsigned long long k = keys[r];
        i_out[r] = (uint32_t)(k >> nb);
        j_out[r] = (uint32_t)(k & ((1ull << nb) - 1ull));
        if (l_out) l_out[r] = (uint8_t)link[r];
    }
}

}  // namespace

int64_t halo_forest(const Binned &B, const BlockSet &S, const uint32_t *safe_lab, const unsigned long long *C,
                    int64_t nC, unsigned long long *A, int64_t nA, uint32_t *err, cudaStream_t s,
                    HostScratch &hs) {
    if (nC <= 0) return 0;
    const int64_t n = B.n;
    const int nb = std::max(1, ceil_log2((uint64_t)n));
    // rank the candidates by (i, j)
    DBuf<unsigned long long> keys(nC, s);
    DBuf<uint32_t> rank_to_c(nC, s);
    k_id_keys<<<grid_for(nC), 256, 0, s>>>(C, nC, B.P4.p, nb, keys.p, rank_to_c.p);
    PC_CHECK_LAUNCH();
    radix_sort_u64((uint64_t *)keys.p, rank_to_c.p, nC, 2 * nb, s);
    keys.release();
    DBuf<unsigned long long> ekey(nC, s), best(n, s), picked(1, s);
    DBuf<uint32_t> eu(nC, s), ev(nC, s), ru(nC, s), rv(nC, s), sel(nC, s), sup(n, s);
    k_forest_setup<<<grid_for(nC), 256, 0, s>>>(C, rank_to_c.p, nC, B.P4.p, safe_lab, S.dev.p, S.doff.p, S.nb,
                                                ekey.p, eu.p, ev.p);
    PC_CHECK_LAUNCH();
    iota_u32(sup.p, n, s);
    k_fill_u64<<<grid_for(n), 256, 0, s>>>(best.p, ~0ull, n);
    PC_CHECK_LAUNCH();
    PC_CUDA(cudaMemsetAsync(sel.p, 0, nC * sizeof(uint32_t), s));
    for (int round = 0; round < 64; ++round) {
        PC_CUDA(cudaMemsetAsync(picked.p, 0, sizeof(unsigned long long), s));
        k_bv_min<<<grid_for(nC), 256, 0, s>>>(ekey.p, eu.p, ev.p, nC, sup.p, ru.p, rv.p, best.p);
        PC_CHECK_LAUNCH();
        k_bv_hook<<<grid_for(nC), 256, 0, s>>>(ekey.p, ru.p, rv.p, nC, sup.p, best.p, sel.p, picked.p, err);
        PC_CHECK_LAUNCH();
        k_bv_reset<<<grid_for(nC), 256, 0, s>>>(ru.p, rv.p, nC, best.p);
        PC_CHECK_LAUNCH();
        const unsigned long long got = *(unsigned long long *)read_back(hs, picked.p, sizeof(unsigned long long), s);
        if (got == 0) break;
    }
    DBuf<uint32_t> pos(nC, s), tot(1, s);
    scan_exclusive_u32(sel.p, pos.p, nC, tot.p, s);
    k_forest_emit<<<grid_for(nC), 256, 0, s>>>(sel.p, pos.p, nC, C, rank_to_c.p, A, nA);
    PC_CHECK_LAUNCH();
    return (int64_t) * (uint32_t *)read_back(hs, tot.p, sizeof(uint32_t), s);
}

void export_pairs(const Binned &B, const BlockSet &S, const unsigned long long *A, int64_t nA, uint32_t *i_out,
                  uint32_t *j_out, uint8_t *link_out, cudaStream_t s) {
    if (nA <= 0) return;
    const int nb = std::max(1, ceil_log2((uint64_t)B.n));
    DBuf<unsigned long long> keys(nA, s);
    DBuf<uint32_t> link(nA, s), di(nA, s), dj(nA, s);
    DBuf<uint8_t> dl(nA, s);
    k_export_keys<<<grid_for(nA), 256, 0, s>>>(A, nA, B.P4.p, S.dev.p, S.doff.p, S.nb, nb, keys.p, link.p);
    PC_CHECK_LAUNCH();
    radix_sort_u64((uint64_t *)keys.p, link.p, nA, 2 * nb, s);
    k_export_split<<<grid_for(nA), 256, 0, s>>>(keys.p, link.p, nA, nb, di.p, dj.p, dl.p);
    PC_CHECK_LAUNCH();
    PC_CUDA(cudaMemcpyAsync(i_out, di.p, nA * sizeof(uint32_t), cudaMemcpyDefault, s));
    PC_CUDA(cudaMemcpyAsync(j_out, dj.p, nA * sizeof(uint32_t), cudaMemcpyDefault, s));
    if (link_out) PC_CUDA(cudaMemcpyAsync(link_out, dl.p, nA, cudaMemcpyDefault, s));
    PC_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- several linking lengths
namespace {

__global__ void k_inverse_order(const uint32_t *__restrict__ order, int64_t n, uint32_t *__restrict__ inv) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        inv[order[p]] = (uint32_t)p;
}

__global__ void k_remap_pairs(const unsigned long long *__restrict__ A, int64_t m, const uint32_t *__restrict__ order_k,
                              const uint32_t *__restrict__ inv, uint8_t t, unsigned long long *__restrict__ out,
                              uint8_t *__restrict__ tout) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long pk = A[r];
        const uint32_t a = inv[order_k[pk >> 32]], b = inv[order_k[pk & 0xffffffffull]];
        out[r] = ((unsigned long long)min(a, b) << 32) | max(a, b);
        tout[r] = t;
    }
}

int remap_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), (int64_t)num_sms() * 16)); }

}  // namespace

void inverse_order(const Binned &B, uint32_t *inv, cudaStream_t s) {
    if (B.n <= 0) return;
    k_inverse_order<<<remap_grid(B.n), 256, 0, s>>>(B.order.p, B.n, inv);
    PC_CHECK_LAUNCH();
}

void remap_pairs(const unsigned long long *A, int64_t m, const uint32_t *order_k, const uint32_t *inv, uint8_t t,
                 unsigned long long *out, uint8_t *tout, cudaStream_t s) {
    if (m <= 0) return;
    k_remap_pairs<<<remap_grid(m), 256, 0, s>>>(A, m, order_k, inv, t, out, tout);
    PC_CHECK_LAUNCH();
}

}  // namespace pc
