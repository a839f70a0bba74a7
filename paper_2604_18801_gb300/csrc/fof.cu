// Input inspection, cell binning, stencil pair search and union-find.
//
// Sec. 2.4 (cell linking, union-find), Sec. 3.1 (vulnerability window) and
// Sec. 3.3 "Identifying safe links and vulnerable pairs" of arXiv 2604.18801.
//
// Binning: cell key = linear index of the cell of each original position,
// stable LSD radix sort of (key, id), then the particles are permuted into
// cell order (float4, w = id bits) and cell_start[] is found by boundary
// detection.  The search visits, for every particle, the 13 forward cells of
// its 27-cell neighbourhood plus the later particles of its own cell, so each
// unordered pair within reach is tested exactly once.  Threads take
// consecutive sorted positions, so a warp walks the same neighbour lists and
// its loads are served from L1.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "pipeline.cuh"

namespace cg = cooperative_groups;

namespace pc {

// ======================================================================= inspect
namespace {

__device__ __forceinline__ uint32_t ord_f32(float f) {   // order-preserving float -> uint
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float unord_f32(uint32_t u) {
    uint32_t v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(v);
#else
    float f;
    memcpy(&f, &v, 4);
    return f;
#endif
}

struct InspectDev {
    uint32_t err;
    uint32_t maxabs;   // float bits of a non-negative value
    uint32_t lo[3];    // ord_f32
    uint32_t hi[3];
};

__global__ void k_inspect(const float *__restrict__ orig, const float *__restrict__ recon, int64_t n, double xi,
                          int periodic, double lo0, double lo1, double lo2, double hi0, double hi1, double hi2,
                          InspectDev *out) {
    const double blo[3] = {lo0, lo1, lo2}, bhi[3] = {hi0, hi1, hi2};
    uint32_t err = 0;
    float mabs = 0.f;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float o = orig[3 * i + d];
            if (!isfinite(o)) { err |= ERR_NONFINITE; continue; }
            mabs = fmaxf(mabs, fabsf(o));
            mn[d] = fminf(mn[d], o);
            mx[d] = fmaxf(mx[d], o);
            // periodic: within a quarter box of the box, so one +-L gives the minimum image
            if (periodic) {
                const double q = 0.25 * (bhi[d] - blo[d]);
                if (!((double)o >= blo[d] - q && (double)o < bhi[d] + q)) err |= ERR_OUTSIDE_BOX;
            }
            if (recon) {
                const float r = recon[3 * i + d];
                if (!isfinite(r)) { err |= ERR_NONFINITE; continue; }
                mabs = fmaxf(mabs, fabsf(r));
                if (fabs((double)r - (double)o) > xi) err |= ERR_BOUND;
            }
        }
    }
    // warp reductions then one atomic per warp
    const unsigned FULL = 0xffffffffu;
    err = __reduce_or_sync(FULL, err);
    uint32_t ma = __reduce_max_sync(FULL, __float_as_uint(mabs));
    uint32_t l[3], h[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        l[d] = __reduce_min_sync(FULL, ord_f32(mn[d]));
        h[d] = __reduce_max_sync(FULL, ord_f32(mx[d]));
    }
    if ((threadIdx.x & 31) == 0) {
        if (err) atomicOr(&out->err, err);
        atomicMax(&out->maxabs, ma);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            atomicMin(&out->lo[d], l[d]);
            atomicMax(&out->hi[d], h[d]);
        }
    }
}

}  // namespace

void *host_scratch(HostScratch &hs, size_t bytes) {
    if (hs.cap < bytes) {
        if (hs.p) cudaFreeHost(hs.p);
        hs.p = nullptr;
        hs.cap = 0;
        PC_CUDA(cudaMallocHost(&hs.p, std::max<size_t>(bytes, 4096)));
        hs.cap = std::max<size_t>(bytes, 4096);
    }
    return hs.p;
}

void *read_back(HostScratch &hs, const void *dev, size_t bytes, cudaStream_t s) {
    void *h = host_scratch(hs, bytes);
    PC_CUDA(cudaMemcpyAsync(h, dev, bytes, cudaMemcpyDeviceToHost, s));
    PC_CUDA(cudaStreamSynchronize(s));
    return h;
}

Inspect inspect_inputs(const float *orig, const float *recon, int64_t n, const pc_params *p, cudaStream_t s,
                       HostScratch &hs) {
    DBuf<InspectDev> d(1, s);
    InspectDev init;
    init.err = 0;
    init.maxabs = 0;
    for (int k = 0; k < 3; ++k) {
        init.lo[k] = 0xffffffffu;
        init.hi[k] = 0u;
    }
    InspectDev *h0 = (InspectDev *)host_scratch(hs, sizeof(InspectDev));
    *h0 = init;
    PC_CUDA(cudaMemcpyAsync(d.p, h0, sizeof(InspectDev), cudaMemcpyHostToDevice, s));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), (int64_t)num_sms() * 8));
    k_inspect<<<grid, 256, 0, s>>>(orig, recon, n, p->xi, p->periodic, p->box_lo[0], p->box_lo[1], p->box_lo[2],
                                   p->box_hi[0], p->box_hi[1], p->box_hi[2], d.p);
    PC_CHECK_LAUNCH();
    InspectDev *h = (InspectDev *)read_back(hs, d.p, sizeof(InspectDev), s);
    Inspect r;
    r.err = h->err;
    uint32_t ma = h->maxabs;
    memcpy(&r.maxabs, &ma, 4);
    for (int k = 0; k < 3; ++k) {
        r.lo[k] = unord_f32(h->lo[k]);
        r.hi[k] = unord_f32(h->hi[k]);
    }
    return r;
}

// ======================================================================= binning
namespace {

__global__ void k_cell_keys(const float *__restrict__ orig, int64_t n, double o0, double o1, double o2, double s0,
                            double s1, double s2, int nx, int ny, int nz, int periodic,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ ids) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int cx = (int)floor(((double)orig[3 * i + 0] - o0) * s0);
        int cy = (int)floor(((double)orig[3 * i + 1] - o1) * s1);
        int cz = (int)floor(((double)orig[3 * i + 2] - o2) * s2);
        if (periodic) {   // positions up to a quarter box outside wrap to their image's cell
            cx = cx < 0 ? cx + nx : (cx >= nx ? cx - nx : cx);
            cy = cy < 0 ? cy + ny : (cy >= ny ? cy - ny : cy);
            cz = cz < 0 ? cz + nz : (cz >= nz ? cz - nz : cz);
        }
        cx = min(max(cx, 0), nx - 1);
        cy = min(max(cy, 0), ny - 1);
        cz = min(max(cz, 0), nz - 1);
        keys[i] = ((uint32_t)cz * (uint32_t)ny + (uint32_t)cy) * (uint32_t)nx + (uint32_t)cx;
        ids[i] = (uint32_t)i;
    }
}

__global__ void k_permute(const float *__restrict__ orig, const uint32_t *__restrict__ order, int64_t n,
                          float4 *__restrict__ P4) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t id = order[k];
        P4[k] = make_float4(orig[3 * (int64_t)id], orig[3 * (int64_t)id + 1], orig[3 * (int64_t)id + 2],
                            __uint_as_float(id));
    }
}

// cell_start[c] = first sorted position with key >= c, for c in [0, ncells].
__global__ void k_cell_bounds(const uint32_t *__restrict__ keys, int64_t n, int64_t ncells,
                              uint32_t *__restrict__ cell_start) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = k == 0 ? -1 : (int64_t)keys[k - 1];
        const int64_t cur = k == n ? ncells : (int64_t)keys[k];
        for (int64_t c = prev + 1; c <= cur; ++c) cell_start[c] = (uint32_t)k;
    }
}

inline int grid_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), (int64_t)num_sms() * 16));
}

}  // namespace

void bin_particles(const float *orig, int64_t n, const Consts &c, Binned &B, cudaStream_t s, HostScratch &hs) {
    B.n = n;
    B.keys.alloc(n, s);
    B.order.alloc(n, s);
    B.P4.alloc(n, s);
    B.cell_start.alloc(c.ncells + 1, s);
    const double o[3] = {c.origin[0], c.origin[1], c.origin[2]};
    double sc[3];
    for (int k = 0; k < 3; ++k) sc[k] = (double)c.inv_w[k];
    k_cell_keys<<<grid_for(n), 256, 0, s>>>(orig, n, o[0], o[1], o[2], sc[0], sc[1], sc[2], c.nc[0], c.nc[1],
                                             c.nc[2], c.periodic, B.keys.p, B.order.p);
    PC_CHECK_LAUNCH();
    radix_sort_u32(B.keys.p, B.order.p, n, c.key_bits, s);
    k_permute<<<grid_for(n), 256, 0, s>>>(orig, B.order.p, n, B.P4.p);
    PC_CHECK_LAUNCH();
    k_cell_bounds<<<grid_for(n + 1), 256, 0, s>>>(B.keys.p, n, c.ncells, B.cell_start.p);
    PC_CHECK_LAUNCH();
    (void)hs;
}

// ======================================================================= union-find
// Parent arrays keep par[x] <= x; the root of a set is its smallest id.
__device__ __forceinline__ uint32_t uf_root(uint32_t *par, uint32_t x) {
    for (int it = 0; it < (1 << 26); ++it) {   // a walk is at most n steps; the cap only guards a broken invariant
        const uint32_t p = __ldcg(par + x);
        if (p == x) return x;
        const uint32_t g = __ldcg(par + p);
        if (g == p) return p;
        __stcg(par + x, g);   // path halving; g is an ancestor of x, so any interleaving is safe
        x = g;                // strictly decreasing: terminates
    }
    return x;
}

constexpr int UF_RETRY_CAP = 1 << 22;

__device__ __forceinline__ void uf_union(uint32_t *par, uint32_t a, uint32_t b, uint32_t *err) {
    for (int it = 0; it < UF_RETRY_CAP; ++it) {
        a = uf_root(par, a);
        b = uf_root(par, b);
        if (a == b) return;
        if (a > b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(par + b, b, a) == b) return;   // hook the larger root under the smaller
    }
    atomicOr(err, ERR_UF_RETRY);
}

namespace {
__global__ void k_uf_flatten(uint32_t *par, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        (void)uf_root(par, (uint32_t)i);
}
__global__ void k_uf_labels(uint32_t *par, int64_t n, uint32_t *lab) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        lab[i] = uf_root(par, (uint32_t)i);
}
}  // namespace

void uf_init(uint32_t *par, int64_t n, cudaStream_t s) { iota_u32(par, n, s); }

// Rewrites par so every entry holds its root (two sweeps: path halving, then roots into a copy).
void uf_flatten(uint32_t *par, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_uf_flatten<<<grid_for(n), 256, 0, s>>>(par, n);
    PC_CHECK_LAUNCH();
    DBuf<uint32_t> lab(n, s);
    k_uf_labels<<<grid_for(n), 256, 0, s>>>(par, n, lab.p);
    PC_CHECK_LAUNCH();
    PC_CUDA(cudaMemcpyAsync(par, lab.p, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
}

// ======================================================================= pair search
namespace {

struct Stencil {
    int n_off;
    int off[14][3];
};

__constant__ Stencil c_stencil;

struct PairArgs {
    uint32_t *fof_par, *safe_par;
    const uint32_t *fof_lab, *safe_lab;
    unsigned long long *A, *C;
    uint64_t capA, capC;
    unsigned long long *counts;
    uint32_t *err;
};

__device__ __forceinline__ void emit_pair(unsigned long long key, unsigned long long *out, uint64_t cap,
                                          unsigned long long *cnt, uint32_t *err) {
    // warp-aggregated reservation: one atomic per group of converged emitting lanes
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(cnt, (unsigned long long)g.size());
    base = g.shfl(base, 0);
    const unsigned long long pos = base + g.thread_rank();
    if (pos < cap) out[pos] = key;
    else atomicOr(err, ERR_INDEX);
}

// PASS 1: union-find + counts.  PASS 2: emission for MODE (0 VP, 1 SC, 2 HF).
template <int PASS, int MODE>
__global__ void __launch_bounds__(256) k_pairs(const float4 *__restrict__ P4, const uint32_t *__restrict__ keys,
                                               const uint32_t *__restrict__ cell_start, int64_t n, Consts c,
                                               PairArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t n_links = 0, n_safe = 0, n_pb = 0, n_pc = 0;
    if (k < n) {
        const float4 p = P4[k];
        const uint32_t id = __float_as_uint(p.w);
        const uint32_t key = keys[k];
        const int nx = c.nc[0], ny = c.nc[1], nz = c.nc[2];
        const int cx = (int)(key % (uint32_t)nx);
        const int cy = (int)((key / (uint32_t)nx) % (uint32_t)ny);
        const int cz = (int)(key / ((uint32_t)nx * (uint32_t)ny));
        const bool per = c.periodic != 0;
        uint32_t my_safe = 0, my_fof = 0;
        if (PASS == 2) {
            if (MODE >= 1) my_safe = a.safe_lab[id];
            if (MODE == 2) my_fof = a.fof_lab[id];
        }
        for (int o = 0; o < c_stencil.n_off; ++o) {
            int qx = cx + c_stencil.off[o][0], qy = cy + c_stencil.off[o][1], qz = cz + c_stencil.off[o][2];
            if (per) {
                qx = qx < 0 ? qx + nx : (qx >= nx ? qx - nx : qx);
                qy = qy < 0 ? qy + ny : (qy >= ny ? qy - ny : qy);
                qz = qz < 0 ? qz + nz : (qz >= nz ? qz - nz : qz);
            } else if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || qz < 0 || qz >= nz) {
                continue;
            }
            const uint32_t cell = ((uint32_t)qz * (uint32_t)ny + (uint32_t)qy) * (uint32_t)nx + (uint32_t)qx;
            int64_t js = min((int64_t)cell_start[cell], n);
            const int64_t je = min((int64_t)cell_start[cell + 1], n);
            if (o == 0) js = k + 1;
            for (int64_t kj = js; kj < je; ++kj) {
                const float4 q = __ldg(P4 + kj);
                const float dx = cdiff(p.x, q.x, per, c.L[0]);
                const float dy = cdiff(p.y, q.y, per, c.L[1]);
                const float dz = cdiff(p.z, q.z, per, c.L[2]);
                const float d2 = cdist2(dx, dy, dz);
                if (d2 > c.hi2) continue;
                const uint32_t jd = __float_as_uint(q.w);
                if (PASS == 1) {
                    if (d2 <= c.lo2) {
                        ++n_safe;
                        ++n_links;
                        if (a.safe_par) uf_union(a.safe_par, id, jd, a.err);
                        if (a.fof_par) uf_union(a.fof_par, id, jd, a.err);
                    } else if (d2 <= c.b2) {
                        ++n_pb;
                        ++n_links;
                        if (a.fof_par) uf_union(a.fof_par, id, jd, a.err);
                    } else {
                        ++n_pc;
                    }
                } else {
                    if (d2 <= c.lo2) continue;   // safe link: never vulnerable
                    const unsigned long long pk = k < kj ? (((unsigned long long)k << 32) | (unsigned long long)kj)
                                                         : (((unsigned long long)kj << 32) | (unsigned long long)k);
                    if (MODE == 0) {
                        emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
                    } else if (MODE == 1) {
                        if (a.safe_lab[jd] != my_safe) emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
                    } else {
                        if (d2 > c.b2) {
                            if (a.fof_lab[jd] != my_fof) emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
                        } else {
                            if (a.safe_lab[jd] != my_safe) emit_pair(pk, a.C, a.capC, a.counts + CNT_C, a.err);
                        }
                    }
                }
            }
        }
    }
    if (PASS == 1) {
        __syncwarp();
        const unsigned FULL = 0xffffffffu;
        n_links = __reduce_add_sync(FULL, n_links);
        n_safe = __reduce_add_sync(FULL, n_safe);
        n_pb = __reduce_add_sync(FULL, n_pb);
        n_pc = __reduce_add_sync(FULL, n_pc);
        if ((threadIdx.x & 31) == 0) {
            if (n_links) atomicAdd(a.counts + CNT_LINKS, (unsigned long long)n_links);
            if (n_safe) atomicAdd(a.counts + CNT_SAFE, (unsigned long long)n_safe);
            if (n_pb) atomicAdd(a.counts + CNT_PB, (unsigned long long)n_pb);
            if (n_pc) atomicAdd(a.counts + CNT_PC, (unsigned long long)n_pc);
        }
    }
}

void upload_stencil(const Consts &c, cudaStream_t s) {
    Stencil st;
    st.n_off = 0;
    // home cell first, then the 13 forward neighbours (lexicographically positive (dz, dy, dx))
    for (int dz = 0; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const bool home = dz == 0 && dy == 0 && dx == 0;
                const bool fwd = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
                if (!home && !fwd) continue;
                // a periodic axis with a single cell has no distinct neighbours along it
                const int d[3] = {dx, dy, dz};
                bool dup = false;
                for (int k = 0; k < 3; ++k)
                    if (c.periodic && c.nc[k] == 1 && d[k] != 0) dup = true;
                if (dup) continue;
                if (home) {
                    // keep the home cell at index 0
                    for (int m = st.n_off; m > 0; --m)
                        for (int k = 0; k < 3; ++k) st.off[m][k] = st.off[m - 1][k];
                    for (int k = 0; k < 3; ++k) st.off[0][k] = d[k];
                } else {
                    for (int k = 0; k < 3; ++k) st.off[st.n_off][k] = d[k];
                }
                st.n_off++;
            }
    PC_CUDA(cudaMemcpyToSymbolAsync(c_stencil, &st, sizeof(st), 0, cudaMemcpyHostToDevice, s));
}

}  // namespace

void pair_pass_union(const Binned &B, const Consts &c, uint32_t *fof_par, uint32_t *safe_par,
                     unsigned long long *counts, uint32_t *err, cudaStream_t s) {
    upload_stencil(c, s);
    PairArgs a = {};
    a.fof_par = fof_par;
    a.safe_par = safe_par;
    a.counts = counts;
    a.err = err;
    const int64_t n = B.n;
    k_pairs<1, 0><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(B.P4.p, B.keys.p, B.cell_start.p, n, c, a);
    PC_CHECK_LAUNCH();
}

void pair_pass_emit(const Binned &B, const Consts &c, int mode, const uint32_t *fof_lab, const uint32_t *safe_lab,
                    unsigned long long *A, uint64_t capA, unsigned long long *C, uint64_t capC,
                    unsigned long long *counts, uint32_t *err, cudaStream_t s) {
    upload_stencil(c, s);
    PairArgs a = {};
    a.fof_lab = fof_lab;
    a.safe_lab = safe_lab;
    a.A = A;
    a.C = C;
    a.capA = capA;
    a.capC = capC;
    a.counts = counts;
    a.err = err;
    const int64_t n = B.n;
    const unsigned g = (unsigned)cdiv(n, 256);
    if (mode == PC_MODE_VP) k_pairs<2, 0><<<g, 256, 0, s>>>(B.P4.p, B.keys.p, B.cell_start.p, n, c, a);
    else if (mode == PC_MODE_SC) k_pairs<2, 1><<<g, 256, 0, s>>>(B.P4.p, B.keys.p, B.cell_start.p, n, c, a);
    else k_pairs<2, 2><<<g, 256, 0, s>>>(B.P4.p, B.keys.p, B.cell_start.p, n, c, a);
    PC_CHECK_LAUNCH();
}

}  // namespace pc
