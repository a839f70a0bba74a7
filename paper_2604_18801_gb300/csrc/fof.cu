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

struct InspectIn {      // per block: what the check needs
    double xi;
    double lo[3], hi[3];
    int periodic;
};

constexpr int TILE = 4096;   // particles per CTA of the inspection (tiles never straddle blocks)

__global__ void k_inspect(const float *__restrict__ orig, const float *__restrict__ recon,
                          const int2 *__restrict__ tiles, const int64_t *__restrict__ off,
                          const InspectIn *__restrict__ bin, InspectDev *out) {
    const int b = tiles[blockIdx.x].x;
    const int64_t start = off[b] + (int64_t)tiles[blockIdx.x].y * TILE;
    const int64_t end = min(off[b + 1], start + TILE);
    const InspectIn B = bin[b];
    uint32_t err = 0;
    float mabs = 0.f;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = start + threadIdx.x; i < end; i += blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float o = orig[3 * i + d];
            if (!isfinite(o)) { err |= ERR_NONFINITE; continue; }
            mabs = fmaxf(mabs, fabsf(o));
            mn[d] = fminf(mn[d], o);
            mx[d] = fmaxf(mx[d], o);
            // periodic: within a quarter box of the box, so one +-L gives the minimum image
            if (B.periodic) {
                const double q = 0.25 * (B.hi[d] - B.lo[d]);
                if (!((double)o >= B.lo[d] - q && (double)o < B.hi[d] + q)) err |= ERR_OUTSIDE_BOX;
            }
            if (recon) {
                const float r = recon[3 * i + d];
                if (!isfinite(r)) { err |= ERR_NONFINITE; continue; }
                mabs = fmaxf(mabs, fabsf(r));
                if (fabs((double)r - (double)o) > B.xi) err |= ERR_BOUND;
            }
        }
    }
    // warp reductions then one atomic per warp into the block's record
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
        InspectDev *o = out + b;
        if (err) atomicOr(&o->err, err);
        atomicMax(&o->maxabs, ma);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            atomicMin(&o->lo[d], l[d]);
            atomicMax(&o->hi[d], h[d]);
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

void inspect_blocks(const float *orig, const float *recon, BlockSet &S, cudaStream_t s, HostScratch &hs) {
    const int nb = S.nb;
    std::vector<InspectIn> bin(nb);
    std::vector<int2> tiles;
    for (int b = 0; b < nb; ++b) {
        const pc_params *p = &S.prm[b];
        bin[b].xi = p->xi;
        bin[b].periodic = p->periodic;
        for (int d = 0; d < 3; ++d) {
            bin[b].lo[d] = p->box_lo[d];
            bin[b].hi[d] = p->box_hi[d];
        }
        const int64_t nt = cdiv(S.off[b + 1] - S.off[b], TILE);
        for (int64_t t = 0; t < nt; ++t) tiles.push_back(make_int2(b, (int)t));
    }
    // one staging area: offsets | per-block inputs | tiles | results
    const size_t b_off = (nb + 1) * sizeof(int64_t), b_in = nb * sizeof(InspectIn), b_t = tiles.size() * sizeof(int2),
                 b_out = nb * sizeof(InspectDev);
    uint8_t *h = (uint8_t *)host_scratch(hs, b_off + b_in + b_t + b_out);
    memcpy(h, S.off.data(), b_off);
    memcpy(h + b_off, bin.data(), b_in);
    memcpy(h + b_off + b_in, tiles.data(), b_t);
    InspectDev *init = (InspectDev *)(h + b_off + b_in + b_t);
    for (int b = 0; b < nb; ++b) {
        init[b].err = 0;
        init[b].maxabs = 0;
        for (int k = 0; k < 3; ++k) {
            init[b].lo[k] = 0xffffffffu;
            init[b].hi[k] = 0u;
        }
    }
    S.doff.alloc(nb + 1, s);
    DBuf<uint8_t> d(b_in + b_t + b_out, s);
    PC_CUDA(cudaMemcpyAsync(S.doff.p, h, b_off, cudaMemcpyHostToDevice, s));
    PC_CUDA(cudaMemcpyAsync(d.p, h + b_off, b_in + b_t + b_out, cudaMemcpyHostToDevice, s));
    InspectIn *din = (InspectIn *)d.p;
    int2 *dt = (int2 *)(d.p + b_in);
    InspectDev *dout = (InspectDev *)(d.p + b_in + b_t);
    if (!tiles.empty()) {
        k_inspect<<<(unsigned)tiles.size(), 256, 0, s>>>(orig, recon, dt, S.doff.p, din, dout);
        PC_CHECK_LAUNCH();
    }
    InspectDev *r = (InspectDev *)read_back(hs, dout, b_out, s);
    S.ins.assign(nb, Inspect());
    for (int b = 0; b < nb; ++b) {
        S.ins[b].err = r[b].err;
        uint32_t ma = r[b].maxabs;
        memcpy(&S.ins[b].maxabs, &ma, 4);
        for (int k = 0; k < 3; ++k) {
            S.ins[b].lo[k] = unord_f32(r[b].lo[k]);
            S.ins[b].hi[k] = unord_f32(r[b].hi[k]);
        }
    }
}

void setup_blocks(BlockSet &S, bool window, cudaStream_t s) {
    const int nb = S.nb;
    S.c.resize(nb);
    std::vector<BlockDev> h(nb);
    int64_t base = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t n = S.off[b + 1] - S.off[b];
        S.c[b] = make_consts(&S.prm[b], S.ins[b], n, window);
        const Consts &c = S.c[b];
        BlockDev &d = h[b];
        memset(&d, 0, sizeof(d));
        d.off = S.off[b];
        d.n = n;
        d.cell_base = base;
        for (int k = 0; k < 3; ++k) {
            d.origin[k] = (double)c.origin[k];
            d.inv_w[k] = (double)c.inv_w[k];
            d.L[k] = c.L[k];
            d.nc[k] = c.nc[k];
        }
        d.b2 = c.b2;
        d.lo2 = c.lo2;
        d.hi2 = c.hi2;
        d.periodic = c.periodic;
        d.mode = S.prm[b].mode;
        base += c.ncells;
    }
    if (base >= (int64_t)0xffffffffll) {
        set_error("too many grid cells for 32-bit cell keys (lower cell_cap_log2)");
        throw Fail{PC_EINVAL};
    }
    S.ncells = base;
    S.key_bits = std::max(1, ceil_log2((uint64_t)base));
    S.dev.alloc(nb, s);
    PC_CUDA(cudaMemcpyAsync(S.dev.p, h.data(), nb * sizeof(BlockDev), cudaMemcpyHostToDevice, s));
    PC_CUDA(cudaStreamSynchronize(s));   // h lives on this stack frame
}

// ======================================================================= binning
namespace {

__global__ void k_cell_keys(const float *__restrict__ orig, int64_t n, const BlockDev *__restrict__ bt,
                            const int64_t *__restrict__ off, int nb, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ ids) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const BlockDev &B = bt[find_block(off, nb, i)];
        const int nx = B.nc[0], ny = B.nc[1], nz = B.nc[2];
        int cx = (int)floor(((double)orig[3 * i + 0] - B.origin[0]) * B.inv_w[0]);
        int cy = (int)floor(((double)orig[3 * i + 1] - B.origin[1]) * B.inv_w[1]);
        int cz = (int)floor(((double)orig[3 * i + 2] - B.origin[2]) * B.inv_w[2]);
        if (B.periodic) {   // positions up to a quarter box outside wrap to their image's cell
            cx = cx < 0 ? cx + nx : (cx >= nx ? cx - nx : cx);
            cy = cy < 0 ? cy + ny : (cy >= ny ? cy - ny : cy);
            cz = cz < 0 ? cz + nz : (cz >= nz ? cz - nz : cz);
        }
        cx = min(max(cx, 0), nx - 1);
        cy = min(max(cy, 0), ny - 1);
        cz = min(max(cz, 0), nz - 1);
        keys[i] = (uint32_t)B.cell_base + ((uint32_t)cz * (uint32_t)ny + (uint32_t)cy) * (uint32_t)nx + (uint32_t)cx;
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

// cell_start[c] = first sorted position with key >= c, for c in [0, ncells].  A warp takes
// the 32 sorted positions k0 .. k0 + 31 (position n stands for key ncells) and writes the
// cells (key[k0 - 1], key[k0 + 31]] 32 consecutive cells at a time: cell c gets k0 plus
// the number of the warp's keys below c (a search over the lanes' keys), so the stores
// stay coalesced however unevenly the particles fill the cells.
__global__ void k_cell_bounds(const uint32_t *__restrict__ keys, int64_t n, int64_t ncells,
                              uint32_t *__restrict__ cell_start) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (n + 1 + 31) / 32;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wk < nwarps; wk += wstride) {
        const int64_t k0 = wk * 32, k = k0 + lane;
        const int64_t cur = k < n ? (int64_t)keys[k] : ncells;   // non-decreasing over the lanes
        const int64_t prev = k0 == 0 ? -1 : (int64_t)keys[k0 - 1];
        const int64_t last = __shfl_sync(FULL, cur, 31);
        for (int64_t c0 = prev + 1; c0 <= last; c0 += 32) {
            const int64_t c = c0 + lane;
            int below = 0;   // lanes whose key is below c (at most 31: the key of lane 31 is >= c)
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int64_t v = __shfl_sync(FULL, cur, below + step - 1);
                if (v < c) below += step;
            }
            if (c <= last) cell_start[c] = (uint32_t)(k0 + below);
        }
    }
}

inline int grid_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), (int64_t)num_sms() * 16));
}

}  // namespace

// Keys are ordered by block (cell bases increase with the block index), so after the
// stable sort the particles of block b occupy sorted positions [off_b, off_b + n_b).
void bin_particles(const float *orig, const BlockSet &S, Binned &B, cudaStream_t s, HostScratch &hs) {
    const int64_t n = S.n;
    B.n = n;
    B.keys.alloc(n, s);
    B.order.alloc(n, s);
    B.P4.alloc(n, s);
    B.cell_start.alloc(S.ncells + 1, s);
    k_cell_keys<<<grid_for(n), 256, 0, s>>>(orig, n, S.dev.p, S.doff.p, S.nb, B.keys.p, B.order.p);
    PC_CHECK_LAUNCH();
    radix_sort_u32(B.keys.p, B.order.p, n, S.key_bits, s);
    k_permute<<<grid_for(n), 256, 0, s>>>(orig, B.order.p, n, B.P4.p);
    PC_CHECK_LAUNCH();
    k_cell_bounds<<<grid_for(n + 1), 256, 0, s>>>(B.keys.p, n, S.ncells, B.cell_start.p);
    PC_CHECK_LAUNCH();
    const int32_t dc = S.prm.empty() ? 0 : S.prm[0].dense_cell;
    cell_maps(B, S, dc > 0 ? (uint32_t)dc : 0u, s, hs);
}

// ======================================================================= union-find
// Parent arrays keep par[x] <= x; the root of a set is its smallest id.
// A walk takes at most n steps; the cap only guards a broken invariant, and reaching it sets
// ERR_UF_RETRY in *err (the caller then fails with PC_ETIMEOUT instead of using the label).
__device__ __forceinline__ uint32_t uf_root(uint32_t *par, uint32_t x, uint32_t *err) {
    for (int it = 0; it < (1 << 26); ++it) {
        const uint32_t p = __ldcg(par + x);
        if (p == x) return x;
        const uint32_t g = __ldcg(par + p);
        if (g == p) return p;
        __stcg(par + x, g);   // path halving; g is an ancestor of x, so any interleaving is safe
        x = g;                // strictly decreasing: terminates
    }
    atomicOr(err, ERR_UF_RETRY);
    return x;
}

constexpr int UF_RETRY_CAP = 1 << 22;

__device__ __forceinline__ void uf_union(uint32_t *par, uint32_t a, uint32_t b, uint32_t *err) {
    for (int it = 0; it < UF_RETRY_CAP; ++it) {
        a = uf_root(par, a, err);
        b = uf_root(par, b, err);
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
__global__ void k_uf_flatten(uint32_t *par, int64_t n, uint32_t *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        (void)uf_root(par, (uint32_t)i, err);
}
__global__ void k_uf_labels(uint32_t *par, int64_t n, uint32_t *lab, uint32_t *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        lab[i] = uf_root(par, (uint32_t)i, err);
}
}  // namespace

void uf_init(uint32_t *par, int64_t n, cudaStream_t s) { iota_u32(par, n, s); }

// Rewrites par so every entry holds its root (two sweeps: path halving, then roots into a copy).
void uf_flatten(uint32_t *par, int64_t n, uint32_t *err, cudaStream_t s) {
    if (n <= 0) return;
    k_uf_flatten<<<grid_for(n), 256, 0, s>>>(par, n, err);
    PC_CHECK_LAUNCH();
    DBuf<uint32_t> lab(n, s);
    k_uf_labels<<<grid_for(n), 256, 0, s>>>(par, n, lab.p, err);
    PC_CHECK_LAUNCH();
    PC_CUDA(cudaMemcpyAsync(par, lab.p, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
}

// ======================================================================= pair search
// Every unordered pair within reach is classified exactly once, by one of two kernels:
//  * k_pairs_sparse: one thread per particle of a sparse cell (fewer than dense_min
//    particles) visits its own cell's later particles and the 13 forward neighbour cells
//    (lexicographically positive (dz, dy, dx)), skipping empty cells on an occupancy
//    bitmap (one bit per cell, small enough to stay in L2) and dense cells;
//  * k_pairs_dense: one warp per chunk of at most 32 particles of a dense cell (one per
//    lane) visits all 27 cells of the neighbourhood: the home cell (later particles), every
//    sparse neighbour, and the dense neighbours in forward directions.  Each neighbour
//    cell is staged in shared memory 32 particles at a time with coalesced float4 loads,
//    and every lane tests its particle against the staged ones (broadcast reads), so the
//    warp's lanes stay busy in dense halos.
// A pair of two sparse cells is visited from the backward cell, a pair with one dense
// cell by that cell's warps, a pair of two dense cells in the forward direction, and a
// pair inside one cell once (later particles only).
namespace {

struct PairArgs {
    unsigned long long *blk_counts;   // pass 1: per block links, safe, pb, pc (may be null)
    unsigned long long *V;            // pass 1: every vulnerable pair (may be null)
    uint64_t capV;
    uint32_t *fof_par, *safe_par;
    const uint32_t *fof_lab, *safe_lab;
    unsigned long long *A, *C;
    uint64_t capA, capC;
    unsigned long long *counts;
    uint32_t *err;
};

__device__ __forceinline__ void emit_pair(unsigned long long key, unsigned long long *out, uint64_t cap,
                                          unsigned long long *cnt, uint32_t *err, uint32_t full = ERR_INDEX) {
    // warp-aggregated reservation: one atomic per group of converged emitting lanes
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(cnt, (unsigned long long)g.size());
    base = g.shfl(base, 0);
    const unsigned long long pos = base + g.thread_rank();
    if (pos < cap) out[pos] = key;
    else atomicOr(err, full);
}

__device__ __forceinline__ unsigned long long pair_key(int64_t k, int64_t kj) {
    return k < kj ? (((unsigned long long)k << 32) | (unsigned long long)kj)
                  : (((unsigned long long)kj << 32) | (unsigned long long)k);
}

// Pass 1 keeps the vulnerable pairs through a buffer per warp in shared memory: a lane
// appends with a shared-memory atomic (no global contention however divergent the lanes
// are), and the warp moves the buffer to V with one global reservation whenever it is
// converged and the buffer is at least half full (and at its end).  A pair that finds the
// buffer full goes to V directly.
constexpr unsigned VBUF = 256;
struct WarpVBuf {
    unsigned long long *key;   // VBUF entries
    unsigned *cnt;
};

__device__ __forceinline__ void vbuf_push(const WarpVBuf &wb, unsigned long long key, const PairArgs &a) {
    const unsigned pos = atomicAdd(wb.cnt, 1u);
    if (pos < VBUF) wb.key[pos] = key;
    else emit_pair(key, a.V, a.capV, a.counts + CNT_V, a.err, ERR_VFULL);
}

// Called by all lanes of a converged warp.
__device__ __forceinline__ void vbuf_flush(const WarpVBuf &wb, bool force, const PairArgs &a) {
    const unsigned FULL = 0xffffffffu;
    __syncwarp();
    const unsigned c = *(volatile unsigned *)wb.cnt;
    if (c == 0 || (!force && c < VBUF / 2)) return;
    const unsigned m = min(c, VBUF);
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 0) base = atomicAdd(a.counts + CNT_V, (unsigned long long)m);
    base = __shfl_sync(FULL, base, 0);
    for (unsigned i = threadIdx.x & 31; i < m; i += 32) {
        if (base + i < a.capV) a.V[base + i] = wb.key[i];
        else atomicOr(a.err, ERR_VFULL);
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) *wb.cnt = 0u;
    __syncwarp();
}

// Home cell first, then the 13 forward neighbours (lexicographically positive (dz, dy, dx)).
__constant__ int c_off[14][3] = {{0, 0, 0},  {-1, -1, 1}, {0, -1, 1}, {1, -1, 1}, {-1, 0, 1},
                                 {0, 0, 1},  {1, 0, 1},   {-1, 1, 1}, {0, 1, 1},  {1, 1, 1},
                                 {-1, 1, 0}, {0, 1, 0},   {1, 1, 0},  {1, 0, 0}};

__device__ __forceinline__ bool cell_bit(const uint32_t *__restrict__ m, uint32_t c) {
    return (__ldg(m + (c >> 5)) >> (c & 31)) & 1u;
}

struct ClassCounts {
    uint32_t links = 0, safe = 0, pb = 0, pc = 0;
};

// One pair within reach (d2 <= hi2; sorted positions k, kj; particle ids id, jd), in one
// pass: pass 1 counts it by class and unites links (FoF) and safe links (safe
// components); pass 2 emits it by the block's mode (VP: every vulnerable pair; SC:
// vulnerable pairs between safe components; HF: created pairs between halos to A, broken
// links between safe components to the forest candidates C).
template <int PASS>
__device__ __forceinline__ void pair_action(float d2, int64_t k, int64_t kj, uint32_t id, uint32_t jd, float lo2,
                                            float b2, int mode, uint32_t my_safe, uint32_t my_fof,
                                            const PairArgs &a, ClassCounts &cn, const WarpVBuf &wb) {
    if (PASS == 1) {
        if (d2 <= lo2) {
            ++cn.safe;
            ++cn.links;
            if (a.safe_par) uf_union(a.safe_par, id, jd, a.err);
            if (a.fof_par) uf_union(a.fof_par, id, jd, a.err);
        } else {
            if (d2 <= b2) {
                ++cn.pb;
                ++cn.links;
                if (a.fof_par) uf_union(a.fof_par, id, jd, a.err);
            } else {
                ++cn.pc;
            }
            if (a.V) vbuf_push(wb, pair_key(k, kj), a);
        }
    } else {
        if (d2 <= lo2) return;   // safe link: never vulnerable
        const unsigned long long pk = pair_key(k, kj);
        if (mode == 0) {
            emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
        } else if (mode == 1) {
            if (a.safe_lab[jd] != my_safe) emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
        } else {
            if (d2 > b2) {
                if (a.fof_lab[jd] != my_fof) emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
            } else {
                if (a.safe_lab[jd] != my_safe) emit_pair(pk, a.C, a.capC, a.counts + CNT_C, a.err);
            }
        }
    }
}

// Pass 1 class counts of a warp: per block (one atomic per warp when the warp lies in one
// block) and in total.
__device__ __forceinline__ void flush_counts(ClassCounts cn, int bk, const PairArgs &a) {
    const unsigned FULL = 0xffffffffu;
    if (a.blk_counts) {
        int same = 0;
        __match_all_sync(FULL, bk, &same);
        if (!same) {
            if (bk >= 0) {
                unsigned long long *c = a.blk_counts + 4 * bk;
                if (cn.links) atomicAdd(c + 0, (unsigned long long)cn.links);
                if (cn.safe) atomicAdd(c + 1, (unsigned long long)cn.safe);
                if (cn.pb) atomicAdd(c + 2, (unsigned long long)cn.pb);
                if (cn.pc) atomicAdd(c + 3, (unsigned long long)cn.pc);
            }
        }
        const unsigned wl = __reduce_add_sync(FULL, cn.links), ws = __reduce_add_sync(FULL, cn.safe),
                       wp = __reduce_add_sync(FULL, cn.pb), wc = __reduce_add_sync(FULL, cn.pc);
        if (same && (threadIdx.x & 31) == 0 && bk >= 0) {
            unsigned long long *c = a.blk_counts + 4 * bk;
            if (wl) atomicAdd(c + 0, (unsigned long long)wl);
            if (ws) atomicAdd(c + 1, (unsigned long long)ws);
            if (wp) atomicAdd(c + 2, (unsigned long long)wp);
            if (wc) atomicAdd(c + 3, (unsigned long long)wc);
        }
    }
    const unsigned wl = __reduce_add_sync(FULL, cn.links), ws = __reduce_add_sync(FULL, cn.safe),
                   wp = __reduce_add_sync(FULL, cn.pb), wc = __reduce_add_sync(FULL, cn.pc);
    if ((threadIdx.x & 31) == 0) {
        if (wl) atomicAdd(a.counts + CNT_LINKS, (unsigned long long)wl);
        if (ws) atomicAdd(a.counts + CNT_SAFE, (unsigned long long)ws);
        if (wp) atomicAdd(a.counts + CNT_PB, (unsigned long long)wp);
        if (wc) atomicAdd(a.counts + CNT_PC, (unsigned long long)wc);
    }
}

// Cell coordinates of a sorted position's cell within its block's grid.
__device__ __forceinline__ void cell_xyz(uint32_t key, const BlockDev &B, int &cx, int &cy, int &cz) {
    const uint32_t l = key - (uint32_t)B.cell_base;
    cx = (int)(l % (uint32_t)B.nc[0]);
    cy = (int)((l / (uint32_t)B.nc[0]) % (uint32_t)B.nc[1]);
    cz = (int)(l / ((uint32_t)B.nc[0] * (uint32_t)B.nc[1]));
}

// Global index of the neighbour cell (cx + ox, cy + oy, cz + oz), or false when it does
// not exist: outside a non-periodic grid, or a step along a periodic axis of one cell
// (which has no distinct neighbour along it; periodic axes have one or at least 3 cells).
__device__ __forceinline__ bool neighbour(const BlockDev &B, int cx, int cy, int cz, int ox, int oy, int oz,
                                          uint32_t &cell) {
    const int nx = B.nc[0], ny = B.nc[1], nz = B.nc[2];
    int qx = cx + ox, qy = cy + oy, qz = cz + oz;
    if (B.periodic) {
        if ((nx == 1 && ox) || (ny == 1 && oy) || (nz == 1 && oz)) return false;
        qx = qx < 0 ? qx + nx : (qx >= nx ? qx - nx : qx);
        qy = qy < 0 ? qy + ny : (qy >= ny ? qy - ny : qy);
        qz = qz < 0 ? qz + nz : (qz >= nz ? qz - nz : qz);
    } else if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || qz < 0 || qz >= nz) {
        return false;
    }
    cell = (uint32_t)B.cell_base + ((uint32_t)qz * (uint32_t)ny + (uint32_t)qy) * (uint32_t)nx + (uint32_t)qx;
    return true;
}

template <int PASS>
__global__ void __launch_bounds__(256, 6) k_pairs_sparse(const float4 *__restrict__ P4, const uint32_t *__restrict__ keys,
                                                      const uint32_t *__restrict__ cell_start, int64_t n,
                                                      const BlockDev *__restrict__ bt, const int64_t *__restrict__ off,
                                                      int nb, CellMaps M, PairArgs a) {
    __shared__ unsigned long long vkey[PASS == 1 ? 8 : 1][PASS == 1 ? VBUF : 1];
    __shared__ unsigned vcnt[8];
    const int w = threadIdx.x >> 5;
    const WarpVBuf wb{vkey[PASS == 1 ? w : 0], vcnt + w};
    const bool keep = PASS == 1 && a.V != nullptr;
    if (keep && (threadIdx.x & 31) == 0) vcnt[w] = 0u;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    ClassCounts cn;
    const int bk = k < n ? find_block(off, nb, k) : -1;
    const bool act = k < n && !cell_bit(M.dense, keys[k]);
    const BlockDev &B = bt[act ? bk : 0];
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t id = 0, my_safe = 0, my_fof = 0;
    int cx = 0, cy = 0, cz = 0;
    if (act) {
        p = P4[k];
        id = __float_as_uint(p.w);
        cell_xyz(keys[k], B, cx, cy, cz);
        if (PASS == 2) {
            if (B.mode >= 1) my_safe = a.safe_lab[id];
            if (B.mode == 2) my_fof = a.fof_lab[id];
        }
    }
    const bool per = B.periodic != 0;
    const float lo2 = B.lo2, b2 = B.b2, hi2 = B.hi2;
    // every lane runs the 14 neighbour steps (a lane without a particle does nothing in
    // them), so the warp is converged after each step and may move its buffer of kept pairs
    for (int o = 0; o < 14; ++o) {
        uint32_t cell;
        if (act && neighbour(B, cx, cy, cz, c_off[o][0], c_off[o][1], c_off[o][2], cell) && cell_bit(M.occ, cell) &&
            (o == 0 || !cell_bit(M.dense, cell))) {   // a dense neighbour's warps take these pairs
            int64_t js = min((int64_t)cell_start[cell], n);
            const int64_t je = min((int64_t)cell_start[cell + 1], n);
            if (o == 0) js = k + 1;
            for (int64_t kj = js; kj < je; ++kj) {
                const float4 q = __ldg(P4 + kj);
                const float d2 = cdist2(cdiff(p.x, q.x, per, B.L[0]), cdiff(p.y, q.y, per, B.L[1]),
                                        cdiff(p.z, q.z, per, B.L[2]));
                if (d2 > hi2) continue;
                pair_action<PASS>(d2, k, kj, id, __float_as_uint(q.w), lo2, b2, B.mode, my_safe, my_fof, a, cn, wb);
            }
        }
        if (keep) vbuf_flush(wb, false, a);
    }
    if (keep) vbuf_flush(wb, true, a);
    if (PASS == 1) {
        __syncwarp();
        flush_counts(cn, bk, a);
    }
}

constexpr int DENSE_WARPS = 8;

template <int PASS>
__global__ void __launch_bounds__(32 * DENSE_WARPS) k_pairs_dense(
    const float4 *__restrict__ P4, const uint32_t *__restrict__ keys, const uint32_t *__restrict__ cell_start,
    int64_t n, const BlockDev *__restrict__ bt, const int64_t *__restrict__ off, int nb, CellMaps M,
    const DenseChunk *__restrict__ chunks, int64_t n_chunks, unsigned long long *work, PairArgs a) {
    __shared__ float4 tile[DENSE_WARPS][32];
    __shared__ unsigned long long vkey[PASS == 1 ? DENSE_WARPS : 1][PASS == 1 ? VBUF : 1];
    __shared__ unsigned vcnt[DENSE_WARPS];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const WarpVBuf wb{vkey[PASS == 1 ? w : 0], vcnt + w};
    const bool keep = PASS == 1 && a.V != nullptr;
    if (keep && lane == 0) vcnt[w] = 0u;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(work, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if ((int64_t)c >= n_chunks) break;
        const DenseChunk ch = chunks[c];
        const int bk = find_block(off, nb, (int64_t)ch.k0);
        const BlockDev &B = bt[bk];
        const int64_t ka = (int64_t)ch.k0 + lane;
        const bool va = lane < (int)ch.cnt;
        const float4 p = va ? P4[ka] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t id = __float_as_uint(p.w);
        int cx, cy, cz;
        cell_xyz(keys[ch.k0], B, cx, cy, cz);
        const bool per = B.periodic != 0;
        const float lo2 = B.lo2, b2 = B.b2, hi2 = B.hi2;
        uint32_t my_safe = 0, my_fof = 0;
        if (PASS == 2 && va) {
            if (B.mode >= 1) my_safe = a.safe_lab[id];
            if (B.mode == 2) my_fof = a.fof_lab[id];
        }
        ClassCounts cn;
        for (int o = 0; o < 27; ++o) {
            const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
            uint32_t cell;
            if (!neighbour(B, cx, cy, cz, ox, oy, oz, cell)) continue;
            if (!cell_bit(M.occ, cell)) continue;
            const bool home = (ox | oy | oz) == 0;
            const bool forward = oz > 0 || (oz == 0 && (oy > 0 || (oy == 0 && ox > 0)));
            if (!home && !forward && cell_bit(M.dense, cell)) continue;   // the other cell's warps take it
            const int64_t js = min((int64_t)cell_start[cell], n), je = min((int64_t)cell_start[cell + 1], n);
            for (int64_t base = js; base < je; base += 32) {
                // stage up to 32 particles of the neighbour cell (one coalesced float4 load)
                const int m = (int)min((int64_t)32, je - base);
                if (lane < m) tile[w][lane] = P4[base + lane];
                __syncwarp();
                for (int j = 0; j < m; ++j) {
                    const float4 q = tile[w][j];
                    const int64_t kj = base + j;
                    if (!va || (home && kj <= ka)) continue;
                    const float d2 = cdist2(cdiff(p.x, q.x, per, B.L[0]), cdiff(p.y, q.y, per, B.L[1]),
                                            cdiff(p.z, q.z, per, B.L[2]));
                    if (d2 > hi2) continue;
                    pair_action<PASS>(d2, ka, kj, id, __float_as_uint(q.w), lo2, b2, B.mode, my_safe, my_fof, a,
                                      cn, wb);
                }
                __syncwarp();
                if (keep) vbuf_flush(wb, false, a);
            }
        }
        if (PASS == 1) flush_counts(cn, bk, a);
    }
    if (keep) vbuf_flush(wb, true, a);
}

// Occupancy and density maps of the grid, and the dense cells cut into chunks of at
// most 32 particles: one thread per cell's first sorted particle.
__global__ void k_cell_maps(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ cell_start, int64_t n,
                            uint32_t dense_min, uint32_t *__restrict__ occ, uint32_t *__restrict__ dense,
                            DenseChunk *__restrict__ chunks, uint64_t cap, unsigned long long *n_chunks,
                            uint32_t *err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = keys[k];
        if (k > 0 && keys[k - 1] == c) continue;
        atomicOr(occ + (c >> 5), 1u << (c & 31));
        const uint32_t cnt = cell_start[c + 1] - (uint32_t)k;
        if (cnt < dense_min) continue;
        atomicOr(dense + (c >> 5), 1u << (c & 31));
        const uint32_t nch = (cnt + 31u) / 32u;
        const unsigned long long at = atomicAdd(n_chunks, (unsigned long long)nch);
        for (uint32_t j = 0; j < nch; ++j) {
            if (at + j < cap) chunks[at + j] = DenseChunk{(uint32_t)k + 32u * j, min(32u, cnt - 32u * j)};
            else atomicOr(err, ERR_INDEX);
        }
    }
}

}  // namespace

void cell_maps(Binned &B, const BlockSet &S, uint32_t dense_min, cudaStream_t s, HostScratch &hs) {
    const int64_t n = B.n;
    const int64_t words = (S.ncells + 32) / 32;
    B.occ.alloc(words, s);
    B.dense.alloc(words, s);
    PC_CUDA(cudaMemsetAsync(B.occ.p, 0, words * sizeof(uint32_t), s));
    PC_CUDA(cudaMemsetAsync(B.dense.p, 0, words * sizeof(uint32_t), s));
    // dense_min = 0: no dense cells (every particle is searched by its own thread)
    const uint64_t cap = dense_min ? (uint64_t)(n / std::max<uint32_t>(2, dense_min) + n / 32 + 1) : 1;
    B.chunks.alloc(cap, s);
    DBuf<unsigned long long> cnt(1, s);
    DBuf<uint32_t> err(1, s);
    PC_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s));
    PC_CUDA(cudaMemsetAsync(err.p, 0, sizeof(uint32_t), s));
    k_cell_maps<<<grid_for(n), 256, 0, s>>>(B.keys.p, B.cell_start.p, n,
                                            dense_min ? std::max<uint32_t>(2, dense_min) : 0xffffffffu, B.occ.p,
                                            B.dense.p, B.chunks.p, cap, cnt.p, err.p);
    PC_CHECK_LAUNCH();
    const unsigned long long *h = (const unsigned long long *)read_back(hs, cnt.p, sizeof(unsigned long long), s);
    B.n_chunks = (int64_t)*h;
    const uint32_t ev = *(const uint32_t *)read_back(hs, err.p, sizeof(uint32_t), s);
    if (ev & ERR_INDEX) fail(PC_ECUDA, "dense-cell chunk list overflowed its bound");
}

namespace {
// One vulnerable pair of pass 1 (key: sorted positions min << 32 | max) sent where pass 2
// would send it, by its block's mode; the squared distance is recomputed from the same
// rounded positions by the same expression (the difference is antisymmetric bit for bit).
__global__ void k_filter_v(const float4 *__restrict__ P4, const unsigned long long *__restrict__ V, uint64_t nV,
                           const BlockDev *__restrict__ bt, const int64_t *__restrict__ off, int nb,
                           const uint32_t *__restrict__ fof_lab, const uint32_t *__restrict__ safe_lab, PairArgs a) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nV;
         t += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long pk = V[t];
        const int64_t k = (int64_t)(pk >> 32), kj = (int64_t)(pk & 0xffffffffull);
        const BlockDev &B = bt[find_block(off, nb, k)];
        if (B.mode == 0) {
            emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
            continue;
        }
        const float4 p = P4[k], q = P4[kj];
        const uint32_t id = __float_as_uint(p.w), jd = __float_as_uint(q.w);
        if (B.mode == 1) {
            if (safe_lab[id] != safe_lab[jd]) emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
            continue;
        }
        const bool per = B.periodic != 0;
        const float d2 = cdist2(cdiff(p.x, q.x, per, B.L[0]), cdiff(p.y, q.y, per, B.L[1]), cdiff(p.z, q.z, per, B.L[2]));
        if (d2 > B.b2) {
            if (fof_lab[id] != fof_lab[jd]) emit_pair(pk, a.A, a.capA, a.counts + CNT_A, a.err);
        } else {
            if (safe_lab[id] != safe_lab[jd]) emit_pair(pk, a.C, a.capC, a.counts + CNT_C, a.err);
        }
    }
}

template <int PASS>
void run_pair_pass(const Binned &B, const BlockSet &S, const PairArgs &a, cudaStream_t s) {
    const int64_t n = B.n;
    const CellMaps M{B.occ.p, B.dense.p};
    k_pairs_sparse<PASS><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(B.P4.p, B.keys.p, B.cell_start.p, n, S.dev.p,
                                                               S.doff.p, S.nb, M, a);
    PC_CHECK_LAUNCH();
    if (B.n_chunks > 0) {
        DBuf<unsigned long long> work(1, s);
        PC_CUDA(cudaMemsetAsync(work.p, 0, sizeof(unsigned long long), s));
        const int grid = (int)std::min<int64_t>(cdiv(B.n_chunks, DENSE_WARPS), (int64_t)num_sms() * 8);
        k_pairs_dense<PASS><<<grid, 32 * DENSE_WARPS, 0, s>>>(B.P4.p, B.keys.p, B.cell_start.p, n, S.dev.p, S.doff.p,
                                                             S.nb, M, B.chunks.p, B.n_chunks, work.p, a);
        PC_CHECK_LAUNCH();
    }
}
}  // namespace

void pair_pass_union(const Binned &B, const BlockSet &S, uint32_t *fof_par, uint32_t *safe_par,
                     unsigned long long *counts, uint32_t *err, cudaStream_t s, unsigned long long *blk_counts,
                     unsigned long long *V, uint64_t capV) {
    PairArgs a = {};
    a.blk_counts = blk_counts;
    a.V = V;
    a.capV = capV;
    a.fof_par = fof_par;
    a.safe_par = safe_par;
    a.counts = counts;
    a.err = err;
    run_pair_pass<1>(B, S, a, s);
}

void pair_pass_emit(const Binned &B, const BlockSet &S, const uint32_t *fof_lab, const uint32_t *safe_lab,
                    unsigned long long *A, uint64_t capA, unsigned long long *C, uint64_t capC,
                    unsigned long long *counts, uint32_t *err, cudaStream_t s) {
    PairArgs a = {};
    a.fof_lab = fof_lab;
    a.safe_lab = safe_lab;
    a.A = A;
    a.C = C;
    a.capA = capA;
    a.capC = capC;
    a.counts = counts;
    a.err = err;
    run_pair_pass<2>(B, S, a, s);
}

void filter_vulnerable(const Binned &B, const BlockSet &S, const uint32_t *fof_lab, const uint32_t *safe_lab,
                       const unsigned long long *V, uint64_t nV, unsigned long long *A, uint64_t capA,
                       unsigned long long *C, uint64_t capC, unsigned long long *counts, uint32_t *err,
                       cudaStream_t s) {
    if (nV == 0) return;
    PairArgs a = {};
    a.A = A;
    a.C = C;
    a.capA = capA;
    a.capC = capC;
    a.counts = counts;
    a.err = err;
    k_filter_v<<<grid_for((int64_t)nV), 256, 0, s>>>(B.P4.p, V, nV, S.dev.p, S.doff.p, S.nb, fof_lab, safe_lab, a);
    PC_CHECK_LAUNCH();
}

}  // namespace pc
