// Host-side interfaces between the translation units of libpc (internal).
#pragma once

#include <vector>

#include "common.cuh"

namespace pc {

// ---------------------------------------------------------------- inputs
struct Inspect {
    uint32_t err = 0;      // ERR_* bits
    float maxabs = 0.f;    // max |coordinate| over orig and recon
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // bounding box of orig
};

// Derived constants; `window` = false sizes the grid for links only (FoF labels).
Consts make_consts(const pc_params *p, const Inspect &ins, int64_t n, bool window);

// ---------------------------------------------------------------- blocks
// A problem set is one or more independent blocks of particles, concatenated:
// block b owns ids (and, after binning, sorted positions) [off_b, off_b + n_b).
// Every kernel finds the block of an index by binary search over the offsets and
// reads that block's constants from the device table; blocks never interact.
struct BlockDev {
    int64_t off, n, cell_base;   // particle range; first global cell of the block's grid
    double origin[3], inv_w[3];  // grid
    float b2, lo2, hi2, L[3];    // link-test bounds, periodic lengths
    int nc[3];
    int periodic, mode;
};

__device__ __forceinline__ int find_block(const int64_t *__restrict__ off, int nb, int64_t i) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct BlockSet {
    int nb = 0;
    int64_t n = 0;                   // all particles
    std::vector<pc_params> prm;      // per block
    std::vector<int64_t> off;        // nb + 1 offsets
    std::vector<Inspect> ins;
    std::vector<Consts> c;
    int64_t ncells = 0;              // all blocks' cells
    int key_bits = 0;
    DBuf<BlockDev> dev;              // nb entries
    DBuf<int64_t> doff;              // nb + 1 offsets
    void release_to_default_stream() {
        dev.s = 0;
        doff.s = 0;
    }
};
// Per-block validation and statistics (finiteness, |recon - orig| <= xi in float64,
// periodic boxes, max |coordinate|, bounding box); recon may be null.  Uploads the
// offsets.  Synchronises the stream.
void inspect_blocks(const float *orig, const float *recon, BlockSet &S, cudaStream_t s, HostScratch &hs);
// Per-block constants (window or links only), global cell bases, device table.
void setup_blocks(BlockSet &S, bool window, cudaStream_t s);

// ---------------------------------------------------------------- binning
// Sorted positions [k0, k0 + cnt) of one dense cell, cnt <= 32 (one warp of the pair search).
struct DenseChunk {
    uint32_t k0, cnt;
};
// Bitmaps over the cells of a binning: occupied cells, and dense cells (at least dense_min
// particles, whose pairs one warp per chunk searches).
struct CellMaps {
    const uint32_t *occ, *dense;
};
struct Binned {
    int64_t n = 0;
    DBuf<uint32_t> keys;        // sorted cell keys (block cell base + local cell)
    DBuf<uint32_t> order;       // sorted position -> particle id
    DBuf<float4> P4;            // sorted original positions, w = id bits
    DBuf<uint32_t> cell_start;  // ncells + 1
    DBuf<uint32_t> occ, dense;  // one bit per cell
    DBuf<DenseChunk> chunks;    // the dense cells in chunks of at most 32 particles
    int64_t n_chunks = 0;
    void release_to_default_stream() {
        keys.s = 0;
        order.s = 0;
        P4.s = 0;
        cell_start.s = 0;
        occ.s = 0;
        dense.s = 0;
        chunks.s = 0;
    }
};
// Binning and the cell maps of the pair search (dense_min from the first block's
// dense_cell parameter; 0, the default, makes no cell dense).
void bin_particles(const float *orig, const BlockSet &S, Binned &B, cudaStream_t s, HostScratch &hs);
void cell_maps(Binned &B, const BlockSet &S, uint32_t dense_min, cudaStream_t s, HostScratch &hs);

// ---------------------------------------------------------------- pair search
enum { CNT_LINKS = 0, CNT_SAFE = 1, CNT_PB = 2, CNT_PC = 3, CNT_A = 4, CNT_C = 5, CNT_V = 6, CNT_N = 8 };

// Capacity of the count pass's buffer of vulnerable pairs: 16 per particle covers the
// workloads at xi <= 0.5 b; a denser problem overflows it and runs the emission pass.
inline int64_t vulnerable_guess(int64_t n) { return std::max<int64_t>(1 << 16, 16 * n); }
// Pass 1: union-find over links (fof_par) and safe links (safe_par), class counts; with V,
// every vulnerable pair is also written to V (counted in CNT_V; ERR_VFULL when capV is
// too small, and the emission pass must run).
void pair_pass_union(const Binned &B, const BlockSet &S, uint32_t *fof_par, uint32_t *safe_par,
                     unsigned long long *counts, uint32_t *err, cudaStream_t s,
                     unsigned long long *blk_counts = nullptr, unsigned long long *V = nullptr,
                     uint64_t capV = 0);
// The selection of pass 2 taken from the vulnerable pairs V of pass 1 instead of a second
// search: the same pairs to A and C, by each block's mode.
void filter_vulnerable(const Binned &B, const BlockSet &S, const uint32_t *fof_lab, const uint32_t *safe_lab,
                       const unsigned long long *V, uint64_t nV, unsigned long long *A, uint64_t capA,
                       unsigned long long *C, uint64_t capC, unsigned long long *counts, uint32_t *err,
                       cudaStream_t s);
// Pass 2: emission of selected pairs as (min_pos << 32 | max_pos), by each block's mode:
//   VP: all vulnerable pairs -> A;  SC: vulnerable pairs joining different safe components -> A;
//   HF: potentially created pairs joining different halos -> A, potentially broken links
//       joining different safe components -> C (spanning-forest candidates).
void pair_pass_emit(const Binned &B, const BlockSet &S, const uint32_t *fof_lab, const uint32_t *safe_lab,
                    unsigned long long *A, uint64_t capA, unsigned long long *C, uint64_t capC,
                    unsigned long long *counts, uint32_t *err, cudaStream_t s);
// Union-find helpers (labels = smallest id of the set)
void uf_init(uint32_t *par, int64_t n, cudaStream_t s);
// Rewrites par so every entry holds its root; a root walk that exceeds its bound sets
// ERR_UF_RETRY in *err (device).
void uf_flatten(uint32_t *par, int64_t n, uint32_t *err, cudaStream_t s);

// ---------------------------------------------------------------- selection (select.cu)
// HF spanning forest: Boruvka on safe-component supernodes over candidate links C
// (key: float32 bits of d2, then (i, j) ids).  Appends the forest links to A
// (positions) starting at *nA; returns the number of forest links.
int64_t halo_forest(const Binned &B, const BlockSet &S, const uint32_t *safe_lab, const unsigned long long *C,
                    int64_t nC, unsigned long long *A, int64_t nA, uint32_t *err, cudaStream_t s,
                    HostScratch &hs);
// Canonical export: (i, j) ids with i < j sorted by (i, j), and the link flag.
void export_pairs(const Binned &B, const BlockSet &S, const unsigned long long *A, int64_t nA, uint32_t *i_out,
                  uint32_t *j_out, uint8_t *link_out, cudaStream_t s);

// ---------------------------------------------------------------- PGD (pgd.cu)
struct PgdResult {       // per block
    int64_t iters = 0, loss_evals = 0, viol0 = 0, viol_final = 0, n_editable = 0;
    double loss0 = 0, loss_final = 0;
    bool converged = false;
    int64_t resets = 0;        // checks that triggered a stall reset
    int64_t row_updates = 0;   // Adam steps applied, summed over the updates
    int64_t pair_evals = 0;    // pairs evaluated in double-float (both directions), summed over the checks
};
struct PgdRun {
    std::vector<PgdResult> blocks;
    double ms = 0;        // iterations + output
    double ms_iter = 0;   // iteration launches only
    double ms_csr = 0;    // CSR and state build
    int64_t launches = 0;
};
// Several linking lengths enforced together in one single-block problem (the union of
// the pairs each selects, Sec. 1 and Sec. 5): the index of each active pair's linking
// length and the constants of every length (at most 4, ascending).
struct ThrSet {
    const uint8_t *Athr = nullptr;   // device, one entry per active pair
    std::vector<Consts> c;
};

// Resumable PGD over every block of a set (Algorithm 1, the loop).  The constructor
// builds E, the CSR of A and the iteration state on stream s (it synchronises s a few
// times); launch() enqueues iteration launches, replaying a captured CUDA graph when
// capture() was called; each block stops on its own check (its later launches return
// at once), so launching past a stop is harmless.  The history outputs require a
// single block.  Not thread safe; every call works on stream s.
class PgdSolver {
  public:
    PgdSolver(const Binned &B, const BlockSet &S, const std::vector<Consts> &cp, const float *orig,
              const float *recon, const unsigned long long *A, int64_t nA, cudaStream_t s, HostScratch &hs,
              double *hist_loss = nullptr, unsigned long long *hist_viol = nullptr, const ThrSet *thr = nullptr);
    ~PgdSolver();
    PgdSolver(const PgdSolver &) = delete;
    PgdSolver &operator=(const PgdSolver &) = delete;
    bool empty() const;                 // no active pair in any block
    int64_t rows() const;               // |E| over all blocks
    int64_t max_launches() const;       // launches after which every block has stopped
    void capture(int k);                // capture k iteration launches into a graph
    int64_t launch(int k);              // enqueue >= k launches (whole graphs when captured); returns the count
    void post_status();                 // enqueue a copy of the stop flags to pinned memory
    bool status_ready() const;          // that copy has landed
    void wait_status() const;
    bool all_stopped() const;           // from the last landed copy
    bool block_stopped(int b) const;
    int64_t active_rows() const;        // rows of the blocks not stopped, from the last landed copy
    void output(float *corrected, int b = -1);   // P + delta of the final buffer: every block, or block b
    void delta_out(double *delta);
    void results(std::vector<PgdResult> &out);   // per block; synchronises
    void block_result(int b, PgdResult &r) const;  // block b, from the last landed status copy
    int64_t launches = 0;
  private:
    struct Impl;
    Impl *im;
};

// PGD for every block of the set; `cp` holds each block's PGD constants (built from
// orig and recon).  The history outputs require a single block.  graph_k > 0 runs the
// iterations as replays of a CUDA graph of graph_k launches.
PgdRun run_pgd(const Binned &B, const BlockSet &S, const std::vector<Consts> &cp, const float *orig,
               const float *recon, const unsigned long long *A, int64_t nA, float *corrected, cudaStream_t s,
               HostScratch &hs, double *delta_out = nullptr, double *hist_loss = nullptr,
               unsigned long long *hist_viol = nullptr, int graph_k = 0, const ThrSet *thr = nullptr);

// ---------------------------------------------------------------- selection (api.cu)
int ctx_device(const pc_ctx *ctx);
void fail(pc_status st, const std::string &msg);                 // set_error + throw
void check_params(const pc_params *p, int64_t n, bool need_pgd);  // PC_EINVAL on bad parameters
void check_inspect(const Inspect &ins);                           // PC_EINVAL / PC_EBOUND on bad input
void check_block_inputs(const BlockSet &S);                       // the same, naming the block
Consts make_consts(const pc_params *p, const Inspect &ins, int64_t n, bool window);

// Selected constraints of a block set, resident on the device.
struct Selection {
    BlockSet S;
    Binned B;
    DBuf<unsigned long long> A;           // active pairs (min_pos << 32 | max_pos)
    int64_t nA = 0;
    std::vector<pc_select_stats> stats;   // per block
    // between the count and the emission passes
    DBuf<unsigned long long> counts, bc;
    DBuf<uint32_t> err, fof, safe;
    DBuf<unsigned long long> V;           // the vulnerable pairs of pass 1 (empty when they overflowed)
    unsigned long long cnt[CNT_N] = {};
    bool any_fof = false, any_safe = false;
    cudaEvent_t ev0 = nullptr;
    ~Selection() {
        if (ev0) cudaEventDestroy(ev0);
    }
};
// Count pass (binning, pass 1 of the pair search): S.prm and S.off must be set.
void select_count(HostScratch &hs, const float *orig, cudaStream_t s, Selection &h);
// Device bytes that select_emit and the PGD state will add (upper estimate from the counts).
int64_t select_more_bytes(const Selection &h);
// Emission pass, halo forest, per-block statistics; releases the count-pass temporaries.
void select_emit(HostScratch &hs, cudaStream_t s, Selection &h);

// Several linking lengths (select.cu): inv[order[p]] = p for a binning, and the pairs of
// another binning's selection (positions, key min << 32 | max) as positions of the binning
// whose inverse is inv, each with the linking-length index t.
void inverse_order(const Binned &B, uint32_t *inv, cudaStream_t s);
void remap_pairs(const unsigned long long *A, int64_t m, const uint32_t *order_k, const uint32_t *inv, uint8_t t,
                 unsigned long long *out, uint8_t *tout, cudaStream_t s);

// Edit stream (edits.cu)
size_t encode_edits(const float *recon, const float *corr, int64_t n, const pc_params *p, uint8_t *out, size_t cap,
                    cudaStream_t s, HostScratch &hs);

// ---------------------------------------------------------------- host scratch
void *host_scratch(HostScratch &hs, size_t bytes);
// Copy `bytes` from device to pinned host scratch and wait.
void *read_back(HostScratch &hs, const void *dev, size_t bytes, cudaStream_t s);

}  // namespace pc
