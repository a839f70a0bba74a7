// Host-side interfaces between the translation units of libpc (internal).
#pragma once

#include "common.cuh"

namespace pc {

// ---------------------------------------------------------------- inputs
struct Inspect {
    uint32_t err = 0;      // ERR_* bits
    float maxabs = 0.f;    // max |coordinate| over orig and recon
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // bounding box of orig
};
// Validates finiteness, |recon - orig| <= xi (float64 compare) and the periodic box;
// recon may be null (labels only).  Synchronises the stream.
Inspect inspect_inputs(const float *orig, const float *recon, int64_t n, const pc_params *p,
                       cudaStream_t s, HostScratch &hs);

// Derived constants; `window` = false sizes the grid for links only (FoF labels).
Consts make_consts(const pc_params *p, const Inspect &ins, int64_t n, bool window);

// ---------------------------------------------------------------- binning
constexpr int CHUNK = 128;   // particles of one home cell handled by one CTA
struct Binned {
    int64_t n = 0;
    DBuf<uint32_t> keys;        // sorted cell keys
    DBuf<uint32_t> order;       // sorted position -> particle id
    DBuf<float4> P4;            // sorted original positions, w = id bits
    DBuf<uint32_t> cell_start;  // ncells + 1
    DBuf<uint32_t> items;       // first sorted position of each home chunk
    int64_t n_items = 0;
};
void bin_particles(const float *orig, int64_t n, const Consts &c, Binned &B, cudaStream_t s, HostScratch &hs);

// ---------------------------------------------------------------- pair search
enum { CNT_LINKS = 0, CNT_SAFE = 1, CNT_PB = 2, CNT_PC = 3, CNT_A = 4, CNT_C = 5, CNT_N = 8 };
// Pass 1: union-find over links (fof_par) and safe links (safe_par), class counts.
void pair_pass_union(const Binned &B, const Consts &c, uint32_t *fof_par, uint32_t *safe_par,
                     unsigned long long *counts, uint32_t *err, cudaStream_t s);
// Pass 2: emission of selected pairs as (min_pos << 32 | max_pos):
//   VP: all vulnerable pairs -> A;  SC: vulnerable pairs joining different safe components -> A;
//   HF: potentially created pairs joining different halos -> A, potentially broken links
//       joining different safe components -> C (spanning-forest candidates).
void pair_pass_emit(const Binned &B, const Consts &c, int mode, const uint32_t *fof_lab,
                    const uint32_t *safe_lab, unsigned long long *A, uint64_t capA, unsigned long long *C,
                    uint64_t capC, unsigned long long *counts, uint32_t *err, cudaStream_t s);
// Union-find helpers (labels = smallest id of the set)
void uf_init(uint32_t *par, int64_t n, cudaStream_t s);
void uf_flatten(uint32_t *par, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------- selection (select.cu)
// HF spanning forest: Boruvka on safe-component supernodes over candidate links C
// (key: float32 bits of d2, then (i, j) ids).  Appends the forest links to A
// (positions) starting at *nA; returns the number of forest links.
int64_t halo_forest(const Binned &B, const Consts &c, const uint32_t *safe_lab, const unsigned long long *C,
                    int64_t nC, unsigned long long *A, int64_t nA, uint32_t *err, cudaStream_t s,
                    HostScratch &hs);
// Canonical export: (i, j) ids with i < j sorted by (i, j), and the link flag.
void export_pairs(const Binned &B, const Consts &c, const unsigned long long *A, int64_t nA, uint32_t *i_out,
                  uint32_t *j_out, uint8_t *link_out, cudaStream_t s);

// ---------------------------------------------------------------- PGD (pgd.cu)
struct PgdResult {
    int64_t iters = 0, loss_evals = 0, viol0 = 0, viol_final = 0, n_editable = 0;
    double loss0 = 0, loss_final = 0;
    bool converged = false;
    double ms = 0;        // iterations + output
    double ms_iter = 0;   // iteration launches only
    int64_t launches = 0;
};
PgdResult run_pgd(const Binned &B, const Consts &c, const pc_params *p, const float *orig, const float *recon,
                  const unsigned long long *A, int64_t nA, float *corrected, cudaStream_t s, HostScratch &hs,
                  double *ms_csr, double *delta_out = nullptr, double *hist_loss = nullptr,
                  unsigned long long *hist_viol = nullptr);

// ---------------------------------------------------------------- host scratch
void *host_scratch(HostScratch &hs, size_t bytes);
// Copy `bytes` from device to pinned host scratch and wait.
void *read_back(HostScratch &hs, const void *dev, size_t bytes, cudaStream_t s);

}  // namespace pc
