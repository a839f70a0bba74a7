/*
 * pc.h -- C ABI of the GB300 cluster-preserving correction pass.
 *
 * Method: arXiv 2604.18801, "Preserving Clusters in Error-Bounded Lossy
 * Compression of Scientific Particle Data".  Given original particle
 * coordinates P, a lossy reconstruction P0 with |P0 - P| <= xi per coordinate,
 * a linking length b and the bound xi, the pass
 *   1. finds friends-of-friends links d <= b and the vulnerable pairs whose
 *      distance lies in (b - 2 sqrt3 xi, b + 2 sqrt3 xi]          (Sec. 2.4, 3.1)
 *   2. labels connected components (union-find)                 (Sec. 2.4)
 *   3. selects active pairs in mode VP, SC or HF                  (Sec. 3.2)
 *   4. runs projected gradient descent (Adam) on the tightened loss of Eq. 3
 *      with every editable coordinate kept within the box         (Alg. 1, Eq. 2-3)
 *   5. encodes the edits as flags + m-bit codes and decodes them  (Sec. 3.3)
 *
 * Conventions for every entry point
 *   - Coordinates are float32, N x 3, C-contiguous (x, y, z per particle).
 *     Pointers named *_dev are CUDA device pointers owned by the caller.
 *   - Calls are issued on the caller's stream.  Entry points that must learn a
 *     size on the device (pair counts, flagged counts) synchronise that stream
 *     before returning; their outputs are complete when they return.
 *   - Negative return codes are errors: outputs are then unspecified and no
 *     library state leaks.  Positive codes are warnings with valid outputs.
 *     pc_last_error() gives a thread-local message for the last failure.
 *   - Link tests use the canonical float32 formula on the original
 *     coordinates: dx = xi - xj in float32, minimum image (periodic boxes) by
 *     one add or subtract of the box length when |dx| > L/2, then
 *     d2 = (dx*dx + dy*dy) + dz*dz rounded per operation (no fused
 *     multiply-add); linked iff d2 <= fl32(b*b).
 *   - The library never allocates with the host heap on the data path; device
 *     temporaries come from the stream-ordered pool of the context's device.
 *   - Particle ids are the row indices 0..N-1; N < 2^31.
 *   - A context keeps pinned host scratch that most calls share: issue calls on one
 *     context from one thread at a time (use one context per thread).  The lossless
 *     calls and pc_cluster_metrics use scratch of their own, and the pc_serve_* calls
 *     are thread safe.
 */
#ifndef PC_H_
#define PC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PC_OK = 0,
    PC_WARN_NOT_CONVERGED = 1, /* PGD hit t_max with violations left; output valid and in the box */
    PC_EINVAL = -1,            /* bad argument: NaN/Inf, n < 2, b <= 0, xi < 0, m outside [2,32], bad box */
    PC_EBOUND = -2,            /* some |recon - orig| > xi: the base compressor broke its bound */
    PC_ENOMEM = -3,            /* device or pinned-host allocation failed */
    PC_ECUDA = -4,             /* a CUDA call failed (message in pc_last_error) */
    PC_EFORMAT = -5,           /* malformed edit stream */
    PC_ETIMEOUT = -6,          /* a bounded device-side wait or retry loop gave up */
    PC_EBUSY = -7              /* server full / ticket unknown */
} pc_status;

typedef enum { PC_MODE_VP = 0, PC_MODE_SC = 1, PC_MODE_HF = 2 } pc_mode;

/* Parameters: the REQUIRE line of Algorithm 1 plus the Adam moments (Sec. 4.2). */
typedef struct {
    double b;              /* linking length b > 0                                        */
    double xi;             /* pointwise bound xi >= 0 (error of the base compressor)       */
    double box_lo[3];      /* periodic boxes: [box_lo, box_hi) per axis; ignored otherwise */
    double box_hi[3];
    int32_t periodic;      /* 1: minimum-image distances; coordinates must lie within a
                              quarter box length of [box_lo, box_hi) (one +-L gives the image) */
    int32_t mode;          /* pc_mode                                                     */
    int32_t m_bits;        /* edit bit depth m in [2, 32] (default 16, Sec. 3.3)            */
    int32_t t_max;         /* maximum number of PGD updates (default 10000)                */
    double alpha_rel;      /* Adam step size in units of xi: alpha = alpha_rel * xi         */
    double beta1, beta2;   /* Adam moments (0.9, 0.999)                                    */
    double eps_rel;        /* Adam epsilon in units of xi (1e-8)                           */
    double loss_tol;       /* eps_L: stop when the tight loss <= loss_tol; 0 (default):
                              stop when no active pair is violated by more than b 2^-40  */
    int32_t replay_iters;  /* >= 0: run exactly this many updates, ignore the loss (-1 off) */
    int32_t cell_cap_log2; /* tuning: at most 2^cell_cap_log2 grid cells (0: cell_factor)    */
    int32_t stall_patience;/* stall reset (not in the paper; 0 = off): after this many checks
                              without progress (doubled after every reset), the next check
                              puts every editable endpoint of a violated pair back at its
                              original position (when the violated pairs' RMS violation
                              exceeds xi / 1024) with cleared
                              Adam moments.  Progress: the loss in units of xi^2 2^-24,
                              summed per violated pair after rounding to an integer, is
                              below best - floor(best / 1024) (best: the lowest so far).  */
    int32_t cell_factor;   /* tuning: at most cell_factor * n grid cells, within [2^16, 2^28]
                              (0 = 8); cells are never smaller than the pair reach.  Only
                              speed depends on it (pc_autotune_cells picks one).          */
    int32_t dense_cell;    /* tuning: grid cells holding at least this many particles are
                              searched by one warp per 32 of their particles, the others by
                              one thread per particle (0 = no such cells).  Only speed
                              depends on it.                                              */
    int32_t screen_chunk;  /* tuning: the PGD screen of a single problem walks its light work
                              items in chunks of at most this many pairs (0 = 1024).  Only
                              speed depends on it.                                        */
} pc_params;

/* Fills defaults: m=16, t_max=10000, alpha_rel=0.2, beta=(0.9,0.999), eps_rel=2e-6,
 * loss_tol=0, replay_iters=-1, cell_cap_log2=0, stall_patience=0 (Algorithm 1 as printed), cell_factor=0,
 * dense_cell=0, screen_chunk=0,
 * unit box, non-periodic, mode VP. */
void pc_params_default(pc_params *p);

typedef struct pc_ctx pc_ctx;
typedef struct pc_constraints pc_constraints;

/* Context on one CUDA device (made current by every call that takes it).
 * arena_bytes: bytes kept in the device pool between calls (0 = keep everything). */
pc_status pc_ctx_create(int device, size_t arena_bytes, pc_ctx **out);
void pc_ctx_destroy(pc_ctx *ctx);

/* Thread-local message of the last failing call ("" if none). */
const char *pc_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all threads). */
uint64_t pc_kernel_launches(void);

/* Friends-of-friends labels (Sec. 2.4): labels_dev[i] = smallest id in i's
 * component of the graph d2 <= b2 (canonical float32 test).  Only b, periodic and
 * the box of params are used.  n_comp (host, may be NULL) receives the number of
 * components.  Synchronises the stream. */
pc_status pc_fof_labels(pc_ctx *ctx, const float *xyz_dev, int64_t n, const pc_params *params,
                        int32_t *labels_dev, int64_t *n_comp, void *stream);

typedef struct {
    int64_t n_links;       /* pairs with d2 <= b2                      */
    int64_t n_safe;        /* safe links d2 <= lo2                     */
    int64_t n_pb;          /* potentially broken: lo2 < d2 <= b2       */
    int64_t n_pc;          /* potentially created: b2 < d2 <= hi2      */
    int64_t n_vulnerable;  /* |V| = n_pb + n_pc                        */
    int64_t n_active;      /* |A| of the selected mode                  */
    int64_t n_active_links;/* active pairs that are original links     */
    int64_t n_halos;       /* FoF components (SC/HF modes; 0 for VP)   */
    int64_t n_safe_comps;  /* safe components (SC/HF modes; 0 for VP)  */
    int64_t n_forest;      /* HF: spanning-forest links kept           */
    double ms;             /* device time of the selection             */
} pc_select_stats;

/* Constraint selection (Sec. 3.2): V, then A for params->mode.  The handle owns
 * device memory of the context's device and is freed with pc_constraints_free.
 * Synchronises the stream. */
pc_status pc_select_constraints(pc_ctx *ctx, const float *orig_dev, int64_t n, const pc_params *params,
                                pc_constraints **out, pc_select_stats *stats, void *stream);

/* Copies the active pairs, canonical order (i < j, sorted by (i, j)), into caller
 * buffers (host or device; each of length >= n_active; link_out may be NULL).
 * link_out[k] = 1 iff the pair is an original link.  Synchronises the stream. */
pc_status pc_constraints_copy(pc_ctx *ctx, const pc_constraints *c, uint32_t *i_out, uint32_t *j_out,
                              uint8_t *link_out, void *stream);
void pc_constraints_free(pc_constraints *c);

typedef struct {
    int64_t iters;         /* T: PGD updates performed                          */
    int64_t loss_evals;    /* tight-loss evaluations (T + 1)                     */
    int64_t viol0;         /* violated active pairs before the first update      */
    int64_t viol_final;    /* violated active pairs at the end (0 if converged)  */
    double loss0, loss_final;
    int64_t n_vulnerable, n_active, n_editable;
    int32_t converged;
    int32_t pad_;
    double ms_setup;       /* binning + pair search + selection + CSR build      */
    double ms_pgd;         /* PGD loop including the output kernels              */
    double ms_pgd_iter;    /* device time of the iteration launches alone        */
    int64_t pgd_launches;  /* iteration kernels launched (>= loss_evals; launches
                              after the stop return at once)                    */
    int64_t resets;        /* stall resets that fired (0 when stall_patience = 0) */
    int64_t row_updates;   /* Adam steps applied to editable particles, summed over
                              the updates (rows with neither a gradient so far nor
                              a projection to do are left as they are)          */
    int64_t pair_evals;    /* active pairs the float32 screen could not certify,
                              evaluated in double-float, summed over the checks
                              (each pair once from each endpoint)               */
} pc_correct_stats;

/* The correction pass (Algorithm 1 up to Delta).  corrected_dev (N x 3) receives
 * P_hat: the reconstruction for particles outside E, orig + delta for editable
 * particles (every |corrected - orig| <= xi).  constraints may be NULL (selected
 * inside) or a handle from pc_select_constraints on the same orig.  Returns PC_OK,
 * PC_WARN_NOT_CONVERGED, or an error.  Synchronises the stream. */
pc_status pc_correct(pc_ctx *ctx, const float *orig_dev, const float *recon_dev, int64_t n,
                     const pc_params *params, const pc_constraints *constraints, float *corrected_dev,
                     pc_correct_stats *stats, void *stream);

/* pc_correct with extra outputs (each may be NULL):
 *   delta_dev     N x 3 float64: P_hat - P (offset of the final iterate) for editable
 *                 particles, 0 for the others; written in float64 from the double-float state.
 *   hist_loss_dev, hist_viol_dev: tight loss (float64) and violated-pair count (uint64) at
 *                 every evaluation t = 0..iters; room for t_max + 1 (or replay_iters + 1) entries.
 * Same errors and synchronisation as pc_correct. */
pc_status pc_correct_detail(pc_ctx *ctx, const float *orig_dev, const float *recon_dev, int64_t n,
                            const pc_params *params, const pc_constraints *constraints, float *corrected_dev,
                            double *delta_dev, double *hist_loss_dev, uint64_t *hist_viol_dev,
                            pc_correct_stats *stats, void *stream);

/* Batched form: independent blocks of particles, concatenated in orig/recon/corrected
 * (block k owns rows [offset_k, offset_k + n_k); the blocks must tile the arrays in
 * order: offset_0 = 0, offset_{k+1} = offset_k + n_k).  Each block has its own
 * parameters (b, xi, mode, box, Adam settings).  Every stage runs once over all
 * blocks -- one sort, one pair search, one selection, and PGD iterations in which all
 * blocks that have not stopped advance together -- and blocks never interact: each
 * block's corrected coordinates are bit-identical to pc_correct on that block alone.
 * stats (host, may be NULL) receives nblocks entries.  Returns PC_OK when every block
 * converged, PC_WARN_NOT_CONVERGED otherwise; errors name the offending block.  This
 * is a batching layer around the method, not part of the paper. */
typedef struct {
    int64_t offset;
    int64_t n;
    pc_params params;
} pc_block;
pc_status pc_correct_batch(pc_ctx *ctx, const float *orig_dev, const float *recon_dev, const pc_block *blocks,
                           int32_t nblocks, float *corrected_dev, pc_correct_stats *stats, void *stream);

/* Autotuner for the cell grid (not part of the paper): runs the selection (binning, pair
 * search, union-find, selection) on the given point set once per candidate cell factor
 * (2, 4, 8, 16, 32 cells per particle), twice each, and returns in *best the factor with
 * the shortest time (CUDA events on the stream).  ms (host, may be NULL) receives the 5
 * times.  The selected pairs do not depend on the factor, only the time does. */
pc_status pc_autotune_cells(pc_ctx *ctx, const float *xyz_dev, int64_t n, const pc_params *params, int32_t *best,
                            double *ms, void *stream);

/* Autotuner for the pair search (not part of the paper): the cell factor as
 * pc_autotune_cells does, then the dense-cell threshold (0 = none, 32, 128, 512) at that
 * factor, each timed over the whole selection on the given point set (the second of two
 * runs).  *tuned receives *params with cell_factor, dense_cell (and cell_cap_log2 = 0)
 * set to the fastest combination; ms (host, may be NULL) receives the 5 + 4 times.  The
 * selected pairs do not depend on either knob.  Synchronises the stream. */
pc_status pc_autotune(pc_ctx *ctx, const float *xyz_dev, int64_t n, const pc_params *params, pc_params *tuned,
                      double *ms, void *stream);

/* Cluster-query metrics of Sec. 4.1 ("Metrics"), for judging an iteration-capped
 * correction (Sec. 4.2 uses a 100-iteration limit).  lab0 / lab1: friends-of-friends
 * labels (smallest id of the component, as pc_fof_labels gives them) of the original and
 * of the decoded data, n entries each on the device.  A halo is a component with at least
 * min_members particles; a particle outside every halo shares a halo with no other.
 *   tp, fp, fn, tn: particle pairs by halo co-membership (same in both / merged /
 *                   split / different in both), exact integers;
 *   ari = 2 (tp tn - fp fn) / ((tp + fn)(fn + tn) + (tp + fp)(fp + tn));
 *   mwm_iou = sum_i |H_i| max_j |H_i and H'_j| / |H_i or H'_j| / sum_i |H_i| over original
 *             halos H_i and decoded halos H'_j (a halo with no overlap scores 0);
 *   halos0 / halos1 / members0: halo counts and particles in original halos.
 * With n_bins > 0 the halo mass functions dn/dlog10 M (mass = members) of both sides are
 * written to hmf0 / hmf1 (host, n_bins each) over n_bins equal-width bins of log10 M from
 * log10(min_members) to log10 of the largest original halo (edges: host, n_bins + 1),
 * normalised by volume and bin width.  Synchronises the stream. */
typedef struct {
    uint64_t tp, fp, fn, tn;
    double ari, mwm_iou;
    int64_t halos0, halos1, members0;
    int64_t pad_;
} pc_cluster_metrics_t;
pc_status pc_cluster_metrics(pc_ctx *ctx, const int32_t *lab0_dev, const int32_t *lab1_dev, int64_t n,
                             int32_t min_members, int32_t n_bins, double volume, pc_cluster_metrics_t *out,
                             double *hmf0, double *hmf1, double *bin_edges, void *stream);

/* Several linking lengths at once (Sec. 1 and Sec. 5: a range of thresholds is
 * supported by enforcing the union of the pairs each threshold selects).  b_list holds
 * n_b linking lengths (1 <= n_b <= 4), finite, positive and strictly ascending;
 * params->b is ignored, every other field applies to each length (mode, xi, box, m,
 * Adam, stop rule).  For each length the active pairs are selected as by
 * pc_select_constraints; a pair active at several lengths is enforced once at each, with
 * the link flag and the thresholds b -/+ delta_t of Eq. 3 of that length.  After
 * convergence the friends-of-friends labels at every length are those of orig.
 * stats: n_vulnerable and n_active are summed over the lengths; the other fields are as
 * for pc_correct.  n_b = 1 is pc_correct with b = b_list[0].  At most 2^29 editable
 * particles with n_b > 1 (PC_EINVAL otherwise).  Synchronises the stream. */
pc_status pc_correct_multi(pc_ctx *ctx, const float *orig_dev, const float *recon_dev, int64_t n,
                           const pc_params *params, const double *b_list, int32_t n_b, float *corrected_dev,
                           pc_correct_stats *stats, void *stream);

/* Edit stream v1 (Algorithm 1 last lines; Sec. 3.3).  Little endian:
 *   0  "PCE1" | 4 u32 version=1 | 8 u64 n | 16 u32 m | 20 u32 mode | 24 u32 periodic | 28 u32 0
 *   32 f64 xi | 40 u64 flagged | 48 u64 flag_bytes=ceil(n/8) | 56 u64 code_bytes
 *   64 flags: particle i -> byte i>>3, bit i&7 (1 = edited)
 *      codes: per flagged particle, ascending id, x y z codes of ceil(m/8) bytes each,
 *      q = clamp(rint((corrected - recon + 2 xi) / s), 0, 2^m - 1), s = 4 xi / (2^m - 1),
 *      evaluated in float64 (ties to even).
 * Without stream_dev (NULL) only *nbytes is computed.  With it, cap must be >= the size.
 * Synchronises the stream. */
pc_status pc_encode_edits(pc_ctx *ctx, const float *recon_dev, const float *corrected_dev, int64_t n,
                          const pc_params *params, uint8_t *stream_dev, size_t cap, size_t *nbytes,
                          void *stream);

/* Decoder (Sec. 3.3, "Reconstruction"): out = recon for unflagged particles and
 * fl32(recon + (-2 xi + q s)) (float64 inside, one rounding) for flagged ones.
 * stream_dev is a device copy of the stream.  PC_EFORMAT on a malformed stream. */
pc_status pc_apply_edits(pc_ctx *ctx, const float *recon_dev, int64_t n, const uint8_t *stream_dev,
                         size_t nbytes, float *out_dev, void *stream);

/* Allocation-free decoder.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory while decoding, for instance a simulation
 * or analysis code that reserves nearly all of the GPU's memory for its own arena at
 * start-up, or a caller working where device allocation is not allowed.  It computes
 * exactly what pc_apply_edits computes, takes no context, and calls no cudaMalloc,
 * cudaFree, pinned-host or pool allocation: its scratch (per-block flag counts and
 * their prefix sums) is one file-scope device array of 512 KB that every GPU which
 * loads the library holds until the process exits.
 *   - n must be in [1, 16,777,216]; larger n returns PC_EINVAL.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before
 *     any stream capture.
 *   - All calls share the array and it keeps the last call's contents (each call
 *     rewrites every entry it reads): calls that overlap on the GPU race, so issue
 *     them on one stream or one after another.
 *   - Synchronises the stream; PC_EFORMAT on a malformed stream. */
pc_status pc_apply_edits_static(const float *recon_dev, int64_t n, const uint8_t *stream_dev, size_t nbytes,
                                float *out_dev, void *stream);

/* Lossless stage (Algorithm 1, last line; Sec. 3.3 "Compaction, quantization, and
 * lossless compression"): canonical Huffman coding of an edit stream v1.  The paper
 * follows the Huffman stage with ZSTD; that stage is not part of this container.
 * Container "PCH1", little endian:
 *   0  "PCH1" | 4 u32 version=1 | 8 u64 raw_bytes | 16 u32 n_lanes | 20 u32 chunk=1024
 *   24 u32 max_len=15 | 28 u32 0 | 32..95 the stream's 64-byte header, verbatim
 *   96 per lane: u64 n_syms | u64 bit_len | u64 n_chunks=ceil(n_syms/1024) |
 *      256 x u8 code length (0 = unused symbol) | n_chunks x u64 bit offset of the chunk |
 *      ceil(bit_len/32) x u32 words
 * Lane 0 holds the flag bytes, lane 1 + k byte k of every code (k < ceil(m/8)).  Each
 * lane has its own code: Huffman lengths (ties taken in order of node id: symbols 0..255,
 * then merged nodes in order of creation) limited to 15 bits (deepest codes folded to 15
 * and the Kraft sum restored by deepening the deepest shorter codes; lengths then dealt
 * from longest to shortest in ascending (frequency, -symbol) order), canonical codes in
 * (length, symbol) order, bits written most significant first from bit 31 of each word.
 * A lane with one distinct symbol codes it with one bit.
 *
 * pc_huff_encode: in_dev is a device copy of an edit stream of nbytes bytes (PC_EFORMAT
 * if it is not one).  With out_dev NULL only *out_bytes is computed; else cap must be at
 * least that size (PC_EINVAL otherwise) and the container is written to out_dev.
 * pc_huff_decode: in_dev is a device copy of a container of nbytes bytes; *out_bytes is
 * set to the stream's size and, with out_dev non-NULL (cap at least that size), the
 * stream is written there.  PC_EFORMAT on a malformed container or an invalid code.
 * The container's buffer (out_dev of the encoder, in_dev of the decoder) must be 4-byte
 * aligned (PC_EINVAL otherwise; cudaMalloc'd pointers are): its words are read and
 * written as u32, and lanes after the first start at 4-byte boundaries.
 * Both synchronise the stream and hold no memory after they return. */
pc_status pc_huff_encode(pc_ctx *ctx, const uint8_t *in_dev, size_t nbytes, uint8_t *out_dev, size_t cap,
                         size_t *out_bytes, void *stream);
pc_status pc_huff_decode(pc_ctx *ctx, const uint8_t *in_dev, size_t nbytes, uint8_t *out_dev, size_t cap,
                         size_t *out_bytes, void *stream);

/* ------------------------------------------------------------------ serving
 * A request loop around pc_correct (not part of the paper).  A server owns one worker
 * thread on the context's device.  Submitted jobs wait in FIFO order until they can be
 * admitted: the jobs admitted together form a cohort that is set up in one pass
 * (validation, binning, pair-search count pass), admitted to the rest (selection, PGD)
 * only when the device-memory estimate from its counts fits the budget, and then
 * iterates on its own stream, replaying a CUDA graph of PGD launches, while later
 * cohorts are admitted and set up beside it (continuous batching: work of jobs that
 * arrived at different times overlaps on the device).  A job finishes as soon as its own
 * block stops: its corrected coordinates are copied out and, when asked, its edit
 * stream is encoded.  Every job's result is bit-identical to pc_correct (and
 * pc_encode_edits) on that job alone, whatever it was batched with.
 *
 * Buffers of a job are device buffers on the server's device; the caller keeps them
 * valid, and its inputs ready and unchanged, from submission until the job is DONE or
 * ERROR.  Thread safe: submit, poll and wait may be called from any thread. */
typedef struct pc_server pc_server;

typedef enum { PC_JOB_PENDING = 0, PC_JOB_RUNNING = 1, PC_JOB_DONE = 2, PC_JOB_ERROR = 3 } pc_job_state;

typedef struct {
    const float *orig_dev;    /* n x 3 original coordinates                              */
    const float *recon_dev;   /* n x 3 reconstruction, |recon - orig| <= xi                */
    int64_t n;
    pc_params params;
    float *corrected_dev;     /* n x 3 output                                             */
    uint8_t *stream_dev;      /* edit stream output, or NULL for none                     */
    size_t stream_cap;        /* bytes available at stream_dev                             */
} pc_job;

typedef struct {
    int32_t state;            /* pc_job_state                                              */
    int32_t status;           /* once DONE or ERROR: PC_OK, PC_WARN_NOT_CONVERGED or an error */
    int64_t submit_ns;        /* steady-clock times of submission, admission and completion */
    int64_t start_ns;
    int64_t done_ns;
    uint64_t stream_bytes;    /* size of the edit stream written (0 without one)            */
    int32_t cohort_jobs;      /* jobs set up together with this one                        */
    int32_t pad_;
    pc_correct_stats stats;
    char error[160];          /* message of an ERROR                                       */
} pc_job_result;

/* mem_budget: device bytes the server's jobs may hold at once (0 = 40 GiB); max_slots:
 * jobs resident at once (0 = 256); max_cohort_particles: particles admitted together in
 * one cohort (0 = 2^24).  A job whose estimate alone exceeds the budget ends in ERROR
 * with PC_ENOMEM. */
pc_status pc_server_create(pc_ctx *ctx, size_t mem_budget, int32_t max_slots, int64_t max_cohort_particles,
                           pc_server **out);
/* Finishes every submitted job, then stops the worker and frees the server. */
void pc_server_destroy(pc_server *srv);
/* Queues a job (parameters are checked at once: PC_EINVAL, no ticket).  Never blocks. */
pc_status pc_serve_submit(pc_server *srv, const pc_job *job, uint64_t *ticket);
/* Current state of a job (PC_EBUSY for an unknown ticket). */
pc_status pc_serve_poll(pc_server *srv, uint64_t ticket, pc_job_result *res);
/* Waits until the job is DONE or ERROR, at most timeout_ms (< 0: no limit); PC_ETIMEOUT
 * when the time ran out (res then holds the current state). */
pc_status pc_serve_wait(pc_server *srv, uint64_t ticket, int64_t timeout_ms, pc_job_result *res);
/* Server counters: jobs submitted, finished, cohorts formed, peak estimated bytes. */
pc_status pc_serve_counters(pc_server *srv, int64_t out[4]);

#ifdef __cplusplus
}
#endif
#endif /* PC_H_ */
