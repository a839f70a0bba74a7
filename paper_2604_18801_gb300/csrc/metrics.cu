// Cluster-query metrics of Sec. 4.1 ("Metrics"): the adjusted Rand index of pairwise
// halo co-membership, the mass-weighted mean IoU of halo membership, and the halo mass
// function.  Used to judge an iteration-capped correction (Sec. 4.2, a 100-iteration
// limit), where membership is improved but not exact.
//
// A halo is a friends-of-friends component with at least min_members particles; a
// particle outside every halo shares a halo with no other particle.  With labels lab0
// (original) and lab1 (decoded), both "smallest id of the component":
//   TP = sum over (halo i, halo j) of C(n_ij, 2)      n_ij = |H_i and H'_j|
//   TP + FN = sum_i C(|H_i|, 2),  TP + FP = sum_j C(|H'_j|, 2),  TN = C(n, 2) - TP - FP - FN
//   IoU_i = max_j n_ij / (|H_i| + |H'_j| - n_ij),  MWM-IoU = sum_i |H_i| IoU_i / sum_i |H_i|
// The pairs (i, j) come from one radix sort of the 64-bit keys (i << 32 | j); all counts
// are integers.  The HMF counts halos per equal-width bin of log10(members).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pipeline.cuh"

namespace pc {
namespace {

#define MGRID(i, n) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
                         i += (int64_t)gridDim.x * blockDim.x)

inline int mgrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

__global__ void k_sizes(const int32_t *__restrict__ lab, int64_t n, uint32_t *__restrict__ sz) {
    MGRID(k, n) atomicAdd(sz + lab[k], 1u);
}

// C(size, 2) over halos (roots with size >= min_members), halo count, largest halo.
__global__ void k_halo_sums(const uint32_t *__restrict__ sz, int64_t n, uint32_t min_members,
                            unsigned long long *__restrict__ out /* [pairs, halos, max, members] */) {
    unsigned long long pairs = 0, halos = 0, members = 0;
    uint32_t mx = 0;
    MGRID(k, n) {
        const uint32_t s = sz[k];
        if (s >= min_members && s > 0) {
            pairs += (unsigned long long)s * (s - 1) / 2;
            halos += 1;
            members += s;
            mx = max(mx, s);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        halos += __shfl_xor_sync(0xffffffffu, halos, o);
        members += __shfl_xor_sync(0xffffffffu, members, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (pairs) atomicAdd(out + 0, pairs);
        if (halos) atomicAdd(out + 1, halos);
        if (mx) atomicMax(out + 2, (unsigned long long)mx);
        if (members) atomicAdd(out + 3, members);
    }
}

// key = (original halo << 32 | decoded halo) for particles in a halo on both sides, else ~0
__global__ void k_pair_keys(const int32_t *__restrict__ lab0, const int32_t *__restrict__ lab1,
                            const uint32_t *__restrict__ sz0, const uint32_t *__restrict__ sz1, int64_t n,
                            uint32_t min_members, unsigned long long *__restrict__ keys) {
    MGRID(k, n) {
        const int32_t a = lab0[k], b = lab1[k];
        const bool in = sz0[a] >= min_members && sz1[b] >= min_members;
        keys[k] = in ? (((unsigned long long)(uint32_t)a << 32) | (unsigned long long)(uint32_t)b) : ~0ull;
    }
}

__global__ void k_run_flags(const unsigned long long *__restrict__ keys, int64_t n, uint32_t *__restrict__ flag) {
    MGRID(k, n) flag[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1u : 0u;
}

__global__ void k_run_starts(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos, int64_t n,
                             uint32_t *__restrict__ start) {
    MGRID(k, n) {
        if (flag[k]) start[pos[k]] = (uint32_t)k;
    }
}

// Runs of equal keys: n_ij, TP += C(n_ij, 2), IoU_i = max_j n_ij / (a_i + b_j - n_ij).
__global__ void k_runs(const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ start,
                       int64_t nruns, int64_t n, const uint32_t *__restrict__ sz0, const uint32_t *__restrict__ sz1,
                       unsigned long long *__restrict__ tp, unsigned long long *__restrict__ iou_bits) {
    unsigned long long acc = 0;
    MGRID(r, nruns) {
        const int64_t k = start[r], e = r + 1 < nruns ? (int64_t)start[r + 1] : n;
        const unsigned long long key = keys[k];
        if (key == ~0ull) continue;
        const unsigned long long nij = (unsigned long long)(e - k);
        acc += nij * (nij - 1) / 2;
        const uint32_t i = (uint32_t)(key >> 32), j = (uint32_t)key;
        const double iou = (double)nij / ((double)sz0[i] + (double)sz1[j] - (double)nij);
        atomicMax(iou_bits + i, (unsigned long long)__double_as_longlong(iou));   // iou >= 0: bits order as values
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(tp, acc);
}

// sum over original halos of |H_i| IoU_i (in fixed point, 2^-32 units, so the sum is exact;
// |H_i| < 2^31 keeps every term and the total below 2^63)
__global__ void k_mwm(const uint32_t *__restrict__ sz0, const unsigned long long *__restrict__ iou_bits, int64_t n,
                      uint32_t min_members, unsigned long long *__restrict__ out) {
    unsigned long long acc = 0;
    MGRID(k, n) {
        const uint32_t s = sz0[k];
        if (s < min_members || s == 0) continue;
        const double iou = __longlong_as_double((long long)iou_bits[k]);
        acc += (unsigned long long)llrint(iou * (double)s * 4294967296.0);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// HMF counts: halo roots with size >= min_members, bin = floor((log10(size) - lo) / width)
__global__ void k_hmf(const uint32_t *__restrict__ sz, int64_t n, uint32_t min_members, double lo, double width,
                      int nbins, unsigned long long *__restrict__ counts) {
    MGRID(k, n) {
        const uint32_t s = sz[k];
        if (s < min_members || s == 0) continue;
        int bin = (int)floor((log10((double)s) - lo) / width);
        bin = min(max(bin, 0), nbins - 1);
        atomicAdd(counts + bin, 1ull);
    }
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" pc_status pc_cluster_metrics(pc_ctx *ctx, const int32_t *lab0, const int32_t *lab1, int64_t n,
                                        int32_t min_members, int32_t n_bins, double volume, pc_cluster_metrics_t *out,
                                        double *hmf0, double *hmf1, double *bin_edges, void *stream) {
    try {
        if (!ctx || !lab0 || !lab1 || !out) {
            set_error("pc_cluster_metrics: NULL argument");
            return PC_EINVAL;
        }
        if (n < 1 || n >= (int64_t)0x7fffffff || min_members < 1 || n_bins < 0 || n_bins > 4096 ||
            (n_bins > 0 && (!hmf0 || !hmf1 || !bin_edges || !(volume > 0.0)))) {
            set_error("pc_cluster_metrics: bad sizes");
            return PC_EINVAL;
        }
        PC_CUDA(cudaSetDevice(ctx_device(ctx)));
        cudaStream_t s = (cudaStream_t)stream;
        HostScratch hs;
        struct HsGuard {
            HostScratch &h;
            ~HsGuard() {
                if (h.p) cudaFreeHost(h.p);
            }
        } hg{hs};
        DBuf<uint32_t> sz0(n, s), sz1(n, s);
        DBuf<unsigned long long> sums(16, s), iou(n, s), keys(n, s), hist(2 * std::max(1, (int)n_bins), s);
        PC_CUDA(cudaMemsetAsync(sz0.p, 0, n * sizeof(uint32_t), s));
        PC_CUDA(cudaMemsetAsync(sz1.p, 0, n * sizeof(uint32_t), s));
        PC_CUDA(cudaMemsetAsync(sums.p, 0, 16 * sizeof(unsigned long long), s));
        PC_CUDA(cudaMemsetAsync(iou.p, 0, n * sizeof(unsigned long long), s));
        PC_CUDA(cudaMemsetAsync(hist.p, 0, 2 * std::max(1, (int)n_bins) * sizeof(unsigned long long), s));
        const uint32_t mm = (uint32_t)min_members;
        k_sizes<<<mgrid(n), 256, 0, s>>>(lab0, n, sz0.p);
        PC_CHECK_LAUNCH();
        k_sizes<<<mgrid(n), 256, 0, s>>>(lab1, n, sz1.p);
        PC_CHECK_LAUNCH();
        k_halo_sums<<<mgrid(n), 256, 0, s>>>(sz0.p, n, mm, sums.p + 0);
        PC_CHECK_LAUNCH();
        k_halo_sums<<<mgrid(n), 256, 0, s>>>(sz1.p, n, mm, sums.p + 4);
        PC_CHECK_LAUNCH();
        k_pair_keys<<<mgrid(n), 256, 0, s>>>(lab0, lab1, sz0.p, sz1.p, n, mm, keys.p);
        PC_CHECK_LAUNCH();
        radix_sort_u64((uint64_t *)keys.p, nullptr, n, 64, s);
        {
            DBuf<uint32_t> flag(n, s), pos(n, s), start(n, s), nr(1, s);
            k_run_flags<<<mgrid(n), 256, 0, s>>>(keys.p, n, flag.p);
            PC_CHECK_LAUNCH();
            scan_exclusive_u32(flag.p, pos.p, n, nr.p, s);
            k_run_starts<<<mgrid(n), 256, 0, s>>>(flag.p, pos.p, n, start.p);
            PC_CHECK_LAUNCH();
            const int64_t nruns = *(const uint32_t *)read_back(hs, nr.p, sizeof(uint32_t), s);
            k_runs<<<mgrid(nruns), 256, 0, s>>>(keys.p, start.p, nruns, n, sz0.p, sz1.p, sums.p + 8, iou.p);
            PC_CHECK_LAUNCH();
        }
        k_mwm<<<mgrid(n), 256, 0, s>>>(sz0.p, iou.p, n, mm, sums.p + 9);
        PC_CHECK_LAUNCH();
        unsigned long long h[16];
        memcpy(h, read_back(hs, sums.p, sizeof(h), s), sizeof(h));
        const unsigned long long p0 = h[0], p1 = h[4], tp = h[8];
        const unsigned long long total = (unsigned long long)n * (unsigned long long)(n - 1) / 2;
        pc_cluster_metrics_t &m = *out;
        memset(&m, 0, sizeof(m));
        m.tp = tp;
        m.fn = p0 - tp;
        m.fp = p1 - tp;
        m.tn = total - tp - m.fn - m.fp;
        m.halos0 = (int64_t)h[1];
        m.halos1 = (int64_t)h[5];
        m.members0 = (int64_t)h[3];
        // ARI = 2 (TP TN - FP FN) / ((TP + FN)(FN + TN) + (TP + FP)(FP + TN)), in long double
        const long double TP = tp, TN = m.tn, FP = m.fp, FN = m.fn;
        const long double den = (TP + FN) * (FN + TN) + (TP + FP) * (FP + TN);
        m.ari = den > 0 ? (double)(2.0L * (TP * TN - FP * FN) / den) : 1.0;
        m.mwm_iou = h[3] ? (double)((long double)h[9] / 4294967296.0L / (long double)h[3]) : 1.0;
        if (n_bins > 0) {
            const double mx = (double)std::max<unsigned long long>(h[2], (unsigned long long)min_members);
            const double lo = std::log10((double)min_members);
            const double hi = std::log10(mx) + 1e-9;
            const double width = (hi - lo) / n_bins;
            for (int k = 0; k <= n_bins; ++k) bin_edges[k] = std::pow(10.0, lo + k * width);
            k_hmf<<<mgrid(n), 256, 0, s>>>(sz0.p, n, mm, lo, width, n_bins, hist.p);
            PC_CHECK_LAUNCH();
            k_hmf<<<mgrid(n), 256, 0, s>>>(sz1.p, n, mm, lo, width, n_bins, hist.p + n_bins);
            PC_CHECK_LAUNCH();
            const unsigned long long *hc =
                (const unsigned long long *)read_back(hs, hist.p, 2 * n_bins * sizeof(unsigned long long), s);
            // dn / dlog10 M: counts per volume and per unit of log10 mass
            for (int k = 0; k < n_bins; ++k) {
                hmf0[k] = (double)hc[k] / (volume * width);
                hmf1[k] = (double)hc[n_bins + k] / (volume * width);
            }
        }
        PC_CUDA(cudaStreamSynchronize(s));
        return PC_OK;
    } catch (const Fail &f) {
        return f.st;
    } catch (...) {
        set_error("pc_cluster_metrics: unexpected failure");
        return PC_ECUDA;
    }
}
