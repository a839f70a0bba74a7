// Allocation-free decoder: pc_apply_edits_static (include/pc.h).
//
// Same result as pc_apply_edits, for callers that cannot allocate device memory
// on the call path (a code that has claimed the device's memory for its own
// arena at start-up, or a caller working inside a region where allocation is
// not allowed).  Its only scratch, the per-block flag counts and their prefix
// sums, lives in one file-scope device array below, sized for at most
// 2^24 particles; the host reads the 64-byte header and one count into stack
// variables.  No cudaMalloc, cudaFree, pinned allocation or pool call is made.
#include <cmath>
#include <cstring>
#include <mutex>

#include "pipeline.cuh"

namespace pc {
namespace {

constexpr int SD_THREADS = 256;                       // particles per block of the count/apply kernels
constexpr int64_t SD_MAX_BLOCKS = 65536;
constexpr int64_t SD_MAX_N = SD_MAX_BLOCKS * SD_THREADS;   // 16,777,216 particles
constexpr int SD_HEADER = 64;
constexpr int SD_SCAN_THREADS = 1024;

// [0, SD_MAX_BLOCKS): flagged count per block; [SD_MAX_BLOCKS, 2*SD_MAX_BLOCKS): exclusive
// prefix; [2*SD_MAX_BLOCKS]: total.  512 KB + 256 B, held by every device that loads the library.
static __device__ __align__(256) uint32_t g_sd_scratch[2 * SD_MAX_BLOCKS + 64];

std::mutex g_sd_mu;
uint32_t *g_sd_ptr[256] = {nullptr};                  // device address of the array, per device

__global__ void k_sd_count(const uint8_t *__restrict__ flags, int64_t n, uint32_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * SD_THREADS + threadIdx.x;
    const bool f = i < n && ((flags[i >> 3] >> (i & 7)) & 1u);
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (uint32_t)c;
}

// One block: exclusive prefix of nblk <= SD_MAX_BLOCKS counts (each thread a consecutive run).
__global__ void k_sd_scan(const uint32_t *__restrict__ cnt, uint32_t *__restrict__ off, int64_t nblk,
                          uint32_t *__restrict__ total) {
    __shared__ uint32_t part[SD_SCAN_THREADS];
    const int64_t per = (nblk + SD_SCAN_THREADS - 1) / SD_SCAN_THREADS;
    const int64_t b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t b = b0; b < b0 + per && b < nblk; ++b) s += cnt[b];
    part[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan of the 1024 run totals
    for (int d = 1; d < SD_SCAN_THREADS; d <<= 1) {
        const uint32_t v = threadIdx.x >= d ? part[threadIdx.x - d] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int64_t b = b0; b < b0 + per && b < nblk; ++b) {
        off[b] = run;
        run += cnt[b];
    }
    if (threadIdx.x == SD_SCAN_THREADS - 1) *total = part[SD_SCAN_THREADS - 1];
}

__global__ void k_sd_apply(const float *__restrict__ recon, int64_t n, const uint8_t *__restrict__ flags,
                           const uint8_t *__restrict__ codes, const uint32_t *__restrict__ off, double xi,
                           double step, int cb, float *__restrict__ out) {
    __shared__ uint32_t wcnt[SD_THREADS / 32];
    const int64_t i = (int64_t)blockIdx.x * SD_THREADS + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool f = i < n && ((flags[i >> 3] >> (i & 7)) & 1u);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    if (i >= n) return;
    if (!f) {
        out[3 * i] = recon[3 * i];
        out[3 * i + 1] = recon[3 * i + 1];
        out[3 * i + 2] = recon[3 * i + 2];
        return;
    }
    uint32_t rank = off[blockIdx.x];
    for (int q = 0; q < w; ++q) rank += wcnt[q];
    rank += __popc(bal & ((1u << lane) - 1u));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uint8_t *src = codes + ((int64_t)rank * 3 + a) * cb;
        unsigned long long q = 0;
        for (int k = 0; k < cb; ++k) q |= (unsigned long long)src[k] << (8 * k);
        out[3 * i + a] = (float)((double)recon[3 * i + a] + (-2.0 * xi + (double)q * step));
    }
}

uint64_t rd64(const uint8_t *o) {
    uint64_t v = 0;
    for (int k = 0; k < 8; ++k) v |= (uint64_t)o[k] << (8 * k);
    return v;
}
uint32_t rd32(const uint8_t *o) {
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) v |= (uint32_t)o[k] << (8 * k);
    return v;
}

// Device address of the scratch array on the current device (looked up once per device).
uint32_t *sd_scratch() {
    int dev = 0;
    PC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("pc_apply_edits_static: device index out of range");
        throw Fail{PC_EINVAL};
    }
    std::lock_guard<std::mutex> lk(g_sd_mu);
    if (!g_sd_ptr[dev]) {
        void *p = nullptr;
        PC_CUDA(cudaGetSymbolAddress(&p, g_sd_scratch));
        g_sd_ptr[dev] = (uint32_t *)p;
    }
    return g_sd_ptr[dev];
}

}  // namespace
}  // namespace pc

extern "C" pc_status pc_apply_edits_static(const float *recon_dev, int64_t n, const uint8_t *stream_dev,
                                           size_t nbytes, float *out_dev, void *stream) {
    using namespace pc;
    try {
        if (!recon_dev || !stream_dev || !out_dev) {
            set_error("pc_apply_edits_static: NULL buffer");
            return PC_EINVAL;
        }
        if (n < 1 || n > SD_MAX_N) {
            set_error("pc_apply_edits_static: n must be in [1, 16777216] (static scratch limit)");
            return PC_EINVAL;
        }
        if (nbytes < (size_t)SD_HEADER) {
            set_error("pc_apply_edits_static: stream shorter than its header");
            return PC_EFORMAT;
        }
        cudaStream_t s = (cudaStream_t)stream;
        uint32_t *scratch = sd_scratch();
        uint8_t hdr[SD_HEADER];
        PC_CUDA(cudaMemcpyAsync(hdr, stream_dev, SD_HEADER, cudaMemcpyDeviceToHost, s));
        PC_CUDA(cudaStreamSynchronize(s));
        const int m = (int)rd32(hdr + 16);
        double xi;
        memcpy(&xi, hdr + 32, 8);
        const uint64_t nf = rd64(hdr + 40), fb = rd64(hdr + 48), codeb = rd64(hdr + 56);
        const int cb = (m + 7) / 8;
        const bool ok = memcmp(hdr, "PCE1", 4) == 0 && rd32(hdr + 4) == 1 && rd64(hdr + 8) == (uint64_t)n && m >= 2 &&
                        m <= 32 && fb == (uint64_t)((n + 7) / 8) && codeb == nf * 3 * (uint64_t)cb &&
                        nbytes >= SD_HEADER + fb + codeb && xi >= 0.0 && nf <= (uint64_t)n;
        if (!ok) {
            set_error("pc_apply_edits_static: malformed edit stream header");
            return PC_EFORMAT;
        }
        const int64_t nblk = cdiv(n, SD_THREADS);
        uint32_t *cnt = scratch, *off = scratch + SD_MAX_BLOCKS, *total = scratch + 2 * SD_MAX_BLOCKS;
        k_sd_count<<<(unsigned)nblk, SD_THREADS, 0, s>>>(stream_dev + SD_HEADER, n, cnt);
        PC_CHECK_LAUNCH();
        k_sd_scan<<<1, SD_SCAN_THREADS, 0, s>>>(cnt, off, nblk, total);
        PC_CHECK_LAUNCH();
        uint32_t seen = 0;
        PC_CUDA(cudaMemcpyAsync(&seen, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        PC_CUDA(cudaStreamSynchronize(s));
        if (seen != nf) {
            set_error("pc_apply_edits_static: flag count does not match the header");
            return PC_EFORMAT;
        }
        const double step = 4.0 * xi / (std::ldexp(1.0, m) - 1.0);
        k_sd_apply<<<(unsigned)nblk, SD_THREADS, 0, s>>>(recon_dev, n, stream_dev + SD_HEADER,
                                                          stream_dev + SD_HEADER + fb, off, xi, step, cb, out_dev);
        PC_CHECK_LAUNCH();
        PC_CUDA(cudaStreamSynchronize(s));
        return PC_OK;
    } catch (const Fail &f) {
        return f.st;
    } catch (...) {
        set_error("pc_apply_edits_static: unexpected failure");
        return PC_ECUDA;
    }
}
