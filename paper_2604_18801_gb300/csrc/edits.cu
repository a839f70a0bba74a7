// Edit stream: flags + m-bit codes (Algorithm 1 last lines; Sec. 3.3
// "Compaction, quantization" and "Reconstruction").
//
// Encode: one thread per particle; a warp ballot of "corrected != recon"
// gives 32 flag bits (little-endian word = particles i..i+31, bit i&7 of byte
// i>>3), per-block flagged counts are scanned, and each flagged particle
// writes its three codes at its rank, so codes appear in ascending id.
// q = clamp(rint((corrected - recon + 2 xi) / s), 0, 2^m - 1), s = 4 xi/(2^m-1),
// in float64.  Decode: the same ranking from the flag bits, then
// out = fl32(recon + (-2 xi + q s)) with the sum in float64.
#include <algorithm>
#include <cstring>

#include "pipeline.cuh"

namespace pc {

namespace {

constexpr int ET = 256;  // particles per block
constexpr int HEADER = 64;

__device__ __forceinline__ bool edited(const float *r, const float *c, int64_t i) {
    return (c[3 * i] != r[3 * i]) | (c[3 * i + 1] != r[3 * i + 1]) | (c[3 * i + 2] != r[3 * i + 2]);
}

// per-block flagged counts
__global__ void k_enc_count(const float *__restrict__ recon, const float *__restrict__ corr, int64_t n,
                            uint32_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * ET + threadIdx.x;
    const bool f = i < n && edited(recon, corr, i);
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (uint32_t)c;
}

__global__ void k_enc_write(const float *__restrict__ recon, const float *__restrict__ corr, int64_t n,
                            const uint32_t *__restrict__ off, double xi, double s, double qmax, int cb,
                            uint8_t *__restrict__ flags, int64_t flag_bytes, uint8_t *__restrict__ codes) {
    __shared__ uint32_t wcnt[ET / 32];
    const int64_t i = (int64_t)blockIdx.x * ET + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool f = i < n && edited(recon, corr, i);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) {
        wcnt[w] = __popc(bal);
        const int64_t byte0 = ((int64_t)blockIdx.x * ET + w * 32) >> 3;
        if (byte0 + 4 <= flag_bytes) {
            *(uint32_t *)(flags + byte0) = bal;
        } else {
            for (int k = 0; k < 4; ++k)
                if (byte0 + k < flag_bytes) flags[byte0 + k] = (uint8_t)(bal >> (8 * k));
        }
    }
    __syncthreads();
    if (!f) return;
    uint32_t rank = off[blockIdx.x];
    for (int q = 0; q < w; ++q) rank += wcnt[q];
    rank += __popc(bal & ((1u << lane) - 1u));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double delta = (double)corr[3 * i + a] - (double)recon[3 * i + a];
        double q = rint((delta + 2.0 * xi) / s);
        q = fmin(qmax, fmax(0.0, q));
        const unsigned long long qi = (unsigned long long)q;
        uint8_t *dst = codes + ((int64_t)rank * 3 + a) * cb;
        for (int k = 0; k < cb; ++k) dst[k] = (uint8_t)(qi >> (8 * k));
    }
}

__global__ void k_dec_count(const uint8_t *__restrict__ flags, int64_t n, uint32_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * ET + threadIdx.x;
    const bool f = i < n && ((flags[i >> 3] >> (i & 7)) & 1u);
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (uint32_t)c;
}

__global__ void k_dec_apply(const float *__restrict__ recon, int64_t n, const uint8_t *__restrict__ flags,
                            const uint8_t *__restrict__ codes, const uint32_t *__restrict__ off, double xi, double s,
                            int cb, float *__restrict__ out) {
    __shared__ uint32_t wcnt[ET / 32];
    const int64_t i = (int64_t)blockIdx.x * ET + threadIdx.x;
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
        out[3 * i + a] = (float)((double)recon[3 * i + a] + (-2.0 * xi + (double)q * s));
    }
}

void put_u32(uint8_t *o, uint32_t v) {
    for (int k = 0; k < 4; ++k) o[k] = (uint8_t)(v >> (8 * k));
}
void put_u64(uint8_t *o, uint64_t v) {
    for (int k = 0; k < 8; ++k) o[k] = (uint8_t)(v >> (8 * k));
}
uint32_t get_u32(const uint8_t *o) {
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) v |= (uint32_t)o[k] << (8 * k);
    return v;
}
uint64_t get_u64(const uint8_t *o) {
    uint64_t v = 0;
    for (int k = 0; k < 8; ++k) v |= (uint64_t)o[k] << (8 * k);
    return v;
}

}  // namespace

// Returns the stream size; writes the stream when out != null (cap already checked by the caller).
size_t encode_edits(const float *recon, const float *corr, int64_t n, const pc_params *p, uint8_t *out, size_t cap,
                    cudaStream_t s, HostScratch &hs) {
    const int m = p->m_bits;
    const int cb = (m + 7) / 8;
    const int64_t nblk = cdiv(n, ET);
    DBuf<uint32_t> cnt(nblk, s), off(nblk, s), tot(1, s);
    k_enc_count<<<(unsigned)nblk, ET, 0, s>>>(recon, corr, n, cnt.p);
    PC_CHECK_LAUNCH();
    scan_exclusive_u32(cnt.p, off.p, nblk, tot.p, s);
    const uint64_t nf = *(uint32_t *)read_back(hs, tot.p, sizeof(uint32_t), s);
    const int64_t fb = (n + 7) / 8;
    const int64_t codeb = (int64_t)nf * 3 * cb;
    const size_t total = HEADER + fb + codeb;
    if (!out) return total;
    if (cap < total) {
        set_error("pc_encode_edits: stream capacity too small");
        throw Fail{PC_EINVAL};
    }
    uint8_t *h = (uint8_t *)host_scratch(hs, HEADER);
    memset(h, 0, HEADER);
    memcpy(h, "PCE1", 4);
    put_u32(h + 4, 1);
    put_u64(h + 8, (uint64_t)n);
    put_u32(h + 16, (uint32_t)m);
    put_u32(h + 20, (uint32_t)p->mode);
    put_u32(h + 24, (uint32_t)p->periodic);
    memcpy(h + 32, &p->xi, 8);
    put_u64(h + 40, nf);
    put_u64(h + 48, (uint64_t)fb);
    put_u64(h + 56, (uint64_t)codeb);
    PC_CUDA(cudaMemcpyAsync(out, h, HEADER, cudaMemcpyHostToDevice, s));
    const double qmax = std::ldexp(1.0, m) - 1.0;
    const double step = 4.0 * p->xi / qmax;
    k_enc_write<<<(unsigned)nblk, ET, 0, s>>>(recon, corr, n, off.p, p->xi, step, qmax, cb, out + HEADER, fb,
                                              out + HEADER + fb);
    PC_CHECK_LAUNCH();
    PC_CUDA(cudaStreamSynchronize(s));
    return total;
}

void apply_edits(const float *recon, int64_t n, const uint8_t *in, size_t nbytes, float *out, cudaStream_t s,
                 HostScratch &hs) {
    if (nbytes < (size_t)HEADER) {
        set_error("pc_apply_edits: stream shorter than its header");
        throw Fail{PC_EFORMAT};
    }
    const uint8_t *h = (const uint8_t *)read_back(hs, in, HEADER, s);
    uint8_t hdr[HEADER];
    memcpy(hdr, h, HEADER);
    const int m = (int)get_u32(hdr + 16);
    double xi;
    memcpy(&xi, hdr + 32, 8);
    const uint64_t nf = get_u64(hdr + 40), fb = get_u64(hdr + 48), codeb = get_u64(hdr + 56);
    const int cb = (m + 7) / 8;
    const bool ok = memcmp(hdr, "PCE1", 4) == 0 && get_u32(hdr + 4) == 1 && get_u64(hdr + 8) == (uint64_t)n &&
                    m >= 2 && m <= 32 && fb == (uint64_t)((n + 7) / 8) && codeb == nf * 3 * (uint64_t)cb &&
                    nbytes >= HEADER + fb + codeb && xi >= 0.0 && nf <= (uint64_t)n;
    if (!ok) {
        set_error("pc_apply_edits: malformed edit stream header");
        throw Fail{PC_EFORMAT};
    }
    const int64_t nblk = cdiv(n, ET);
    DBuf<uint32_t> cnt(nblk, s), off(nblk, s), tot(1, s);
    k_dec_count<<<(unsigned)nblk, ET, 0, s>>>(in + HEADER, n, cnt.p);
    PC_CHECK_LAUNCH();
    scan_exclusive_u32(cnt.p, off.p, nblk, tot.p, s);
    const uint32_t seen = *(uint32_t *)read_back(hs, tot.p, sizeof(uint32_t), s);
    if (seen != nf) {
        set_error("pc_apply_edits: flag count does not match the header");
        throw Fail{PC_EFORMAT};
    }
    const double step = 4.0 * xi / (std::ldexp(1.0, m) - 1.0);
    k_dec_apply<<<(unsigned)nblk, ET, 0, s>>>(recon, n, in + HEADER, in + HEADER + fb, off.p, xi, step, cb, out);
    PC_CHECK_LAUNCH();
    PC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pc
