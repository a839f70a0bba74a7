// Lossless stage of the edit stream (Algorithm 1, last line; Sec. 3.3 "Compaction,
// quantization, and lossless compression"): canonical Huffman coding of the stream's
// bytes, container "PCH1" (include/pc.h).  The paper follows Huffman with ZSTD; this
// container holds the Huffman stage only.
//
// The stream body is split into lanes (flag bytes; byte k of every code), each coded with
// its own canonical code of at most 15 bits.  On the device: one 256-bin histogram per
// lane, the bit length of every 1024-symbol chunk, a scan of the chunk lengths (the
// chunks' bit offsets, kept in the container so that every chunk decodes on its own),
// and the codes written with one 32-bit atomic OR per word they touch.  The code lengths
// and canonical codes (256 symbols per lane) are built on the host.
#include <algorithm>
#include <cstring>
#include <functional>
#include <queue>
#include <vector>

#include "pipeline.cuh"

namespace pc {
namespace {

constexpr int HMAX = 15;          // longest code
constexpr int HCHUNK = 1024;      // symbols per independently decodable chunk
constexpr int ENC_SPT = HCHUNK / 256;   // symbols per thread of k_encode (256 threads per chunk)
constexpr int HHEAD = 64;         // bytes of the edit stream's own header
constexpr int CONT_HEAD = 96;     // container header: 32 bytes + the stream header

#define HGRID(i, n) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
                         i += (int64_t)gridDim.x * blockDim.x)

// A lane: n symbols at base + i * stride.
struct Lane {
    int64_t off, n;
    int stride;
};

__global__ void k_hist(const uint8_t *__restrict__ src, Lane L, unsigned long long *__restrict__ hist) {
    __shared__ unsigned int h[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) h[k] = 0;
    __syncthreads();
    HGRID(i, L.n) atomicAdd(&h[src[L.off + i * L.stride]], 1u);
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
        if (h[k]) atomicAdd(hist + k, (unsigned long long)h[k]);
}

// bit length of each chunk (one block per chunk)
__global__ void k_chunk_bits(const uint8_t *__restrict__ src, Lane L, const uint8_t *__restrict__ lens,
                             unsigned long long *__restrict__ chunk_bits) {
    __shared__ uint8_t ln[256];
    __shared__ unsigned long long part[8];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) ln[k] = lens[k];
    __syncthreads();
    const int64_t c = blockIdx.x, i0 = c * HCHUNK, i1 = min((int64_t)HCHUNK * (c + 1), L.n);
    unsigned long long acc = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += ln[src[L.off + i * L.stride]];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        chunk_bits[c] = t;
    }
}

// Codes of one chunk per block: each thread takes ENC_SPT consecutive symbols, a block scan of
// their bit lengths places them, and every code is ORed into the (zeroed) words it spans.
__global__ void k_encode(const uint8_t *__restrict__ src, Lane L, const uint8_t *__restrict__ lens,
                         const uint32_t *__restrict__ codes, const unsigned long long *__restrict__ chunk_off,
                         uint32_t *__restrict__ words) {
    __shared__ uint8_t ln[256];
    __shared__ uint32_t cd[256];
    __shared__ unsigned int scan[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
        ln[k] = lens[k];
        cd[k] = codes[k];
    }
    __syncthreads();
    const int64_t c = blockIdx.x;
    const int64_t i0 = c * HCHUNK + (int64_t)threadIdx.x * ENC_SPT;
    const int64_t i1 = min(i0 + ENC_SPT, min((int64_t)HCHUNK * (c + 1), L.n));
    unsigned int mine = 0;
    for (int64_t i = i0; i < i1; ++i) mine += ln[src[L.off + i * L.stride]];
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int d = 1; d < 256; d <<= 1) {   // inclusive Hillis-Steele scan over the 256 threads
        const unsigned int v = threadIdx.x >= (unsigned)d ? scan[threadIdx.x - d] : 0u;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long pos = chunk_off[c] + (scan[threadIdx.x] - mine);
    for (int64_t i = i0; i < i1; ++i) {
        const uint8_t s = src[L.off + i * L.stride];
        const int l = ln[s];
        const uint32_t code = cd[s];
        const int b = (int)(pos & 31);
        const int64_t w = (int64_t)(pos >> 5);
        if (b + l <= 32) {
            atomicOr(words + w, code << (32 - b - l));
        } else {
            atomicOr(words + w, code >> (b + l - 32));
            atomicOr(words + w + 1, code << (64 - b - l));
        }
        pos += l;
    }
}

// Canonical decoding tables of one lane.
struct DecTab {
    uint32_t first[HMAX + 2];   // first code of each length
    uint32_t count[HMAX + 2];   // codes of each length
    uint32_t index[HMAX + 2];   // position of the first symbol of each length in sym[]
    uint8_t sym[256];           // symbols ordered by (length, symbol)
};
static_assert(sizeof(DecTab) % 4 == 0, "DecTab is copied as words");

constexpr int LUT_BITS = 11;     // codes up to this length decode with one table lookup
constexpr int DEC_THREADS = 32;  // one warp per block, one chunk per thread
constexpr int MAX_LANES = 5;     // flags + up to 4 code bytes

struct DecLane {
    const uint32_t *words;       // the lane's words (4-byte aligned)
    const uint32_t *chunk_off;   // its chunk bit offsets (u64 at 4-byte boundaries)
    const DecTab *T;
    unsigned long long bit_len;
    int64_t nchunks, block0;     // first block of this lane in the launch
    Lane L;
};
struct DecArgs {
    DecLane lane[MAX_LANES];
    int nl;
};

// A u64 of the container at a 4-byte boundary (lanes after the first start on one).
__device__ __forceinline__ unsigned long long ld_u64_a4(const uint32_t *p, int64_t k) {
    return (unsigned long long)p[2 * k] | ((unsigned long long)p[2 * k + 1] << 32);
}

// Every lane in one launch: the blocks of lane l start at block0; each block builds the
// lane's LUT_BITS-bit lookup table (symbol | length << 8; 0 for a prefix of a longer code)
// in shared memory, then each thread decodes one chunk, its next bits held left-aligned in
// a 64-bit register.  Codes longer than LUT_BITS continue length by length on the
// canonical tables.  Any code that is invalid, or runs past its chunk, sets *err.
__global__ void __launch_bounds__(DEC_THREADS) k_decode(DecArgs A, uint8_t *__restrict__ dst,
                                                        uint32_t *__restrict__ err) {
    __shared__ uint16_t lut[1 << LUT_BITS];
    __shared__ DecTab tab;
    int l = 0;
    while (l + 1 < A.nl && (int64_t)blockIdx.x >= A.lane[l + 1].block0) ++l;
    const DecLane &D = A.lane[l];
    for (int k = threadIdx.x; k < (int)(sizeof(DecTab) / 4); k += DEC_THREADS)
        ((uint32_t *)&tab)[k] = ((const uint32_t *)D.T)[k];
    __syncthreads();
    for (int e = threadIdx.x; e < (1 << LUT_BITS); e += DEC_THREADS) {
        uint16_t v = 0;
        for (int len = 1; len <= LUT_BITS; ++len) {
            const uint32_t code = (uint32_t)e >> (LUT_BITS - len);
            if (code - tab.first[len] < tab.count[len]) {
                v = (uint16_t)(tab.sym[tab.index[len] + code - tab.first[len]] | (len << 8));
                break;
            }
        }
        lut[e] = v;
    }
    __syncthreads();
    const int64_t c = ((int64_t)blockIdx.x - D.block0) * DEC_THREADS + threadIdx.x;
    if (c >= D.nchunks) return;
    const int64_t nw = (int64_t)((D.bit_len + 31) >> 5);
    const uint32_t *W = D.words;
    unsigned long long pos = ld_u64_a4(D.chunk_off, c);
    const unsigned long long end = c + 1 < D.nchunks ? ld_u64_a4(D.chunk_off, c + 1) : D.bit_len;
    if (pos > end || end > D.bit_len) {
        atomicOr(err, 1u);
        return;
    }
    int64_t w = (int64_t)(pos >> 5);
    unsigned long long buf = (((unsigned long long)(w < nw ? W[w] : 0u) << 32) | (w + 1 < nw ? W[w + 1] : 0u))
                             << (pos & 31);
    int avail = 64 - (int)(pos & 31);
    w += 2;
    const int64_t i1 = min((int64_t)HCHUNK * (c + 1), D.L.n);
    for (int64_t i = (int64_t)HCHUNK * c; i < i1; ++i) {
        if (avail < 32) {
            buf |= (unsigned long long)(w < nw ? W[w] : 0u) << (32 - avail);
            avail += 32;
            ++w;
        }
        const uint16_t e = lut[buf >> (64 - LUT_BITS)];
        int len = e >> 8;
        uint8_t sym = (uint8_t)(e & 255);
        if (len == 0) {
            bool ok = false;
            for (len = LUT_BITS + 1; len <= HMAX; ++len) {
                const uint32_t code = (uint32_t)(buf >> (64 - len));
                if (code - tab.first[len] < tab.count[len]) {
                    sym = tab.sym[tab.index[len] + code - tab.first[len]];
                    ok = true;
                    break;
                }
            }
            if (!ok) {
                atomicOr(err, 1u);
                return;
            }
        }
        if (pos + len > end) {
            atomicOr(err, 1u);
            return;
        }
        dst[D.L.off + i * D.L.stride] = sym;
        buf <<= len;
        avail -= len;
        pos += len;
    }
    if (pos != end) atomicOr(err, 1u);   // the chunk ends where the next starts
}

// ---------------------------------------------------------------- host side
uint64_t rd_u64(const uint8_t *p) {
    uint64_t v = 0;
    for (int k = 0; k < 8; ++k) v |= (uint64_t)p[k] << (8 * k);
    return v;
}
uint32_t rd_u32(const uint8_t *p) {
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) v |= (uint32_t)p[k] << (8 * k);
    return v;
}
void wr_u64(uint8_t *p, uint64_t v) {
    for (int k = 0; k < 8; ++k) p[k] = (uint8_t)(v >> (8 * k));
}
void wr_u32(uint8_t *p, uint32_t v) {
    for (int k = 0; k < 4; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

// Huffman code lengths (ties: smaller node id first; symbols are ids 0..255, merged nodes
// 256, 257, ... in order of creation), limited to HMAX bits.
void huff_lengths(const unsigned long long *freq, uint8_t *len) {
    std::memset(len, 0, 256);
    std::vector<int> used;
    for (int s = 0; s < 256; ++s)
        if (freq[s]) used.push_back(s);
    if (used.empty()) return;
    if (used.size() == 1) {
        len[used[0]] = 1;
        return;
    }
    typedef std::pair<unsigned long long, int> Node;
    std::priority_queue<Node, std::vector<Node>, std::greater<Node>> pq;
    for (int s : used) pq.push(Node(freq[s], s));
    std::vector<int> parent(512, -1);
    int next = 256;
    while (pq.size() > 1) {
        const Node a = pq.top();
        pq.pop();
        const Node b = pq.top();
        pq.pop();
        parent[a.second] = next;
        parent[b.second] = next;
        pq.push(Node(a.first + b.first, next));
        ++next;
    }
    int depth[256] = {0}, maxd = 0;
    for (int s : used) {
        int d = 0;
        for (int x = s; parent[x] >= 0; x = parent[x]) ++d;
        depth[s] = d;
        maxd = std::max(maxd, d);
    }
    if (maxd <= HMAX) {
        for (int s : used) len[s] = (uint8_t)depth[s];
        return;
    }
    // fold the deeper codes into HMAX, then restore the Kraft sum: each step moves the
    // deepest code shorter than HMAX one level down, with a folded code as its sibling
    std::vector<long long> bl(HMAX + 1, 0);
    for (int s : used) bl[std::min(depth[s], HMAX)] += 1;
    long long excess = -(1ll << HMAX);
    for (int l = 1; l <= HMAX; ++l) excess += bl[l] << (HMAX - l);
    while (excess > 0) {
        int b = HMAX - 1;
        while (bl[b] == 0) --b;
        bl[b] -= 1;
        bl[b + 1] += 2;
        bl[HMAX] -= 1;
        excess -= 1;
    }
    std::vector<int> order(used);
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        return freq[x] != freq[y] ? freq[x] < freq[y] : x > y;   // rarest first, then larger symbol
    });
    size_t i = 0;
    for (int l = HMAX; l >= 1; --l)
        for (long long k = 0; k < bl[l]; ++k) len[order[i++]] = (uint8_t)l;
}

void canonical(const uint8_t *len, uint32_t *code, DecTab *tab) {
    std::vector<int> syms;
    for (int s = 0; s < 256; ++s)
        if (len[s]) syms.push_back(s);
    std::sort(syms.begin(), syms.end(), [&](int a, int b) { return len[a] != len[b] ? len[a] < len[b] : a < b; });
    uint32_t c = 0;
    int prev = 0;
    if (tab) std::memset(tab, 0, sizeof(DecTab));
    for (size_t k = 0; k < syms.size(); ++k) {
        const int s = syms[k];
        c <<= (len[s] - prev);
        prev = len[s];
        if (code) code[s] = c;
        if (tab) {
            if (tab->count[len[s]] == 0) {
                tab->first[len[s]] = c;
                tab->index[len[s]] = (uint32_t)k;
            }
            tab->count[len[s]] += 1;
            tab->sym[k] = (uint8_t)s;
        }
        ++c;
    }
}

// The lanes of an edit stream v1 with the given header.
std::vector<Lane> stream_lanes(const uint8_t *hdr, size_t nbytes) {
    const uint64_t n = rd_u64(hdr + 8);
    const uint32_t m = rd_u32(hdr + 16);
    const uint64_t fb = rd_u64(hdr + 48), codeb = rd_u64(hdr + 56);
    const int cb = (int)((m + 7) / 8);
    if (memcmp(hdr, "PCE1", 4) != 0 || rd_u32(hdr + 4) != 1 || m < 2 || m > 32 || fb != (n + 7) / 8 || codeb % (uint64_t)cb != 0 ||
        nbytes != (size_t)(HHEAD + fb + codeb))
        fail(PC_EFORMAT, "not an edit stream v1");
    std::vector<Lane> lanes;
    lanes.push_back(Lane{HHEAD, (int64_t)fb, 1});
    for (int k = 0; k < cb; ++k) lanes.push_back(Lane{(int64_t)(HHEAD + fb + k), (int64_t)(codeb / cb), cb});
    return lanes;
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" pc_status pc_huff_encode(pc_ctx *ctx, const uint8_t *in, size_t nbytes, uint8_t *out, size_t cap,
                                    size_t *out_bytes, void *stream) {
    try {
        if (!ctx || !in || !out_bytes) fail(PC_EINVAL, "pc_huff_encode: NULL argument");
        if (nbytes < (size_t)HHEAD) fail(PC_EFORMAT, "pc_huff_encode: stream shorter than its header");
        PC_CUDA(cudaSetDevice(ctx_device(ctx)));
        cudaStream_t s = (cudaStream_t)stream;
        HostScratch hs;
        struct G {
            HostScratch &h;
            ~G() {
                if (h.p) cudaFreeHost(h.p);
            }
        } g{hs};
        uint8_t hdr[HHEAD];
        memcpy(hdr, read_back(hs, in, HHEAD, s), HHEAD);
        const std::vector<Lane> lanes = stream_lanes(hdr, nbytes);
        const int nl = (int)lanes.size();
        // per lane: histogram -> lengths -> codes -> chunk bits -> offsets
        std::vector<std::vector<uint8_t>> lens(nl, std::vector<uint8_t>(256));
        std::vector<DBuf<unsigned long long>> offs(nl);
        std::vector<uint64_t> bits(nl), nch(nl);
        DBuf<unsigned long long> hist(256 * nl, s);
        PC_CUDA(cudaMemsetAsync(hist.p, 0, 256 * nl * sizeof(unsigned long long), s));
        for (int l = 0; l < nl; ++l) {
            if (lanes[l].n > 0) {
                k_hist<<<(unsigned)std::min<int64_t>(1024, cdiv(lanes[l].n, 256)), 256, 0, s>>>(in, lanes[l],
                                                                                             hist.p + 256 * l);
                PC_CHECK_LAUNCH();
            }
        }
        std::vector<unsigned long long> hh(256 * nl);
        memcpy(hh.data(), read_back(hs, hist.p, 256 * nl * sizeof(unsigned long long), s), hh.size() * 8);
        DBuf<uint8_t> dlen(256 * nl, s);
        DBuf<uint32_t> dcode(256 * nl, s);
        std::vector<uint32_t> codes(256 * nl);
        for (int l = 0; l < nl; ++l) {
            huff_lengths(hh.data() + 256 * l, lens[l].data());
            canonical(lens[l].data(), codes.data() + 256 * l, nullptr);
        }
        {
            uint8_t *h = (uint8_t *)host_scratch(hs, 256 * nl * 5);
            for (int l = 0; l < nl; ++l) memcpy(h + 256 * l, lens[l].data(), 256);
            memcpy(h + 256 * nl, codes.data(), 256 * nl * 4);
            PC_CUDA(cudaMemcpyAsync(dlen.p, h, 256 * nl, cudaMemcpyHostToDevice, s));
            PC_CUDA(cudaMemcpyAsync(dcode.p, h + 256 * nl, 256 * nl * 4, cudaMemcpyHostToDevice, s));
            PC_CUDA(cudaStreamSynchronize(s));
        }
        DBuf<unsigned long long> cbits;
        for (int l = 0; l < nl; ++l) {
            nch[l] = (uint64_t)cdiv(lanes[l].n, HCHUNK);
            offs[l].alloc(std::max<uint64_t>(1, nch[l] + 1), s);
            if (nch[l] == 0) {
                bits[l] = 0;
                continue;
            }
            cbits.alloc(nch[l], s);
            k_chunk_bits<<<(unsigned)nch[l], 256, 0, s>>>(in, lanes[l], dlen.p + 256 * l, cbits.p);
            PC_CHECK_LAUNCH();
            scan_exclusive_u64((const uint64_t *)cbits.p, (uint64_t *)offs[l].p, (int64_t)nch[l],
                               (uint64_t *)(offs[l].p + nch[l]), s);
            bits[l] = *(const unsigned long long *)read_back(hs, offs[l].p + nch[l], 8, s);
        }
        // container layout
        std::vector<size_t> lane_at(nl), words_at(nl);
        size_t total = CONT_HEAD;
        for (int l = 0; l < nl; ++l) {
            lane_at[l] = total;
            total += 24 + 256 + 8 * nch[l];
            words_at[l] = total;
            total += 4 * ((bits[l] + 31) / 32);
        }
        *out_bytes = total;
        if (!out) return PC_OK;
        if (cap < total) fail(PC_EINVAL, "pc_huff_encode: output buffer too small");
        if ((uintptr_t)out % 4 != 0) fail(PC_EINVAL, "pc_huff_encode: out_dev must be 4-byte aligned");
        PC_CUDA(cudaMemsetAsync(out, 0, total, s));
        {
            const size_t hb = CONT_HEAD + nl * (24 + 256);
            uint8_t *h = (uint8_t *)host_scratch(hs, hb);
            memset(h, 0, hb);
            memcpy(h, "PCH1", 4);
            wr_u32(h + 4, 1);
            wr_u64(h + 8, nbytes);
            wr_u32(h + 16, (uint32_t)nl);
            wr_u32(h + 20, HCHUNK);
            wr_u32(h + 24, HMAX);
            memcpy(h + 32, hdr, HHEAD);
            PC_CUDA(cudaMemcpyAsync(out, h, CONT_HEAD, cudaMemcpyHostToDevice, s));
            for (int l = 0; l < nl; ++l) {
                uint8_t *lh = h + CONT_HEAD + l * (24 + 256);
                wr_u64(lh, (uint64_t)lanes[l].n);
                wr_u64(lh + 8, bits[l]);
                wr_u64(lh + 16, nch[l]);
                memcpy(lh + 24, lens[l].data(), 256);
                PC_CUDA(cudaMemcpyAsync(out + lane_at[l], lh, 24 + 256, cudaMemcpyHostToDevice, s));
                if (nch[l])
                    PC_CUDA(cudaMemcpyAsync(out + lane_at[l] + 24 + 256, offs[l].p, 8 * nch[l],
                                            cudaMemcpyDeviceToDevice, s));
            }
            for (int l = 0; l < nl; ++l) {
                if (nch[l] == 0) continue;
                k_encode<<<(unsigned)nch[l], 256, 0, s>>>(in, lanes[l], dlen.p + 256 * l, dcode.p + 256 * l,
                                                          offs[l].p, (uint32_t *)(out + words_at[l]));
                PC_CHECK_LAUNCH();
            }
            PC_CUDA(cudaStreamSynchronize(s));   // the staging area is reused on return
        }
        return PC_OK;
    } catch (const Fail &f) {
        return f.st;
    } catch (...) {
        set_error("pc_huff_encode: unexpected failure");
        return PC_ECUDA;
    }
}

extern "C" pc_status pc_huff_decode(pc_ctx *ctx, const uint8_t *in, size_t nbytes, uint8_t *out, size_t cap,
                                    size_t *out_bytes, void *stream) {
    try {
        if (!ctx || !in || !out_bytes) fail(PC_EINVAL, "pc_huff_decode: NULL argument");
        if (nbytes < (size_t)CONT_HEAD) fail(PC_EFORMAT, "pc_huff_decode: shorter than the container header");
        if ((uintptr_t)in % 4 != 0) fail(PC_EINVAL, "pc_huff_decode: in_dev must be 4-byte aligned");
        PC_CUDA(cudaSetDevice(ctx_device(ctx)));
        cudaStream_t s = (cudaStream_t)stream;
        HostScratch hs;
        struct G {
            HostScratch &h;
            ~G() {
                if (h.p) cudaFreeHost(h.p);
            }
        } g{hs};
        uint8_t head[CONT_HEAD];
        memcpy(head, read_back(hs, in, CONT_HEAD, s), CONT_HEAD);
        if (memcmp(head, "PCH1", 4) != 0 || rd_u32(head + 4) != 1 || rd_u32(head + 20) != HCHUNK ||
            rd_u32(head + 24) != HMAX)
            fail(PC_EFORMAT, "pc_huff_decode: not a PCH1 container");
        const uint64_t raw = rd_u64(head + 8);
        const std::vector<Lane> lanes = stream_lanes(head + 32, raw);
        if ((int)rd_u32(head + 16) != (int)lanes.size()) fail(PC_EFORMAT, "pc_huff_decode: lane count");
        *out_bytes = raw;
        if (!out) return PC_OK;
        if (cap < raw) fail(PC_EINVAL, "pc_huff_decode: output buffer too small");
        PC_CUDA(cudaMemcpyAsync(out, in + 32, HHEAD, cudaMemcpyDeviceToDevice, s));
        DBuf<uint32_t> err(1, s);
        PC_CUDA(cudaMemsetAsync(err.p, 0, 4, s));
        const int nl = (int)lanes.size();
        if (nl > MAX_LANES) fail(PC_EFORMAT, "pc_huff_decode: lane count");
        DBuf<DecTab> tabs(nl, s);
        std::vector<DecTab> ht(nl);
        DecArgs args;
        memset(&args, 0, sizeof(args));
        args.nl = nl;
        int64_t blocks = 0;
        size_t at = CONT_HEAD;
        for (int l = 0; l < nl; ++l) {
            if (at + 24 + 256 > nbytes) fail(PC_EFORMAT, "pc_huff_decode: truncated lane header");
            uint8_t lh[24 + 256];
            memcpy(lh, read_back(hs, in + at, sizeof(lh), s), sizeof(lh));
            const uint64_t n = rd_u64(lh), bits = rd_u64(lh + 8), nch = rd_u64(lh + 16);
            if ((int64_t)n != lanes[l].n || nch != (uint64_t)cdiv((int64_t)n, HCHUNK))
                fail(PC_EFORMAT, "pc_huff_decode: lane size");
            uint64_t kraft = 0;   // sum of 2^(HMAX - length): at most 2^HMAX for a prefix code
            for (int k = 0; k < 256; ++k) {
                if (lh[24 + k] > HMAX) fail(PC_EFORMAT, "pc_huff_decode: code length");
                if (lh[24 + k]) kraft += 1ull << (HMAX - lh[24 + k]);
            }
            if (kraft > (1ull << HMAX) || (n > 0 && kraft == 0)) fail(PC_EFORMAT, "pc_huff_decode: not a prefix code");
            if (bits > 8ull * nbytes) fail(PC_EFORMAT, "pc_huff_decode: bit length");
            canonical(lh + 24, nullptr, &ht[l]);
            const size_t off_at = at + 24 + 256, words_at = off_at + 8 * nch;
            at = words_at + 4 * ((bits + 31) / 32);
            if (at > nbytes) fail(PC_EFORMAT, "pc_huff_decode: truncated lane");
            DecLane &D = args.lane[l];
            D.words = (const uint32_t *)(in + words_at);
            D.chunk_off = (const uint32_t *)(in + off_at);
            D.T = tabs.p + l;
            D.bit_len = bits;
            D.nchunks = (int64_t)nch;
            D.block0 = blocks;
            D.L = lanes[l];
            blocks += cdiv((int64_t)nch, DEC_THREADS);
        }
        PC_CUDA(cudaMemcpyAsync(tabs.p, ht.data(), nl * sizeof(DecTab), cudaMemcpyHostToDevice, s));
        if (blocks > 0) {
            k_decode<<<(unsigned)blocks, DEC_THREADS, 0, s>>>(args, out, err.p);
            PC_CHECK_LAUNCH();
        }
        if (*(const uint32_t *)read_back(hs, err.p, 4, s)) fail(PC_EFORMAT, "pc_huff_decode: invalid code");
        return PC_OK;
    } catch (const Fail &f) {
        return f.st;
    } catch (...) {
        set_error("pc_huff_decode: unexpected failure");
        return PC_ECUDA;
    }
}
