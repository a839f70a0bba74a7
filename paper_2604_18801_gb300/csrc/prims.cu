// Device-wide primitives: exclusive scan and a stable LSD radix sort.
//
// Both are plain three-phase designs (tile reduce -> scan of tile totals ->
// tile scan / scatter) with deterministic results: the sort is stable, so
// equal keys keep their input order, and the scan adds in a fixed order.
#include "common.cuh"

namespace pc {

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; the block total goes to *total.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T *total) {
    constexpr int NW = SCAN_THREADS / 32;
    __shared__ T wsum[NW];
    __shared__ T tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const T inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const T x = lane < NW ? wsum[lane] : T(0);
        const T xi = warp_incl_scan(x);
        if (lane < NW) wsum[lane] = xi - x;
        if (lane == NW - 1) tot = xi;
    }
    __syncthreads();
    const T excl = wsum[w] + inc - v;
    *total = tot;
    __syncthreads();
    return excl;
}

template <class T>
__global__ void k_tile_reduce(const T *__restrict__ in, T *__restrict__ sums, int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    T tot;
    block_excl_scan<T>(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class T>
__global__ void k_tile_scan(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                            const T *__restrict__ tile_off, T *total_dev) {
    __shared__ T sh[SCAN_TILE];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        sh[k * SCAN_THREADS + threadIdx.x] = i < n ? in[i] : T(0);
    }
    __syncthreads();
    T loc[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        loc[k] = sh[threadIdx.x * SCAN_ITEMS + k];
        s += loc[k];
    }
    T tot;
    T ex = block_excl_scan<T>(s, &tot);
    const T off = tile_off ? tile_off[blockIdx.x] : T(0);
    ex += off;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        sh[threadIdx.x * SCAN_ITEMS + k] = ex;
        ex += loc[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) out[i] = sh[k * SCAN_THREADS + threadIdx.x];
    }
    if (total_dev && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_dev = off + tot;
}

template <class T>
void scan_impl(const T *in, T *out, int64_t n, T *total_dev, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) PC_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(T), s));
        return;
    }
    const int64_t tiles = cdiv(n, SCAN_TILE);
    if (tiles == 1) {
        k_tile_scan<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr, total_dev);
        PC_CHECK_LAUNCH();
        return;
    }
    DBuf<T> sums(tiles, s), offs(tiles, s);
    k_tile_reduce<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, sums.p, n);
    PC_CHECK_LAUNCH();
    scan_impl<T>(sums.p, offs.p, tiles, nullptr, s);
    k_tile_scan<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs.p, total_dev);
    PC_CHECK_LAUNCH();
}

// ------------------------------- radix sort -------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

template <class K, class O>
__global__ void k_rs_hist(const K *__restrict__ keys, int64_t n, int shift, O *__restrict__ hist,
                          int64_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int k = 0; k < RS_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// O: type of the output positions (32-bit below 2^32 elements, else 64-bit).
template <class K, bool HAS_V, class O>
__global__ void k_rs_scatter(const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
                             uint32_t *__restrict__ vout, int64_t n, int shift,
                             const O *__restrict__ off, int64_t ntiles) {
    __shared__ O run[256];
    __shared__ O wc[RS_WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    run[tid] = off[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) wc[q][tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + (int64_t)r * RS_THREADS + tid;
        const bool valid = i < n;
        K k = valid ? kin[i] : K(0);
        uint32_t v = (HAS_V && valid) ? vin[i] : 0u;
        const uint32_t d = valid ? ((uint32_t)(k >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wc[w][d] = (O)__popc(peers);
        __syncthreads();
        {
            O s = run[tid];
#pragma unroll
            for (int q = 0; q < RS_WARPS; ++q) {
                const O c = wc[q][tid];
                wc[q][tid] = s;
                s += c;
            }
            run[tid] = s;
        }
        __syncthreads();
        if (valid) {
            const O pos = wc[w][d] + (O)rank;
            kout[pos] = k;
            if (HAS_V) vout[pos] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RS_WARPS; ++q) wc[q][tid] = 0;
        __syncthreads();
    }
}

template <class K, class O>
void radix_passes(K *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    const int64_t ntiles = cdiv(n, RS_TILE);
    DBuf<K> k2(n, s);
    DBuf<uint32_t> v2(vals ? n : 0, s);
    DBuf<O> hist(256 * ntiles, s);
    K *ka = keys, *kb = k2.p;
    uint32_t *va = vals, *vb = v2.p;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        k_rs_hist<K, O><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, hist.p, ntiles);
        PC_CHECK_LAUNCH();
        scan_impl<O>(hist.p, hist.p, 256 * ntiles, nullptr, s);
        if (vals)
            k_rs_scatter<K, true, O><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, hist.p,
                                                                             ntiles);
        else
            k_rs_scatter<K, false, O><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, nullptr, kb, nullptr, n, shift,
                                                                              hist.p, ntiles);
        PC_CHECK_LAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {
        PC_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
        if (vals) PC_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

template <class K>
void radix_impl(K *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    // positions (histogram offsets) are 32-bit below 2^32 elements and 64-bit above
    if (n < (int64_t)0xffffffffll) radix_passes<K, uint32_t>(keys, vals, n, bits, s);
    else radix_passes<K, unsigned long long>(keys, vals, n, bits, s);
}

__global__ void k_fill_u32(uint32_t *p, uint32_t v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void k_iota_u32(uint32_t *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

}  // namespace

void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev, cudaStream_t s) {
    scan_impl<uint32_t>(in, out, n, total_dev, s);
}
void scan_exclusive_u64(const uint64_t *in, uint64_t *out, int64_t n, uint64_t *total_dev, cudaStream_t s) {
    scan_impl<unsigned long long>((const unsigned long long *)in, (unsigned long long *)out, n,
                                  (unsigned long long *)total_dev, s);
}
void radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    radix_impl<uint32_t>(keys, vals, n, bits, s);
}
void radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    radix_impl<uint64_t>(keys, vals, n, bits, s);
}
void fill_u32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int g = (int)std::min<int64_t>(cdiv(n, 256), (int64_t)num_sms() * 8);
    k_fill_u32<<<g, 256, 0, s>>>(p, v, n);
    PC_CHECK_LAUNCH();
}
void iota_u32(uint32_t *p, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int g = (int)std::min<int64_t>(cdiv(n, 256), (int64_t)num_sms() * 8);
    k_iota_u32<<<g, 256, 0, s>>>(p, n);
    PC_CHECK_LAUNCH();
}

}  // namespace pc
