// Internal definitions shared by the CUDA translation units of libpc.
// (Nothing here is visible through the C ABI in include/pc.h.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>

#include "../../include/pc.h"

namespace pc {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
struct Fail {
    pc_status st;
};
#define PC_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            ::pc::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));            \
            throw ::pc::Fail{e_ == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA};       \
        }                                                                                   \
    } while (0)
void count_launch();
void add_launches(int64_t k);   // graph replays (k > 0) and captured launches that did not run (k < 0)
#define PC_CHECK_LAUNCH()             \
    do {                              \
        ::pc::count_launch();         \
        PC_CUDA(cudaGetLastError());  \
    } while (0)

// Device error word bits (set by kernels with atomicOr, read by the host).
enum : uint32_t {
    ERR_NONFINITE = 1u,
    ERR_BOUND = 2u,
    ERR_OUTSIDE_BOX = 4u,
    ERR_UF_RETRY = 8u,      // a union-find retry loop exceeded its bound
    ERR_INDEX = 16u,        // an index check failed (should never happen)
    ERR_VFULL = 32u,        // the count pass's buffer of vulnerable pairs is full (the emission pass runs)
};

// ---------------------------------------------------------------------------
// Derived constants (Sec. 3.1 window, Sec. 3.3 quantisation / tight margin)
// ---------------------------------------------------------------------------
struct Consts {
    // float32 link-test bounds on the canonical d2
    float b2, lo2, hi2;
    float L[3];            // periodic box lengths
    int periodic;
    // grid
    float origin[3];
    float inv_w[3];
    int nc[3];
    int key_bits;
    int64_t ncells;
    // PGD (float32 on the device)
    float thr_link, thr_non;   // b -/+ delta_t
    float xi_box;
    float alpha, beta1, beta2, eps_adam;
    // double copies kept for the host
    double xi, b, eps_q, u, dt, xi_box_d, M;
    // periodic boxes: a particle whose position lies in [in_lo, in_hi] on every axis has
    // no active pair that wraps (set only when every original position is inside the box)
    int interior_ok;
    double in_lo[3], in_hi[3];
};

// Canonical float32 difference with minimum image (exact: one add/sub of L when |d| > L/2).
__device__ __forceinline__ float cdiff(float a, float b, bool periodic, float L) {
    float d = __fsub_rn(a, b);
    if (periodic) {
        const float h = 0.5f * L;
        if (d > h) d = __fsub_rn(d, L);
        else if (d < -h) d = __fadd_rn(d, L);
    }
    return d;
}

// Canonical squared distance: (dx*dx + dy*dy) + dz*dz, each op rounded, no FMA.
__device__ __forceinline__ float cdist2(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ---------------------------------------------------------------------------
// Stream-ordered device temporaries
// ---------------------------------------------------------------------------
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = 0;
    DBuf() = default;
    DBuf(size_t count, cudaStream_t st) { alloc(count, st); }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        if (count) PC_CUDA(cudaMallocAsync((void **)&p, count * sizeof(T), st));
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    ~DBuf() { release(); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
        return *this;
    }
};

// Pinned host scratch for small device->host reads.
struct HostScratch {
    void *p = nullptr;
    size_t cap = 0;
};

// ---------------------------------------------------------------------------
// Primitives (prims.cu)
// ---------------------------------------------------------------------------
// Exclusive scan of n unsigned values; returns nothing; total written to *total_dev if non-null.
void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev, cudaStream_t s);
void scan_exclusive_u64(const uint64_t *in, uint64_t *out, int64_t n, uint64_t *total_dev, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the key.
// keys/vals are sorted in place (temporaries taken from the stream pool).  vals may be null.
void radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s);
void radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s);
// Fill helpers
void fill_u32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t s);
void iota_u32(uint32_t *p, int64_t n, cudaStream_t s);

int num_sms();
inline int ceil_log2(uint64_t x) {
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace pc
