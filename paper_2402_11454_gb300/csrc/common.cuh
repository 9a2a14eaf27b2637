// common.cuh -- shared device/host helpers of libgsp (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/gsp.h"

namespace gsp {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
struct Error {
    gsp_status status;
};

#define GSP_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            ::gsp::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            throw ::gsp::Error{e_ == cudaErrorMemoryAllocation ? GSP_ERR_NOMEM : GSP_ERR_CUDA}; \
        }                                                                                   \
    } while (0)

void count_launch();
#define GSP_CHECK_LAUNCH()          \
    do {                            \
        ::gsp::count_launch();      \
        GSP_CUDA(cudaGetLastError()); \
    } while (0)

#define GSP_REQUIRE(cond, ...)                                                              \
    do {                                                                                    \
        if (!(cond)) {                                                                      \
            ::gsp::set_error(__VA_ARGS__);                                                  \
            throw ::gsp::Error{GSP_ERR_INVALID};                                            \
        }                                                                                   \
    } while (0)

// ------------------------------------------------------------ workspace
// One device workspace per device, grown on demand (cudaMalloc of new
// chunks) and kept across calls.  Bump allocation with 256-byte alignment;
// mark()/release() bracket temporaries, reset() starts a call.
class Arena {
  public:
    void *alloc(size_t bytes);
    template <typename T> T *get(size_t count) { return static_cast<T *>(alloc(count * sizeof(T))); }
    size_t mark();
    void release(size_t m);
    void reset();
    void free_all();
};
Arena &arena();
Arena &io_arena();  // host-buffer entry points stage their device copies here

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int sm_count();  // SMs of the current device (cached per device)
// Grid caps are given in blocks per SM: sms(k) = k blocks on every SM.
inline unsigned sms(unsigned per_sm) { return per_sm * (unsigned)sm_count(); }
// Grid of a grid-stride kernel that fits the device at once: the blocks of
// `fn` resident per SM (registers and shared memory), at most per_sm_cap,
// times the SM count.  Launching more blocks than are resident leaves a
// partial second generation of blocks running on idle SMs.
unsigned resident_grid(const void *fn, int threads, size_t dyn_smem, unsigned per_sm_cap);
inline unsigned grid_for(uint64_t work, unsigned block, unsigned cap = 0) {
    if (!cap) cap = sms(16);
    uint64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// --------------------------------------------------------- device helpers
// Row of CSR entry p (offsets non-decreasing, off[n] > p): the last row with
// off[row] <= p, searched forward from a row r known to have off[r] <= p:
// first the row itself and the next, then by doubling the step and halving
// it.  Consecutive entries of a lane lie a row or so apart, so the search
// mostly ends after one or two cached loads.
__device__ __forceinline__ uint32_t row_from(const uint64_t *__restrict__ off, uint32_t n, uint64_t p, uint32_t r) {
    if ((uint64_t)r + 1 >= n || __ldg(off + r + 1) > p) return r;
    r += 1;
    uint64_t step = 1;
    while ((uint64_t)r + step < n && __ldg(off + r + step) <= p) {
        r += (uint32_t)step;
        step <<= 1;
    }
    for (step >>= 1; step > 0; step >>= 1)
        if ((uint64_t)r + step < n && __ldg(off + r + step) <= p) r += (uint32_t)step;
    return r;
}

// The same row by bisection over all rows (a block's first entry).
__device__ __forceinline__ uint32_t row_of(const uint64_t *__restrict__ off, uint32_t n, uint64_t p) {
    uint32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo + 1) / 2;
        if (__ldg(off + mid) <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double wload(const float *w, uint64_t e) { return (double)__ldg(w + e); }
__device__ __forceinline__ double wload(const double *w, uint64_t e) { return __ldg(w + e); }
__device__ __forceinline__ float wloadf(const float *w, uint64_t e) { return __ldg(w + e); }
__device__ __forceinline__ float wloadf(const double *w, uint64_t e) { return (float)__ldg(w + e); }

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Block-wide sum; every thread gets the result.  `scratch` holds >= 32 T.
template <typename T> __device__ T block_sum(T v, T *scratch) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    T t = (threadIdx.x < (unsigned)nw) ? scratch[threadIdx.x] : T(0);
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) scratch[0] = t;
    __syncthreads();
    T r = scratch[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) { return x * 0x9E3779B1u; }

// Host launch helpers (scan.cu)
void exclusive_scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, cudaStream_t s);
void exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s);
void exclusive_scan_u8_to_u32(const uint8_t *in, uint32_t *out, uint64_t n, cudaStream_t s);
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, cudaStream_t s);

// radix sort (sort.cu): sorts (keys, vals) in place over bits [0, bits) using
// alternate buffers of the same size; stable.
void radix_sort_u64_f32(uint64_t *keys, float *vals, uint64_t *keys_alt, float *vals_alt, uint64_t n,
                        int bits, cudaStream_t s);
void radix_sort_u64_u32(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n,
                        int bits, cudaStream_t s);

}  // namespace gsp
