// scan.cu -- exclusive prefix sums written for this library (no CUB).
//
// Reduce-then-scan over tiles of SCAN_THREADS * SCAN_ITEMS elements: one
// kernel reduces every tile, the tile sums are scanned (recursively, or by a
// single block when they fit one tile), and a second kernel rescans each tile
// with its offset.  out has n+1 entries; out[n] is the total.  Used for the
// community offsets of aggregation (Algorithm 5: exclusiveScan), community
// renumbering and CSR construction.
#include "common.cuh"

namespace gsp {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr uint64_t SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T> __device__ T block_exclusive_scan(T v, T *warp_tot, T &total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : T(0);
        T s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = s - t;
        if (lane == SCAN_THREADS / 32 - 1) warp_tot[SCAN_THREADS / 32] = s;
    }
    __syncthreads();
    T r = warp_tot[wid] + x - v;
    total = warp_tot[SCAN_THREADS / 32];
    __syncthreads();
    return r;
}

template <typename In, typename Out>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_reduce(const In *__restrict__ in, uint64_t n,
                                                              Out *__restrict__ partial) {
    __shared__ Out scratch[32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    Out s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        uint64_t idx = base + (uint64_t)k * SCAN_THREADS + threadIdx.x;
        if (idx < n) s += (Out)in[idx];
    }
    s = block_sum<Out>(s, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Rescan each tile; thread t owns elements [t*ITEMS, t*ITEMS+ITEMS) of the
// tile, staged through shared memory so that global accesses coalesce.
template <typename In, typename Out>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const In *__restrict__ in, uint64_t n,
                                                            const Out *__restrict__ offs,
                                                            Out *__restrict__ out, int write_total) {
    __shared__ Out tile[SCAN_TILE];
    __shared__ Out warp_tot[SCAN_THREADS / 32 + 1];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        uint64_t li = (uint64_t)k * SCAN_THREADS + threadIdx.x;
        tile[li] = (base + li < n) ? (Out)in[base + li] : Out(0);
    }
    __syncthreads();
    Out v[SCAN_ITEMS];
    Out s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = tile[threadIdx.x * SCAN_ITEMS + k];
        s += v[k];
    }
    Out total;
    Out run = block_exclusive_scan<Out>(s, warp_tot, total) + (offs ? offs[blockIdx.x] : Out(0));
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        tile[threadIdx.x * SCAN_ITEMS + k] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        uint64_t li = (uint64_t)k * SCAN_THREADS + threadIdx.x;
        if (base + li < n) out[base + li] = tile[li];
    }
    if (write_total && threadIdx.x == SCAN_THREADS - 1 && blockIdx.x == gridDim.x - 1)
        out[n] = run;  // run = exclusive prefix after the tile's last element
}

template <typename In, typename Out> static void scan_impl(const In *in, Out *out, uint64_t n, cudaStream_t s) {
    if (n == 0) {
        GSP_CUDA(cudaMemsetAsync(out, 0, sizeof(Out), s));
        return;
    }
    uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_tile_scan<In, Out><<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out, 1);
        GSP_CHECK_LAUNCH();
        return;
    }
    size_t mk = arena().mark();
    Out *partial = arena().get<Out>(tiles + 1);
    k_tile_reduce<In, Out><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, partial);
    GSP_CHECK_LAUNCH();
    scan_impl<Out, Out>(partial, partial, tiles, s);  // in place is safe: tile-local staging
    k_tile_scan<In, Out><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, partial, out, 1);
    GSP_CHECK_LAUNCH();
    arena().release(mk);
}

void exclusive_scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, cudaStream_t s) {
    scan_impl<uint32_t, uint64_t>(in, out, n, s);
}
void exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s) {
    scan_impl<uint64_t, uint64_t>(in, out, n, s);
}
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, cudaStream_t s) {
    scan_impl<uint32_t, uint32_t>(in, out, n, s);
}
void exclusive_scan_u8_to_u32(const uint8_t *in, uint32_t *out, uint64_t n, cudaStream_t s) {
    scan_impl<uint8_t, uint32_t>(in, out, n, s);
}

}  // namespace gsp
