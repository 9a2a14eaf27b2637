// sort.cu -- stable LSD radix sort of 64-bit keys with 32-bit payloads,
// written for this library (no CUB).  8-bit digits; per pass: a tile
// histogram kernel, a scan of the digit-major histogram matrix, and a
// scatter kernel that ranks every element among the equal digits of its tile
// (warp match + per-warp counts), so that the pass is stable.
#include "common.cuh"

namespace gsp {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;
constexpr uint64_t RS_TILE = (uint64_t)RS_THREADS * RS_ROUNDS;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *__restrict__ keys, uint64_t n,
                                                        int shift, uint32_t *__restrict__ hist,
                                                        uint32_t tiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        uint64_t i = base + (uint64_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

template <typename V>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t *__restrict__ keys,
                                                           const V *__restrict__ vals, uint64_t n,
                                                           int shift, const uint32_t *__restrict__ offs,
                                                           uint32_t tiles, uint64_t *__restrict__ keys_out,
                                                           V *__restrict__ vals_out) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t run[256];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    run[threadIdx.x] = offs[(uint64_t)threadIdx.x * tiles + blockIdx.x];
    for (int r = 0; r < RS_ROUNDS; r++) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        uint64_t i = base + (uint64_t)r * RS_THREADS + threadIdx.x;
        bool valid = i < n;
        uint64_t k = valid ? keys[i] : 0;
        uint32_t dig = valid ? (uint32_t)((k >> shift) & 0xFF) : 256u + lane;  // invalid lanes never match
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig);
        uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[wid][dig] = __popc(peers);
        __syncthreads();
        {   // per digit: prefix over warps, offset by the running tile count
            uint32_t d = threadIdx.x;
            uint32_t acc = run[d];
#pragma unroll
            for (int w = 0; w < RS_WARPS; w++) {
                uint32_t c = wcnt[w][d];
                wcnt[w][d] = acc;
                acc += c;
            }
            run[d] = acc;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wcnt[wid][dig] + rank;
            keys_out[pos] = k;
            vals_out[pos] = vals[i];
        }
        __syncthreads();
    }
}


template <typename V>
static void radix_sort_impl(uint64_t *keys, V *vals, uint64_t *keys_alt, V *vals_alt, uint64_t n, int bits,
                            cudaStream_t s) {
    GSP_REQUIRE(n < (1ull << 32), "radix sort supports fewer than 2^32 elements");
    if (n <= 1 || bits <= 0) return;
    uint32_t tiles = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
    size_t mk = arena().mark();
    uint32_t *hist = arena().get<uint32_t>((size_t)256 * tiles + 1);
    uint64_t *ks = keys, *kd = keys_alt;
    V *vs = vals, *vd = vals_alt;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        k_rs_hist<<<tiles, RS_THREADS, 0, s>>>(ks, n, shift, hist, tiles);
        GSP_CHECK_LAUNCH();
        exclusive_scan_u32(hist, hist, (uint64_t)256 * tiles, s);
        k_rs_scatter<V><<<tiles, RS_THREADS, 0, s>>>(ks, vs, n, shift, hist, tiles, kd, vd);
        GSP_CHECK_LAUNCH();
        uint64_t *tk = ks; ks = kd; kd = tk;
        V *tv = vs; vs = vd; vd = tv;
    }
    if (ks != keys) {
        GSP_CUDA(cudaMemcpyAsync(keys, ks, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        GSP_CUDA(cudaMemcpyAsync(vals, vs, n * sizeof(V), cudaMemcpyDeviceToDevice, s));
    }
    arena().release(mk);
}

void radix_sort_u64_f32(uint64_t *keys, float *vals, uint64_t *keys_alt, float *vals_alt, uint64_t n, int bits,
                        cudaStream_t s) {
    radix_sort_impl<float>(keys, vals, keys_alt, vals_alt, n, bits, s);
}
void radix_sort_u64_u32(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n,
                        int bits, cudaStream_t s) {
    radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, bits, s);
}

}  // namespace gsp
