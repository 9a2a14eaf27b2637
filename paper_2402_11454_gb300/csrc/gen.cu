// gen.cu -- seeded synthetic graphs drawn on the device (R-MAT, batched
// planted partition, 2-D grid), bit-identical to the host generators of the
// Python package: the same counter-based SplitMix64 stream (Steele, Lea and
// Flood, OOPSLA 2014), integer-only draws, and the same merge rule.
//
// Each generator writes both directions of every sampled pair as a 64-bit key
// (src << b | dst), self-loops as an all-ones key; one stable radix sort,
// a run-length merge that keeps the smallest weight of each pair, and a count
// + exclusive scan give the symmetric CSR.  These are input generators, not
// part of the community-detection method.
#include <math.h>

#include <vector>

#include "internal.cuh"

namespace gsp {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint64_t STREAM_MUL = 0xD1B54A32D192ED03ull;
constexpr uint64_t STREAM_RMAT = 1, STREAM_PLANTED = 2, STREAM_GRID_KEEP = 3, STREAM_GRID_WEIGHT = 4,
                   STREAM_GRID_LONG = 5;
constexpr uint64_t INVALID_KEY = ~0ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return mix64(seed * GAMMA + stream * STREAM_MUL);
}
__device__ __forceinline__ uint64_t rand_u64(uint64_t key, uint64_t ctr) { return mix64(key + (ctr + 1) * GAMMA); }
__device__ __forceinline__ uint64_t uniform_int(uint64_t r, uint64_t N) { return ((r >> 32) * N) >> 32; }

__device__ __forceinline__ void emit_pair(uint64_t *keys, float *vals, uint64_t slot, uint64_t u, uint64_t v,
                                          float w, int b) {
    if (u == v) {
        keys[2 * slot] = INVALID_KEY;
        keys[2 * slot + 1] = INVALID_KEY;
    } else {
        keys[2 * slot] = (u << b) | v;
        keys[2 * slot + 1] = (v << b) | u;
    }
    vals[2 * slot] = w;
    vals[2 * slot + 1] = w;
}

__global__ void k_gen_rmat(uint64_t S, int scale, uint64_t key, uint64_t t1, uint64_t t2, uint64_t t3, int b,
                           uint64_t *keys, float *vals) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < S; e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t u = 0, v = 0;
        for (int l = 0; l < scale; l++) {
            uint64_t r = rand_u64(key, e * (uint64_t)scale + l) >> 11;
            uint64_t bit = 1ull << (scale - 1 - l);
            if (r >= t2) u |= bit;
            if ((r >= t1 && r < t2) || r >= t3) v |= bit;
        }
        emit_pair(keys, vals, e, u, v, 1.0f, b);
    }
}

struct PlantedParams {
    const uint64_t *n, *k, *p53, *key, *vbase, *ebase;
    uint32_t G;
};

__global__ void k_gen_planted(PlantedParams P, uint64_t S, int b, uint64_t *keys, float *vals) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < S; t += (uint64_t)gridDim.x * blockDim.x) {
        // graph of sample t: last g with ebase[g] <= t
        uint32_t lo = 0, hi = P.G - 1;
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (P.ebase[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        uint32_t g = lo;
        uint64_t e = t - P.ebase[g];
        uint64_t n = P.n[g], k = P.k[g], key = P.key[g];
        uint64_t r0 = rand_u64(key, 4 * e) >> 11;
        uint64_t r1 = rand_u64(key, 4 * e + 1);
        uint64_t r2 = rand_u64(key, 4 * e + 2);
        uint64_t r3 = rand_u64(key, 4 * e + 3);
        uint64_t u, v;
        if (r0 < P.p53[g]) {
            uint64_t c = uniform_int(r1, k);
            uint64_t sz = (n - c + k - 1) / k;
            u = c + k * uniform_int(r2, sz);
            v = c + k * uniform_int(r3, sz);
        } else {
            u = uniform_int(r2, n);
            v = uniform_int(r3, n);
        }
        emit_pair(keys, vals, t, u + P.vbase[g], v + P.vbase[g], 1.0f, b);
    }
}

__device__ __forceinline__ float grid_weight(uint64_t r, double lo, double hi) {
    double x = (double)(r >> 40) * 0x1p-24;
    return __double2float_rn(__dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), x)));
}

__global__ void k_gen_grid(uint32_t R, uint32_t Cc, uint64_t remove53, uint64_t L, double lo, double hi,
                           uint64_t seed, int b, uint64_t *keys, float *vals) {
    uint64_t nh = (uint64_t)R * (Cc - 1), nv = (uint64_t)(R - 1) * Cc, E = nh + nv;
    uint64_t N = (uint64_t)R * Cc;
    uint64_t kk = stream_key(seed, STREAM_GRID_KEEP), kw = stream_key(seed, STREAM_GRID_WEIGHT),
             kl = stream_key(seed, STREAM_GRID_LONG);
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E + L;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t u, v;
        float w = grid_weight(rand_u64(kw, e), lo, hi);
        if (e < E) {
            if (e < nh) {
                uint64_t r = e / (Cc - 1), c = e % (Cc - 1);
                u = r * Cc + c;
                v = u + 1;
            } else {
                u = e - nh;
                v = u + Cc;
            }
            if ((rand_u64(kk, e) >> 11) < remove53) u = v;  // removed: dropped like a self-loop
        } else {
            uint64_t t = e - E;
            u = uniform_int(rand_u64(kl, 2 * t), N);
            v = uniform_int(rand_u64(kl, 2 * t + 1), N);
        }
        emit_pair(keys, vals, e, u, v, w, b);
    }
}

// Run heads of the sorted keys; at each head, the smallest weight of its run.
__global__ void k_dedup_heads(const uint64_t *__restrict__ keys, const float *__restrict__ vals, uint64_t n,
                              uint8_t *head, float *minw) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        bool h = k != INVALID_KEY && (i == 0 || keys[i - 1] != k);
        head[i] = h;
        if (h) {
            float m = vals[i];
            for (uint64_t j = i + 1; j < n && keys[j] == k; j++) m = fminf(m, vals[j]);
            minw[i] = m;
        }
    }
}

__global__ void k_dedup_write(const uint64_t *__restrict__ keys, const uint8_t *__restrict__ head,
                              const uint32_t *__restrict__ pos, const float *__restrict__ minw, uint64_t n, int b,
                              uint32_t *tgt, float *w, uint32_t *rowcnt) {
    uint64_t mask = (1ull << b) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        uint64_t k = keys[i];
        uint32_t p = pos[i];
        tgt[p] = (uint32_t)(k & mask);
        w[p] = minw[i];
        atomicAdd(rowcnt + (k >> b), 1u);
    }
}

// Library-owned storage of the last generated graph.
static struct {
    uint64_t *off = nullptr;
    uint32_t *tgt = nullptr;
    float *w = nullptr;
} g_graph;

static void release_graph() {
    cudaFree(g_graph.off);
    cudaFree(g_graph.tgt);
    cudaFree(g_graph.w);
    g_graph.off = nullptr;
    g_graph.tgt = nullptr;
    g_graph.w = nullptr;
}

static int bits_for(uint64_t n) {
    int b = 1;
    while ((1ull << b) < n) b++;
    return b;
}

// keys/vals hold 2*S entries; build the CSR of n vertices into g_graph.
static void build_csr(uint64_t *keys, float *vals, uint64_t nkeys, uint32_t n, int b, gsp_device_graph *out,
                      cudaStream_t s) {
    GSP_REQUIRE(nkeys < (1ull << 32), "generator: too many edge samples (limit 2^31 pairs)");
    uint64_t *k2 = arena().get<uint64_t>(nkeys);
    float *v2 = arena().get<float>(nkeys);
    radix_sort_u64_f32(keys, vals, k2, v2, nkeys, 2 * b, s);
    uint8_t *head = reinterpret_cast<uint8_t *>(k2);  // k2 is free after the sort
    float *minw = v2;
    uint32_t *pos = arena().get<uint32_t>(nkeys + 1);
    unsigned gr = grid_for(nkeys, 256, sms(32));
    k_dedup_heads<<<gr, 256, 0, s>>>(keys, vals, nkeys, head, minw);
    GSP_CHECK_LAUNCH();
    exclusive_scan_u8_to_u32(head, pos, nkeys, s);
    uint32_t nnz;
    GSP_CUDA(cudaMemcpyAsync(&nnz, pos + nkeys, sizeof(nnz), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    release_graph();
    GSP_CUDA(cudaMalloc(&g_graph.off, sizeof(uint64_t) * ((size_t)n + 1)));
    GSP_CUDA(cudaMalloc(&g_graph.tgt, sizeof(uint32_t) * ((size_t)nnz + 1)));
    GSP_CUDA(cudaMalloc(&g_graph.w, sizeof(float) * ((size_t)nnz + 1)));
    uint32_t *rowcnt = arena().get<uint32_t>(n);
    GSP_CUDA(cudaMemsetAsync(rowcnt, 0, sizeof(uint32_t) * n, s));
    k_dedup_write<<<gr, 256, 0, s>>>(keys, head, pos, minw, nkeys, b, g_graph.tgt, g_graph.w, rowcnt);
    GSP_CHECK_LAUNCH();
    exclusive_scan_u32_to_u64(rowcnt, g_graph.off, n, s);
    GSP_CUDA(cudaStreamSynchronize(s));
    out->n = n;
    out->nnz = nnz;
    out->offsets = g_graph.off;
    out->targets = g_graph.tgt;
    out->weights = g_graph.w;
}

}  // namespace gsp

using namespace gsp;

#define GEN_BEGIN try {
#define GEN_END                           \
    return GSP_OK;                        \
    }                                     \
    catch (const gsp::Error &e) {         \
        return e.status;                  \
    }                                     \
    catch (...) {                         \
        set_error("unexpected exception"); \
        return GSP_ERR_CUDA;              \
    }

extern "C" {

gsp_status gsp_gen_rmat(uint32_t scale, uint32_t edge_factor, uint64_t t1, uint64_t t2, uint64_t t3, uint64_t seed,
                        gsp_device_graph *out, void *stream) {
    GEN_BEGIN
    GSP_REQUIRE(scale >= 1 && scale <= 30 && edge_factor >= 1 && out, "invalid R-MAT parameters");
    GSP_REQUIRE(t1 <= t2 && t2 <= t3 && t3 <= (1ull << 53), "R-MAT thresholds must rise within 2^53");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    arena().reset();
    uint64_t S = (uint64_t)edge_factor << scale;
    uint32_t n = 1u << scale;
    int b = bits_for(n);
    uint64_t *keys = arena().get<uint64_t>(2 * S);
    float *vals = arena().get<float>(2 * S);
    k_gen_rmat<<<grid_for(S, 256, sms(32)), 256, 0, s>>>(S, scale, stream_key(seed, STREAM_RMAT), t1, t2, t3, b,
                                                         keys, vals);
    GSP_CHECK_LAUNCH();
    build_csr(keys, vals, 2 * S, n, b, out, s);
    arena().reset();
    GEN_END
}

gsp_status gsp_gen_planted_batch(uint32_t num_graphs, const uint64_t *n_g, const uint64_t *k_g,
                                 const uint64_t *edges_g, const uint64_t *p_intra53_g, const uint64_t *seed_g,
                                 gsp_device_graph *out, void *stream) {
    GEN_BEGIN
    GSP_REQUIRE(num_graphs >= 1 && n_g && k_g && edges_g && p_intra53_g && seed_g && out, "invalid arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    arena().reset();
    std::vector<uint64_t> vbase(num_graphs), ebase(num_graphs), keyv(num_graphs);
    uint64_t nv = 0, S = 0;
    for (uint32_t g = 0; g < num_graphs; g++) {
        GSP_REQUIRE(n_g[g] >= 1 && k_g[g] >= 1 && k_g[g] <= n_g[g], "graph %u: need 1 <= k <= n", g);
        vbase[g] = nv;
        ebase[g] = S;
        keyv[g] = stream_key(seed_g[g], STREAM_PLANTED);
        nv += n_g[g];
        S += edges_g[g];
    }
    GSP_REQUIRE(nv < (1ull << 31), "too many vertices");
    uint64_t *d = arena().get<uint64_t>(6ull * num_graphs);
    const uint64_t *srcs[6] = {n_g, k_g, p_intra53_g, keyv.data(), vbase.data(), ebase.data()};
    for (int i = 0; i < 6; i++)
        GSP_CUDA(cudaMemcpyAsync(d + (size_t)i * num_graphs, srcs[i], sizeof(uint64_t) * num_graphs,
                                 cudaMemcpyHostToDevice, s));
    PlantedParams P{d, d + num_graphs, d + 2 * num_graphs, d + 3 * num_graphs, d + 4 * num_graphs,
                    d + 5 * num_graphs, num_graphs};
    int b = bits_for(nv);
    uint64_t *keys = arena().get<uint64_t>(2 * S + 2);
    float *vals = arena().get<float>(2 * S + 2);
    if (S) {
        k_gen_planted<<<grid_for(S, 256, sms(32)), 256, 0, s>>>(P, S, b, keys, vals);
        GSP_CHECK_LAUNCH();
    }
    build_csr(keys, vals, 2 * S, (uint32_t)nv, b, out, s);
    arena().reset();
    GEN_END
}

gsp_status gsp_gen_grid(uint32_t R, uint32_t Cc, uint64_t remove53, uint64_t n_long, float wlo, float whi,
                        uint64_t seed, gsp_device_graph *out, void *stream) {
    GEN_BEGIN
    GSP_REQUIRE(R >= 2 && Cc >= 2 && (uint64_t)R * Cc < (1ull << 31) && out, "invalid grid size");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    arena().reset();
    uint64_t E = (uint64_t)R * (Cc - 1) + (uint64_t)(R - 1) * Cc;
    uint64_t S = E + n_long;
    uint32_t n = R * Cc;
    int b = bits_for(n);
    uint64_t *keys = arena().get<uint64_t>(2 * S);
    float *vals = arena().get<float>(2 * S);
    k_gen_grid<<<grid_for(S, 256, sms(32)), 256, 0, s>>>(R, Cc, remove53, n_long, (double)wlo, (double)whi, seed, b,
                                                         keys, vals);
    GSP_CHECK_LAUNCH();
    build_csr(keys, vals, 2 * S, n, b, out, s);
    arena().reset();
    GEN_END
}

void gsp_release_graph(void) { release_graph(); }

}  // extern "C"
