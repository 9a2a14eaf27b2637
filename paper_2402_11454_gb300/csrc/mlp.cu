// mlp.cu -- the learned vertex-pruning predictor: a 6 -> 32 -> 32 -> 1 MLP
// (ReLU hidden layers, sigmoid output) with weights rounded to bfloat16 and
// float32 accumulation; forward, binary cross-entropy backward, SGD and Adam steps.
//
// Parameter layout (float32 master copy): W1[32][6], b1[32], W2[32][32],
// b2[32], W3[32], b3.  One thread evaluates one row (about 1.2 K FMA); the
// rounded weights sit in shared memory.  The backward pass reduces every
// parameter's per-row contribution over a warp with shuffles, then over the
// block in shared memory, then adds it to the global gradient.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace gsp {

constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_H * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H;
constexpr int OFF_B3 = OFF_W3 + MLP_H;
static_assert(OFF_B3 + 1 == MLP_PARAMS, "parameter layout");

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ void load_params_bf16(const float *__restrict__ params, float *sp) {
    for (int i = threadIdx.x; i < MLP_PARAMS; i += blockDim.x) sp[i] = bf16r(params[i]);
    __syncthreads();
}

// Forward pass of one row; h1, h2 receive the hidden activations; returns z.
__device__ __forceinline__ float mlp_row(const float *sp, const float *x, float *h1, float *h2) {
#pragma unroll
    for (int j = 0; j < MLP_H; j++) {
        float a = sp[OFF_B1 + j];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) a = fmaf(sp[OFF_W1 + j * MLP_IN + i], x[i], a);
        h1[j] = fmaxf(a, 0.0f);
    }
#pragma unroll
    for (int j = 0; j < MLP_H; j++) {
        float a = sp[OFF_B2 + j];
#pragma unroll
        for (int i = 0; i < MLP_H; i++) a = fmaf(sp[OFF_W2 + j * MLP_H + i], h1[i], a);
        h2[j] = fmaxf(a, 0.0f);
    }
    float z = sp[OFF_B3];
#pragma unroll
    for (int i = 0; i < MLP_H; i++) z = fmaf(sp[OFF_W3 + i], h2[i], z);
    return z;
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

__device__ float mlp_prob(const float *sp, const float *x) {
    float h1[MLP_H], h2[MLP_H];
    return sigmoidf(mlp_row(sp, x, h1, h2));
}

__global__ void k_mlp_forward(const float *__restrict__ params, const float *__restrict__ x, uint32_t rows,
                              float *__restrict__ p) {
    __shared__ float sp[MLP_PARAMS];
    load_params_bf16(params, sp);
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        float xr[MLP_IN];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) xr[i] = x[(size_t)r * MLP_IN + i];
        p[r] = mlp_prob(sp, xr);
    }
}

// Per-warp accumulation of one parameter's contributions.
__device__ __forceinline__ void acc_param(float *wsum, int idx, float v) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) wsum[idx] += v;
}

constexpr int MLP_BWD_THREADS = 128;

__global__ void __launch_bounds__(MLP_BWD_THREADS) k_mlp_backward(const float *__restrict__ params,
                                                                  const float *__restrict__ x,
                                                                  const uint8_t *__restrict__ y, uint32_t rows,
                                                                  float *grad, double *loss) {
    __shared__ float sp[MLP_PARAMS];
    __shared__ float ws[MLP_BWD_THREADS / 32][MLP_PARAMS];
    __shared__ double red[32];
    const int wid = threadIdx.x >> 5;
    for (int i = threadIdx.x & 31; i < MLP_PARAMS; i += 32) ws[wid][i] = 0.0f;
    load_params_bf16(params, sp);
    float *wsum = ws[wid];
    double lsum = 0.0;
    const float inv_n = 1.0f / (float)rows;
    // every lane of a warp runs the same number of iterations (shuffles)
    uint32_t stride = gridDim.x * blockDim.x;
    uint32_t base0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (uint32_t base = base0; base < rows; base += stride) {
        uint32_t r = base + (threadIdx.x & 31);
        bool valid = r < rows;
        float xr[MLP_IN], h1[MLP_H], h2[MLP_H];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) xr[i] = valid ? x[(size_t)r * MLP_IN + i] : 0.0f;
        float z = mlp_row(sp, xr, h1, h2);
        float yr = valid ? (float)y[r] : 0.0f;
        float p = sigmoidf(z);
        // BCE = softplus(z) - y z, in a stable form
        if (valid) lsum += (double)(fmaxf(z, 0.0f) - yr * z + log1pf(expf(-fabsf(z))));
        float dz = valid ? (p - yr) * inv_n : 0.0f;
        acc_param(wsum, OFF_B3, dz);
        float dh2[MLP_H];
#pragma unroll
        for (int j = 0; j < MLP_H; j++) {
            acc_param(wsum, OFF_W3 + j, dz * h2[j]);
            dh2[j] = h2[j] > 0.0f ? dz * sp[OFF_W3 + j] : 0.0f;
        }
        float dh1[MLP_H];
#pragma unroll
        for (int i = 0; i < MLP_H; i++) dh1[i] = 0.0f;
#pragma unroll
        for (int j = 0; j < MLP_H; j++) {
            acc_param(wsum, OFF_B2 + j, dh2[j]);
#pragma unroll
            for (int i = 0; i < MLP_H; i++) {
                acc_param(wsum, OFF_W2 + j * MLP_H + i, dh2[j] * h1[i]);
                dh1[i] = fmaf(dh2[j], sp[OFF_W2 + j * MLP_H + i], dh1[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < MLP_H; i++) {
            float d = h1[i] > 0.0f ? dh1[i] : 0.0f;
            acc_param(wsum, OFF_B1 + i, d);
#pragma unroll
            for (int k = 0; k < MLP_IN; k++) acc_param(wsum, OFF_W1 + i * MLP_IN + k, d * xr[k]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < MLP_PARAMS; i += blockDim.x) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < MLP_BWD_THREADS / 32; w++) t += ws[w][i];
        if (t != 0.0f) atomicAdd(grad + i, t);
    }
    lsum = block_sum(lsum, red);
    if (threadIdx.x == 0) atomicAdd(loss, lsum);
}

__global__ void k_mlp_sgd(float *params, const float *__restrict__ grad, float lr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_PARAMS; i += gridDim.x * blockDim.x)
        params[i] -= lr * grad[i];
}

__global__ void k_mlp_adam(float *params, const float *__restrict__ grad, float *m, float *v, float lr, float b1,
                           float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_PARAMS; i += gridDim.x * blockDim.x) {
        float g = grad[i];
        float mi = b1 * m[i] + (1.0f - b1) * g;
        float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Learned pruning: one thread per vertex; active vertices predicted not to
// move sit out the sweep (flag cleared, skip set) and are counted as skipped.
__global__ void k_mlp_prune(const float *__restrict__ params, const uint64_t *__restrict__ off,
                            const double *__restrict__ K, const float *__restrict__ kept,
                            const float *__restrict__ gain, const float *__restrict__ last_gain,
                            const uint8_t *__restrict__ moved, uint8_t *act, uint8_t *skip, uint32_t n,
                            float max_logk, float iter_frac, float thr, MoveCounters *ctr) {
    __shared__ float sp[MLP_PARAMS];
    __shared__ unsigned long long red[32];
    __shared__ double redd[32];
    load_params_bf16(params, sp);
    unsigned long long skipped = 0;
    double expect = 0.0;  // expected gain of the put-off vertices: P(move) x last best gain
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!act[i]) continue;
        uint32_t deg = (uint32_t)(off[i + 1] - off[i]);
        if (!deg) continue;
        float x[MLP_IN];
        predictor_features(deg, K[i], kept[i], gain[i], moved[i], max_logk, iter_frac, x);
        const float p = mlp_prob(sp, x);
        if (p < thr) {
            act[i] = 0;
            skip[i] = 1;
            skipped++;
            expect += (double)p * (double)fmaxf(last_gain[i], 0.0f);
        }
    }
    skipped = block_sum(skipped, red);
    expect = block_sum(expect, redd);
    if (threadIdx.x == 0 && skipped) {
        atomicAdd(&ctr->skipped, skipped);
        atomicAdd(&ctr->skipped_gain, expect);
    }
}

void mlp_prune(const DevGraph &g, MoveBuffers &mb, int iteration, int max_iterations, float threshold,
               cudaStream_t s) {
    float frac = max_iterations > 0 ? (float)iteration / (float)max_iterations : 0.0f;
    k_mlp_prune<<<grid_for(g.n, 256, sms(8)), 256, 0, s>>>(mb.mlp, g.off, mb.K, mb.feat_kept, mb.feat_gain,
                                                            mb.last_gain, mb.moved_last, mb.act, mb.skip, g.n,
                                                            mb.max_logk, frac, threshold, mb.ctr);
    GSP_CHECK_LAUNCH();
}

__global__ void k_mlp_unskip(uint8_t *act, uint8_t *skip, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (skip[i]) {
            act[i] = 1;
            skip[i] = 0;
        }
}

void mlp_unskip(const DevGraph &g, MoveBuffers &mb, cudaStream_t s) {
    k_mlp_unskip<<<grid_for(g.n, 256), 256, 0, s>>>(mb.act, mb.skip, g.n);
    GSP_CHECK_LAUNCH();
}

}  // namespace gsp

using namespace gsp;

#define MLP_BEGIN try {
#define MLP_END                             \
    return GSP_OK;                          \
    }                                       \
    catch (const gsp::Error &e) {           \
        return e.status;                    \
    }                                       \
    catch (...) {                           \
        set_error("unexpected exception");  \
        return GSP_ERR_CUDA;                \
    }

extern "C" {

int gsp_mlp_param_count(void) { return MLP_PARAMS; }

gsp_status gsp_mlp_forward(const float *params, const float *x, uint32_t rows, float *p, void *stream) {
    MLP_BEGIN
    GSP_REQUIRE(params && (rows == 0 || (x && p)), "invalid arguments");
    if (!rows) return GSP_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_mlp_forward<<<grid_for(rows, 256), 256, 0, s>>>(params, x, rows, p);
    GSP_CHECK_LAUNCH();
    GSP_CUDA(cudaStreamSynchronize(s));
    MLP_END
}

gsp_status gsp_mlp_backward(const float *params, const float *x, const uint8_t *y, uint32_t rows, float *grad,
                            double *loss_host, void *stream) {
    MLP_BEGIN
    GSP_REQUIRE(params && grad && rows > 0 && x && y, "invalid arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t mk = arena().mark();
    double *loss = arena().get<double>(1);
    GSP_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * MLP_PARAMS, s));
    GSP_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
    k_mlp_backward<<<grid_for(rows, MLP_BWD_THREADS, sms(4)), MLP_BWD_THREADS, 0, s>>>(params, x, y, rows, grad,
                                                                                        loss);
    GSP_CHECK_LAUNCH();
    double h;
    GSP_CUDA(cudaMemcpyAsync(&h, loss, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    if (loss_host) *loss_host = h / rows;
    MLP_END
}

gsp_status gsp_mlp_sgd(float *params, const float *grad, float lr, void *stream) {
    MLP_BEGIN
    GSP_REQUIRE(params && grad, "invalid arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_mlp_sgd<<<grid_for(MLP_PARAMS, 256), 256, 0, s>>>(params, grad, lr);
    GSP_CHECK_LAUNCH();
    MLP_END
}

gsp_status gsp_mlp_adam(float *params, const float *grad, float *m, float *v, float lr, float beta1, float beta2,
                        float eps, int t, void *stream) {
    MLP_BEGIN
    GSP_REQUIRE(params && grad && m && v, "invalid arguments");
    GSP_REQUIRE(t >= 1, "Adam step number must be >= 1");
    GSP_REQUIRE(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f,
                "Adam hyper-parameters out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float c1 = (float)(1.0 - pow((double)beta1, t)), c2 = (float)(1.0 - pow((double)beta2, t));
    k_mlp_adam<<<grid_for(MLP_PARAMS, 256), 256, 0, s>>>(params, grad, m, v, lr, beta1, beta2, eps, c1, c2);
    GSP_CHECK_LAUNCH();
    MLP_END
}

}  // extern "C"
