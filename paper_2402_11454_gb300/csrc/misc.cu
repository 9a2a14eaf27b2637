// misc.cu -- vertex weights (Section 3), modularity (Equation 1), community
// renumbering and dendrogram lookup (Algorithm 1), the final numbering, and
// the disconnected-community count (Algorithm 6).
//
// Row sums use one thread per row up to 64 entries, one warp per row up to
// 8192 and one block per longer row.  Their sums of weights are exact and so
// do not depend on the order: in integer units of the weights' lowest set bit
// when the total fits 2^52 such units (exact_lsb), otherwise in float64 over
// float32-representable weights whose partial sums stay representable.
#include <cmath>

#include "internal.cuh"

namespace gsp {

constexpr uint32_t SHORT_ROW = 64;

// Smallest lowest-set-bit exponent over the weights and their (rounded) sum.
template <typename WT>
__global__ void k_weight_range(const WT *__restrict__ w, uint64_t nnz, int *minlow, double *sum) {
    int lo = INT_MAX;
    float acc = 0.0f;  // an estimate for the range test (float64 is slow here)
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nnz; p += (uint64_t)gridDim.x * blockDim.x) {
        const WT x = w[p];
        lo = min(lo, low_bit_exp(x));
        acc += (float)x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(minlow, lo);
        atomicAdd(sum, (double)acc);
    }
}

// exact_lsb: the exponent lsb such that every weight is a multiple of 2^lsb
// and the total weight is below 2^52 * 2^lsb, so that every sum of weights is
// an integer number of units below 2^52, exact both as uint64 and as float64;
// INT_MIN when no such exponent in [-1000, 1000] exists (zero, negative or
// non-finite weights, or too wide a range of magnitudes).  The total is
// estimated with float32 partial sums (relative error far below the factor 2
// of margin kept under 2^53).
template <typename WT>
static int exact_lsb_t(const DevGraph &g, cudaStream_t s) {
    if (!g.nnz || !g.w) return INT_MIN;
    size_t mk = arena().mark();
    int *dlo = arena().get<int>(1);
    double *dsum = arena().get<double>(1);
    const int init = INT_MAX;
    GSP_CUDA(cudaMemcpyAsync(dlo, &init, sizeof(int), cudaMemcpyHostToDevice, s));
    GSP_CUDA(cudaMemsetAsync(dsum, 0, sizeof(double), s));
    k_weight_range<WT><<<grid_for(g.nnz, 256, sms(8)), 256, 0, s>>>(static_cast<const WT *>(g.w), g.nnz, dlo, dsum);
    GSP_CHECK_LAUNCH();
    int lo = 0;
    double sum = 0.0;
    GSP_CUDA(cudaMemcpyAsync(&lo, dlo, sizeof(int), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaMemcpyAsync(&sum, dsum, sizeof(double), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    if (lo < -1000 || lo > 1000) return INT_MIN;
    // the sum is an estimate: keep a factor 2 of margin below 2^53
    if (!(sum > 0.0) || !(sum < std::ldexp(1.0, 52 + lo))) return INT_MIN;
    return lo;
}

int exact_lsb(const DevGraph &g, cudaStream_t s) {
    return g.wt == GSP_W_F64 ? exact_lsb_t<double>(g, s) : exact_lsb_t<float>(g, s);
}


__global__ void k_iota(uint32_t *p, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}
void iota_u32(uint32_t *p, uint32_t n, cudaStream_t s) {
    if (!n) return;
    k_iota<<<grid_for(n, 256), 256, 0, s>>>(p, n);
    GSP_CHECK_LAUNCH();
}

// Owner of every task of a chunked work split: one warp per item writes the
// item's index over its task range.
__global__ void k_task_items(const uint64_t *__restrict__ prefix, uint32_t nitems, uint32_t *out) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t base = prefix[0];
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nitems;
         t += (gridDim.x * blockDim.x) >> 5) {
        const uint64_t b = prefix[t] - base, e = prefix[t + 1] - base;
        for (uint64_t k = b + lane; k < e; k += 32) out[k] = t;
    }
}
void task_items(const uint64_t *prefix, uint32_t nitems, uint32_t *out, cudaStream_t s) {
    if (!nitems) return;
    k_task_items<<<grid_for((uint64_t)nitems * 32, 256), 256, 0, s>>>(prefix, nitems, out);
    GSP_CHECK_LAUNCH();
}

// Per row i: K_i, and the intra-community part sum_{j: C_j = C_i} w_ij when C
// is given; Sigma_c += K_i when Sig is given.  Long rows are deferred to a
// list for the block kernel.
template <typename WT, typename AV>
__global__ void k_row_sums(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tgt,
                           const WT *__restrict__ w, uint32_t n, const uint32_t *__restrict__ C, double *K,
                           double *Sig, AV *acc /* [0]=2m, [1]=intra */, uint32_t *longlist,
                           uint32_t *nlong, int lsb) {
    __shared__ AV red[32];
    AV two_m = 0, intra = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint64_t b = off[i], e = off[i + 1];
        if (e - b > SHORT_ROW) {
            longlist[atomicAdd(nlong, 1u)] = i;
            continue;
        }
        AV k = 0, in = 0;
        uint32_t ci = C ? C[i] : 0;
        uint64_t p = b;
        for (; p + 4 <= e; p += 4) {  // four independent loads in flight
            AV wv[4];
            uint32_t cj[4];
#pragma unroll
            for (int u = 0; u < 4; u++) wv[u] = Acc<AV>::of(w[p + u], lsb);
            if (C) {
#pragma unroll
                for (int u = 0; u < 4; u++) cj[u] = C[tgt[p + u]];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                k += wv[u];
                if (C && cj[u] == ci) in += wv[u];
            }
        }
        for (; p < e; p++) {
            const AV wv = Acc<AV>::of(w[p], lsb);
            k += wv;
            if (C && C[tgt[p]] == ci) in += wv;
        }
        const double kd = Acc<AV>::val(k, lsb);
        if (K) K[i] = kd;
        if (Sig) atomicAdd(Sig + ci, kd);
        two_m += k;
        intra += in;
    }
    two_m = block_sum(two_m, red);
    intra = block_sum(intra, red);
    if (threadIdx.x == 0) {
        atomicAdd(acc, two_m);
        if (C) atomicAdd(acc + 1, intra);
    }
}

// Long rows: one warp per row up to 8192 entries, one block per longer row.
constexpr uint32_t WARP_ROW = 8192;

template <typename WT, typename AV>
__global__ void k_row_sums_long(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tgt,
                                const WT *__restrict__ w, const uint32_t *__restrict__ C, double *K, double *Sig,
                                AV *acc, const uint32_t *longlist, const uint32_t *nlong, int lsb) {
    __shared__ AV red[32];
    uint32_t cnt = *nlong;
    const int lane = threadIdx.x & 31;
    uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    AV wk = 0, win = 0;
    for (uint32_t t = warp; t < cnt; t += nwarps) {
        uint32_t i = longlist[t];
        uint64_t b = off[i], e = off[i + 1];
        if (e - b > WARP_ROW) continue;
        uint32_t ci = C ? C[i] : 0;
        AV k = 0, in = 0;
        uint64_t p = b + lane;
        for (; p + 96 < e; p += 128) {  // four independent loads per lane in flight
            AV wv[4];
            uint32_t cj[4];
#pragma unroll
            for (int u = 0; u < 4; u++) wv[u] = Acc<AV>::of(w[p + 32 * u], lsb);
            if (C) {
#pragma unroll
                for (int u = 0; u < 4; u++) cj[u] = C[tgt[p + 32 * u]];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                k += wv[u];
                if (C && cj[u] == ci) in += wv[u];
            }
        }
        for (; p < e; p += 32) {
            const AV wv = Acc<AV>::of(w[p], lsb);
            k += wv;
            if (C && C[tgt[p]] == ci) in += wv;
        }
        k = warp_sum(k);
        in = warp_sum(in);
        if (lane == 0) {
            const double kd = Acc<AV>::val(k, lsb);
            if (K) K[i] = kd;
            if (Sig) atomicAdd(Sig + ci, kd);
            wk += k;
            win += in;
        }
    }
    // rows longer than WARP_ROW: one block each
    for (uint32_t t = blockIdx.x; t < cnt; t += gridDim.x) {
        uint32_t i = longlist[t];
        uint64_t b = off[i], e = off[i + 1];
        if (e - b <= WARP_ROW) continue;
        uint32_t ci = C ? C[i] : 0;
        AV k = 0, in = 0;
        uint64_t p = b + threadIdx.x;
        const uint64_t st = blockDim.x;
        for (; p + 3 * st < e; p += 4 * st) {
            AV wv[4];
            uint32_t cj[4];
#pragma unroll
            for (int u = 0; u < 4; u++) wv[u] = Acc<AV>::of(w[p + st * u], lsb);
            if (C) {
#pragma unroll
                for (int u = 0; u < 4; u++) cj[u] = C[tgt[p + st * u]];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                k += wv[u];
                if (C && cj[u] == ci) in += wv[u];
            }
        }
        for (; p < e; p += st) {
            const AV wv = Acc<AV>::of(w[p], lsb);
            k += wv;
            if (C && C[tgt[p]] == ci) in += wv;
        }
        k = block_sum(k, red);
        in = block_sum(in, red);
        if (threadIdx.x == 0) {
            const double kd = Acc<AV>::val(k, lsb);
            if (K) K[i] = kd;
            if (Sig) atomicAdd(Sig + ci, kd);
            wk += k;
            win += in;
        }
    }
    wk = block_sum(wk, red);
    win = block_sum(win, red);
    if (threadIdx.x == 0) {
        if (wk != AV(0)) atomicAdd(acc, wk);
        if (C && win != AV(0)) atomicAdd(acc + 1, win);
    }
}

template <typename WT, typename AV>
static void row_sums(const DevGraph &g, const uint32_t *C, double *K, double *Sig, AV *acc, int lsb, cudaStream_t s) {
    size_t mk = arena().mark();
    uint32_t *longlist = arena().get<uint32_t>(g.n + 1);
    uint32_t *nlong = arena().get<uint32_t>(1);
    GSP_CUDA(cudaMemsetAsync(nlong, 0, sizeof(uint32_t), s));
    const WT *w = static_cast<const WT *>(g.w);
    k_row_sums<WT, AV><<<grid_for(g.n, 256), 256, 0, s>>>(g.off, g.tgt, w, g.n, C, K, Sig, acc, longlist, nlong, lsb);
    GSP_CHECK_LAUNCH();
    // as many warps as fit: each long row is a chain of loads per lane
    k_row_sums_long<WT, AV><<<resident_grid((const void *)k_row_sums_long<WT, AV>, 256, 0, 8), 256, 0, s>>>(
        g.off, g.tgt, w, C, K, Sig, acc, longlist, nlong, lsb);
    GSP_CHECK_LAUNCH();
    arena().release(mk);
}

// x[k] = u[k] units of 2^lsb as float64 (exact: u < 2^52).
__global__ void k_units_to_f64(const unsigned long long *u, int cnt, int lsb, double *x) {
    if ((int)threadIdx.x < cnt) x[threadIdx.x] = Acc<unsigned long long>::val(u[threadIdx.x], lsb);
}

// Row sums into float64 accumulators (acc: [0] = 2m, [1] = intra), or, when
// lsb != INT_MIN, in integer units accumulated in acc_u and converted here
// (exactly) into the same float64 values.
static void row_sums_any(const DevGraph &g, const uint32_t *C, double *K, double *Sig, double *acc,
                         unsigned long long *acc_u, int lsb, cudaStream_t s) {
    if (lsb != INT_MIN) {
        if (g.wt == GSP_W_F64) row_sums<double, unsigned long long>(g, C, K, Sig, acc_u, lsb, s);
        else row_sums<float, unsigned long long>(g, C, K, Sig, acc_u, lsb, s);
        k_units_to_f64<<<1, 32, 0, s>>>(acc_u, 2, lsb, acc);
        GSP_CHECK_LAUNCH();
        return;
    }
    if (g.wt == GSP_W_F64) row_sums<double, double>(g, C, K, Sig, acc, INT_MIN, s);
    else row_sums<float, double>(g, C, K, Sig, acc, INT_MIN, s);
}

__global__ void k_half(const double *acc, double *m_dev) { *m_dev = acc[0] / 2.0; }

double vertex_weights(const DevGraph &g, double *K, double *m_dev, cudaStream_t s, int lsb) {
    size_t mk = arena().mark();
    double *acc = arena().get<double>(2);
    unsigned long long *acc_u = arena().get<unsigned long long>(2);
    GSP_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
    GSP_CUDA(cudaMemsetAsync(acc_u, 0, 2 * sizeof(unsigned long long), s));
    row_sums_any(g, nullptr, K, nullptr, acc, acc_u, lsb, s);
    if (m_dev) {
        k_half<<<1, 1, 0, s>>>(acc, m_dev);
        GSP_CHECK_LAUNCH();
    }
    double h[2];
    GSP_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    return h[0] / 2.0;
}

__global__ void k_sum_sq(const double *Sig, uint32_t n, double *out) {
    __shared__ double red[32];
    double t = 0;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double x = Sig[c];
        t += x * x;
    }
    t = block_sum(t, red);
    if (threadIdx.x == 0) atomicAdd(out, t);
}

// Equation 1, second form: Q = sum_c sigma_c / 2m - sum_c (Sigma_c / 2m)^2,
// with sum_c sigma_c = the weight of all intra-community entries.
double modularity(const DevGraph &g, const uint32_t *C, cudaStream_t s, int lsb) {
    size_t mk = arena().mark();
    double *acc = arena().get<double>(4);
    unsigned long long *acc_u = arena().get<unsigned long long>(2);
    double *Sig = arena().get<double>(g.n);
    GSP_CUDA(cudaMemsetAsync(acc, 0, 4 * sizeof(double), s));
    GSP_CUDA(cudaMemsetAsync(acc_u, 0, 2 * sizeof(unsigned long long), s));
    GSP_CUDA(cudaMemsetAsync(Sig, 0, sizeof(double) * g.n, s));
    row_sums_any(g, C, nullptr, Sig, acc, acc_u, lsb, s);
    k_sum_sq<<<grid_for(g.n, 256), 256, 0, s>>>(Sig, g.n, acc + 2);
    GSP_CHECK_LAUNCH();
    double h[4];
    GSP_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    double two_m = h[0];
    if (!(two_m > 0.0)) return 0.0;
    return h[1] / two_m - h[2] / (two_m * two_m);
}

// Equation 1 with caller-provided scratch instead of the workspace: Sig (n
// doubles), acc (4 doubles), longlist (n entries) and nlong (1 entry).
// Allocates nothing.
template <typename WT>
static double modularity_scratch_t(const DevGraph &g, const uint32_t *C, double *Sig, double *acc, uint32_t *longlist,
                                   uint32_t *nlong, cudaStream_t s) {
    const WT *w = static_cast<const WT *>(g.w);
    GSP_CUDA(cudaMemsetAsync(acc, 0, 4 * sizeof(double), s));
    GSP_CUDA(cudaMemsetAsync(Sig, 0, sizeof(double) * g.n, s));
    GSP_CUDA(cudaMemsetAsync(nlong, 0, sizeof(uint32_t), s));
    k_row_sums<WT, double><<<grid_for(g.n, 256), 256, 0, s>>>(g.off, g.tgt, w, g.n, C, nullptr, Sig, acc, longlist,
                                                              nlong, INT_MIN);
    GSP_CHECK_LAUNCH();
    k_row_sums_long<WT, double><<<sms(4), 256, 0, s>>>(g.off, g.tgt, w, C, nullptr, Sig, acc, longlist, nlong,
                                                       INT_MIN);
    GSP_CHECK_LAUNCH();
    k_sum_sq<<<grid_for(g.n, 256), 256, 0, s>>>(Sig, g.n, acc + 2);
    GSP_CHECK_LAUNCH();
    double h[4];
    GSP_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    double two_m = h[0];
    if (!(two_m > 0.0)) return 0.0;
    return h[1] / two_m - h[2] / (two_m * two_m);
}

double modularity_scratch(const DevGraph &g, const uint32_t *C, double *Sig, double *acc, uint32_t *longlist,
                          uint32_t *nlong, cudaStream_t s) {
    if (g.wt == GSP_W_F64) return modularity_scratch_t<double>(g, C, Sig, acc, longlist, nlong, s);
    return modularity_scratch_t<float>(g, C, Sig, acc, longlist, nlong, s);
}

__global__ void k_count_ge(const uint32_t *__restrict__ x, uint64_t n, uint32_t bound, unsigned long long *out) {
    unsigned long long b = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (x[i] >= bound) b++;
    if (b) atomicAdd(out, b);
}

// Number of entries x[i] >= bound (i < n), counted in *counter
// (caller-provided, no allocation).
unsigned long long count_out_of_range(const uint32_t *x, uint64_t n, uint32_t bound, unsigned long long *counter,
                                      cudaStream_t s) {
    GSP_CUDA(cudaMemsetAsync(counter, 0, sizeof(*counter), s));
    if (n) {
        k_count_ge<<<grid_for(n, 256), 256, 0, s>>>(x, n, bound, counter);
        GSP_CHECK_LAUNCH();
    }
    unsigned long long h = 0;
    GSP_CUDA(cudaMemcpyAsync(&h, counter, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    return h;
}

__global__ void k_count_bad_offsets(const uint64_t *__restrict__ off, uint32_t n, uint64_t nnz,
                                    unsigned long long *out) {
    unsigned long long b = 0;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint64_t i = tid; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (off[i + 1] < off[i]) b++;
    if (tid == 0 && (off[0] != 0 || off[n] != nnz)) b++;
    if (b) atomicAdd(out, b);
}

// CSR structure for the phase entry points: offsets rise from 0 to nnz and
// every target is < n; raises GSP_ERR_INVALID otherwise.  *counter is
// caller-provided scratch (no allocation).
void check_csr(const uint64_t *off, const uint32_t *tgt, uint32_t n, uint64_t nnz, unsigned long long *counter,
               cudaStream_t s) {
    GSP_CUDA(cudaMemsetAsync(counter, 0, sizeof(*counter), s));
    k_count_bad_offsets<<<grid_for(n, 256), 256, 0, s>>>(off, n, nnz, counter);
    GSP_CHECK_LAUNCH();
    unsigned long long h = 0;
    GSP_CUDA(cudaMemcpyAsync(&h, counter, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    GSP_REQUIRE(h == 0, "invalid graph: offsets must rise from 0 to nnz");
    h = count_out_of_range(tgt, nnz, n, counter, s);
    GSP_REQUIRE(h == 0, "invalid graph: %llu targets out of range (must be < %u)", h, n);
}

// ---------------------------------------------------------------- renumber
__global__ void k_mark_used(const uint32_t *__restrict__ C, uint32_t n, uint8_t *used) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) used[C[i]] = 1;
}
__global__ void k_apply_rank(const uint32_t *__restrict__ C, uint32_t n, const uint32_t *__restrict__ rank,
                             uint32_t *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = rank[C[i]];
}

uint32_t renumber(uint32_t n, const uint32_t *C, uint32_t *C_dense, cudaStream_t s) {
    size_t mk = arena().mark();
    uint8_t *used = arena().get<uint8_t>(n);
    uint32_t *rank = arena().get<uint32_t>((size_t)n + 1);
    GSP_CUDA(cudaMemsetAsync(used, 0, n, s));
    k_mark_used<<<grid_for(n, 256), 256, 0, s>>>(C, n, used);
    GSP_CHECK_LAUNCH();
    exclusive_scan_u8_to_u32(used, rank, n, s);
    k_apply_rank<<<grid_for(n, 256), 256, 0, s>>>(C, n, rank, C_dense);
    GSP_CHECK_LAUNCH();
    uint32_t k;
    GSP_CUDA(cudaMemcpyAsync(&k, rank + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    return k;
}

__global__ void k_lookup(uint32_t *Ctop, uint32_t n, const uint32_t *__restrict__ Cp) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) Ctop[i] = Cp[Ctop[i]];
}
void lookup(uint32_t n_top, uint32_t *C_top, const uint32_t *C_pass, cudaStream_t s) {
    if (!n_top) return;
    k_lookup<<<grid_for(n_top, 256), 256, 0, s>>>(C_top, n_top, C_pass);
    GSP_CHECK_LAUNCH();
}

// ------------------------------------------------------- final numbering
__global__ void k_first_vertex(const uint32_t *__restrict__ C, uint32_t n, uint32_t *first) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicMin(first + C[i], i);
}
__global__ void k_is_first(const uint32_t *__restrict__ C, uint32_t n, const uint32_t *__restrict__ first,
                           uint8_t *flag) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = first[C[i]] == i;
}
__global__ void k_apply_first(uint32_t *C, uint32_t n, const uint32_t *__restrict__ first,
                              const uint32_t *__restrict__ rank) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        C[i] = rank[first[C[i]]];
}

uint32_t canonical_numbering(uint32_t n, uint32_t *C, cudaStream_t s) {
    size_t mk = arena().mark();
    uint32_t *first = arena().get<uint32_t>(n);
    uint8_t *flag = arena().get<uint8_t>(n);
    uint32_t *rank = arena().get<uint32_t>((size_t)n + 1);
    GSP_CUDA(cudaMemsetAsync(first, 0xFF, sizeof(uint32_t) * n, s));
    unsigned gr = grid_for(n, 256);
    k_first_vertex<<<gr, 256, 0, s>>>(C, n, first);
    GSP_CHECK_LAUNCH();
    k_is_first<<<gr, 256, 0, s>>>(C, n, first, flag);
    GSP_CHECK_LAUNCH();
    exclusive_scan_u8_to_u32(flag, rank, n, s);
    k_apply_first<<<gr, 256, 0, s>>>(C, n, first, rank);
    GSP_CHECK_LAUNCH();
    uint32_t k;
    GSP_CUDA(cudaMemcpyAsync(&k, rank + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    return k;
}

// ------------------------------------------ Algorithm 6 (disconnected count)
// A community is disconnected exactly when its vertices fall in more than
// one connected component of the intra-community subgraph.
__global__ void k_count_roots(const uint32_t *__restrict__ C, const uint32_t *__restrict__ lab, uint32_t n,
                              uint32_t *ncomp) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (lab[i] == i) atomicAdd(ncomp + C[i], 1u);
}
__global__ void k_flag_disconnected(const uint32_t *__restrict__ ncomp, uint32_t n, uint8_t *flags,
                                    unsigned long long *count) {
    __shared__ unsigned long long red[32];
    unsigned long long t = 0;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        uint8_t f = ncomp[c] > 1;
        if (flags) flags[c] = f;
        t += f;
    }
    t = block_sum(t, red);
    if (threadIdx.x == 0 && t) atomicAdd(count, t);
}

uint32_t count_disconnected(const DevGraph &g, const uint32_t *C, uint8_t *flags, cudaStream_t s) {
    size_t mk = arena().mark();
    uint32_t *lab = arena().get<uint32_t>(g.n);
    uint32_t *ncomp = arena().get<uint32_t>(g.n);
    unsigned long long *cnt = arena().get<unsigned long long>(1);
    Classes cl;
    classify_vertices(g, cl, 1, s);
    split_labels(g, cl, C, GSP_SPLIT_SV, lab, s);  // every technique gives the same labels
    GSP_CUDA(cudaMemsetAsync(ncomp, 0, sizeof(uint32_t) * g.n, s));
    GSP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    unsigned gr = grid_for(g.n, 256);
    k_count_roots<<<gr, 256, 0, s>>>(C, lab, g.n, ncomp);
    GSP_CHECK_LAUNCH();
    k_flag_disconnected<<<gr, 256, 0, s>>>(ncomp, g.n, flags, cnt);
    GSP_CHECK_LAUNCH();
    unsigned long long h;
    GSP_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    return (uint32_t)h;
}

}  // namespace gsp
