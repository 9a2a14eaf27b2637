// refine.cu -- refinement phase of the Leiden algorithm (Section 3.5), the
// step that turns GSP-Louvain into the GSP-Leiden variant: the refined
// partition R of each bound community b (the membership local moving and
// the split left) starts from singletons, and a vertex still alone in R may
// join the refined community c of a neighbour inside b when
//   E(v, b-v) >= K_v (S_b - K_v) / 2m     (v well connected to b),
//   E(c, b-c) >= S_c (S_b - S_c) / 2m     (c well connected to b),
//   g_c = E(v, c) - K_v S_c / 2m >= 0     (m times Equation 2),
// chosen with probability proportional to exp(g_c / theta) among the
// eligible c and staying (gain 0): the largest g / theta plus Gumbel noise
// -ln(-ln u), u drawn per (vertex, candidate) from SplitMix64 used as a
// counter-based generator, so that the choice does not depend on the order
// in which the table lists the candidates.  theta = 0 is the greedy limit
// (largest g > 0, ties to the lowest id).
//
// Parallel form: every vertex is visited once, in the frozen-state waves of
// local moving (the class/wave lists of classify_vertices); a wave's
// decisions read the wave's start state, and a mover whose own singleton is
// another mover's target in the same wave stays, so every target keeps its
// members.  E(c, b-c) is kept per refined community: a joiner adds its
// E(v, b-v), less twice its edges to c's earlier members and less its edges
// to the wave's other joiners of c (each such edge is met from both ends).
//
// Scores are float64 in every precision mode, each operation rounded as
// written (no fused multiply-add).  Table sums and the per-community totals
// are float64 additions in an unspecified order, exact -- and so equal to a
// sequential evaluation -- when the weights are integer multiples of a power
// of two with totals below 2^53 units.
#include "internal.cuh"

namespace gsp {

namespace {

constexpr int RF_THREADS = 256;
constexpr int RF_WARPS = RF_THREADS / 32;
constexpr int RF_WARP_SLOTS = 256;  // per-warp table: degrees up to GROUP_MAX_LIMIT (128)
constexpr uint64_t GOLDEN_GAMMA = 0x9e3779b97f4a7c15ull;

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output for generator
// state x (the state advanced by the golden gamma, then the mixer).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + GOLDEN_GAMMA;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Gumbel noise -ln(-ln u) for (vertex, candidate); pass_key is the pass's
// stream of the seed, splitmix64(seed + gamma * (pass + 1)).
__device__ __forceinline__ double gumbel(uint64_t pass_key, uint32_t v, uint32_t c) {
    uint64_t r = splitmix64(pass_key ^ (((uint64_t)v << 32) | c));
    double u = __dmul_rn(__dadd_rn((double)(r >> 12), 0.5), 0x1.0p-52);
    return -log(-log(u));
}

struct RefineState {
    const uint64_t *off;
    const uint32_t *tgt;
    const void *w;
    const uint32_t *B;   // bound membership (ids < n)
    uint32_t *R;         // refined membership (seed vertex ids)
    const double *K;
    const double *SB;    // S_b per bound community
    double *SR;          // S_c per refined community
    double *ext;         // E(c, b-c) per refined community
    uint32_t *size;      // members per refined community
    uint32_t *T;         // decision of each vertex of the current wave
    double *wvt;         // E(v, T[v]) at the decision
    uint8_t *targeted;   // refined communities some mover of the wave targets
    uint8_t *joined;     // movers of the wave that joined their target
    unsigned long long *moves;
    double two_m;
    double theta;
    uint64_t pass_key;
};

// Up to NUM_CLS slices of the class/wave list, addressed as one sequence.
struct Slices {
    const uint32_t *list;
    uint32_t begin[NUM_CLS];
    uint32_t prefix[NUM_CLS + 1];
    int n;
    __device__ __forceinline__ uint32_t at(uint32_t i) const {
        int k = 0;
        while (k + 1 < n && i >= prefix[k + 1]) k++;
        return list[begin[k] + (i - prefix[k])];
    }
    __host__ __device__ __forceinline__ uint32_t total() const { return prefix[n]; }
};

Slices make_slices(const Classes &cl, int wave, const int *cls, int ncls) {
    Slices s;
    s.list = cl.list;
    s.n = ncls;
    s.prefix[0] = 0;
    for (int k = 0; k < ncls; k++) {
        s.begin[k] = cl.begin(cls[k], wave);
        s.prefix[k + 1] = s.prefix[k] + cl.count(cls[k], wave);
    }
    return s;
}

// v may move only while it is alone in R and well connected to its bound
// community.
__device__ __forceinline__ bool may_move(const RefineState &a, uint32_t v) {
    if (a.R[v] != v || a.size[v] != 1) return false;
    double Kv = a.K[v];
    double thr = __ddiv_rn(__dmul_rn(Kv, __dsub_rn(a.SB[a.B[v]], Kv)), a.two_m);
    return a.ext[v] >= thr;
}

// Candidate c with E(v, c) = Hc: its score, or false when c is not eligible.
__device__ __forceinline__ bool candidate_score(const RefineState &a, uint32_t v, double Kv, double SBb,
                                                uint32_t c, double Hc, double *score) {
    double SRc = a.SR[c];
    double thr = __ddiv_rn(__dmul_rn(SRc, __dsub_rn(SBb, SRc)), a.two_m);
    if (!(a.ext[c] >= thr)) return false;
    double gain = __dsub_rn(Hc, __ddiv_rn(__dmul_rn(Kv, SRc), a.two_m));
    if (a.theta > 0.0) {
        if (gain < 0.0) return false;
        *score = __dadd_rn(__ddiv_rn(gain, a.theta), gumbel(a.pass_key, v, c));
    } else {
        if (!(gain > 0.0)) return false;
        *score = gain;
    }
    return true;
}

struct Best {
    double s;
    double h;
    uint32_t c;
    int have;
};

__device__ __forceinline__ bool better(const Best &x, const Best &y) {
    if (!x.have) return false;
    if (!y.have) return true;
    return x.s > y.s || (x.s == y.s && x.c < y.c);
}

__device__ __forceinline__ Best warp_best(Best b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Best y;
        y.s = __shfl_xor_sync(0xFFFFFFFFu, b.s, o);
        y.h = __shfl_xor_sync(0xFFFFFFFFu, b.h, o);
        y.c = __shfl_xor_sync(0xFFFFFFFFu, b.c, o);
        y.have = __shfl_xor_sync(0xFFFFFFFFu, b.have, o);
        if (better(y, b)) b = y;
    }
    return b;
}

// Staying is a candidate (gain 0) of the random choice only.
__device__ __forceinline__ Best initial_best(const RefineState &a, uint32_t v, bool first) {
    Best b{0.0, 0.0, v, 0};
    if (first && a.theta > 0.0) {
        b.have = 1;
        b.s = gumbel(a.pass_key, v, v);
    }
    return b;
}

__device__ __forceinline__ void record(const RefineState &a, uint32_t v, const Best &b) {
    uint32_t c = b.have ? b.c : v;
    a.T[v] = c;
    a.wvt[v] = c != v ? b.h : 0.0;
}

// Degrees up to the group classes' bound: one warp per vertex, a 256-slot
// table per warp in shared memory.
template <typename WT>
__global__ void __launch_bounds__(RF_THREADS) k_refine_decide_warp(RefineState a, Slices sl) {
    __shared__ uint32_t skeys[RF_WARPS][RF_WARP_SLOTS];
    __shared__ double svals[RF_WARPS][RF_WARP_SLOTS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *keys = skeys[wid];
    double *vals = svals[wid];
    const WT *w = static_cast<const WT *>(a.w);
    const uint32_t total = sl.total();
    for (uint32_t t = blockIdx.x * RF_WARPS + wid; t < total; t += gridDim.x * RF_WARPS) {
        const uint32_t v = sl.at(t);
        if (!may_move(a, v)) {
            if (lane == 0) record(a, v, Best{0.0, 0.0, v, 0});
            continue;
        }
        for (int s = lane; s < RF_WARP_SLOTS; s += 32) {
            keys[s] = EMPTY;
            vals[s] = 0.0;
        }
        __syncwarp();
        const uint32_t b = a.B[v];
        for (uint64_t e = a.off[v] + lane; e < a.off[v + 1]; e += 32) {
            uint32_t u = a.tgt[e];
            if (u != v && a.B[u] == b) ht_add<double>(keys, vals, 8, a.R[u], wload(w, e));
        }
        __syncwarp();
        const double Kv = a.K[v], SBb = a.SB[b];
        Best best = initial_best(a, v, lane == 0);
        for (int s = lane; s < RF_WARP_SLOTS; s += 32) {
            uint32_t c = keys[s];
            if (c == EMPTY) continue;
            Best y{0.0, vals[s], c, 0};
            if (candidate_score(a, v, Kv, SBb, c, y.h, &y.s)) {
                y.have = 1;
                if (better(y, best)) best = y;
            }
        }
        best = warp_best(best);
        if (lane == 0) record(a, v, best);
        __syncwarp();
    }
}

// Larger degrees: one block per vertex; the table (2^logcap slots) in
// dynamic shared memory, or for the largest degrees in the hub pool (slots
// pool_off[t] .. pool_off[t+1] of the vertex at position t).
template <typename WT, bool POOL>
__global__ void __launch_bounds__(RF_THREADS) k_refine_decide_block(RefineState a, Slices sl, int logcap,
                                                                    const uint64_t *pool_off, uint32_t *pool_keys,
                                                                    double *pool_vals) {
    extern __shared__ __align__(16) unsigned char rf_smem[];
    __shared__ Best sbest[RF_WARPS];
    __shared__ int s_go;
    const WT *w = static_cast<const WT *>(a.w);
    const uint32_t total = sl.total();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        const uint32_t v = sl.at(t);
        if (threadIdx.x == 0) s_go = may_move(a, v);
        __syncthreads();
        if (!s_go) {
            if (threadIdx.x == 0) record(a, v, Best{0.0, 0.0, v, 0});
            __syncthreads();
            continue;
        }
        uint32_t *keys;
        double *vals;
        uint32_t cap;
        int lg;
        if (POOL) {
            keys = pool_keys + pool_off[t];
            vals = pool_vals + pool_off[t];
            cap = (uint32_t)(pool_off[t + 1] - pool_off[t]);
            lg = 31 - __clz(cap);
        } else {
            cap = 1u << logcap;
            lg = logcap;
            vals = reinterpret_cast<double *>(rf_smem);
            keys = reinterpret_cast<uint32_t *>(rf_smem + sizeof(double) * cap);
        }
        for (uint32_t s = threadIdx.x; s < cap; s += blockDim.x) {
            keys[s] = EMPTY;
            vals[s] = 0.0;
        }
        __syncthreads();
        const uint32_t b = a.B[v];
        for (uint64_t e = a.off[v] + threadIdx.x; e < a.off[v + 1]; e += blockDim.x) {
            uint32_t u = a.tgt[e];
            if (u != v && a.B[u] == b) ht_add<double>(keys, vals, lg, a.R[u], wload(w, e));
        }
        __syncthreads();
        const double Kv = a.K[v], SBb = a.SB[b];
        Best best = initial_best(a, v, threadIdx.x == 0);
        for (uint32_t s = threadIdx.x; s < cap; s += blockDim.x) {
            uint32_t c = keys[s];
            if (c == EMPTY) continue;
            Best y{0.0, vals[s], c, 0};
            if (candidate_score(a, v, Kv, SBb, c, y.h, &y.s)) {
                y.have = 1;
                if (better(y, best)) best = y;
            }
        }
        best = warp_best(best);
        if (lane == 0) sbest[wid] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            Best r = sbest[0];
            for (int k = 1; k < RF_WARPS; k++)
                if (better(sbest[k], r)) r = sbest[k];
            record(a, v, r);
        }
        __syncthreads();
    }
}

__global__ void k_refine_mark(RefineState a, Slices sl) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < sl.total(); t += gridDim.x * blockDim.x) {
        uint32_t v = sl.at(t);
        uint32_t c = a.T[v];
        if (c != v) a.targeted[c] = 1;
    }
}

__global__ void k_refine_apply(RefineState a, Slices sl) {
    unsigned long long moved = 0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < sl.total(); t += gridDim.x * blockDim.x) {
        uint32_t v = sl.at(t);
        uint32_t c = a.T[v];
        bool j = c != v && !a.targeted[v];
        a.joined[v] = j;
        if (!j) continue;
        a.R[v] = c;
        atomicAdd(&a.size[c], 1u);
        a.size[v] = 0;
        atomicAdd(&a.SR[c], a.K[v]);
        moved++;
    }
    moved = warp_sum(moved);
    if ((threadIdx.x & 31) == 0 && moved) atomicAdd(a.moves, moved);
}

// E(c, b-c) of each target: one warp per joiner.
template <typename WT>
__global__ void k_refine_ext_update(RefineState a, Slices sl) {
    const int lane = threadIdx.x & 31;
    const WT *w = static_cast<const WT *>(a.w);
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < sl.total(); t += warps) {
        uint32_t v = sl.at(t);
        if (!a.joined[v]) continue;
        const uint32_t c = a.T[v];
        double co = 0.0;
        for (uint64_t e = a.off[v] + lane; e < a.off[v + 1]; e += 32) {
            uint32_t u = a.tgt[e];
            if (u != v && a.joined[u] && a.T[u] == c) co += wload(w, e);
        }
        co = warp_sum(co);
        if (lane == 0) atomicAdd(&a.ext[c], __dsub_rn(__dsub_rn(a.ext[v], __dmul_rn(2.0, a.wvt[v])), co));
    }
}

__global__ void k_refine_clear(RefineState a, Slices sl) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < sl.total(); t += gridDim.x * blockDim.x) {
        uint32_t v = sl.at(t);
        a.targeted[a.T[v]] = 0;
        a.joined[v] = 0;
    }
}

__global__ void k_refine_init(const uint32_t *B, const double *K, uint32_t *R, double *SR, uint32_t *size,
                              double *SB, uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        R[v] = v;
        SR[v] = K[v];
        size[v] = 1;
        atomicAdd(&SB[B[v]], K[v]);
    }
}

// E(v, b-v) of every vertex: one warp per vertex.
template <typename WT>
__global__ void k_refine_ext_init(const uint64_t *off, const uint32_t *tgt, const WT *w, const uint32_t *B,
                                  double *ext, uint32_t n) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint32_t b = B[v];
        double x = 0.0;
        for (uint64_t e = off[v] + lane; e < off[v + 1]; e += 32) {
            uint32_t u = tgt[e];
            if (u != v && B[u] == b) x += wload(w, e);
        }
        x = warp_sum(x);
        if (lane == 0) ext[v] = x;
    }
}

template <typename K>
unsigned block_grid(K kernel, size_t smem, uint32_t work) {
    if (!work) return 0;
    unsigned g = resident_grid(reinterpret_cast<const void *>(kernel), RF_THREADS, smem, 8);
    return work < g ? work : g;
}

template <typename WT>
uint32_t refine_impl(const DevGraph &g, const Classes &cl, const uint32_t *B, uint32_t *R, const double *K, double m,
                     double theta, uint64_t seed, uint32_t pass, cudaStream_t s) {
    const uint32_t n = g.n;
    size_t mk = arena().mark();
    RefineState a;
    a.off = g.off;
    a.tgt = g.tgt;
    a.w = g.w;
    a.B = B;
    a.R = R;
    a.K = K;
    double *SB = arena().get<double>(n);
    a.SB = SB;
    a.SR = arena().get<double>(n);
    a.ext = arena().get<double>(n);
    a.size = arena().get<uint32_t>(n);
    a.T = arena().get<uint32_t>(n);
    a.wvt = arena().get<double>(n);
    a.targeted = arena().get<uint8_t>(n);
    a.joined = arena().get<uint8_t>(n);
    a.moves = arena().get<unsigned long long>(1);
    a.two_m = 2.0 * m;
    a.theta = theta;
    a.pass_key = splitmix64(seed + GOLDEN_GAMMA * ((uint64_t)pass + 1));
    GSP_CUDA(cudaMemsetAsync(SB, 0, sizeof(double) * n, s));
    GSP_CUDA(cudaMemsetAsync(a.targeted, 0, n, s));
    GSP_CUDA(cudaMemsetAsync(a.joined, 0, n, s));
    GSP_CUDA(cudaMemsetAsync(a.moves, 0, sizeof(unsigned long long), s));
    k_refine_init<<<grid_for(n, 256), 256, 0, s>>>(B, K, R, a.SR, a.size, SB, n);
    GSP_CHECK_LAUNCH();
    k_refine_ext_init<WT><<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(g.off, g.tgt, static_cast<const WT *>(g.w),
                                                                            B, a.ext, n);
    GSP_CHECK_LAUNCH();
    if (!(m > 0.0)) {  // edgeless: every vertex stays alone
        unsigned long long z = 0;
        arena().release(mk);
        return (uint32_t)z;
    }
    // hub tables in a pool of their own (keys, then values)
    uint32_t nh = cl.cls_count(CLS_HUGE);
    uint32_t *pkeys = nullptr;
    double *pvals = nullptr;
    if (nh) {
        size_t sa = align_up(cl.pool_slots, 64);
        pvals = arena().get<double>(sa);
        pkeys = arena().get<uint32_t>(sa);
    }
    const int small[] = {CLS_G4, CLS_G8, CLS_G16, CLS_G32};
    const int mid[] = {CLS_W512, CLS_BLOCK};
    const int big[] = {CLS_BIG};
    const int huge[] = {CLS_HUGE};
    const int all[] = {CLS_G4, CLS_G8, CLS_G16, CLS_G32, CLS_W512, CLS_BLOCK, CLS_BIG, CLS_HUGE};
    constexpr int MID_LOG = 12, BIG_LOG = 14;  // 2x the classes' largest degrees
    const size_t mid_smem = (sizeof(double) + sizeof(uint32_t)) << MID_LOG;
    const size_t big_smem = (sizeof(double) + sizeof(uint32_t)) << BIG_LOG;
    static_assert((1u << MID_LOG) >= 2 * BLOCK_MAX_LIMIT && (1u << BIG_LOG) >= 2 * BIG_MAX_LIMIT,
                  "refinement tables hold twice the largest degree of their classes");
    static_assert(RF_WARP_SLOTS >= 2 * GROUP_MAX_LIMIT, "warp tables hold twice the group classes' degrees");
    auto kmid = k_refine_decide_block<WT, false>;
    auto kpool = k_refine_decide_block<WT, true>;
    GSP_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(kmid), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)big_smem));
    for (int wv = 0; wv < cl.W; wv++) {
        Slices ss = make_slices(cl, wv, small, 4), sm = make_slices(cl, wv, mid, 2),
               sb = make_slices(cl, wv, big, 1), sh = make_slices(cl, wv, huge, 1),
               sa = make_slices(cl, wv, all, NUM_CLS);
        if (!sa.total()) continue;
        if (ss.total()) {
            k_refine_decide_warp<WT><<<grid_for(ss.total(), RF_WARPS, sms(8)), RF_THREADS, 0, s>>>(a, ss);
            GSP_CHECK_LAUNCH();
        }
        if (sm.total()) {
            kmid<<<block_grid(kmid, mid_smem, sm.total()), RF_THREADS, mid_smem, s>>>(a, sm, MID_LOG, nullptr,
                                                                                      nullptr, nullptr);
            GSP_CHECK_LAUNCH();
        }
        if (sb.total()) {
            kmid<<<block_grid(kmid, big_smem, sb.total()), RF_THREADS, big_smem, s>>>(a, sb, BIG_LOG, nullptr,
                                                                                      nullptr, nullptr);
            GSP_CHECK_LAUNCH();
        }
        if (sh.total()) {
            const uint64_t *po = cl.pool_off + (cl.begin(CLS_HUGE, wv) - cl.cls_begin(CLS_HUGE));
            kpool<<<block_grid(kpool, 0, sh.total()), RF_THREADS, 0, s>>>(a, sh, 0, po, pkeys, pvals);
            GSP_CHECK_LAUNCH();
        }
        const unsigned gv = grid_for(sa.total(), 256, sms(8));
        k_refine_mark<<<gv, 256, 0, s>>>(a, sa);
        GSP_CHECK_LAUNCH();
        k_refine_apply<<<gv, 256, 0, s>>>(a, sa);
        GSP_CHECK_LAUNCH();
        k_refine_ext_update<WT><<<grid_for((uint64_t)sa.total() * 32, 256, sms(8)), 256, 0, s>>>(a, sa);
        GSP_CHECK_LAUNCH();
        k_refine_clear<<<gv, 256, 0, s>>>(a, sa);
        GSP_CHECK_LAUNCH();
    }
    unsigned long long moves = 0;
    GSP_CUDA(cudaMemcpyAsync(&moves, a.moves, sizeof(moves), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    return (uint32_t)moves;
}

}  // namespace

namespace {
__global__ void k_sigma_from_membership(const uint32_t *C, const double *K, double *Sigma, uint32_t *size,
                                        uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        atomicAdd(&Sigma[C[v]], K[v]);
        atomicAdd(&size[C[v]], 1u);
    }
}

__global__ void k_scatter_bound(const uint32_t *R, const uint32_t *B, uint32_t *C_next, uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) C_next[R[v]] = B[v];
}
}  // namespace

void sigma_from_membership(const uint32_t *C, const double *K, double *Sigma, uint32_t *size, uint32_t n,
                           cudaStream_t s) {
    GSP_CUDA(cudaMemsetAsync(Sigma, 0, sizeof(double) * n, s));
    GSP_CUDA(cudaMemsetAsync(size, 0, sizeof(uint32_t) * n, s));
    k_sigma_from_membership<<<grid_for(n, 256), 256, 0, s>>>(C, K, Sigma, size, n);
    GSP_CHECK_LAUNCH();
}

void scatter_bound(const uint32_t *R, const uint32_t *B, uint32_t *C_next, uint32_t n, cudaStream_t s) {
    k_scatter_bound<<<grid_for(n, 256), 256, 0, s>>>(R, B, C_next, n);
    GSP_CHECK_LAUNCH();
}

uint32_t refine_partition(const DevGraph &g, const Classes &cl, const uint32_t *B, uint32_t *R, const double *K,
                          double m, double theta, uint64_t seed, uint32_t pass, cudaStream_t s) {
    GSP_REQUIRE(theta >= 0.0 && theta == theta, "refine_theta must be >= 0");
    if (g.wt == GSP_W_F64) return refine_impl<double>(g, cl, B, R, K, m, theta, seed, pass, s);
    return refine_impl<float>(g, cl, B, R, K, m, theta, seed, pass, s);
}

}  // namespace gsp
