// move.cu -- local-moving phase of GSP-Louvain (Algorithm 4, louvainMove and
// scanCommunities) on sm_103a.
//
// Each active vertex i gathers K_{i->c} for every neighbouring community c
// (self-loop excluded) into an open-addressing hashtable, scores every
// candidate with Equation 2 and takes the argmax (ties to the lowest id);
// it moves only on a strictly positive gain.  The work is binned by degree:
//   groups of G = 4/8/16/32 lanes per vertex, table in shared memory;
//   one block per vertex, table in shared memory (degree <= 4096);
//   one block per vertex, table in a global-memory pool (larger degrees).
// Duplicate community keys meet in the table through atomicCAS on the key and
// atomicAdd on the value.
//
// Precision: FP64 evaluates Equation 2 term by term with round-to-nearest
// intrinsics (no fused multiply-add), exactly as written, so its choices can
// be compared with a sequential FP64 evaluation.  MIXED accumulates K_{i->c}
// in float32 and compares the scaled score s_c = K_{i->c} - K_i * Sigma_c / 2m
// in float32 (m * dQ_{i:d->c} = s_c - s_d with Sigma_d taken without K_i);
// m and Sigma stay float64.
//
// Modes: SYNC reads the state of the sweep's start and writes the next state
// (deterministic); ASYNC reads and writes one state in place, as the
// paper's parallel loop does, with L2-coherent loads (ld.global.cg) for
// values other threads update.
#include <type_traits>

#include "internal.cuh"

namespace gsp {

struct MoveArgs {
    const uint64_t *off;
    const uint32_t *tgt;
    const void *w;
    const uint32_t *C;     // read
    uint32_t *Cw;          // write
    const double *K;
    const double *Sig;     // read
    double *Sigw;          // write (atomics)
    const uint32_t *size;  // read
    uint32_t *sizew;
    const uint8_t *act;    // read
    uint8_t *actw;         // write (re-marking); ASYNC: same as act
    const double *m;
    MoveCounters *ctr;
    int rule;
    // learned pruning
    const float *mlp;
    float *feat_dq;
    uint8_t *moved_last;
    int learned;
};

template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
__device__ __forceinline__ uint8_t ldcg(const uint8_t *p) {
    return (uint8_t)__ldcg(reinterpret_cast<const unsigned char *>(p));
}

template <bool SYNC, typename T> __device__ __forceinline__ T ld_state(const T *p) {
    if constexpr (SYNC) return __ldg(p);
    else return ldcg(p);
}

template <typename V, typename WT> __device__ __forceinline__ V load_w(const WT *w, uint64_t e) {
    return (V)__ldg(w + e);
}

// Equation 2, evaluated in the order written, with no contraction.
__device__ __forceinline__ double eq2(double Kic, double Kid, double Ki, double Sc, double Sd, double m) {
    double t1 = __ddiv_rn(__dsub_rn(Kic, Kid), m);
    double t2 = __dmul_rn(Ki, __dsub_rn(__dadd_rn(Ki, Sc), Sd));
    double den = __dmul_rn(__dmul_rn(2.0, m), m);
    return __dsub_rn(t1, __ddiv_rn(t2, den));
}

template <typename S> __device__ __forceinline__ bool better(S s1, uint32_t c1, S s2, uint32_t c2) {
    return s1 > s2 || (s1 == s2 && c1 < c2);
}

// Per-vertex scoring context.
template <bool F64> struct Score;
template <> struct Score<true> {
    using S = double;
    double Ki, Kid, Sd, m;
    __device__ S score(double kic, double Sc) const { return eq2(kic, Kid, Ki, Sc, Sd, m); }
    __device__ double gain(S best) const { return best; }           // in units of Q
};
template <> struct Score<false> {
    using S = float;
    float kif, sd;
    double m;
    __device__ S score(float kic, double Sc) const { return kic - kif * (float)Sc; }
    __device__ double gain(S best) const { return (double)(best - sd) / m; }
};

template <bool F64>
__device__ __forceinline__ Score<F64> make_score(double Ki, double kid, double Sd, double m);
template <> __device__ __forceinline__ Score<true> make_score<true>(double Ki, double kid, double Sd, double m) {
    Score<true> s;
    s.Ki = Ki; s.Kid = kid; s.Sd = Sd; s.m = m;
    return s;
}
template <> __device__ __forceinline__ Score<false> make_score<false>(double Ki, double kid, double Sd, double m) {
    Score<false> s;
    double inv2m = 0.5 / m;
    s.kif = (float)(Ki * inv2m);
    s.sd = (float)kid - (float)(Ki * inv2m) * (float)(Sd - Ki);
    s.m = m;
    return s;
}

// Decide and apply the move of i (called by one thread).
template <bool SYNC>
__device__ __forceinline__ bool apply_move(const MoveArgs &a, uint32_t i, uint32_t d, uint32_t c, double Ki) {
    if (c == EMPTY || c == d) return false;
    if (a.rule) {
        uint32_t sd = ld_state<SYNC>(a.size + d), sc = ld_state<SYNC>(a.size + c);
        if (sd == 1 && sc == 1 && c > d) return false;
    }
    a.Cw[i] = c;
    atomicAdd(a.Sigw + d, -Ki);
    atomicAdd(a.Sigw + c, Ki);
    atomicSub(a.sizew + d, 1u);
    atomicAdd(a.sizew + c, 1u);
    return true;
}

struct LocalCtr {
    double dq = 0;
    unsigned long long moved = 0, vertices = 0, edges = 0, candidates = 0, marked = 0;
};

__device__ void flush_counters(const LocalCtr &l, MoveCounters *g) {
    __shared__ double sd[32];
    __shared__ unsigned long long su[32];
    double dq = block_sum<double>(l.dq, sd);
    unsigned long long mv = block_sum<unsigned long long>(l.moved, su);
    unsigned long long vx = block_sum<unsigned long long>(l.vertices, su);
    unsigned long long ed = block_sum<unsigned long long>(l.edges, su);
    unsigned long long ca = block_sum<unsigned long long>(l.candidates, su);
    unsigned long long mk = block_sum<unsigned long long>(l.marked, su);
    if (threadIdx.x == 0) {
        if (mk) atomicAdd(&g->marked, mk);
        if (dq != 0.0) atomicAdd(&g->dq, dq);
        if (mv) atomicAdd(&g->moved, mv);
        if (vx) atomicAdd(&g->vertices, vx);
        if (ed) atomicAdd(&g->edges, ed);
        if (ca) atomicAdd(&g->candidates, ca);
    }
}

// --------------------------------------------------------------------------
// Groups of G lanes, one vertex per group, table of up to CAP slots per group.
// --------------------------------------------------------------------------
template <int G, int CAP, typename WT, bool F64, bool SYNC>
__global__ void __launch_bounds__(256) k_move_group(MoveArgs a, const uint32_t *__restrict__ list,
                                                    uint32_t count) {
    using V = typename std::conditional<F64, double, float>::type;
    using SC = Score<F64>;
    using S = typename SC::S;
    constexpr int NG = 256 / G;
    __shared__ uint32_t s_keys[NG][CAP];
    __shared__ V s_vals[NG][CAP];
    const int lane = threadIdx.x % G;
    const int grp = threadIdx.x / G;
    const unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    uint32_t *keys = s_keys[grp];
    V *vals = s_vals[grp];
    const WT *w = static_cast<const WT *>(a.w);
    const double m = *a.m;
    LocalCtr lc;
    for (uint32_t idx = blockIdx.x * NG + grp; idx < count; idx += gridDim.x * NG) {
        uint32_t i = list[idx];
        // one lane reads the flag (other threads may be re-marking it) and
        // marks the vertex processed; the group follows its decision
        int go = 0;
        if (lane == 0) {
            go = ld_state<SYNC>(a.act + i);
            if (!SYNC && go) a.actw[i] = 0;
        }
        go = __shfl_sync(gmask, go, (threadIdx.x & 31) & ~(G - 1));
        if (!go) continue;
        uint32_t d = ld_state<SYNC>(a.C + i);
        uint64_t b = a.off[i], e = a.off[i + 1];
        uint32_t deg = (uint32_t)(e - b);
        int logcap = ceil_log2(2 * deg);
        if (logcap < 1) logcap = 1;
        uint32_t cap = 1u << logcap;
        for (uint32_t s = lane; s < cap; s += G) { keys[s] = EMPTY; vals[s] = V(0); }
        __syncwarp(gmask);
        V kid = 0;
        for (uint64_t p = b + lane; p < e; p += G) {
            uint32_t j = __ldg(a.tgt + p);
            if (j == i) continue;
            V wv = load_w<V>(w, p);
            uint32_t c = ld_state<SYNC>(a.C + j);
            if (c == d) kid += wv;
            else ht_add<V>(keys, vals, logcap, c, wv);
        }
        __syncwarp(gmask);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) kid += __shfl_xor_sync(gmask, kid, o);
        double Ki = a.K[i];
        double Sd = ld_state<SYNC>(a.Sig + d);
        Sd = __shfl_sync(gmask, Sd, (threadIdx.x & 31) & ~(G - 1));
        SC sc = make_score<F64>(Ki, (double)kid, Sd, m);
        S best = -INFINITY;
        uint32_t bestc = EMPTY;
        uint32_t ncand = 0;
        for (uint32_t s = lane; s < cap; s += G) {
            uint32_t c = keys[s];
            if (c == EMPTY) continue;
            ncand++;
            S v = sc.score(vals[s], ld_state<SYNC>(a.Sig + c));
            if (better(v, c, best, bestc)) { best = v; bestc = c; }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            S v2 = __shfl_xor_sync(gmask, best, o);
            uint32_t c2 = __shfl_xor_sync(gmask, bestc, o);
            if (better(v2, c2, best, bestc)) { best = v2; bestc = c2; }
        }
        lc.candidates += ncand;
        double gain = (bestc == EMPTY) ? 0.0 : sc.gain(best);
        int mv = 0;
        if (lane == 0) {
            lc.vertices++;
            lc.edges += deg;
            if (gain > 0.0) mv = apply_move<SYNC>(a, i, d, bestc, Ki);
            if (mv) { lc.moved++; lc.dq += gain; lc.marked += deg; }
        }
        mv = __shfl_sync(gmask, mv, (threadIdx.x & 31) & ~(G - 1));
        if (mv) {
            for (uint64_t p = b + lane; p < e; p += G) {
                uint32_t j = __ldg(a.tgt + p);
                if (j != i) a.actw[j] = 1;
            }
        }
        __syncwarp(gmask);
    }
    flush_counters(lc, a.ctr);
}

// --------------------------------------------------------------------------
// One block per vertex; table in shared memory (CAP > 0) or in the global
// pool (CAP == 0, slots at pool_off[idx]).
// --------------------------------------------------------------------------
template <int CAP, typename WT, bool F64, bool SYNC>
__global__ void __launch_bounds__(256) k_move_block(MoveArgs a, const uint32_t *__restrict__ list, uint32_t count,
                                                    const uint64_t *__restrict__ pool_off, uint32_t *pool_keys,
                                                    void *pool_vals) {
    using V = typename std::conditional<F64, double, float>::type;
    using SC = Score<F64>;
    using S = typename SC::S;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    uint32_t *s_keys = reinterpret_cast<uint32_t *>(dyn_smem);
    V *s_vals = reinterpret_cast<V *>(dyn_smem + (size_t)CAP * sizeof(uint32_t));
    __shared__ S red_s[32];
    __shared__ uint32_t red_c[32];
    __shared__ V red_k[32];
    __shared__ int s_mv;
    __shared__ double s_Sd;
    const WT *w = static_cast<const WT *>(a.w);
    const double m = *a.m;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    LocalCtr lc;
    for (uint32_t idx = blockIdx.x; idx < count; idx += gridDim.x) {
        uint32_t i = list[idx];
        __syncthreads();  // previous vertex done with the table and reductions
        if (threadIdx.x == 0) {
            int go = ld_state<SYNC>(a.act + i);
            if (!SYNC && go) a.actw[i] = 0;
            s_mv = go;
            if (go) s_Sd = ld_state<SYNC>(a.Sig + ld_state<SYNC>(a.C + i));
        }
        __syncthreads();
        if (!s_mv) continue;
        uint32_t d = ld_state<SYNC>(a.C + i);
        uint64_t b = a.off[i], e = a.off[i + 1];
        uint32_t deg = (uint32_t)(e - b);
        int logcap = ceil_log2(2 * deg);
        if (logcap < 1) logcap = 1;
        uint32_t cap = 1u << logcap;
        uint32_t *keys = s_keys;
        V *vals = s_vals;
        if (CAP == 0) {
            keys = pool_keys + pool_off[idx];
            vals = static_cast<V *>(pool_vals) + pool_off[idx];
        }
        for (uint32_t s = threadIdx.x; s < cap; s += blockDim.x) { keys[s] = EMPTY; vals[s] = V(0); }
        __syncthreads();
        V kid = 0;
        for (uint64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
            uint32_t j = __ldg(a.tgt + p);
            if (j == i) continue;
            V wv = load_w<V>(w, p);
            uint32_t c = ld_state<SYNC>(a.C + j);
            if (c == d) kid += wv;
            else ht_add<V>(keys, vals, logcap, c, wv);
        }
        kid = warp_sum(kid);
        if (lane == 0) red_k[wid] = kid;
        __syncthreads();
        kid = 0;
        for (int t = 0; t < nw; t++) kid += red_k[t];
        double Ki = a.K[i];
        SC sc = make_score<F64>(Ki, (double)kid, s_Sd, m);
        S best = -INFINITY;
        uint32_t bestc = EMPTY;
        uint32_t ncand = 0;
        for (uint32_t s = threadIdx.x; s < cap; s += blockDim.x) {
            uint32_t c = keys[s];
            if (c == EMPTY) continue;
            ncand++;
            S v = sc.score(vals[s], ld_state<SYNC>(a.Sig + c));
            if (better(v, c, best, bestc)) { best = v; bestc = c; }
        }
        lc.candidates += ncand;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S v2 = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            uint32_t c2 = __shfl_xor_sync(0xFFFFFFFFu, bestc, o);
            if (better(v2, c2, best, bestc)) { best = v2; bestc = c2; }
        }
        if (lane == 0) { red_s[wid] = best; red_c[wid] = bestc; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = 1; t < nw; t++)
                if (better(red_s[t], red_c[t], best, bestc)) { best = red_s[t]; bestc = red_c[t]; }
            double gain = (bestc == EMPTY) ? 0.0 : sc.gain(best);
            int mv = 0;
            if (gain > 0.0) mv = apply_move<SYNC>(a, i, d, bestc, Ki);
            lc.vertices++;
            lc.edges += deg;
            if (mv) { lc.moved++; lc.dq += gain; lc.marked += deg; }
            s_mv = mv;
        }
        __syncthreads();
        if (s_mv) {
            for (uint64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
                uint32_t j = __ldg(a.tgt + p);
                if (j != i) a.actw[j] = 1;
            }
        }
    }
    __syncthreads();
    flush_counters(lc, a.ctr);
}

// --------------------------------------------------------------------------
// Degree classes
// --------------------------------------------------------------------------
__device__ __forceinline__ int class_of(uint64_t deg) {
    if (deg <= 8) return CLS_G4;
    if (deg <= 16) return CLS_G8;
    if (deg <= 32) return CLS_G16;
    if (deg <= 128) return CLS_G32;
    if (deg <= 4096) return CLS_BLOCK;
    return CLS_HUGE;
}

__global__ void k_classify_count(const uint64_t *__restrict__ off, uint32_t n, uint32_t *counts) {
    __shared__ uint32_t sc[NUM_CLS];
    if (threadIdx.x < NUM_CLS) sc[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t deg = off[v + 1] - off[v];
        if (deg) atomicAdd(&sc[class_of(deg)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NUM_CLS && sc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sc[threadIdx.x]);
}

__global__ void k_classify_fill(const uint64_t *__restrict__ off, uint32_t n, uint32_t *cursor, uint32_t *list) {
    int lane = threadIdx.x & 31;
    for (uint32_t v0 = blockIdx.x * blockDim.x; v0 < n; v0 += gridDim.x * blockDim.x) {
        uint32_t v = v0 + threadIdx.x;
        uint64_t deg = (v < n) ? off[v + 1] - off[v] : 0;
        int cls = deg ? class_of(deg) : -1;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, cls);
        int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && cls >= 0) base = atomicAdd(&cursor[cls], (uint32_t)__popc(peers));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (cls >= 0) list[base + __popc(peers & ((1u << lane) - 1u))] = v;
    }
}

__global__ void k_pool_caps(const uint64_t *__restrict__ off, const uint32_t *__restrict__ list, uint32_t count,
                            uint64_t *caps) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        uint32_t v = list[t];
        uint64_t deg = off[v + 1] - off[v];
        uint64_t cap = 2;
        while (cap < 2 * deg) cap <<= 1;
        caps[t] = cap;
    }
}

void classify_vertices(const DevGraph &g, Classes &cl, cudaStream_t s) {
    uint32_t *counts = arena().get<uint32_t>(2 * NUM_CLS);
    GSP_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * NUM_CLS, s));
    unsigned grid = grid_for(g.n, 256, 152 * 8);
    k_classify_count<<<grid, 256, 0, s>>>(g.off, g.n, counts);
    GSP_CHECK_LAUNCH();
    uint32_t h[NUM_CLS];
    GSP_CUDA(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    cl.start[0] = 0;
    for (int c = 0; c < NUM_CLS; c++) cl.start[c + 1] = cl.start[c] + h[c];
    uint32_t *cursor = counts + NUM_CLS;
    GSP_CUDA(cudaMemcpyAsync(cursor, cl.start, sizeof(uint32_t) * NUM_CLS, cudaMemcpyHostToDevice, s));
    cl.list = arena().get<uint32_t>(cl.start[NUM_CLS] + 1);
    k_classify_fill<<<grid, 256, 0, s>>>(g.off, g.n, cursor, cl.list);
    GSP_CHECK_LAUNCH();
    uint32_t nh = cl.start[CLS_HUGE + 1] - cl.start[CLS_HUGE];
    cl.pool_off = arena().get<uint64_t>(nh + 1);
    cl.pool_slots = 0;
    if (nh) {
        uint64_t *caps = arena().get<uint64_t>(nh);
        k_pool_caps<<<grid_for(nh, 256), 256, 0, s>>>(g.off, cl.list + cl.start[CLS_HUGE], nh, caps);
        GSP_CHECK_LAUNCH();
        exclusive_scan_u64(caps, cl.pool_off, nh, s);
        GSP_CUDA(cudaMemcpyAsync(&cl.pool_slots, cl.pool_off + nh, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
    }
}

// --------------------------------------------------------------------------
// Host launcher for one sweep
// --------------------------------------------------------------------------
template <typename WT, bool F64, bool SYNC>
static void launch_sweep(const Classes &cl, const MoveArgs &a, cudaStream_t s) {
    auto cnt = [&](int c) { return cl.start[c + 1] - cl.start[c]; };
    auto lst = [&](int c) { return cl.list + cl.start[c]; };
    const unsigned maxg = 152 * 8;
    if (cnt(CLS_G4)) {
        k_move_group<4, 16, WT, F64, SYNC><<<grid_for((uint64_t)cnt(CLS_G4) * 4, 256, maxg), 256, 0, s>>>(
            a, lst(CLS_G4), cnt(CLS_G4));
        GSP_CHECK_LAUNCH();
    }
    if (cnt(CLS_G8)) {
        k_move_group<8, 32, WT, F64, SYNC><<<grid_for((uint64_t)cnt(CLS_G8) * 8, 256, maxg), 256, 0, s>>>(
            a, lst(CLS_G8), cnt(CLS_G8));
        GSP_CHECK_LAUNCH();
    }
    if (cnt(CLS_G16)) {
        k_move_group<16, 64, WT, F64, SYNC><<<grid_for((uint64_t)cnt(CLS_G16) * 16, 256, maxg), 256, 0, s>>>(
            a, lst(CLS_G16), cnt(CLS_G16));
        GSP_CHECK_LAUNCH();
    }
    if (cnt(CLS_G32)) {
        k_move_group<32, 256, WT, F64, SYNC><<<grid_for((uint64_t)cnt(CLS_G32) * 32, 256, maxg), 256, 0, s>>>(
            a, lst(CLS_G32), cnt(CLS_G32));
        GSP_CHECK_LAUNCH();
    }
    if (cnt(CLS_BLOCK)) {
        using V = typename std::conditional<F64, double, float>::type;
        constexpr int CAP = 8192;
        constexpr size_t smem = (size_t)CAP * (sizeof(uint32_t) + sizeof(V));
        static bool attr = false;
        if (!attr) {
            GSP_CUDA(cudaFuncSetAttribute(k_move_block<CAP, WT, F64, SYNC>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = true;
        }
        k_move_block<CAP, WT, F64, SYNC><<<grid_for(cnt(CLS_BLOCK), 1, 152 * 2), 256, smem, s>>>(
            a, lst(CLS_BLOCK), cnt(CLS_BLOCK), nullptr, nullptr, nullptr);
        GSP_CHECK_LAUNCH();
    }
}

template <typename WT, bool F64, bool SYNC>
static void launch_huge(const Classes &cl, const MoveArgs &a, uint32_t *pool_keys, void *pool_vals, cudaStream_t s) {
    uint32_t nh = cl.start[CLS_HUGE + 1] - cl.start[CLS_HUGE];
    if (!nh) return;
    k_move_block<0, WT, F64, SYNC><<<grid_for(nh, 1, 152 * 4), 256, 0, s>>>(
        a, cl.list + cl.start[CLS_HUGE], nh, cl.pool_off, pool_keys, pool_vals);
    GSP_CHECK_LAUNCH();
}

void move_sweep(const DevGraph &g, const Classes &cl, MoveBuffers &mb, bool sync, bool fp64, bool rule,
                bool learned, cudaStream_t s) {
    MoveArgs a;
    a.off = g.off;
    a.tgt = g.tgt;
    a.w = g.w;
    a.C = mb.C;
    a.Cw = sync ? mb.C2 : mb.C;
    a.K = mb.K;
    a.Sig = mb.Sigma;
    a.Sigw = sync ? mb.Sigma2 : mb.Sigma;
    a.size = mb.size;
    a.sizew = sync ? mb.size2 : mb.size;
    a.act = mb.act;
    a.actw = sync ? mb.act2 : mb.act;
    a.m = mb.m_dev;
    a.ctr = mb.ctr;
    a.rule = rule ? 1 : 0;
    a.mlp = mb.mlp;
    a.feat_dq = mb.feat_dq;
    a.moved_last = mb.moved_last;
    a.learned = learned ? 1 : 0;
    uint32_t *pool_keys = static_cast<uint32_t *>(mb.pool);
    void *pool_vals = pool_keys ? static_cast<void *>(pool_keys + align_up(cl.pool_slots, 64)) : nullptr;
#define GSP_SWEEP(WT, F64, SYNC)                                   \
    do {                                                           \
        launch_sweep<WT, F64, SYNC>(cl, a, s);                     \
        launch_huge<WT, F64, SYNC>(cl, a, pool_keys, pool_vals, s); \
    } while (0)
    if (g.wt == GSP_W_F32) {
        if (fp64) { if (sync) GSP_SWEEP(float, true, true); else GSP_SWEEP(float, true, false); }
        else { if (sync) GSP_SWEEP(float, false, true); else GSP_SWEEP(float, false, false); }
    } else {
        if (fp64) { if (sync) GSP_SWEEP(double, true, true); else GSP_SWEEP(double, true, false); }
        else { if (sync) GSP_SWEEP(double, false, true); else GSP_SWEEP(double, false, false); }
    }
#undef GSP_SWEEP
}

}  // namespace gsp
