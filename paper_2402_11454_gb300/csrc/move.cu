// move.cu -- local-moving phase of GSP-Louvain (Algorithm 4, louvainMove and
// scanCommunities) on sm_103a.
//
// Each active vertex i gathers K_{i->c} for every neighbouring community c
// (self-loop excluded) into an open-addressing hashtable, scores every
// candidate with Equation 2 and takes the argmax (ties to the lowest id);
// it moves only on a strictly positive gain.  The work is binned by degree:
//   groups of G = 4/8/16/32 lanes per vertex, table in shared memory (one
//     fused launch for the four group classes);
//   one warp per vertex, 1024-slot shared table (degree <= 512);
//   one block per vertex, table in shared memory (degree <= 2048);
//   the whole grid per vertex for larger degrees ("hubs"): edge-chunk tasks
//     combined in shared memory, published to a global-memory table.
// Duplicate community keys meet in the table through atomicCAS on the key and
// atomicAdd on the value.
//
// Parallel semantics.  Frozen-state mode (deterministic): the vertices of a
// sweep are split into W interleaved waves (vertex i in wave i mod W); a wave
// reads C, Sigma and the community sizes left by the earlier waves, appends
// its moves to a list, and apply_moves() applies them (Sigma/size atomics,
// neighbour re-marking) before the next wave.  In-place mode: the paper's
// parallel loop as written, every move applied at once, with L2-coherent
// loads (ld.global.cg) for values other threads update.
//
// Precision: FP64 evaluates Equation 2 term by term with round-to-nearest
// intrinsics (no fused multiply-add), in the order written.  MIXED accumulates
// K_{i->c} in float32 and compares the scaled score s_c = K_{i->c} - K_i *
// Sigma_c / 2m in float32 (m * dQ_{i:d->c} = s_c - s_d with Sigma_d taken
// without K_i); m and Sigma stay float64.
#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace gsp {

struct MoveArgs {
    const uint64_t *off;
    const uint32_t *tgt;
    const void *w;
    uint32_t *C;
    const double *K;
    double *Sig;
    uint32_t *size;
    uint8_t *act;
    uint8_t *mark;  // re-marking target: a separate array merged after a frozen-state wave, act in place
    const double *m;
    // batches of independent graphs: graph of each vertex, m of each graph,
    // per-graph summed gains (null for a single graph)
    const uint32_t *gid;
    const double *m_g;
    const double *minv_g;  // 1/m of each graph
    double *dq_g;
    int lsb;  // K in exact integer units of 2^lsb (INT_MIN: float64 deltas)
    MoveCounters *ctr;
    int rule;
    // no-return rule: from iteration no_return_from on (0: never) a vertex
    // does not move back to the community it left in the previous iteration
    uint32_t *left;   // community each vertex last left
    int *left_it;     // iteration of that move (-2: none in this pass)
    const int *iteration;  // device scalar: the sweep's iteration (set before each launch or graph replay)
    int no_return_from;
    uint32_t *mv_vtx, *mv_cmt, *mv_cnt;  // frozen-state move list
    uint32_t *choice;                    // optional per-vertex decision
    // last-visit features for the learned predictor (optional)
    float *feat_kept, *feat_gain, *last_gain;
    uint8_t *moved_last;
    uint8_t *deferred;  // learned pruning: vertices the predictor put off (cleared when visited)
    // trace rows (optional): features before the visit, label = moved
    float *trace_x;
    uint8_t *trace_y;
    uint32_t *trace_cnt;
    uint64_t *trace_keys;  // optional: trace_tag | iteration << 48 | vertex per row
    uint64_t trace_tag;    // pass << 56 | repeat << 40
    uint32_t trace_cap, trace_every;
    float max_logk;
    int max_iterations;  // the iteration's position in the pass (a feature) is *iteration / max_iterations
    uint32_t salt;       // trace sampling: per pass; the iteration is mixed in on the device
};

template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
__device__ __forceinline__ uint8_t ldcg(const uint8_t *p) {
    return (uint8_t)__ldcg(reinterpret_cast<const unsigned char *>(p));
}
// SYNC: 0 = in-place updates (the paper's loop), 1 = frozen-state wave in its
// own launch, 2 = frozen-state wave inside the persistent sweep kernel.  A
// frozen-state wave reads data that no thread writes during the wave; in its
// own launch that data is read-only for the whole launch (read-only cache
// path), inside the persistent kernel earlier phases of the same launch wrote
// it, so the loads go to L2 (the per-SM L1 is not coherent).
template <int SYNC, typename T> __device__ __forceinline__ T ld_state(const T *p) {
    if constexpr (SYNC == 1) return __ldg(p);
    else return ldcg(p);
}

template <typename V, typename WT> __device__ __forceinline__ V load_w(const WT *w, uint64_t e) {
    return (V)__ldg(w + e);
}

// Scan the edges [b, e) of vertex i with stride `step` starting at b + lane:
// the self-loop is skipped, K_{i->d} accumulates in kid, other communities
// go to ins(c, w).  U edges per thread per round, their loads issued before
// their use, so that U gathers of C[j] are in flight at once.
template <int U, int SYNC, typename V, typename WT, typename F>
__device__ __forceinline__ void scan_edges(const uint32_t *__restrict__ tgt, const WT *__restrict__ w,
                                           const uint32_t *C, uint32_t i, uint32_t d, uint64_t b, uint64_t e,
                                           uint32_t lane, uint32_t step, V &kid, F &&ins) {
    for (uint64_t p0 = b + lane; p0 < e; p0 += (uint64_t)U * step) {
        uint32_t j[U];
        V wv[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            uint64_t p = p0 + (uint64_t)u * step;
            bool ok = p < e;
            j[u] = ok ? __ldg(tgt + p) : i;
            wv[u] = ok ? (V)__ldg(w + p) : V(0);
        }
        uint32_t c[U];
#pragma unroll
        for (int u = 0; u < U; u++) c[u] = (j[u] != i) ? ld_state<SYNC>(C + j[u]) : EMPTY;
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (c[u] == EMPTY) continue;
            if (c[u] == d) kid += wv[u];
            else ins(c[u], wv[u]);
        }
    }
}

template <typename S> __device__ __forceinline__ bool better(S s1, uint32_t c1, S s2, uint32_t c2) {
    return s1 > s2 || (s1 == s2 && c1 < c2);
}

// Score the entries of a table: slots s = lane, lane + step, ... < cap (or
// the listed slots occ[...] when occ is given).  U entries per round, with
// the gathers of Sigma_c issued together.
template <int U, int SYNC, typename SC, typename S, typename V>
__device__ __forceinline__ void score_table(const uint32_t *keys, const V *vals, const uint16_t *occ, uint32_t cap,
                                            uint32_t lane, uint32_t step, const double *Sig, const SC &sc, S &best,
                                            uint32_t &bestc, uint32_t &ncand) {
    for (uint32_t s0 = lane; s0 < cap; s0 += U * step) {
        uint32_t c[U];
        V v[U];
        double sg[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            uint32_t s = s0 + u * step;
            uint32_t slot = s < cap ? (occ ? (uint32_t)occ[s] : s) : 0;
            c[u] = s < cap ? keys[slot] : EMPTY;
            v[u] = s < cap ? vals[slot] : V(0);
        }
#pragma unroll
        for (int u = 0; u < U; u++) sg[u] = c[u] != EMPTY ? ld_state<SYNC>(Sig + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (c[u] == EMPTY) continue;
            ncand++;
            S val = sc.score(v[u], sg[u]);
            if (better(val, c[u], best, bestc)) { best = val; bestc = c[u]; }
        }
    }
}

// Equation 2, evaluated in the order written, with no contraction.
__device__ __forceinline__ double eq2(double Kic, double Kid, double Ki, double Sc, double Sd, double m) {
    double t1 = __ddiv_rn(__dsub_rn(Kic, Kid), m);
    double t2 = __dmul_rn(Ki, __dsub_rn(__dadd_rn(Ki, Sc), Sd));
    double den = __dmul_rn(__dmul_rn(2.0, m), m);
    return __dsub_rn(t1, __ddiv_rn(t2, den));
}

// Per-vertex scoring context.
template <bool F64> struct Score;
template <> struct Score<true> {
    using S = double;
    double Ki, Kid, Sd, m;
    __device__ S score(double kic, double Sc) const { return eq2(kic, Kid, Ki, Sc, Sd, m); }
    __device__ double gain(S best) const { return best; }  // in units of Q
};
// Float64 is a narrow pipe on this GPU: the mixed-precision scores take 1/m
// precomputed (0.5/m is 0.5 * RN(1/m) exactly, so K_i/2m is unchanged) and
// the gain of the chosen community is a product, not a division.
template <> struct Score<false> {
    using S = float;
    float kif, sd;
    double inv_m;
    __device__ S score(float kic, double Sc) const { return kic - kif * (float)Sc; }
    __device__ double gain(S best) const { return (double)(best - sd) * inv_m; }
};

// m and inv_m = 1/m of the vertex's graph (the float64 score uses m only).
template <bool F64>
__device__ __forceinline__ Score<F64> make_score(double Ki, double kid, double Sd, double m, double inv_m);
template <>
__device__ __forceinline__ Score<true> make_score<true>(double Ki, double kid, double Sd, double m, double) {
    Score<true> s;
    s.Ki = Ki; s.Kid = kid; s.Sd = Sd; s.m = m;
    return s;
}
template <>
__device__ __forceinline__ Score<false> make_score<false>(double Ki, double kid, double Sd, double, double inv_m) {
    Score<false> s;
    const double inv2m = 0.5 * inv_m;
    s.kif = (float)(Ki * inv2m);
    s.sd = (float)kid - s.kif * (float)(Sd - Ki);
    s.inv_m = inv_m;
    return s;
}

// m of vertex i's graph (batches) or of the single graph.
__device__ __forceinline__ double vertex_m(const MoveArgs &a, uint32_t i, double m0) {
    return a.gid ? a.m_g[a.gid[i]] : m0;
}
__device__ __forceinline__ double vertex_inv_m(const MoveArgs &a, uint32_t i, double inv0) {
    return a.gid ? a.minv_g[a.gid[i]] : inv0;
}
__device__ __forceinline__ void add_graph_gain(const MoveArgs &a, uint32_t i, double gain) {
    if (a.dq_g) atomicAdd(a.dq_g + a.gid[i], gain);
}

// Decide the move of i toward c (one thread).  Frozen-state: record it in the
// move list; in place: apply it now.  Returns whether i moves.
template <int SYNC>
__device__ __forceinline__ bool decide_move(const MoveArgs &a, uint32_t i, uint32_t d, uint32_t c, double Ki) {
    if (c == EMPTY || c == d) return false;
    if (a.rule) {
        uint32_t sd = ld_state<SYNC>(a.size + d), sc = ld_state<SYNC>(a.size + c);
        if (sd == 1 && sc == 1 && c > d) return false;
    }
    if (a.no_return_from > 0 && a.left[i] == c) {
        const int it = *a.iteration;
        if (it >= a.no_return_from && a.left_it[i] == it - 1) return false;
    }
    if (a.choice) a.choice[i] = c;
    if constexpr (SYNC) {
        uint32_t slot = atomicAdd(a.mv_cnt, 1u);
        a.mv_vtx[slot] = i;
        a.mv_cmt[slot] = c;
    } else {
        a.left[i] = d;
        a.left_it[i] = *a.iteration;
        a.C[i] = c;
        atomicAdd(a.Sig + d, -Ki);
        atomicAdd(a.Sig + c, Ki);
        atomicSub(a.size + d, 1u);
        atomicAdd(a.size + c, 1u);
    }
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
        if (dq != 0.0) atomicAdd(&g->dq, dq);
        if (mv) atomicAdd(&g->moved, mv);
        if (vx) atomicAdd(&g->vertices, vx);
        if (ed) atomicAdd(&g->edges, ed);
        if (ca) atomicAdd(&g->candidates, ca);
        if (mk) atomicAdd(&g->marked, mk);
    }
}

__device__ __forceinline__ void vertex_features(const MoveArgs &a, uint32_t i, uint32_t deg, double Ki, float *x) {
    const float iter_frac = a.max_iterations > 0 ? (float)*a.iteration / (float)a.max_iterations : 0.0f;
    predictor_features(deg, Ki, a.feat_kept[i], a.feat_gain[i], a.moved_last[i], a.max_logk, iter_frac, x);
}

// After a visit: record last-visit features and, for sampled visits, a trace
// row (features before the visit, label = moved).
__device__ __forceinline__ void record_visit(const MoveArgs &a, uint32_t i, uint32_t deg, double Ki, double kid,
                                             double gain, double m, int moved) {
    if (!a.feat_kept) return;
    if (a.trace_x && (hash32(i ^ ((uint32_t)*a.iteration * 0x9E3779B9u + a.salt)) % a.trace_every) == 0) {
        float x[MLP_IN];
        vertex_features(a, i, deg, Ki, x);
        uint32_t slot = atomicAdd(a.trace_cnt, 1u);
        if (slot < a.trace_cap) {
#pragma unroll
            for (int k = 0; k < MLP_IN; k++) a.trace_x[(size_t)slot * MLP_IN + k] = x[k];
            a.trace_y[slot] = (uint8_t)moved;
            if (a.trace_keys) a.trace_keys[slot] = a.trace_tag | ((uint64_t)(*a.iteration & 0xFF) << 48) | i;
        }
    }
    float kept = Ki > 0.0 ? (float)(kid / Ki) : 0.0f;
    float g = Ki > 0.0 ? (float)(gain * m / Ki) : 0.0f;
    a.feat_kept[i] = kept;
    a.feat_gain[i] = fminf(fmaxf(g, -1.0f), 1.0f);
    if (a.last_gain) a.last_gain[i] = (float)gain;
    a.moved_last[i] = (uint8_t)moved;
}

// --------------------------------------------------------------------------
// Groups of G lanes, one vertex per group, table of up to CAP slots per group
// (slots carved out of the block's shared buffer).
// --------------------------------------------------------------------------
template <int G, int CAP, typename WT, bool F64, int SYNC>
__device__ void group_body(const MoveArgs &a, const uint32_t *__restrict__ list, uint32_t count, uint32_t lb,
                           uint32_t nb, unsigned char *smem, LocalCtr &lc) {
    using V = typename std::conditional<F64, double, float>::type;
    using SC = Score<F64>;
    using S = typename SC::S;
    constexpr int NG = 256 / G;
    const int lane = threadIdx.x % G;
    const int grp = threadIdx.x / G;
    const int leader = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << leader);
    uint32_t *keys = reinterpret_cast<uint32_t *>(smem) + grp * CAP;
    V *vals = reinterpret_cast<V *>(smem + (size_t)NG * CAP * sizeof(uint32_t)) + grp * CAP;
    const WT *w = static_cast<const WT *>(a.w);
    const double m0 = *a.m;
    const double inv0 = 1.0 / m0;
    // counters accumulate in the caller's lc
    // The warp's list entries are wbase, wbase + wstep, ...; 32 of them are
    // claimed at once (each lane reads one flag and marks its vertex
    // processed), and the active ones are dealt to the warp's groups round
    // by round, so that the inactive vertices of later sweeps cost one
    // parallel round of loads per 32 entries and the groups of a warp stay
    // in step.
    constexpr int NGW = 32 / G;  // groups per warp
    const int wl = threadIdx.x & 31, gw = wl / G;
    const uint32_t wbase = lb * 8 + (threadIdx.x >> 5), wstep = nb * 8;
    for (uint64_t kb = 0; wbase + kb * wstep < count; kb += 32) {
        const uint64_t my = wbase + (kb + wl) * wstep;
        uint32_t vi = 0;
        int claim = 0;
        if (my < count) {
            vi = list[my];
            claim = ld_state<SYNC>(a.act + vi);
            if (claim) {
                a.act[vi] = 0;
                if (a.deferred) a.deferred[vi] = 0;
            }
        }
        const unsigned amask = __ballot_sync(0xFFFFFFFFu, claim);
        const int nact = __popc(amask);
        for (int r0 = 0; r0 < nact; r0 += NGW) {
        const int q = r0 + gw;  // this group's active entry in the round
        const uint32_t i = __shfl_sync(0xFFFFFFFFu, vi, q < nact ? select_bit(amask, q) : 0);
        if (q >= nact) continue;
        uint32_t d = ld_state<SYNC>(a.C + i);
        uint64_t b = a.off[i], e = a.off[i + 1];
        uint32_t deg = (uint32_t)(e - b);
        int logcap = ceil_log2(2 * deg);
        if (logcap < 1) logcap = 1;
        uint32_t cap = 1u << logcap;
        for (uint32_t s = lane; s < cap; s += G) { keys[s] = EMPTY; vals[s] = V(0); }
        __syncwarp(gmask);
        V kid = 0;
        scan_edges<(CAP >= 1024 ? 4 : 2), SYNC, V>(a.tgt, w, a.C, i, d, b, e, lane, G, kid,
                                                    [&](uint32_t c, V wv) { ht_add<V>(keys, vals, logcap, c, wv); });
        __syncwarp(gmask);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) kid += __shfl_xor_sync(gmask, kid, o);
        double Ki = a.K[i];
        double Sd = ld_state<SYNC>(a.Sig + d);
        Sd = __shfl_sync(gmask, Sd, leader);
        const double m = vertex_m(a, i, m0);
        SC sc = make_score<F64>(Ki, (double)kid, Sd, m, vertex_inv_m(a, i, inv0));
        S best = -INFINITY;
        uint32_t bestc = EMPTY;
        uint32_t ncand = 0;
        score_table<(CAP >= 1024 ? 4 : 2), SYNC>(keys, vals, (const uint16_t *)nullptr, cap, lane, G, a.Sig, sc, best,
                                                  bestc, ncand);
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
            if (gain > 0.0) mv = decide_move<SYNC>(a, i, d, bestc, Ki);
            if (mv) { lc.moved++; lc.dq += gain; add_graph_gain(a, i, gain); }
            record_visit(a, i, deg, Ki, (double)kid, gain, m, mv);
        }
        // movers re-mark their neighbours (frozen-state waves write a separate
        // array merged after the wave, so that the wave never sees its marks)
        mv = __shfl_sync(gmask, mv, leader);
        if (mv) {
            if (lane == 0) lc.marked += deg;
            for (uint64_t p = b + lane; p < e; p += G) {
                uint32_t j = __ldg(a.tgt + p);
                if (j != i) a.mark[j] = 1;
            }
        }
        __syncwarp(gmask);
        }
    }
    __syncthreads();  // the block's tables are free for the next body
}

struct GroupLists {
    const uint32_t *list[4];
    uint32_t count[4];
    uint32_t bstart[5];  // block ranges of the four classes
};

constexpr size_t GROUP_SMEM_F64 = 2048 * (sizeof(uint32_t) + sizeof(double));
constexpr size_t GROUP_SMEM_F32 = 2048 * (sizeof(uint32_t) + sizeof(float));

template <typename WT, bool F64, int SYNC>
__global__ void __launch_bounds__(256) k_move_groups(MoveArgs a, GroupLists gl) {
    __shared__ __align__(16) unsigned char smem[F64 ? GROUP_SMEM_F64 : GROUP_SMEM_F32];
    uint32_t b = blockIdx.x;
    LocalCtr lc;
    if (b < gl.bstart[1])
        group_body<4, 16, WT, F64, SYNC>(a, gl.list[0], gl.count[0], b, gl.bstart[1], smem, lc);
    else if (b < gl.bstart[2])
        group_body<8, 32, WT, F64, SYNC>(a, gl.list[1], gl.count[1], b - gl.bstart[1], gl.bstart[2] - gl.bstart[1],
                                         smem, lc);
    else if (b < gl.bstart[3])
        group_body<16, 64, WT, F64, SYNC>(a, gl.list[2], gl.count[2], b - gl.bstart[2],
                                          gl.bstart[3] - gl.bstart[2], smem, lc);
    else
        group_body<32, 256, WT, F64, SYNC>(a, gl.list[3], gl.count[3], b - gl.bstart[3],
                                           gl.bstart[4] - gl.bstart[3], smem, lc);
    flush_counters(lc, a.ctr);
}

// Degrees 129..512: one warp per vertex, 1024-slot table per warp.
constexpr int W512_CAP = 1024;
template <typename WT, bool F64, int SYNC>
__global__ void __launch_bounds__(256) k_move_w512(MoveArgs a, const uint32_t *__restrict__ list, uint32_t count) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    LocalCtr lc;
    group_body<32, W512_CAP, WT, F64, SYNC>(a, list, count, blockIdx.x, gridDim.x, dyn_smem, lc);
    flush_counters(lc, a.ctr);
}

// --------------------------------------------------------------------------
// One block per vertex; table in shared memory (CAP > 0) or in the global
// pool (CAP == 0, slots at pool_off[idx]).
// --------------------------------------------------------------------------
template <int CAP, typename WT, bool F64, int SYNC>
__device__ void block_body(const MoveArgs &a, const uint32_t *__restrict__ list, uint32_t count, uint32_t lb,
                           uint32_t nb, unsigned char *dyn_smem, LocalCtr &lc) {
    using V = typename std::conditional<F64, double, float>::type;
    using SC = Score<F64>;
    using S = typename SC::S;
    // table: keys, values and the list of occupied slots (scoring and
    // clearing touch only those)
    uint32_t *keys = reinterpret_cast<uint32_t *>(dyn_smem);
    V *vals = reinterpret_cast<V *>(dyn_smem + (size_t)CAP * sizeof(uint32_t));
    uint16_t *occ = reinterpret_cast<uint16_t *>(dyn_smem + (size_t)CAP * (sizeof(uint32_t) + sizeof(V)));
    __shared__ S red_s[32];
    __shared__ uint32_t red_c[32];
    __shared__ V red_k[32];
    __shared__ int s_mv;
    __shared__ uint32_t s_d, s_nocc;
    __shared__ double s_Sd;
    const WT *w = static_cast<const WT *>(a.w);
    const double m0 = *a.m;
    const double inv0 = 1.0 / m0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    // counters accumulate in the caller's lc
    __shared__ uint32_t s_todo[256], s_ntodo, s_wcnt[8];
    for (uint32_t s = threadIdx.x; s < CAP; s += blockDim.x) { keys[s] = EMPTY; vals[s] = V(0); }
    // The block's entries are lb + k * nb; blockDim.x of them are claimed at
    // once (one flag per thread) and the active ones listed in shared memory,
    // so inactive vertices cost no serial round trip.
    for (uint64_t kb = 0; lb + kb * nb < count; kb += blockDim.x) {
        const uint64_t my = lb + (kb + threadIdx.x) * nb;
        uint32_t vi = 0;
        int claim = 0;
        if (my < count) {
            vi = list[my];
            claim = ld_state<SYNC>(a.act + vi);
            if (claim) {
                a.act[vi] = 0;
                if (a.deferred) a.deferred[vi] = 0;
            }
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, claim);
        __syncthreads();  // the loop's previous step is done with s_todo
        if (lane == 0) s_wcnt[wid] = __popc(bal);
        __syncthreads();
        if (claim) {
            uint32_t pos = __popc(bal & ((1u << lane) - 1u));
            for (int k = 0; k < wid; k++) pos += s_wcnt[k];
            s_todo[pos] = vi;
        }
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int k = 0; k < nw; k++) t += s_wcnt[k];
            s_ntodo = t;
        }
        __syncthreads();
        const uint32_t ntodo = s_ntodo;
    for (uint32_t kk = 0; kk < ntodo; kk++) {
        const uint32_t i = s_todo[kk];
        __syncthreads();  // previous vertex done with the table and reductions
        if (threadIdx.x == 0) {
            s_nocc = 0;
            s_d = ld_state<SYNC>(a.C + i);
            s_Sd = ld_state<SYNC>(a.Sig + s_d);
        }
        __syncthreads();
        uint32_t d = s_d;
        uint64_t b = a.off[i], e = a.off[i + 1];
        uint32_t deg = (uint32_t)(e - b);
        int logcap = ceil_log2(2 * deg);
        V kid = 0;
        constexpr int U = CAP >= 16384 ? 8 : 4;  // hubs: more gathers in flight per thread
        scan_edges<U, SYNC, V>(a.tgt, w, a.C, i, d, b, e, threadIdx.x, blockDim.x, kid,
                               [&](uint32_t c, V wv) { smem_add<V>(keys, vals, logcap, occ, &s_nocc, c, wv); });
        kid = warp_sum(kid);
        if (lane == 0) red_k[wid] = kid;
        __syncthreads();
        kid = 0;
        for (int t = 0; t < nw; t++) kid += red_k[t];
        double Ki = a.K[i];
        const double m = vertex_m(a, i, m0);
        SC sc = make_score<F64>(Ki, (double)kid, s_Sd, m, vertex_inv_m(a, i, inv0));
        S best = -INFINITY;
        uint32_t bestc = EMPTY;
        uint32_t nocc = s_nocc;
        uint32_t ncand = 0;
        score_table<U, SYNC>(keys, vals, occ, nocc, threadIdx.x, blockDim.x, a.Sig, sc, best, bestc, ncand);
        __syncthreads();  // every slot scored before the table is emptied
        for (uint32_t k = threadIdx.x; k < nocc; k += blockDim.x) {
            uint32_t slot = occ[k];
            keys[slot] = EMPTY;  // leave the table empty for the next vertex
            vals[slot] = V(0);
        }
        if (threadIdx.x == 0) lc.candidates += nocc;
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
            if (gain > 0.0) mv = decide_move<SYNC>(a, i, d, bestc, Ki);
            lc.vertices++;
            lc.edges += deg;
            if (mv) { lc.moved++; lc.dq += gain; add_graph_gain(a, i, gain); }
            record_visit(a, i, deg, Ki, (double)kid, gain, m, mv);
            s_mv = mv;
        }
        __syncthreads();
        if (s_mv) {
            if (threadIdx.x == 0) lc.marked += deg;
            for (uint64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
                uint32_t j = __ldg(a.tgt + p);
                if (j != i) a.mark[j] = 1;
            }
        }
    }
    }
    __syncthreads();
    __syncthreads();  // the block's table is free for the next body
}

template <int CAP, typename WT, bool F64, int SYNC>
__global__ void __launch_bounds__(256) k_move_block(MoveArgs a, const uint32_t *__restrict__ list, uint32_t count) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    LocalCtr lc;
    block_body<CAP, WT, F64, SYNC>(a, list, count, blockIdx.x, gridDim.x, dyn_smem, lc);
    flush_counters(lc, a.ctr);
}

// --------------------------------------------------------------------------
// Apply a frozen-state wave's moves: C, Sigma and size updates (float64
// atomics of exactly representable values, so the result does not depend on
// their order).  The movers' neighbours were already re-marked, into the
// separate mark array, by the kernels that decided the moves (hub movers by
// k_mark_big).
// --------------------------------------------------------------------------

// Community totals change by +-K_i per move; movers of a wave crowd into a
// few large communities, so the deltas are first summed per block in a
// shared table (float64 sums of exactly representable values, exact in any
// order) and then applied with one atomic per community per block.
constexpr int APPLY_SLOG = 11;

// The block's delta of Sigma_c is summed either in float64 or, when K is in
// exact integer units of 2^lsb (lsb != INT_MIN), as a signed 64-bit integer
// (two's complement in an unsigned atomic add: one native shared-memory
// operation, where a float64 add loops on compare-and-swap under contention).
// Both sums are exact, so Sigma ends up the same.
__device__ __forceinline__ double signed_units_val(unsigned long long u, int lsb) {
    const long long v = (long long)u;
    return v < 0 ? -Acc<unsigned long long>::val((unsigned long long)(-v), lsb)
                 : Acc<unsigned long long>::val((unsigned long long)v, lsb);
}

__device__ __forceinline__ void apply_delta(uint32_t *keys, double *ds, int *dn, uint32_t c, double k, int n,
                                            double *Sig, uint32_t *size, int lsb) {
    uint32_t mask = (1u << APPLY_SLOG) - 1u;
    uint32_t h = hash32(c) >> (32 - APPLY_SLOG);
    for (uint32_t probe = 0; probe < 64; probe++) {
        uint32_t old = atomicCAS(&keys[h], EMPTY, c);
        if (old == EMPTY || old == c) {
            if (lsb != INT_MIN) {
                const unsigned long long u = units_of(k < 0.0 ? -k : k, lsb);
                atomicAdd(reinterpret_cast<unsigned long long *>(ds) + h, k < 0.0 ? 0ull - u : u);
            } else {
                atomicAdd(&ds[h], k);
            }
            atomicAdd(&dn[h], n);
            return;
        }
        h = (h + 1) & mask;
    }
    atomicAdd(Sig + c, k);  // crowded table: apply directly
    atomicAdd(size + c, (uint32_t)n);
}

// Flush a block's delta table (slot t) into Sigma and size.
__device__ __forceinline__ void flush_delta(const uint32_t *keys, const double *ds, const int *dn, int t, double *Sig,
                                            uint32_t *size, int lsb) {
    const uint32_t c = keys[t];
    if (c == EMPTY) return;
    if (lsb != INT_MIN) {
        const unsigned long long u = reinterpret_cast<const unsigned long long *>(ds)[t];
        if (u) atomicAdd(Sig + c, signed_units_val(u, lsb));
    } else if (ds[t] != 0.0) {
        atomicAdd(Sig + c, ds[t]);
    }
    if (dn[t] != 0) atomicAdd(size + c, (uint32_t)dn[t]);
}

__global__ void __launch_bounds__(256) k_apply_moves(const uint32_t *__restrict__ mv_vtx,
                                                     const uint32_t *__restrict__ mv_cmt,
                                                     const uint32_t *__restrict__ mv_cnt, const double *__restrict__ K,
                                                     uint32_t *C, double *Sig, uint32_t *size, int lsb, uint32_t *left,
                                                     int *left_it, const int *iteration_dev) {
    __shared__ uint32_t skeys[1 << APPLY_SLOG];
    __shared__ double sds[1 << APPLY_SLOG];
    __shared__ int sdn[1 << APPLY_SLOG];
    for (int t = threadIdx.x; t < (1 << APPLY_SLOG); t += blockDim.x) { skeys[t] = EMPTY; sds[t] = 0.0; sdn[t] = 0; }
    __syncthreads();
    uint32_t cnt = *mv_cnt;
    const int iteration = *iteration_dev;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        uint32_t i = mv_vtx[t], c = mv_cmt[t];
        uint32_t d = C[i];
        double Ki = K[i];
        C[i] = c;
        left[i] = d;
        left_it[i] = iteration;
        apply_delta(skeys, sds, sdn, d, -Ki, -1, Sig, size, lsb);
        apply_delta(skeys, sds, sdn, c, Ki, 1, Sig, size, lsb);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < (1 << APPLY_SLOG); t += blockDim.x) flush_delta(skeys, sds, sdn, t, Sig, size, lsb);
}

// act |= mark, mark = 0 (16 bytes per thread step).
__global__ void k_merge_marks(uint8_t *act, uint8_t *mark, uint32_t n) {
    uint32_t n16 = n / 16;
    uint4 *a4 = reinterpret_cast<uint4 *>(act);
    uint4 *m4 = reinterpret_cast<uint4 *>(mark);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n16; t += gridDim.x * blockDim.x) {
        uint4 mk = m4[t];
        if (mk.x | mk.y | mk.z | mk.w) {
            uint4 ac = a4[t];
            ac.x |= mk.x; ac.y |= mk.y; ac.z |= mk.z; ac.w |= mk.w;
            a4[t] = ac;
            m4[t] = make_uint4(0, 0, 0, 0);
        }
    }
    for (uint32_t v = n16 * 16 + blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (mark[v]) { act[v] = 1; mark[v] = 0; }
    }
}

// Re-mark the neighbours of the big movers: block column x takes movers
// x, x + gridDim.x, ...; the gridDim.y blocks of a column split each mover's
// edges into interleaved slices.
__global__ void k_mark_big(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tgt,
                           const uint32_t *__restrict__ big, const uint32_t *__restrict__ nbig, uint8_t *act) {
    uint32_t cnt = *nbig;
    uint64_t step = (uint64_t)gridDim.y * blockDim.x;
    for (uint32_t t = blockIdx.x; t < cnt; t += gridDim.x) {
        uint32_t i = big[t];
        uint64_t b = off[i], e = off[i + 1];
        for (uint64_t p = b + (uint64_t)blockIdx.y * blockDim.x + threadIdx.x; p < e; p += step) {
            uint32_t j = tgt[p];
            if (j != i) act[j] = 1;
        }
    }
}

// --------------------------------------------------------------------------
// Persistent sweep: for graphs with no hub (every degree <= 2048) and at most
// a million or so vertices, a sweep of W waves costs 4-6 launches per wave on
// the normal path, and on small graphs those dependent launches, not the
// work, set the time.  Here one cooperative launch runs the whole sweep: per
// run of a wave, every block takes its share of each degree class (the same device
// bodies as the per-class kernels, frozen-state decisions into the wave's
// move list), a grid barrier, the moves applied and the re-marks merged,
// and a grid barrier.  Data written by earlier phases are read through L2
// (SYNC mode 2).  The barrier spins a bounded number of times: a block that
// gives up flags the sweep (MoveCounters::stalled) and the kernel returns.
// --------------------------------------------------------------------------
constexpr unsigned long long GRID_SYNC_SPINS = 1ull << 22;  // x 64 ns sleeps: about 0.3 s

__device__ bool grid_sync(GridBar *b, unsigned nb, MoveCounters *ctr) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ok = 1;
        volatile unsigned *vgen = &b->gen;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(&b->arrive, 1u) == nb - 1) {
            b->arrive = 0;
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == g) {
                if (++spins > GRID_SYNC_SPINS || *(volatile unsigned *)&b->err) {
                    atomicExch(&b->err, 1u);
                    atomicAdd(&ctr->stalled, 1ull);
                    ok = 0;
                    break;
                }
                if (spins > 256) __nanosleep(32);  // poll tightly first: most waits are short
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Moves of a wave applied as k_apply_moves does, reading the move list, C
// and the count through L2; `smem` holds the block's delta table.
__device__ void apply_body_l2(const uint32_t *mv_vtx, const uint32_t *mv_cmt, const uint32_t *mv_cnt,
                              const double *__restrict__ K, uint32_t *C, double *Sig, uint32_t *size, uint32_t lb,
                              uint32_t nb, unsigned char *smem, int lsb, uint32_t *left, int *left_it, int iteration) {
    uint32_t *skeys = reinterpret_cast<uint32_t *>(smem);
    double *sds = reinterpret_cast<double *>(smem + sizeof(uint32_t) * (1u << APPLY_SLOG));
    int *sdn = reinterpret_cast<int *>(smem + (sizeof(uint32_t) + sizeof(double)) * (1u << APPLY_SLOG));
    for (int t = threadIdx.x; t < (1 << APPLY_SLOG); t += blockDim.x) { skeys[t] = EMPTY; sds[t] = 0.0; sdn[t] = 0; }
    __syncthreads();
    const uint32_t cnt = __ldcg(mv_cnt);
    for (uint32_t t = lb * blockDim.x + threadIdx.x; t < cnt; t += nb * blockDim.x) {
        const uint32_t i = __ldcg(mv_vtx + t), c = __ldcg(mv_cmt + t);
        const uint32_t d = __ldcg(C + i);
        const double Ki = K[i];
        C[i] = c;
        left[i] = d;
        left_it[i] = iteration;
        apply_delta(skeys, sds, sdn, d, -Ki, -1, Sig, size, lsb);
        apply_delta(skeys, sds, sdn, c, Ki, 1, Sig, size, lsb);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < (1 << APPLY_SLOG); t += blockDim.x) flush_delta(skeys, sds, sdn, t, Sig, size, lsb);
    __syncthreads();
}

__device__ void merge_body_l2(uint8_t *act, uint8_t *mark, uint32_t n, uint32_t lb, uint32_t nb) {
    const uint32_t n16 = n / 16;
    uint4 *a4 = reinterpret_cast<uint4 *>(act);
    uint4 *m4 = reinterpret_cast<uint4 *>(mark);
    for (uint32_t t = lb * blockDim.x + threadIdx.x; t < n16; t += nb * blockDim.x) {
        const uint4 mk = __ldcg(m4 + t);
        if (mk.x | mk.y | mk.z | mk.w) {
            uint4 ac = __ldcg(a4 + t);
            ac.x |= mk.x; ac.y |= mk.y; ac.z |= mk.z; ac.w |= mk.w;
            a4[t] = ac;
            m4[t] = make_uint4(0, 0, 0, 0);
        }
    }
    for (uint32_t v = n16 * 16 + lb * blockDim.x + threadIdx.x; v < n; v += nb * blockDim.x) {
        if (ldcg(mark + v)) { act[v] = 1; mark[v] = 0; }
    }
}

template <typename WT, bool F64>
__global__ void __launch_bounds__(256) k_sweep_persistent(MoveArgs a, const uint32_t *__restrict__ list,
                                                          const uint32_t *__restrict__ start, int W, int R,
                                                          uint32_t n, uint32_t *mv_cnts, GridBar *bar) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const uint32_t lb = blockIdx.x, nb = gridDim.x;
    LocalCtr lc;  // one flush per block per sweep
    if (lb == 0)
        for (int t = threadIdx.x; t < W * R; t += blockDim.x) mv_cnts[t] = 0;
    if (!grid_sync(bar, nb, a.ctr)) return;
    for (int wr = 0; wr < W * R; wr++) {  // wave wr / R, repeat wr % R
        const int wv = wr / R;
        uint32_t cb[CLS_HUGE], cc[CLS_HUGE], tot = 0;
#pragma unroll
        for (int k = 0; k < CLS_HUGE; k++) {
            cb[k] = start[k * W + wv];
            cc[k] = start[k * W + wv + 1] - cb[k];
            tot += cc[k];
        }
        if (!tot) continue;  // the same for every block
        MoveArgs aw = a;
        aw.mv_cnt = mv_cnts + wr;
        if (cc[CLS_G4]) group_body<4, 16, WT, F64, 2>(aw, list + cb[CLS_G4], cc[CLS_G4], lb, nb, dyn_smem, lc);
        if (cc[CLS_G8]) group_body<8, 32, WT, F64, 2>(aw, list + cb[CLS_G8], cc[CLS_G8], lb, nb, dyn_smem, lc);
        if (cc[CLS_G16]) group_body<16, 64, WT, F64, 2>(aw, list + cb[CLS_G16], cc[CLS_G16], lb, nb, dyn_smem, lc);
        if (cc[CLS_G32]) group_body<32, 256, WT, F64, 2>(aw, list + cb[CLS_G32], cc[CLS_G32], lb, nb, dyn_smem, lc);
        if (cc[CLS_W512])
            group_body<32, W512_CAP, WT, F64, 2>(aw, list + cb[CLS_W512], cc[CLS_W512], lb, nb, dyn_smem, lc);
        if (cc[CLS_BLOCK])
            block_body<4096, WT, F64, 2>(aw, list + cb[CLS_BLOCK], cc[CLS_BLOCK], lb, nb, dyn_smem, lc);
        if (!grid_sync(bar, nb, a.ctr)) return;
        apply_body_l2(a.mv_vtx, a.mv_cmt, mv_cnts + wr, a.K, a.C, a.Sig, a.size, lb, nb, dyn_smem, a.lsb, a.left,
                      a.left_it, *a.iteration);
        merge_body_l2(a.act, a.mark, n, lb, nb);
        if (!grid_sync(bar, nb, a.ctr)) return;
    }
    flush_counters(lc, a.ctr);
}

// --------------------------------------------------------------------------
// Hub vertices (degree > 2048), processed by the whole grid:
//   prepare: read and clear each hub's flag, snapshot its community;
//   insert:  the hub's edges are cut into HUB_CHUNK-edge tasks; a block
//            combines a task's communities in a shared-memory table, then
//            publishes the distinct ones to the hub's global table (new keys
//            append their slot to the hub's occupied list);
//   score:   all threads stride over the occupied list (and reset the slots
//            for the next sweep); per-block best per hub;
//   decide:  one warp per hub reduces the block bests and decides the move.
// --------------------------------------------------------------------------
constexpr int HUB_SLOG = 11;  // shared table of 2 * HUB_CHUNK slots

struct HubArgs {
    const uint32_t *hubs;
    uint32_t nh;
    const uint64_t *pool_off;  // per hub
    const uint64_t *tasks;     // per hub: prefix of chunk counts (nh + 1 entries, tasks[0] = base)
    uint32_t *keys;
    void *vals;
    uint32_t *occ;
    uint32_t *occ_n;    // per hub
    void *kid;          // per hub, V
    uint8_t *go;        // per hub
    uint32_t *d;        // per hub
    void *best_s;       // per task, S
    uint32_t *best_c;   // per task
    uint32_t *big, *nbig;
};

template <int SYNC>
__global__ void k_hub_prepare(MoveArgs a, HubArgs h) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < h.nh; t += gridDim.x * blockDim.x) {
        uint32_t i = h.hubs[t];
        uint8_t go = ld_state<SYNC>(a.act + i);
        if (go) {
            a.act[i] = 0;
            if (a.deferred) a.deferred[i] = 0;
        }
        h.go[t] = go;
        h.d[t] = ld_state<SYNC>(a.C + i);
    }
}

template <typename WT, bool F64, int SYNC>
__global__ void __launch_bounds__(256) k_hub_insert(MoveArgs a, HubArgs h) {
    using V = typename std::conditional<F64, double, float>::type;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    uint32_t *skeys = reinterpret_cast<uint32_t *>(dyn_smem);
    V *svals = reinterpret_cast<V *>(dyn_smem + sizeof(uint32_t) * (1u << HUB_SLOG));
    uint16_t *socc = reinterpret_cast<uint16_t *>(dyn_smem + (sizeof(uint32_t) + sizeof(V)) * (1u << HUB_SLOG));
    __shared__ V red[32];
    __shared__ uint32_t s_nocc;
    const WT *w = static_cast<const WT *>(a.w);
    V *kidv = static_cast<V *>(h.kid);
    for (uint32_t s = threadIdx.x; s < (1u << HUB_SLOG); s += blockDim.x) { skeys[s] = EMPTY; svals[s] = V(0); }
    if (threadIdx.x == 0) s_nocc = 0;
    const uint64_t base = h.tasks[0], total = h.tasks[h.nh] - base;
    for (uint64_t task = blockIdx.x; task < total; task += gridDim.x) {
        uint32_t t = task_item(h.tasks, h.nh, task + base);
        if (!h.go[t]) continue;
        uint64_t chunk = task + base - h.tasks[t];
        uint32_t i = h.hubs[t], d = h.d[t];
        uint64_t e1 = a.off[i + 1];
        uint64_t b = a.off[i] + chunk * HUB_CHUNK;
        uint64_t e = min(b + HUB_CHUNK, e1);
        V kid = 0;
        scan_edges<4, SYNC, V>(a.tgt, w, a.C, i, d, b, e, threadIdx.x, blockDim.x, kid,
                               [&](uint32_t c, V wv) { smem_add<V>(skeys, svals, HUB_SLOG, socc, &s_nocc, c, wv); });
        kid = block_sum<V>(kid, red);
        if (threadIdx.x == 0 && kid != V(0)) atomicAdd(kidv + t, kid);
        int glog = ceil_log2((uint32_t)(2 * (e1 - a.off[i])));
        publish_block_table<V>(skeys, svals, socc, &s_nocc, h.keys + h.pool_off[t],
                               static_cast<V *>(h.vals) + h.pool_off[t], glog, h.occ + h.pool_off[t], h.occ_n + t);
    }
}

// Scoring uses the insert's task split: task k of a hub scores occupied
// entries [k*HUB_CHUNK, (k+1)*HUB_CHUNK) (a hub has at most one distinct
// community per edge) and leaves its best in best[task].
template <typename WT, bool F64, int SYNC>
__global__ void __launch_bounds__(256) k_hub_score(MoveArgs a, HubArgs h) {
    using V = typename std::conditional<F64, double, float>::type;
    using SC = Score<F64>;
    using S = typename SC::S;
    __shared__ S red_s[32];
    __shared__ uint32_t red_c[32];
    const V *kidv = static_cast<const V *>(h.kid);
    S *bs = static_cast<S *>(h.best_s);
    const double m0 = *a.m;
    const double inv0 = 1.0 / m0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t base = h.tasks[0], total = h.tasks[h.nh] - base;
    for (uint64_t task = blockIdx.x; task < total; task += gridDim.x) {
        uint32_t t = task_item(h.tasks, h.nh, task + base);
        if (!h.go[t]) continue;
        uint64_t k0 = (task + base - h.tasks[t]) * HUB_CHUNK;
        uint32_t i = h.hubs[t], d = h.d[t];
        uint32_t *keys = h.keys + h.pool_off[t];
        V *vals = static_cast<V *>(h.vals) + h.pool_off[t];
        const uint32_t *occ = h.occ + h.pool_off[t];
        uint64_t k1 = min(k0 + HUB_CHUNK, (uint64_t)h.occ_n[t]);
        SC sc = make_score<F64>(a.K[i], (double)kidv[t], ld_state<SYNC>(a.Sig + d), vertex_m(a, i, m0),
                                vertex_inv_m(a, i, inv0));
        S best = -INFINITY;
        uint32_t bestc = EMPTY;
        // U entries per thread per round; each level of the gather chain
        // (occupied list -> slot -> Sigma) is issued for all U at once
        constexpr int U = 8;
        for (uint64_t kb = k0 + threadIdx.x; kb < k1; kb += (uint64_t)U * blockDim.x) {
            uint32_t slot[U], c[U];
            V val[U];
            double sg[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                uint64_t k = kb + (uint64_t)u * blockDim.x;
                slot[u] = k < k1 ? occ[k] : EMPTY;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                c[u] = slot[u] != EMPTY ? keys[slot[u]] : EMPTY;
                val[u] = slot[u] != EMPTY ? vals[slot[u]] : V(0);
            }
#pragma unroll
            for (int u = 0; u < U; u++) sg[u] = c[u] != EMPTY ? ld_state<SYNC>(a.Sig + c[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (c[u] == EMPTY) continue;
                S v = sc.score(val[u], sg[u]);
                if (better(v, c[u], best, bestc)) { best = v; bestc = c[u]; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S v2 = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            uint32_t c2 = __shfl_xor_sync(0xFFFFFFFFu, bestc, o);
            if (better(v2, c2, best, bestc)) { best = v2; bestc = c2; }
        }
        __syncthreads();
        if (lane == 0) { red_s[wid] = best; red_c[wid] = bestc; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < (int)(blockDim.x >> 5); k++)
                if (better(red_s[k], red_c[k], best, bestc)) { best = red_s[k]; bestc = red_c[k]; }
            bs[task] = best;
            h.best_c[task] = bestc;
        }
    }
}

template <bool F64, int SYNC>
__global__ void k_hub_decide(MoveArgs a, HubArgs h) {
    using V = typename std::conditional<F64, double, float>::type;
    using SC = Score<F64>;
    using S = typename SC::S;
    const V *kidv = static_cast<const V *>(h.kid);
    const S *bs = static_cast<const S *>(h.best_s);
    const double m0 = *a.m;
    const double inv0 = 1.0 / m0;
    const int lane = threadIdx.x & 31;
    uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint64_t base = h.tasks[0];
    LocalCtr lc;
    for (uint32_t t = warp; t < h.nh; t += nwarps) {
        if (!h.go[t]) continue;
        uint32_t i = h.hubs[t], d = h.d[t];
        S best = -INFINITY;
        uint32_t bestc = EMPTY;
        for (uint64_t k = h.tasks[t] - base + lane; k < h.tasks[t + 1] - base; k += 32) {
            S v = bs[k];
            uint32_t c = h.best_c[k];
            if (c != EMPTY && better(v, c, best, bestc)) { best = v; bestc = c; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S v2 = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            uint32_t c2 = __shfl_xor_sync(0xFFFFFFFFu, bestc, o);
            if (better(v2, c2, best, bestc)) { best = v2; bestc = c2; }
        }
        if (lane == 0) {
            double Ki = a.K[i];
            uint64_t deg = a.off[i + 1] - a.off[i];
            const double m = vertex_m(a, i, m0);
            SC sc = make_score<F64>(Ki, (double)kidv[t], ld_state<SYNC>(a.Sig + d), m, vertex_inv_m(a, i, inv0));
            double gain = (bestc == EMPTY) ? 0.0 : sc.gain(best);
            int mv = 0;
            if (gain > 0.0) mv = decide_move<SYNC>(a, i, d, bestc, Ki);
            lc.vertices++;
            lc.edges += deg;
            lc.candidates += h.occ_n[t];
            h.occ_n[t] = 0;
            if (mv) {  // neighbours are re-marked by k_mark_big
                lc.moved++;
                lc.dq += gain;
                add_graph_gain(a, i, gain);
                lc.marked += deg;
                h.big[atomicAdd(h.nbig, 1u)] = i;
            }
            record_visit(a, i, (uint32_t)deg, Ki, (double)kidv[t], gain, m, mv);
        }
    }
    flush_counters(lc, a.ctr);
}

__global__ void k_hub_tasks(const uint64_t *__restrict__ off, const uint32_t *__restrict__ list, uint32_t count,
                            uint64_t *ntask) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        uint32_t v = list[t];
        ntask[t] = (off[v + 1] - off[v] + HUB_CHUNK - 1) / HUB_CHUNK;
    }
}

// --------------------------------------------------------------------------
// Degree classes
// --------------------------------------------------------------------------
__device__ __forceinline__ int class_of(uint64_t deg, const ClassBounds &cb) {
    if (deg <= 8) return CLS_G4;
    if (deg <= 16) return CLS_G8;
    if (deg <= 32) return CLS_G16;
    if (deg <= cb.group_max) return CLS_G32;
    if (deg <= cb.warp_max) return CLS_W512;
    if (deg <= cb.block_max) return CLS_BLOCK;
    if (deg <= cb.big_max) return CLS_BIG;
    return CLS_HUGE;
}

// Wave of vertex v: a hash of its index within its graph, mod W.  The hash
// (the MurmurHash3 32-bit finaliser, Appleby) keeps arithmetic patterns of
// ids out of the waves: with the index itself, every community of a planted
// graph whose community count shares a factor with W (vertex v in community
// v mod k) fell into few waves, decided at once and cycled.
__device__ __forceinline__ uint32_t wave_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ int wave_of(uint32_t v, int W, const uint32_t *gid, const uint64_t *gvo) {
    const uint32_t local = gid ? (uint32_t)(v - gvo[gid[v]]) : v;
    return (int)(wave_hash(local) % (uint32_t)W);
}

__global__ void k_classify_count(const uint64_t *__restrict__ off, uint32_t n, int W, uint32_t *counts,
                                 const uint32_t *__restrict__ gid, const uint64_t *__restrict__ gvo, ClassBounds cb) {
    __shared__ uint32_t sc[NUM_CLS * MAX_WAVES];
    for (int t = threadIdx.x; t < NUM_CLS * W; t += blockDim.x) sc[t] = 0;
    __syncthreads();
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t deg = off[v + 1] - off[v];
        if (deg) atomicAdd(&sc[class_of(deg, cb) * W + wave_of(v, W, gid, gvo)], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NUM_CLS * W; t += blockDim.x)
        if (sc[t]) atomicAdd(&counts[t], sc[t]);
}

__global__ void k_classify_fill(const uint64_t *__restrict__ off, uint32_t n, int W, uint32_t *cursor,
                                uint32_t *list, const uint32_t *__restrict__ gid, const uint64_t *__restrict__ gvo,
                                ClassBounds cb) {
    int lane = threadIdx.x & 31;
    for (uint32_t v0 = blockIdx.x * blockDim.x; v0 < n; v0 += gridDim.x * blockDim.x) {
        uint32_t v = v0 + threadIdx.x;
        uint64_t deg = (v < n) ? off[v + 1] - off[v] : 0;
        int key = deg ? class_of(deg, cb) * W + wave_of(v, W, gid, gvo) : -1;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
        int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && key >= 0) base = atomicAdd(&cursor[key], (uint32_t)__popc(peers));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (key >= 0) list[base + __popc(peers & ((1u << lane) - 1u))] = v;
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

void classify_vertices(const DevGraph &g, Classes &cl, int waves, cudaStream_t s, const uint32_t *gid,
                       const uint64_t *gvo) {
    GSP_REQUIRE(waves >= 1 && waves <= MAX_WAVES, "waves must be in [1, %d]", MAX_WAVES);
    const int W = waves;
    const int NK = NUM_CLS * W;
    cl.W = W;
    uint32_t *counts = arena().get<uint32_t>(2 * NK);
    GSP_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * NK, s));
    unsigned grid = grid_for(g.n, 256, sms(8));
    const Tuning tn = tuning();
    const ClassBounds cb{tn.group_max, tn.warp_max, tn.block_max, tn.big_max};
    k_classify_count<<<grid, 256, 0, s>>>(g.off, g.n, W, counts, gid, gvo, cb);
    GSP_CHECK_LAUNCH();
    uint32_t h[NUM_CLS * MAX_WAVES];
    GSP_CUDA(cudaMemcpyAsync(h, counts, sizeof(uint32_t) * NK, cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    cl.start[0] = 0;
    for (int k = 0; k < NK; k++) cl.start[k + 1] = cl.start[k] + h[k];
    uint32_t *cursor = counts + NK;
    GSP_CUDA(cudaMemcpyAsync(cursor, cl.start, sizeof(uint32_t) * NK, cudaMemcpyHostToDevice, s));
    cl.list = arena().get<uint32_t>(cl.start[NK] + 1);
    k_classify_fill<<<grid, 256, 0, s>>>(g.off, g.n, W, cursor, cl.list, gid, gvo, cb);
    GSP_CHECK_LAUNCH();
    cl.dstart = arena().get<uint32_t>(NK + 1);
    GSP_CUDA(cudaMemcpyAsync(cl.dstart, cl.start, sizeof(uint32_t) * (NK + 1), cudaMemcpyHostToDevice, s));
    uint32_t nh = cl.cls_count(CLS_HUGE);
    cl.pool_off = arena().get<uint64_t>(nh + 1);
    cl.pool_slots = 0;
    if (nh) {
        uint64_t *caps = arena().get<uint64_t>(nh);
        k_pool_caps<<<grid_for(nh, 256), 256, 0, s>>>(g.off, cl.list + cl.cls_begin(CLS_HUGE), nh, caps);
        GSP_CHECK_LAUNCH();
        exclusive_scan_u64(caps, cl.pool_off, nh, s);
        cl.host_pool_off.resize(nh + 1);
        GSP_CUDA(cudaMemcpyAsync(cl.host_pool_off.data(), cl.pool_off, sizeof(uint64_t) * (nh + 1),
                                 cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        cl.pool_slots = cl.host_pool_off[nh];
        uint64_t *ntask = arena().get<uint64_t>(nh);
        cl.hub_tasks = arena().get<uint64_t>(nh + 1);
        k_hub_tasks<<<grid_for(nh, 256), 256, 0, s>>>(g.off, cl.list + cl.cls_begin(CLS_HUGE), nh, ntask);
        GSP_CHECK_LAUNCH();
        exclusive_scan_u64(ntask, cl.hub_tasks, nh, s);
        cl.host_hub_tasks.resize(nh + 1);
        GSP_CUDA(cudaMemcpyAsync(cl.host_hub_tasks.data(), cl.hub_tasks, sizeof(uint64_t) * (nh + 1),
                                 cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        cl.hub_occ_n = arena().get<uint32_t>(nh);
        GSP_CUDA(cudaMemsetAsync(cl.hub_occ_n, 0, sizeof(uint32_t) * nh, s));
    }
}

// --------------------------------------------------------------------------
// Host launchers
// --------------------------------------------------------------------------
SideStreams &side_streams() {
    static SideStreams ss[16];
    static bool made[16] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 15;
    if (!made[dev]) {
        for (int k = 0; k < SideStreams::N; k++)
            GSP_CUDA(cudaStreamCreateWithFlags(&ss[dev].side[k], cudaStreamNonBlocking));
        for (int f = 0; f < 64; f++) {
            GSP_CUDA(cudaEventCreateWithFlags(&ss[dev].fork_ev[f], cudaEventDisableTiming));
            for (int k = 0; k < SideStreams::N; k++)
                GSP_CUDA(cudaEventCreateWithFlags(&ss[dev].join_ev[f][k], cudaEventDisableTiming));
        }
        made[dev] = true;
    }
    return ss[dev];
}

// The class kernels of a wave touch disjoint vertices and only append to the
// move list, so they run as parallel branches: W512 and the block class on
// side streams 0 and 1, the hub chain on side stream 2, the big-table block
// class on side stream 3, the group classes on the main stream; all join
// before the wave's moves are applied.
template <typename WT, bool F64, int SYNC>
static void launch_wave(const Classes &cl, const MoveArgs &a, int wave, uint32_t *pool_keys, void *pool_vals,
                        uint32_t *pool_occ, uint32_t *big, uint32_t *nbig, cudaStream_t main) {
    using V = typename std::conditional<F64, double, float>::type;
    SideStreams &ss = side_streams();
    const int f = ss.next;
    ss.next = (ss.next + 1) & 63;
    bool used[SideStreams::N] = {false, false, false, false};
    GSP_CUDA(cudaEventRecord(ss.fork_ev[f], main));
    auto on = [&](int k) -> cudaStream_t {
        if (!used[k]) {
            GSP_CUDA(cudaStreamWaitEvent(ss.side[k], ss.fork_ev[f], 0));
            used[k] = true;
        }
        return ss.side[k];
    };
    cudaStream_t s = main;
    const Tuning tn = tuning();
    const int sm = sm_count();
    GroupLists gl;
    const int G[4] = {4, 8, 16, 32};
    uint32_t blocks = 0;
    for (int c = 0; c < 4; c++) {
        gl.list[c] = cl.list + cl.begin(c, wave);
        gl.count[c] = cl.count(c, wave);
        gl.bstart[c] = blocks;
        if (gl.count[c]) blocks += grid_for((uint64_t)gl.count[c] * G[c], 256, (uint32_t)(sm * tn.groups));
    }
    gl.bstart[4] = blocks;
    if (blocks) {
        k_move_groups<WT, F64, SYNC><<<blocks, 256, 0, s>>>(a, gl);
        GSP_CHECK_LAUNCH();
    }
    uint32_t nw5 = cl.count(CLS_W512, wave);
    if (nw5) {
        constexpr size_t smem = (size_t)8 * W512_CAP * (sizeof(uint32_t) + sizeof(V));
        static bool attr = false;
        if (!attr) {
            GSP_CUDA(cudaFuncSetAttribute(k_move_w512<WT, F64, SYNC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            attr = true;
        }
        k_move_w512<WT, F64, SYNC><<<grid_for((uint64_t)nw5 * 32, 256, (uint32_t)(sm * tn.w512)), 256, smem, on(0)>>>(
            a, cl.list + cl.begin(CLS_W512, wave), nw5);
        GSP_CHECK_LAUNCH();
    }
    uint32_t nb = cl.count(CLS_BLOCK, wave);
    if (nb) {
        constexpr int CAP = 4096;
        constexpr size_t smem = (size_t)CAP * (sizeof(uint32_t) + sizeof(V) + sizeof(uint16_t));
        static bool attr = false;
        if (!attr) {
            GSP_CUDA(cudaFuncSetAttribute(k_move_block<CAP, WT, F64, SYNC>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = true;
        }
        k_move_block<CAP, WT, F64, SYNC><<<grid_for(nb, 1, (uint32_t)(sm * tn.block)), 256, smem, on(1)>>>(
            a, cl.list + cl.begin(CLS_BLOCK, wave), nb);
        GSP_CHECK_LAUNCH();
    }
    uint32_t ng = cl.count(CLS_BIG, wave);
    if (ng) {
        // 2049..8192 edges: one block per vertex with a 16384-slot shared
        // table (at most 2 x 8192 distinct keys), one block per SM
        constexpr int CAP = 16384;
        constexpr size_t smem = (size_t)CAP * (sizeof(uint32_t) + sizeof(V) + sizeof(uint16_t));
        static bool attr = false;
        if (!attr) {
            GSP_CUDA(cudaFuncSetAttribute(k_move_block<CAP, WT, F64, SYNC>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = true;
        }
        k_move_block<CAP, WT, F64, SYNC><<<grid_for(ng, 1, (uint32_t)sm), 256, smem, on(3)>>>(
            a, cl.list + cl.begin(CLS_BIG, wave), ng);
        GSP_CHECK_LAUNCH();
    }
    uint32_t nh = cl.count(CLS_HUGE, wave);
    if (nh) {
        cudaStream_t s = on(2);
        using S = typename Score<F64>::S;
        uint32_t rel = cl.begin(CLS_HUGE, wave) - cl.cls_begin(CLS_HUGE);
        size_t mk = arena().mark();
        HubArgs h;
        h.hubs = cl.list + cl.begin(CLS_HUGE, wave);
        h.nh = nh;
        h.pool_off = cl.pool_off + rel;
        h.tasks = cl.hub_tasks + rel;
        h.keys = pool_keys;
        h.vals = pool_vals;
        h.occ = pool_occ;
        h.occ_n = cl.hub_occ_n + rel;
        h.kid = arena().alloc(sizeof(V) * nh);
        h.go = arena().get<uint8_t>(nh);
        h.d = arena().get<uint32_t>(nh);
        uint64_t ntasks = cl.host_hub_tasks[rel + nh] - cl.host_hub_tasks[rel];
        h.best_s = arena().alloc(sizeof(S) * ntasks);
        h.best_c = arena().get<uint32_t>(ntasks);
        h.big = big;
        h.nbig = nbig;
        // this wave's tables: one contiguous slice of the pool, cleared with
        // coalesced memsets
        uint64_t first = cl.host_pool_off[rel], last = cl.host_pool_off[rel + nh];
        GSP_CUDA(cudaMemsetAsync(pool_keys + first, 0xFF, sizeof(uint32_t) * (last - first), s));
        GSP_CUDA(cudaMemsetAsync(static_cast<V *>(pool_vals) + first, 0, sizeof(V) * (last - first), s));
        GSP_CUDA(cudaMemsetAsync(h.kid, 0, sizeof(V) * nh, s));
        k_hub_prepare<SYNC><<<grid_for(nh, 256), 256, 0, s>>>(a, h);
        GSP_CHECK_LAUNCH();
        constexpr size_t hsmem = (sizeof(uint32_t) + sizeof(V) + sizeof(uint16_t)) << HUB_SLOG;
        static bool attr = false;
        if (!attr) {
            GSP_CUDA(cudaFuncSetAttribute(k_hub_insert<WT, F64, SYNC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)hsmem));
            attr = true;
        }
        // one block per task at most: small waves launch only what they use
        const unsigned hub_grid = (unsigned)std::min<uint64_t>(ntasks, (uint64_t)sm * tn.hub);
        k_hub_insert<WT, F64, SYNC><<<hub_grid, 256, hsmem, s>>>(a, h);
        GSP_CHECK_LAUNCH();
        k_hub_score<WT, F64, SYNC><<<hub_grid, 256, 0, s>>>(a, h);
        GSP_CHECK_LAUNCH();
        k_hub_decide<F64, SYNC><<<grid_for((uint64_t)nh * 32, 256), 256, 0, s>>>(a, h);
        GSP_CHECK_LAUNCH();
        arena().release(mk);
    }
    for (int k = 0; k < SideStreams::N; k++) {
        if (!used[k]) continue;
        GSP_CUDA(cudaEventRecord(ss.join_ev[f][k], ss.side[k]));
        GSP_CUDA(cudaStreamWaitEvent(main, ss.join_ev[f][k], 0));
    }
}

static MoveArgs make_move_args(const DevGraph &g, const MoveBuffers &mb, bool sync, bool rule, int iteration,
                               int max_iterations) {
    MoveArgs a;
    a.off = g.off;
    a.tgt = g.tgt;
    a.w = g.w;
    a.C = mb.C;
    a.K = mb.K;
    a.Sig = mb.Sigma;
    a.size = mb.size;
    a.act = mb.act;
    a.mark = sync ? mb.mark : mb.act;
    a.m = mb.m_dev;
    a.gid = mb.gid;
    a.m_g = mb.m_g;
    a.minv_g = mb.minv_g;
    a.lsb = mb.lsb;
    a.dq_g = mb.dq_g;
    a.ctr = mb.ctr;
    a.rule = rule ? 1 : 0;
    a.left = mb.left;
    a.left_it = mb.left_it;
    a.iteration = mb.it_dev;
    a.no_return_from = mb.no_return_from;
    a.mv_vtx = mb.mv_vtx;
    a.mv_cmt = mb.mv_cmt;
    a.mv_cnt = mb.mv_cnt;
    a.choice = mb.choice;
    a.feat_kept = mb.feat_kept;
    a.feat_gain = mb.feat_gain;
    a.last_gain = mb.last_gain;
    a.moved_last = mb.moved_last;
    a.deferred = mb.skip;
    a.trace_x = mb.trace_x;
    a.trace_y = mb.trace_y;
    a.trace_cnt = mb.trace_cnt;
    a.trace_cap = mb.trace_cap;
    a.trace_keys = mb.trace_keys;
    a.trace_tag = ((uint64_t)(mb.trace_pass & 0xFF) << 56) | ((uint64_t)(mb.cur_repeat & 0xFF) << 40);
    a.trace_every = mb.trace_every ? mb.trace_every : 1;
    a.max_logk = mb.max_logk;
    a.max_iterations = max_iterations;
    a.salt = mb.trace_salt;
    return a;
}

template <typename WT, bool F64>
static bool launch_persistent(const MoveArgs &a, const Classes &cl, uint32_t n, MoveBuffers &mb, int iteration,
                              cudaStream_t s) {
    using V = typename std::conditional<F64, double, float>::type;
    constexpr size_t smem = std::max(std::max((size_t)8 * W512_CAP * (sizeof(uint32_t) + sizeof(V)),
                                              (size_t)4096 * (sizeof(uint32_t) + sizeof(V) + sizeof(uint16_t))),
                                     (size_t)(sizeof(uint32_t) + sizeof(double) + sizeof(int)) << APPLY_SLOG);
    static int per_sm[64] = {0};  // resident blocks per SM, per device (-1: cannot run)
    int dev = 0;
    GSP_CUDA(cudaGetDevice(&dev));
    dev &= 63;
    if (!per_sm[dev]) {
        GSP_CUDA(cudaFuncSetAttribute(k_sweep_persistent<WT, F64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        int coop = 0, nblk = 0;
        GSP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        GSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, k_sweep_persistent<WT, F64>, 256, smem));
        per_sm[dev] = (coop && nblk > 0) ? nblk : -1;
    }
    if (per_sm[dev] < 0) return false;
    MoveArgs aa = a;
    const uint32_t *list = cl.list;
    const uint32_t *start = cl.dstart;
    int W = cl.W;
    int R = std::min(wave_repeats_at(mb, iteration), MAX_REPEATS);
    uint32_t nn = n;
    uint32_t *cnts = mb.mv_cnts;
    GridBar *bar = mb.bar;
    void *args[] = {&aa, &list, &start, &W, &R, &nn, &cnts, &bar};
    GSP_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBar), s));
    GSP_CUDA(cudaLaunchCooperativeKernel((const void *)k_sweep_persistent<WT, F64>, dim3(per_sm[dev] * sm_count()),
                                         dim3(256), args, smem, s));
    count_launch();
    return true;
}

bool sweep_persistent(const DevGraph &g, const Classes &cl, MoveBuffers &mb, bool fp64, bool rule, int iteration,
                      int max_iterations, cudaStream_t s) {
    if (cl.cls_count(CLS_HUGE) || cl.cls_count(CLS_BIG) || mb.feat_kept || mb.choice || !cl.dstart || !mb.bar)
        return false;
    if (g.n > tuning().persist_max_vertices) return false;
    MoveArgs a = make_move_args(g, mb, true, rule, iteration, max_iterations);
    if (g.wt == GSP_W_F32) return fp64 ? launch_persistent<float, true>(a, cl, g.n, mb, iteration, s)
                                       : launch_persistent<float, false>(a, cl, g.n, mb, iteration, s);
    return fp64 ? launch_persistent<double, true>(a, cl, g.n, mb, iteration, s)
                : launch_persistent<double, false>(a, cl, g.n, mb, iteration, s);
}

void move_wave(const DevGraph &g, const Classes &cl, MoveBuffers &mb, int wave, bool sync, bool fp64, bool rule,
               bool learned, int iteration, int max_iterations, cudaStream_t s) {
    (void)learned;
    MoveArgs a = make_move_args(g, mb, sync, rule, iteration, max_iterations);
    // pool layout: keys (u32), values (8 bytes per slot), occupied-slot list (u32)
    uint32_t *pool_keys = static_cast<uint32_t *>(mb.pool);
    const size_t sa = align_up(cl.pool_slots, 64);
    void *pool_vals = pool_keys ? static_cast<void *>(pool_keys + sa) : nullptr;
    uint32_t *pool_occ = pool_keys ? pool_keys + 3 * sa : nullptr;
    GSP_CUDA(cudaMemsetAsync(mb.nbig, 0, sizeof(uint32_t), s));
#define GSP_WAVE(WT, F64, SYNC) \
    launch_wave<WT, F64, SYNC>(cl, a, wave, pool_keys, pool_vals, pool_occ, mb.big, mb.nbig, s)
    if (g.wt == GSP_W_F32) {
        if (fp64) { if (sync) GSP_WAVE(float, true, true); else GSP_WAVE(float, true, false); }
        else { if (sync) GSP_WAVE(float, false, true); else GSP_WAVE(float, false, false); }
    } else {
        if (fp64) { if (sync) GSP_WAVE(double, true, true); else GSP_WAVE(double, true, false); }
        else { if (sync) GSP_WAVE(double, false, true); else GSP_WAVE(double, false, false); }
    }
#undef GSP_WAVE
    if (cl.count(CLS_HUGE, wave)) {  // hub movers re-mark their neighbours
        k_mark_big<<<dim3(sm_count(), 16), 256, 0, s>>>(g.off, g.tgt, mb.big, mb.nbig, a.mark);
        GSP_CHECK_LAUNCH();
    }
}

void apply_moves(const DevGraph &g, MoveBuffers &mb, uint32_t n_hint, cudaStream_t s) {
    k_apply_moves<<<grid_for(n_hint, 256, sms(4)), 256, 0, s>>>(mb.mv_vtx, mb.mv_cmt, mb.mv_cnt, mb.K, mb.C,
                                                                 mb.Sigma, mb.size, mb.lsb, mb.left, mb.left_it,
                                                                 mb.it_dev);
    GSP_CHECK_LAUNCH();
    k_merge_marks<<<grid_for(g.n / 16 + 1, 256, sms(8)), 256, 0, s>>>(mb.act, mb.mark, g.n);
    GSP_CHECK_LAUNCH();
}

}  // namespace gsp
