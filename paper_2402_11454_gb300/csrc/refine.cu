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
// The well-connectedness of each refined community is a flag, computed in
// float64 for every singleton and again for each community that gained
// members in a wave.
//
// Precision.  FP64: table sums, gains and scores in float64, each operation
// rounded as written (no fused multiply-add), as the sequential evaluation
// does.  MIXED: table sums, gains (K_v times S_c / 2m, the quotient formed
// in float64 per community) and scores in float32, the Gumbel noise from
// 23 random bits; the well-connectedness flags stay float64.  float64 sums
// are additions in an unspecified order, exact -- and so equal to a
// sequential evaluation -- when the weights are integer multiples of a power
// of two with totals below 2^53 units.
//
// Only candidates whose gain is within GUMBEL_SPAN * theta of the vertex's
// best gain draw their noise: the noise of a draw is bounded, so the others
// cannot win, and skipping them changes no choice.
#include "internal.cuh"

namespace gsp {

namespace {

constexpr int RF_THREADS = 256;
constexpr int RF_WARPS = RF_THREADS / 32;
constexpr uint64_t GOLDEN_GAMMA = 0x9e3779b97f4a7c15ull;

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output for generator
// state x (the state advanced by the golden gamma, then the mixer).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + GOLDEN_GAMMA;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// The draw of (vertex, candidate) in the pass's stream of the seed
// (pass_key = splitmix64(seed + gamma * (pass + 1))).
__device__ __forceinline__ uint64_t draw(uint64_t pass_key, uint32_t v, uint32_t c) {
    return splitmix64(pass_key ^ (((uint64_t)v << 32) | c));
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
    float *SRf;          // S_c / 2m per refined community, as float32 (MIXED gains)
    double *ext;         // E(c, b-c) per refined community
    uint32_t *size;      // members per refined community
    uint8_t *wc;         // refined community well connected to its bound community
    uint32_t *T;         // decision of each vertex of the current wave
    uint8_t *targeted;   // refined communities some mover of the wave targets
    uint8_t *joined;     // movers of the wave that joined their target
    unsigned long long *moves;
    double two_m;
    double theta;
    uint64_t pass_key;
    // batches of graphs: graph of each vertex, 2m of each graph, first vertex
    // of each graph (NULL for one graph); the draws are keyed by indices
    // within the graph, so that a graph refines as it does alone
    const uint32_t *gid;
    const double *two_m_g;
    const uint64_t *gvo;
};

// 2m of vertex v's graph.
__device__ __forceinline__ double two_m_of(const RefineState &a, uint32_t v) {
    return a.gid ? a.two_m_g[a.gid[v]] : a.two_m;
}

// Index of vertex v within its graph.
__device__ __forceinline__ uint32_t local_id(const RefineState &a, uint32_t v) {
    return a.gid ? (uint32_t)(v - a.gvo[a.gid[v]]) : v;
}

// Score arithmetic of the two precision modes.  SPAN: a bound on the spread
// of the Gumbel noise, -ln(-ln u) for the smallest and the largest draw
// (52 bits: [-3.604, 36.737]; 23 bits: [-2.812, 16.636]), with room for the
// rounding of the scores.
template <typename S> struct Score;
template <> struct Score<double> {
    static constexpr double SPAN = 48.0;
    template <typename WT> __device__ static double weight(const WT *w, uint64_t e) { return wload(w, e); }
    __device__ static double kv(const RefineState &a, uint32_t v) { return a.K[v]; }
    __device__ static double gain(const RefineState &a, double Kv, uint32_t c, double H) {
        return __dsub_rn(H, __ddiv_rn(__dmul_rn(Kv, a.SR[c]), two_m_of(a, c)));
    }
    __device__ static double noise(const RefineState &a, uint32_t v, uint32_t c) {
        uint64_t r = draw(a.pass_key, local_id(a, v), local_id(a, c));
        double u = __dmul_rn(__dadd_rn((double)(r >> 12), 0.5), 0x1.0p-52);
        return -log(-log(u));
    }
    __device__ static double score(const RefineState &a, uint32_t v, uint32_t c, double g) {
        return __dadd_rn(__ddiv_rn(g, a.theta), noise(a, v, c));
    }
    __device__ static double theta(const RefineState &a) { return a.theta; }
};
template <> struct Score<float> {
    static constexpr float SPAN = 28.0f;
    template <typename WT> __device__ static float weight(const WT *w, uint64_t e) { return wloadf(w, e); }
    __device__ static float kv(const RefineState &a, uint32_t v) { return (float)a.K[v]; }
    __device__ static float gain(const RefineState &a, float Kv, uint32_t c, float H) { return H - Kv * a.SRf[c]; }
    __device__ static float noise(const RefineState &a, uint32_t v, uint32_t c) {
        uint64_t r = draw(a.pass_key, local_id(a, v), local_id(a, c));
        float u = ((float)(uint32_t)(r >> 41) + 0.5f) * 0x1.0p-23f;
        return -logf(-logf(u));
    }
    __device__ static float score(const RefineState &a, uint32_t v, uint32_t c, float g) {
        return g / (float)a.theta + noise(a, v, c);
    }
    __device__ static float theta(const RefineState &a) { return (float)a.theta; }
};

// Up to NUM_CLS slices of the class/wave list, addressed as one sequence.
struct Slices {
    const uint32_t *list;
    uint32_t begin[NUM_CLS];
    uint32_t prefix[NUM_CLS + 1];
    uint32_t count;  // prefix[n]
    int n;
    __device__ __forceinline__ uint32_t at(uint32_t i) const {
        // unrolled with constant indices, so the arrays stay in parameter space
        uint32_t b = begin[0], p = prefix[0];
#pragma unroll
        for (int k = 1; k < NUM_CLS; k++)
            if (k < n && i >= prefix[k]) {
                b = begin[k];
                p = prefix[k];
            }
        return list[b + (i - p)];
    }
    __host__ __device__ __forceinline__ uint32_t total() const { return count; }
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
    s.count = s.prefix[ncls];
    return s;
}

// Vertices of classes [lo, hi) over all waves: one contiguous slice.
Slices class_range(const Classes &cl, int lo, int hi) {
    Slices s;
    s.list = cl.list;
    s.n = 1;
    s.begin[0] = cl.start[lo * cl.W];
    s.prefix[0] = 0;
    s.prefix[1] = cl.start[hi * cl.W] - cl.start[lo * cl.W];
    s.count = s.prefix[1];
    return s;
}

// E(c, b-c) >= S_c (S_b - S_c) / 2m, rounded as written.
__device__ __forceinline__ bool well_connected(double ext, double S, double Sb, double two_m) {
    return ext >= __ddiv_rn(__dmul_rn(S, __dsub_rn(Sb, S)), two_m);
}

// v may move only while it is alone in R and well connected to its bound
// community (its singleton's flag).
__device__ __forceinline__ bool may_move(const RefineState &a, uint32_t v) {
    return a.R[v] == v && a.size[v] == 1 && a.wc[v];
}

// Gain of joining c (E(v, c) = H), or false when c is not eligible: not
// well connected, or a gain below 0 (theta > 0) or not above 0 (greedy).
template <typename S>
__device__ __forceinline__ bool candidate_gain(const RefineState &a, S Kv, uint32_t c, S H, S *gain) {
    if (!a.wc[c]) return false;
    S g = Score<S>::gain(a, Kv, c, H);
    *gain = g;
    return a.theta > 0.0 ? g >= S(0) : g > S(0);
}

template <typename S> struct Best {
    S s;
    uint32_t c;
    int have;
};

template <typename S> __device__ __forceinline__ bool better(const Best<S> &x, const Best<S> &y) {
    if (!x.have) return false;
    if (!y.have) return true;
    return x.s > y.s || (x.s == y.s && x.c < y.c);
}

template <typename S> __device__ __forceinline__ void offer(Best<S> &best, S s, uint32_t c) {
    Best<S> y{s, c, 1};
    if (better(y, best)) best = y;
}

// An eligible candidate with gain g: its gain (greedy), or g / theta plus
// its noise when it is near enough the best gain gmax.
template <typename S>
__device__ __forceinline__ void offer_scored(const RefineState &a, Best<S> &best, uint32_t v, uint32_t c, S g,
                                             S gmax) {
    if (a.theta > 0.0) {
        if (g >= gmax - Score<S>::SPAN * Score<S>::theta(a)) offer(best, Score<S>::score(a, v, c, g), c);
    } else {
        offer(best, g, c);
    }
}

// Staying (gain 0) is a candidate of the random choice only.
template <typename S> __device__ __forceinline__ void offer_stay(const RefineState &a, Best<S> &best, uint32_t v, S gmax) {
    if (a.theta > 0.0 && S(0) >= gmax - Score<S>::SPAN * Score<S>::theta(a)) offer(best, Score<S>::noise(a, v, v), v);
}

template <typename S> __device__ __forceinline__ void record(const RefineState &a, uint32_t v, const Best<S> &b) {
    a.T[v] = b.have ? b.c : v;
}

template <int G, typename S> __device__ __forceinline__ Best<S> group_best(Best<S> b) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        Best<S> y;
        y.s = __shfl_xor_sync(0xFFFFFFFFu, b.s, o);
        y.c = __shfl_xor_sync(0xFFFFFFFFu, b.c, o);
        y.have = __shfl_xor_sync(0xFFFFFFFFu, b.have, o);
        if (better(y, b)) b = y;
    }
    return b;
}

template <int G, typename S> __device__ __forceinline__ S group_max(S x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
    return x;
}

// Degrees up to 2G (the classes of 8, 16 and 32 edges): G lanes per vertex,
// two edges per lane, no table: each lane sums the group's weights of the
// refined communities its edges reach (shuffles in lane order) and scores
// them; equal communities held by several lanes score alike.
template <int G, typename WT, typename S>
__global__ void __launch_bounds__(RF_THREADS) k_refine_decide_group(RefineState a, Slices sl) {
    constexpr uint32_t PER_WARP = 32 / G;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), base = lane & ~(G - 1);
    const WT *w = static_cast<const WT *>(a.w);
    const uint32_t total = sl.total();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t0 = warp * PER_WARP; t0 < total; t0 += nwarps * PER_WARP) {  // warp-uniform
        const uint32_t t = t0 + lane / G;
        const bool valid = t < total;
        const uint32_t v = valid ? sl.at(t) : 0u;
        const bool go = valid && may_move(a, v);
        uint32_t k0 = EMPTY, k1 = EMPTY;
        S w0 = S(0), w1 = S(0);
        if (go) {
            const uint32_t b = a.B[v];
            const uint64_t end = a.off[v + 1];
            uint64_t e = a.off[v] + gl;
            if (e < end) {
                uint32_t u = a.tgt[e];
                if (u != v && a.B[u] == b) { k0 = a.R[u]; w0 = Score<S>::weight(w, e); }
            }
            e += G;
            if (e < end) {
                uint32_t u = a.tgt[e];
                if (u != v && a.B[u] == b) { k1 = a.R[u]; w1 = Score<S>::weight(w, e); }
            }
        }
        S s0 = S(0), s1 = S(0);
#pragma unroll
        for (int j = 0; j < G; j++) {
            const uint32_t kj0 = __shfl_sync(0xFFFFFFFFu, k0, base + j), kj1 = __shfl_sync(0xFFFFFFFFu, k1, base + j);
            const S wj0 = __shfl_sync(0xFFFFFFFFu, w0, base + j), wj1 = __shfl_sync(0xFFFFFFFFu, w1, base + j);
            if (kj0 == k0) s0 += wj0;
            if (kj1 == k0) s0 += wj1;
            if (kj0 == k1) s1 += wj0;
            if (kj1 == k1) s1 += wj1;
        }
        S g0 = S(0), g1 = S(0);
        bool e0 = false, e1 = false;
        const S Kv = go ? Score<S>::kv(a, v) : S(0);
        if (k0 != EMPTY) e0 = candidate_gain<S>(a, Kv, k0, s0, &g0);
        if (k1 != EMPTY) e1 = candidate_gain<S>(a, Kv, k1, s1, &g1);
        S gmax = S(-INFINITY);
        if (a.theta > 0.0) gmax = group_max<G, S>(fmax(e0 ? g0 : S(-INFINITY), e1 ? g1 : S(-INFINITY)));
        Best<S> best{S(0), v, 0};
        if (go && gl == 0) offer_stay<S>(a, best, v, gmax);
        if (e0) offer_scored<S>(a, best, v, k0, g0, gmax);
        if (e1) offer_scored<S>(a, best, v, k1, g1, gmax);
        best = group_best<G, S>(best);
        if (valid && gl == 0) record(a, v, best);
    }
}

// Table scans of the warp and block kernels.  First scan: each occupied
// slot's gain replaces E(v, c), ineligible slots are emptied, and the
// thread's largest gain (greedy: its best candidate) is kept.  Second scan
// (theta > 0, once the vertex's largest gain is known): the scores.
template <typename S>
__device__ __forceinline__ S scan_gains(const RefineState &a, S Kv, uint32_t *keys, S *vals, uint32_t cap,
                                        uint32_t first, uint32_t stride, Best<S> &best) {
    S gmax = S(-INFINITY);
    for (uint32_t s = first; s < cap; s += stride) {
        uint32_t c = keys[s];
        if (c == EMPTY) continue;
        S g;
        if (!candidate_gain<S>(a, Kv, c, vals[s], &g)) {
            keys[s] = EMPTY;
            continue;
        }
        vals[s] = g;
        gmax = fmax(gmax, g);
        if (!(a.theta > 0.0)) offer(best, g, c);
    }
    return gmax;
}

template <typename S>
__device__ __forceinline__ void scan_scores(const RefineState &a, uint32_t v, const uint32_t *keys, const S *vals,
                                            uint32_t cap, uint32_t first, uint32_t stride, S gmax, Best<S> &best) {
    for (uint32_t s = first; s < cap; s += stride) {
        uint32_t c = keys[s];
        if (c != EMPTY) offer_scored<S>(a, best, v, c, vals[s], gmax);
    }
}

// Degrees up to SLOTS / 2: one warp per vertex, a table per warp in dynamic
// shared memory (SLOTS values, then SLOTS keys per warp), of which a vertex
// uses the next power of two at or above twice its degree.
template <int SLOTS, typename WT, typename S>
__global__ void __launch_bounds__(RF_THREADS) k_refine_decide_warp(RefineState a, Slices sl) {
    extern __shared__ __align__(16) unsigned char rf_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    S *vals = reinterpret_cast<S *>(rf_smem) + wid * SLOTS;
    uint32_t *keys = reinterpret_cast<uint32_t *>(rf_smem + sizeof(S) * RF_WARPS * SLOTS) + wid * SLOTS;
    const WT *w = static_cast<const WT *>(a.w);
    const uint32_t total = sl.total();
    for (uint32_t t = blockIdx.x * RF_WARPS + wid; t < total; t += gridDim.x * RF_WARPS) {
        const uint32_t v = sl.at(t);
        if (!may_move(a, v)) {
            if (lane == 0) a.T[v] = v;
            continue;
        }
        const uint64_t e0 = a.off[v], e1 = a.off[v + 1];
        const int lg = ceil_log2((uint32_t)(2 * (e1 - e0)));
        const uint32_t cap = 1u << lg;
        for (uint32_t s = lane; s < cap; s += 32) {
            keys[s] = EMPTY;
            vals[s] = S(0);
        }
        __syncwarp();
        const uint32_t b = a.B[v];
        for (uint64_t e = e0 + lane; e < e1; e += 32) {
            uint32_t u = a.tgt[e];
            if (u != v && a.B[u] == b) ht_add<S>(keys, vals, lg, a.R[u], Score<S>::weight(w, e));
        }
        __syncwarp();
        Best<S> best{S(0), v, 0};
        S gmax = scan_gains<S>(a, Score<S>::kv(a, v), keys, vals, cap, lane, 32, best);
        if (a.theta > 0.0) {
            gmax = group_max<32, S>(gmax);
            if (lane == 0) offer_stay<S>(a, best, v, gmax);
            scan_scores<S>(a, v, keys, vals, cap, lane, 32, gmax, best);
        }
        best = group_best<32, S>(best);
        if (lane == 0) record(a, v, best);
        __syncwarp();
    }
}

// Larger degrees: one block per vertex, the table in dynamic shared memory
// (the next power of two at or above twice the degree).
template <typename WT, typename S>
__global__ void __launch_bounds__(RF_THREADS) k_refine_decide_block(RefineState a, Slices sl, uint32_t smem_slots) {
    extern __shared__ __align__(16) unsigned char rf_smem[];
    __shared__ Best<S> sbest[RF_WARPS];
    __shared__ S sgmax[RF_WARPS];
    __shared__ int s_go;
    const WT *w = static_cast<const WT *>(a.w);
    const uint32_t total = sl.total();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    S *vals = reinterpret_cast<S *>(rf_smem);
    uint32_t *keys = reinterpret_cast<uint32_t *>(rf_smem + sizeof(S) * smem_slots);
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        const uint32_t v = sl.at(t);
        if (threadIdx.x == 0) s_go = may_move(a, v);
        __syncthreads();
        if (!s_go) {
            if (threadIdx.x == 0) a.T[v] = v;
            __syncthreads();
            continue;
        }
        const uint64_t e0 = a.off[v], e1 = a.off[v + 1];
        const int lg = ceil_log2((uint32_t)(2 * (e1 - e0)));
        const uint32_t cap = 1u << lg;
        for (uint32_t s = threadIdx.x; s < cap; s += blockDim.x) {
            keys[s] = EMPTY;
            vals[s] = S(0);
        }
        __syncthreads();
        const uint32_t b = a.B[v];
        for (uint64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            uint32_t u = a.tgt[e];
            if (u != v && a.B[u] == b) ht_add<S>(keys, vals, lg, a.R[u], Score<S>::weight(w, e));
        }
        __syncthreads();
        Best<S> best{S(0), v, 0};
        S gmax = scan_gains<S>(a, Score<S>::kv(a, v), keys, vals, cap, threadIdx.x, blockDim.x, best);
        if (a.theta > 0.0) {
            gmax = group_max<32, S>(gmax);
            if (lane == 0) sgmax[wid] = gmax;
            __syncthreads();
            gmax = sgmax[0];
            for (int k = 1; k < RF_WARPS; k++) gmax = fmax(gmax, sgmax[k]);
            if (threadIdx.x == 0) offer_stay<S>(a, best, v, gmax);
            scan_scores<S>(a, v, keys, vals, cap, threadIdx.x, blockDim.x, gmax, best);
        }
        best = group_best<32, S>(best);
        if (lane == 0) sbest[wid] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            Best<S> r = sbest[0];
            for (int k = 1; k < RF_WARPS; k++)
                if (better(sbest[k], r)) r = sbest[k];
            record(a, v, r);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- hubs
// Vertices above the 16384-slot tables: their edges are cut into HUB_CHUNK-
// edge tasks (the hub task prefix of the class lists) that blocks insert
// into the hub's table in the hub pool; then every slot of the wave's hub
// tables is scored by its own thread, and the hub's choice is the best
// (score, id) pair, found with ordered 64-bit atomics.
struct HubArgs {
    const uint32_t *hubs;       // the wave's hubs (class list)
    const uint64_t *pool_off;   // table slots of the wave's hubs (pool offsets; hw + 1 entries)
    const uint64_t *tasks;      // task prefix of the wave's hubs (hw + 1 entries)
    const uint32_t *owner;      // hub (index within the wave) of each of the wave's tasks
    uint32_t nhubs;
    uint64_t slot0, slot1;      // the wave's table slots [slot0, slot1) of the pool
    uint32_t *keys;             // the hub pool
    void *vals;
    unsigned long long *best;   // per hub: best gain, then (nhubs on) best score, as ordered keys
    uint32_t *best_c;           // per hub: lowest id among the best
};

// Ordered keys of floating-point values: unsigned order equals value order.
__device__ __forceinline__ unsigned long long ordered(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ unsigned long long ordered(float x) { return ordered((double)x); }
template <typename S> __device__ __forceinline__ S from_ordered(unsigned long long k);
template <> __device__ __forceinline__ double from_ordered<double>(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}
template <> __device__ __forceinline__ float from_ordered<float>(unsigned long long k) {
    return (float)from_ordered<double>(k);
}

// Owner hub of slot s of the wave's tables (binary search of pool_off).
__device__ __forceinline__ uint32_t slot_owner(const HubArgs &h, uint64_t s) {
    uint32_t lo = 0, hi = h.nhubs;  // pool_off[lo] <= s < pool_off[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (h.pool_off[mid] <= s) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename WT, typename S>
__global__ void __launch_bounds__(RF_THREADS) k_refine_hub_insert(RefineState a, HubArgs h, uint32_t ntasks) {
    const WT *w = static_cast<const WT *>(a.w);
    S *vals = static_cast<S *>(h.vals);
    for (uint32_t t = blockIdx.x; t < ntasks; t += gridDim.x) {
        const uint32_t k = h.owner[t];
        const uint32_t v = h.hubs[k];
        if (!may_move(a, v)) continue;
        const uint32_t b = a.B[v];
        const uint64_t base = h.pool_off[k], cap = h.pool_off[k + 1] - base;  // absolute pool slots
        const int lg = 63 - __clzll((long long)cap);
        const uint64_t e0 = a.off[v] + (uint64_t)(t - (uint32_t)(h.tasks[k] - h.tasks[0])) * HUB_CHUNK;
        const uint64_t e1 = min(e0 + HUB_CHUNK, a.off[v + 1]);
        for (uint64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            uint32_t u = a.tgt[e];
            if (u != v && a.B[u] == b) ht_add<S>(h.keys + base, vals + base, lg, a.R[u], Score<S>::weight(w, e));
        }
    }
}

// Pass 0: gains (ineligible slots emptied) and each hub's best gain.
// Pass 1 (theta > 0): scores of the candidates near the best gain and each
// hub's best score.  Pass 2: the lowest id among the slots at the best.
template <typename S> __global__ void k_refine_hub_slots(RefineState a, HubArgs h, int pass) {
    S *vals = static_cast<S *>(h.vals);
    for (uint64_t s = h.slot0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < h.slot1;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = h.keys[s];
        if (c == EMPTY) continue;
        const uint32_t k = slot_owner(h, s);
        const uint32_t v = h.hubs[k];
        if (!may_move(a, v)) continue;
        if (pass == 0) {
            S g;
            if (!candidate_gain<S>(a, Score<S>::kv(a, v), c, vals[s], &g)) {
                h.keys[s] = EMPTY;
                continue;
            }
            vals[s] = g;
            atomicMax(&h.best[k], ordered(g));
        } else if (pass == 1) {
            const S gmax = from_ordered<S>(h.best[k]);
            const S g = vals[s];
            if (g >= gmax - Score<S>::SPAN * Score<S>::theta(a)) {
                const S sc = Score<S>::score(a, v, c, g);
                vals[s] = sc;
                atomicMax(&h.best[h.nhubs + k], ordered(sc));
            } else {
                h.keys[s] = EMPTY;
            }
        } else {
            const unsigned long long top = a.theta > 0.0 ? h.best[h.nhubs + k] : h.best[k];
            if (ordered(vals[s]) == top) atomicMin(&h.best_c[k], c);
        }
    }
}

// Each hub's decision: the best candidate (with the stay option of the
// random choice, its score the noise of (v, v)), or v.
template <typename S> __global__ void k_refine_hub_decide(RefineState a, HubArgs h) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < h.nhubs; k += gridDim.x * blockDim.x) {
        const uint32_t v = h.hubs[k];
        if (!may_move(a, v)) {
            a.T[v] = v;
            continue;
        }
        Best<S> best{S(0), v, 0};
        if (h.best_c[k] != EMPTY) {
            best.have = 1;
            best.c = h.best_c[k];
            best.s = from_ordered<S>(a.theta > 0.0 ? h.best[h.nhubs + k] : h.best[k]);
        }
        if (a.theta > 0.0) {
            const S gmax = h.best[k] ? from_ordered<S>(h.best[k]) : S(-INFINITY);
            offer_stay<S>(a, best, v, gmax);
        }
        record(a, v, best);
    }
}

// --------------------------------------------------------- apply, E, flags
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

// E(c, b-c) of each target, G lanes (1 or 32) per joiner: E(v, b-v), less
// twice the edges to c's earlier members and the edges to the wave's other
// joiners of c (after the moves, both have R[u] = c).
template <int G, typename WT>
__global__ void k_refine_ext_update(RefineState a, Slices sl) {
    constexpr uint32_t PER_WARP = 32 / G;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const WT *w = static_cast<const WT *>(a.w);
    const uint32_t total = sl.total();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t0 = warp * PER_WARP; t0 < total; t0 += nwarps * PER_WARP) {  // warp-uniform
        const uint32_t t = t0 + lane / G;
        const uint32_t v = t < total ? sl.at(t) : 0u;
        const bool j = t < total && a.joined[v];
        double old = 0.0, co = 0.0;
        const uint32_t c = j ? a.T[v] : 0u;
        if (j)
            for (uint64_t e = a.off[v] + gl; e < a.off[v + 1]; e += G) {
                uint32_t u = a.tgt[e];
                if (u == v || a.R[u] != c) continue;
                if (a.joined[u]) co += wload(w, e);
                else old += wload(w, e);
            }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            co += __shfl_xor_sync(0xFFFFFFFFu, co, o);
            old += __shfl_xor_sync(0xFFFFFFFFu, old, o);
        }
        if (j && gl == 0) atomicAdd(&a.ext[c], __dsub_rn(__dsub_rn(a.ext[v], __dmul_rn(2.0, old)), co));
    }
}

// The flags (and S_c / 2m) of every refined community that gained members in
// the wave (recomputed from each joiner; same value).
__global__ void k_refine_wc_targets(RefineState a, Slices sl) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < sl.total(); t += gridDim.x * blockDim.x) {
        uint32_t v = sl.at(t);
        if (!a.joined[v]) continue;
        uint32_t c = a.T[v];
        const double tm = two_m_of(a, c);
        a.wc[c] = well_connected(a.ext[c], a.SR[c], a.SB[a.B[c]], tm);
        a.SRf[c] = (float)(a.SR[c] / tm);
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

// The singletons' flags: E(v, b-v) >= K_v (S_b - K_v) / 2m; and K_v / 2m.
__global__ void k_refine_wc_init(RefineState a, uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double tm = two_m_of(a, v);
        if (!(tm > 0.0)) {  // a graph without edges: nothing to join
            a.wc[v] = 0;
            a.SRf[v] = 0.0f;
            continue;
        }
        a.wc[v] = well_connected(a.ext[v], a.SR[v], a.SB[a.B[v]], tm);
        a.SRf[v] = (float)(a.SR[v] / tm);
    }
}

// E(v, b-v) of the vertices of a class list: G lanes (1 or 32) per vertex.
template <int G, typename WT>
__global__ void k_refine_ext_init(const uint64_t *off, const uint32_t *tgt, const WT *w, const uint32_t *B,
                                  double *ext, Slices sl) {
    constexpr uint32_t PER_WARP = 32 / G;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const uint32_t total = sl.total();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t0 = warp * PER_WARP; t0 < total; t0 += nwarps * PER_WARP) {  // warp-uniform
        const uint32_t t = t0 + lane / G;
        const uint32_t v = t < total ? sl.at(t) : 0u;
        double x = 0.0;
        if (t < total) {
            const uint32_t b = B[v];
            for (uint64_t e = off[v] + gl; e < off[v + 1]; e += G) {
                uint32_t u = tgt[e];
                if (u != v && B[u] == b) x += wload(w, e);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        if (t < total && gl == 0) ext[v] = x;
    }
}

// E(v, b-v) of the largest vertices: one block per HUB_CHUNK-edge task of the
// class list's hubs (task prefix `tasks`, owner of each task `owner`),
// each adding its part.
template <typename WT>
__global__ void k_refine_ext_init_tasks(const uint64_t *off, const uint32_t *tgt, const WT *w, const uint32_t *B,
                                        double *ext, const uint32_t *hubs, const uint64_t *tasks,
                                        const uint32_t *owner, uint32_t ntasks) {
    __shared__ double scratch[32];
    for (uint32_t t = blockIdx.x; t < ntasks; t += gridDim.x) {
        const uint32_t k = owner[t];
        const uint32_t v = hubs[k];
        const uint32_t b = B[v];
        const uint64_t e0 = off[v] + (uint64_t)(t - (uint32_t)(tasks[k] - tasks[0])) * HUB_CHUNK;
        const uint64_t e1 = min(e0 + HUB_CHUNK, off[v + 1]);
        double x = 0.0;
        for (uint64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            uint32_t u = tgt[e];
            if (u != v && B[u] == b) x += wload(w, e);
        }
        x = block_sum(x, scratch);
        if (threadIdx.x == 0 && x != 0.0) atomicAdd(&ext[v], x);
    }
}

template <int G, typename WT> void launch_ext_init(const DevGraph &g, const uint32_t *B, double *ext, const Slices &sl,
                                                   cudaStream_t s) {
    if (!sl.total()) return;
    k_refine_ext_init<G, WT><<<grid_for((uint64_t)sl.total() * G, 256, sms(8)), 256, 0, s>>>(
        g.off, g.tgt, static_cast<const WT *>(g.w), B, ext, sl);
    GSP_CHECK_LAUNCH();
}

template <int G, typename WT> void launch_ext_update(const RefineState &a, const Slices &sl, cudaStream_t s) {
    if (!sl.total()) return;
    k_refine_ext_update<G, WT><<<grid_for((uint64_t)sl.total() * G, 256, sms(8)), 256, 0, s>>>(a, sl);
    GSP_CHECK_LAUNCH();
}

template <int G, typename WT, typename S> void launch_group(const RefineState &a, const Slices &sl, cudaStream_t s) {
    if (!sl.total()) return;
    k_refine_decide_group<G, WT, S><<<grid_for((uint64_t)sl.total() * G, RF_THREADS, sms(8)), RF_THREADS, 0, s>>>(
        a, sl);
    GSP_CHECK_LAUNCH();
}

template <typename K> unsigned block_grid(K kernel, size_t smem, uint32_t work) {
    if (!work) return 0;
    unsigned g = resident_grid(reinterpret_cast<const void *>(kernel), RF_THREADS, smem, 8);
    return work < g ? work : g;
}

template <typename WT, typename S>
uint32_t refine_impl(const DevGraph &g, const Classes &cl, const uint32_t *B, uint32_t *R, const double *K, double m,
                     double theta, uint64_t seed, uint32_t pass, const RefineBatch &batch, cudaStream_t s) {
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
    a.SRf = arena().get<float>(n);
    a.ext = arena().get<double>(n);
    a.size = arena().get<uint32_t>(n);
    a.wc = arena().get<uint8_t>(n);
    a.T = arena().get<uint32_t>(n);
    a.targeted = arena().get<uint8_t>(n);
    a.joined = arena().get<uint8_t>(n);
    a.moves = arena().get<unsigned long long>(1);
    a.two_m = 2.0 * m;
    a.gid = batch.gid;
    a.two_m_g = batch.two_m_g;
    a.gvo = batch.gvo;
    a.theta = theta;
    a.pass_key = splitmix64(seed + GOLDEN_GAMMA * ((uint64_t)pass + 1));
    GSP_CUDA(cudaMemsetAsync(SB, 0, sizeof(double) * n, s));
    GSP_CUDA(cudaMemsetAsync(a.targeted, 0, n, s));
    GSP_CUDA(cudaMemsetAsync(a.joined, 0, n, s));
    GSP_CUDA(cudaMemsetAsync(a.moves, 0, sizeof(unsigned long long), s));
    k_refine_init<<<grid_for(n, 256), 256, 0, s>>>(B, K, R, a.SR, a.size, SB, n);
    GSP_CHECK_LAUNCH();
    if (!batch.gid && !(m > 0.0)) {  // edgeless: every vertex stays alone
        arena().release(mk);
        return 0;
    }
    // hubs (the class above the 16384-slot tables): task owners, tables
    const uint32_t nh = cl.cls_count(CLS_HUGE);
    uint32_t *owner = nullptr, *pkeys = nullptr, *best_c = nullptr;
    void *pvals = nullptr;
    unsigned long long *hbest = nullptr;
    const uint32_t *hub_list = cl.list + cl.cls_begin(CLS_HUGE);
    if (nh) {
        const uint64_t ntasks = cl.host_hub_tasks[nh];
        owner = arena().get<uint32_t>(ntasks);
        task_items(cl.hub_tasks, nh, owner, s);
        const size_t sa = align_up(cl.pool_slots, 64);
        pvals = arena().alloc(sizeof(S) * sa);
        pkeys = arena().get<uint32_t>(sa);
        hbest = arena().get<unsigned long long>(2 * (size_t)nh);  // per wave: its hubs only
        best_c = arena().get<uint32_t>(nh);
    }
    // E(v, b-v): a thread per vertex up to 16 edges, a warp up to 2048, a
    // block up to 8192, tasks of HUB_CHUNK edges above (vertices without
    // edges keep 0)
    GSP_CUDA(cudaMemsetAsync(a.ext, 0, sizeof(double) * n, s));
    launch_ext_init<1, WT>(g, B, a.ext, class_range(cl, CLS_G4, CLS_G16), s);
    launch_ext_init<32, WT>(g, B, a.ext, class_range(cl, CLS_G16, CLS_HUGE), s);
    if (nh) {
        const uint32_t ntasks = (uint32_t)cl.host_hub_tasks[nh];
        k_refine_ext_init_tasks<WT><<<grid_for(ntasks, 1, sms(8)), 256, 0, s>>>(
            g.off, g.tgt, static_cast<const WT *>(g.w), B, a.ext, hub_list, cl.hub_tasks, owner, ntasks);
        GSP_CHECK_LAUNCH();
    }
    k_refine_wc_init<<<grid_for(n, 256), 256, 0, s>>>(a, n);
    GSP_CHECK_LAUNCH();

    const int c4[] = {CLS_G4}, c8[] = {CLS_G8}, c16[] = {CLS_G16}, c32[] = {CLS_G32}, c512[] = {CLS_W512},
              cblock[] = {CLS_BLOCK}, cbig[] = {CLS_BIG};
    const int small[] = {CLS_G4, CLS_G8}, rest[] = {CLS_G16, CLS_G32, CLS_W512, CLS_BLOCK, CLS_BIG, CLS_HUGE};
    const int all[] = {CLS_G4, CLS_G8, CLS_G16, CLS_G32, CLS_W512, CLS_BLOCK, CLS_BIG, CLS_HUGE};
    // table sizes: twice the largest degree each class can hold
    constexpr int W32_SLOTS = 2 * GROUP_MAX_LIMIT, W512_SLOTS = 2 * WARP_MAX_LIMIT;
    constexpr uint32_t BLOCK_SLOTS = 2 * BLOCK_MAX_LIMIT, BIG_SLOTS = 2 * BIG_MAX_LIMIT;
    const size_t slot_bytes = sizeof(S) + sizeof(uint32_t);
    const size_t w32_smem = slot_bytes * RF_WARPS * W32_SLOTS, w512_smem = slot_bytes * RF_WARPS * W512_SLOTS;
    const size_t block_smem = slot_bytes * BLOCK_SLOTS, big_smem = slot_bytes * BIG_SLOTS;
    auto kw32 = k_refine_decide_warp<W32_SLOTS, WT, S>;
    auto kw512 = k_refine_decide_warp<W512_SLOTS, WT, S>;
    auto kblk = k_refine_decide_block<WT, S>;
    GSP_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(kw512), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)w512_smem));
    GSP_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(kblk), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)big_smem));
    for (int wv = 0; wv < cl.W; wv++) {
        const Slices sa = make_slices(cl, wv, all, NUM_CLS);
        if (!sa.total()) continue;
        launch_group<4, WT, S>(a, make_slices(cl, wv, c4, 1), s);
        launch_group<8, WT, S>(a, make_slices(cl, wv, c8, 1), s);
        launch_group<16, WT, S>(a, make_slices(cl, wv, c16, 1), s);
        const Slices s32 = make_slices(cl, wv, c32, 1), s512 = make_slices(cl, wv, c512, 1),
                     sblk = make_slices(cl, wv, cblock, 1), sbig = make_slices(cl, wv, cbig, 1);
        if (s32.total()) {
            kw32<<<grid_for(s32.total(), RF_WARPS, sms(8)), RF_THREADS, w32_smem, s>>>(a, s32);
            GSP_CHECK_LAUNCH();
        }
        if (s512.total()) {
            kw512<<<grid_for(s512.total(), RF_WARPS, sms(8)), RF_THREADS, w512_smem, s>>>(a, s512);
            GSP_CHECK_LAUNCH();
        }
        if (sblk.total()) {
            kblk<<<block_grid(kblk, block_smem, sblk.total()), RF_THREADS, block_smem, s>>>(a, sblk, BLOCK_SLOTS);
            GSP_CHECK_LAUNCH();
        }
        if (sbig.total()) {
            kblk<<<block_grid(kblk, big_smem, sbig.total()), RF_THREADS, big_smem, s>>>(a, sbig, BIG_SLOTS);
            GSP_CHECK_LAUNCH();
        }
        const uint32_t hw = cl.count(CLS_HUGE, wv);
        if (hw) {
            // the wave's hubs are consecutive in the class list, and so are
            // their tables and tasks
            const uint32_t r0 = cl.begin(CLS_HUGE, wv) - cl.cls_begin(CLS_HUGE);
            const uint64_t t0 = cl.host_hub_tasks[r0], t1 = cl.host_hub_tasks[r0 + hw];
            HubArgs h;
            h.hubs = hub_list + r0;
            h.nhubs = hw;
            h.pool_off = cl.pool_off + r0;
            h.tasks = cl.hub_tasks + r0;
            h.slot0 = cl.host_pool_off[r0];
            h.slot1 = cl.host_pool_off[r0 + hw];
            h.keys = pkeys;
            h.vals = pvals;
            h.best = hbest;
            h.best_c = best_c;
            uint32_t *wave_owner = arena().get<uint32_t>(t1 - t0);
            task_items(cl.hub_tasks + r0, hw, wave_owner, s);  // hub index within the wave
            h.owner = wave_owner;
            const uint64_t nslots = h.slot1 - h.slot0;
            GSP_CUDA(cudaMemsetAsync(pkeys + h.slot0, 0xFF, sizeof(uint32_t) * nslots, s));
            GSP_CUDA(cudaMemsetAsync(static_cast<S *>(pvals) + h.slot0, 0, sizeof(S) * nslots, s));
            GSP_CUDA(cudaMemsetAsync(hbest, 0, sizeof(unsigned long long) * 2 * hw, s));
            GSP_CUDA(cudaMemsetAsync(best_c, 0xFF, sizeof(uint32_t) * hw, s));
            k_refine_hub_insert<WT, S><<<grid_for(t1 - t0, 1, sms(8)), RF_THREADS, 0, s>>>(a, h, (uint32_t)(t1 - t0));
            GSP_CHECK_LAUNCH();
            const unsigned gs = grid_for(nslots, 256, sms(8));
            for (int p = 0; p < 3; p++) {
                if (p == 1 && !(theta > 0.0)) continue;
                k_refine_hub_slots<S><<<gs, 256, 0, s>>>(a, h, p);
                GSP_CHECK_LAUNCH();
            }
            k_refine_hub_decide<S><<<grid_for(hw, 256), 256, 0, s>>>(a, h);
            GSP_CHECK_LAUNCH();
        }
        const unsigned gv = grid_for(sa.total(), 256, sms(8));
        k_refine_mark<<<gv, 256, 0, s>>>(a, sa);
        GSP_CHECK_LAUNCH();
        k_refine_apply<<<gv, 256, 0, s>>>(a, sa);
        GSP_CHECK_LAUNCH();
        launch_ext_update<1, WT>(a, make_slices(cl, wv, small, 2), s);
        launch_ext_update<32, WT>(a, make_slices(cl, wv, rest, 6), s);
        k_refine_wc_targets<<<gv, 256, 0, s>>>(a, sa);
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
                          double m, double theta, uint64_t seed, uint32_t pass, bool fp64, cudaStream_t s,
                          const RefineBatch &batch) {
    GSP_REQUIRE(theta >= 0.0 && theta == theta, "refine_theta must be >= 0");
    if (fp64) {
        if (g.wt == GSP_W_F64) return refine_impl<double, double>(g, cl, B, R, K, m, theta, seed, pass, batch, s);
        return refine_impl<float, double>(g, cl, B, R, K, m, theta, seed, pass, batch, s);
    }
    if (g.wt == GSP_W_F64) return refine_impl<double, float>(g, cl, B, R, K, m, theta, seed, pass, batch, s);
    return refine_impl<float, float>(g, cl, B, R, K, m, theta, seed, pass, batch, s);
}

}  // namespace gsp
