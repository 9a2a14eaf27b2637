// internal.cuh -- host-side interfaces between the translation units of libgsp.
#pragma once

#include <climits>
#include <vector>

#include "common.cuh"

namespace gsp {

struct DevGraph {
    uint32_t n = 0;
    uint64_t nnz = 0;
    const uint64_t *off = nullptr;
    const uint32_t *tgt = nullptr;
    const void *w = nullptr;  // float (wt == GSP_W_F32) or double (GSP_W_F64)
    int wt = GSP_W_F32;
};

// Launch geometry of the local-moving kernels: grid caps in blocks per SM
// (the kernels are grid-stride loops, so any positive value is correct; the
// result of a sweep does not depend on it).  Set by gsp_set_tuning or chosen
// by gsp_autotune.
struct Tuning {
    int groups = 8;  // k_move_groups (degrees <= group_max)
    int w512 = 3;    // k_move_w512 (group_max+1 .. warp_max)
    int block = 4;   // k_move_block, 4096-slot table (warp_max+1 .. block_max)
    int hub = 4;     // k_hub_insert / k_hub_score (> big_max)
    uint32_t persist_max_vertices = 0;  // graphs up to this size (no hubs) sweep in one launch (0: off)
    // class boundaries (largest degree of each class); each at most what its
    // kernel's table holds (twice as many slots as edges)
    uint32_t group_max = 128, warp_max = 512, block_max = 2048, big_max = 8192;
};
// Largest degree each class's table can hold.
constexpr uint32_t GROUP_MAX_LIMIT = 128, WARP_MAX_LIMIT = 512, BLOCK_MAX_LIMIT = 2048, BIG_MAX_LIMIT = 8192;
// Class boundaries as the classify kernels take them.
struct ClassBounds {
    uint32_t group_max, warp_max, block_max, big_max;
};
Tuning &tuning();

// Degree classes of a vertex list.  Small degrees are served by groups of G
// lanes with a shared-memory table, mid degrees by one block with a
// shared-memory table (4096 slots up to 2048 edges, 16384 slots, one block
// per SM, up to 8192), the largest by the whole grid with tables in a global
// pool.  Each class is further split into W waves (vertex v in wave v mod W):
// the list holds key = class * W + wave in increasing order.
enum { CLS_G4 = 0, CLS_G8, CLS_G16, CLS_G32, CLS_W512, CLS_BLOCK, CLS_BIG, CLS_HUGE, NUM_CLS };
constexpr int MAX_WAVES = 64;
// Edges of one task of the largest class (the hub task prefix of Classes).
constexpr uint32_t HUB_CHUNK = 1024;
constexpr int MAX_REPEATS = 8;  // repeats of a wave (gsp_opts.wave_repeats)

struct Classes {
    uint32_t *list = nullptr;
    uint32_t *dstart = nullptr;  // device copy of start[]
    int W = 1;
    uint32_t start[NUM_CLS * MAX_WAVES + 1] = {0};
    uint64_t *pool_off = nullptr;  // huge class (all waves): hashtable slot offsets
    std::vector<uint64_t> host_pool_off;
    uint64_t pool_slots = 0;
    uint64_t *hub_tasks = nullptr;  // huge class: prefix of edge-chunk counts (count+1)
    std::vector<uint64_t> host_hub_tasks;
    uint32_t *hub_occ_n = nullptr;  // huge class: occupied-slot count of each hub table
    uint32_t begin(int cls, int wave) const { return start[cls * W + wave]; }
    uint32_t count(int cls, int wave) const { return start[cls * W + wave + 1] - start[cls * W + wave]; }
    uint32_t cls_begin(int cls) const { return start[cls * W]; }
    uint32_t cls_count(int cls) const { return start[(cls + 1) * W] - start[cls * W]; }
};

// Build the class/wave lists of g's vertices (degree 0 vertices are left out).
// With gid/gvo (batches of graphs: graph of each vertex, per-graph first
// vertex), a vertex's wave is its index within its graph, mod W.
void classify_vertices(const DevGraph &g, Classes &cl, int waves, cudaStream_t s, const uint32_t *gid = nullptr,
                       const uint64_t *gvo = nullptr);

struct MoveCounters {  // device-side accumulators of one sweep
    double dq;
    unsigned long long moved;
    unsigned long long vertices;
    unsigned long long edges;
    unsigned long long candidates;
    unsigned long long skipped;
    unsigned long long marked;  // edges of moved vertices (neighbour re-marking)
    unsigned long long stalled; // persistent sweep: grid barriers that gave up waiting
    double skipped_gain;        // learned pruning: sum over put-off vertices of P(move) x last gain
};

// Grid-wide barrier state of the persistent sweep kernel (zero at start).
struct GridBar {
    unsigned arrive, gen, err, pad;
};

struct MoveBuffers {
    uint32_t *C = nullptr;       // membership
    double *Sigma = nullptr;     // community totals
    uint32_t *size = nullptr;    // community sizes (singleton rule)
    uint8_t *act = nullptr;      // unprocessed flags
    uint8_t *mark = nullptr;     // re-marks of a frozen-state wave (merged into act after it)
    const double *K = nullptr;
    double *m_dev = nullptr;     // device copy of m
    const uint32_t *gid = nullptr;   // batches: graph of each vertex
    const double *m_g = nullptr;     // batches: m of each graph
    const double *minv_g = nullptr;  // batches: 1/m of each graph
    int lsb = INT_MIN;               // weights in exact integer units of 2^lsb (exact_lsb)
    int repeats = 1;                 // repeats of a wave in a pass's first iteration (wave_repeats_at)
    int no_return_from = 0;          // gsp_opts.no_return_from
    uint32_t *left = nullptr;        // community each vertex last left (no-return rule)
    int *left_it = nullptr;          // iteration of that move, -2 before any in the pass
    int *it_dev = nullptr;           // the sweep's iteration, read by the kernels (set_iteration)
    double *dq_g = nullptr;          // batches: summed gain of each graph in a sweep
    MoveCounters *ctr = nullptr;
    void *pool = nullptr;        // huge-class hashtables
    uint32_t *mv_vtx = nullptr;  // moves decided in the current wave (frozen-state mode)
    uint32_t *mv_cmt = nullptr;
    uint32_t *mv_cnt = nullptr;
    uint32_t *mv_cnts = nullptr; // persistent sweep: one move counter per repeat of a wave
    GridBar *bar = nullptr;      // persistent sweep: grid barrier
    uint32_t *choice = nullptr;  // optional: decision of each vertex (single-sweep API)
    uint32_t *big = nullptr;     // movers whose neighbours all blocks re-mark together
    uint32_t *nbig = nullptr;
    // learned pruning (optional)
    const float *mlp = nullptr;
    float *feat_kept = nullptr;  // K_{i->C_i} / K_i at the vertex's last visit
    float *feat_gain = nullptr;  // scaled best gain at the last visit
    float *last_gain = nullptr;  // best gain at the last visit, in units of Q (not clamped)
    uint8_t *moved_last = nullptr;
    uint8_t *skip = nullptr;     // vertices the predictor put off and no sweep has visited since
    float max_logk = 1.0f;
    // move/no-move trace rows (optional)
    float *trace_x = nullptr;
    uint8_t *trace_y = nullptr;
    uint32_t *trace_cnt = nullptr;
    uint64_t *trace_keys = nullptr;  // optional: (pass, iteration, repeat, vertex) of each row
    uint32_t trace_cap = 0, trace_every = 1, trace_salt = 0;
    int trace_pass = 0, cur_repeat = 0;
};

// Side streams for the independent kernels of a wave (fork/join with
// events); created once per device.
struct SideStreams {
    static constexpr int N = 4;
    cudaStream_t side[N];
    cudaEvent_t fork_ev[64], join_ev[64][N];
    int next = 0;
};
SideStreams &side_streams();

// One wave of a sweep over the active vertices.  sync: frozen-state wave
// (decisions go to the move list; apply_moves() applies them); otherwise
// in-place updates as the paper's parallel loop.
void move_wave(const DevGraph &g, const Classes &cl, MoveBuffers &mb, int wave, bool sync, bool fp64, bool rule,
               bool learned, int iteration, int max_iterations, cudaStream_t s);
void apply_moves(const DevGraph &g, MoveBuffers &mb, uint32_t n_hint, cudaStream_t s);
// A whole frozen-state sweep (all waves) as one cooperative launch, for graphs
// with no vertex above 2048 edges and at most tuning().persist_max_vertices
// vertices.  Returns false (launching nothing) when the graph or the run does
// not qualify.
bool sweep_persistent(const DevGraph &g, const Classes &cl, MoveBuffers &mb, bool fp64, bool rule, int iteration,
                      int max_iterations, cudaStream_t s);

// Scratch of one call taken from a caller's device buffer (gsp_opts.workspace)
// for as long as the object lives; base == NULL leaves the internal workspace
// in use.  workspace_peak(): most bytes the current workspace held at once
// since the call began.
struct UserWorkspace {
    struct Impl;
    Impl *impl = nullptr;
    UserWorkspace(void *base, size_t bytes);
    ~UserWorkspace();
    UserWorkspace(const UserWorkspace &) = delete;
    UserWorkspace &operator=(const UserWorkspace &) = delete;
};
size_t workspace_peak();

// driver.cu helpers shared with the batched driver
int wave_repeats_at(const MoveBuffers &mb, int iteration);  // runs of each wave in that iteration
// gsp_opts.waves, with 0 read as the mode's default: 17 frozen-state waves,
// 64 in-place ones
int effective_waves(int waves, bool sync);
void sweep_launches(const DevGraph &g, const Classes &cl, MoveBuffers &mb, bool sync, bool fp64, bool rule,
                    bool pruned, int it, int max_it, const uint32_t *wave_n, bool reset_ctr, cudaStream_t s);
bool graphs_enabled();
bool persistent_enabled();
cudaStream_t capture_stream();
void alloc_move_state(MoveBuffers &mb, uint32_t n);
void reset_left(MoveBuffers &mb, uint32_t n, cudaStream_t s);
// Store the iteration of the next sweep where its kernels read it; called
// before each sweep's launches or graph replay (a captured graph keeps the
// kernel arguments of its capture).
void set_iteration(MoveBuffers &mb, int iteration, cudaStream_t s);
void alloc_pool(MoveBuffers &mb, const Classes &cl, cudaStream_t s);
double sweep_bytes(const MoveCounters &h, int wt);
cudaEvent_t pool_event();
void reset_event_pool();
void check_graph(const uint64_t *off, const uint32_t *tgt, const float *w, uint32_t n, uint64_t nnz, cudaStream_t s);
void check_opts(const gsp_opts &o);
DevGraph make_graph(const uint64_t *off, const uint32_t *tgt, const void *w, int wt, uint32_t n, uint64_t nnz);

struct LouvainTimers;

// One GSP-Louvain run (Algorithm 1) on a validated graph, on stream s; the
// body of gsp_louvain (trace: optional visit recording of gsp_louvain_trace).
struct TraceSpec;
void louvain_run(const DevGraph &g0, const gsp_opts &o, uint32_t *membership, double *modularity_out,
                 gsp_stats *st, cudaStream_t s, const TraceSpec *trace = nullptr);

// Batched GSP-Louvain on the concatenated graphs (h_gvo0: host vertex offsets
// of the num_graphs graphs), per-graph modularity into q_out (device); the
// body of gsp_louvain_batched.  check_batch validates its arguments.
void check_batch(uint32_t num_graphs, const uint64_t *h_gvo0, uint32_t n, const gsp_opts &o);
void louvain_batched_run(const DevGraph &g0, uint32_t num_graphs, const uint64_t *h_gvo0, const gsp_opts &o,
                         uint32_t *membership, double *q_out, gsp_stats *st, cudaStream_t caller);

// Leiden refinement (Section 3.5) of the bound membership B (ids < n) into R
// (each refined community named by one of its vertices), in the waves of
// `cl` (built for g), scores in float64 (fp64) or float32; returns the number
// of vertices that joined another refined community.
// Batches: graph of each vertex, 2m of each graph (device), first vertex of
// each graph (device); all NULL for one graph.
struct RefineBatch {
    const uint32_t *gid = nullptr;
    const double *two_m_g = nullptr;
    const uint64_t *gvo = nullptr;
};
uint32_t refine_partition(const DevGraph &g, const Classes &cl, const uint32_t *B, uint32_t *R, const double *K,
                          double m, double theta, uint64_t seed, uint32_t pass, bool fp64, cudaStream_t s,
                          const RefineBatch &batch = RefineBatch());
// Sigma[c] = sum of K over the vertices of community c, size[c] = their
// count (C ids < n).
void sigma_from_membership(const uint32_t *C, const double *K, double *Sigma, uint32_t *size, uint32_t n,
                           cudaStream_t s);
// C_next[R[i]] = B[i]: each super-vertex of the refined partition R (dense)
// starts the next pass in the bound community B (dense) of its members.
void scatter_bound(const uint32_t *R, const uint32_t *B, uint32_t *C_next, uint32_t n, cudaStream_t s);

// Split (Algorithms 2, 3): labels = smallest vertex of the component.
void split_labels(const DevGraph &g, const Classes &cl, const uint32_t *C, int mode, uint32_t *labels,
                  cudaStream_t s);

// Renumber: C_dense[v] = rank of C[v] among the distinct ids; returns k.
uint32_t renumber(uint32_t n, const uint32_t *C, uint32_t *C_dense, cudaStream_t s);

// Aggregation (Algorithm 5) into out (offsets k+1, targets/weights nnz); returns nnz''.
// sorted: rows in increasing target order (the canonical form); otherwise
// each row's entries come in table order.  lsb_cache (optional) carries the
// exponent of the exact fixed-point unit of the weights between the passes
// of one run (INT_MAX: not known yet; the weights of every aggregated graph
// are sums of the input weights, so the input's unit and bound hold for all).
uint64_t aggregate(const DevGraph &g, const uint32_t *Cd, uint32_t k, uint64_t *out_off, uint32_t *out_tgt,
                   double *out_w, cudaStream_t s, bool sorted = true, int *lsb_cache = nullptr);

// Exponent lsb such that every weight of g is a multiple of 2^lsb and the
// total weight is below 2^52 * 2^lsb, or INT_MIN (then sums stay float64).
// Aggregated graphs carry sums of the input weights, so the input's lsb holds
// for every pass of a run.
int exact_lsb(const DevGraph &g, cudaStream_t s);

// K and m (m also written to *m_dev when non-null); returns m.  lsb: the
// graph's exact_lsb (INT_MIN: float64 sums).
double vertex_weights(const DevGraph &g, double *K, double *m_dev, cudaStream_t s, int lsb = INT_MIN);
double modularity(const DevGraph &g, const uint32_t *C, cudaStream_t s, int lsb = INT_MIN);
double modularity_scratch(const DevGraph &g, const uint32_t *C, double *Sig, double *acc, uint32_t *longlist,
                          uint32_t *nlong, cudaStream_t s);
unsigned long long count_out_of_range(const uint32_t *x, uint64_t n, uint32_t bound, unsigned long long *counter,
                                      cudaStream_t s);
void check_csr(const uint64_t *off, const uint32_t *tgt, uint32_t n, uint64_t nnz, unsigned long long *counter,
               cudaStream_t s);
uint32_t count_disconnected(const DevGraph &g, const uint32_t *C, uint8_t *flags, cudaStream_t s);
void lookup(uint32_t n_top, uint32_t *C_top, const uint32_t *C_pass, cudaStream_t s);
// Renumber membership by smallest vertex id (final numbering); returns k.
uint32_t canonical_numbering(uint32_t n, uint32_t *C, cudaStream_t s);

void iota_u32(uint32_t *p, uint32_t n, cudaStream_t s);
// out[k] = the item that owns task prefix[0] + k of a chunked work split
// (tasks [prefix[i], prefix[i+1]) belong to item i); out holds
// prefix[nitems] - prefix[0] entries.  Replaces a per-task search of prefix.
void task_items(const uint64_t *prefix, uint32_t nitems, uint32_t *out, cudaStream_t s);

// MLP (mlp.cu)
constexpr int MLP_IN = 6, MLP_H = 32;
constexpr int MLP_PARAMS = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;

// Inputs of the learned pruning predictor for vertex i, from the state its
// last visit left: log-degree, log-weighted-degree (normalised by the pass
// maximum), fraction of K_i kept inside its community, last scaled gain,
// whether it moved, and the iteration's position in the pass.
__device__ __forceinline__ void predictor_features(uint32_t deg, double Ki, float kept, float gain, uint8_t moved,
                                                   float max_logk, float iter_frac, float *x) {
    x[0] = log1pf((float)deg) * (1.0f / 16.0f);
    x[1] = log1pf((float)Ki) / max_logk;
    x[2] = kept;
    x[3] = gain;
    x[4] = (float)moved;
    x[5] = iter_frac;
}

// Learned pruning before a sweep: active vertices whose predicted move
// probability is below threshold are marked processed and put off
// (mb.skip); a later visit (a neighbour's move re-marks them) clears that.
void mlp_prune(const DevGraph &g, MoveBuffers &mb, int iteration, int max_iterations, float threshold,
               cudaStream_t s);
// Before a plain sweep: every vertex still put off is unprocessed again, so
// that the plain sweep reconsiders it.
void mlp_unskip(const DevGraph &g, MoveBuffers &mb, cudaStream_t s);

__device__ __forceinline__ int ceil_log2(uint32_t x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// Position of the q-th (from 0) set bit of m; q < popcount(m).
__device__ __forceinline__ int select_bit(unsigned m, int q) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const unsigned low = m & ((1u << w) - 1u);
        const int c = __popc(low);
        if (q >= c) {
            q -= c;
            m >>= w;
            pos += w;
        } else {
            m = low;
        }
    }
    return pos;
}


// Open-addressing insert of (c, w) with linear probing: the key is claimed
// with atomicCAS, the value accumulated with atomicAdd.  The table holds
// 2^logcap slots, more than the number of distinct keys inserted, so a free
// slot always exists; the probe loop still stops after one full cycle.
// Returns 1 when c was new to the table, 0 when it was present, -1 when the
// table was full (which the sizing rules out).
template <typename V>
__device__ __forceinline__ int ht_add(uint32_t *keys, V *vals, int logcap, uint32_t c, V w) {
    uint32_t mask = (1u << logcap) - 1u;
    uint32_t h = logcap ? (hash32(c) >> (32 - logcap)) : 0u;
    volatile uint32_t *vk = keys;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        uint32_t k = vk[h];
        if (k == c) { atomicAdd(&vals[h], w); return 0; }
        if (k == EMPTY) {
            uint32_t old = atomicCAS(&keys[h], EMPTY, c);
            if (old == EMPTY) { atomicAdd(&vals[h], w); return 1; }
            if (old == c) { atomicAdd(&vals[h], w); return 0; }
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// Global-table insert that claims with atomicCAS first (one round trip when
// the home slot is free or already holds c); reports the slot used.
template <typename V>
__device__ __forceinline__ int ht_add_slot_cas(uint32_t *keys, V *vals, int logcap, uint32_t c, V w, uint32_t *slot) {
    uint32_t mask = (1u << logcap) - 1u;
    uint32_t h = logcap ? (hash32(c) >> (32 - logcap)) : 0u;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        uint32_t old = atomicCAS(&keys[h], EMPTY, c);
        if (old == EMPTY || old == c) {
            atomicAdd(&vals[h], w);
            *slot = h;
            return old == EMPTY;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// As ht_add, also reporting the slot used (for occupied-slot lists).
template <typename V>
__device__ __forceinline__ int ht_add_slot(uint32_t *keys, V *vals, int logcap, uint32_t c, V w, uint32_t *slot) {
    uint32_t mask = (1u << logcap) - 1u;
    uint32_t h = logcap ? (hash32(c) >> (32 - logcap)) : 0u;
    volatile uint32_t *vk = keys;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        uint32_t k = vk[h];
        if (k == c) { atomicAdd(&vals[h], w); *slot = h; return 0; }
        if (k == EMPTY) {
            uint32_t old = atomicCAS(&keys[h], EMPTY, c);
            if (old == EMPTY || old == c) { atomicAdd(&vals[h], w); *slot = h; return old == EMPTY; }
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// Combine-then-publish: the block's shared table (2^slog slots, whose
// occupied slots are listed in socc[0..*s_nocc)) is merged into a global
// table (2^glog slots); keys new to the global table append their slot to
// occ (count in *occ_n).  The shared table is left empty.  Every thread of
// the block must call this.
constexpr uint32_t PUBLISH_MAX = 2048;  // most distinct keys one block publishes at once

template <typename V>
__device__ void publish_block_table(uint32_t *skeys, V *svals, uint16_t *socc, uint32_t *s_nocc, uint32_t *gkeys,
                                    V *gvals, int glog, uint32_t *occ, uint32_t *occ_n) {
    __shared__ uint32_t s_newslot[PUBLISH_MAX];
    __shared__ uint32_t s_new, s_base;
    __syncthreads();
    if (threadIdx.x == 0) s_new = 0;
    __syncthreads();
    uint32_t n = min(*s_nocc, PUBLISH_MAX);
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
        uint32_t s = socc[t];
        uint32_t slot;
        if (ht_add_slot_cas<V>(gkeys, gvals, glog, skeys[s], svals[s], &slot) == 1)
            s_newslot[atomicAdd(&s_new, 1u)] = slot;
        skeys[s] = EMPTY;
        svals[s] = V(0);
    }
    __syncthreads();
    // one reservation per block in the global occupied list
    if (threadIdx.x == 0) s_base = s_new ? atomicAdd(occ_n, s_new) : 0;
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < s_new; t += blockDim.x) occ[s_base + t] = s_newslot[t];
    __syncthreads();
    if (threadIdx.x == 0) *s_nocc = 0;
    __syncthreads();
}

// Insert into a shared table, listing slots new to it in socc.
template <typename V>
__device__ __forceinline__ void smem_add(uint32_t *skeys, V *svals, int slog, uint16_t *socc, uint32_t *s_nocc,
                                         uint32_t c, V w) {
    uint32_t slot;
    if (ht_add_slot<V>(skeys, svals, slog, c, w, &slot) == 1) socc[atomicAdd(s_nocc, 1u)] = (uint16_t)slot;
}

// Exact sums of edge weights.  They are accumulated either as float64
// (AV = double) or, when every weight of the graph is a multiple of 2^lsb and
// the total weight is below 2^52 units (exact_lsb), as 64-bit integers in
// units of 2^lsb (AV = unsigned long long): a float32 or float64 weight
// becomes its integer mantissa shifted by its exponent, with no floating-point
// arithmetic (float64 is a narrow pipe on this GPU), and a shared-memory
// integer atomic add is a single native operation.  Both sum exactly, so they
// give identical results.
__device__ __forceinline__ unsigned long long units_of(float x, int lsb) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFFu);
    const unsigned long long m = e ? ((b & 0x7FFFFFu) | 0x800000u) : (b & 0x7FFFFFu);
    const int sh = (e ? e : 1) - 150 - lsb;  // x = m * 2^(sh + lsb); sh >= -ctz(m)
    return sh >= 0 ? m << sh : m >> -sh;
}
__device__ __forceinline__ unsigned long long units_of(double x, int lsb) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FFu);
    const unsigned long long m = e ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : (b & 0xFFFFFFFFFFFFFull);
    const int sh = (e ? e : 1) - 1075 - lsb;
    return sh >= 0 ? m << sh : m >> -sh;
}
template <typename AV> struct Acc;
template <> struct Acc<double> {
    template <typename WT> __device__ static double of(WT x, int) { return (double)x; }
    __device__ static double val(double v, int) { return v; }
};
template <> struct Acc<unsigned long long> {
    template <typename WT> __device__ static unsigned long long of(WT x, int lsb) { return units_of(x, lsb); }
    // v < 2^52: the conversion is exact, and so is the power-of-two scaling
    // done on the exponent field (lsb >= -1000 keeps the result normal)
    __device__ static double val(unsigned long long v, int lsb) {
        if (!v) return 0.0;
        const double d = (double)v;
        return __longlong_as_double(__double_as_longlong(d) + ((long long)lsb << 52));
    }
};

// Exponent of the lowest set bit of a positive finite weight (INT_MIN for a
// value that is not, INT_MAX for zero).
__device__ __forceinline__ int low_bit_exp(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    if ((b >> 31) || e == 0xFFu) return INT_MIN;
    if (e == 0) return m ? -149 + (__ffs((int)m) - 1) : INT_MAX;
    return (int)e - 150 + (__ffs((int)(m | 0x800000u)) - 1);
}
__device__ __forceinline__ int low_bit_exp(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FFu);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if ((b >> 63) || e == 0x7FF) return INT_MIN;
    if (e == 0) return m ? -1074 + (__ffsll((long long)m) - 1) : INT_MAX;
    return e - 1075 + (__ffsll((long long)(m | (1ull << 52))) - 1);
}

// Chunked work over items (hubs, communities) of different sizes: task ids
// [prefix[i], prefix[i+1]) belong to item i; returns the item of a task.
__device__ __forceinline__ uint32_t task_item(const uint64_t *prefix, uint32_t nitems, uint64_t task) {
    uint32_t lo = 0, hi = nitems - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= task) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace gsp
