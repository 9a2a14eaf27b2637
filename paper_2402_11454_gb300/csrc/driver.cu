// driver.cu -- GSP-Louvain pass loop (Algorithm 1), the device workspace,
// error reporting and the C ABI of include/gsp.h for the phase entry points.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace gsp {

// ---------------------------------------------------------------- errors
static thread_local char g_err[512] = "";
static unsigned long long g_launches = 0;
void count_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// ------------------------------------------------------------- workspace
// Chunked bump allocator: chunks are cudaMalloc'd on demand and kept for the
// next call, so a repeated call of the same size allocates nothing.
struct ChunkArena {
    struct Chunk {
        char *base;
        size_t cap;
    };
    std::vector<Chunk> chunks;
    size_t cur = 0, top = 0;
    size_t peak = 0;       // most bytes in use since the last reset (chunk tails skipped count as used)
    bool fixed = false;    // a caller's workspace: one chunk, never grown
    size_t in_use() const {
        size_t b = top;
        for (size_t k = 0; k < cur && k < chunks.size(); k++) b += chunks[k].cap;
        return b;
    }
    void *alloc(size_t bytes) {
        bytes = align_up(bytes ? bytes : 1, 256);
        while (cur < chunks.size()) {
            if (top + bytes <= chunks[cur].cap) {
                void *p = chunks[cur].base + top;
                top += bytes;
                peak = std::max(peak, in_use());
                return p;
            }
            if (fixed) {
                set_error("caller workspace too small: %zu of %zu bytes used, %zu more requested", top,
                          chunks[cur].cap, bytes);
                throw Error{GSP_ERR_CAPACITY};
            }
            cur++;
            top = 0;
        }
        // chunks double from 64 MB up to 4 GB; a larger request gets a chunk
        // of its own size (doubling without a cap reserved about twice the
        // peak of an R-MAT scale-26 run)
        size_t last = chunks.empty() ? 0 : chunks.back().cap;
        size_t grow = std::min<size_t>(std::max<size_t>(last * 2, (size_t)64 << 20), (size_t)4 << 30);
        size_t sz = std::max(bytes, grow);
        char *p = nullptr;
        cudaError_t e = cudaMalloc(&p, sz);
        if (e != cudaSuccess && sz > bytes) {
            cudaGetLastError();
            sz = bytes;
            e = cudaMalloc(&p, sz);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("device workspace: cudaMalloc(%zu) failed: %s", sz, cudaGetErrorString(e));
            throw Error{GSP_ERR_NOMEM};
        }
        chunks.push_back({p, sz});
        cur = chunks.size() - 1;
        top = bytes;
        peak = std::max(peak, in_use());
        return p;
    }
    size_t mark() const { return (cur << 40) | top; }
    void release(size_t m) {
        cur = m >> 40;
        top = m & ((1ull << 40) - 1);
    }
    void reset() { cur = top = peak = 0; }
    void free_all() {
        for (auto &k : chunks) cudaFree(k.base);
        chunks.clear();
        reset();
    }
};

static ChunkArena g_work[16], g_io[16];
static int cur_dev() {
    int d = 0;
    cudaGetDevice(&d);
    return d & 15;
}

// A call given a caller workspace (gsp_opts.workspace) takes all its scratch
// from it; the internal workspace is left alone.
static thread_local ChunkArena *g_user_ws = nullptr;
struct UserWorkspace::Impl {
    ChunkArena ws;
};
UserWorkspace::UserWorkspace(void *base, size_t bytes) {
    if (!base) return;
    GSP_REQUIRE(bytes >= 256 && (reinterpret_cast<uintptr_t>(base) & 255) == 0,
                "workspace must be 256-byte aligned and hold at least 256 bytes");
    impl = new Impl;
    impl->ws.chunks.push_back({static_cast<char *>(base), bytes & ~(size_t)255});
    impl->ws.fixed = true;
    g_user_ws = &impl->ws;
}
UserWorkspace::~UserWorkspace() {
    if (!impl) return;
    if (g_user_ws == &impl->ws) g_user_ws = nullptr;
    impl->ws.chunks.clear();  // the caller's memory: never freed here
    delete impl;
}

static Arena g_work_facade, g_io_facade;
Arena &arena() { return g_work_facade; }
Arena &io_arena() { return g_io_facade; }
static ChunkArena &backing(const Arena *a) {
    if (a == &g_io_facade) return g_io[cur_dev()];
    return g_user_ws ? *g_user_ws : g_work[cur_dev()];
}
size_t workspace_peak() { return backing(&g_work_facade).peak; }
void *Arena::alloc(size_t bytes) { return backing(this).alloc(bytes); }
size_t Arena::mark() { return backing(this).mark(); }
void Arena::release(size_t m) { backing(this).release(m); }
void Arena::reset() { backing(this).reset(); }
void Arena::free_all() { backing(this).free_all(); }

// ---------------------------------------------------------- small kernels
__global__ void k_fill_u32_(uint32_t *p, uint32_t n, uint32_t v) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_community_sizes(const uint32_t *__restrict__ C, uint32_t n, uint32_t *size) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(size + C[i], 1u);
}

// Input checks.  Offsets: non-decreasing from 0 to nnz (checked first: the
// entry kernel below trusts them).  Entries: targets < n, weights finite and
// > 0.  Symmetry (Section 3: G is undirected, w_ij = w_ji): every stored
// entry (i, j, w) with i != j hashes the unordered pair and the weight's bits
// to 64 bits and adds the hash (and 1) when i < j, subtracts it (and 1) when
// i > j, modulo 2^64.  A symmetric CSR stores the same multiset of (pair,
// weight) on both sides, so both differences end at 0; an asymmetric one
// passes only if its hash difference vanishes by chance.  The hash is the
// MurmurHash3 64-bit finaliser (Appleby) of the pair with the weight's bits
// mixed in by a multiplication with the 64-bit golden ratio.
struct GraphCheck {
    unsigned long long bad;    // offset, target and weight violations
    unsigned long long below;  // entries below the diagonal (i < j)
    unsigned long long cntd;   // entries below minus above, modulo 2^64
    unsigned long long fpd;    // hashes below minus above, modulo 2^64
};

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

struct CheckAcc {
    unsigned long long bad = 0, below = 0, cntd = 0, fpd = 0;
    // entry (i, j) of weight x (has_w = 0: no weights to check)
    __device__ void entry(uint32_t i, uint32_t j, float x, bool has_w, uint32_t n) {
        uint32_t wb = 0;
        if (has_w) {
            if (!(x > 0.0f) || isinf(x)) bad++;
            wb = __float_as_uint(x);
        }
        if (j >= n) { bad++; return; }
        if (i == j) return;
        const uint64_t key = ((uint64_t)min(i, j) << 32) | max(i, j);
        const uint64_t h = fmix64(key ^ ((uint64_t)wb * 0x9E3779B97F4A7C15ull));
        if (i < j) {
            fpd += h;
            cntd++;
            below++;
        } else {
            fpd -= h;
            cntd--;
        }
    }
    __device__ void flush(GraphCheck *g) {
        unsigned long long v[4] = {bad, below, cntd, fpd};
        unsigned long long *dst[4] = {&g->bad, &g->below, &g->cntd, &g->fpd};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const unsigned long long t = warp_sum(v[k]);
            if ((threadIdx.x & 31) == 0 && t) atomicAdd(dst[k], t);
        }
    }
};

__global__ void k_check_offsets(const uint64_t *__restrict__ off, uint32_t n, uint64_t nnz, GraphCheck *g) {
    unsigned long long b = 0;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint64_t i = tid; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (off[i + 1] < off[i]) b++;
    if (tid == 0 && (off[0] != 0 || off[n] != nnz)) b++;
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&g->bad, b);
}

constexpr int CHECK_UNROLL = 4;  // entries a thread loads before checking them

// Entry checks, edge-parallel, in chunks of CHECK_CHUNK consecutive entries
// whose first rows a bisection kernel finds ahead; warp w takes chunks w,
// w + warps, ..., its lanes consecutive entries (coalesced loads whatever the
// row lengths; a lane's next entry lies 32 entries on, so its row search
// moves a row or so).  Dealing the chunks round the warps spreads the
// stretches of empty rows, where the searches run longest, over all SMs.
constexpr uint64_t CHECK_CHUNK = 1024;

__global__ void k_chunk_rows(const uint64_t *__restrict__ off, uint32_t n, uint64_t nchunks, uint32_t *rows) {
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < nchunks;
         c += (uint64_t)gridDim.x * blockDim.x)
        rows[c] = row_of(off, n, c * CHECK_CHUNK);
}

__global__ void __launch_bounds__(256, 6) k_check_entries(const uint64_t *__restrict__ off,
                                                          const uint32_t *__restrict__ tgt,
                                                          const float *__restrict__ w, uint32_t n, uint64_t nnz,
                                                          const uint32_t *__restrict__ chunk_rows,
                                                          uint64_t nchunks, GraphCheck *g) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    CheckAcc a;
    const bool has_w = w != nullptr;
    for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += warps) {
        const uint64_t c0 = c * CHECK_CHUNK, c1 = min(c0 + CHECK_CHUNK, nnz);
        uint32_t r = __ldg(chunk_rows + c);
        for (uint64_t p = c0 + lane; p < c1; p += 32ull * CHECK_UNROLL) {
            uint32_t t[CHECK_UNROLL];
            float x[CHECK_UNROLL];
#pragma unroll
            for (int k = 0; k < CHECK_UNROLL; k++) {
                const uint64_t q = p + 32ull * k;
                t[k] = q < c1 ? __ldg(tgt + q) : 0u;
                x[k] = (has_w && q < c1) ? __ldg(w + q) : 1.0f;
            }
#pragma unroll
            for (int k = 0; k < CHECK_UNROLL; k++) {
                const uint64_t q = p + 32ull * k;
                if (q < c1) {
                    r = row_from(off, n, q, r);
                    a.entry(r, t[k], x[k], has_w, n);
                }
            }
        }
    }
    a.flush(g);
}

void check_graph(const uint64_t *off, const uint32_t *tgt, const float *w, uint32_t n, uint64_t nnz,
                 cudaStream_t s) {
    size_t mk = arena().mark();
    GraphCheck *d = arena().get<GraphCheck>(1);
    GraphCheck h;
    GSP_CUDA(cudaMemsetAsync(d, 0, sizeof(GraphCheck), s));
    k_check_offsets<<<grid_for(n, 256), 256, 0, s>>>(off, n, nnz, d);
    GSP_CHECK_LAUNCH();
    GSP_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    if (h.bad) arena().release(mk);
    GSP_REQUIRE(h.bad == 0, "invalid graph: offsets must rise from 0 to nnz (%llu violations)", h.bad);
    if (nnz) {
        const uint64_t nchunks = (nnz + CHECK_CHUNK - 1) / CHECK_CHUNK;
        uint32_t *chunk_rows = arena().get<uint32_t>(nchunks);
        k_chunk_rows<<<grid_for(nchunks, 256), 256, 0, s>>>(off, n, nchunks, chunk_rows);
        GSP_CHECK_LAUNCH();
        const unsigned grid = std::min(grid_for(nchunks, 8, sms(8)),
                                       resident_grid((const void *)k_check_entries, 256, 0, 6));
        k_check_entries<<<grid, 256, 0, s>>>(off, tgt, w, n, nnz, chunk_rows, nchunks, d);
        GSP_CHECK_LAUNCH();
        GSP_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
    }
    arena().release(mk);
    GSP_REQUIRE(h.bad == 0, "invalid graph: %llu violations (targets must be < n, weights finite and > 0)", h.bad);
    if (h.cntd != 0 || h.fpd != 0) {
        set_error("graph is not symmetric: %llu entries below the diagonal, %llu above, or their (pair, weight) "
                  "multisets differ (Section 3 needs w_ij = w_ji for every stored entry)",
                  h.below, h.below - h.cntd);
        throw Error{GSP_ERR_NOT_SYMMETRIC};
    }
}

__global__ void k_check_ids(const uint32_t *__restrict__ C, uint32_t n, uint32_t bound, unsigned long long *bad) {
    unsigned long long b = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (C[i] >= bound) b++;
    if (b) atomicAdd(bad, b);
}

// Caller-supplied ids must be < bound (community ids index arrays of that size).
static void check_ids(const uint32_t *C, uint32_t n, uint32_t bound, const char *what, cudaStream_t s) {
    size_t mk = arena().mark();
    unsigned long long *bad = arena().get<unsigned long long>(1);
    GSP_CUDA(cudaMemsetAsync(bad, 0, sizeof(*bad), s));
    k_check_ids<<<grid_for(n, 256), 256, 0, s>>>(C, n, bound, bad);
    GSP_CHECK_LAUNCH();
    unsigned long long h = 0;
    GSP_CUDA(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    GSP_REQUIRE(h == 0, "%s: %llu ids out of range (must be < %u)", what, h, bound);
}

// ------------------------------------------------------------ move loop
struct EventPool {
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    cudaEvent_t get() {
        if (used == ev.size()) {
            cudaEvent_t e;
            GSP_CUDA(cudaEventCreate(&e));
            ev.push_back(e);
        }
        return ev[used++];
    }
    void reset() { used = 0; }
};
static EventPool g_events;
cudaEvent_t pool_event() { return g_events.get(); }
void reset_event_pool() { g_events.reset(); }

struct MoveLoopResult {
    int iterations;
    uint64_t vertices, edges, candidates, skipped;
    double bytes;     // algorithmic bytes of the sweep kernels
    float ms_kernels; // their device time
};

// Algorithmic bytes of one sweep (per processed vertex: list entry 4, flag 1,
// C_i 4, two offsets 16, K_i 8, Sigma_d 8; per scanned edge: target 4, weight
// 4 or 8, C_j 4; per candidate community: Sigma_c 8; per move: move-list
// entry 8 written and read, C_i 4, two Sigma and two size updates 24, plus
// one flag byte per neighbour).
double sweep_bytes(const MoveCounters &h, int wt) {
    double wb = wt == GSP_W_F64 ? 8.0 : 4.0;
    return 41.0 * h.vertices + (8.0 + wb) * h.edges + 8.0 * h.candidates + 44.0 * h.moved + 1.0 * h.marked;
}

struct PruneCtx {
    bool learned = false;
    int full_every = 4;
    float threshold = 0.5f;
};

// One sweep: cl.W waves, each run wave_repeats_at(it) times (mb.repeats in
// the first iteration of a pass, once afterwards).  In frozen-state mode the
// moves of each repeat are applied (and the movers' neighbours re-marked)
// before the next; a repeat takes the vertices of the wave that the earlier
// repeats re-marked, on the state those moves left.
int effective_waves(int waves, bool sync) { return waves > 0 ? waves : (sync ? 17 : 64); }

int wave_repeats_at(const MoveBuffers &mb, int it) { return (it == 0 && mb.repeats > 1) ? mb.repeats : 1; }

void sweep_launches(const DevGraph &g, const Classes &cl, MoveBuffers &mb, bool sync, bool fp64, bool rule,
                    bool pruned, int it, int max_it, const uint32_t *wave_n, bool reset_ctr, cudaStream_t s) {
    if (reset_ctr) GSP_CUDA(cudaMemsetAsync(mb.ctr, 0, sizeof(MoveCounters), s));
    const int R = wave_repeats_at(mb, it);
    for (int wv = 0; wv < cl.W; wv++) {
        if (!wave_n[wv]) continue;
        for (int r = 0; r < R; r++) {
            mb.cur_repeat = r;
            if (sync) GSP_CUDA(cudaMemsetAsync(mb.mv_cnt, 0, sizeof(uint32_t), s));
            move_wave(g, cl, mb, wv, sync, fp64, rule, pruned, it, max_it, s);
            if (sync) apply_moves(g, mb, wave_n[wv], s);
        }
        mb.cur_repeat = 0;
    }
}

bool graphs_enabled() {
    const char *e = getenv("GSP_NO_GRAPH");
    return !(e && e[0] == '1');
}

bool persistent_enabled() { return tuning().persist_max_vertices > 0; }

// louvainMove (Algorithm 4): iterate sweeps until the summed gain of a sweep
// is <= tau or max_iterations is reached.  The launches of a sweep do not
// change within a pass: the first sweep runs directly, the second is captured
// into a CUDA graph that the following sweeps replay.
// Library-owned stream for graph capture (the caller's stream may be the
// legacy default stream, which cannot be captured).
cudaStream_t capture_stream() {
    static cudaStream_t cs[16];
    static bool made[16] = {false};
    int d = cur_dev();
    if (!made[d]) {
        GSP_CUDA(cudaStreamCreateWithFlags(&cs[d], cudaStreamNonBlocking));
        made[d] = true;
    }
    return cs[d];
}

static MoveLoopResult move_loop_on(const DevGraph &g, const Classes &cl, MoveBuffers &mb, double tau, int max_it,
                                   bool sync, bool fp64, bool rule, const PruneCtx &pr, cudaStream_t s);

static MoveLoopResult move_loop(const DevGraph &g, const Classes &cl, MoveBuffers &mb, double tau, int max_it,
                                bool sync, bool fp64, bool rule, const PruneCtx &pr, cudaStream_t caller) {
    cudaStream_t s = capture_stream();
    cudaEvent_t in = g_events.get(), out = g_events.get();
    GSP_CUDA(cudaEventRecord(in, caller));
    GSP_CUDA(cudaStreamWaitEvent(s, in, 0));
    MoveLoopResult r = move_loop_on(g, cl, mb, tau, max_it, sync, fp64, rule, pr, s);
    GSP_CUDA(cudaEventRecord(out, s));
    GSP_CUDA(cudaStreamWaitEvent(caller, out, 0));
    return r;
}

static MoveLoopResult move_loop_on(const DevGraph &g, const Classes &cl, MoveBuffers &mb, double tau, int max_it,
                                   bool sync, bool fp64, bool rule, const PruneCtx &pr, cudaStream_t s) {
    MoveLoopResult r{0, 0, 0, 0, 0, 0.0, 0.0f};
    MoveCounters h;
    cudaEvent_t e0 = g_events.get(), e1 = g_events.get();
    uint32_t wave_n[MAX_WAVES];
    for (int wv = 0; wv < cl.W; wv++) {
        wave_n[wv] = 0;
        for (int c = 0; c < NUM_CLS; c++) wave_n[wv] += cl.count(c, wv);
    }
    // every per-iteration value the kernels need (the iteration itself, the
    // features' iteration position, trace sampling) comes from the device
    // scalar set before each replay, so every run replays its graph
    const bool use_graph = graphs_enabled();
    bool use_persist = sync && persistent_enabled();  // small graphs: one launch per sweep
    cudaGraphExec_t exec = nullptr;
    side_streams();
    try {
        // Learned pruning: the first sweep of a pass is plain (no vertex has a
        // visit history yet); a pruned sweep puts off the vertices predicted
        // not to move (they stay off until a neighbour's move re-marks them);
        // every full_every-th sweep, and the sweep after a pruned sweep whose
        // gain fell to tau while vertices were put off, is plain and takes the
        // put-off vertices back.  Only a plain sweep ends the pass.
        bool force_full = false;
        uint64_t deferred = 0;  // put off since the last plain sweep (an upper bound)
        for (int it = 0; it < max_it; it++) {
            const bool pruned = pr.learned && !force_full && it > 0 && pr.full_every > 0 &&
                                (it % pr.full_every) != pr.full_every - 1;
            set_iteration(mb, it, s);
            if (pr.learned && !pruned && deferred) {
                mlp_unskip(g, mb, s);
                deferred = 0;
            }
            bool persisted = false;
            if (use_persist) {
                GSP_CUDA(cudaMemsetAsync(mb.ctr, 0, sizeof(MoveCounters), s));
                GSP_CUDA(cudaEventRecord(e0, s));
                persisted = sweep_persistent(g, cl, mb, fp64, rule, it, max_it, s);
                use_persist = persisted;
            }
            if (!persisted) {
                GSP_CUDA(cudaEventRecord(e0, s));
                GSP_CUDA(cudaMemsetAsync(mb.ctr, 0, sizeof(MoveCounters), s));
                if (pruned) mlp_prune(g, mb, it, max_it, pr.threshold, s);
                if (use_graph && it >= 1) {
                    if (!exec) {
                        cudaGraph_t graph;
                        GSP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
                        sweep_launches(g, cl, mb, sync, fp64, rule, false, it, max_it, wave_n, false, s);
                        GSP_CUDA(cudaStreamEndCapture(s, &graph));
                        GSP_CUDA(cudaGraphInstantiate(&exec, graph, 0));
                        GSP_CUDA(cudaGraphDestroy(graph));
                    }
                    GSP_CUDA(cudaGraphLaunch(exec, s));
                } else {
                    sweep_launches(g, cl, mb, sync, fp64, rule, pruned, it, max_it, wave_n, false, s);
                }
            }
            GSP_CUDA(cudaEventRecord(e1, s));
            GSP_CUDA(cudaMemcpyAsync(&h, mb.ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
            GSP_CUDA(cudaStreamSynchronize(s));
            if (h.stalled) {
                set_error("persistent sweep: a grid barrier gave up waiting");
                throw Error{GSP_ERR_TIMEOUT};
            }
            float ms = 0;
            GSP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            r.ms_kernels += ms;
            r.bytes += sweep_bytes(h, g.wt);
            r.iterations = it + 1;
            r.vertices += h.vertices;
            r.edges += h.edges;
            r.candidates += h.candidates;
            r.skipped += h.skipped;
            deferred += h.skipped;
            // the gain of a pruned sweep misses what its put-off vertices
            // would add; their expected gain (P(move) x last gain, summed by
            // the predictor) counts with it, and when the two together stay
            // at tau the pass ends as a plain sweep's gain would end it
            if (h.dq <= tau) {
                if (!pruned || deferred == 0 || h.dq + h.skipped_gain <= tau) break;
                force_full = true;
            } else {
                force_full = false;
            }
        }
    } catch (...) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaGraph_t gdead;
            cudaStreamEndCapture(s, &gdead);
            if (gdead) cudaGraphDestroy(gdead);
        }
        throw;
    }
    if (exec) GSP_CUDA(cudaGraphExecDestroy(exec));
    return r;
}

// Allocate the move state for a graph of n vertices.
__global__ void k_set_int(int *p, int v) { *p = v; }
void set_iteration(MoveBuffers &mb, int iteration, cudaStream_t s) {
    k_set_int<<<1, 1, 0, s>>>(mb.it_dev, iteration);
    GSP_CHECK_LAUNCH();
}

// No vertex has left a community yet (left_it = -2 matches no iteration - 1).
void reset_left(MoveBuffers &mb, uint32_t n, cudaStream_t s) {
    if (!n) return;
    k_fill_u32_<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<uint32_t *>(mb.left_it), n, 0xFFFFFFFEu);
    GSP_CHECK_LAUNCH();
}

void alloc_move_state(MoveBuffers &mb, uint32_t n) {
    mb.C = arena().get<uint32_t>(n);
    mb.Sigma = arena().get<double>(n);
    mb.size = arena().get<uint32_t>(n);
    mb.act = arena().get<uint8_t>(n);
    mb.mark = arena().get<uint8_t>(n);
    mb.mv_vtx = arena().get<uint32_t>(n);
    mb.mv_cmt = arena().get<uint32_t>(n);
    mb.mv_cnt = arena().get<uint32_t>(1);
    mb.mv_cnts = arena().get<uint32_t>(MAX_WAVES * MAX_REPEATS);
    mb.bar = arena().get<GridBar>(1);
    mb.big = arena().get<uint32_t>(n);
    mb.nbig = arena().get<uint32_t>(1);
    mb.left = arena().get<uint32_t>(n);
    mb.left_it = arena().get<int>(n);
    mb.it_dev = arena().get<int>(1);
    mb.m_dev = arena().get<double>(1);
    mb.ctr = arena().get<MoveCounters>(1);
}

static void alloc_features(MoveBuffers &mb, uint32_t n, cudaStream_t s) {
    mb.feat_kept = arena().get<float>(n);
    mb.feat_gain = arena().get<float>(n);
    mb.last_gain = arena().get<float>(n);
    mb.moved_last = arena().get<uint8_t>(n);
    mb.skip = arena().get<uint8_t>(n);
    GSP_CUDA(cudaMemsetAsync(mb.skip, 0, n, s));
}

__global__ void k_init_features(float *kept, float *gain, float *last_gain, uint8_t *moved, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        kept[i] = 0.0f;
        gain[i] = 1.0f;
        last_gain[i] = 0.0f;
        moved[i] = 1;
    }
}

__global__ void k_max_double(const double *x, uint32_t n, unsigned long long *out) {
    unsigned long long mx = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        mx = max(mx, (unsigned long long)__double_as_longlong(x[i]));  // x >= 0: bits order as values
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

static double max_value(const double *x, uint32_t n, cudaStream_t s) {
    size_t mk = arena().mark();
    unsigned long long *d = arena().get<unsigned long long>(1);
    GSP_CUDA(cudaMemsetAsync(d, 0, sizeof(*d), s));
    k_max_double<<<grid_for(n, 256), 256, 0, s>>>(x, n, d);
    GSP_CHECK_LAUNCH();
    unsigned long long h = 0;
    GSP_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    arena().release(mk);
    double v;
    memcpy(&v, &h, sizeof(v));
    return v;
}

// Hub hashtables: keys (u32), values (8 bytes) and an occupied-slot list
// (u32) per slot.  The tables start empty; each sweep's scoring empties them.
void alloc_pool(MoveBuffers &mb, const Classes &cl, cudaStream_t s) {
    mb.pool = nullptr;
    if (!cl.pool_slots) return;
    size_t sa = align_up(cl.pool_slots, 64);
    mb.pool = arena().alloc(sa * 16);
    GSP_CUDA(cudaMemsetAsync(mb.pool, 0xFF, sa * sizeof(uint32_t), s));
    GSP_CUDA(cudaMemsetAsync(static_cast<uint32_t *>(mb.pool) + sa, 0, sa * sizeof(double), s));
}

// --------------------------------------------------------- GSP-Louvain run
struct Timer {
    cudaEvent_t a;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        a = g_events.get();
        GSP_CUDA(cudaEventRecord(a, s));
    }
    float lap() {  // ms since the previous lap
        cudaEvent_t b = g_events.get();
        GSP_CUDA(cudaEventRecord(b, s));
        GSP_CUDA(cudaEventSynchronize(b));
        float ms = 0;
        GSP_CUDA(cudaEventElapsedTime(&ms, a, b));
        a = b;
        return ms;
    }
};

struct TraceSpec {
    float *x = nullptr;
    uint8_t *y = nullptr;
    uint64_t *keys = nullptr;
    uint32_t cap = 0, every = 1;
    uint32_t *cnt = nullptr;  // device counter
};

void louvain_run(const DevGraph &g0, const gsp_opts &o, uint32_t *membership, double *modularity_out,
                 gsp_stats *st, cudaStream_t s, const TraceSpec *trace) {
    g_events.reset();
    const uint32_t n0 = g0.n;
    const bool sync = o.move == GSP_MOVE_SYNC;
    const int W = effective_waves(o.waves, sync);
    const bool fp64 = o.precision == GSP_PREC_FP64;
    PruneCtx pr;
    pr.learned = o.prune == GSP_PRUNE_LEARNED && o.mlp_params && !trace;
    pr.full_every = o.full_sweep_every;
    pr.threshold = o.prune_threshold;
    const bool features = pr.learned || trace;
    gsp_stats local;
    memset(&local, 0, sizeof(local));
    Timer total(s), t(s);

    MoveBuffers mb;
    alloc_move_state(mb, n0);
    double *K = arena().get<double>(n0);
    uint32_t *labels = arena().get<uint32_t>(n0);
    uint32_t *Cd = arena().get<uint32_t>(n0);
    mb.K = K;
    mb.repeats = o.wave_repeats;
    mb.no_return_from = o.no_return_from;
    mb.mlp = static_cast<const float *>(o.mlp_params);
    if (features) alloc_features(mb, n0, s);
    if (trace) {
        mb.trace_x = trace->x;
        mb.trace_y = trace->y;
        mb.trace_cnt = trace->cnt;
        mb.trace_keys = trace->keys;
        mb.trace_cap = trace->cap;
        mb.trace_every = trace->every;
    }
    // ping-pong buffers for the aggregated graphs (float64 weights)
    uint64_t *goff[2];
    uint32_t *gtgt[2];
    double *gw[2];
    for (int b = 0; b < 2; b++) {
        goff[b] = arena().get<uint64_t>((size_t)n0 + 1);
        gtgt[b] = arena().get<uint32_t>(g0.nnz + 1);
        gw[b] = arena().get<double>(g0.nnz + 1);
    }
    iota_u32(membership, n0, s);
    DevGraph cur = g0;
    double tau = o.tolerance;
    const bool split_pass = o.split != GSP_SPLIT_NONE && o.split_when == GSP_SPLIT_PASS;
    const bool refine = o.refine != 0;
    int passes = 0;
    uint32_t *Cp = mb.C;  // membership of the current graph's vertices
    int pb = 0;
    // exact integer unit of the input weights (INT_MIN: float64 sums), valid
    // for every pass: aggregated weights are sums of input weights
    int lsb_cache = exact_lsb(g0, s);
    mb.lsb = lsb_cache;
    for (int lp = 0; lp < o.max_passes; lp++) {
        const uint32_t nv = cur.n;
        size_t pass_mark = arena().mark();
        t.lap();
        // K' = Sigma' = vertexWeights(G'), C' = [0..|V'|), all unprocessed;
        // with refinement, after an aggregation, C' holds each super-vertex's
        // bound community and Sigma' sums K' over it
        double m = vertex_weights(cur, K, mb.m_dev, s, lsb_cache);
        if (refine && lp > 0) {
            sigma_from_membership(mb.C, K, mb.Sigma, mb.size, nv, s);
        } else {
            GSP_CUDA(cudaMemcpyAsync(mb.Sigma, K, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
            iota_u32(mb.C, nv, s);
            k_fill_u32_<<<grid_for(nv, 256), 256, 0, s>>>(mb.size, nv, 1u);
            GSP_CHECK_LAUNCH();
        }
        reset_left(mb, nv, s);
        GSP_CUDA(cudaMemsetAsync(mb.act, 1, nv, s));
        GSP_CUDA(cudaMemsetAsync(mb.mark, 0, nv, s));
        if (features) {
            k_init_features<<<grid_for(nv, 256), 256, 0, s>>>(mb.feat_kept, mb.feat_gain, mb.last_gain,
                                                              mb.moved_last, nv);
            GSP_CHECK_LAUNCH();
            GSP_CUDA(cudaMemsetAsync(mb.skip, 0, nv, s));
            mb.max_logk = (float)log1p(max_value(K, nv, s));
            if (!(mb.max_logk > 0.0f)) mb.max_logk = 1.0f;
            mb.trace_salt = 0x85EBCA6Bu * (uint32_t)(lp + 1);
            mb.trace_pass = lp;
        }
        Classes cl;
        classify_vertices(cur, cl, W, s);
        alloc_pool(mb, cl, s);
        float ms_other = t.lap();
        MoveLoopResult mr{0, 0, 0, 0, 0, 0.0, 0.0f};
        if (m > 0.0) mr = move_loop(cur, cl, mb, tau, o.max_iterations, sync, fp64, o.singleton_rule != 0, pr, s);
        int li = mr.iterations;
        Cp = mb.C;
        float ms_move = t.lap();
        if (split_pass) {
            split_labels(cur, cl, Cp, o.split, labels, s);
            Cp = labels;
        }
        // |Gamma| = communities after the split; |Gamma_old| = |V'|
        uint32_t k = renumber(nv, Cp, Cd, s);
        float ms_split = t.lap();
        passes = lp + 1;
        if (lp < GSP_MAX_PASS_STATS) {
            local.iterations[lp] = li;
            local.vertices[lp] = nv;
            local.communities[lp] = k;
            local.edges[lp] = cur.nnz;
            local.ms_move[lp] = ms_move;
            local.ms_split[lp] = ms_split;
            local.ms_other[lp] = ms_other;
            local.vertices_processed[lp] = mr.vertices;
            local.edges_scanned[lp] = mr.edges;
            local.vertices_skipped[lp] = mr.skipped;
            local.move_bytes[lp] = mr.bytes;
            local.ms_move_kernels[lp] = mr.ms_kernels;
        }
        if (li <= 1) break;  // globally converged
        // the partition to aggregate: C' itself, or its refinement (GSP-Leiden)
        const uint32_t *A = Cd;
        if (refine) {
            uint32_t *Rf = arena().get<uint32_t>(nv);
            uint32_t *Rd = arena().get<uint32_t>(nv);
            refine_partition(cur, cl, Cp, Rf, K, m, o.refine_theta, o.seed, (uint32_t)lp, fp64, s);
            k = renumber(nv, Rf, Rd, s);
            A = Rd;
            float ms_ref = t.lap();
            if (lp < GSP_MAX_PASS_STATS) {
                local.refined[lp] = k;
                local.ms_refine[lp] = ms_ref;
            }
        }
        if ((double)k / (double)nv > o.aggregation_tolerance) break;  // low shrink
        // renumber, dendrogram lookup, aggregate, threshold scaling
        lookup(n0, membership, A, s);
        DevGraph nxt;
        nxt.n = k;
        nxt.off = goff[pb];
        nxt.tgt = gtgt[pb];
        nxt.w = gw[pb];
        nxt.wt = GSP_W_F64;
        nxt.nnz = aggregate(cur, A, k, goff[pb], gtgt[pb], gw[pb], s, /*sorted=*/false, &lsb_cache);
        pb ^= 1;
        cur = nxt;
        tau = tau / o.tolerance_drop;
        // C' on the new graph: the identity, or each super-vertex's bound community
        if (refine) scatter_bound(A, Cd, mb.C, nv, s);
        float ms_agg = t.lap();
        if (lp < GSP_MAX_PASS_STATS) local.ms_aggregate[lp] = ms_agg;
        arena().release(pass_mark);
        if (!refine) iota_u32(mb.C, cur.n, s);
        Cp = mb.C;
    }
    // Equation 1 of the result.  Aggregation keeps every weight (self-loops
    // included), so the intra-community weight, 2m and each Sigma_c of the
    // input graph under the looked-up membership equal those of the last
    // level's graph under its own membership: Q is taken there, on the
    // smaller graph, unless a last split changes the membership on the input.
    const bool split_last = o.split != GSP_SPLIT_NONE && o.split_when == GSP_SPLIT_LAST;
    double q = split_last ? 0.0 : modularity(cur, Cp, s, lsb_cache);
    lookup(n0, membership, Cp, s);
    if (split_last) {
        Classes cl;
        classify_vertices(g0, cl, 1, s);
        split_labels(g0, cl, membership, o.split, labels, s);
        GSP_CUDA(cudaMemcpyAsync(membership, labels, sizeof(uint32_t) * n0, cudaMemcpyDeviceToDevice, s));
    }
    uint32_t kf = canonical_numbering(n0, membership, s);
    if (split_last) q = modularity(g0, membership, s, lsb_cache);
    local.passes = passes;
    local.final_communities = kf;
    local.modularity = q;
    local.ms_total = total.lap();
    local.disconnected = o.count_disconnected ? count_disconnected(g0, membership, nullptr, s) : GSP_NOT_COUNTED;
    local.workspace_bytes = workspace_peak();
    if (modularity_out) *modularity_out = q;
    if (st) *st = local;
}

}  // namespace gsp

// =============================================================== C ABI
using namespace gsp;

#define GSP_API_BEGIN try {
#define GSP_API_END                                              \
    return GSP_OK;                                               \
    }                                                            \
    catch (const gsp::Error &e) {                                \
        return e.status;                                         \
    }                                                            \
    catch (...) {                                                \
        set_error("unexpected C++ exception");                   \
        return GSP_ERR_CUDA;                                     \
    }

static cudaStream_t S(void *p) { return static_cast<cudaStream_t>(p); }

namespace gsp {
DevGraph make_graph(const uint64_t *off, const uint32_t *tgt, const void *w, int wt, uint32_t n,
                           uint64_t nnz) {
    GSP_REQUIRE(n > 0, "n must be > 0");
    GSP_REQUIRE(off != nullptr, "offsets must not be NULL");
    GSP_REQUIRE(nnz == 0 || (tgt != nullptr && w != nullptr), "targets/weights must not be NULL");
    GSP_REQUIRE(wt == GSP_W_F32 || wt == GSP_W_F64, "unknown weight type %d", wt);
    DevGraph g;
    g.n = n;
    g.nnz = nnz;
    g.off = off;
    g.tgt = tgt;
    g.w = w;
    g.wt = wt;
    return g;
}

void check_opts(const gsp_opts &o) {
    GSP_REQUIRE(o.max_passes >= 1 && o.max_passes <= 1000, "max_passes out of range");
    GSP_REQUIRE(o.max_iterations >= 1 && o.max_iterations <= 100000, "max_iterations out of range");
    GSP_REQUIRE(o.tolerance >= 0.0 && o.tolerance_drop > 0.0, "tolerance out of range");
    GSP_REQUIRE(o.aggregation_tolerance > 0.0, "aggregation_tolerance must be > 0");
    GSP_REQUIRE(o.split >= GSP_SPLIT_NONE && o.split <= GSP_SPLIT_SV, "unknown split mode");
    GSP_REQUIRE(o.split_when == GSP_SPLIT_PASS || o.split_when == GSP_SPLIT_LAST, "unknown split_when");
    GSP_REQUIRE(o.move == GSP_MOVE_ASYNC || o.move == GSP_MOVE_SYNC, "unknown move mode");
    GSP_REQUIRE(o.waves >= 0 && o.waves <= MAX_WAVES, "waves must be in [0, %d]", MAX_WAVES);
    GSP_REQUIRE(o.wave_repeats >= 1 && o.wave_repeats <= MAX_REPEATS, "wave_repeats must be in [1, %d]",
                MAX_REPEATS);
    GSP_REQUIRE(o.no_return_from >= 0, "no_return_from must be >= 0");
    GSP_REQUIRE(o.prune_threshold >= 0.0f && o.prune_threshold <= 1.0f, "prune_threshold must be in [0, 1]");
    GSP_REQUIRE(o.precision == GSP_PREC_MIXED || o.precision == GSP_PREC_FP64, "unknown precision");
    GSP_REQUIRE(o.prune == GSP_PRUNE_FLAGS || o.prune == GSP_PRUNE_LEARNED, "unknown prune mode");
    GSP_REQUIRE(o.prune != GSP_PRUNE_LEARNED || o.mlp_params != nullptr, "learned pruning needs mlp_params");
    GSP_REQUIRE(o.workspace == nullptr || o.workspace_bytes >= 256, "workspace_bytes too small");
    GSP_REQUIRE(o.refine == 0 || o.refine == 1, "refine must be 0 or 1");
    GSP_REQUIRE(o.refine_theta >= 0.0, "refine_theta must be >= 0");
}
}  // namespace gsp

extern "C" {

void gsp_default_opts(gsp_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->max_passes = 10;
    o->max_iterations = 20;
    o->tolerance = 1e-2;
    o->tolerance_drop = 10.0;
    o->aggregation_tolerance = 0.8;
    o->split = GSP_SPLIT_LPP;
    o->split_when = GSP_SPLIT_PASS;
    o->move = GSP_MOVE_SYNC;
    o->waves = 0;
    o->wave_repeats = 3;
    o->no_return_from = 3;
    o->precision = GSP_PREC_MIXED;
    o->singleton_rule = 1;
    o->prune = GSP_PRUNE_FLAGS;
    o->mlp_params = nullptr;
    o->full_sweep_every = 4;
    o->prune_threshold = 0.5f;
    o->count_disconnected = 0;
    o->refine = 0;
    o->refine_theta = 0.01;
    o->seed = 0;
    o->workspace = nullptr;
    o->workspace_bytes = 0;
    o->stream = nullptr;
}

const char *gsp_status_string(gsp_status s) {
    switch (s) {
    case GSP_OK: return "ok";
    case GSP_ERR_INVALID: return "invalid argument";
    case GSP_ERR_NOMEM: return "out of device memory";
    case GSP_ERR_CUDA: return "CUDA error";
    case GSP_ERR_TIMEOUT: return "device wait timed out";
    case GSP_ERR_CAPACITY: return "capacity exceeded";
    case GSP_ERR_NOT_SYMMETRIC: return "graph not symmetric";
    }
    return "unknown status";
}

const char *gsp_last_error(void) { return g_err; }

uint64_t gsp_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

void gsp_release_workspace(void) {
    const int d = cur_dev();
    cudaDeviceSynchronize();
    g_work[d].free_all();
    g_io[d].free_all();
}

uint64_t gsp_workspace_reserved(void) {
    uint64_t b = 0;
    for (int d = 0; d < 16; d++) {
        for (const auto &c : g_work[d].chunks) b += c.cap;
        for (const auto &c : g_io[d].chunks) b += c.cap;
    }
    return b;
}

gsp_status gsp_louvain(const uint64_t *offsets, const uint32_t *targets, const float *weights, uint32_t n,
                       uint64_t nnz, const gsp_opts *opts, uint32_t *membership, double *modularity,
                       gsp_stats *stats) {
    GSP_API_BEGIN
    gsp_opts o;
    if (opts) o = *opts;
    else gsp_default_opts(&o);
    check_opts(o);
    GSP_REQUIRE(membership != nullptr, "membership must not be NULL");
    DevGraph g = make_graph(offsets, targets, weights, GSP_W_F32, n, nnz);
    cudaStream_t s = S(o.stream);
    UserWorkspace uw(o.workspace, o.workspace_bytes);
    arena().reset();
    check_graph(offsets, targets, weights, n, nnz, s);
    louvain_run(g, o, membership, modularity, stats, s);
    GSP_API_END
}

gsp_status gsp_louvain_host(const uint64_t *offsets, const uint32_t *targets, const float *weights, uint32_t n,
                            uint64_t nnz, const gsp_opts *opts, uint32_t *membership, double *modularity,
                            gsp_stats *stats) {
    GSP_API_BEGIN
    gsp_opts o;
    if (opts) o = *opts;
    else gsp_default_opts(&o);
    check_opts(o);
    GSP_REQUIRE(n > 0 && offsets && membership && (nnz == 0 || (targets && weights)), "invalid host buffers");
    cudaStream_t s = S(o.stream);
    io_arena().reset();
    uint64_t *doff = io_arena().get<uint64_t>((size_t)n + 1);
    uint32_t *dtgt = io_arena().get<uint32_t>(nnz + 1);
    float *dw = io_arena().get<float>(nnz + 1);
    uint32_t *dC = io_arena().get<uint32_t>(n);
    GSP_CUDA(cudaMemcpyAsync(doff, offsets, sizeof(uint64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
    if (nnz) {
        GSP_CUDA(cudaMemcpyAsync(dtgt, targets, sizeof(uint32_t) * nnz, cudaMemcpyHostToDevice, s));
        GSP_CUDA(cudaMemcpyAsync(dw, weights, sizeof(float) * nnz, cudaMemcpyHostToDevice, s));
    }
    DevGraph g = make_graph(doff, dtgt, dw, GSP_W_F32, n, nnz);
    UserWorkspace uw(o.workspace, o.workspace_bytes);
    arena().reset();
    check_graph(doff, dtgt, dw, n, nnz, s);
    louvain_run(g, o, dC, modularity, stats, s);
    GSP_CUDA(cudaMemcpyAsync(membership, dC, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    GSP_API_END
}

gsp_status gsp_vertex_weights(const uint64_t *offsets, const uint32_t *targets, const void *weights, int wt,
                              uint32_t n, uint64_t nnz, double *K, double *m_host, void *stream) {
    GSP_API_BEGIN
    DevGraph g = make_graph(offsets, targets, weights, wt, n, nnz);
    GSP_REQUIRE(K != nullptr, "K must not be NULL");
    arena().reset();
    check_csr(offsets, targets, n, nnz, arena().get<unsigned long long>(1), S(stream));
    double m = vertex_weights(g, K, nullptr, S(stream), exact_lsb(g, S(stream)));
    if (m_host) *m_host = m;
    GSP_API_END
}

gsp_status gsp_modularity(const uint64_t *offsets, const uint32_t *targets, const void *weights, int wt, uint32_t n,
                          uint64_t nnz, const uint32_t *C, double *q_host, void *stream) {
    GSP_API_BEGIN
    DevGraph g = make_graph(offsets, targets, weights, wt, n, nnz);
    GSP_REQUIRE(C != nullptr && q_host != nullptr, "C and q_host must not be NULL");
    arena().reset();
    check_csr(offsets, targets, n, nnz, arena().get<unsigned long long>(1), S(stream));
    check_ids(C, n, n, "membership", S(stream));
    *q_host = modularity(g, C, S(stream), exact_lsb(g, S(stream)));
    GSP_API_END
}

gsp_status gsp_move_sweep(const uint64_t *offsets, const uint32_t *targets, const void *weights, int wt, uint32_t n,
                          uint64_t nnz, const uint32_t *C, const double *K, const double *Sigma, double m,
                          const uint8_t *active, int precision, int singleton_rule, uint32_t *choice,
                          double *dq_host, uint32_t *moved_host, void *stream) {
    GSP_API_BEGIN
    DevGraph g = make_graph(offsets, targets, weights, wt, n, nnz);
    GSP_REQUIRE(C && K && Sigma && choice, "C, K, Sigma and choice must not be NULL");
    GSP_REQUIRE(m > 0.0, "m must be > 0");
    GSP_REQUIRE(precision == GSP_PREC_MIXED || precision == GSP_PREC_FP64, "unknown precision");
    cudaStream_t s = S(stream);
    arena().reset();
    check_csr(offsets, targets, n, nnz, arena().get<unsigned long long>(1), s);
    check_ids(C, n, n, "membership", s);
    // one frozen-state wave over all vertices; decisions go to `choice`,
    // nothing is applied (C and Sigma are only read)
    MoveBuffers mb;
    alloc_move_state(mb, n);
    mb.K = K;
    mb.choice = choice;
    GSP_CUDA(cudaMemcpyAsync(mb.C, C, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    GSP_CUDA(cudaMemcpyAsync(mb.Sigma, Sigma, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    GSP_CUDA(cudaMemcpyAsync(mb.m_dev, &m, sizeof(double), cudaMemcpyHostToDevice, s));
    GSP_CUDA(cudaMemcpyAsync(choice, C, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    GSP_CUDA(cudaMemsetAsync(mb.size, 0, sizeof(uint32_t) * n, s));
    k_community_sizes<<<grid_for(n, 256), 256, 0, s>>>(C, n, mb.size);
    GSP_CHECK_LAUNCH();
    if (active) GSP_CUDA(cudaMemcpyAsync(mb.act, active, n, cudaMemcpyDeviceToDevice, s));
    else GSP_CUDA(cudaMemsetAsync(mb.act, 1, n, s));
    GSP_CUDA(cudaMemsetAsync(mb.ctr, 0, sizeof(MoveCounters), s));
    GSP_CUDA(cudaMemsetAsync(mb.mv_cnt, 0, sizeof(uint32_t), s));
    GSP_CUDA(cudaMemsetAsync(mb.mark, 0, n, s));
    Classes cl;
    classify_vertices(g, cl, 1, s);
    alloc_pool(mb, cl, s);
    set_iteration(mb, 0, s);
    move_wave(g, cl, mb, 0, true, precision == GSP_PREC_FP64, singleton_rule != 0, false, 0, 1, s);
    MoveCounters h;
    GSP_CUDA(cudaMemcpyAsync(&h, mb.ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    if (dq_host) *dq_host = h.dq;
    if (moved_host) *moved_host = (uint32_t)h.moved;
    GSP_API_END
}

gsp_status gsp_local_move(const uint64_t *offsets, const uint32_t *targets, const void *weights, int wt, uint32_t n,
                          uint64_t nnz, uint32_t *C, const double *K, double *Sigma, double m, double tolerance,
                          int max_iterations, int move, int waves, int wave_repeats, int no_return_from,
                          int precision, int singleton_rule, int *iterations_host, void *stream) {
    GSP_API_BEGIN
    DevGraph g = make_graph(offsets, targets, weights, wt, n, nnz);
    GSP_REQUIRE(C && K && Sigma, "C, K and Sigma must not be NULL");
    GSP_REQUIRE(m > 0.0 && max_iterations >= 1, "m must be > 0 and max_iterations >= 1");
    GSP_REQUIRE(move == GSP_MOVE_ASYNC || move == GSP_MOVE_SYNC, "unknown move mode");
    GSP_REQUIRE(waves >= 0 && waves <= MAX_WAVES, "waves must be in [0, %d]", MAX_WAVES);
    GSP_REQUIRE(wave_repeats >= 1 && wave_repeats <= MAX_REPEATS, "wave_repeats must be in [1, %d]", MAX_REPEATS);
    GSP_REQUIRE(no_return_from >= 0, "no_return_from must be >= 0");
    GSP_REQUIRE(precision == GSP_PREC_MIXED || precision == GSP_PREC_FP64, "unknown precision");
    cudaStream_t s = S(stream);
    arena().reset();
    g_events.reset();
    check_csr(offsets, targets, n, nnz, arena().get<unsigned long long>(1), s);
    check_ids(C, n, n, "membership", s);
    bool sync = move == GSP_MOVE_SYNC;
    MoveBuffers mb;
    alloc_move_state(mb, n);
    mb.K = K;
    mb.repeats = wave_repeats;
    mb.no_return_from = no_return_from;
    reset_left(mb, n, s);
    GSP_CUDA(cudaMemcpyAsync(mb.m_dev, &m, sizeof(double), cudaMemcpyHostToDevice, s));
    GSP_CUDA(cudaMemcpyAsync(mb.C, C, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    GSP_CUDA(cudaMemcpyAsync(mb.Sigma, Sigma, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    GSP_CUDA(cudaMemsetAsync(mb.size, 0, sizeof(uint32_t) * n, s));
    k_community_sizes<<<grid_for(n, 256), 256, 0, s>>>(C, n, mb.size);
    GSP_CHECK_LAUNCH();
    GSP_CUDA(cudaMemsetAsync(mb.act, 1, n, s));
    GSP_CUDA(cudaMemsetAsync(mb.mark, 0, n, s));
    Classes cl;
    classify_vertices(g, cl, effective_waves(waves, sync), s);
    alloc_pool(mb, cl, s);
    PruneCtx pr;
    MoveLoopResult r = move_loop(g, cl, mb, tolerance, max_iterations, sync, precision == GSP_PREC_FP64,
                                 singleton_rule != 0, pr, s);
    GSP_CUDA(cudaMemcpyAsync(C, mb.C, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    GSP_CUDA(cudaMemcpyAsync(Sigma, mb.Sigma, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    if (iterations_host) *iterations_host = r.iterations;
    GSP_API_END
}

gsp_status gsp_louvain_trace(const uint64_t *offsets, const uint32_t *targets, const float *weights, uint32_t n,
                             uint64_t nnz, const gsp_opts *opts, float *features, uint8_t *labels,
                             uint64_t *keys, uint32_t capacity, uint32_t sample_every, uint32_t *rows_host) {
    GSP_API_BEGIN
    gsp_opts o;
    if (opts) o = *opts;
    else gsp_default_opts(&o);
    o.prune = GSP_PRUNE_FLAGS;
    check_opts(o);
    GSP_REQUIRE(features && labels && capacity > 0 && sample_every >= 1, "invalid trace buffers");
    DevGraph g = make_graph(offsets, targets, weights, GSP_W_F32, n, nnz);
    cudaStream_t s = S(o.stream);
    arena().reset();
    check_graph(offsets, targets, weights, n, nnz, s);
    uint32_t *membership = arena().get<uint32_t>(n);
    TraceSpec tr;
    tr.x = features;
    tr.y = labels;
    tr.keys = keys;
    tr.cap = capacity;
    tr.every = sample_every;
    tr.cnt = arena().get<uint32_t>(1);
    GSP_CUDA(cudaMemsetAsync(tr.cnt, 0, sizeof(uint32_t), s));
    louvain_run(g, o, membership, nullptr, nullptr, s, &tr);
    uint32_t rows = 0;
    GSP_CUDA(cudaMemcpyAsync(&rows, tr.cnt, sizeof(rows), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    if (rows_host) *rows_host = std::min(rows, capacity);
    GSP_API_END
}

gsp_status gsp_refine(const uint64_t *offsets, const uint32_t *targets, const void *weights, int wt, uint32_t n,
                      uint64_t nnz, const uint32_t *B, uint32_t *R, double theta, uint64_t seed, uint32_t pass,
                      int waves, int precision, uint32_t *moves_host, void *stream) {
    GSP_API_BEGIN
    DevGraph g = make_graph(offsets, targets, weights, wt, n, nnz);
    GSP_REQUIRE(B && R, "B and R must not be NULL");
    GSP_REQUIRE(theta >= 0.0, "theta must be >= 0");
    GSP_REQUIRE(waves >= 0 && waves <= MAX_WAVES, "waves must be in [0, %d]", MAX_WAVES);
    GSP_REQUIRE(precision == GSP_PREC_MIXED || precision == GSP_PREC_FP64, "unknown precision");
    cudaStream_t s = S(stream);
    arena().reset();
    check_csr(offsets, targets, n, nnz, arena().get<unsigned long long>(1), s);
    check_ids(B, n, n, "bound membership", s);
    double *K = arena().get<double>(n);
    double *m_dev = arena().get<double>(1);
    double m = vertex_weights(g, K, m_dev, s, exact_lsb(g, s));
    Classes cl;
    classify_vertices(g, cl, effective_waves(waves, true), s);
    uint32_t moves = refine_partition(g, cl, B, R, K, m, theta, seed, pass, precision == GSP_PREC_FP64, s);
    if (moves_host) *moves_host = moves;
    GSP_API_END
}

gsp_status gsp_split(const uint64_t *offsets, const uint32_t *targets, uint32_t n, uint64_t nnz, const uint32_t *C,
                     int mode, uint32_t *labels, uint32_t *k_host, void *stream) {
    GSP_API_BEGIN
    GSP_REQUIRE(mode == GSP_SPLIT_LP || mode == GSP_SPLIT_LPP || mode == GSP_SPLIT_BFS || mode == GSP_SPLIT_SV,
                "unknown split mode");
    GSP_REQUIRE(C && labels && n > 0 && offsets && (nnz == 0 || targets), "invalid arguments");
    DevGraph g = make_graph(offsets, targets, targets ? (const void *)targets : (const void *)offsets, GSP_W_F32, n,
                            nnz);
    cudaStream_t s = S(stream);
    arena().reset();
    check_csr(offsets, targets, n, nnz, arena().get<unsigned long long>(1), s);
    check_ids(C, n, n, "membership", s);
    Classes cl;
    classify_vertices(g, cl, 1, s);
    split_labels(g, cl, C, mode, labels, s);
    if (k_host) {
        uint32_t *tmp = arena().get<uint32_t>(n);
        *k_host = renumber(n, labels, tmp, s);
    }
    GSP_CUDA(cudaStreamSynchronize(s));
    GSP_API_END
}

gsp_status gsp_renumber(uint32_t n, const uint32_t *C, uint32_t *C_dense, uint32_t *k_host, void *stream) {
    GSP_API_BEGIN
    GSP_REQUIRE(n > 0 && C && C_dense, "invalid arguments");
    arena().reset();
    check_ids(C, n, n, "membership", S(stream));
    uint32_t k = renumber(n, C, C_dense, S(stream));
    if (k_host) *k_host = k;
    GSP_API_END
}

gsp_status gsp_lookup(uint32_t n_top, uint32_t *C_top, const uint32_t *C_pass, void *stream) {
    GSP_API_BEGIN
    GSP_REQUIRE(C_top && C_pass, "invalid arguments");
    lookup(n_top, C_top, C_pass, S(stream));
    GSP_CUDA(cudaStreamSynchronize(S(stream)));
    GSP_API_END
}

gsp_status gsp_aggregate(const uint64_t *offsets, const uint32_t *targets, const void *weights, int wt, uint32_t n,
                         uint64_t nnz, const uint32_t *C, uint32_t k, uint64_t *out_offsets, uint32_t *out_targets,
                         double *out_weights, uint64_t *out_nnz_host, void *stream) {
    GSP_API_BEGIN
    DevGraph g = make_graph(offsets, targets, weights, wt, n, nnz);
    GSP_REQUIRE(C && out_offsets && k > 0 && k <= n, "invalid arguments");
    GSP_REQUIRE(nnz == 0 || (out_targets && out_weights), "output arrays must not be NULL");
    arena().reset();
    check_csr(offsets, targets, n, nnz, arena().get<unsigned long long>(1), S(stream));
    check_ids(C, n, k, "membership", S(stream));
    uint64_t e = aggregate(g, C, k, out_offsets, out_targets, out_weights, S(stream));
    GSP_CUDA(cudaStreamSynchronize(S(stream)));
    if (out_nnz_host) *out_nnz_host = e;
    GSP_API_END
}

gsp_status gsp_count_disconnected(const uint64_t *offsets, const uint32_t *targets, uint32_t n, uint64_t nnz,
                                  const uint32_t *C, uint8_t *flags, uint32_t *count_host, void *stream) {
    GSP_API_BEGIN
    GSP_REQUIRE(C && n > 0 && offsets && (nnz == 0 || targets), "invalid arguments");
    DevGraph g = make_graph(offsets, targets, targets ? (const void *)targets : (const void *)offsets, GSP_W_F32, n,
                            nnz);
    arena().reset();
    check_csr(offsets, targets, n, nnz, arena().get<unsigned long long>(1), S(stream));
    check_ids(C, n, n, "membership", S(stream));
    uint32_t c = count_disconnected(g, C, flags, S(stream));
    if (count_host) *count_host = c;
    GSP_API_END
}

}  // extern "C"
