// tune.cu -- launch-geometry tuning of the local-moving kernels.
//
// Each degree class of local moving (Algorithm 4) runs as a grid-stride
// kernel whose grid is capped at a number of blocks per SM, and the degree
// boundaries between the classes decide which kernel (table size, lanes per
// vertex) serves a vertex.  The best choices depend on the graph's degree
// distribution (how many vertices of each class a wave holds, how unbalanced
// the hubs are), so gsp_autotune (one graph) and gsp_autotune_batched (a
// batch, timed through the batched call) pick them on the caller's input by
// timing whole runs under candidate caps and boundaries, one knob at a time.
// Caps and boundaries change only which threads do the work: in frozen-state
// mode a run's result is the same under every setting.
#include <string.h>

#include <algorithm>
#include <functional>
#include <mutex>

#include "internal.cuh"

namespace gsp {

static Tuning g_tuning;
static std::mutex g_tuning_mu;

Tuning &tuning() { return g_tuning; }

int sm_count() {
    static int cached[64] = {0};
    int d = 0;
    GSP_CUDA(cudaGetDevice(&d));
    GSP_REQUIRE(d >= 0 && d < 64, "device index %d out of range", d);
    if (!cached[d]) {
        int v = 0;
        GSP_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d));
        cached[d] = v > 0 ? v : 1;
    }
    return cached[d];
}

unsigned resident_grid(const void *fn, int threads, size_t dyn_smem, unsigned per_sm_cap) {
    int nb = 0;
    GSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, dyn_smem));
    unsigned per = nb > 0 ? (unsigned)nb : 1u;
    return sms(per < per_sm_cap ? per : per_sm_cap);
}

constexpr int TUNE_MAX = 32;  // blocks per SM, upper limit of every cap

static void check_tuning(const gsp_tuning &t) {
    GSP_REQUIRE(t.groups_blocks_per_sm >= 1 && t.groups_blocks_per_sm <= TUNE_MAX &&
                    t.w512_blocks_per_sm >= 1 && t.w512_blocks_per_sm <= TUNE_MAX &&
                    t.block_blocks_per_sm >= 1 && t.block_blocks_per_sm <= TUNE_MAX &&
                    t.hub_blocks_per_sm >= 1 && t.hub_blocks_per_sm <= TUNE_MAX,
                "tuning caps must be in [1, %d] blocks per SM", TUNE_MAX);
    GSP_REQUIRE(t.group_max_degree >= 33 && t.group_max_degree <= GROUP_MAX_LIMIT &&
                    t.warp_max_degree > t.group_max_degree && t.warp_max_degree <= WARP_MAX_LIMIT &&
                    t.block_max_degree > t.warp_max_degree && t.block_max_degree <= BLOCK_MAX_LIMIT &&
                    t.big_max_degree > t.block_max_degree && t.big_max_degree <= BIG_MAX_LIMIT,
                "class boundaries must rise: 33 <= group_max <= %u < warp_max <= %u < block_max <= %u < "
                "big_max <= %u",
                GROUP_MAX_LIMIT, WARP_MAX_LIMIT, BLOCK_MAX_LIMIT, BIG_MAX_LIMIT);
}

static gsp_tuning to_abi(const Tuning &t) {
    gsp_tuning o;
    o.groups_blocks_per_sm = t.groups;
    o.w512_blocks_per_sm = t.w512;
    o.block_blocks_per_sm = t.block;
    o.hub_blocks_per_sm = t.hub;
    o.persist_max_vertices = t.persist_max_vertices;
    o.group_max_degree = t.group_max;
    o.warp_max_degree = t.warp_max;
    o.block_max_degree = t.block_max;
    o.big_max_degree = t.big_max;
    return o;
}

static Tuning from_abi(const gsp_tuning &t) {
    Tuning o;
    o.groups = t.groups_blocks_per_sm;
    o.w512 = t.w512_blocks_per_sm;
    o.block = t.block_blocks_per_sm;
    o.hub = t.hub_blocks_per_sm;
    o.persist_max_vertices = t.persist_max_vertices;
    o.group_max = t.group_max_degree;
    o.warp_max = t.warp_max_degree;
    o.block_max = t.block_max_degree;
    o.big_max = t.big_max_degree;
    return o;
}

}  // namespace gsp

using namespace gsp;

extern "C" {

gsp_status gsp_get_tuning(gsp_tuning *out) {
    if (!out) {
        set_error("gsp_get_tuning: out must not be NULL");
        return GSP_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    *out = to_abi(g_tuning);
    return GSP_OK;
}

gsp_status gsp_set_tuning(const gsp_tuning *t) {
    try {
        GSP_REQUIRE(t != nullptr, "gsp_set_tuning: t must not be NULL");
        check_tuning(*t);
        std::lock_guard<std::mutex> lock(g_tuning_mu);
        g_tuning = from_abi(*t);
        return GSP_OK;
    } catch (const gsp::Error &e) {
        return e.status;
    }
}

}  // extern "C"

namespace gsp {

// Device buffers of the trials, outside the workspace (which a trial may
// free: candidates with other class boundaries allocate in another order, and
// the chunked workspace then grows), and the trials' own events (a run resets
// the event pool).
struct TuneBuffers {
    uint32_t *membership = nullptr;
    double *q = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // allocated after construction, so that the destructor frees what a
    // failing later allocation leaves behind
    void alloc(uint32_t n, uint32_t num_q) {
        GSP_CUDA(cudaMalloc(&membership, sizeof(uint32_t) * (size_t)n));
        if (num_q) GSP_CUDA(cudaMalloc(&q, sizeof(double) * (size_t)num_q));
        GSP_CUDA(cudaEventCreate(&e0));
        GSP_CUDA(cudaEventCreate(&e1));
    }
    ~TuneBuffers() {
        if (membership) cudaFree(membership);
        if (q) cudaFree(q);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Validation shared by both entry points; returns the stream the trials run on.
static cudaStream_t tune_prologue(const DevGraph &g, const uint64_t *offsets, const uint32_t *targets,
                                  const float *weights, const gsp_opts &o) {
    cudaStream_t caller = static_cast<cudaStream_t>(o.stream);
    arena().reset();
    reset_event_pool();
    check_graph(offsets, targets, weights, g.n, g.nnz, caller);
    GSP_CUDA(cudaStreamSynchronize(caller));
    cudaStream_t s = capture_stream();
    size_t mk = arena().mark();
    double *K = arena().get<double>(g.n);
    double *m_dev = arena().get<double>(1);
    const double m = vertex_weights(g, K, m_dev, s);
    arena().release(mk);
    GSP_REQUIRE(m > 0.0, "gsp_autotune: the graph has no edges");
    return s;
}

// The search.  A trial is whole calls through `one_run` on the caller's
// options (the caps act on local moving, whose share and degree mix change
// from pass to pass, so no part of a run stands in for it); whole runs repeat
// within a few tenths of a percent.
static void autotune_search(const std::function<void()> &one_run, TuneBuffers &tb_, cudaStream_t s,
                            gsp_tuning *chosen, float *ms_default, float *ms_tuned) {
    auto run = [&]() -> float {
        arena().reset();
        GSP_CUDA(cudaEventRecord(tb_.e0, s));
        one_run();
        GSP_CUDA(cudaEventRecord(tb_.e1, s));
        GSP_CUDA(cudaEventSynchronize(tb_.e1));
        float ms = 0;
        GSP_CUDA(cudaEventElapsedTime(&ms, tb_.e0, tb_.e1));
        return ms;
    };
    // A candidate with other class boundaries allocates in another order:
    // the workspace is freed and rebuilt by an untimed run first.  Caps alone
    // allocate the same; should a run still grow the workspace, it is timed
    // again, and a workspace above 1.5 x its first size is rebuilt before the
    // next run.
    uint64_t limit = 0;
    ClassBounds ran{0, 0, 0, 0};
    auto trial = [&]() -> float {
        const Tuning &t = g_tuning;
        const bool moved = ran.group_max != t.group_max || ran.warp_max != t.warp_max ||
                           ran.block_max != t.block_max || ran.big_max != t.big_max;
        if (moved || (limit && gsp_workspace_reserved() > limit)) {
            gsp_release_workspace();
            run();
            ran = ClassBounds{t.group_max, t.warp_max, t.block_max, t.big_max};
        }
        const uint64_t before = gsp_workspace_reserved();
        if (!limit) limit = before + before / 2;
        float ms = run();
        if (gsp_workspace_reserved() > before) ms = run();
        return std::min(ms, run());  // the better of two runs
    };
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    const Tuning start = g_tuning;
    Tuning best = start;
    float t0 = 0.0f, tb = 0.0f;
    try {
        trial();  // first-touch effects (workspace, instruction cache)
        t0 = tb = trial();
        // a candidate replaces the current choice only when it is faster by
        // more than the run-to-run spread of a trial
        constexpr float ACCEPT = 0.99f;
        struct Knob {
            int Tuning::*field;
            int cand[5];
        };
        const Knob knobs[] = {{&Tuning::groups, {4, 6, 8, 12, 16}},
                              {&Tuning::w512, {1, 2, 3, 4, 6}},
                              {&Tuning::block, {2, 3, 4, 5, 8}},
                              {&Tuning::hub, {2, 4, 8, 16, 32}}};
        // class boundaries: each class may hand its upper half to the next
        // (larger) kernel; a boundary only moves down from the limit its
        // table allows
        struct Bound {
            uint32_t Tuning::*field;
            uint32_t cand[2];
        };
        const Bound bounds[] = {{&Tuning::group_max, {GROUP_MAX_LIMIT, GROUP_MAX_LIMIT / 2}},
                                {&Tuning::warp_max, {WARP_MAX_LIMIT, WARP_MAX_LIMIT / 2}},
                                {&Tuning::block_max, {BLOCK_MAX_LIMIT, BLOCK_MAX_LIMIT / 2}},
                                {&Tuning::big_max, {BIG_MAX_LIMIT, BIG_MAX_LIMIT / 2}}};
        auto valid = [](const Tuning &t) {
            return t.group_max >= 33 && t.warp_max > t.group_max && t.block_max > t.warp_max &&
                   t.big_max > t.block_max;
        };
        for (const Knob &k : knobs) {
            for (int v : k.cand) {
                if (v == best.*(k.field)) continue;
                g_tuning = best;
                g_tuning.*(k.field) = v;
                float t = trial();
                if (t < tb * ACCEPT) {
                    tb = t;
                    best = g_tuning;
                }
            }
        }
        for (const Bound &b : bounds) {
            for (uint32_t v : b.cand) {
                if (v == best.*(b.field)) continue;
                Tuning c = best;
                c.*(b.field) = v;
                if (!valid(c)) continue;
                g_tuning = c;
                float t = trial();
                if (t < tb * ACCEPT) {
                    tb = t;
                    best = g_tuning;
                }
            }
        }
        // the pick is the best of many noisy trials: time it against the
        // starting settings once more and keep whichever is faster; the two
        // times reported are then those of this last pair
        if (!(best.groups == start.groups && best.w512 == start.w512 && best.block == start.block &&
              best.hub == start.hub && best.group_max == start.group_max && best.warp_max == start.warp_max &&
              best.block_max == start.block_max && best.big_max == start.big_max)) {
            g_tuning = start;
            const float ts = trial();
            g_tuning = best;
            const float tbest = trial();
            t0 = ts;
            if (ts <= tbest) {
                best = start;
                tb = ts;
            } else {
                tb = tbest;
            }
        }
    } catch (...) {
        g_tuning = start;
        throw;
    }
    g_tuning = best;
    if (chosen) *chosen = to_abi(best);
    if (ms_default) *ms_default = t0;
    if (ms_tuned) *ms_tuned = tb;
    GSP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gsp

extern "C" {

gsp_status gsp_autotune(const uint64_t *offsets, const uint32_t *targets, const float *weights, uint32_t n,
                        uint64_t nnz, const gsp_opts *opts, gsp_tuning *chosen, float *ms_default,
                        float *ms_tuned) {
    try {
        gsp_opts o;
        if (opts) o = *opts;
        else gsp_default_opts(&o);
        check_opts(o);
        DevGraph g = make_graph(offsets, targets, weights, GSP_W_F32, n, nnz);
        cudaStream_t s = tune_prologue(g, offsets, targets, weights, o);
        TuneBuffers buf;
        buf.alloc(n, 0);
        gsp_opts ro = o;
        ro.count_disconnected = 0;
        ro.stream = s;
        autotune_search([&]() { louvain_run(g, ro, buf.membership, nullptr, nullptr, s); }, buf, s, chosen,
                        ms_default, ms_tuned);
        return GSP_OK;
    } catch (const gsp::Error &e) {
        return e.status;
    } catch (...) {
        set_error("unexpected C++ exception");
        return GSP_ERR_CUDA;
    }
}

gsp_status gsp_autotune_batched(uint32_t num_graphs, const uint64_t *graph_vertex_offsets, const uint64_t *offsets,
                                const uint32_t *targets, const float *weights, uint32_t n, uint64_t nnz,
                                const gsp_opts *opts, gsp_tuning *chosen, float *ms_default, float *ms_tuned) {
    try {
        gsp_opts o;
        if (opts) o = *opts;
        else gsp_default_opts(&o);
        check_opts(o);
        check_batch(num_graphs, graph_vertex_offsets, n, o);
        DevGraph g = make_graph(offsets, targets, weights, GSP_W_F32, n, nnz);
        cudaStream_t s = tune_prologue(g, offsets, targets, weights, o);
        TuneBuffers buf;
        buf.alloc(n, num_graphs);
        gsp_opts ro = o;
        ro.count_disconnected = 0;
        ro.stream = s;
        autotune_search(
            [&]() { louvain_batched_run(g, num_graphs, graph_vertex_offsets, ro, buf.membership, buf.q, nullptr, s); },
            buf, s, chosen, ms_default, ms_tuned);
        return GSP_OK;
    } catch (const gsp::Error &e) {
        return e.status;
    } catch (...) {
        set_error("unexpected C++ exception");
        return GSP_ERR_CUDA;
    }
}

}  // extern "C"
