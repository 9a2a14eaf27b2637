// batched.cu -- GSP-Louvain (Algorithm 1) over a batch of independent graphs
// in one set of launches.
//
// The graphs are concatenated into one CSR (no edge crosses graphs) and every
// kernel runs over the union, with per-graph state so that each graph follows
// the run it would have alone:
//   * a vertex scores moves (Equation 2) with the m of its own graph;
//   * waves use the vertex's index within its graph;
//   * the gains of a sweep are summed per graph, and a graph stops iterating
//     when its own sum is <= tau (its vertices are then left unprocessed);
//   * after the split each graph takes its own decisions (l_i <= 1, low
//     shrink) and finishes on its own.  A finished graph's membership is fixed
//     and it is collapsed to one super-vertex, so it costs one vertex and one
//     self-loop in the passes that follow;
//   * communities never cross graphs, so split, renumbering and aggregation
//     run on the union unchanged, and every graph's super-vertices stay one
//     contiguous id range.
// Membership values of a graph that finishes are rewritten to the smallest
// input vertex of each community (an id unique across graphs and levels);
// the final numbering then orders communities by that vertex.
#include <string.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "internal.cuh"

namespace gsp {

// gid[v] = the graph owning vertex v: the last g with gvo[g] <= v (empty
// graphs own no vertex).
__global__ void k_graph_of(const uint64_t *__restrict__ gvo, uint32_t G, uint32_t n, uint32_t *gid) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = G - 1;
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo + 1) / 2;
            if (gvo[mid] <= v) lo = mid;
            else hi = mid - 1;
        }
        gid[v] = lo;
    }
}

// Entries whose target lies outside the vertex range of their row's graph,
// edge-parallel: warp w of the grid takes the contiguous entries
// [nnz w / warps, nnz (w+1) / warps), its lanes consecutive entries.
constexpr int CROSS_UNROLL = 4;
__global__ void __launch_bounds__(256) k_cross_edges(const uint64_t *__restrict__ off,
                                                     const uint32_t *__restrict__ tgt,
                                                     const uint32_t *__restrict__ gid,
                                                     const uint64_t *__restrict__ gvo, uint32_t n, uint64_t nnz,
                                                     unsigned long long *bad) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t wid = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t w0 = nnz * wid / warps, w1 = nnz * (wid + 1) / warps;
    uint32_t r = 0;
    if (lane == 0 && w0 < w1) r = row_of(off, n, w0);
    r = __shfl_sync(0xffffffffu, r, 0);
    unsigned long long cnt = 0;
    for (uint64_t p = w0 + lane; p < w1; p += 32ull * CROSS_UNROLL) {
        uint32_t t[CROSS_UNROLL];
#pragma unroll
        for (int k = 0; k < CROSS_UNROLL; k++) {
            const uint64_t q = p + 32ull * k;
            t[k] = q < w1 ? __ldg(tgt + q) : 0u;
        }
#pragma unroll
        for (int k = 0; k < CROSS_UNROLL; k++) {
            const uint64_t q = p + 32ull * k;
            if (q < w1) {
                r = row_from(off, n, q, r);
                const uint32_t g = __ldg(gid + r);
                cnt += t[k] < __ldg(gvo + g) || t[k] >= __ldg(gvo + g + 1);
            }
        }
    }
    cnt = warp_sum(cnt);
    if (lane == 0 && cnt) atomicAdd(bad, cnt);
}

__global__ void k_fill_ones(uint32_t *p, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 1u;
}

// m of each graph: half its K total.
__global__ void k_graph_m(const double *__restrict__ K, const uint32_t *__restrict__ gid, uint32_t n, double *m_g) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (K[v] != 0.0) atomicAdd(m_g + gid[v], 0.5 * K[v]);
}

// Unprocessed flags: set for the vertices of the graphs still iterating.
__global__ void k_set_active(uint8_t *act, const uint32_t *__restrict__ gid, const uint8_t *__restrict__ live,
                             uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        act[v] = live[gid[v]];
}
__global__ void k_clear_stopped(uint8_t *act, const uint32_t *__restrict__ gid, const uint8_t *__restrict__ live,
                                uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (!live[gid[v]] && act[v]) act[v] = 0;
}

// Communities of each graph: community ids are vertex ids of the same graph,
// so mark the ids in use and count them by the graph owning the id.
__global__ void k_mark_ids(const uint32_t *__restrict__ C, uint32_t n, uint8_t *used) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) used[C[v]] = 1;
}
__global__ void k_count_ids(const uint8_t *__restrict__ used, const uint32_t *__restrict__ gid, uint32_t n,
                            uint32_t *k_g) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (used[v]) atomicAdd(k_g + gid[v], 1u);
}

// Graphs in `sel`: membership of their input vertices := the smallest input
// vertex of their community (community = lab[C_top[v]]).
__global__ void k_rep_min(const uint32_t *__restrict__ C_top, const uint32_t *__restrict__ lab,
                          const uint32_t *__restrict__ gid0, const uint8_t *__restrict__ sel, uint32_t n0,
                          uint32_t *first) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += gridDim.x * blockDim.x)
        if (sel[gid0[v]]) atomicMin(first + lab[C_top[v]], v);
}
__global__ void k_rep_apply(uint32_t *C_top, const uint32_t *__restrict__ lab, const uint32_t *__restrict__ gid0,
                            const uint8_t *__restrict__ sel, uint32_t n0, const uint32_t *__restrict__ first) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += gridDim.x * blockDim.x)
        if (sel[gid0[v]]) C_top[v] = first[lab[C_top[v]]];
}

// Finished graphs collapse to their first vertex; the others keep their label.
__global__ void k_collapse(const uint32_t *__restrict__ lab, const uint32_t *__restrict__ gid,
                           const uint8_t *__restrict__ done, const uint64_t *__restrict__ gvo, uint32_t n,
                           uint32_t *out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t g = gid[v];
        out[v] = done[g] ? (uint32_t)gvo[g] : lab[v];
    }
}

// Dendrogram lookup for the graphs still open.
__global__ void k_lookup_open(uint32_t *C_top, const uint32_t *__restrict__ Cd, const uint32_t *__restrict__ gid0,
                              const uint8_t *__restrict__ done, uint32_t n0) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += gridDim.x * blockDim.x)
        if (!done[gid0[v]]) C_top[v] = Cd[C_top[v]];
}

// Equation 1 per graph on the input graphs, with the union-wide community ids
// C: 2m, the intra-community weight and Sigma of each community.
template <typename WT, typename AV>
__global__ void k_graph_q_rows(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tgt,
                               const WT *__restrict__ w, const uint32_t *__restrict__ C,
                               const uint32_t *__restrict__ gid0, uint32_t n0, double *two_m, double *intra,
                               double *Sig, uint32_t *comm_graph, int lsb) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += gridDim.x * blockDim.x) {
        AV k = 0, in = 0;
        const uint32_t cv = C[v], g = gid0[v];
        for (uint64_t p = off[v]; p < off[v + 1]; p++) {
            const AV x = Acc<AV>::of(w[p], lsb);
            k += x;
            if (C[tgt[p]] == cv) in += x;
        }
        comm_graph[cv] = g;  // every member writes the same value
        if (k != AV(0)) {
            const double kd = Acc<AV>::val(k, lsb);
            atomicAdd(two_m + g, kd);
            atomicAdd(Sig + cv, kd);
        }
        if (in != AV(0)) atomicAdd(intra + g, Acc<AV>::val(in, lsb));
    }
}
__global__ void k_graph_q_sq(const double *__restrict__ Sig, const uint32_t *__restrict__ comm_graph, uint32_t k,
                             double *sumsq) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
        double x = Sig[c];
        if (x != 0.0) atomicAdd(sumsq + comm_graph[c], x * x);
    }
}
// Q_g = intra/2m - sum Sigma^2/(2m)^2, 0 when 2m = 0; base[g] = the union id
// of the community of the graph's first vertex (its smallest id).
__global__ void k_graph_q_final(const double *__restrict__ two_m, const double *__restrict__ intra,
                                const double *__restrict__ sumsq, const uint32_t *__restrict__ C,
                                const uint64_t *__restrict__ gvo0, uint32_t G, double *q, uint32_t *base) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        double t = two_m[g];
        q[g] = t > 0.0 ? intra[g] / t - sumsq[g] / (t * t) : 0.0;
        base[g] = gvo0[g + 1] > gvo0[g] ? C[gvo0[g]] : 0u;
    }
}
__global__ void k_localise(uint32_t *C, const uint32_t *__restrict__ gid0, const uint32_t *__restrict__ base,
                           uint32_t n0) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += gridDim.x * blockDim.x)
        C[v] -= base[gid0[v]];
}

struct Lap {
    cudaStream_t s;
    cudaEvent_t a;
    explicit Lap(cudaStream_t st) : s(st) {
        a = pool_event();
        GSP_CUDA(cudaEventRecord(a, s));
    }
    float operator()() {
        cudaEvent_t b = pool_event();
        GSP_CUDA(cudaEventRecord(b, s));
        GSP_CUDA(cudaEventSynchronize(b));
        float ms = 0;
        GSP_CUDA(cudaEventElapsedTime(&ms, a, b));
        a = b;
        return ms;
    }
};

struct BatchMove {
    uint64_t vertices = 0, edges = 0;
    double bytes = 0;
    float ms_kernels = 0;
};

// louvainMove (Algorithm 4) for every open graph at once, with per-graph gains
// and stopping.  h_live (in/out) flags the graphs still iterating; h_li
// receives each graph's l_i.  Sweeps after the first replay a CUDA graph.
static BatchMove batch_move_loop(const DevGraph &g, const Classes &cl, MoveBuffers &mb, uint32_t G, double tau,
                                 const gsp_opts &o, std::vector<uint8_t> &h_live, std::vector<int> &h_li,
                                 uint8_t *live, cudaStream_t s) {
    const bool sync = o.move == GSP_MOVE_SYNC;
    const bool fp64 = o.precision == GSP_PREC_FP64;
    const bool rule = o.singleton_rule != 0;
    BatchMove r;
    uint32_t nlive = 0;
    for (uint32_t gi = 0; gi < G; gi++) nlive += h_live[gi];
    if (!nlive) return r;
    uint32_t wave_n[MAX_WAVES];
    for (int wv = 0; wv < cl.W; wv++) {
        wave_n[wv] = 0;
        for (int c = 0; c < NUM_CLS; c++) wave_n[wv] += cl.count(c, wv);
    }
    std::vector<double> h_dq(G);
    MoveCounters h;
    cudaEvent_t e0 = pool_event(), e1 = pool_event();
    cudaGraphExec_t exec = nullptr;
    const bool use_graph = graphs_enabled();
    bool use_persist = sync && persistent_enabled();  // small graphs: one launch per sweep
    side_streams();
    try {
        for (int it = 0; it < o.max_iterations && nlive; it++) {
            GSP_CUDA(cudaMemsetAsync(mb.dq_g, 0, sizeof(double) * G, s));
            set_iteration(mb, it, s);
            bool persisted = false;
            if (use_persist) {
                GSP_CUDA(cudaMemsetAsync(mb.ctr, 0, sizeof(MoveCounters), s));
                GSP_CUDA(cudaEventRecord(e0, s));
                persisted = sweep_persistent(g, cl, mb, fp64, rule, it, o.max_iterations, s);
                use_persist = persisted;
            }
            if (persisted) {
            } else {
            GSP_CUDA(cudaEventRecord(e0, s));
            if (use_graph && it >= 1) {
                if (!exec) {
                    cudaGraph_t graph;
                    GSP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
                    sweep_launches(g, cl, mb, sync, fp64, rule, false, it, o.max_iterations, wave_n, true, s);
                    GSP_CUDA(cudaStreamEndCapture(s, &graph));
                    GSP_CUDA(cudaGraphInstantiate(&exec, graph, 0));
                    GSP_CUDA(cudaGraphDestroy(graph));
                }
                GSP_CUDA(cudaGraphLaunch(exec, s));
            } else {
                sweep_launches(g, cl, mb, sync, fp64, rule, false, it, o.max_iterations, wave_n, true, s);
            }
            }
            GSP_CUDA(cudaEventRecord(e1, s));
            GSP_CUDA(cudaMemcpyAsync(&h, mb.ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
            GSP_CUDA(cudaMemcpyAsync(h_dq.data(), mb.dq_g, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
            GSP_CUDA(cudaStreamSynchronize(s));
            if (h.stalled) {
                set_error("persistent sweep: a grid barrier gave up waiting");
                throw Error{GSP_ERR_TIMEOUT};
            }
            float ms = 0;
            GSP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            r.ms_kernels += ms;
            r.bytes += sweep_bytes(h, g.wt);
            r.vertices += h.vertices;
            r.edges += h.edges;
            bool stopped = false;
            for (uint32_t gi = 0; gi < G; gi++) {
                if (!h_live[gi]) continue;
                h_li[gi] = it + 1;
                if (h_dq[gi] <= tau) {
                    h_live[gi] = 0;
                    nlive--;
                    stopped = true;
                }
            }
            if (stopped && nlive) {
                GSP_CUDA(cudaMemcpyAsync(live, h_live.data(), G, cudaMemcpyHostToDevice, s));
                k_clear_stopped<<<grid_for(g.n, 256), 256, 0, s>>>(mb.act, mb.gid, live, g.n);
                GSP_CHECK_LAUNCH();
            }
        }
    } catch (...) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaStreamCaptureStatus cst;
        if (cudaStreamIsCapturing(s, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
            cudaGraph_t gdead = nullptr;
            cudaStreamEndCapture(s, &gdead);
            if (gdead) cudaGraphDestroy(gdead);
        }
        throw;
    }
    if (exec) GSP_CUDA(cudaGraphExecDestroy(exec));
    return r;
}

// Membership of the graphs in h_sel := smallest input vertex of the community
// that lab gives their current-level vertex.
static void to_representatives(uint32_t *membership, const uint32_t *lab, uint32_t nv, const uint32_t *gid0,
                               uint32_t n0, uint8_t *sel, const std::vector<uint8_t> &h_sel, uint32_t *first,
                               cudaStream_t s) {
    GSP_CUDA(cudaMemcpyAsync(sel, h_sel.data(), h_sel.size(), cudaMemcpyHostToDevice, s));
    GSP_CUDA(cudaMemsetAsync(first, 0xFF, sizeof(uint32_t) * nv, s));
    k_rep_min<<<grid_for(n0, 256), 256, 0, s>>>(membership, lab, gid0, sel, n0, first);
    GSP_CHECK_LAUNCH();
    k_rep_apply<<<grid_for(n0, 256), 256, 0, s>>>(membership, lab, gid0, sel, n0, first);
    GSP_CHECK_LAUNCH();
}

void louvain_batched_run(const DevGraph &g0, uint32_t G, const uint64_t *h_gvo0, const gsp_opts &o,
                         uint32_t *membership, double *q_out, gsp_stats *st, cudaStream_t caller) {
    reset_event_pool();
    cudaStream_t s = capture_stream();
    {
        cudaEvent_t in = pool_event();
        GSP_CUDA(cudaEventRecord(in, caller));
        GSP_CUDA(cudaStreamWaitEvent(s, in, 0));
    }
    const uint32_t n0 = g0.n;
    const int W = effective_waves(o.waves, o.move == GSP_MOVE_SYNC);
    gsp_stats local;
    memset(&local, 0, sizeof(local));
    Lap total(s), lap(s);

    MoveBuffers mb;
    alloc_move_state(mb, n0);
    mb.repeats = o.wave_repeats;
    mb.no_return_from = o.no_return_from;
    double *K = arena().get<double>(n0);
    uint32_t *labels = arena().get<uint32_t>(n0);
    uint32_t *Cd = arena().get<uint32_t>(n0);
    uint32_t *first = arena().get<uint32_t>(n0);
    uint8_t *used = arena().get<uint8_t>(n0);
    uint32_t *gid = arena().get<uint32_t>(n0);   // graph of each current-level vertex
    uint32_t *gid0 = arena().get<uint32_t>(n0);  // graph of each input vertex
    double *m_g = arena().get<double>(G);
    double *minv_g = arena().get<double>(G);
    double *dq_g = arena().get<double>(G);
    uint32_t *k_g = arena().get<uint32_t>(G);
    uint8_t *live = arena().get<uint8_t>(G);
    uint8_t *done = arena().get<uint8_t>(G);
    uint8_t *sel = arena().get<uint8_t>(G);
    uint64_t *gvo = arena().get<uint64_t>((size_t)G + 1);
    uint64_t *gvo0 = arena().get<uint64_t>((size_t)G + 1);
    // GSP-Leiden: refined partition, its dense ids, the bound communities
    // collapsed and dense, 2m of each graph
    const bool refine = o.refine != 0;
    uint32_t *Rf = refine ? arena().get<uint32_t>(n0) : nullptr;
    uint32_t *Bl = refine ? arena().get<uint32_t>(n0) : nullptr;
    uint32_t *Bd = refine ? arena().get<uint32_t>(n0) : nullptr;
    double *two_m_g = refine ? arena().get<double>(G) : nullptr;
    mb.K = K;
    mb.gid = gid;
    mb.m_g = m_g;
    mb.minv_g = minv_g;
    uint64_t *goff[2];
    uint32_t *gtgt[2];
    double *gw[2];
    for (int b = 0; b < 2; b++) {
        goff[b] = arena().get<uint64_t>((size_t)n0 + 1);
        gtgt[b] = arena().get<uint32_t>(g0.nnz + 1);
        gw[b] = arena().get<double>(g0.nnz + 1);
    }
    std::vector<uint64_t> hvo(h_gvo0, h_gvo0 + G + 1);
    GSP_CUDA(cudaMemcpyAsync(gvo0, hvo.data(), sizeof(uint64_t) * (G + 1), cudaMemcpyHostToDevice, s));
    GSP_CUDA(cudaMemcpyAsync(gvo, gvo0, sizeof(uint64_t) * (G + 1), cudaMemcpyDeviceToDevice, s));
    k_graph_of<<<grid_for(n0, 256), 256, 0, s>>>(gvo0, G, n0, gid0);
    GSP_CHECK_LAUNCH();
    {
        size_t mk = arena().mark();
        unsigned long long *bad = arena().get<unsigned long long>(1);
        GSP_CUDA(cudaMemsetAsync(bad, 0, sizeof(*bad), s));
        if (g0.nnz) {
            const unsigned grid = std::min(grid_for(g0.nnz, 256 * CROSS_UNROLL, sms(8)),
                                           resident_grid((const void *)k_cross_edges, 256, 0, 8));
            k_cross_edges<<<grid, 256, 0, s>>>(g0.off, g0.tgt, gid0, gvo0, n0, g0.nnz, bad);
            GSP_CHECK_LAUNCH();
        }
        unsigned long long hb = 0;
        GSP_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        arena().release(mk);
        GSP_REQUIRE(hb == 0, "%llu edges cross graphs of the batch", hb);
    }
    GSP_CUDA(cudaMemcpyAsync(gid, gid0, sizeof(uint32_t) * n0, cudaMemcpyDeviceToDevice, s));
    GSP_CUDA(cudaMemsetAsync(done, 0, G, s));
    iota_u32(membership, n0, s);

    std::vector<uint8_t> h_done(G, 0), h_live(G, 0), h_sel(G, 0);
    std::vector<int> h_li(G, 0);
    std::vector<uint32_t> h_k(G, 0), h_kr(G, 0);
    std::vector<double> h_m(G, 0.0), h_minv(G, 0.0), h_two_m(G, 0.0);
    DevGraph cur = g0;
    double tau = o.tolerance;
    const bool split_pass = o.split != GSP_SPLIT_NONE && o.split_when == GSP_SPLIT_PASS;
    uint32_t *Cp = mb.C;
    int pb = 0, passes = 0;
    // exact integer unit of the input weights (INT_MIN: float64 sums), valid
    // for every pass: aggregated weights are sums of input weights
    int lsb_cache = exact_lsb(g0, s);
    mb.lsb = lsb_cache;
    uint32_t remaining = G;
    for (int lp = 0; lp < o.max_passes && remaining; lp++) {
        const uint32_t nv = cur.n;
        size_t pass_mark = arena().mark();
        lap();
        // K' = Sigma' = vertexWeights(G'), C' = identity; each graph's m
        vertex_weights(cur, K, mb.m_dev, s, lsb_cache);
        GSP_CUDA(cudaMemsetAsync(m_g, 0, sizeof(double) * G, s));
        k_graph_m<<<grid_for(nv, 256), 256, 0, s>>>(K, gid, nv, m_g);
        GSP_CHECK_LAUNCH();
        GSP_CUDA(cudaMemcpyAsync(h_m.data(), m_g, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        for (uint32_t gi = 0; gi < G; gi++) {
            h_live[gi] = !h_done[gi] && h_m[gi] > 0.0;
            h_li[gi] = 0;
            h_minv[gi] = h_m[gi] > 0.0 ? 1.0 / h_m[gi] : 0.0;  // graphs without edges are never scored
        }
        GSP_CUDA(cudaMemcpyAsync(live, h_live.data(), G, cudaMemcpyHostToDevice, s));
        GSP_CUDA(cudaMemcpyAsync(minv_g, h_minv.data(), sizeof(double) * G, cudaMemcpyHostToDevice, s));
        if (refine && lp > 0) {
            // each super-vertex starts in the bound community of its members
            sigma_from_membership(mb.C, K, mb.Sigma, mb.size, nv, s);
        } else {
            GSP_CUDA(cudaMemcpyAsync(mb.Sigma, K, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
            iota_u32(mb.C, nv, s);
            k_fill_ones<<<grid_for(nv, 256), 256, 0, s>>>(mb.size, nv);
            GSP_CHECK_LAUNCH();
        }
        reset_left(mb, nv, s);
        k_set_active<<<grid_for(nv, 256), 256, 0, s>>>(mb.act, gid, live, nv);
        GSP_CHECK_LAUNCH();
        GSP_CUDA(cudaMemsetAsync(mb.mark, 0, nv, s));
        Classes cl;
        classify_vertices(cur, cl, W, s, gid, gvo);
        alloc_pool(mb, cl, s);
        float ms_other = lap();
        mb.dq_g = dq_g;
        BatchMove mr = batch_move_loop(cur, cl, mb, G, tau, o, h_live, h_li, live, s);
        mb.dq_g = nullptr;
        float ms_move = lap();
        Cp = mb.C;
        if (split_pass) {
            split_labels(cur, cl, Cp, o.split, labels, s);
            Cp = labels;
        }
        // |Gamma| of each graph (communities after the split)
        GSP_CUDA(cudaMemsetAsync(used, 0, nv, s));
        GSP_CUDA(cudaMemsetAsync(k_g, 0, sizeof(uint32_t) * G, s));
        k_mark_ids<<<grid_for(nv, 256), 256, 0, s>>>(Cp, nv, used);
        GSP_CHECK_LAUNCH();
        k_count_ids<<<grid_for(nv, 256), 256, 0, s>>>(used, gid, nv, k_g);
        GSP_CHECK_LAUNCH();
        GSP_CUDA(cudaMemcpyAsync(h_k.data(), k_g, sizeof(uint32_t) * G, cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        passes = lp + 1;
        // GSP-Leiden: each graph's refinement of its bound communities; the
        // low-shrink test counts refined communities
        float ms_ref = 0.0f, ms_split_part = 0.0f;
        if (refine) {
            for (uint32_t gi = 0; gi < G; gi++) h_two_m[gi] = 2.0 * h_m[gi];
            GSP_CUDA(cudaMemcpyAsync(two_m_g, h_two_m.data(), sizeof(double) * G, cudaMemcpyHostToDevice, s));
            RefineBatch rb;
            rb.gid = gid;
            rb.two_m_g = two_m_g;
            rb.gvo = gvo;
            ms_split_part = lap();
            refine_partition(cur, cl, Cp, Rf, K, 0.0, o.refine_theta, o.seed, (uint32_t)lp,
                             o.precision == GSP_PREC_FP64, s, rb);
            GSP_CUDA(cudaMemsetAsync(used, 0, nv, s));
            GSP_CUDA(cudaMemsetAsync(k_g, 0, sizeof(uint32_t) * G, s));
            k_mark_ids<<<grid_for(nv, 256), 256, 0, s>>>(Rf, nv, used);
            GSP_CHECK_LAUNCH();
            k_count_ids<<<grid_for(nv, 256), 256, 0, s>>>(used, gid, nv, k_g);
            GSP_CHECK_LAUNCH();
            GSP_CUDA(cudaMemcpyAsync(h_kr.data(), k_g, sizeof(uint32_t) * G, cudaMemcpyDeviceToHost, s));
            GSP_CUDA(cudaStreamSynchronize(s));
            ms_ref = lap();
        }
        // per-graph convergence: l_i <= 1 (converged) or |Gamma|/|Gamma_old| > tau_agg
        uint32_t finishing = 0, k_open = 0;
        int max_li = 0;
        for (uint32_t gi = 0; gi < G; gi++) {
            h_sel[gi] = 0;
            if (h_done[gi]) continue;
            max_li = std::max(max_li, h_li[gi]);
            k_open += h_k[gi];
            const uint64_t ng = hvo[gi + 1] - hvo[gi];
            const uint32_t kk = refine ? h_kr[gi] : h_k[gi];
            if (h_li[gi] <= 1 || (double)kk / (double)ng > o.aggregation_tolerance) {
                h_sel[gi] = 1;
                finishing++;
            }
        }
        float ms_split = ms_split_part + lap();
        if (lp < GSP_MAX_PASS_STATS) {
            local.iterations[lp] = max_li;
            local.vertices[lp] = nv;
            local.communities[lp] = k_open;
            if (refine) {
                uint32_t kr_open = 0;
                for (uint32_t gi = 0; gi < G; gi++)
                    if (!h_done[gi]) kr_open += h_kr[gi];
                local.refined[lp] = kr_open;
                local.ms_refine[lp] = ms_ref;
            }
            local.edges[lp] = cur.nnz;
            local.ms_move[lp] = ms_move;
            local.ms_split[lp] = ms_split;
            local.ms_other[lp] = ms_other;
            local.vertices_processed[lp] = mr.vertices;
            local.edges_scanned[lp] = mr.edges;
            local.move_bytes[lp] = mr.bytes;
            local.ms_move_kernels[lp] = mr.ms_kernels;
        }
        if (finishing) {
            to_representatives(membership, Cp, nv, gid0, n0, sel, h_sel, first, s);
            for (uint32_t gi = 0; gi < G; gi++)
                if (h_sel[gi]) {
                    h_done[gi] = 1;
                    remaining--;
                }
            GSP_CUDA(cudaMemcpyAsync(done, h_done.data(), G, cudaMemcpyHostToDevice, s));
        }
        if (!remaining) break;
        // open graphs: renumber, lookup, aggregate, tau scaling; finished
        // graphs collapse to one super-vertex each
        if (refine) {  // the bound communities, collapsed the same way, for the next pass's start
            k_collapse<<<grid_for(nv, 256), 256, 0, s>>>(Cp, gid, done, gvo, nv, Bl);
            GSP_CHECK_LAUNCH();
        }
        k_collapse<<<grid_for(nv, 256), 256, 0, s>>>(refine ? Rf : Cp, gid, done, gvo, nv, labels);
        GSP_CHECK_LAUNCH();
        const uint32_t k = renumber(nv, labels, Cd, s);
        k_lookup_open<<<grid_for(n0, 256), 256, 0, s>>>(membership, Cd, gid0, done, n0);
        GSP_CHECK_LAUNCH();
        DevGraph nxt;
        nxt.n = k;
        nxt.off = goff[pb];
        nxt.tgt = gtgt[pb];
        nxt.w = gw[pb];
        nxt.wt = GSP_W_F64;
        nxt.nnz = aggregate(cur, Cd, k, goff[pb], gtgt[pb], gw[pb], s, /*sorted=*/false, &lsb_cache);
        pb ^= 1;
        cur = nxt;
        tau = tau / o.tolerance_drop;
        std::vector<uint64_t> nvo(G + 1, 0);  // the next level's vertex ranges
        for (uint32_t gi = 0; gi < G; gi++) {
            const uint64_t ng = hvo[gi + 1] - hvo[gi];
            nvo[gi + 1] = nvo[gi] + (h_done[gi] ? (ng ? 1 : 0) : (refine ? h_kr[gi] : h_k[gi]));
        }
        GSP_REQUIRE(nvo[G] == k, "batched aggregation: %llu super-vertices expected, %u made",
                    (unsigned long long)nvo[G], k);
        hvo.swap(nvo);
        if (refine) {  // super-vertex r starts the next pass in the bound community of its members
            renumber(nv, Bl, Bd, s);
            scatter_bound(Cd, Bd, mb.C, nv, s);
        }
        float ms_agg = lap();
        if (lp < GSP_MAX_PASS_STATS) local.ms_aggregate[lp] = ms_agg;
        arena().release(pass_mark);
        GSP_CUDA(cudaMemcpyAsync(gvo, hvo.data(), sizeof(uint64_t) * (G + 1), cudaMemcpyHostToDevice, s));
        k_graph_of<<<grid_for(k, 256), 256, 0, s>>>(gvo, G, k, gid);
        GSP_CHECK_LAUNCH();
        if (!refine) iota_u32(mb.C, cur.n, s);
        Cp = mb.C;
    }
    if (remaining) {  // max_passes reached: the open graphs keep their last labels
        for (uint32_t gi = 0; gi < G; gi++) h_sel[gi] = !h_done[gi];
        to_representatives(membership, Cp, cur.n, gid0, n0, sel, h_sel, first, s);
    }
    if (o.split != GSP_SPLIT_NONE && o.split_when == GSP_SPLIT_LAST) {
        Classes cl;
        classify_vertices(g0, cl, 1, s);
        split_labels(g0, cl, membership, o.split, labels, s);
        GSP_CUDA(cudaMemcpyAsync(membership, labels, sizeof(uint32_t) * n0, cudaMemcpyDeviceToDevice, s));
    }
    const uint32_t kf = canonical_numbering(n0, membership, s);
    // global ids here: no community spans two graphs
    local.disconnected = o.count_disconnected ? count_disconnected(g0, membership, nullptr, s) : GSP_NOT_COUNTED;
    // per-graph Equation 1, then graph-local numbering
    {
        size_t mk = arena().mark();
        double *two_m = arena().get<double>(G);
        double *intra = arena().get<double>(G);
        double *sumsq = arena().get<double>(G);
        double *Sig = arena().get<double>(kf);
        uint32_t *comm_graph = arena().get<uint32_t>(kf);
        uint32_t *base = arena().get<uint32_t>(G);
        GSP_CUDA(cudaMemsetAsync(two_m, 0, sizeof(double) * G, s));
        GSP_CUDA(cudaMemsetAsync(intra, 0, sizeof(double) * G, s));
        GSP_CUDA(cudaMemsetAsync(sumsq, 0, sizeof(double) * G, s));
        GSP_CUDA(cudaMemsetAsync(Sig, 0, sizeof(double) * kf, s));
#define GSP_QROWS(WT, AV)                                                                                 \
    k_graph_q_rows<WT, AV><<<grid_for(n0, 256), 256, 0, s>>>(g0.off, g0.tgt, static_cast<const WT *>(g0.w),   \
                                                              membership, gid0, n0, two_m, intra, Sig, comm_graph, \
                                                              lsb_cache)
        if (g0.wt == GSP_W_F64) {
            if (lsb_cache != INT_MIN) GSP_QROWS(double, unsigned long long);
            else GSP_QROWS(double, double);
        } else {
            if (lsb_cache != INT_MIN) GSP_QROWS(float, unsigned long long);
            else GSP_QROWS(float, double);
        }
#undef GSP_QROWS
        GSP_CHECK_LAUNCH();
        k_graph_q_sq<<<grid_for(kf, 256), 256, 0, s>>>(Sig, comm_graph, kf, sumsq);
        GSP_CHECK_LAUNCH();
        k_graph_q_final<<<grid_for(G, 256), 256, 0, s>>>(two_m, intra, sumsq, membership, gvo0, G, q_out, base);
        GSP_CHECK_LAUNCH();
        k_localise<<<grid_for(n0, 256), 256, 0, s>>>(membership, gid0, base, n0);
        GSP_CHECK_LAUNCH();
        std::vector<double> hq(G);
        GSP_CUDA(cudaMemcpyAsync(hq.data(), q_out, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        double qs = 0;
        for (double x : hq) qs += x;
        local.modularity = qs / G;  // mean over the graphs
        arena().release(mk);
    }
    local.passes = passes;
    local.final_communities = kf;
    local.ms_total = total();
    local.workspace_bytes = workspace_peak();
    if (st) *st = local;
    cudaEvent_t out = pool_event();
    GSP_CUDA(cudaEventRecord(out, s));
    GSP_CUDA(cudaStreamWaitEvent(caller, out, 0));
}

void check_batch(uint32_t num_graphs, const uint64_t *gvo, uint32_t n, const gsp_opts &o) {
    GSP_REQUIRE(o.prune == GSP_PRUNE_FLAGS, "batched runs support flag pruning only");
    GSP_REQUIRE(num_graphs >= 1 && gvo, "need at least one graph and its vertex offsets");
    GSP_REQUIRE(gvo[0] == 0 && gvo[num_graphs] == n, "graph_vertex_offsets must run from 0 to n");
    for (uint32_t g = 0; g < num_graphs; g++)
        GSP_REQUIRE(gvo[g + 1] >= gvo[g], "graph_vertex_offsets must not decrease");
}

}  // namespace gsp

using namespace gsp;

extern "C" gsp_status gsp_louvain_batched(uint32_t num_graphs, const uint64_t *graph_vertex_offsets,
                                          const uint64_t *offsets, const uint32_t *targets, const float *weights,
                                          uint32_t n, uint64_t nnz, const gsp_opts *opts, uint32_t *membership,
                                          double *modularity, gsp_stats *stats) {
    try {
        gsp_opts o;
        if (opts) o = *opts;
        else gsp_default_opts(&o);
        check_opts(o);
        check_batch(num_graphs, graph_vertex_offsets, n, o);
        GSP_REQUIRE(membership && modularity, "membership and modularity must not be NULL");
        DevGraph g = make_graph(offsets, targets, weights, GSP_W_F32, n, nnz);
        cudaStream_t s = static_cast<cudaStream_t>(o.stream);
        UserWorkspace uw(o.workspace, o.workspace_bytes);
        arena().reset();
        check_graph(offsets, targets, weights, n, nnz, s);
        louvain_batched_run(g, num_graphs, graph_vertex_offsets, o, membership, modularity, stats, s);
        GSP_CUDA(cudaStreamSynchronize(s));
        return GSP_OK;
    } catch (const gsp::Error &e) {
        return e.status;
    } catch (...) {
        set_error("unexpected C++ exception");
        return GSP_ERR_CUDA;
    }
}
