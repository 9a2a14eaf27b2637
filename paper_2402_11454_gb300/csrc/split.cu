// split.cu -- the split step of GSP-Louvain (Section 4.1): break every
// community into the connected components of its intra-community edges.
//
//   LP  (Algorithm 2): labels start at the vertex id; every sweep each vertex
//        takes the minimum label over its same-community neighbours, in place,
//        until a sweep changes nothing.  Labels only decrease, so the in-place
//        updates of concurrent threads converge to the same fixpoint.
//   LPP (Algorithm 2 with pruning): only vertices flagged unprocessed are
//        visited; a vertex whose label drops flags its same-community
//        neighbours.
//   SV  (not in the paper): hooking and shortcutting (Shiloach-Vishkin) on
//        the intra-community edges, O(log n) sweeps on high-diameter graphs.
//   BFS (Algorithm 3): rounds of multi-source, level-synchronous,
//        frontier-compacted BFS.  In each round the seed of a community is its
//        smallest unvisited vertex, found with atomicMin; vertices are claimed
//        with atomicCAS on their label.  The busy flags of the paper's
//        per-thread BFS become unnecessary: every community is searched from
//        one seed per round by the whole GPU.
// The seed of a round is the smallest vertex of its component (the smaller
// vertices of the community are already visited, and components are
// disjoint), so every mode yields label = smallest vertex id of the component.
#include "internal.cuh"

namespace gsp {

template <typename T> __device__ __forceinline__ T ldcg_(const T *p) { return __ldcg(p); }
__device__ __forceinline__ uint8_t ldcg_(const uint8_t *p) {
    return (uint8_t)__ldcg(reinterpret_cast<const unsigned char *>(p));
}

// min over the same-community neighbours' labels of the edges b + first,
// b + first + step, ... < e; four gathers of C and lab in flight per thread.
__device__ __forceinline__ uint32_t min_label(const uint32_t *__restrict__ tgt, const uint32_t *__restrict__ C,
                                              const uint32_t *lab, uint32_t ci, uint64_t b, uint64_t e,
                                              uint32_t first, uint32_t step, uint32_t mn) {
    uint64_t p = b + first;
    for (; p + 3 * (uint64_t)step < e; p += 4 * (uint64_t)step) {
        uint32_t j[4], cj[4];
#pragma unroll
        for (int u = 0; u < 4; u++) j[u] = tgt[p + (uint64_t)u * step];
#pragma unroll
        for (int u = 0; u < 4; u++) cj[u] = C[j[u]];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (cj[u] == ci) mn = min(mn, ldcg_(lab + j[u]));
    }
    for (; p < e; p += step) {
        const uint32_t j = tgt[p];
        if (C[j] == ci) mn = min(mn, ldcg_(lab + j));
    }
    return mn;
}

// ----------------------------------------------------------------- LP / LPP
// HOOK (the hooking split): besides lowering its own label, a vertex whose
// smallest neighbouring label mn is below its label p hooks p's tree under
// mn (lab[p] = min(lab[p], mn)); with the shortcut kernel between sweeps the
// labels then converge in O(log n) sweeps instead of O(diameter).
template <int G, bool PRUNE, bool HOOK = false>
__global__ void __launch_bounds__(256) k_lp_group(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tgt,
                                                  const uint32_t *__restrict__ C, uint32_t *lab, uint8_t *flag,
                                                  const uint32_t *__restrict__ list, uint32_t count,
                                                  unsigned long long *changed) {
    const int lane = threadIdx.x % G;
    const unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    unsigned long long ch = 0;
    // 32 list entries per warp and round: each lane reads (and, pruned,
    // clears) one flag; the flagged vertices are dealt to the warp's groups
    constexpr int NGW = 32 / G;
    const int wl = threadIdx.x & 31, gw = wl / G;
    const uint32_t wbase = blockIdx.x * 8 + (threadIdx.x >> 5), wstep = gridDim.x * 8;
    for (uint64_t kb = 0; wbase + kb * wstep < count; kb += 32) {
        const uint64_t my = wbase + (kb + wl) * wstep;
        uint32_t vi = 0;
        int claim = 0;
        if (my < count) {
            vi = list[my];
            claim = 1;
            if (PRUNE) {
                claim = ldcg_(flag + vi);
                if (claim) flag[vi] = 0;
            }
        }
        const unsigned amask = __ballot_sync(0xFFFFFFFFu, claim);
        const int nact = __popc(amask);
        // a consumed flag was set after its setter's label store: order the
        // label reads below after the flag reads
        if (PRUNE && nact) __threadfence();
        for (int r0 = 0; r0 < nact; r0 += NGW) {
        const int qa = r0 + gw;
        const uint32_t i = __shfl_sync(0xFFFFFFFFu, vi, qa < nact ? select_bit(amask, qa) : 0);
        if (qa >= nact) continue;
        uint32_t ci = C[i];
        uint32_t cur = ldcg_(lab + i);
        uint32_t mn = cur;
        uint64_t b = off[i], e = off[i + 1];
        mn = min_label(tgt, C, lab, ci, b, e, lane, G, mn);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(gmask, mn, o));
        if (mn < cur) {
            if (lane == 0) {
                if (HOOK) {
                    atomicMin(lab + cur, mn);
                    atomicMin(lab + i, mn);
                } else {
                    lab[i] = mn;
                }
                ch++;
            }
            if (PRUNE) {
                // the new label must be visible before any neighbour sees its
                // flag (a neighbour that consumes the flag re-reads it once)
                __syncwarp(gmask);
                __threadfence();
            }
            if (PRUNE)
                for (uint64_t p = b + lane; p < e; p += G) {
                    uint32_t j = tgt[p];
                    if (C[j] == ci) flag[j] = 1;
                }
        }
        __syncwarp(gmask);
        }
    }
    __shared__ unsigned long long red[32];
    ch = block_sum(ch, red);
    if (threadIdx.x == 0 && ch) atomicAdd(changed, ch);
}

template <bool PRUNE, bool HOOK = false>
__global__ void __launch_bounds__(256) k_lp_block(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tgt,
                                                  const uint32_t *__restrict__ C, uint32_t *lab, uint8_t *flag,
                                                  const uint32_t *__restrict__ list, uint32_t count,
                                                  unsigned long long *changed) {
    __shared__ uint32_t red[32];
    __shared__ uint32_t s_todo[256], s_ntodo, s_wcnt[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long ch = 0;
    // 256 list entries per block and round (blockIdx.x + k * gridDim.x):
    // each thread reads (and, pruned, clears) one flag; the flagged vertices
    // are listed in shared memory and processed one by one
    for (uint64_t kb = 0; blockIdx.x + kb * gridDim.x < count; kb += blockDim.x) {
        const uint64_t my = blockIdx.x + (kb + threadIdx.x) * gridDim.x;
        uint32_t vi = 0;
        int claim = 0;
        if (my < count) {
            vi = list[my];
            claim = 1;
            if (PRUNE) {
                claim = ldcg_(flag + vi);
                if (claim) flag[vi] = 0;
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
            for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s_wcnt[k];
            s_ntodo = t;
        }
        __syncthreads();
        const uint32_t ntodo = s_ntodo;
        if (PRUNE && ntodo) __threadfence();  // flags consumed before the labels are read
    for (uint32_t kk = 0; kk < ntodo; kk++) {
        const uint32_t i = s_todo[kk];
        __syncthreads();  // previous vertex done with red
        uint32_t ci = C[i];
        uint32_t cur = ldcg_(lab + i);
        uint32_t mn = cur;
        uint64_t b = off[i], e = off[i + 1];
        mn = min_label(tgt, C, lab, ci, b, e, threadIdx.x, blockDim.x, mn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mn;
        __syncthreads();
        mn = red[0];
        for (int t = 1; t < (int)(blockDim.x >> 5); t++) mn = min(mn, red[t]);
        if (mn < cur) {
            if (threadIdx.x == 0) {
                if (HOOK) {
                    atomicMin(lab + cur, mn);
                    atomicMin(lab + i, mn);
                } else {
                    lab[i] = mn;
                }
                ch++;
            }
            if (PRUNE) {  // the new label visible before the neighbours' flags
                __syncthreads();
                __threadfence();
            }
            if (PRUNE)
                for (uint64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
                    uint32_t j = tgt[p];
                    if (C[j] == ci) flag[j] = 1;
                }
        }
    }
    }
    __shared__ unsigned long long r2[32];
    __syncthreads();
    ch = block_sum(ch, r2);
    if (threadIdx.x == 0 && ch) atomicAdd(changed, ch);
}

static void split_lp(const DevGraph &g, const Classes &cl, const uint32_t *C, bool prune, uint32_t *lab,
                     cudaStream_t s) {
    size_t mk = arena().mark();
    uint8_t *flag = prune ? arena().get<uint8_t>(g.n) : nullptr;
    unsigned long long *changed = arena().get<unsigned long long>(1);
    iota_u32(lab, g.n, s);
    if (prune) GSP_CUDA(cudaMemsetAsync(flag, 1, g.n, s));
    // every class with all its waves (class c spans [cls_begin(c), cls_begin(c+1)))
    auto cnt = [&](int c) { return cl.cls_count(c); };
    auto lst = [&](int c) { return cl.list + cl.cls_begin(c); };
    const unsigned maxg = sms(8);
    uint32_t nbig = cl.cls_count(CLS_BLOCK) + cl.cls_count(CLS_BIG) + cl.cls_count(CLS_HUGE);
    for (int it = 0; it < (1 << 30); it++) {
        GSP_CUDA(cudaMemsetAsync(changed, 0, sizeof(unsigned long long), s));
#define LPG(G, CLS)                                                                                  \
    if (cnt(CLS)) {                                                                                  \
        if (prune)                                                                                   \
            k_lp_group<G, true><<<grid_for((uint64_t)cnt(CLS) * G, 256, maxg), 256, 0, s>>>(        \
                g.off, g.tgt, C, lab, flag, lst(CLS), cnt(CLS), changed);                            \
        else                                                                                         \
            k_lp_group<G, false><<<grid_for((uint64_t)cnt(CLS) * G, 256, maxg), 256, 0, s>>>(       \
                g.off, g.tgt, C, lab, flag, lst(CLS), cnt(CLS), changed);                            \
        GSP_CHECK_LAUNCH();                                                                          \
    }
        LPG(4, CLS_G4) LPG(8, CLS_G8) LPG(16, CLS_G16) LPG(32, CLS_G32) LPG(32, CLS_W512)
#undef LPG
        if (nbig) {
            if (prune)
                k_lp_block<true><<<grid_for(nbig, 1, sms(4)), 256, 0, s>>>(g.off, g.tgt, C, lab, flag,
                                                                              lst(CLS_BLOCK), nbig, changed);
            else
                k_lp_block<false><<<grid_for(nbig, 1, sms(4)), 256, 0, s>>>(g.off, g.tgt, C, lab, flag,
                                                                               lst(CLS_BLOCK), nbig, changed);
            GSP_CHECK_LAUNCH();
        }
        unsigned long long h;
        GSP_CUDA(cudaMemcpyAsync(&h, changed, sizeof(h), cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        if (h == 0) break;
    }
    arena().release(mk);
}

// ------------------------------------------------------------ hooking split
// Shiloach-Vishkin-style connected components restricted to intra-community
// edges: hooking sweeps (k_lp_group/k_lp_block with HOOK) alternate with a
// shortcut pass that points every vertex at the root of its tree.  Labels
// only decrease and always name a vertex of the same component, so at the
// fixpoint every component carries its smallest vertex id, as LP and BFS.
__global__ void k_sv_shortcut(uint32_t *lab, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t x = ldcg_(lab + i);
        // lab[x] <= x, so the chain strictly decreases and ends at a root
        for (;;) {
            const uint32_t y = ldcg_(lab + x);
            if (y == x) break;
            x = y;
        }
        lab[i] = x;
    }
}

static void split_sv(const DevGraph &g, const Classes &cl, const uint32_t *C, uint32_t *lab, cudaStream_t s) {
    size_t mk = arena().mark();
    unsigned long long *changed = arena().get<unsigned long long>(1);
    iota_u32(lab, g.n, s);
    auto cnt = [&](int c) { return cl.cls_count(c); };
    auto lst = [&](int c) { return cl.list + cl.cls_begin(c); };
    const unsigned maxg = sms(8);
    const uint32_t nbig = cl.cls_count(CLS_BLOCK) + cl.cls_count(CLS_BIG) + cl.cls_count(CLS_HUGE);
    for (int it = 0; it < (1 << 30); it++) {
        GSP_CUDA(cudaMemsetAsync(changed, 0, sizeof(unsigned long long), s));
#define SVG(G, CLS)                                                                                            \
    if (cnt(CLS)) {                                                                                            \
        k_lp_group<G, false, true><<<grid_for((uint64_t)cnt(CLS) * G, 256, maxg), 256, 0, s>>>(               \
            g.off, g.tgt, C, lab, nullptr, lst(CLS), cnt(CLS), changed);                                       \
        GSP_CHECK_LAUNCH();                                                                                    \
    }
        SVG(4, CLS_G4) SVG(8, CLS_G8) SVG(16, CLS_G16) SVG(32, CLS_G32) SVG(32, CLS_W512)
#undef SVG
        if (nbig) {
            k_lp_block<false, true><<<grid_for(nbig, 1, sms(4)), 256, 0, s>>>(g.off, g.tgt, C, lab, nullptr,
                                                                               lst(CLS_BLOCK), nbig, changed);
            GSP_CHECK_LAUNCH();
        }
        k_sv_shortcut<<<grid_for(g.n, 256), 256, 0, s>>>(lab, g.n);
        GSP_CHECK_LAUNCH();
        unsigned long long h;
        GSP_CUDA(cudaMemcpyAsync(&h, changed, sizeof(h), cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        if (h == 0) break;
    }
    arena().release(mk);
}

// --------------------------------------------------------------------- BFS
// Seeds of a round: the smallest unvisited vertex of every community that
// still has one.  `cand` lists the vertices unvisited after the previous
// round (all vertices in the first round).
__global__ void k_bfs_seed_min(const uint32_t *__restrict__ C, const uint32_t *__restrict__ lab,
                               const uint32_t *__restrict__ cand, const uint32_t *__restrict__ ncand, uint32_t n,
                               uint32_t *seed) {
    uint32_t cnt = cand ? *ncand : n;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        uint32_t v = cand ? cand[t] : t;
        if (lab[v] == EMPTY) atomicMin(seed + C[v], v);
    }
}

// Warp-aggregated append of the lanes with `want` set.
__device__ __forceinline__ void push_warp(bool want, uint32_t v, uint32_t *q, uint32_t *qn) {
    uint32_t ballot = __ballot_sync(0xFFFFFFFFu, want);
    if (!ballot) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(ballot) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(qn, (uint32_t)__popc(ballot));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (want) q[base + __popc(ballot & ((1u << lane) - 1u))] = v;
}

// Label the seeds and start the frontier; the other unvisited vertices form
// the candidate list of the next round.
__global__ void k_bfs_seed_push(const uint32_t *__restrict__ C, uint32_t *lab, const uint32_t *__restrict__ cand,
                                const uint32_t *__restrict__ ncand, uint32_t n, const uint32_t *__restrict__ seed,
                                uint32_t *q, uint32_t *qn, uint32_t *rest, uint32_t *nrest) {
    uint32_t cnt = cand ? *ncand : n;
    for (uint32_t t0 = blockIdx.x * blockDim.x; t0 < cnt; t0 += gridDim.x * blockDim.x) {
        uint32_t t = t0 + threadIdx.x;
        bool is_seed = false, keep = false;
        uint32_t v = 0;
        if (t < cnt) {
            v = cand ? cand[t] : t;
            if (lab[v] == EMPTY) {
                if (seed[C[v]] == v) {
                    lab[v] = v;
                    is_seed = true;
                } else {
                    keep = true;
                }
            }
        }
        push_warp(is_seed, v, q, qn);
        push_warp(keep, v, rest, nrest);
    }
}

__global__ void k_bfs_seed_reset(const uint32_t *__restrict__ C, const uint32_t *__restrict__ q,
                                 const uint32_t *__restrict__ qn, uint32_t *seed) {
    uint32_t cnt = *qn;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x)
        seed[C[q[t]]] = EMPTY;
}

constexpr uint32_t BFS_BIG = 1024;

__device__ __forceinline__ void bfs_visit_edges(const uint32_t *__restrict__ tgt, const uint32_t *__restrict__ C,
                                                uint32_t *lab, uint64_t p0, uint64_t e, uint64_t step, uint32_t cu,
                                                uint32_t lu, uint32_t *nq, uint32_t *nqn) {
    // all 32 lanes of the warp run the same trip count (push_warp ballots)
    for (uint64_t pb = p0; pb < e + (threadIdx.x & 31) && pb - (threadIdx.x & 31) < e; pb += step) {
        uint64_t p = pb;
        bool want = false;
        uint32_t j = 0;
        if (p < e) {
            j = tgt[p];
            if (C[j] == cu && ldcg_(lab + j) == EMPTY) want = atomicCAS(lab + j, EMPTY, lu) == EMPTY;
        }
        push_warp(want, j, nq, nqn);
    }
}

// One level: a warp per frontier vertex claims unvisited same-community
// neighbours with atomicCAS and appends them to the next frontier; frontier
// vertices of degree > BFS_BIG go to a list for k_bfs_expand_big.
__global__ void k_bfs_expand(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tgt,
                             const uint32_t *__restrict__ C, uint32_t *lab, const uint32_t *__restrict__ q,
                             const uint32_t *__restrict__ qn, uint32_t *nq, uint32_t *nqn, uint32_t *big,
                             uint32_t *nbig) {
    uint32_t cnt = *qn;
    int lane = threadIdx.x & 31;
    uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t = warp; t < cnt; t += nwarps) {
        uint32_t u = q[t];
        uint64_t b = off[u], e = off[u + 1];
        if (e - b > BFS_BIG) {
            if (lane == 0) big[atomicAdd(nbig, 1u)] = u;
            continue;
        }
        uint32_t cu = C[u], lu = ldcg_(lab + u);
        bfs_visit_edges(tgt, C, lab, b + lane, e, 32, cu, lu, nq, nqn);
    }
}

// The big frontier vertices: every warp of the grid strides over each one's
// edges in turn.
__global__ void k_bfs_expand_big(const uint64_t *__restrict__ off, const uint32_t *__restrict__ tgt,
                                 const uint32_t *__restrict__ C, uint32_t *lab, const uint32_t *__restrict__ big,
                                 const uint32_t *__restrict__ nbig, uint32_t *nq, uint32_t *nqn) {
    uint32_t cnt = *nbig;
    uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    for (uint32_t t = 0; t < cnt; t++) {
        uint32_t u = big[t];
        uint32_t cu = C[u], lu = ldcg_(lab + u);
        bfs_visit_edges(tgt, C, lab, off[u] + tid, off[u + 1], T, cu, lu, nq, nqn);
    }
}

// Rounds of multi-source BFS.  Levels are launched in batches of
// BFS_LEVEL_BATCH between host checks of the frontier size (an empty
// frontier makes the remaining launches of a batch return at once).
constexpr int BFS_LEVEL_BATCH = 6;

static void split_bfs(const DevGraph &g, const uint32_t *C, uint32_t *lab, cudaStream_t s) {
    size_t mk = arena().mark();
    uint32_t n = g.n;
    uint32_t *seed = arena().get<uint32_t>(n);
    uint32_t *fr[BFS_LEVEL_BATCH + 1];
    for (int k = 0; k <= BFS_LEVEL_BATCH; k++) fr[k] = nullptr;
    uint32_t *qa = arena().get<uint32_t>(n);
    uint32_t *qb = arena().get<uint32_t>(n);
    uint32_t *candA = arena().get<uint32_t>(n);
    uint32_t *candB = arena().get<uint32_t>(n);
    uint32_t *big = arena().get<uint32_t>(n);
    // counters: [0] seeds, [1] rest, [2 .. 2+BATCH] frontier sizes, big counts after
    uint32_t *cnts = arena().get<uint32_t>(4 + 2 * (BFS_LEVEL_BATCH + 1));
    uint32_t *ncandA = cnts + 0;  // candidate counts live beside the seed/rest counters
    GSP_CUDA(cudaMemsetAsync(lab, 0xFF, sizeof(uint32_t) * n, s));
    GSP_CUDA(cudaMemsetAsync(seed, 0xFF, sizeof(uint32_t) * n, s));
    const uint32_t *cand = nullptr;  // first round: every vertex
    uint32_t *cand_cnt = nullptr;
    uint32_t h_cand = n;
    uint32_t *cbuf[2] = {candA, candB};
    uint32_t *ccnt[2] = {cnts + 2 + 2 * (BFS_LEVEL_BATCH + 1), cnts + 3 + 2 * (BFS_LEVEL_BATCH + 1)};
    (void)ncandA;
    int cb = 0;
    for (int round = 0; h_cand > 0; round++) {
        uint32_t *rest = cbuf[cb], *nrest = ccnt[cb];
        uint32_t *qn = cnts + 0;
        GSP_CUDA(cudaMemsetAsync(cnts, 0, sizeof(uint32_t) * (2 + 2 * (BFS_LEVEL_BATCH + 1)), s));
        GSP_CUDA(cudaMemsetAsync(nrest, 0, sizeof(uint32_t), s));
        unsigned gr = grid_for(h_cand, 256);
        k_bfs_seed_min<<<gr, 256, 0, s>>>(C, lab, cand, cand_cnt, n, seed);
        GSP_CHECK_LAUNCH();
        k_bfs_seed_push<<<gr, 256, 0, s>>>(C, lab, cand, cand_cnt, n, seed, qa, qn, rest, nrest);
        GSP_CHECK_LAUNCH();
        k_bfs_seed_reset<<<gr, 256, 0, s>>>(C, qa, qn, seed);
        GSP_CHECK_LAUNCH();
        // levels, in batches
        uint32_t *q = qa, *nq = qb;
        uint32_t *fcnt = cnts + 2;        // fcnt[k]: frontier size of level k in the batch
        uint32_t *bcnt = cnts + 2 + (BFS_LEVEL_BATCH + 1);
        GSP_CUDA(cudaMemcpyAsync(fcnt, qn, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        for (;;) {
            for (int k = 0; k < BFS_LEVEL_BATCH; k++) {
                k_bfs_expand<<<sms(8), 256, 0, s>>>(g.off, g.tgt, C, lab, q, fcnt + k, nq, fcnt + k + 1, big,
                                                    bcnt + k);
                GSP_CHECK_LAUNCH();
                k_bfs_expand_big<<<sms(4), 256, 0, s>>>(g.off, g.tgt, C, lab, big, bcnt + k, nq,
                                                                 fcnt + k + 1);
                GSP_CHECK_LAUNCH();
                uint32_t *t = q; q = nq; nq = t;
            }
            uint32_t last;
            GSP_CUDA(cudaMemcpyAsync(&last, fcnt + BFS_LEVEL_BATCH, sizeof(last), cudaMemcpyDeviceToHost, s));
            GSP_CUDA(cudaStreamSynchronize(s));
            if (last == 0) break;
            GSP_CUDA(cudaMemcpyAsync(fcnt, fcnt + BFS_LEVEL_BATCH, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
            GSP_CUDA(cudaMemsetAsync(fcnt + 1, 0, sizeof(uint32_t) * BFS_LEVEL_BATCH, s));
            GSP_CUDA(cudaMemsetAsync(bcnt, 0, sizeof(uint32_t) * (BFS_LEVEL_BATCH + 1), s));
        }
        // vertices still unvisited become the next round's candidates
        GSP_CUDA(cudaMemcpyAsync(&h_cand, nrest, sizeof(h_cand), cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        cand = rest;
        cand_cnt = nrest;
        cb ^= 1;
    }
    arena().release(mk);
}

void split_labels(const DevGraph &g, const Classes &cl, const uint32_t *C, int mode, uint32_t *labels,
                  cudaStream_t s) {
    if (mode == GSP_SPLIT_BFS) split_bfs(g, C, labels, s);
    else if (mode == GSP_SPLIT_SV) split_sv(g, cl, C, labels, s);
    else split_lp(g, cl, C, mode == GSP_SPLIT_LPP, labels, s);
}

}  // namespace gsp
