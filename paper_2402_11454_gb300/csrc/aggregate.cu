// aggregate.cu -- aggregation phase of GSP-Louvain (Algorithm 5,
// louvainAggregate) on sm_103a.
//
//  1. community-vertex CSR: countCommunityVertices, exclusive scan, scatter;
//  2. super-vertex row bounds: communityTotalDegree, exclusive scan (the
//     paper's "holey" CSR with gaps);
//  3. per community, an open-addressing table over the edges of all members
//     (self-loops included) merges the weights per neighbouring community:
//       total degree <= 512  : one warp, 1024-slot table in shared memory
//       total degree <= 2048 : one block, 4096-slot table in shared memory
//       larger               : the whole grid, edge-chunk tasks combined in
//                              shared memory and published to a global table;
//  4. the rows are compacted (exclusive scan of the row lengths) and, for the
//     canonical form, each row is sorted by target: warp bitonic sort (<= 32
//     entries), block bitonic sort in shared memory (<= 2048), and one
//     segmented LSD radix sort for all longer rows together.  Inside a run
//     the rows stay unsorted: no later step depends on their order (moves,
//     split and aggregation sum exactly representable weights, and ties go
//     to the lowest id), so only the phase entry point sorts.
// Weights are stored in float64; sums of float32-exact weights are exact in
// float64, so every merged weight is order-independent and the output is
// canonical.  The tables accumulate in integer units of the weights' lowest
// set bit (64-bit integer atomics, native in shared memory) whenever the total
// weight stays below 2^52 such units, and in float64 otherwise; the two give
// the same sums.
#include <climits>
#include <cmath>

#include "internal.cuh"

namespace gsp {

enum { ACLS_W = 0, ACLS_B, ACLS_L, NUM_ACLS };
constexpr uint64_t ACLS_MAX[NUM_ACLS] = {512, 2048, ~0ull};
enum { RCLS_W = 0, RCLS_B, RCLS_L, NUM_RCLS };
constexpr uint64_t RCLS_MAX[NUM_RCLS] = {32, 2048, ~0ull};

template <typename WT>
__global__ void k_agg_count(const uint64_t *__restrict__ off, const uint32_t *__restrict__ Cd, uint32_t n,
                            uint32_t *cnt, unsigned long long *cdeg) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t c = Cd[v];
        atomicAdd(cnt + c, 1u);
        uint64_t deg = off[v + 1] - off[v];
        if (deg) atomicAdd(cdeg + c, (unsigned long long)deg);
    }
}

__global__ void k_agg_scatter(const uint32_t *__restrict__ Cd, uint32_t n, const uint64_t *__restrict__ coff,
                              uint32_t *cnt, uint32_t *cverts) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t c = Cd[v];
        uint32_t pos = atomicSub(cnt + c, 1u) - 1u;
        cverts[coff[c] + pos] = v;
    }
}

// Classify ids 0..k-1 by a 64-bit size (entries of size 0 are left out).
template <int NC>
__global__ void k_cls_count(const uint64_t *__restrict__ sz, uint32_t k, const uint64_t *maxes, uint32_t *counts) {
    __shared__ uint32_t sc[NC];
    if (threadIdx.x < NC) sc[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
        uint64_t x = sz[c];
        if (!x) continue;
        int cls = 0;
        while (cls < NC - 1 && x > maxes[cls]) cls++;
        atomicAdd(&sc[cls], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NC && sc[threadIdx.x]) atomicAdd(counts + threadIdx.x, sc[threadIdx.x]);
}

template <int NC>
__global__ void k_cls_fill(const uint64_t *__restrict__ sz, uint32_t k, const uint64_t *maxes, uint32_t *cursor,
                           uint32_t *list) {
    int lane = threadIdx.x & 31;
    for (uint32_t c0 = blockIdx.x * blockDim.x; c0 < k; c0 += gridDim.x * blockDim.x) {
        uint32_t c = c0 + threadIdx.x;
        int cls = -1;
        if (c < k) {
            uint64_t x = sz[c];
            if (x) {
                cls = 0;
                while (cls < NC - 1 && x > maxes[cls]) cls++;
            }
        }
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, cls);
        int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && cls >= 0) base = atomicAdd(cursor + cls, (uint32_t)__popc(peers));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (cls >= 0) list[base + __popc(peers & ((1u << lane) - 1u))] = c;
    }
}

struct IdClasses {
    uint32_t *list = nullptr;
    uint32_t start[4] = {0, 0, 0, 0};
};

template <int NC>
static void classify_ids(const uint64_t *sz, uint32_t k, const uint64_t (&maxes)[NC], IdClasses &ic, cudaStream_t s) {
    uint64_t *dmax = arena().get<uint64_t>(NC);
    uint32_t *counts = arena().get<uint32_t>(2 * NC);
    GSP_CUDA(cudaMemcpyAsync(dmax, maxes, sizeof(uint64_t) * NC, cudaMemcpyHostToDevice, s));
    GSP_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * NC, s));
    unsigned gr = grid_for(k, 256, sms(8));
    k_cls_count<NC><<<gr, 256, 0, s>>>(sz, k, dmax, counts);
    GSP_CHECK_LAUNCH();
    uint32_t h[NC];
    GSP_CUDA(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    ic.start[0] = 0;
    for (int c = 0; c < NC; c++) ic.start[c + 1] = ic.start[c] + h[c];
    GSP_CUDA(cudaMemcpyAsync(counts + NC, ic.start, sizeof(uint32_t) * NC, cudaMemcpyHostToDevice, s));
    ic.list = arena().get<uint32_t>(ic.start[NC] + 1);
    k_cls_fill<NC><<<gr, 256, 0, s>>>(sz, k, dmax, counts + NC, ic.list);
    GSP_CHECK_LAUNCH();
}

struct AggArgs {
    const uint64_t *off;
    const uint32_t *tgt;
    const void *w;
    const uint32_t *Cd;
    const uint64_t *coff;
    const uint32_t *cverts;
    const unsigned long long *cdeg;
    const uint64_t *yoff;
    uint32_t *htgt;
    double *hw;
    uint32_t *rowlen;
    uint32_t k;
    int xlsb;  // exact fixed-point accumulation: values in integer units of 2^xlsb
};

// Append the occupied slots of a table to row c of the holey CSR.
__device__ __forceinline__ void emit_slot(const AggArgs &a, uint32_t c, uint32_t key, double val, bool valid,
                                          uint32_t *cursor) {
    uint32_t ballot = __ballot_sync(0xFFFFFFFFu, valid);
    if (!ballot) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(ballot) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cursor, (uint32_t)__popc(ballot));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (valid) {
        uint64_t pos = a.yoff[c] + base + __popc(ballot & ((1u << lane) - 1u));
        a.htgt[pos] = key;
        a.hw[pos] = val;
    }
}

// Visits the edges of the rows list[q0..q1) (row v = list[q] owns edges
// off[v]..off[v+1]) with a whole warp: the bounds of 32 rows are read at once
// and their edges dealt out 32 per round with every lane busy, a lane finding
// its row by a 5-step search over the lanes' running edge totals.  fn(p,
// valid) is called by all 32 lanes every round.  The edges of 32 consecutive
// rows must number fewer than 2^32.
template <typename F>
__device__ __forceinline__ void warp_row_edges(const uint32_t *__restrict__ list, uint64_t q0, uint64_t q1,
                                               const uint64_t *__restrict__ off, F &&fn) {
    const uint32_t FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    for (uint64_t qb = q0; qb < q1; qb += 32) {
        const uint64_t q = qb + lane;
        uint64_t b = 0;
        uint32_t len = 0;
        if (q < q1) {
            const uint32_t v = list[q];
            b = off[v];
            len = (uint32_t)(off[v + 1] - b);
        }
        uint32_t end = len;  // inclusive prefix over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, end, o);
            if (lane >= o) end += t;
        }
        const uint32_t start = end - len;
        const uint32_t total = __shfl_sync(FULL, end, 31);
        for (uint32_t e0 = 0; e0 < total; e0 += 32) {
            const uint32_t e = e0 + lane;
            int r = 0;  // first lane whose running total exceeds e
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint32_t ev = __shfl_sync(FULL, end, r + step - 1);
                if (ev <= e) r += step;
            }
            r &= 31;
            const uint64_t rb = __shfl_sync(FULL, b, r);
            const uint32_t rs = __shfl_sync(FULL, start, r);
            fn(rb + (e - rs), e < total);
        }
    }
}

constexpr int AGG_WCAP = 1024;
constexpr int AGG_WWARPS = 4;

template <typename WT, typename AV>
__global__ void __launch_bounds__(AGG_WWARPS * 32) k_agg_merge_warp(AggArgs a, const uint32_t *__restrict__ list,
                                                                    uint32_t count) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    __shared__ uint32_t s_cur[AGG_WWARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *keys = reinterpret_cast<uint32_t *>(dyn_smem) + wid * AGG_WCAP;
    AV *vals = reinterpret_cast<AV *>(dyn_smem + sizeof(uint32_t) * AGG_WCAP * AGG_WWARPS) + wid * AGG_WCAP;
    const WT *w = static_cast<const WT *>(a.w);
    for (uint32_t t = blockIdx.x * AGG_WWARPS + wid; t < count; t += gridDim.x * AGG_WWARPS) {
        uint32_t c = list[t];
        uint64_t cd = a.cdeg[c];
        uint64_t bound = cd < a.k ? cd : a.k;
        int logcap = ceil_log2((uint32_t)(2 * bound));
        if (logcap < 1) logcap = 1;
        uint32_t cap = 1u << logcap;
        for (uint32_t s = lane; s < cap; s += 32) { keys[s] = EMPTY; vals[s] = AV(0); }
        if (lane == 0) s_cur[wid] = 0;
        __syncwarp();
        // edges inside the community (the super-vertex's self-loop) are summed
        // in registers: they are the most frequent key of the table
        AV selfw = AV(0);
        uint32_t nself = 0;
        warp_row_edges(a.cverts, a.coff[c], a.coff[c + 1], a.off, [&](uint64_t p, bool valid) {
            if (!valid) return;
            const uint32_t d = a.Cd[a.tgt[p]];
            const WT x = w[p];
            if (d == c) { selfw += Acc<AV>::of(x, a.xlsb); nself++; }
            else ht_add<AV>(keys, vals, logcap, d, Acc<AV>::of(x, a.xlsb));
        });
        selfw = warp_sum(selfw);
        nself = warp_sum(nself);
        __syncwarp();
        if (lane == 0 && nself) ht_add<AV>(keys, vals, logcap, c, selfw);
        __syncwarp();
        for (uint32_t s0 = 0; s0 < cap; s0 += 32) {
            uint32_t s = s0 + lane;
            uint32_t key = s < cap ? keys[s] : EMPTY;
            emit_slot(a, c, key, s < cap ? Acc<AV>::val(vals[s], a.xlsb) : 0.0, key != EMPTY, &s_cur[wid]);
        }
        __syncwarp();
        if (lane == 0) a.rowlen[c] = s_cur[wid];
        __syncwarp();
    }
}

// One block per community; 4096-slot table in dynamic shared memory with a
// list of occupied slots (emission and clearing touch only those).  The
// members' edges are numbered through a prefix of member degrees in shared
// memory and dealt out evenly over the block (a member-per-warp split leaves
// warps waiting on the longest member).
constexpr int AGG_BCAP = 4096;
constexpr int AGG_BMEM = 2048;  // members staged in shared memory (total degree <= 2048 bounds them)

template <typename WT, typename AV>
__global__ void __launch_bounds__(256) k_agg_merge_block(AggArgs a, const uint32_t *__restrict__ list, uint32_t count) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    uint32_t *keys = reinterpret_cast<uint32_t *>(dyn_smem);
    AV *vals = reinterpret_cast<AV *>(dyn_smem + sizeof(uint32_t) * AGG_BCAP);
    uint16_t *occ = reinterpret_cast<uint16_t *>(dyn_smem + (sizeof(uint32_t) + sizeof(double)) * AGG_BCAP);
    uint64_t *s_base = reinterpret_cast<uint64_t *>(
        dyn_smem + (sizeof(uint32_t) + sizeof(double) + sizeof(uint16_t)) * AGG_BCAP);
    uint32_t *s_pre = reinterpret_cast<uint32_t *>(s_base + AGG_BMEM);  // AGG_BMEM + 1 entries
    __shared__ uint32_t s_cur, s_nocc;
    __shared__ AV s_red[32];
    __shared__ uint32_t s_redn[32], s_wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const WT *w = static_cast<const WT *>(a.w);
    for (uint32_t s = threadIdx.x; s < AGG_BCAP; s += blockDim.x) { keys[s] = EMPTY; vals[s] = AV(0); }
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        uint32_t c = list[t];
        uint64_t cd = a.cdeg[c];
        uint64_t bound = cd < a.k ? cd : a.k;
        int logcap = ceil_log2((uint32_t)(2 * bound));
        if (logcap < 1) logcap = 1;
        __syncthreads();
        if (threadIdx.x == 0) { s_cur = 0; s_nocc = 0; }
        __syncthreads();
        uint64_t q0 = a.coff[c], q1 = a.coff[c + 1];
        const uint32_t nm = (uint32_t)(q1 - q0);
        AV selfw = AV(0);
        uint32_t nself = 0;
        auto visit = [&](uint64_t p) {
            const uint32_t d = a.Cd[a.tgt[p]];
            const WT x = w[p];
            if (d == c) { selfw += Acc<AV>::of(x, a.xlsb); nself++; }
            else smem_add<AV>(keys, vals, logcap, occ, &s_nocc, d, Acc<AV>::of(x, a.xlsb));
        };
        if (nm <= AGG_BMEM) {
            // member degrees -> exclusive prefix s_pre[0..nm], bases s_base
            constexpr int PER = AGG_BMEM / 256;
            uint32_t len[PER];
            uint32_t tsum = 0;
#pragma unroll
            for (int u = 0; u < PER; u++) {
                const uint32_t j = threadIdx.x * PER + u;
                len[u] = 0;
                if (j < nm) {
                    const uint32_t v = a.cverts[q0 + j];
                    const uint64_t b = a.off[v];
                    s_base[j] = b;
                    len[u] = (uint32_t)(a.off[v + 1] - b);
                }
                tsum += len[u];
            }
            uint32_t incl = tsum;  // block-wide exclusive scan of the thread sums
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += x;
            }
            if (lane == 31) s_wsum[wid] = incl;
            __syncthreads();
            uint32_t wbase = 0;
            for (int k = 0; k < wid; k++) wbase += s_wsum[k];
            uint32_t run = wbase + incl - tsum;
#pragma unroll
            for (int u = 0; u < PER; u++) {
                const uint32_t j = threadIdx.x * PER + u;
                if (j < nm) s_pre[j] = run;
                run += len[u];
            }
            if (threadIdx.x == blockDim.x - 1) s_pre[nm] = run;
            __syncthreads();
            const uint32_t E = s_pre[nm];
            for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
                uint32_t lo = 0, hi = nm - 1;  // last member with s_pre <= e
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (s_pre[mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                visit(s_base[lo] + (e - s_pre[lo]));
            }
        } else {
            for (uint64_t q = q0 + wid; q < q1; q += nw) {
                uint32_t v = a.cverts[q];
                uint64_t b = a.off[v], e = a.off[v + 1];
                for (uint64_t p = b + lane; p < e; p += 32) visit(p);
            }
        }
        selfw = block_sum(selfw, s_red);
        nself = block_sum(nself, s_redn);
        if (threadIdx.x == 0 && nself) smem_add<AV>(keys, vals, logcap, occ, &s_nocc, c, selfw);
        __syncthreads();
        uint32_t nocc = s_nocc;
        for (uint32_t k0 = wid * 32; k0 < nocc; k0 += blockDim.x) {
            uint32_t k = k0 + lane;
            uint32_t slot = k < nocc ? occ[k] : 0;
            emit_slot(a, c, k < nocc ? keys[slot] : EMPTY, k < nocc ? Acc<AV>::val(vals[slot], a.xlsb) : 0.0, k < nocc,
                      &s_cur);
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < nocc; k += blockDim.x) {
            uint32_t slot = occ[k];
            keys[slot] = EMPTY;
            vals[slot] = AV(0);
        }
        if (threadIdx.x == 0) a.rowlen[c] = s_cur;
    }
}

// Large communities (total degree > 2048), processed by the whole grid.  A
// community's edges are numbered through the member-edge prefix medge (scan
// of member degrees in community-vertex order, so community c owns
// [yoff[c], yoff[c+1])) and cut into AGG_CHUNK-edge tasks.  A block combines a
// task's neighbour communities in a shared-memory table (each warp finds its
// first member by binary search and walks the members forward), then
// publishes the distinct ones to the community's global table; keys new to it
// append their slot to the community's occupied list, which the extraction
// walks.
constexpr uint32_t AGG_CHUNK = 2048;
constexpr uint32_t AGG_TASK_WARPS = 8;                    // k_agg_large_insert runs 256-thread blocks
constexpr uint32_t AGG_SUB = AGG_CHUNK / AGG_TASK_WARPS;  // edges of a task per warp
constexpr int AGG_SLOG = 12;  // shared table of 2 * AGG_CHUNK slots

__global__ void k_member_deg(const uint64_t *__restrict__ off, const uint32_t *__restrict__ cverts, uint32_t n,
                             uint64_t *mdeg) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        uint32_t v = cverts[q];
        mdeg[q] = off[v + 1] - off[v];
    }
}

__global__ void k_agg_tasks(const unsigned long long *__restrict__ cdeg, const uint32_t *__restrict__ list,
                            uint32_t count, uint64_t *ntask) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x)
        ntask[t] = (cdeg[list[t]] + AGG_CHUNK - 1) / AGG_CHUNK;
}

// First member of every warp's slice of every task: the last member q of
// the community with medge[q] <= the slice's first edge (a binary search per
// slice, all slices at once, ahead of the insert kernel).
__global__ void k_agg_warp_starts(AggArgs a, const uint32_t *__restrict__ list, const uint64_t *__restrict__ tasks,
                                  uint32_t count, const uint32_t *__restrict__ task_c,
                                  const uint64_t *__restrict__ medge, uint32_t *wstart) {
    const uint64_t total = tasks[count] * AGG_TASK_WARPS;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < total;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t task = x / AGG_TASK_WARPS;
        const uint32_t t = task_c[task], c = list[t];
        const uint64_t ch = a.yoff[c] + (task - tasks[t]) * AGG_CHUNK + (x % AGG_TASK_WARPS) * AGG_SUB;
        uint64_t lo = a.coff[c];
        if (ch < a.yoff[c + 1]) {
            uint64_t hi = a.coff[c + 1] - 1;
            while (lo < hi) {
                uint64_t mid = (lo + hi + 1) >> 1;
                if (medge[mid] <= ch) lo = mid;
                else hi = mid - 1;
            }
        }
        wstart[x] = (uint32_t)lo;
    }
}

template <typename WT, typename AV>
__global__ void __launch_bounds__(256) k_agg_large_insert(AggArgs a, const uint32_t *__restrict__ list, uint32_t count,
                                                          const uint64_t *__restrict__ tasks,
                                                          const uint32_t *__restrict__ task_c,
                                                          const uint32_t *__restrict__ wstart,
                                                          const uint64_t *__restrict__ medge,
                                                          const uint64_t *__restrict__ pool_off, uint32_t *pool_keys,
                                                          AV *pool_vals, uint32_t *pool_occ, uint32_t *occ_n) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    uint32_t *skeys = reinterpret_cast<uint32_t *>(dyn_smem);
    AV *svals = reinterpret_cast<AV *>(dyn_smem + sizeof(uint32_t) * (1u << AGG_SLOG));
    uint16_t *socc = reinterpret_cast<uint16_t *>(dyn_smem + (sizeof(uint32_t) + sizeof(AV)) * (1u << AGG_SLOG));
    __shared__ uint32_t s_nocc;
    __shared__ AV s_red[32];
    __shared__ uint32_t s_redn[32];
    const WT *w = static_cast<const WT *>(a.w);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t s = threadIdx.x; s < (1u << AGG_SLOG); s += blockDim.x) { skeys[s] = EMPTY; svals[s] = AV(0); }
    if (threadIdx.x == 0) s_nocc = 0;
    const uint64_t total = tasks[count];
    for (uint64_t task = blockIdx.x; task < total; task += gridDim.x) {
        uint32_t t = task_c[task];
        uint32_t c = list[t];
        uint64_t E1 = a.yoff[c + 1];
        uint64_t q1 = a.coff[c + 1];
        uint64_t ch = a.yoff[c] + (task - tasks[t]) * AGG_CHUNK + (uint64_t)wid * AGG_SUB;
        uint64_t cend = min(ch + AGG_SUB, E1);
        AV selfw = AV(0);
        uint32_t nself = 0;
        if (ch < E1) {
            const uint64_t lo = wstart[task * AGG_TASK_WARPS + wid];  // last member with medge <= ch
            // A window of 32 members (lane l: member q + l, its end in the
            // member-edge numbering and its first edge in the CSR) is read at
            // once; each round deals out up to 32 edges of the window, every
            // lane finding its member by a 5-step search over the window's
            // ends.  Members of high degree keep the window for many rounds,
            // short ones are consumed 32 at a time.
            const uint32_t FULL = 0xFFFFFFFFu;
            uint64_t q = lo, t0 = ch, wq = ~0ull;
            uint64_t wend_l = 0, wbase_l = 0, wstart = 0;
            while (t0 < cend) {
                if (q != wq) {
                    const uint64_t ql = q + lane;
                    wend_l = medge[ql < q1 ? ql + 1 : q1];
                    wbase_l = ql < q1 ? a.off[a.cverts[ql]] : 0;
                    wstart = medge[q];
                    wq = q;
                }
                const uint64_t wend = __shfl_sync(FULL, wend_l, 31);
                uint64_t rend = min(min(wend, cend), t0 + 32);
                if (rend <= t0) {  // every member of the window ends before t0
                    q += 32;
                    continue;
                }
                const uint64_t tt = t0 + lane;
                int r = 0;  // first window member ending after tt
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const uint64_t ev = __shfl_sync(FULL, wend_l, r + step - 1);
                    if (ev <= tt) r += step;
                }
                r &= 31;
                const uint64_t rbase = __shfl_sync(FULL, wbase_l, r);
                const uint64_t rprev = __shfl_sync(FULL, wend_l, (r + 31) & 31);
                const uint64_t rstart = r ? rprev : wstart;
                if (tt < rend) {
                    const uint64_t p = rbase + (tt - rstart);
                    const uint32_t dd = a.Cd[a.tgt[p]];
                    if (dd == c) { selfw += Acc<AV>::of(w[p], a.xlsb); nself++; }
                    else smem_add<AV>(skeys, svals, AGG_SLOG, socc, &s_nocc, dd, Acc<AV>::of(w[p], a.xlsb));
                }
                // members ending at or before rend are done
                q += __popc(__ballot_sync(FULL, wend_l <= rend));
                t0 = rend;
            }
        }
        // the task's edges inside the community enter the table once
        selfw = block_sum(selfw, s_red);
        nself = block_sum(nself, s_redn);
        if (threadIdx.x == 0 && nself)
            smem_add<AV>(skeys, svals, AGG_SLOG, socc, &s_nocc, c, selfw);
        uint64_t cd = a.cdeg[c];
        uint64_t bound = cd < a.k ? cd : a.k;
        int glog = ceil_log2((uint32_t)(2 * bound));
        if (glog < 1) glog = 1;
        publish_block_table<AV>(skeys, svals, socc, &s_nocc, pool_keys + pool_off[t], pool_vals + pool_off[t],
                                    glog, pool_occ + pool_off[t], occ_n + t);
    }
}

// Extraction uses the insert's task split: task k of a community emits its
// occupied entries [k * AGG_CHUNK, (k+1) * AGG_CHUNK) (a community has at
// most one distinct neighbour community per edge).
template <typename AV>
__global__ void __launch_bounds__(256) k_agg_large_extract(AggArgs a, const uint32_t *__restrict__ list,
                                                           uint32_t count, const uint64_t *__restrict__ tasks,
                                                           const uint32_t *__restrict__ task_c,
                                                           const uint64_t *__restrict__ pool_off,
                                                           const uint32_t *__restrict__ pool_keys,
                                                           const AV *__restrict__ pool_vals,
                                                           const uint32_t *__restrict__ pool_occ,
                                                           const uint32_t *__restrict__ occ_n) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t total = tasks[count];
    for (uint64_t task = blockIdx.x; task < total; task += gridDim.x) {
        uint32_t t = task_c[task];
        uint32_t c = list[t];
        const uint32_t *keys = pool_keys + pool_off[t];
        const AV *vals = pool_vals + pool_off[t];
        const uint32_t *occ = pool_occ + pool_off[t];
        uint64_t k0 = (task - tasks[t]) * AGG_CHUNK;
        uint64_t k1 = min(k0 + AGG_CHUNK, (uint64_t)occ_n[t]);
        // warp-uniform trip counts so emit_slot's ballots see full warps
        for (uint64_t kb = k0 + wid * 32; kb < k1; kb += blockDim.x) {
            uint64_t k = kb + lane;
            bool valid = k < k1;
            uint32_t slot = valid ? occ[k] : 0;
            emit_slot(a, c, valid ? keys[slot] : EMPTY, valid ? Acc<AV>::val(vals[slot], a.xlsb) : 0.0, valid,
                      a.rowlen + c);
        }
    }
}

__global__ void k_agg_pool_caps(const unsigned long long *__restrict__ cdeg, const uint32_t *__restrict__ list,
                                uint32_t count, uint32_t k, uint64_t *caps) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        uint64_t cd = cdeg[list[t]];
        uint64_t bound = cd < k ? cd : k;
        uint64_t cap = 2;
        while (cap < 2 * bound) cap <<= 1;
        caps[t] = cap;
    }
}

// ------------------------------------------------------------ row sorting
__global__ void k_rowlen64(const uint32_t *__restrict__ rowlen, uint32_t k, uint64_t *out) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) out[c] = rowlen[c];
}

// Rows of <= 32 entries: one warp, bitonic network over the lanes.
__global__ void k_sort_rows_warp(const uint32_t *__restrict__ list, uint32_t count, const uint64_t *__restrict__ yoff,
                                 const uint32_t *__restrict__ htgt, const double *__restrict__ hw,
                                 const uint64_t *__restrict__ noff, uint32_t *otgt, double *ow) {
    const int lane = threadIdx.x & 31;
    uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t = warp; t < count; t += nwarps) {
        uint32_t c = list[t];
        uint64_t dst = noff[c];
        uint32_t L = (uint32_t)(noff[c + 1] - dst);
        uint64_t src = yoff[c];
        uint32_t key = lane < L ? htgt[src + lane] : EMPTY;
        double val = lane < L ? hw[src + lane] : 0.0;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                uint32_t ok = __shfl_xor_sync(0xFFFFFFFFu, key, j);
                double ov = __shfl_xor_sync(0xFFFFFFFFu, val, j);
                bool up = (lane & k) == 0;
                bool lower = (lane & j) == 0;
                bool take = (lower == up) ? (ok < key) : (ok > key);
                if (take) { key = ok; val = ov; }
            }
        }
        if (lane < L) { otgt[dst + lane] = key; ow[dst + lane] = val; }
    }
}

constexpr int SORT_BCAP = 2048;
// Rows of <= 2048 entries: one block, bitonic sort in shared memory.
__global__ void __launch_bounds__(256) k_sort_rows_block(const uint32_t *__restrict__ list, uint32_t count,
                                                         const uint64_t *__restrict__ yoff,
                                                         const uint32_t *__restrict__ htgt,
                                                         const double *__restrict__ hw,
                                                         const uint64_t *__restrict__ noff, uint32_t *otgt,
                                                         double *ow) {
    __shared__ uint32_t sk[SORT_BCAP];
    __shared__ double sv[SORT_BCAP];
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        uint32_t c = list[t];
        uint64_t dst = noff[c];
        uint32_t L = (uint32_t)(noff[c + 1] - dst);
        uint64_t src = yoff[c];
        uint32_t P = 1u << ceil_log2(L);
        __syncthreads();
        for (uint32_t x = threadIdx.x; x < P; x += blockDim.x) {
            sk[x] = x < L ? htgt[src + x] : EMPTY;
            sv[x] = x < L ? hw[src + x] : 0.0;
        }
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t x = threadIdx.x; x < P; x += blockDim.x) {
                    uint32_t y = x ^ j;
                    if (y > x) {
                        bool up = (x & k) == 0;
                        uint32_t kx = sk[x], ky = sk[y];
                        if ((kx > ky) == up) {
                            sk[x] = ky; sk[y] = kx;
                            double tv = sv[x]; sv[x] = sv[y]; sv[y] = tv;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t x = threadIdx.x; x < L; x += blockDim.x) { otgt[dst + x] = sk[x]; ow[dst + x] = sv[x]; }
    }
}

// Long rows: copy unsorted, and stage (row rank << kbits | target, position)
// pairs for one segmented radix sort.
__global__ void k_stage_long(const uint32_t *__restrict__ list, uint32_t count, const uint64_t *__restrict__ yoff,
                             const uint32_t *__restrict__ htgt, const double *__restrict__ hw,
                             const uint64_t *__restrict__ noff, const uint64_t *__restrict__ gpre, int kbits,
                             uint64_t *keys, uint32_t *pos, double *wtmp) {
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        uint32_t c = list[t];
        uint64_t dst = noff[c];
        uint32_t L = (uint32_t)(noff[c + 1] - dst);
        uint64_t src = yoff[c], g = gpre[t];
        for (uint32_t x = threadIdx.x; x < L; x += blockDim.x) {
            keys[g + x] = ((uint64_t)t << kbits) | htgt[src + x];
            pos[g + x] = (uint32_t)(g + x);
            wtmp[g + x] = hw[src + x];
        }
    }
}

__global__ void k_unstage_long(const uint32_t *__restrict__ list, const uint64_t *__restrict__ keys,
                               const uint32_t *__restrict__ pos, uint64_t total, const double *__restrict__ wtmp,
                               const uint64_t *__restrict__ gpre, const uint64_t *__restrict__ noff, int kbits,
                               uint32_t *otgt, double *ow) {
    uint64_t mask = (1ull << kbits) - 1ull;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t key = keys[q];
        uint32_t t = (uint32_t)(key >> kbits);
        uint64_t dst = noff[list[t]] + (q - gpre[t]);
        otgt[dst] = (uint32_t)(key & mask);
        ow[dst] = wtmp[pos[q]];
    }
}

__global__ void k_rowlen_gather(const uint32_t *__restrict__ list, uint32_t count, const uint32_t *__restrict__ rowlen,
                                uint64_t *out) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x)
        out[t] = rowlen[list[t]];
}

// Unsorted compaction of the holey rows (rows in any order of targets):
// one warp per row for rows of <= 2048 entries, one block per longer row.
__global__ void k_compact_rows_warp(const uint32_t *__restrict__ list, uint32_t count,
                                    const uint64_t *__restrict__ yoff, const uint32_t *__restrict__ htgt,
                                    const double *__restrict__ hw, const uint64_t *__restrict__ noff, uint32_t *otgt,
                                    double *ow) {
    const int lane = threadIdx.x & 31;
    uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t = warp; t < count; t += nwarps) {
        uint32_t c = list[t];
        uint64_t dst = noff[c], src = yoff[c];
        uint32_t L = (uint32_t)(noff[c + 1] - dst);
        for (uint32_t x = lane; x < L; x += 32) {
            otgt[dst + x] = htgt[src + x];
            ow[dst + x] = hw[src + x];
        }
    }
}

__global__ void k_compact_rows_block(const uint32_t *__restrict__ list, uint32_t count,
                                     const uint64_t *__restrict__ yoff, const uint32_t *__restrict__ htgt,
                                     const double *__restrict__ hw, const uint64_t *__restrict__ noff, uint32_t *otgt,
                                     double *ow) {
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        uint32_t c = list[t];
        uint64_t dst = noff[c], src = yoff[c];
        uint64_t L = noff[c + 1] - dst;
        for (uint64_t x = threadIdx.x; x < L; x += blockDim.x) {
            otgt[dst + x] = htgt[src + x];
            ow[dst + x] = hw[src + x];
        }
    }
}

static int ceil_log2_host(uint64_t x) {
    int b = 0;
    while ((1ull << b) < x) b++;
    return b;
}


// Per-community tables of the three size classes, emitted into the holey CSR.
template <typename WT, typename AV>
static void merge_tables(const DevGraph &g, const AggArgs &a, const IdClasses &ic, const unsigned long long *cdeg,
                         const uint32_t *cverts, uint32_t k, uint32_t n, cudaStream_t s) {
    auto cnt_of = [&](int c) { return ic.start[c + 1] - ic.start[c]; };
    if (cnt_of(ACLS_W)) {
        constexpr size_t smem = (size_t)AGG_WWARPS * AGG_WCAP * (sizeof(uint32_t) + sizeof(AV));
        static bool wattr = false;
        if (!wattr) {
            GSP_CUDA(cudaFuncSetAttribute(k_agg_merge_warp<WT, AV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            wattr = true;
        }
        k_agg_merge_warp<WT, AV><<<grid_for((uint64_t)cnt_of(ACLS_W) * 32, AGG_WWARPS * 32, sms(4)), AGG_WWARPS * 32,
                               smem, s>>>(a, ic.list + ic.start[ACLS_W], cnt_of(ACLS_W));
        GSP_CHECK_LAUNCH();
    }
    if (cnt_of(ACLS_B)) {
        constexpr size_t smem = (size_t)AGG_BCAP * (sizeof(uint32_t) + sizeof(AV) + sizeof(uint16_t)) +
                                (size_t)AGG_BMEM * sizeof(uint64_t) + (size_t)(AGG_BMEM + 1) * sizeof(uint32_t);
        static bool attr = false;
        if (!attr) {
            GSP_CUDA(cudaFuncSetAttribute(k_agg_merge_block<WT, AV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            attr = true;
        }
        k_agg_merge_block<WT, AV><<<grid_for(cnt_of(ACLS_B), 1, sms(4)), 256, smem, s>>>(a, ic.list + ic.start[ACLS_B],
                                                                                     cnt_of(ACLS_B));
        GSP_CHECK_LAUNCH();
    }
    uint32_t nl = cnt_of(ACLS_L);
    if (nl) {
        uint64_t *caps = arena().get<uint64_t>(nl);
        uint64_t *poff = arena().get<uint64_t>((size_t)nl + 1);
        k_agg_pool_caps<<<grid_for(nl, 256), 256, 0, s>>>(cdeg, ic.list + ic.start[ACLS_L], nl, k, caps);
        GSP_CHECK_LAUNCH();
        exclusive_scan_u64(caps, poff, nl, s);
        uint64_t slots;
        GSP_CUDA(cudaMemcpyAsync(&slots, poff + nl, sizeof(slots), cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        uint32_t *pk = arena().get<uint32_t>(slots);
        AV *pv = arena().get<AV>(slots);
        uint32_t *po = arena().get<uint32_t>(slots);
        uint32_t *on = arena().get<uint32_t>(nl);
        GSP_CUDA(cudaMemsetAsync(pk, 0xFF, sizeof(uint32_t) * slots, s));
        GSP_CUDA(cudaMemsetAsync(pv, 0, sizeof(AV) * slots, s));
        GSP_CUDA(cudaMemsetAsync(on, 0, sizeof(uint32_t) * nl, s));
        uint64_t *medge = arena().get<uint64_t>((size_t)n + 1);
        uint64_t *mdeg = arena().get<uint64_t>(n);
        k_member_deg<<<grid_for(n, 256), 256, 0, s>>>(g.off, cverts, n, mdeg);
        GSP_CHECK_LAUNCH();
        exclusive_scan_u64(mdeg, medge, n, s);
        const uint32_t *llist = ic.list + ic.start[ACLS_L];
        uint64_t *ntask = arena().get<uint64_t>(nl);
        uint64_t *tasks = arena().get<uint64_t>((size_t)nl + 1);
        k_agg_tasks<<<grid_for(nl, 256), 256, 0, s>>>(cdeg, llist, nl, ntask);
        GSP_CHECK_LAUNCH();
        exclusive_scan_u64(ntask, tasks, nl, s);
        // at most one task per AGG_CHUNK edges plus one partial task per community
        const uint64_t task_bound = g.nnz / AGG_CHUNK + nl + 1;
        uint32_t *task_c = arena().get<uint32_t>(task_bound);
        task_items(tasks, nl, task_c, s);
        uint32_t *wstart = arena().get<uint32_t>(task_bound * AGG_TASK_WARPS);
        k_agg_warp_starts<<<grid_for(task_bound * AGG_TASK_WARPS, 256, sms(16)), 256, 0, s>>>(
            a, llist, tasks, nl, task_c, medge, wstart);
        GSP_CHECK_LAUNCH();
        constexpr size_t lsmem = (sizeof(uint32_t) + sizeof(AV) + sizeof(uint16_t)) << AGG_SLOG;
        static bool lattr = false;
        if (!lattr) {
            GSP_CUDA(cudaFuncSetAttribute(k_agg_large_insert<WT, AV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)lsmem));
            lattr = true;
        }
        const unsigned lgrid = resident_grid((const void *)k_agg_large_insert<WT, AV>, AGG_TASK_WARPS * 32, lsmem, 4);
        k_agg_large_insert<WT, AV><<<lgrid, AGG_TASK_WARPS * 32, lsmem, s>>>(a, llist, nl, tasks, task_c, wstart, medge,
                                                                          poff, pk, pv, po, on);
        GSP_CHECK_LAUNCH();
        k_agg_large_extract<AV><<<sms(4), 256, 0, s>>>(a, llist, nl, tasks, task_c, poff, pk, pv, po, on);
        GSP_CHECK_LAUNCH();
    }

}

template <typename WT>
static uint64_t aggregate_impl(const DevGraph &g, const uint32_t *Cd, uint32_t k, uint64_t *out_off,
                               uint32_t *out_tgt, double *out_w, bool sorted, int *lsb_cache, cudaStream_t s) {
    size_t mk = arena().mark();
    uint32_t n = g.n;
    uint32_t *cnt = arena().get<uint32_t>(k);
    unsigned long long *cdeg = arena().get<unsigned long long>(k);
    uint64_t *coff = arena().get<uint64_t>((size_t)k + 1);
    uint64_t *yoff = arena().get<uint64_t>((size_t)k + 1);
    uint32_t *cverts = arena().get<uint32_t>(n);
    uint32_t *rowlen = arena().get<uint32_t>(k);
    uint32_t *htgt = arena().get<uint32_t>(g.nnz + 1);
    double *hw = arena().get<double>(g.nnz + 1);
    GSP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * k, s));
    GSP_CUDA(cudaMemsetAsync(cdeg, 0, sizeof(unsigned long long) * k, s));
    GSP_CUDA(cudaMemsetAsync(rowlen, 0, sizeof(uint32_t) * k, s));
    unsigned gr = grid_for(n, 256);
    k_agg_count<WT><<<gr, 256, 0, s>>>(g.off, Cd, n, cnt, cdeg);
    GSP_CHECK_LAUNCH();
    exclusive_scan_u32_to_u64(cnt, coff, k, s);
    exclusive_scan_u64(reinterpret_cast<const uint64_t *>(cdeg), yoff, k, s);
    k_agg_scatter<<<gr, 256, 0, s>>>(Cd, n, coff, cnt, cverts);
    GSP_CHECK_LAUNCH();

    IdClasses ic;
    classify_ids<NUM_ACLS>(reinterpret_cast<const uint64_t *>(cdeg), k, ACLS_MAX, ic, s);
    AggArgs a{g.off, g.tgt, g.w, Cd, coff, cverts, cdeg, yoff, htgt, hw, rowlen, k, 0};
    // exact fixed-point table values when the weights allow it (same result,
    // native shared-memory integer atomics instead of float64 ones)
    int lsb = lsb_cache ? *lsb_cache : INT_MAX;
    if (lsb == INT_MAX) lsb = exact_lsb(g, s);
    if (lsb_cache) *lsb_cache = lsb;
    if (lsb != INT_MIN) {
        a.xlsb = lsb;
        merge_tables<WT, unsigned long long>(g, a, ic, cdeg, cverts, k, n, s);
    } else {
        merge_tables<WT, double>(g, a, ic, cdeg, cverts, k, n, s);
    }
    // compact + sort rows
    exclusive_scan_u32_to_u64(rowlen, out_off, k, s);
    uint64_t nnz2;
    GSP_CUDA(cudaMemcpyAsync(&nnz2, out_off + k, sizeof(nnz2), cudaMemcpyDeviceToHost, s));
    GSP_CUDA(cudaStreamSynchronize(s));
    uint64_t *rl64 = arena().get<uint64_t>(k);
    k_rowlen64<<<grid_for(k, 256), 256, 0, s>>>(rowlen, k, rl64);
    GSP_CHECK_LAUNCH();
    IdClasses rc;
    classify_ids<NUM_RCLS>(rl64, k, RCLS_MAX, rc, s);
    auto rcnt = [&](int c) { return rc.start[c + 1] - rc.start[c]; };
    if (!sorted) {
        const uint32_t nshort = rcnt(RCLS_W) + rcnt(RCLS_B);  // classes W and B are adjacent in the list
        if (nshort) {
            k_compact_rows_warp<<<grid_for((uint64_t)nshort * 32, 256, sms(16)), 256, 0, s>>>(
                rc.list + rc.start[RCLS_W], nshort, yoff, htgt, hw, out_off, out_tgt, out_w);
            GSP_CHECK_LAUNCH();
        }
        if (rcnt(RCLS_L)) {
            k_compact_rows_block<<<grid_for(rcnt(RCLS_L), 1, sms(4)), 256, 0, s>>>(
                rc.list + rc.start[RCLS_L], rcnt(RCLS_L), yoff, htgt, hw, out_off, out_tgt, out_w);
            GSP_CHECK_LAUNCH();
        }
        arena().release(mk);
        return nnz2;
    }
    if (rcnt(RCLS_W)) {
        k_sort_rows_warp<<<grid_for((uint64_t)rcnt(RCLS_W) * 32, 256, sms(16)), 256, 0, s>>>(
            rc.list + rc.start[RCLS_W], rcnt(RCLS_W), yoff, htgt, hw, out_off, out_tgt, out_w);
        GSP_CHECK_LAUNCH();
    }
    if (rcnt(RCLS_B)) {
        k_sort_rows_block<<<grid_for(rcnt(RCLS_B), 1, sms(4)), 256, 0, s>>>(
            rc.list + rc.start[RCLS_B], rcnt(RCLS_B), yoff, htgt, hw, out_off, out_tgt, out_w);
        GSP_CHECK_LAUNCH();
    }
    uint32_t nlong = rcnt(RCLS_L);
    if (nlong) {
        const uint32_t *llist = rc.list + rc.start[RCLS_L];
        uint64_t *lens = arena().get<uint64_t>(nlong);
        uint64_t *gpre = arena().get<uint64_t>((size_t)nlong + 1);
        // lengths of the long rows, in list order
        k_rowlen_gather<<<grid_for(nlong, 256), 256, 0, s>>>(llist, nlong, rowlen, lens);
        GSP_CHECK_LAUNCH();
        exclusive_scan_u64(lens, gpre, nlong, s);
        uint64_t total;
        GSP_CUDA(cudaMemcpyAsync(&total, gpre + nlong, sizeof(total), cudaMemcpyDeviceToHost, s));
        GSP_CUDA(cudaStreamSynchronize(s));
        GSP_REQUIRE(total < (1ull << 32), "aggregation: long rows exceed 2^32 entries");
        int kbits = ceil_log2_host(k);
        if (kbits < 1) kbits = 1;
        int bits = kbits + ceil_log2_host(nlong) + 1;
        uint64_t *keys = arena().get<uint64_t>(total);
        uint64_t *keys2 = arena().get<uint64_t>(total);
        uint32_t *pos = arena().get<uint32_t>(total);
        uint32_t *pos2 = arena().get<uint32_t>(total);
        double *wtmp = arena().get<double>(total);
        k_stage_long<<<grid_for(nlong, 1, sms(4)), 256, 0, s>>>(llist, nlong, yoff, htgt, hw, out_off, gpre, kbits,
                                                                  keys, pos, wtmp);
        GSP_CHECK_LAUNCH();
        radix_sort_u64_u32(keys, pos, keys2, pos2, total, bits, s);
        k_unstage_long<<<grid_for(total, 256), 256, 0, s>>>(llist, keys, pos, total, wtmp, gpre, out_off, kbits,
                                                             out_tgt, out_w);
        GSP_CHECK_LAUNCH();
    }
    arena().release(mk);
    return nnz2;
}

uint64_t aggregate(const DevGraph &g, const uint32_t *Cd, uint32_t k, uint64_t *out_off, uint32_t *out_tgt,
                   double *out_w, cudaStream_t s, bool sorted, int *lsb_cache) {
    if (g.wt == GSP_W_F64) return aggregate_impl<double>(g, Cd, k, out_off, out_tgt, out_w, sorted, lsb_cache, s);
    return aggregate_impl<float>(g, Cd, k, out_off, out_tgt, out_w, sorted, lsb_cache, s);
}

}  // namespace gsp
