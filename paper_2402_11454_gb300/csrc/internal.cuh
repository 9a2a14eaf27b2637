// internal.cuh -- host-side interfaces between the translation units of libgsp.
#pragma once
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

// Degree classes of a vertex (or community) list.  Small degrees are served
// by groups of G lanes with a shared-memory table, mid degrees by one block
// with a shared-memory table, the largest by one block with a table in a
// global-memory pool.
enum { CLS_G4 = 0, CLS_G8, CLS_G16, CLS_G32, CLS_BLOCK, CLS_HUGE, NUM_CLS };
constexpr uint32_t CLS_MAXDEG[NUM_CLS] = {8, 16, 32, 128, 4096, 0xFFFFFFFFu};

struct Classes {
    uint32_t *list = nullptr;  // vertex ids grouped by class (class c at [start[c], start[c+1]))
    uint32_t start[NUM_CLS + 1] = {0};
    uint64_t *pool_off = nullptr;  // huge class: hashtable slot offsets (count+1)
    uint64_t pool_slots = 0;
};

// Build the class lists of g's vertices (degree 0 vertices are left out).
void classify_vertices(const DevGraph &g, Classes &cl, cudaStream_t s);

struct MoveCounters {  // device-side accumulators of one sweep
    double dq;
    unsigned long long moved;
    unsigned long long vertices;
    unsigned long long edges;
    unsigned long long candidates;
    unsigned long long skipped;
    unsigned long long marked;  // edges of moved vertices (neighbour re-marking)
};

struct MoveBuffers {
    uint32_t *C = nullptr, *C2 = nullptr;       // membership (C2: next, frozen-state sweeps)
    double *Sigma = nullptr, *Sigma2 = nullptr;
    uint32_t *size = nullptr, *size2 = nullptr;
    uint8_t *act = nullptr, *act2 = nullptr;     // unprocessed flags
    const double *K = nullptr;
    double *m_dev = nullptr;                     // device copy of m
    MoveCounters *ctr = nullptr;
    void *pool = nullptr;                        // huge-class hashtables
    // learned pruning (optional)
    const float *mlp = nullptr;
    float *feat_dq = nullptr;     // last delta-modularity gain seen per vertex (scaled)
    uint8_t *moved_last = nullptr;
    float *nbr_moved = nullptr;
};

struct SweepResult {
    double dq;
    uint64_t moved, vertices, edges, candidates, skipped;
};

// One sweep over the active vertices.  sync: frozen-state (reads C/Sigma/size/act,
// writes C2/Sigma2/size2/act2, which must hold copies of C/Sigma/size and zeros).
void move_sweep(const DevGraph &g, const Classes &cl, MoveBuffers &mb, bool sync, bool fp64, bool rule,
                bool learned, cudaStream_t s);

struct LouvainTimers;

// Split (Algorithms 2, 3): labels = smallest vertex of the component.
void split_labels(const DevGraph &g, const Classes &cl, const uint32_t *C, int mode, uint32_t *labels,
                  cudaStream_t s);

// Renumber: C_dense[v] = rank of C[v] among the distinct ids; returns k.
uint32_t renumber(uint32_t n, const uint32_t *C, uint32_t *C_dense, cudaStream_t s);

// Aggregation (Algorithm 5) into out (offsets k+1, targets/weights nnz); returns nnz''.
uint64_t aggregate(const DevGraph &g, const uint32_t *Cd, uint32_t k, uint64_t *out_off, uint32_t *out_tgt,
                   double *out_w, cudaStream_t s);

// K and m (m also written to *m_dev when non-null); returns m.
double vertex_weights(const DevGraph &g, double *K, double *m_dev, cudaStream_t s);
double modularity(const DevGraph &g, const uint32_t *C, cudaStream_t s);
uint32_t count_disconnected(const DevGraph &g, const uint32_t *C, uint8_t *flags, cudaStream_t s);
void lookup(uint32_t n_top, uint32_t *C_top, const uint32_t *C_pass, cudaStream_t s);
// Renumber membership by smallest vertex id (final numbering); returns k.
uint32_t canonical_numbering(uint32_t n, uint32_t *C, cudaStream_t s);

void iota_u32(uint32_t *p, uint32_t n, cudaStream_t s);

// MLP (mlp.cu)
constexpr int MLP_IN = 6, MLP_H = 32;
constexpr int MLP_PARAMS = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;

__device__ __forceinline__ int ceil_log2(uint32_t x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

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

}  // namespace gsp
