/*
 * gsp.h -- C ABI of the GB300-native GSP-Louvain library (libgsp.so).
 *
 * GSP-Louvain (Sahu, arXiv 2402.11454) is the Louvain method of community
 * detection with a split step after the local-moving phase of every pass,
 * which breaks each community into its connected components so that no
 * returned community is internally disconnected.
 *
 * Conventions for every entry point:
 *  - Graphs are symmetric CSR: offsets (n+1 x uint64), targets (nnz x uint32),
 *    weights (nnz x float32, or float64 where a gsp_wtype says so).  Both
 *    directions of every undirected edge are stored; a self-loop is stored
 *    once in its row.  Weights must be finite and > 0.  (Section 3: G(V,E,w),
 *    w_ij = w_ji, unit weight for unweighted graphs.)
 *  - Unless a parameter says "host", every pointer is a DEVICE pointer owned by
 *    the caller; the library never frees caller memory.  Work runs on the
 *    cudaStream_t passed as `stream` (NULL = legacy default stream); calls that
 *    return host values synchronise that stream before returning.
 *  - Nothing throws across the ABI.  Every call returns a gsp_status; invalid
 *    sizes or options give GSP_ERR_INVALID before any device work; a CUDA
 *    failure gives GSP_ERR_CUDA; gsp_last_error() returns a message.
 *  - The library keeps one internal device workspace, grown on demand with
 *    cudaMalloc and reused across calls.  Calls must not run concurrently
 *    from several host threads.
 *  - The naming clash of the paper (m = total edge weight, M = edge count) is
 *    avoided by calling the edge count nnz.
 */
#ifndef GSP_H
#define GSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSP_OK = 0,
    GSP_ERR_INVALID = -1,     /* bad size, pointer or option */
    GSP_ERR_NOMEM = -2,       /* device allocation failed */
    GSP_ERR_CUDA = -3,        /* a CUDA runtime call or kernel failed */
    GSP_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    GSP_ERR_CAPACITY = -5,    /* a fixed-size buffer was too small */
    GSP_ERR_NOT_SYMMETRIC = -6 /* the CSR is not symmetric (w_ij != w_ji, or an entry lacks its mirror) */
} gsp_status;

/* Split techniques of Section 4.1: none (GVE-Louvain), min-label propagation
 * (Algorithm 2), min-label propagation with pruning (Algorithm 2, LPP), and
 * breadth-first search (Algorithm 3); SV (not in the paper) is hooking and
 * shortcutting (Shiloach-Vishkin) on the intra-community edges, for graphs of
 * high diameter.  All give the same labels. */
typedef enum {
    GSP_SPLIT_NONE = 0,
    GSP_SPLIT_LP = 1,
    GSP_SPLIT_LPP = 2,
    GSP_SPLIT_BFS = 3,
    GSP_SPLIT_SV = 4
} gsp_split_mode;
/* Split Pass (after the local-moving phase of every pass) or Split Last
 * (once, after the passes converge); Section 4.1. */
typedef enum { GSP_SPLIT_PASS = 0, GSP_SPLIT_LAST = 1 } gsp_split_when;
/* Local moving (Algorithm 4): ASYNC updates memberships in place as the paper
 * does (results depend on thread timing); SYNC lets every vertex of an
 * iteration read the state of the iteration's start (deterministic). */
typedef enum { GSP_MOVE_ASYNC = 0, GSP_MOVE_SYNC = 1 } gsp_move_mode;
/* An iteration is split into `waves` waves: vertex i belongs to wave
 * h(i) mod waves, h the MurmurHash3 32-bit finaliser of its index (of its
 * index within its graph in a batch), and every vertex of a wave reads the
 * state left by the earlier waves (SYNC, waves = 1: fully synchronous; more
 * waves approach the one-thread order).  The hash keeps arithmetic patterns
 * of the ids out of the waves: with wave i mod 17, every community of a
 * planted graph with 17, 34 or 51 communities (vertex v in community v mod k)
 * fell into one wave, decided at once and cycled.  In the first iteration of
 * a pass each wave runs `wave_repeats` times (later iterations once): a
 * repeat takes the vertices of the wave that the previous repeat's moves
 * marked unprocessed again (the pruning rule of Algorithm 4 applied inside
 * the wave), on the state those moves left.  Three repeats
 * bring the frozen-state schedule close to the modularity of the one-thread
 * loop (on R-MAT scales 19, 20 and 21, 0.0002, 0.0007 and 0.0013 below it on
 * average, where a single pass fell 0.0022, 0.0029 and 0.0033 short) for about
 * 1.45 times the edge visits; an odd count does better than the next even
 * one, and repeats in the later iterations cost more than they gain.  From
 * iteration `no_return_from` of a pass on, a vertex does not move back to the
 * community it left in the previous iteration: the one-thread loop raises Q
 * with every move and cannot cycle, but simultaneous decisions can fall into
 * a two-iteration cycle whose claimed gains stay above tau (grids ran their
 * later passes to MAX_ITERATIONS).  In ASYNC mode the waves, repeats and the
 * no-return rule order the in-place updates the same way; there the default
 * is 64 waves: with 17, the thousands of vertices of a wave that run at once
 * ended up to 0.0026 below the one-thread loop on R-MAT 16-18, with 64 within
 * 0.0008, and with one wave (the loop as written, every vertex at once) 0.03
 * to 0.08 below. */
/* MIXED: per-community weights K_{i->c} and delta-modularity in float32,
 * while m, Sigma_tot and modularity stay float64.  FP64: everything float64,
 * Equation 2 evaluated term by term (the parity mode). */
typedef enum { GSP_PREC_MIXED = 0, GSP_PREC_FP64 = 1 } gsp_precision;
/* Vertex pruning of Algorithm 4 (processed/unprocessed flags), optionally
 * narrowed by a learned skip predictor (a small MLP). */
typedef enum { GSP_PRUNE_FLAGS = 0, GSP_PRUNE_LEARNED = 1 } gsp_prune_mode;
typedef enum { GSP_W_F32 = 0, GSP_W_F64 = 1 } gsp_wtype;

typedef struct {
    int max_passes;                 /* MAX_PASSES (Algorithm 1); default 10 */
    int max_iterations;             /* MAX_ITERATIONS (Algorithm 4); default 20 */
    double tolerance;               /* tau (Algorithm 4); default 1e-2 */
    double tolerance_drop;          /* TOLERANCE_DROP (Algorithm 1); default 10 */
    double aggregation_tolerance;   /* tau_agg (Algorithm 1); default 0.8 */
    int split;                      /* gsp_split_mode; default GSP_SPLIT_LPP */
    int split_when;                 /* gsp_split_when; default GSP_SPLIT_PASS */
    int move;                       /* gsp_move_mode; default GSP_MOVE_SYNC */
    int waves;                      /* waves per iteration, 1..64, or 0 (the default): 17 for SYNC, 64
                                       for ASYNC */
    int wave_repeats;               /* times each wave runs in a pass's first iteration, 1..8; default 3 */
    int no_return_from;             /* no move back to the community left the iteration before, from this
                                       iteration of a pass on (0: never); default 3 */
    int precision;                  /* gsp_precision; default GSP_PREC_MIXED */
    int singleton_rule;             /* 1: a vertex alone in its community moves to another
                                       singleton community only if that id is lower; default 1 */
    int prune;                      /* gsp_prune_mode; default GSP_PRUNE_FLAGS */
    const void *mlp_params;         /* device pointer to gsp_mlp_param_count() floats (learned pruning) */
    int full_sweep_every;           /* learned pruning: every k-th iteration is a plain sweep; default 4 */
    float prune_threshold;          /* learned pruning: skip a vertex when P(move) < this; default 0.5 */
    int count_disconnected;         /* 1: count internally-disconnected communities of the result
                                       (Algorithm 6) into gsp_stats.disconnected; default 0 */
    int refine;                     /* 1: GSP-Leiden -- the refinement phase of the Leiden algorithm
                                       (Section 3.5, gsp_refine) runs after each pass's split, the
                                       refined partition is aggregated, and each super-vertex starts
                                       the next pass in its bound community (in a batch each graph
                                       refines as it does alone); default 0 */
    double refine_theta;            /* randomness of the refinement's choice, >= 0 (0: greedy); default
                                       0.01 */
    uint64_t seed;                  /* seed of the refinement's draws; default 0 */
    void *workspace;                /* optional device scratch owned by the caller (256-byte aligned); NULL:
                                       the library's internal workspace.  With a workspace the call
                                       allocates no device memory and fails with GSP_ERR_CAPACITY when
                                       it runs short; gsp_stats.workspace_bytes of an earlier call on
                                       the same graph and options gives the size it needs */
    size_t workspace_bytes;         /* size of `workspace` in bytes */
    void *stream;                   /* cudaStream_t; NULL = default stream */
} gsp_opts;

#define GSP_MAX_PASS_STATS 32
typedef struct {
    int passes;
    int iterations[GSP_MAX_PASS_STATS];          /* l_i of each pass */
    uint32_t vertices[GSP_MAX_PASS_STATS];       /* |V'| at the start of each pass */
    uint32_t communities[GSP_MAX_PASS_STATS];    /* communities after each pass's split */
    uint64_t edges[GSP_MAX_PASS_STATS];          /* nnz of each pass's graph */
    float ms_move[GSP_MAX_PASS_STATS];
    float ms_split[GSP_MAX_PASS_STATS];
    float ms_aggregate[GSP_MAX_PASS_STATS];
    float ms_other[GSP_MAX_PASS_STATS];
    uint64_t vertices_processed[GSP_MAX_PASS_STATS];  /* vertex visits of local moving */
    uint64_t edges_scanned[GSP_MAX_PASS_STATS];       /* edge visits of local moving */
    uint64_t vertices_skipped[GSP_MAX_PASS_STATS];    /* visits dropped by the learned predictor */
    double move_bytes[GSP_MAX_PASS_STATS];            /* algorithmic bytes of the local-moving kernels */
    float ms_move_kernels[GSP_MAX_PASS_STATS];        /* device time of those kernels (CUDA events) */
    uint32_t final_communities;
    double modularity;
    float ms_total;
    uint32_t disconnected;          /* internally-disconnected communities of the result (Algorithm 6),
                                       GSP_NOT_COUNTED unless gsp_opts.count_disconnected is set */
    uint64_t workspace_bytes;       /* most device scratch bytes the call held at once */
    uint32_t refined[GSP_MAX_PASS_STATS];        /* refined communities of each pass (gsp_opts.refine) */
    float ms_refine[GSP_MAX_PASS_STATS];
} gsp_stats;
#define GSP_NOT_COUNTED 0xFFFFFFFFu

/* Fill *o with the defaults listed in gsp_opts. */
void gsp_default_opts(gsp_opts *o);
const char *gsp_status_string(gsp_status s);
/* Message of the last failing call on this thread (static storage). */
const char *gsp_last_error(void);

/*
 * GSP-Louvain (Algorithm 1).  Input: the graph (float32 weights).  Output:
 * membership[n] (device), each vertex's community numbered 0..k-1 in order of
 * the smallest vertex id of each community; *modularity (host) = Equation 1
 * of that membership on the input graph, reduced in float64; *stats (host,
 * may be NULL).  n == 0 is GSP_ERR_INVALID.  An edgeless graph returns the
 * identity membership and modularity 0 (2m = 0 leaves Equation 1 undefined).
 */
gsp_status gsp_louvain(const uint64_t *offsets, const uint32_t *targets, const float *weights,
                       uint32_t n, uint64_t nnz, const gsp_opts *opts,
                       uint32_t *membership, double *modularity, gsp_stats *stats);

/* As gsp_louvain, but offsets/targets/weights/membership are HOST arrays: the
 * call copies the graph to the device and the membership back. */
gsp_status gsp_louvain_host(const uint64_t *offsets, const uint32_t *targets, const float *weights,
                            uint32_t n, uint64_t nnz, const gsp_opts *opts,
                            uint32_t *membership, double *modularity, gsp_stats *stats);

/*
 * Batched GSP-Louvain over num_graphs independent graphs concatenated into one
 * CSR: graph g owns vertices [graph_vertex_offsets[g], graph_vertex_offsets[g+1])
 * (host array of num_graphs+1 entries) and no edge crosses graphs.  Each graph
 * keeps its own m, tolerance and convergence, as if run alone.  membership is
 * per graph local (0..k_g-1, ordered by smallest vertex); modularity (device,
 * num_graphs doubles) receives each graph's Equation 1 value.
 */
gsp_status gsp_louvain_batched(uint32_t num_graphs, const uint64_t *graph_vertex_offsets,
                               const uint64_t *offsets, const uint32_t *targets, const float *weights,
                               uint32_t n, uint64_t nnz, const gsp_opts *opts,
                               uint32_t *membership, double *modularity, gsp_stats *stats);

/* ---------------------------------------------------------------------------
 * Phase entry points (each one step of Algorithm 1), for reuse and parity
 * tests.  `wt` gives the weight type of `weights`.
 *
 * Sums of weights (K, m, Sigma, aggregated weights, the terms of Q) are
 * exact, and so do not depend on the order of the parallel additions,
 * whenever every weight is a multiple of 2^lsb for some lsb in [-1000, 1000]
 * with the total weight below 2^52 * 2^lsb (then they are taken as 64-bit
 * integers in units of 2^lsb); otherwise they are float64 additions in an
 * unspecified order, exact only while the partial sums stay representable.
 * ------------------------------------------------------------------------- */

/* Section 3: K[i] = sum_j w_ij (self-loop included), float64; *m_host =
 * sum K / 2 (host). */
gsp_status gsp_vertex_weights(const uint64_t *offsets, const uint32_t *targets, const void *weights,
                              int wt, uint32_t n, uint64_t nnz, double *K, double *m_host, void *stream);

/* Equation 1 (second form) for membership C (ids < n); *q_host receives Q. */
gsp_status gsp_modularity(const uint64_t *offsets, const uint32_t *targets, const void *weights,
                          int wt, uint32_t n, uint64_t nnz, const uint32_t *C, double *q_host,
                          void *stream);

/*
 * One frozen-state sweep of local moving (Algorithm 4 with every vertex
 * reading C, Sigma and the community sizes of the sweep's start).  Vertices
 * with active[i] != 0 (active may be NULL = all) pick the best neighbouring
 * community by Equation 2 (ties to the lowest id; a move needs a strictly
 * positive gain; with singleton_rule a singleton moves to a singleton only
 * toward a lower id) and choice[i] receives it (C[i] when not moving).
 * precision is a gsp_precision.  *dq_host receives the summed gain of the
 * moves and *moved_host their count (host pointers, may be NULL).
 */
gsp_status gsp_move_sweep(const uint64_t *offsets, const uint32_t *targets, const void *weights,
                          int wt, uint32_t n, uint64_t nnz, const uint32_t *C, const double *K,
                          const double *Sigma, double m, const uint8_t *active, int precision,
                          int singleton_rule, uint32_t *choice, double *dq_host,
                          uint32_t *moved_host, void *stream);

/*
 * louvainMove (Algorithm 4) from membership C (in/out) and Sigma (in/out,
 * must equal the per-community sums of K).  move is a gsp_move_mode, waves
 * the wave count (1..64, 0: the mode's default), wave_repeats the repeats of a wave in the first
 * iteration (1..8) and no_return_from the first iteration of the no-return
 * rule (0: never), as in gsp_opts.  Returns l_i, the iterations executed,
 * in *iterations_host.
 */
gsp_status gsp_local_move(const uint64_t *offsets, const uint32_t *targets, const void *weights,
                          int wt, uint32_t n, uint64_t nnz, uint32_t *C, const double *K,
                          double *Sigma, double m, double tolerance, int max_iterations, int move,
                          int waves, int wave_repeats, int no_return_from, int precision,
                          int singleton_rule, int *iterations_host, void *stream);

/*
 * Split (Algorithms 2 and 3): labels[i] = the smallest vertex id of the
 * connected component of i in the subgraph of edges (i,j) with C[i] = C[j].
 * Every mode returns the same labels.  *k_host (may be NULL) = number of
 * components.  mode is a gsp_split_mode other than NONE.
 */
gsp_status gsp_split(const uint64_t *offsets, const uint32_t *targets, uint32_t n, uint64_t nnz,
                     const uint32_t *C, int mode, uint32_t *labels, uint32_t *k_host, void *stream);

/*
 * Refinement phase of the Leiden algorithm (Section 3.5), the step of the
 * GSP-Leiden variant.  B: bound membership (ids < n), e.g. local moving's
 * result after the split.  R (output, n entries) receives the refined
 * partition, each refined community named by one of its vertices; every
 * refined community lies inside one bound community and is connected.
 * Within each bound community b, R starts from singletons and every vertex
 * is visited once, in `waves` frozen-state waves (vertex i in wave h(i) mod
 * waves as in local moving; 0 = 17); a vertex still alone in R may join the
 * refined community c of a neighbour in b when E(v, b-v) >= K_v (S_b - K_v)
 * / 2m, E(c, b-c) >= S_c (S_b - S_c) / 2m and the gain g = E(v, c) - K_v S_c
 * / 2m is >= 0 (E the weight between vertex sets, S the sum of K).  It picks
 * among those c and staying (g = 0) with probability proportional to exp(g /
 * theta), drawn as the largest g / theta - ln(-ln u), u a SplitMix64 draw
 * keyed by (seed, pass, vertex, candidate); theta = 0 takes the largest g > 0
 * (ties to the lowest id).  A mover whose own singleton is another mover's
 * target in the same wave stays.  precision (gsp_precision): FP64 computes
 * sums, gains and scores in float64, as a sequential evaluation does; MIXED
 * in float32 (the well-connectedness tests stay float64).  *moves_host (may
 * be NULL) receives the number of vertices that joined another community.
 */
gsp_status gsp_refine(const uint64_t *offsets, const uint32_t *targets, const void *weights, int wt, uint32_t n,
                      uint64_t nnz, const uint32_t *B, uint32_t *R, double theta, uint64_t seed, uint32_t pass,
                      int waves, int precision, uint32_t *moves_host, void *stream);

/* Renumber communities (Algorithm 1): distinct ids of C (all < n) ranked by
 * increasing value become 0..k-1, written to C_dense; *k_host = k. */
gsp_status gsp_renumber(uint32_t n, const uint32_t *C, uint32_t *C_dense, uint32_t *k_host,
                        void *stream);

/* Dendrogram lookup (Algorithm 1): C_top[v] = C_pass[C_top[v]] for v < n_top. */
gsp_status gsp_lookup(uint32_t n_top, uint32_t *C_top, const uint32_t *C_pass, void *stream);

/*
 * louvainAggregate (Algorithm 5): super-vertex graph of membership C (dense,
 * 0..k-1).  Row c of the output holds, for every community d adjacent to c,
 * the summed weight of all edges (i,j) with C[i] = c, C[j] = d, self-loops
 * included, in increasing d, with no gaps.  out_offsets has k+1 entries;
 * out_targets/out_weights (float64) must hold nnz entries.  *out_nnz_host
 * receives the super-edge count.
 */
gsp_status gsp_aggregate(const uint64_t *offsets, const uint32_t *targets, const void *weights,
                         int wt, uint32_t n, uint64_t nnz, const uint32_t *C, uint32_t k,
                         uint64_t *out_offsets, uint32_t *out_targets, double *out_weights,
                         uint64_t *out_nnz_host, void *stream);

/* disconnectedCommunities (Algorithm 6): *count_host = number of communities
 * of C (ids < n) whose vertices are not all connected inside the community;
 * flags (may be NULL, n bytes) receives a 1 at each such community id. */
gsp_status gsp_count_disconnected(const uint64_t *offsets, const uint32_t *targets, uint32_t n,
                                  uint64_t nnz, const uint32_t *C, uint8_t *flags,
                                  uint32_t *count_host, void *stream);

/*
 * Move/no-move traces of the plain method, for training the learned pruning
 * predictor: runs gsp_louvain (opts as given; learned pruning ignored) and,
 * for a sample of vertex visits of local moving (about one in sample_every;
 * every visit when it is 1), records the visit's 6 predictor features (taken
 * before the visit) into features[rows][6] and whether the vertex moved into
 * labels[rows] (device arrays of `capacity` rows).  keys (device, capacity
 * entries, may be NULL) receives each row's visit as pass << 56 |
 * iteration << 48 | repeat << 40 | vertex (vertex of that pass's graph).
 * Rows come in no particular order.  *rows_host = rows written (<= capacity).
 */
gsp_status gsp_louvain_trace(const uint64_t *offsets, const uint32_t *targets, const float *weights,
                             uint32_t n, uint64_t nnz, const gsp_opts *opts, float *features,
                             uint8_t *labels, uint64_t *keys, uint32_t capacity, uint32_t sample_every,
                             uint32_t *rows_host);

/* ---------------------------------------------------------------------------
 * Learned vertex pruning: a 6 -> 32 -> 32 -> 1 MLP (ReLU, sigmoid output)
 * predicting whether a vertex will move.  Parameters are one packed float32
 * array of gsp_mlp_param_count() entries: W1[32][6], b1[32], W2[32][32],
 * b2[32], W3[32], b3.  Features are gsp_mlp_features() rows of 6 floats.
 * ------------------------------------------------------------------------- */
int gsp_mlp_param_count(void);

/* p[r] = sigmoid(MLP(x[r])) for r < rows; weights are rounded to bfloat16,
 * products accumulate in float32. */
gsp_status gsp_mlp_forward(const float *params, const float *x, uint32_t rows, float *p,
                           void *stream);

/* Mean binary cross-entropy of p against labels y (0/1 bytes) with its
 * gradient: grad (gsp_mlp_param_count floats, overwritten) = d loss / d params
 * at the bfloat16-rounded weights; *loss_host = the loss. */
gsp_status gsp_mlp_backward(const float *params, const float *x, const uint8_t *y, uint32_t rows,
                            float *grad, double *loss_host, void *stream);

/* params -= lr * grad (plain SGD step, float32 master weights). */
gsp_status gsp_mlp_sgd(float *params, const float *grad, float lr, void *stream);

/* One Adam step (Kingma & Ba, 2015) of step number t >= 1: with g = grad,
 * m = beta1 m + (1 - beta1) g, v = beta2 v + (1 - beta2) g^2 (m, v: device
 * arrays of gsp_mlp_param_count() floats, zero before the first step),
 * params -= lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps). */
gsp_status gsp_mlp_adam(float *params, const float *grad, float *m, float *v, float lr, float beta1,
                        float beta2, float eps, int t, void *stream);

/* ---------------------------------------------------------------------------
 * Seeded synthetic graphs, drawn on the device with the same counter-based
 * SplitMix64 stream as the host generators.  Each writes a symmetric CSR
 * (self-loops dropped, duplicate pairs merged keeping the smallest weight)
 * into library-owned device memory valid until the next generator call or
 * gsp_release_graph(); pointers are returned through the out arguments.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t n;
    uint64_t nnz;
    uint64_t *offsets;
    uint32_t *targets;
    float *weights;
} gsp_device_graph;

/* R-MAT: edge_factor << scale samples with quadrant thresholds t1<t2<t3 on the
 * top 53 bits of each draw (a, a+b, a+b+c scaled by 2^53). */
gsp_status gsp_gen_rmat(uint32_t scale, uint32_t edge_factor, uint64_t t1, uint64_t t2, uint64_t t3,
                        uint64_t seed, gsp_device_graph *out, void *stream);
/* Batch of planted-partition graphs (host parameter arrays of num_graphs
 * entries: vertices, communities, edge samples, intra threshold on 53 bits,
 * per-graph seed); one graph alone is the single planted-partition case. */
gsp_status gsp_gen_planted_batch(uint32_t num_graphs, const uint64_t *n_g, const uint64_t *k_g,
                                 const uint64_t *edges_g, const uint64_t *p_intra53_g,
                                 const uint64_t *seed_g, gsp_device_graph *out, void *stream);
/* R x Cc grid with random removal (threshold on 53 bits), floor(p_long * E)
 * long-range pairs and weights uniform in [wlo, whi). */
gsp_status gsp_gen_grid(uint32_t R, uint32_t Cc, uint64_t remove53, uint64_t n_long, float wlo,
                        float whi, uint64_t seed, gsp_device_graph *out, void *stream);
void gsp_release_graph(void);

/*
 * Modularity for callers that cannot allocate device memory (embedders whose
 * device memory comes from a fixed pool, such as an inference server or
 * another framework's allocator holding the device; processes that must not
 * grow their device footprint after start-up).  It returns the same value as
 * gsp_modularity, with the same arguments and the same checks (offsets,
 * target and membership ids), but its scratch is one fixed __device__ array
 * inside the library instead of the library workspace: it calls no
 * cudaMalloc, cudaFree or allocating library routine.  Like gsp_modularity it
 * waits for `stream` and returns Q in host memory.  The paper has no
 * counterpart; this is an interface convenience.
 *  - Limit: n <= GSP_STATIC_MAX_VERTICES; larger n returns GSP_ERR_CAPACITY
 *    with a message (use gsp_modularity).
 *  - Every device that loads the library holds GSP_STATIC_SCRATCH_BYTES for
 *    the array until the process exits.
 *  - The first call made in a device's context looks up the array's device
 *    address (with that device current); later calls in that context reuse
 *    it.
 *  - All calls share the one array: calls that overlap on the GPU (several
 *    streams, several host threads) race and give wrong results; serialise
 *    them.  Each call clears the parts of the array it needs.
 */
#define GSP_STATIC_MAX_VERTICES (1u << 20)
#define GSP_STATIC_SCRATCH_BYTES (12ull * GSP_STATIC_MAX_VERTICES + 4 * 8 + 8 + 256)
gsp_status gsp_modularity_static(const uint64_t *offsets, const uint32_t *targets, const void *weights,
                                 int wt, uint32_t n, uint64_t nnz, const uint32_t *C, double *q_host,
                                 void *stream);

/* Number of kernels this library has launched since it was loaded (all
 * devices, all threads); a diagnostic for counting launches in a region. */
uint64_t gsp_kernel_launches(void);

/* Bytes of device memory the library's internal workspaces hold (all
 * devices); a diagnostic: it grows only when a call needs more scratch than
 * any earlier call did. */
uint64_t gsp_workspace_reserved(void);

/* Free the internal workspace of the current device (after waiting for the
 * device to be idle); the next call grows it again.  For callers that
 * switch between graphs of very different sizes. */
void gsp_release_workspace(void);

/* ---------------------------------------------------------------------------
 * Launch geometry of local moving (an implementation choice; the paper has no
 * counterpart).  Each degree class runs as a grid-stride kernel whose grid is
 * capped at a number of blocks per SM: groups of lanes per vertex (degree <=
 * 128), a warp per vertex (129..512), a block per vertex (513..2048) and the
 * grid-wide hub pipeline (> 8192).  Vertices of 2049..8192 edges take one
 * block each with a 16384-slot shared table, one block per SM (no cap).  Any
 * cap in [1, 32] gives the same result in frozen-state (SYNC) mode; only the
 * speed differs.  The setting is
 * process-wide (all devices) and applies to calls started after it is set.
 * ------------------------------------------------------------------------- */
typedef struct {
    int groups_blocks_per_sm;  /* default 8 */
    int w512_blocks_per_sm;    /* default 3 */
    int block_blocks_per_sm;   /* default 4 */
    int hub_blocks_per_sm;     /* default 4 */
    /* SYNC sweeps of graphs with at most this many vertices and no vertex
     * above 2048 edges run as one cooperative launch (a persistent kernel
     * with grid-wide barriers) instead of several launches per wave; 0
     * disables it.  Default 0: on a GB300 the per-wave launches replayed
     * from a CUDA graph were as fast (a wave's dependent loads, not its
     * launches, set the time).  The result is the same either way. */
    uint32_t persist_max_vertices;
    /* Class boundaries: the largest degree served by the group kernel (33..128,
     * default 128), the warp kernel (..512, default 512), the 4096-slot block
     * kernel (..2048, default 2048) and the 16384-slot block kernel (..8192,
     * default 8192); larger degrees go to the hub pipeline.  They must rise. */
    uint32_t group_max_degree;
    uint32_t warp_max_degree;
    uint32_t block_max_degree;
    uint32_t big_max_degree;
} gsp_tuning;

/* Current caps into *out (host).  GSP_ERR_INVALID if out is NULL. */
gsp_status gsp_get_tuning(gsp_tuning *out);

/* Install caps and boundaries (host struct); GSP_ERR_INVALID if a cap is
 * outside [1, 32] or the boundaries break their limits (persist_max_vertices
 * may be any value). */
gsp_status gsp_set_tuning(const gsp_tuning *t);

/*
 * Pick the caps and class boundaries for this graph and install them: times
 * whole gsp_louvain calls on opts (its move mode, waves, wave repeats,
 * precision, split and refinement) under candidate caps and boundaries (each
 * boundary at its limit or half of it), one knob at a time, each trial the
 * better of two calls; keeps a candidate only when it is more than 1 % faster
 * than the current choice, and finally times the pick against the settings
 * in effect at the call once more, keeping the faster.  Device graph as for
 * gsp_louvain (float32 weights); the graph is not modified.  *chosen
 * receives the installed settings, *ms_default the time of a call under the
 * settings in effect at the call, *ms_tuned under the chosen ones, both from
 * the final pair of trials when the search moved (so ms_tuned <= ms_default;
 * host pointers, each may be NULL).  The trials allocate a membership array of n
 * entries outside the workspace and may free and rebuild the workspace.  An
 * edgeless graph is GSP_ERR_INVALID.  Not safe to run concurrently with
 * other calls.
 */
gsp_status gsp_autotune(const uint64_t *offsets, const uint32_t *targets, const float *weights,
                        uint32_t n, uint64_t nnz, const gsp_opts *opts, gsp_tuning *chosen,
                        float *ms_default, float *ms_tuned);

/*
 * As gsp_autotune, timing gsp_louvain_batched calls on the batch (arguments
 * as for gsp_louvain_batched: host graph_vertex_offsets of num_graphs + 1
 * entries, device CSR of the concatenated graphs).  A batch stops each graph
 * on its own gain and runs its passes over the graphs still open, so its
 * degree mix per pass differs from that of one call on the same CSR taken
 * as a single graph.  A batch without any edge is GSP_ERR_INVALID.
 */
gsp_status gsp_autotune_batched(uint32_t num_graphs, const uint64_t *graph_vertex_offsets,
                                const uint64_t *offsets, const uint32_t *targets, const float *weights,
                                uint32_t n, uint64_t nnz, const gsp_opts *opts, gsp_tuning *chosen,
                                float *ms_default, float *ms_tuned);

#ifdef __cplusplus
}
#endif
#endif /* GSP_H */
