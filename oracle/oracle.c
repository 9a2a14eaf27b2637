/*
 * oracle.c -- sequential CPU oracle for GSP-Louvain (Sahu, "An Approach for
 * Addressing Internally-Disconnected Communities in Louvain Algorithm",
 * arXiv 2402.11454).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the package-level smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Plain, slow, obviously correct: every quantity is FP64, every loop runs in
 * vertex order on one thread, and the per-vertex "hashtable" H of the paper
 * is a dense array indexed by community id plus a list of the ids touched.
 * Each function names the passage of the paper it follows.
 *
 * Build with -ffp-contract=off so that a*b+c is never fused: the oracle then
 * rounds identically on x86-64 and AArch64.
 *
 * Graph model (Section 3): undirected G(V,E,w) stored as a symmetric CSR,
 * w_ij = w_ji > 0, self-loops allowed and stored once in their row.
 * K_i = sum_j w_ij (self-loop included), m = sum_{i,j} w_ij / 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t n;            /* |V| */
    uint64_t nnz;          /* directed CSR entries (both directions stored) */
    const uint64_t *off;   /* n+1 row offsets */
    const uint32_t *tgt;   /* nnz neighbour ids */
    const double *w;       /* nnz weights */
} og_graph;

typedef struct {
    int max_passes;             /* MAX_PASSES, Algorithm 1 */
    int max_iterations;         /* MAX_ITERATIONS, Algorithm 4 */
    double tolerance;           /* tau, Algorithm 4 */
    double tolerance_drop;      /* TOLERANCE_DROP, Algorithm 1 */
    double aggregation_tolerance; /* tau_agg, Algorithm 1 */
    int split;                  /* 0 none (GVE-Louvain), 1 LP, 2 LPP, 3 BFS */
    int split_last;             /* 0 Split Pass (SP), 1 Split Last (SL) */
    int sync;                   /* 0 asynchronous in-place moves, 1 frozen-state waves */
    int waves;                  /* frozen-state waves per iteration */
    int wave_hash;              /* 1: vertex i in wave og_wave_hash(i) mod waves; 0: i mod waves */
    int wave_repeats;           /* frozen-state repeats of a wave in the first iteration of a pass */
    int no_return_from;         /* frozen-state: from this iteration on no move back to the community left
                                   in the previous iteration (0: never) */
    int singleton_rule;         /* frozen-state sweeps only: singleton -> singleton moves go to lower ids */
    int refine;                 /* 1: Leiden refinement (Section 3.5) before each aggregation (GSP-Leiden) */
    double refine_theta;        /* randomness theta of the refinement choice (0: greedy) */
    uint64_t seed;              /* seed of the refinement draws */
} og_opts;

typedef struct {
    int passes;
    int iterations[64];
    uint32_t vertices[64];      /* |V'| at the start of each pass */
    uint32_t communities[64];   /* communities after the split of each pass */
    double modularity;
    uint32_t final_communities;
} og_stats;

/* ------------------------------------------------------------------ */
/* Section 3: weighted degree K_i and total weight m.                   */
/* ------------------------------------------------------------------ */
double og_vertex_weights(const og_graph *g, double *K)
{
    double two_m = 0.0;
    for (uint32_t i = 0; i < g->n; i++) {
        double k = 0.0;
        for (uint64_t e = g->off[i]; e < g->off[i + 1]; e++) k += g->w[e];
        K[i] = k;
        two_m += k;
    }
    return two_m / 2.0;
}

/* ------------------------------------------------------------------ */
/* Equation 1, second form: Q = sum_c [ sigma_c/2m - (Sigma_c/2m)^2 ],  */
/* sigma_c = weight of directed entries (i,j) with C_i = C_j = c,       */
/* Sigma_c = sum of K_i over i in c.  Community ids must be < n.        */
/* An edgeless graph (2m = 0) has Q := 0.                               */
/* ------------------------------------------------------------------ */
double og_modularity(const og_graph *g, const uint32_t *C)
{
    uint32_t n = g->n;
    double *sigma = calloc(n ? n : 1, sizeof(double));
    double *Sigma = calloc(n ? n : 1, sizeof(double));
    double two_m = 0.0;
    for (uint32_t i = 0; i < n; i++) {
        for (uint64_t e = g->off[i]; e < g->off[i + 1]; e++) {
            uint32_t j = g->tgt[e];
            Sigma[C[i]] += g->w[e];
            if (C[i] == C[j]) sigma[C[i]] += g->w[e];
            two_m += g->w[e];
        }
    }
    double q = 0.0;
    if (two_m > 0.0) {
        for (uint32_t c = 0; c < n; c++) {
            double a = Sigma[c] / two_m;
            q += sigma[c] / two_m - a * a;
        }
    }
    free(sigma);
    free(Sigma);
    return q;
}

/* ------------------------------------------------------------------ */
/* Equation 2: delta-modularity of moving i from community d to c.      */
/* K_{i->c}, K_{i->d} exclude the self-loop of i; Sigma_d includes K_i. */
/* ------------------------------------------------------------------ */
double og_delta_modularity(double Kic, double Kid, double Ki, double Sc, double Sd, double m)
{
    return (Kic - Kid) / m - Ki * (Ki + Sc - Sd) / (2.0 * m * m);
}

/* scanCommunities (Algorithm 4): H[C[j]] += w over the edges of i,      */
/* skipping the self-loop unless self is set.  H is a dense array that  */
/* starts at zero; every id touched for the first time is appended to   */
/* list, and the list length is returned.                               */
static uint32_t scan_communities(const og_graph *g, const uint32_t *C, uint32_t i, int self,
                                 double *H, uint8_t *seen, uint32_t *list, uint32_t len)
{
    for (uint64_t e = g->off[i]; e < g->off[i + 1]; e++) {
        uint32_t j = g->tgt[e];
        if (!self && j == i) continue;
        uint32_t c = C[j];
        if (!seen[c]) { seen[c] = 1; list[len++] = c; }
        H[c] += g->w[e];
    }
    return len;
}

static void clear_table(double *H, uint8_t *seen, const uint32_t *list, uint32_t len)
{
    for (uint32_t t = 0; t < len; t++) { H[list[t]] = 0.0; seen[list[t]] = 0; }
}

/*
 * Best move of vertex i (Algorithm 4: "best community linked to i" and its
 * delta-modularity, by Equation 2).  Candidates are the communities c != d
 * present in H; ties go to the lowest community id.  Returns d (no move)
 * unless the best delta-modularity is strictly positive.  best/second
 * receive the two largest candidate values (-inf when absent) so that a
 * caller can tell near-ties apart.  size/singleton_rule implement the
 * lower-id rule for a vertex alone in its community moving to another
 * singleton community (frozen-state sweeps only).
 */
static uint32_t best_move(const og_graph *g, const uint32_t *C, const double *K, const double *Sigma,
                          const uint32_t *size, int singleton_rule, double m, uint32_t i,
                          double *H, uint8_t *seen, uint32_t *list, double *best_out, double *second_out,
                          double *kid_out)
{
    uint32_t d = C[i];
    uint32_t len = scan_communities(g, C, i, 0, H, seen, list, 0);
    double Kid = H[d];   /* zero when no neighbour lies in d */
    if (kid_out) *kid_out = Kid;
    double best = -INFINITY, second = -INFINITY;
    uint32_t cbest = d;
    for (uint32_t t = 0; t < len; t++) {          /* the best candidate */
        uint32_t c = list[t];
        if (c == d) continue;
        double dq = og_delta_modularity(H[c], Kid, K[i], Sigma[c], Sigma[d], m);
        if (dq > best || (dq == best && c < cbest)) { best = dq; cbest = c; }
    }
    for (uint32_t t = 0; t < len; t++) {          /* the runner-up */
        uint32_t c = list[t];
        if (c == d || c == cbest) continue;
        double dq = og_delta_modularity(H[c], Kid, K[i], Sigma[c], Sigma[d], m);
        if (dq > second) second = dq;
    }
    clear_table(H, seen, list, len);
    if (best_out) *best_out = best;
    if (second_out) *second_out = second;
    if (cbest == d || !(best > 0.0)) return d;
    if (singleton_rule && size && size[d] == 1 && size[cbest] == 1 && cbest > d) return d;
    return cbest;
}

/*
 * One frozen-state sweep of the local-moving phase (Algorithm 4, with every
 * vertex reading the C and Sigma of the sweep's start).  Processes the
 * vertices with active[i] != 0 and writes the chosen community to choice[i]
 * (C[i] for inactive vertices or no move), plus the best and second-best
 * candidate delta-modularity.  Nothing is applied.
 */
void og_move_sweep_sync(const og_graph *g, const uint32_t *C, const double *K, const double *Sigma,
                        const uint32_t *size, int singleton_rule, double m, const uint8_t *active,
                        uint32_t *choice, double *best, double *second)
{
    uint32_t n = g->n;
    double *H = calloc(n, sizeof(double));
    uint8_t *seen = calloc(n, 1);
    uint32_t *list = malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t i = 0; i < n; i++) {
        double b = -INFINITY, s = -INFINITY;
        choice[i] = C[i];
        if (active && !active[i]) { best[i] = b; second[i] = s; continue; }
        choice[i] = best_move(g, C, K, Sigma, size, singleton_rule, m, i, H, seen, list, &b, &s, NULL);
        best[i] = b;
        second[i] = s;
    }
    free(H); free(seen); free(list);
}

/*
 * louvainMove (Algorithm 4).  Updates C and Sigma in place and returns l_i,
 * the number of iterations executed (including the one that met the
 * tolerance).  Every vertex starts unprocessed; a processed vertex is marked
 * processed, and a vertex that moves marks its neighbours unprocessed.
 *   sync = 0: one thread walks the unprocessed vertices in id order and each
 *             move is applied at once (the in-place form of the paper).
 *   sync = 1: the parallel loop is made deterministic by waves: the vertices
 *             of an iteration are split into `waves` waves, taken in order;
 *             every vertex of a wave reads the C, Sigma and community sizes
 *             left by the earlier waves, and the wave's moves are applied
 *             after it.  Vertex i belongs to wave og_wave_hash(i) mod waves
 *             (wave_hash = 1), so that no arithmetic pattern of the ids
 *             (vertex v of a planted community v mod k, R-MAT's bit-structured
 *             ids) gathers a community into one wave, or to wave i mod waves
 *             (wave_hash = 0).  waves = 1 is the fully synchronous loop; with
 *             wave_hash = 0, waves = |V'| is the one-thread loop in id order.
 *             In the first iteration a wave runs `repeats` times (at least
 *             once; later iterations once): a repeat takes the vertices of the
 *             wave that the previous repeat's moves marked unprocessed again,
 *             on the state those moves left (the pruning rule of Algorithm 4
 *             applied within the wave).  With one vertex per wave a vertex
 *             never marks itself, so repeats change nothing there.  From
 *             iteration no_return_from on (0: never), a vertex does not move
 *             back to the community it left in the previous iteration: the
 *             one-thread loop raises Q with every move and cannot cycle,
 *             while simultaneous decisions can fall into a two-iteration cycle
 *             whose claimed gains stay above tau.
 * dq_iter (optional) receives the total delta-modularity of each iteration.
 */
/*
 * Visit trace for the learned pruning predictor (not part of the paper's
 * method; the predictor is an addition checked against this record).  Every
 * vertex visit of local moving appends one record of OG_TRACE_FIELDS
 * doubles: pass, iteration, repeat, vertex, degree, K_i, then the state the
 * vertex's previous visit in this pass left (the fraction K_{i->C_i}/K_i of
 * its weight inside its community, its best candidate's delta-modularity
 * times m/K_i clamped to [-1, 1] (0 without a candidate), whether it moved;
 * before a first visit 0, 1, 1), whether this visit moved it, and the
 * largest K of the pass's graph.  Records beyond cap are counted, not kept.
 */
#define OG_TRACE_FIELDS 11
typedef struct {
    double *rec;
    uint64_t cap, len;
    int pass;
    double max_K;
    double *kept, *gain;      /* per vertex of the pass's graph */
    uint8_t *moved;
} og_trace;

static void trace_visit(og_trace *tr, const og_graph *g, int it, int rep, uint32_t i, double Ki, double kid,
                        double best, double m, int moved)
{
    if (!tr) return;
    if (tr->len < tr->cap) {
        double *r = tr->rec + tr->len * OG_TRACE_FIELDS;
        r[0] = tr->pass; r[1] = it; r[2] = rep; r[3] = i;
        r[4] = (double)(g->off[i + 1] - g->off[i]); r[5] = Ki;
        r[6] = tr->kept[i]; r[7] = tr->gain[i]; r[8] = tr->moved[i];
        r[9] = moved; r[10] = tr->max_K;
    }
    tr->len++;
    double gain = isfinite(best) ? best : 0.0;
    double x = Ki > 0.0 ? gain * m / Ki : 0.0;
    tr->kept[i] = Ki > 0.0 ? kid / Ki : 0.0;
    tr->gain[i] = x < -1.0 ? -1.0 : (x > 1.0 ? 1.0 : x);
    tr->moved[i] = (uint8_t)moved;
}

/* Wave hash: the MurmurHash3 32-bit finaliser (Appleby) of the vertex id. */
uint32_t og_wave_hash(uint32_t i)
{
    i ^= i >> 16;
    i *= 0x85ebca6bu;
    i ^= i >> 13;
    i *= 0xc2b2ae35u;
    i ^= i >> 16;
    return i;
}

static int move_impl(const og_graph *g, uint32_t *C, const double *K, double *Sigma, double m, double tau,
                     int max_iterations, int sync, int waves, int wave_hash, int repeats, int no_return_from,
                     int singleton_rule, double *dq_iter, og_trace *tr)
{
    uint32_t n = g->n;
    double *H = calloc(n ? n : 1, sizeof(double));
    uint8_t *seen = calloc(n ? n : 1, 1);
    uint32_t *list = malloc(sizeof(uint32_t) * (n ? n : 1));
    uint8_t *unprocessed = malloc(n ? n : 1);
    uint32_t *choice = malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *size = calloc(n ? n : 1, sizeof(uint32_t));
    memset(unprocessed, 1, n);
    for (uint32_t i = 0; i < n; i++) size[C[i]]++;
    /* frozen-state schedule: the vertices of each wave in id order, the
     * community each vertex last left and the iteration it left it */
    uint32_t W = waves < 1 ? 1u : (uint32_t)waves;
    uint32_t *wstart = calloc((size_t)W + 1, sizeof(uint32_t));
    uint32_t *wlist = malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *left = malloc(sizeof(uint32_t) * (n ? n : 1));
    int *left_it = malloc(sizeof(int) * (n ? n : 1));
    for (uint32_t i = 0; i < n; i++) {
        wstart[(wave_hash ? og_wave_hash(i) : i) % W + 1]++;
        left_it[i] = -2;
    }
    for (uint32_t k = 0; k < W; k++) wstart[k + 1] += wstart[k];
    {
        uint32_t *fill = malloc(sizeof(uint32_t) * ((size_t)W + 1));
        memcpy(fill, wstart, sizeof(uint32_t) * ((size_t)W + 1));
        for (uint32_t i = 0; i < n; i++) wlist[fill[(wave_hash ? og_wave_hash(i) : i) % W]++] = i;
        free(fill);
    }
    int li = 0;
    for (int it = 0; it < max_iterations; it++) {
        double dQ = 0.0;
        li = it + 1;
        if (!sync) {
            for (uint32_t i = 0; i < n; i++) {
                if (!unprocessed[i]) continue;
                unprocessed[i] = 0;
                double b, kid;
                uint32_t c = best_move(g, C, K, Sigma, NULL, 0, m, i, H, seen, list, &b, NULL, &kid);
                trace_visit(tr, g, it, 0, i, K[i], kid, b, m, c != C[i]);
                if (c == C[i]) continue;
                Sigma[C[i]] -= K[i];
                Sigma[c] += K[i];
                size[C[i]]--; size[c]++;
                C[i] = c;
                dQ += b;
                for (uint64_t e = g->off[i]; e < g->off[i + 1]; e++)
                    if (g->tgt[e] != i) unprocessed[g->tgt[e]] = 1;
            }
        } else {
            int R = (it == 0 && repeats > 1) ? repeats : 1;
            int no_return = no_return_from > 0 && it >= no_return_from;
            for (uint32_t wv = 0; wv < W; wv++) {
                for (int r = 0; r < R; r++) {
                    /* decide: every unprocessed vertex of the wave, frozen state */
                    for (uint32_t t = wstart[wv]; t < wstart[wv + 1]; t++) {
                        uint32_t i = wlist[t];
                        choice[i] = C[i];
                        if (!unprocessed[i]) continue;
                        unprocessed[i] = 0;
                        double b, kid;
                        choice[i] = best_move(g, C, K, Sigma, size, singleton_rule, m, i, H, seen, list, &b, NULL,
                                              &kid);
                        if (no_return && choice[i] == left[i] && left_it[i] == it - 1) choice[i] = C[i];
                        trace_visit(tr, g, it, r, i, K[i], kid, b, m, choice[i] != C[i]);
                        if (choice[i] != C[i]) dQ += b;
                    }
                    /* apply the wave's moves; movers mark their neighbours */
                    for (uint32_t t = wstart[wv]; t < wstart[wv + 1]; t++) {
                        uint32_t i = wlist[t];
                        if (choice[i] == C[i]) continue;
                        Sigma[C[i]] -= K[i];
                        Sigma[choice[i]] += K[i];
                        size[C[i]]--; size[choice[i]]++;
                        for (uint64_t e = g->off[i]; e < g->off[i + 1]; e++)
                            if (g->tgt[e] != i) unprocessed[g->tgt[e]] = 1;
                        left[i] = C[i];
                        left_it[i] = it;
                        C[i] = choice[i];
                    }
                }
            }
        }
        if (dq_iter) dq_iter[it] = dQ;
        if (dQ <= tau) break;
    }
    free(H); free(seen); free(list); free(unprocessed); free(choice); free(size);
    free(wstart); free(wlist); free(left); free(left_it);
    return li;
}

int og_move(const og_graph *g, uint32_t *C, const double *K, double *Sigma, double m, double tau,
            int max_iterations, int sync, int waves, int wave_hash, int repeats, int no_return_from,
            int singleton_rule, double *dq_iter)
{
    return move_impl(g, C, K, Sigma, m, tau, max_iterations, sync, waves, wave_hash, repeats, no_return_from,
                     singleton_rule, dq_iter, NULL);
}

/* ------------------------------------------------------------------ */
/* splitDisconnectedLp (Algorithm 2).  Labels start at the vertex id;  */
/* each vertex takes the minimum label over its same-community         */
/* neighbours until no label changes.  prune != 0 is the LPP variant:  */
/* only unprocessed vertices are visited, and a vertex whose label     */
/* changed marks its same-community neighbours unprocessed.  Returns   */
/* the number of iterations.                                           */
/* ------------------------------------------------------------------ */
int og_split_lp(const og_graph *g, const uint32_t *C, uint32_t *Cp, int prune)
{
    uint32_t n = g->n;
    uint8_t *unprocessed = malloc(n ? n : 1);
    for (uint32_t i = 0; i < n; i++) { unprocessed[i] = 1; Cp[i] = i; }
    int iters = 0;
    for (;;) {
        uint64_t dN = 0;
        iters++;
        for (uint32_t i = 0; i < n; i++) {
            if (!unprocessed[i]) continue;
            if (prune) unprocessed[i] = 0;
            uint32_t cmin = Cp[i];
            for (uint64_t e = g->off[i]; e < g->off[i + 1]; e++) {
                uint32_t j = g->tgt[e];
                if (C[j] == C[i] && Cp[j] < cmin) cmin = Cp[j];
            }
            if (cmin == Cp[i]) continue;
            Cp[i] = cmin;
            dN++;
            if (prune)
                for (uint64_t e = g->off[i]; e < g->off[i + 1]; e++)
                    if (C[g->tgt[e]] == C[i]) unprocessed[g->tgt[e]] = 1;
        }
        if (dN == 0) break;
    }
    free(unprocessed);
    return iters;
}

/* bfsVisitForEach: breadth-first search from s over the vertices j with  */
/* C[j] == c, marking vis; calls back by writing label into Cp (when Cp  */
/* is given) and returns the number of vertices reached.                */
static uint64_t bfs_visit(const og_graph *g, const uint32_t *C, uint32_t c, uint32_t s, uint8_t *vis,
                          uint32_t *queue, uint32_t *Cp, uint32_t label)
{
    uint64_t head = 0, tail = 0;
    vis[s] = 1;
    queue[tail++] = s;
    while (head < tail) {
        uint32_t u = queue[head++];
        if (Cp) Cp[u] = label;
        for (uint64_t e = g->off[u]; e < g->off[u + 1]; e++) {
            uint32_t j = g->tgt[e];
            if (vis[j] || C[j] != c) continue;
            vis[j] = 1;
            queue[tail++] = j;
        }
    }
    return tail;
}

/* ------------------------------------------------------------------ */
/* splitDisconnectedBfs (Algorithm 3) with one thread: vertices are    */
/* scanned in id order; an unvisited vertex i seeds a BFS inside its   */
/* community C[i], labelling everything reached with C'[i] = i.  (The  */
/* BFS condition is read as C[j] = C[i]; the printed condition compares */
/* C[j] with itself.)  With one thread the busy flags never block.     */
/* ------------------------------------------------------------------ */
void og_split_bfs(const og_graph *g, const uint32_t *C, uint32_t *Cp)
{
    uint32_t n = g->n;
    uint8_t *vis = calloc(n ? n : 1, 1);
    uint32_t *queue = malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t i = 0; i < n; i++) Cp[i] = i;
    for (uint32_t i = 0; i < n; i++) {
        if (vis[i]) continue;
        bfs_visit(g, C, C[i], i, vis, queue, Cp, Cp[i]);
    }
    free(vis); free(queue);
}

/* Renumber communities (Algorithm 1): distinct ids ranked by increasing */
/* value become 0..k-1.  Ids must be < n.  Returns k.                   */
uint32_t og_renumber(uint32_t n, uint32_t *C)
{
    uint32_t *rank = malloc(sizeof(uint32_t) * (n ? n : 1));
    uint8_t *used = calloc(n ? n : 1, 1);
    for (uint32_t i = 0; i < n; i++) used[C[i]] = 1;
    uint32_t k = 0;
    for (uint32_t c = 0; c < n; c++) rank[c] = used[c] ? k++ : 0;
    for (uint32_t i = 0; i < n; i++) C[i] = rank[C[i]];
    free(rank); free(used);
    return k;
}

/* Dendrogram lookup (Algorithm 1): C[v] <- C'[C[v]]. */
void og_lookup(uint64_t n_top, uint32_t *C, const uint32_t *Cp)
{
    for (uint64_t v = 0; v < n_top; v++) C[v] = Cp[C[v]];
}

/* ------------------------------------------------------------------ */
/* louvainAggregate (Algorithm 5).  C must be dense in [0,k).          */
/*  1. community-vertex CSR: count, exclusive scan, scatter;            */
/*  2. super-vertex offsets from each community's total degree;         */
/*  3. per community, H over the edges of its members (self = true),    */
/*     then the (d, w) pairs become the edges of super-vertex c.        */
/* The holey CSR of the paper is compacted, and each row is emitted in  */
/* increasing d, so that the result is canonical.  out_off has k+1      */
/* entries; out_tgt/out_w need room for nnz entries.  Returns the       */
/* number of super-edges.                                               */
/* ------------------------------------------------------------------ */
uint64_t og_aggregate(const og_graph *g, const uint32_t *C, uint32_t k,
                      uint64_t *out_off, uint32_t *out_tgt, double *out_w)
{
    uint32_t n = g->n;
    uint64_t *coff = calloc((size_t)k + 1, sizeof(uint64_t));
    uint32_t *cverts = malloc(sizeof(uint32_t) * (n ? n : 1));
    uint64_t *fill = malloc(sizeof(uint64_t) * ((size_t)k + 1));
    /* countCommunityVertices + exclusiveScan */
    for (uint32_t i = 0; i < n; i++) coff[C[i] + 1]++;
    for (uint32_t c = 0; c < k; c++) coff[c + 1] += coff[c];
    memcpy(fill, coff, sizeof(uint64_t) * ((size_t)k + 1));
    for (uint32_t i = 0; i < n; i++) cverts[fill[C[i]]++] = i;
    /* communityTotalDegree + exclusiveScan: the super-vertex row bounds */
    uint64_t *yoff = calloc((size_t)k + 1, sizeof(uint64_t));
    for (uint32_t i = 0; i < n; i++) yoff[C[i] + 1] += g->off[i + 1] - g->off[i];
    for (uint32_t c = 0; c < k; c++) yoff[c + 1] += yoff[c];
    /* per-community hashtable; rows written gap-free and sorted */
    double *H = calloc(k ? k : 1, sizeof(double));
    uint8_t *seen = calloc(k ? k : 1, 1);
    uint32_t *list = malloc(sizeof(uint32_t) * (k ? k : 1));
    uint64_t pos = 0;
    out_off[0] = 0;
    for (uint32_t c = 0; c < k; c++) {
        uint32_t len = 0;
        for (uint64_t t = coff[c]; t < coff[c + 1]; t++)
            len = scan_communities(g, C, cverts[t], 1, H, seen, list, len);
        /* emit in increasing d: walk the touched ids after sorting them */
        for (uint32_t a = 1; a < len; a++) {          /* insertion sort */
            uint32_t x = list[a];
            uint32_t b = a;
            while (b > 0 && list[b - 1] > x) { list[b] = list[b - 1]; b--; }
            list[b] = x;
        }
        for (uint32_t t = 0; t < len; t++) {
            out_tgt[pos] = list[t];
            out_w[pos] = H[list[t]];
            pos++;
        }
        clear_table(H, seen, list, len);
        out_off[c + 1] = pos;
    }
    free(coff); free(cverts); free(fill); free(yoff); free(H); free(seen); free(list);
    return pos;
}

/* ------------------------------------------------------------------ */
/* disconnectedCommunities (Algorithm 6) with one thread: S = community */
/* sizes; the first vertex met of each community seeds a BFS inside it; */
/* the community is flagged when fewer than S[c] vertices are reached.  */
/* D (optional, n entries) receives the flags.  Returns how many.       */
/* ------------------------------------------------------------------ */
uint32_t og_disconnected(const og_graph *g, const uint32_t *C, uint8_t *D)
{
    uint32_t n = g->n;
    uint64_t *S = calloc(n ? n : 1, sizeof(uint64_t));
    uint8_t *vis = calloc(n ? n : 1, 1);
    uint32_t *queue = malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t count = 0;
    if (D) memset(D, 0, n);
    for (uint32_t i = 0; i < n; i++) S[C[i]]++;
    for (uint32_t i = 0; i < n; i++) {
        uint32_t c = C[i];
        if (S[c] == 0) continue;
        uint64_t reached = bfs_visit(g, C, c, i, vis, queue, NULL, 0);
        if (reached < S[c]) { if (D) D[c] = 1; count++; }
        S[c] = 0;
    }
    free(S); free(vis); free(queue);
    return count;
}

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output of the   */
/* generator whose state has reached x, i.e. x advanced by the golden  */
/* gamma and passed through the variant-13 mixer.                      */
/* ------------------------------------------------------------------ */
uint64_t og_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Uniform draw in (0,1) for the refinement choice of vertex v among    */
/* candidate c in a pass: SplitMix64 as a counter-based generator, the  */
/* key (v, c) mixed into a per-pass stream of the seed.  52 random bits */
/* plus one half, so the value is exact and never 0 or 1.               */
double og_refine_uniform(uint64_t seed, uint32_t pass, uint32_t v, uint32_t c)
{
    uint64_t s = og_splitmix64(seed + 0x9e3779b97f4a7c15ull * ((uint64_t)pass + 1));
    uint64_t r = og_splitmix64(s ^ (((uint64_t)v << 32) | c));
    return ((double)(r >> 12) + 0.5) * 0x1.0p-52;
}

/* ------------------------------------------------------------------ */
/* Refinement phase of the Leiden algorithm (Section 3.5), for the      */
/* GSP-Leiden variant the conclusion mentions.  B is the bound          */
/* membership left by local moving (ids < n); R receives the refined    */
/* membership, each refined community named by one of its vertices.     */
/*                                                                      */
/* R starts from singletons.  A vertex v that is still alone in R may   */
/* join the refined community c of a neighbour inside its own bound     */
/* community b when                                                     */
/*   - v is well connected to b:  E(v, b-v) >= K_v (S_b - K_v) / 2m,    */
/*   - c is well connected to b:  E(c, b-c) >= S_c (S_b - S_c) / 2m,    */
/*   - the gain is not negative:  g_c = E(v, c) - K_v S_c / 2m >= 0     */
/* (g_c is m times Equation 2 for v leaving its singleton; S_b, S_c sum */
/* K over b and c; E(x, y) is the weight between vertex sets x and y).  */
/* With theta > 0 the choice among the eligible c and staying (gain 0)  */
/* is random with weight exp(g / theta), drawn as the largest           */
/* g / theta + Gumbel noise, the noise -ln(-ln u) of an independent     */
/* uniform u per (v, candidate); theta = 0 is the greedy limit: the     */
/* largest strictly positive gain, ties to the lowest id.               */
/*                                                                      */
/* Parallel form: the vertices are visited once, in the frozen-state    */
/* waves of local moving (vertex i in wave hash(i) mod W, or i mod W);  */
/* all decisions of a wave read the wave's start state, and a mover     */
/* whose own singleton is another mover's target in the same wave       */
/* stays, so that every target keeps its members.  E(c, b-c) is kept   */
/* per refined community and updated as vertices join.  Returns the     */
/* number of vertices that joined another refined community.            */
/* ------------------------------------------------------------------ */
uint32_t og_refine(const og_graph *g, const uint32_t *B, uint32_t *R, double theta, uint64_t seed, uint32_t pass,
                   int waves, int wave_hash)
{
    uint32_t n = g->n;
    size_t nn = n ? n : 1;
    double *K = malloc(sizeof(double) * nn);
    double *SB = calloc(nn, sizeof(double));      /* S_b per bound community */
    double *SR = malloc(sizeof(double) * nn);     /* S_c per refined community */
    double *ext = calloc(nn, sizeof(double));     /* E(c, b - c) per refined community */
    double *H = calloc(nn, sizeof(double));       /* E(v, c) of the vertex being decided */
    double *wvt = malloc(sizeof(double) * nn);    /* E(v, target) at the decision */
    uint32_t *size = malloc(sizeof(uint32_t) * nn);
    uint32_t *T = malloc(sizeof(uint32_t) * nn);
    uint32_t *list = malloc(sizeof(uint32_t) * nn);
    uint8_t *seen = calloc(nn, 1);
    uint8_t *targeted = calloc(nn, 1);
    uint8_t *joined = calloc(nn, 1);
    double m = og_vertex_weights(g, K);
    for (uint32_t v = 0; v < n; v++) {
        SB[B[v]] += K[v];
        R[v] = v; SR[v] = K[v]; size[v] = 1;
    }
    for (uint32_t v = 0; v < n; v++)
        for (uint64_t e = g->off[v]; e < g->off[v + 1]; e++) {
            uint32_t u = g->tgt[e];
            if (u != v && B[u] == B[v]) ext[v] += g->w[e];
        }
    uint32_t moves = 0;
    uint32_t W = waves < 1 ? 1u : (uint32_t)waves;
    uint32_t *wstart = calloc((size_t)W + 1, sizeof(uint32_t));
    uint32_t *wlist = malloc(sizeof(uint32_t) * nn);
    for (uint32_t i = 0; i < n; i++) wstart[(wave_hash ? og_wave_hash(i) : i) % W + 1]++;
    for (uint32_t k = 0; k < W; k++) wstart[k + 1] += wstart[k];
    {
        uint32_t *fill = malloc(sizeof(uint32_t) * ((size_t)W + 1));
        memcpy(fill, wstart, sizeof(uint32_t) * ((size_t)W + 1));
        for (uint32_t i = 0; i < n; i++) wlist[fill[(wave_hash ? og_wave_hash(i) : i) % W]++] = i;
        free(fill);
    }
    double two_m = 2.0 * m;
    for (uint32_t wv = 0; m > 0.0 && wv < W; wv++) {
        /* decide, every vertex of the wave from the wave's start state */
        for (uint32_t t = wstart[wv]; t < wstart[wv + 1]; t++) {
            uint32_t v = wlist[t];
            T[v] = v;
            wvt[v] = 0.0;
            if (size[v] != 1 || R[v] != v) continue;             /* only singletons move */
            uint32_t b = B[v];
            if (!(ext[v] >= K[v] * (SB[b] - K[v]) / two_m)) continue;
            uint32_t len = 0;
            for (uint64_t e = g->off[v]; e < g->off[v + 1]; e++) {
                uint32_t u = g->tgt[e];
                if (u == v || B[u] != b) continue;
                uint32_t c = R[u];
                if (!seen[c]) { seen[c] = 1; list[len++] = c; }
                H[c] += g->w[e];
            }
            int have = 0;
            double best = 0.0;
            uint32_t bc = v;
            if (theta > 0.0) { have = 1; best = -log(-log(og_refine_uniform(seed, pass, v, v))); }
            for (uint32_t k = 0; k < len; k++) {
                uint32_t c = list[k];
                if (!(ext[c] >= SR[c] * (SB[b] - SR[c]) / two_m)) continue;
                double gain = H[c] - K[v] * SR[c] / two_m;
                double s;
                if (theta > 0.0) {
                    if (gain < 0.0) continue;
                    s = gain / theta + -log(-log(og_refine_uniform(seed, pass, v, c)));
                } else {
                    if (!(gain > 0.0)) continue;
                    s = gain;
                }
                if (!have || s > best || (s == best && c < bc)) { have = 1; best = s; bc = c; }
            }
            T[v] = bc;
            if (bc != v) wvt[v] = H[bc];
            for (uint32_t k = 0; k < len; k++) { H[list[k]] = 0.0; seen[list[k]] = 0; }
        }
        /* a mover whose singleton is targeted by another mover stays */
        for (uint32_t t = wstart[wv]; t < wstart[wv + 1]; t++) {
            uint32_t v = wlist[t];
            if (T[v] != v) targeted[T[v]] = 1;
        }
        for (uint32_t t = wstart[wv]; t < wstart[wv + 1]; t++) {
            uint32_t v = wlist[t];
            joined[v] = (T[v] != v && !targeted[v]);
        }
        for (uint32_t t = wstart[wv]; t < wstart[wv + 1]; t++) {
            uint32_t v = wlist[t];
            if (!joined[v]) continue;
            uint32_t c = T[v];
            R[v] = c;
            size[c]++; size[v] = 0;
            SR[c] += K[v];
            moves++;
        }
        /* E(c, b - c) of each target: plus the joiner's edges to the rest  */
        /* of b, less its edges to the target's earlier members (counted   */
        /* from both sides) and to the wave's other joiners of that target */
        for (uint32_t t = wstart[wv]; t < wstart[wv + 1]; t++) {
            uint32_t v = wlist[t];
            if (!joined[v]) continue;
            double co = 0.0;
            for (uint64_t e = g->off[v]; e < g->off[v + 1]; e++) {
                uint32_t u = g->tgt[e];
                if (u != v && joined[u] && T[u] == T[v]) co += g->w[e];
            }
            ext[T[v]] += ext[v] - 2.0 * wvt[v] - co;
        }
        for (uint32_t t = wstart[wv]; t < wstart[wv + 1]; t++) {
            uint32_t v = wlist[t];
            targeted[T[v]] = 0;
            joined[v] = 0;
        }
    }
    free(K); free(SB); free(SR); free(ext); free(H); free(wvt); free(size); free(T); free(list);
    free(seen); free(targeted); free(joined); free(wstart); free(wlist);
    return moves;
}

static void run_split(const og_graph *g, const uint32_t *C, uint32_t *Cp, int mode)
{
    if (mode == 1) og_split_lp(g, C, Cp, 0);
    else if (mode == 2) og_split_lp(g, C, Cp, 1);
    else if (mode == 3) og_split_bfs(g, C, Cp);
    else memcpy(Cp, C, sizeof(uint32_t) * g->n);
}

/* Final numbering: communities ranked by their smallest vertex id. */
static uint32_t canonical_numbering(uint32_t n, uint32_t *C)
{
    uint32_t *id = malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t c = 0; c < n; c++) id[c] = UINT32_MAX;
    uint32_t k = 0;
    for (uint32_t v = 0; v < n; v++) {
        if (id[C[v]] == UINT32_MAX) id[C[v]] = k++;
        C[v] = id[C[v]];
    }
    free(id);
    return k;
}

/* ------------------------------------------------------------------ */
/* louvain (Algorithm 1), GSP-Louvain driver.  G is the input graph;   */
/* C receives the final membership numbered 0..k-1 by smallest vertex   */
/* id.  Each pass: K' = vertexWeights(G'), Sigma' from C' (identity),  */
/* louvainMove, split (Split Pass), global convergence when l_i <= 1,   */
/* low-shrink stop when |Gamma|/|V'| > tau_agg, renumber, dendrogram    */
/* lookup, louvainAggregate, tau /= TOLERANCE_DROP.  A final lookup     */
/* follows the loop.  With split_last the split runs once, on G and the */
/* final membership.  With refine (GSP-Leiden) the refined partition  */
/* of C' (og_refine) is what the low-shrink test counts, the lookup     */
/* follows and the aggregation merges, and each super-vertex starts   */
/* the next pass in the bound community of its members (Section 3.5). */
/* Returns the number of passes.                                        */
/* ------------------------------------------------------------------ */
static int louvain_impl(const og_graph *g, const og_opts *o, uint32_t *C, og_stats *st, og_trace *tr)
{
    uint32_t n = g->n;
    for (uint32_t v = 0; v < n; v++) C[v] = v;
    if (st) memset(st, 0, sizeof(*st));
    /* the current graph G' (owned copies after the first aggregation) */
    og_graph cur = *g;
    uint64_t *own_off = NULL; uint32_t *own_tgt = NULL; double *own_w = NULL;
    double *K = malloc(sizeof(double) * (n ? n : 1));
    double *Sigma = malloc(sizeof(double) * (n ? n : 1));
    uint32_t *Cp = malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *Cs = malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *Rf = malloc(sizeof(uint32_t) * (n ? n : 1));
    double tau = o->tolerance;
    int passes = 0;
    int split_each_pass = (o->split != 0 && !o->split_last);
    /* C' of the first pass is the identity; after an aggregation it is the */
    /* identity too, or with refinement the bound community of each super- */
    /* vertex; Sigma' sums K' over the communities of C'                    */
    for (uint32_t i = 0; i < n; i++) Cp[i] = i;
    for (int lp = 0; lp < o->max_passes; lp++) {
        uint32_t nv = cur.n;
        double m = og_vertex_weights(&cur, K);
        memset(Sigma, 0, sizeof(double) * nv);
        for (uint32_t i = 0; i < nv; i++) Sigma[Cp[i]] += K[i];
        if (tr) {
            tr->pass = lp;
            tr->max_K = 0.0;
            for (uint32_t i = 0; i < nv; i++) {
                if (K[i] > tr->max_K) tr->max_K = K[i];
                tr->kept[i] = 0.0; tr->gain[i] = 1.0; tr->moved[i] = 1;
            }
        }
        int li = (m > 0.0) ? move_impl(&cur, Cp, K, Sigma, m, tau, o->max_iterations, o->sync, o->waves,
                                       o->wave_hash, o->wave_repeats, o->no_return_from, o->singleton_rule, NULL,
                                       tr)
                           : 0;
        if (split_each_pass) {
            run_split(&cur, Cp, Cs, o->split);
            memcpy(Cp, Cs, sizeof(uint32_t) * nv);
        }
        passes = lp + 1;
        /* |Gamma| = communities in C' after the split; |Gamma_old| = |V'| */
        uint32_t *tmp = malloc(sizeof(uint32_t) * (nv ? nv : 1));
        memcpy(tmp, Cp, sizeof(uint32_t) * nv);
        uint32_t k = og_renumber(nv, tmp);
        free(tmp);
        if (st && lp < 64) { st->iterations[lp] = li; st->vertices[lp] = nv; st->communities[lp] = k; }
        if (li <= 1) break;
        /* the partition aggregated: C' itself, or with refinement the     */
        /* refined partition of C' (its super-vertices start the next pass */
        /* in their bound communities)                                     */
        uint32_t *A = Cp;
        if (o->refine) {
            og_refine(&cur, Cp, Rf, o->refine_theta, o->seed, (uint32_t)lp, o->waves, o->wave_hash);
            k = og_renumber(nv, Rf);
            A = Rf;
        }
        if ((double)k / (double)nv > o->aggregation_tolerance) break;
        k = og_renumber(nv, A);
        if (o->refine) og_renumber(nv, Cp);
        og_lookup(n, C, A);
        uint64_t *noff = malloc(sizeof(uint64_t) * ((size_t)k + 1));
        uint32_t *ntgt = malloc(sizeof(uint32_t) * (cur.nnz ? cur.nnz : 1));
        double *nw = malloc(sizeof(double) * (cur.nnz ? cur.nnz : 1));
        uint64_t nnz2 = og_aggregate(&cur, A, k, noff, ntgt, nw);
        free(own_off); free(own_tgt); free(own_w);
        own_off = noff; own_tgt = ntgt; own_w = nw;
        cur.n = k; cur.nnz = nnz2; cur.off = noff; cur.tgt = ntgt; cur.w = nw;
        tau = tau / o->tolerance_drop;
        if (o->refine) {
            /* super-vertex r starts in the bound community of its members */
            for (uint32_t i = 0; i < nv; i++) Cs[Rf[i]] = Cp[i];
            memcpy(Cp, Cs, sizeof(uint32_t) * k);
        } else {
            /* the pass that aggregated leaves C' as identity on the new graph */
            for (uint32_t i = 0; i < k; i++) Cp[i] = i;
        }
    }
    og_lookup(n, C, Cp);
    if (o->split != 0 && o->split_last) {
        run_split(g, C, Cs, o->split);
        memcpy(C, Cs, sizeof(uint32_t) * n);
    }
    uint32_t k = canonical_numbering(n, C);
    if (st) {
        st->passes = passes;
        st->final_communities = k;
        st->modularity = og_modularity(g, C);
    }
    free(own_off); free(own_tgt); free(own_w); free(K); free(Sigma); free(Cp); free(Cs); free(Rf);
    return passes;
}

int og_louvain(const og_graph *g, const og_opts *o, uint32_t *C, og_stats *st)
{
    return louvain_impl(g, o, C, st, NULL);
}

/* og_louvain that also records every local-moving visit (og_trace) into
 * rec[cap][OG_TRACE_FIELDS]; *len receives the number of visits (possibly
 * more than cap). */
int og_louvain_trace(const og_graph *g, const og_opts *o, uint32_t *C, og_stats *st, double *rec, uint64_t cap,
                     uint64_t *len)
{
    uint32_t n = g->n ? g->n : 1;
    og_trace tr;
    tr.rec = rec; tr.cap = cap; tr.len = 0; tr.pass = 0; tr.max_K = 0.0;
    tr.kept = malloc(sizeof(double) * n);
    tr.gain = malloc(sizeof(double) * n);
    tr.moved = malloc(n);
    int passes = louvain_impl(g, o, C, st, &tr);
    free(tr.kept); free(tr.gain); free(tr.moved);
    if (len) *len = tr.len;
    return passes;
}
