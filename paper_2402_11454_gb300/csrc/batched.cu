// batched.cu -- batched GSP-Louvain over many independent graphs.
#include "internal.cuh"

using namespace gsp;

extern "C" gsp_status gsp_louvain_batched(uint32_t num_graphs, const uint64_t *graph_vertex_offsets,
                                          const uint64_t *offsets, const uint32_t *targets, const float *weights,
                                          uint32_t n, uint64_t nnz, const gsp_opts *opts, uint32_t *membership,
                                          double *modularity, gsp_stats *stats) {
    (void)num_graphs; (void)graph_vertex_offsets; (void)offsets; (void)targets; (void)weights; (void)n;
    (void)nnz; (void)opts; (void)membership; (void)modularity; (void)stats;
    set_error("gsp_louvain_batched: not available in this build");
    return GSP_ERR_INVALID;
}
