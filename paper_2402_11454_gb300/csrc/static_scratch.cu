// static_scratch.cu -- modularity (Equation 1) for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: embedders whose device memory is owned
// by a fixed pool (inference servers, other frameworks' allocators that hold
// the whole device), or processes that must not grow their device footprint
// after start-up.  gsp_modularity_static computes the same value as
// gsp_modularity but takes its scratch from one file-scope __device__ array
// instead of the library workspace, so it allocates nothing.  Like
// gsp_modularity it waits for the stream and returns Q in host memory.
//
// The array is part of the module image: every device that loads the library
// holds GSP_STATIC_SCRATCH_BYTES for it until the process exits.  Host code
// cannot use the array's name as a device address (it is a host-side
// stand-in), so the set-up looks the address up with cudaGetSymbolAddress
// while the device is current, once per device context: a context created
// anew (after cudaDeviceReset) gets a fresh lookup.
#include <cuda.h>  // CUcontext and the cuCtxGetCurrent signature (resolved at run time)

#include <mutex>

#include "internal.cuh"

namespace gsp {

constexpr uint32_t STATIC_MAX_N = GSP_STATIC_MAX_VERTICES;
// layout: Sigma[STATIC_MAX_N] (double) | acc[4] (double) | counter (u64) |
//         nlong (u32, padded) | longlist[STATIC_MAX_N] (u32)
constexpr size_t SO_SIGMA = 0;
constexpr size_t SO_ACC = SO_SIGMA + sizeof(double) * STATIC_MAX_N;
constexpr size_t SO_COUNTER = SO_ACC + 4 * sizeof(double);
constexpr size_t SO_NLONG = SO_COUNTER + sizeof(unsigned long long);
constexpr size_t SO_LONG = SO_NLONG + 256;
constexpr size_t SCRATCH_BYTES = SO_LONG + sizeof(uint32_t) * STATIC_MAX_N;
static_assert(SCRATCH_BYTES == GSP_STATIC_SCRATCH_BYTES, "scratch size in gsp.h");

static __device__ __align__(256) unsigned char g_static_scratch[SCRATCH_BYTES];

struct ScratchSlot {
    CUcontext ctx;
    char *addr;
};
static ScratchSlot g_scratch_addr[64];
static std::mutex g_scratch_mu;

// The current context, through the driver entry point the runtime hands out
// (the library links no driver library); nullptr when unavailable.
static CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(p);
        else
            cudaGetLastError();
    }
    CUcontext ctx = nullptr;
    if (!fn || fn(&ctx) != CUDA_SUCCESS) return nullptr;
    return ctx;
}

// Device address of the scratch array on the current device: looked up with
// that device current the first time a context of it calls, and again when
// the device's context has changed since (cudaDeviceReset makes a new one).
static char *scratch_address() {
    int dev = 0;
    GSP_CUDA(cudaGetDevice(&dev));
    GSP_REQUIRE(dev >= 0 && dev < 64, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    CUcontext ctx = current_context();
    ScratchSlot &slot = g_scratch_addr[dev];
    if (!slot.addr || !ctx || ctx != slot.ctx) {
        void *p = nullptr;
        GSP_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));  // initialises the context when needed
        slot.addr = static_cast<char *>(p);
        slot.ctx = current_context();
    }
    return slot.addr;
}

}  // namespace gsp

using namespace gsp;

extern "C" gsp_status gsp_modularity_static(const uint64_t *offsets, const uint32_t *targets, const void *weights,
                                            int wt, uint32_t n, uint64_t nnz, const uint32_t *C, double *q_host,
                                            void *stream) {
    try {
        GSP_REQUIRE(n > 0, "n must be > 0");
        GSP_REQUIRE(offsets && C && q_host, "offsets, C and q_host must not be NULL");
        GSP_REQUIRE(nnz == 0 || (targets && weights), "targets/weights must not be NULL");
        GSP_REQUIRE(wt == GSP_W_F32 || wt == GSP_W_F64, "unknown weight type %d", wt);
        if (n > STATIC_MAX_N) {
            set_error("gsp_modularity_static: n = %u exceeds the static scratch limit of %u vertices "
                      "(use gsp_modularity)", n, STATIC_MAX_N);
            return GSP_ERR_CAPACITY;
        }
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        char *base = scratch_address();
        unsigned long long *counter = reinterpret_cast<unsigned long long *>(base + SO_COUNTER);
        check_csr(offsets, targets, n, nnz, counter, s);
        unsigned long long bad = count_out_of_range(C, n, n, counter, s);
        GSP_REQUIRE(bad == 0, "membership: %llu ids out of range (must be < %u)", bad, n);
        DevGraph g;
        g.n = n;
        g.nnz = nnz;
        g.off = offsets;
        g.tgt = targets;
        g.w = weights;
        g.wt = wt;
        *q_host = modularity_scratch(g, C, reinterpret_cast<double *>(base + SO_SIGMA),
                                     reinterpret_cast<double *>(base + SO_ACC),
                                     reinterpret_cast<uint32_t *>(base + SO_LONG),
                                     reinterpret_cast<uint32_t *>(base + SO_NLONG), s);
        return GSP_OK;
    } catch (const gsp::Error &e) {
        return e.status;
    } catch (...) {
        set_error("unexpected exception");
        return GSP_ERR_CUDA;
    }
}
