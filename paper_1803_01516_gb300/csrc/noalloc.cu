// gs_maxflow_solve_noalloc: the max-flow solve with its scratch memory in a
// fixed, library-owned device array instead of a caller workspace.
//
// Some callers cannot allocate device memory when they solve: a real-time
// stereo loop that reserves all its memory at start-up and must not touch the
// CUDA allocator afterwards, or a plug-in inside a host application that owns
// the device allocator and gives the plug-in no way to request scratch space.
// They still pass the graph state and the status word; the scratch the solver
// needs lives in g_scratch below.
#include <mutex>

#include "gs_internal.cuh"

namespace gs {

// Scratch for one solve: the control block, per-node words and per-tile
// flags of the tiled solver.  Every GPU that loads this library holds these
// bytes until the process exits.
constexpr size_t kNoallocScratchBytes = 16u << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
static void *g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of g_scratch on the current device, looked up once per
// device.  (In host code the name g_scratch is only a host-side stand-in.)
static int scratch_address(void **out) {
    int dev = 0;
    GS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_INVAL;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_noalloc_scratch_bytes(void) { return kNoallocScratchBytes; }

extern "C" int gs_maxflow_solve_noalloc(void *graph, const gs_params *p, const gs_solve_opts *o,
                                        int32_t *status, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !o || !graph || !status) return GS_ERR_INVAL;
    if (o->engine != GS_ENGINE_TILED) return GS_ERR_INVAL;
    if (work_bytes(g) > kNoallocScratchBytes) return GS_ERR_TOO_LARGE;
    void *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != GS_OK) return rc;
    // The solve clears the control block it needs on the stream before use;
    // the other scratch words are written before they are read.
    return gs_maxflow_solve(graph, p, o, scratch, status, stream);
}
