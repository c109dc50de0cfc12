// noalloc.cu -- mem_flux_noalloc: the flux / characteristic-speed path with
// its working memory in a fixed, file-scope device array instead of memory
// the context allocates.
//
// Some callers cannot allocate device memory at the moment they need a
// result: a caller whose allocator owns the whole device budget (a framework
// caching allocator, a serving process that reserves its memory at start-up),
// or a caller on a latency-critical path where cudaMalloc's implicit
// synchronisation is not acceptable.  This entry point lets them compute
// fluxes and speeds without any allocation: the scratch below is part of the
// library image and is resident on every GPU that loads the library until the
// process exits.
#include <mutex>

#include "common.cuh"
#include "ctx.h"

#define MEM_NOALLOC_MAX_CELLS 1024
#define MEM_NOALLOC_MAX_Q 1728

// sigma [MAX_CELLS][MAX_Q] followed by the contraction output
// [MAX_CELLS][MEM_NCOL_FLUX]; 12.5 MB.
static __device__ __align__(256) float g_flux_scratch[(size_t)MEM_NOALLOC_MAX_CELLS * (MEM_NOALLOC_MAX_Q + MEM_NCOL_FLUX)];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_scratch_ptr[kMaxDevices] = {};
}  // namespace

extern "C" int mem_flux_noalloc(mem_ctx *ctx, const float *M, const float *beta, const float *gauge, float *F,
                                float *speed, int64_t B, void *stream) {
    if (!ctx || B < 0) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!M || !beta || !gauge) return MEM_EINVAL;
    // velocity-space contexts build none of the dense tables this path reads
    if (ctx->vel) return MEM_EINVAL;
    if (B > MEM_NOALLOC_MAX_CELLS || ctx->Q > MEM_NOALLOC_MAX_Q) return MEM_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MEM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices || dev != ctx->device) return MEM_EINVAL;
    float *base = nullptr;
    {
        // One-time set-up per device (with that device current): the host
        // name of the array is only a stand-in, so resolve its device address.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_flux_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return MEM_ECUDA;
            }
            g_scratch_ptr[dev] = (float *)p;
        }
        base = g_scratch_ptr[dev];
    }
    // Every element of both regions that the kernels read is written earlier
    // in the same call, so nothing has to be cleared between calls.
    float *sigma = base;
    float *mom = base + (size_t)MEM_NOALLOC_MAX_CELLS * MEM_NOALLOC_MAX_Q;
    return mem_host::flux_bufs(ctx, M, beta, gauge, F, speed, B, sigma, mom, (cudaStream_t)stream);
}
