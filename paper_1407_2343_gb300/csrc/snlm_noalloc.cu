// snlm_denoise_noalloc: the separable NLM of snlm_denoise for callers that must
// not allocate device memory at run time, using a fixed scratch area that is part
// of the library's device image instead of memory from cudaMalloc.
//
// Who needs this: programs that may not call cudaMalloc/cudaFree once they are
// running — real-time loops (an allocation can synchronise the whole device and
// take an unbounded time), plug-ins whose host application owns all device memory
// through its own allocator, and programs that must keep a fixed device-memory
// footprint after start-up. They pass their own input and output buffers; the
// intermediate images live in the static array below.
//
// The array is shared by every call in the process on a given device and keeps
// whatever the last call left in it. Nothing in it has to start at zero: every
// pass writes its intermediate image in full before the next pass reads it, and
// every CTA writes its own partial-sum record. Two calls whose device work
// overlaps in time (different streams, or different host threads without
// ordering) race on the array and corrupt each other's results; serialise them.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/snlm.h"

namespace {

// Fixed scratch of snlm_denoise_noalloc (32 MiB). Every device that loads the
// library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SNLM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

}  // namespace

extern "C" int snlm_denoise_noalloc(const void *img, int dtype, int H, int W, int pitch, int S, int K,
                                    float h, int profile, int order, float sigma, float beta, float *out,
                                    void *stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SNLM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices)
        return SNLM_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    {
        // First call on this device: look up where the static array lives in the
        // device's memory (host code only knows a host-side stand-in symbol).
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return SNLM_ERR_CUDA;
            }
            g_addr[dev] = p;
        }
        scratch = g_addr[dev];
    }
    // The regular entry point with caller-provided scratch does the rest; it
    // rejects an image whose scratch would not fit (SNLM_ERR_ARG) before any launch
    // and allocates nothing.
    return snlm_denoise_ws(img, dtype, H, W, pitch, S, K, h, profile, order, sigma, beta, out, scratch,
                           (size_t)SNLM_NOALLOC_SCRATCH_BYTES, nullptr, stream);
}
