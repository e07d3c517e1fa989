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
#include <cuda_runtime.h>

#include "../../include/snlm.h"

namespace {

// Fixed scratch of snlm_denoise_noalloc (32 MiB). Every device that loads the
// library holds it until the process exits. Host code sees only a stand-in for
// this symbol; its device address is looked up on every call (below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SNLM_NOALLOC_SCRATCH_BYTES];

}  // namespace

extern "C" int snlm_denoise_noalloc(const void *img, int dtype, int H, int W, int pitch, int S, int K,
                                    float h, int profile, int order, float sigma, float beta, float *out,
                                    void *stream)
{
    // Where the static array lives in the memory of the device (and context) that
    // is current now. A static __device__ array has one copy per context, so the
    // address is not cached: after cudaDeviceReset, or with another context made
    // current on the same device, a remembered address would point at freed or
    // foreign memory. The lookup is a host-side query; no device work is queued.
    void *scratch = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
    if (e != cudaSuccess || !scratch) {
        cudaGetLastError();
        return SNLM_ERR_CUDA;
    }
    // The regular entry point with caller-provided scratch does the rest; it
    // rejects an image whose scratch would not fit (SNLM_ERR_ARG) before any launch
    // and allocates nothing.
    return snlm_denoise_ws(img, dtype, H, W, pitch, S, K, h, profile, order, sigma, beta, out, scratch,
                           (size_t)SNLM_NOALLOC_SCRATCH_BYTES, nullptr, stream);
}
