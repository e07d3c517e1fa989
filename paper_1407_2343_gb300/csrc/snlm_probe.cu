// snlm_probe_peaks: measured issue rates of the arithmetic the passes are bound by
// (no counterpart in the paper; a measurement aid for the roofline of the 1-D
// passes): FP32 lane-operations per second through packed FP32x2 FMAs and through
// scalar FMAs, and MUFU.EX2 results per second. Each kernel runs independent
// dependency chains in every thread of a grid that fills every SM, so the pipe,
// not latency, sets its rate; the device time comes from CUDA events on the
// caller's stream.
#include <cuda_runtime.h>

#include "../../include/snlm.h"

namespace {

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 pack2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int kChains = 8;

// Where a kernel would write its chains' sum (one float per thread of a CTA of 256);
// the condition that guards the write never holds, but the compiler cannot know,
// so the chains are not removed as dead code.
static __device__ float g_probe_sink[256];

// kChains packed chains x <- x * m + a (two lanes each); the fixed point of the
// map is a / (1 - m), so the values stay bounded and normal.
__global__ void __launch_bounds__(256) probe_fma2_kernel(float *sink, int iters, float m, float a)
{
    f32x2 x[kChains];
    const f32x2 mm = pack2(m, m), aa = pack2(a, a);
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = pack2(threadIdx.x * 1e-3f + c, c * 0.5f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            x[c] = fma2(x[c], mm, aa);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 12345.678f)
        sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) probe_fma_kernel(float *sink, int iters, float m, float a)
{
    float x[2 * kChains];
#pragma unroll
    for (int c = 0; c < 2 * kChains; ++c)
        x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 2 * kChains; ++c)
            asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(m), "f"(a));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 2 * kChains; ++c)
        s += x[c];
    if (s == 12345.678f)
        sink[threadIdx.x] = s;
}

// kChains chains x <- 2^(-x): for x in (0, 1] the result stays in [1/2, 1).
__global__ void __launch_bounds__(256) probe_ex2_kernel(float *sink, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = 0.1f + 0.1f * c + threadIdx.x * 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            x[c] = ex2(-x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    if (s == 12345.678f)
        sink[threadIdx.x] = s;
}

template <typename F>
int timed(F launch, cudaStream_t st, float *ms)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess)
        return SNLM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SNLM_ERR_CUDA;
    }
    launch();                           // warm-up (clocks up, code loaded)
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r)
        launch();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    return e == cudaSuccess ? SNLM_OK : SNLM_ERR_CUDA;
}

}  // namespace

extern "C" int snlm_probe_peaks(double *rates, void *stream)
{
    if (!rates)
        return SNLM_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return SNLM_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *sink = nullptr;
    if (cudaGetSymbolAddress((void **)&sink, g_probe_sink) != cudaSuccess || !sink) {
        cudaGetLastError();
        return SNLM_ERR_CUDA;
    }
    const int blocks = sms * 8, threads = 256;
    const double nthreads = (double)blocks * threads;
    const int it_fma = 40000, it_ex2 = 20000;
    float ms = 0.f;
    int rc = timed([&] { probe_fma2_kernel<<<blocks, threads, 0, st>>>(sink, it_fma, 0.999f, 1e-3f); }, st, &ms);
    if (rc != SNLM_OK)
        return rc;
    rates[0] = 3.0 * nthreads * it_fma * kChains * 2 / (ms * 1e-3);
    rc = timed([&] { probe_fma_kernel<<<blocks, threads, 0, st>>>(sink, it_fma, 0.999f, 1e-3f); }, st, &ms);
    if (rc != SNLM_OK)
        return rc;
    rates[1] = 3.0 * nthreads * it_fma * kChains * 2 / (ms * 1e-3);
    rc = timed([&] { probe_ex2_kernel<<<blocks, threads, 0, st>>>(sink, it_ex2); }, st, &ms);
    if (rc != SNLM_OK)
        return rc;
    rates[2] = 3.0 * nthreads * it_ex2 * kChains / (ms * 1e-3);
    return SNLM_OK;
}
