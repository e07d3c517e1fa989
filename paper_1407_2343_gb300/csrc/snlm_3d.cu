// Data movement of the separable 3-D extension (the volume form that the paper's
// conclusion names as a direct extension of separable NLM): the 1-D passes along x
// and z read a (z, y, x) volume with a single line stride; the pass along y needs
// the (y, z, x) order, in which its lines again have one stride. These kernels swap
// the two outer dimensions (converting the samples to float32 on the way) and
// accumulate the average of several orders.
#include <cuda_fp16.h>

#include "snlm_host.h"
#include "snlm_internal.h"

namespace snlm {

namespace {

constexpr int kSwapThreads = 256;

template <typename T>
__device__ __forceinline__ float to_f32(T v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

// out row (a, b) = in row (b, a): in is B x A rows of W samples, out A x B rows.
template <typename T>
__global__ void __launch_bounds__(kSwapThreads) swap_outer_kernel(const T *__restrict__ in, float *__restrict__ out,
                                                                  int A, int B, int W)
{
    const long long rows = (long long)A * B;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int a = (int)(r / B), b = (int)(r - (long long)a * B);
        const T *src = in + ((long long)b * A + a) * W;
        float *dst = out + r * W;
        for (int x = threadIdx.x; x < W; x += kSwapThreads)
            dst[x] = to_f32(__ldg(src + x));
    }
}

// out = alpha * x + beta * out (beta = 0 overwrites)
__global__ void __launch_bounds__(kSwapThreads) axpby_kernel(const float *__restrict__ x, float *__restrict__ out,
                                                             float alpha, float beta, long long n)
{
    for (long long i = blockIdx.x * (long long)kSwapThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kSwapThreads)
        out[i] = beta == 0.f ? alpha * x[i] : fmaf(alpha, x[i], beta * out[i]);
}

int grid_for(long long items, int per_block)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (items + per_block - 1) / per_block;
    return (int)std::max(1LL, std::min(want, (long long)sms * 16));
}

}  // namespace

int preload_3d()
{
    return preload_kernel((const void *)swap_outer_kernel<unsigned char>) +
           preload_kernel((const void *)swap_outer_kernel<__half>) +
           preload_kernel((const void *)swap_outer_kernel<float>) + preload_kernel((const void *)axpby_kernel);
}

cudaError_t launch_swap_outer(const void *in, int dtype, float *out, int A, int B, int W, cudaStream_t st)
{
    const int grid = grid_for((long long)A * B, 1);
    if (dtype == DT_U8)
        swap_outer_kernel<unsigned char><<<grid, kSwapThreads, 0, st>>>(static_cast<const unsigned char *>(in), out,
                                                                         A, B, W);
    else if (dtype == DT_F16)
        swap_outer_kernel<__half><<<grid, kSwapThreads, 0, st>>>(static_cast<const __half *>(in), out, A, B, W);
    else
        swap_outer_kernel<float><<<grid, kSwapThreads, 0, st>>>(static_cast<const float *>(in), out, A, B, W);
    return cudaGetLastError();
}

cudaError_t launch_axpby(const float *x, float *out, float alpha, float beta, long long n, cudaStream_t st)
{
    axpby_kernel<<<grid_for(n, kSwapThreads), kSwapThreads, 0, st>>>(x, out, alpha, beta, n);
    return cudaGetLastError();
}

}  // namespace snlm
