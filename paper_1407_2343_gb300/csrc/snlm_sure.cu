// SURE-optimal combination of the two separable orders (Sec. III-A, Alg. 4):
// reduce the per-CTA partial sums of the last pass of each order, solve the 2x2
// system A theta = b of Eqs. (19) and (25), and form theta1 f_rc + theta2 f_cr
// (Eq. (14)).
#include <cuda_fp16.h>

#include "snlm_internal.h"
#include "snlm_sure_impl.cuh"

namespace snlm {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kSolveBlocks = kSolveScratchRecords;   // first-level slices of the records

// First level: block b sums records [b*per, min(n, (b+1)*per)) in a fixed order.
__global__ void __launch_bounds__(kSolveThreads) sure_partial_kernel(const double *part, int n, int per,
                                                                     double *out)
{
    __shared__ double sh[kPartials * kSolveThreads];
    const int lo = blockIdx.x * per, hi = min(n, lo + per);
    double r[kPartials];
    reduce_records(part + (long long)lo * kPartials, max(0, hi - lo), sh, r);
    if (threadIdx.x < kPartials)
        out[(long long)blockIdx.x * kPartials + threadIdx.x] = r[threadIdx.x];
}

// The SURE objective of Eq. (17) is minimised over f~ = theta1 f_rc + theta2 f_cr
// (Eq. (14)). It is solved here in the basis m = (f_rc + f_cr)/2, d = (f_rc - f_cr)/2,
// f~ = alpha m + beta d, theta1 = (alpha + beta)/2, theta2 = (alpha - beta)/2: the
// same minimiser (a linear change of variables; det/trace^2 is unchanged), but the
// sums that fix the nearly singular direction (beta) are made of the small
// differences d, so float32 per-pixel products keep them accurate.
//
// Both levels and the solve run in one launch: block b reduces slice b of each record
// set into scratch (fixed order, as sure_partial_kernel), then takes a ticket; the
// block that takes the last one (every slice is in scratch by then: each block
// fences its writes before its ticket) reduces the slices in a fixed order and
// solves. No block waits for another. The ticket word must be zero at launch.
__global__ void __launch_bounds__(kSolveThreads) sure_reduce_solve_kernel(const double *part_rc, int n_rc,
                                                                          int per_rc, const double *part_cr,
                                                                          int n_cr, int per_cr, double *scratch,
                                                                          unsigned *ticket, double sigma2,
                                                                          double *info)
{
    __shared__ double sh[kPartials * kSolveThreads];
    __shared__ bool last;
    double r[kPartials];
    {
        const int lo = blockIdx.x * per_rc, hi = min(n_rc, lo + per_rc);
        reduce_records(part_rc + (long long)lo * kPartials, max(0, hi - lo), sh, r);
        if (threadIdx.x < kPartials)
            scratch[(long long)blockIdx.x * kPartials + threadIdx.x] = r[threadIdx.x];
    }
    {
        const int lo = blockIdx.x * per_cr, hi = min(n_cr, lo + per_cr);
        reduce_records(part_cr + (long long)lo * kPartials, max(0, hi - lo), sh, r);
        if (threadIdx.x < kPartials)
            scratch[(long long)(gridDim.x + blockIdx.x) * kPartials + threadIdx.x] = r[threadIdx.x];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    double rc[kPartials], cr[kPartials];
    reduce_records(scratch, gridDim.x, sh, rc);
    reduce_records(scratch + (long long)gridDim.x * kPartials, gridDim.x, sh, cr);
    if (threadIdx.x == 0)
        sure_finish(rc, cr, sigma2, info);
}

// out = theta1 * frc + theta2 * out, with theta split into float hi + lo parts so
// the weights keep ~48 bits.
__global__ void combine_kernel(const float4 *__restrict__ frc, float4 *__restrict__ out,
                               const double *__restrict__ info, long long n4)
{
    const double t0 = info[0], t1 = info[1];
    const float h0 = (float)t0, h1 = (float)t1;
    const float l0 = (float)(t0 - (double)h0), l1 = (float)(t1 - (double)h1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 a = frc[i];
        float4 b = out[i];
        b.x = fmaf(h0, a.x, fmaf(h1, b.x, fmaf(l0, a.x, l1 * b.x)));
        b.y = fmaf(h0, a.y, fmaf(h1, b.y, fmaf(l0, a.y, l1 * b.y)));
        b.z = fmaf(h0, a.z, fmaf(h1, b.z, fmaf(l0, a.z, l1 * b.z)));
        b.w = fmaf(h0, a.w, fmaf(h1, b.w, fmaf(l0, a.w, l1 * b.w)));
        out[i] = b;
    }
}

__global__ void combine_scalar_kernel(const float *__restrict__ frc, float *__restrict__ out,
                                      const double *__restrict__ info, long long start, long long n)
{
    const double t0 = info[0], t1 = info[1];
    const float h0 = (float)t0, h1 = (float)t1;
    const float l0 = (float)(t0 - (double)h0), l1 = (float)(t1 - (double)h1);
    for (long long i = start + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = fmaf(h0, frc[i], fmaf(h1, out[i], fmaf(l0, frc[i], l1 * out[i])));
}

// The seven sums of a band, in the basis m, d (no solve).
__global__ void __launch_bounds__(kSolveThreads) sure_sums_kernel(const double *part_rc, int n_rc,
                                                                  const double *part_cr, int n_cr, double *sums)
{
    __shared__ double sh[kPartials * kSolveThreads];
    double rc[kPartials], cr[kPartials];
    reduce_records(part_rc, n_rc, sh, rc);
    reduce_records(part_cr, n_cr, sh, cr);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 5; ++k)
            sums[k] = cr[k];
        sums[5] = rc[5];
        sums[6] = cr[5];
    }
}

// out = theta1 frc + theta2 fcr (theta split into float hi + lo parts).
__global__ void combine_theta_kernel(const float *__restrict__ frc, const float *fcr, float *out, long long n,
                                     double t0, double t1)
{
    const float h0 = (float)t0, h1 = (float)t1;
    const float l0 = (float)(t0 - (double)h0), l1 = (float)(t1 - (double)h1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float a = frc[i], b = fcr[i];
        out[i] = fmaf(h0, a, fmaf(h1, b, fmaf(l0, a, l1 * b)));
    }
}

// Partial records of the SURE sums over whole images, for the passes that form no
// records of their own (the recursive profile's): block b takes rows r0 + b,
// r0 + b + gridDim.x, ... of [r0, r1), thread t the columns t, t + 256, ... of each,
// and forms in float32
//   m = (frc + fcr)/2, d = (frc - fcr)/2:  m^2, m d, d^2, f m, f d, delta
// (frc == NULL: delta only). A thread sums its at most ceil(W/256) terms of a row in
// float32 (as the pass kernels sum a lane's run) and adds the row's partial in FP64
// (FP64 arithmetic is slow on this GPU, so it is kept to one add per row and sum);
// the block is reduced in a fixed tree into record b (kPartials doubles, the unused
// ones zero).
__global__ void __launch_bounds__(kSolveThreads) image_sums_kernel(const float *__restrict__ frc,
                                                                   const float *__restrict__ fcr, Lines f, int W,
                                                                   int r0, int r1, const float *__restrict__ delta,
                                                                   double *records)
{
    __shared__ double sh[kPartials * kSolveThreads];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int r = r0 + (int)blockIdx.x; r < r1; r += (int)gridDim.x) {
        const long long row = (long long)r * W, fo = (long long)r * f.line_step;
        float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = (int)threadIdx.x; c < W; c += (int)blockDim.x) {
            s[5] += delta[row + c];
            if (frc) {
                const float a = frc[row + c], b = fcr[row + c];
                const float m = 0.5f * (a + b), d = 0.5f * (a - b);
                const float fv = f.dtype == DT_U8 ? (float)static_cast<const unsigned char *>(f.ptr)[fo + c]
                                 : f.dtype == DT_F16 ? __half2float(static_cast<const __half *>(f.ptr)[fo + c])
                                                     : static_cast<const float *>(f.ptr)[fo + c];
                s[0] = fmaf(m, m, s[0]);
                s[1] = fmaf(m, d, s[1]);
                s[2] = fmaf(d, d, s[2]);
                s[3] = fmaf(fv, m, s[3]);
                s[4] = fmaf(fv, d, s[4]);
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            acc[k] += (double)s[k];
    }
    for (int k = 0; k < kPartials; ++k)
        sh[k * kSolveThreads + threadIdx.x] = k < 6 ? acc[k] : 0.0;
    __syncthreads();
    for (int stride = kSolveThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride)
            for (int k = 0; k < kPartials; ++k)
                sh[k * kSolveThreads + threadIdx.x] += sh[k * kSolveThreads + threadIdx.x + stride];
        __syncthreads();
    }
    if (threadIdx.x < kPartials)
        records[(long long)blockIdx.x * kPartials + threadIdx.x] = sh[threadIdx.x * kSolveThreads];
}

__global__ void set_theta_kernel(double *info, double t0, double t1)
{
    if (threadIdx.x < 10)
        info[threadIdx.x] = threadIdx.x == 0 ? t0 : (threadIdx.x == 1 ? t1 : 0.0);
}

}  // namespace

int preload_sure()
{
    const void *f[] = {(const void *)sure_partial_kernel, (const void *)sure_reduce_solve_kernel,
                       (const void *)combine_kernel,      (const void *)combine_scalar_kernel,
                       (const void *)sure_sums_kernel,    (const void *)combine_theta_kernel,
                       (const void *)image_sums_kernel,   (const void *)set_theta_kernel};
    int n = 0;
    for (const void *k : f)
        n += preload_kernel(k);
    return n;
}

cudaError_t launch_sure_solve(const double *part_rc, int n_rc, const double *part_cr, int n_cr,
                              double sigma2, double *info, double *scratch, unsigned *ticket, cudaStream_t st)
{
    // two fixed-order levels, kSolveBlocks slices per record set and then one block,
    // in a single launch (the last block to finish does the second level)
    const int per_rc = (n_rc + kSolveBlocks - 1) / kSolveBlocks;
    const int per_cr = (n_cr + kSolveBlocks - 1) / kSolveBlocks;
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess)
        return e;
    sure_reduce_solve_kernel<<<kSolveBlocks, kSolveThreads, 0, st>>>(part_rc, n_rc, per_rc, part_cr, n_cr, per_cr,
                                                                     scratch, ticket, sigma2, info);
    return cudaGetLastError();
}

cudaError_t launch_combine(const float *frc, float *out_fcr, const double *info, long long n,
                           cudaStream_t st)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool aligned = ((reinterpret_cast<uintptr_t>(frc) | reinterpret_cast<uintptr_t>(out_fcr)) & 15) == 0;
    const long long n4 = aligned ? n / 4 : 0;
    if (n4 > 0) {
        long long blocks = (n4 + 255) / 256;
        if (blocks > (long long)sms * 8)
            blocks = (long long)sms * 8;
        combine_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const float4 *>(frc),
                                                         reinterpret_cast<float4 *>(out_fcr), info, n4);
    }
    const long long rest = n - n4 * 4;
    if (rest > 0) {
        long long blocks = (rest + 255) / 256;
        if (blocks > (long long)sms * 8)
            blocks = (long long)sms * 8;
        combine_scalar_kernel<<<(unsigned)blocks, 256, 0, st>>>(frc, out_fcr, info, n4 * 4, n);
    }
    return cudaGetLastError();
}

cudaError_t launch_sure_sums(const double *part_rc, int n_rc, const double *part_cr, int n_cr, double *sums,
                             double *scratch, cudaStream_t st)
{
    const int per_rc = (n_rc + kSolveBlocks - 1) / kSolveBlocks;
    const int per_cr = (n_cr + kSolveBlocks - 1) / kSolveBlocks;
    sure_partial_kernel<<<kSolveBlocks, kSolveThreads, 0, st>>>(part_rc, n_rc, per_rc, scratch);
    sure_partial_kernel<<<kSolveBlocks, kSolveThreads, 0, st>>>(part_cr, n_cr, per_cr,
                                                                scratch + kSolveBlocks * kPartials);
    sure_sums_kernel<<<1, kSolveThreads, 0, st>>>(scratch, kSolveBlocks, scratch + kSolveBlocks * kPartials,
                                                  kSolveBlocks, sums);
    return cudaGetLastError();
}

cudaError_t launch_combine_theta(const float *frc, const float *fcr, float *out, long long n, double theta1,
                                 double theta2, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)sms * 8)
        blocks = (long long)sms * 8;
    combine_theta_kernel<<<(unsigned)blocks, 256, 0, st>>>(frc, fcr, out, n, theta1, theta2);
    return cudaGetLastError();
}

cudaError_t launch_image_sums(const float *frc, const float *fcr, const Lines &f, int W, int r0, int r1,
                              const float *delta, double *records, int n_records, cudaStream_t st)
{
    image_sums_kernel<<<n_records, kSolveThreads, 0, st>>>(frc, fcr, f, W, r0, r1, delta, records);
    return cudaGetLastError();
}

cudaError_t launch_set_theta(double *info, double t1, double t2, cudaStream_t st)
{
    set_theta_kernel<<<1, 32, 0, st>>>(info, t1, t2);
    return cudaGetLastError();
}

}  // namespace snlm
