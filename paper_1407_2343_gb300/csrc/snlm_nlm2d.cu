// The 2-D non-local means of Eqs. (1)-(2) (Sec. I): the workload that the run-time
// tables of Sec. IV-B compare separable NLM against. At pixel i,
//   NLM[f](i) = sum_j w_ij f(j) / sum_j w_ij over the (2S+1)^2 window centred at i,
//   w_ij = exp(-(1/h^2) sum_{k in [-K,K]^2} G(k) (f(i+k) - f(j+k))^2),
// G(k1, k2) = g(k1) g(k2) (box: 1; Gaussian: exp(-|k|^2 / (2 alpha^2))), with the
// samples read through the half-sample symmetric extension along each axis (the
// boundary reading of the 1-D passes).
//
// Evaluated exactly, offset by offset. A CTA owns a 32 x 16 tile of outputs and
// stages its input with an (S+K)-wide halo in shared memory once; then, for every
// offset s of the window: (1) the squared differences E = (f(x) - f(x+s))^2 over
// the tile plus a K-wide halo, (2) E filtered along the rows with g, (3) along the
// columns with g, giving the patch distance of every output pixel for this offset,
// (4) the weight 2^(c2 d) (c2 = -log2(e) / h^2) accumulated in centred form,
// f(i) + sum w (f(j) - f(i)) / sum w (the offset 0 has weight 1), each window row
// summed apart before it joins the totals (FP32 sums of 2S+1 terms at both levels,
// not one chain of (2S+1)^2). The separable patch sum makes the cost O(S^2 K) a
// pixel instead of the O(S^2 K^2) of the plain double sum, for both profiles.
#include "snlm_host.h"
#include "snlm_internal.h"

#include <utility>

#include <cuda_fp16.h>

namespace snlm {

namespace {

constexpr int kN2Tx = 32;                 // output columns per CTA
constexpr int kN2Ty = 16;                 // output rows per CTA
constexpr int kN2Threads = 256;
constexpr int kN2Cg = 4;                  // row-filter outputs per thread

struct Nlm2dArgs {
    const void *img;
    int dtype;
    int H, W;
    long long pitch;
    float *out;
    int S;
    float c2;                             // -log2(e) / h^2
    float g[2 * kMaxK + 1];               // the 1-D profile; G = g x g
};

__device__ __forceinline__ int n2_reflect(int x, int n)
{
    if (x >= 0 && x < n)
        return x;
    const int p = 2 * n;
    int y = x % p;
    if (y < 0)
        y += p;
    return y < n ? y : p - 1 - y;
}

__device__ __forceinline__ float n2_load(const Nlm2dArgs &p, int y, int x)
{
    const long long o = (long long)y * p.pitch + x;
    if (p.dtype == DT_U8)
        return (float)__ldg(static_cast<const unsigned char *>(p.img) + o);
    if (p.dtype == DT_F16)
        return __half2float(__ldg(static_cast<const __half *>(p.img) + o));
    return __ldg(static_cast<const float *>(p.img) + o);
}

__device__ __forceinline__ float n2_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Shared-memory layout (floats): F (input tile with halo S+K), E, Hs.
struct N2Layout {
    int R, FW, FH, EW, EH, f, e, hs, total;
    __host__ __device__ N2Layout(int S, int K)
    {
        R = S + K;
        FW = kN2Tx + 2 * R;
        FH = kN2Ty + 2 * R;
        EW = kN2Tx + 2 * K;
        EH = kN2Ty + 2 * K;
        f = 0;
        e = FW * FH;
        hs = e + EW * EH;
        total = hs + kN2Tx * EH;
    }
};

template <int K>
__global__ void __launch_bounds__(kN2Threads) nlm2d_kernel(const __grid_constant__ Nlm2dArgs p)
{
    constexpr int D = 2 * K + 1;
    extern __shared__ __align__(16) float sm[];
    const int S = p.S;
    const N2Layout L(S, K);
    float *F = sm + L.f, *E = sm + L.e, *Hs = sm + L.hs;
    const int x0 = blockIdx.x * kN2Tx, y0 = blockIdx.y * kN2Ty;
    const int tid = threadIdx.x;

    for (int i = tid; i < L.FW * L.FH; i += kN2Threads) {
        const int r = i / L.FW, c = i - r * L.FW;
        F[i] = n2_load(p, n2_reflect(y0 - L.R + r, p.H), n2_reflect(x0 - L.R + c, p.W));
    }
    __syncthreads();

    // outputs of this thread: column oc, rows 2 orp and 2 orp + 1 of the tile
    const int oc = tid & 31, orp = tid >> 5;
    const int fr0 = 2 * orp + L.R, fc0 = oc + L.R;          // centre in F
    const float c0 = F[fr0 * L.FW + fc0], c1 = F[(fr0 + 1) * L.FW + fc0];
    float num0 = 0.f, num1 = 0.f, den0 = 0.f, den1 = 0.f;
    // row-filter work item of this thread: row hr of E, columns hc .. hc + 3
    const int hr = tid / (kN2Tx / kN2Cg), hc = kN2Cg * (tid - hr * (kN2Tx / kN2Cg));
    const bool h_on = hr < L.EH;

#pragma unroll 1
    for (int sy = -S; sy <= S; ++sy) {
        // the offsets of one window row are summed apart and then added to the
        // totals: two levels of 2S+1 terms instead of one chain of (2S+1)^2
        float rn0 = 0.f, rn1 = 0.f, rd0 = 0.f, rd1 = 0.f;
#pragma unroll 1
        for (int sx = -S; sx <= S; ++sx) {
            // (1) squared differences over the tile + K halo
            for (int i = tid; i < L.EW * L.EH; i += kN2Threads) {
                const int r = i / L.EW, c = i - r * L.EW;
                const int a = (r + S) * L.FW + c + S;
                const float d = F[a] - F[a + sy * L.FW + sx];
                E[i] = d * d;
            }
            __syncthreads();
            // (2) along the rows
            if (h_on) {
                float e[kN2Cg + 2 * K];
#pragma unroll
                for (int j = 0; j < kN2Cg + 2 * K; ++j)
                    e[j] = E[hr * L.EW + hc + j];
#pragma unroll
                for (int q = 0; q < kN2Cg; ++q) {
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        acc = fmaf(p.g[k], e[q + k], acc);
                    Hs[hr * kN2Tx + hc + q] = acc;
                }
            }
            __syncthreads();
            // (3) along the columns, (4) weights and centred accumulation
            float h[D + 1];
#pragma unroll
            for (int k = 0; k <= D; ++k)
                h[k] = Hs[(2 * orp + k) * kN2Tx + oc];
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                d0 = fmaf(p.g[k], h[k], d0);
                d1 = fmaf(p.g[k], h[k + 1], d1);
            }
            const float w0 = n2_ex2(p.c2 * d0), w1 = n2_ex2(p.c2 * d1);
            const int js = (fr0 + sy) * L.FW + fc0 + sx;
            rn0 = fmaf(w0, F[js] - c0, rn0);
            rn1 = fmaf(w1, F[js + L.FW] - c1, rn1);
            rd0 += w0;
            rd1 += w1;
        }
        num0 += rn0;
        num1 += rn1;
        den0 += rd0;
        den1 += rd1;
    }
    const int x = x0 + oc, y = y0 + 2 * orp;
    if (x < p.W) {
        if (y < p.H)
            p.out[(long long)y * p.W + x] = c0 + num0 / den0;
        if (y + 1 < p.H)
            p.out[(long long)(y + 1) * p.W + x] = c1 + num1 / den1;
    }
}

template <int K>
cudaError_t launch_n2(const Nlm2dArgs &a, cudaStream_t st)
{
    const N2Layout L(a.S, K);
    const size_t smem = (size_t)L.total * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(nlm2d_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dim3 grid((unsigned)div_up(a.W, kN2Tx), (unsigned)div_up(a.H, kN2Ty));
    nlm2d_kernel<K><<<grid, kN2Threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int... K>
int preload_n2(std::integer_sequence<int, K...>)
{
    return (preload_kernel((const void *)nlm2d_kernel<K>) + ...);
}

}  // namespace

int preload_nlm2d()
{
    return preload_n2(std::make_integer_sequence<int, 8>{});
}

}  // namespace snlm

using namespace snlm;

extern "C" int snlm_nlm_2d(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h, int profile,
                           float alpha, float *out, void *stream)
{
    if (H < 1 || W < 1 || pitch < W || (long long)H * pitch >= (1LL << 31) || (long long)H * W >= (1LL << 31))
        return SNLM_ERR_ARG;
    if (profile == SNLM_GAUSS_IIR)
        return SNLM_ERR_UNSUPPORTED;
    if (S < 0 || K < 0 || !valid_dtype(dtype) || (profile != SNLM_BOX && profile != SNLM_GAUSS))
        return SNLM_ERR_ARG;
    if (!(h > 0.f) || !std::isfinite(h))
        return SNLM_ERR_ARG;
    if (S > kMaxS2d || K > kMaxK || div_up(H, kN2Ty) > 65535)
        return SNLM_ERR_UNSUPPORTED;                    // (the grid's y extent holds the row tiles)
    if (!is_device_ptr(img) || !is_device_ptr(out))
        return SNLM_ERR_ARG;
    Nlm2dArgs a;
    a.img = img;
    a.dtype = dtype;
    a.H = H;
    a.W = W;
    a.pitch = pitch;
    a.out = out;
    a.S = S;
    a.c2 = (float)(-1.4426950408889634 / ((double)h * h));
    const double beta = alpha > 0.f ? (double)alpha : (K > 0 ? K / 2.0 : 1.0);
    for (int k = 0; k < 2 * kMaxK + 1; ++k)
        a.g[k] = 0.f;
    for (int k = -K; k <= K; ++k)
        a.g[k + K] = profile == SNLM_BOX ? 1.f : (float)std::exp(-(double)(k * k) / (2.0 * beta * beta));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TraceScope ts(SNLM_K_NLM_2D, st);
    cudaError_t e;
    switch (K) {
    case 0: e = launch_n2<0>(a, st); break;
    case 1: e = launch_n2<1>(a, st); break;
    case 2: e = launch_n2<2>(a, st); break;
    case 3: e = launch_n2<3>(a, st); break;
    case 4: e = launch_n2<4>(a, st); break;
    case 5: e = launch_n2<5>(a, st); break;
    case 6: e = launch_n2<6>(a, st); break;
    default: e = launch_n2<7>(a, st); break;
    }
    return status_of(e);
}
