// Bilateral post-filter of Sec. III-B, Eq. (BF): SNLM[f](i) is the average of the
// samples f~(i - j) over the integer offsets j of [-R, R]^2, R = floor(3 sigma_s),
// weighted by w(j) g(f~(i - j) - f~(i)) with w(j) = exp(-|j|^2 / (2 sigma_s^2)) and
// g(t) = exp(-t^2 / (2 sigma_r^2)); samples outside the image are read through the
// half-sample symmetric extension (the boundary reading of the NLM passes).
//
// On the GPU the direct sum is cheap (R = 2 for the parameter rules of Sec. IV-A
// at sigma <= 60, i.e. 24 taps a pixel), so the filter is computed exactly rather
// than through the trigonometric approximation of the range kernel that the paper
// uses on the CPU. Each tap costs one ex2: w(j) g(t) = 2^(lw(j) + cr t^2) with
// lw(j) = -log2(e) |j|^2 / (2 sigma_s^2) (kernel parameters, read from the constant
// bank) and cr = -log2(e) / (2 sigma_r^2). The result is formed in centred form,
// f~(i) + sum w g t / sum w g with t = f~(i - j) - f~(i); the centre tap is 1.
//
// A CTA filters a 128 x 32 tile: it stages the tile with its R-wide halo in shared
// memory (reflected at the image borders), then each thread filters 4 consecutive
// pixels of 4 rows, reading each window row with 16-byte shared-memory loads and
// treating its pixels in pairs with packed FP32x2 arithmetic (the ex2 stays scalar).
#include "snlm_host.h"
#include "snlm_internal.h"

#include <utility>

namespace snlm {

namespace {

constexpr int kBfPx = 4;                      // consecutive pixels of a row per thread
constexpr int kBfTileW = 32 * kBfPx;          // columns per CTA
constexpr int kBfWarps = 8;
constexpr int kBfRowsPerThread = 4;
constexpr int kBfTileH = kBfWarps * kBfRowsPerThread;
constexpr int kBfTaps = (2 * kBfMaxR + 1) * (2 * kBfMaxR + 1);

struct BfArgs {
    const float *in;
    float *out;
    long long in_pitch, out_pitch;
    int H, W;
    float2 cr2;              // (cr, cr), cr = -log2(e) / (2 sigma_r^2)
    float2 lw2[kBfTaps];     // (lw, lw) of tap dy * (2R + 1) + dx: -log2(e) ((dx-R)^2 + (dy-R)^2) / (2 sigma_s^2)
};

// Two floats in one 64-bit register pair for the packed FP32x2 instructions (two
// pixels per issue slot).
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f32x2 pk2(float2 v) { return pk(v.x, v.y); }
__device__ __forceinline__ float lo_of(f32x2 v)
{
    float a;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(a) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi_of(f32x2 v)
{
    float a;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(a) : "l"(v));
    return a;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Half-sample symmetric extension into [0, n), 2n-periodic.
__device__ __forceinline__ int bf_reflect(int x, int n)
{
    if (x >= 0 && x < n)
        return x;
    const int p = 2 * n;
    int y = x % p;
    if (y < 0)
        y += p;
    return y < n ? y : p - 1 - y;
}

__device__ __forceinline__ float bf_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int R>
__global__ void __launch_bounds__(kBfWarps * 32) bilateral_kernel(const __grid_constant__ BfArgs p)
{
    constexpr int D = 2 * R + 1;
    constexpr int NV = (kBfPx + 2 * R + 3) / 4;          // 16-byte loads per window row
    constexpr int SW = 4 * (31 + NV);                    // shared row: columns x0 - R + [0, SW)
    constexpr int SH = kBfTileH + 2 * R;
    __shared__ __align__(16) float tile[SH * SW];

    const int x0 = blockIdx.x * kBfTileW, y0 = blockIdx.y * kBfTileH;
    for (int i = threadIdx.x; i < SH * SW; i += blockDim.x) {
        const int r = i / SW, q = i - r * SW;
        const int y = bf_reflect(y0 - R + r, p.H), x = bf_reflect(x0 - R + q, p.W);
        tile[i] = __ldg(p.in + (long long)y * p.in_pitch + x);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool vec_out = ((reinterpret_cast<uintptr_t>(p.out) | (unsigned long long)p.out_pitch * 4) & 15) == 0;
#pragma unroll 1
    for (int rr = 0; rr < kBfRowsPerThread; ++rr) {
        const int ty = wid + kBfWarps * rr;
        const int y = y0 + ty;
        if (y >= p.H)
            break;
        // pixel pairs (0, 1) and (2, 3): centre, numerator and denominator as float pairs
        f32x2 C2[kBfPx / 2], N2[kBfPx / 2], D2[kBfPx / 2];
#pragma unroll
        for (int q = 0; q < kBfPx / 2; ++q) {
            C2[q] = pk(tile[(ty + R) * SW + 4 * lane + R + 2 * q], tile[(ty + R) * SW + 4 * lane + R + 2 * q + 1]);
            N2[q] = pk(0.f, 0.f);
            D2[q] = pk(1.f, 1.f);                         // the centre tap
        }
        const f32x2 cr2 = pk2(p.cr2);
#pragma unroll
        for (int dy = 0; dy < D; ++dy) {
            float v[4 * NV];
            const float4 *row = reinterpret_cast<const float4 *>(tile + (ty + dy) * SW) + lane;
#pragma unroll
            for (int b = 0; b < NV; ++b) {
                const float4 t = row[b];
                v[4 * b] = t.x;
                v[4 * b + 1] = t.y;
                v[4 * b + 2] = t.z;
                v[4 * b + 3] = t.w;
            }
            // window pairs starting at every position j (even j: the loaded pairs)
            f32x2 V2[4 * NV - 1];
#pragma unroll
            for (int j = 0; j + 1 < 4 * NV; ++j)
                V2[j] = pk(v[j], v[j + 1]);
#pragma unroll
            for (int dx = 0; dx < D; ++dx) {
                const f32x2 lw = pk2(p.lw2[dy * D + dx]);
#pragma unroll
                for (int q = 0; q < kBfPx / 2; ++q) {
                    if (dy == R && dx == R)
                        continue;
                    const f32x2 t = sub2(V2[2 * q + dx], C2[q]);
                    const f32x2 e = fma2(mul2(t, cr2), t, lw);
                    const f32x2 wg = pk(bf_ex2(lo_of(e)), bf_ex2(hi_of(e)));
                    N2[q] = fma2(wg, t, N2[q]);
                    D2[q] = add2(D2[q], wg);
                }
            }
        }
        float c[kBfPx], num[kBfPx], den[kBfPx];
#pragma unroll
        for (int q = 0; q < kBfPx / 2; ++q) {
            c[2 * q] = lo_of(C2[q]);
            c[2 * q + 1] = hi_of(C2[q]);
            num[2 * q] = lo_of(N2[q]);
            num[2 * q + 1] = hi_of(N2[q]);
            den[2 * q] = lo_of(D2[q]);
            den[2 * q + 1] = hi_of(D2[q]);
        }
        float o[kBfPx];
#pragma unroll
        for (int k = 0; k < kBfPx; ++k)
            o[k] = c[k] + num[k] / den[k];
        const int x = x0 + 4 * lane;
        float *dst = p.out + (long long)y * p.out_pitch + x;
        if (vec_out && x + kBfPx <= p.W) {
            *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
            for (int k = 0; k < kBfPx; ++k)
                if (x + k < p.W)
                    dst[k] = o[k];
        }
    }
}

template <int R>
cudaError_t launch_bf(const BfArgs &a, cudaStream_t st)
{
    dim3 grid((unsigned)div_up(a.W, kBfTileW), (unsigned)div_up(a.H, kBfTileH));
    bilateral_kernel<R><<<grid, kBfWarps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

template <int... R>
int preload_bf(std::integer_sequence<int, R...>)
{
    return (preload_kernel((const void *)bilateral_kernel<R>) + ...);
}

bool overlaps(const float *a, long long na, const float *b, long long nb)
{
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
    return a0 < b0 + (uintptr_t)nb * 4 && b0 < a0 + (uintptr_t)na * 4;
}

}  // namespace

int bilateral_radius(float sigma_s) { return (int)std::floor(3.0 * (double)sigma_s); }

int run_bilateral(const float *in, int H, int W, long long in_pitch, float sigma_s, float sigma_r, float *out,
                  long long out_pitch, cudaStream_t st)
{
    const int R = bilateral_radius(sigma_s);
    BfArgs a;
    a.in = in;
    a.out = out;
    a.in_pitch = in_pitch;
    a.out_pitch = out_pitch;
    a.H = H;
    a.W = W;
    const double log2e = 1.4426950408889634;
    const double ss = (double)sigma_s, sr = (double)sigma_r;
    const float cr = (float)(-log2e / (2.0 * sr * sr));
    a.cr2 = make_float2(cr, cr);
    for (int i = 0; i < kBfTaps; ++i)
        a.lw2[i] = make_float2(0.f, 0.f);
    const int D = 2 * R + 1;
    for (int dy = 0; dy < D; ++dy)
        for (int dx = 0; dx < D; ++dx) {
            const double j2 = (double)((dx - R) * (dx - R) + (dy - R) * (dy - R));
            const float lw = (float)(-log2e * j2 / (2.0 * ss * ss));
            a.lw2[dy * D + dx] = make_float2(lw, lw);
        }
    TraceScope ts(SNLM_K_BILATERAL, st);
    cudaError_t e;
    switch (R) {
    case 0: e = launch_bf<0>(a, st); break;
    case 1: e = launch_bf<1>(a, st); break;
    case 2: e = launch_bf<2>(a, st); break;
    case 3: e = launch_bf<3>(a, st); break;
    case 4: e = launch_bf<4>(a, st); break;
    case 5: e = launch_bf<5>(a, st); break;
    case 6: e = launch_bf<6>(a, st); break;
    case 7: e = launch_bf<7>(a, st); break;
    default: e = launch_bf<8>(a, st); break;
    }
    return status_of(e);
}

int check_bilateral(const float *in, int H, int W, long long in_pitch, float sigma_s, float sigma_r,
                    const float *out, long long out_pitch)
{
    if (H < 1 || W < 1 || in_pitch < W || out_pitch < W || (long long)H * in_pitch >= (1LL << 31) ||
        (long long)H * out_pitch >= (1LL << 31))
        return SNLM_ERR_ARG;
    if (!(sigma_s > 0.f) || !std::isfinite(sigma_s) || !(sigma_r > 0.f) || !std::isfinite(sigma_r))
        return SNLM_ERR_ARG;
    if (bilateral_radius(sigma_s) > kBfMaxR || div_up(H, kBfTileH) > 65535)
        return SNLM_ERR_UNSUPPORTED;                    // (the grid's y extent holds the row tiles)
    if (!is_device_ptr(in) || !is_device_ptr(out))
        return SNLM_ERR_ARG;
    if (overlaps(in, (long long)(H - 1) * in_pitch + W, out, (long long)(H - 1) * out_pitch + W))
        return SNLM_ERR_ARG;
    return SNLM_OK;
}

int preload_bilateral()
{
    return preload_bf(std::make_integer_sequence<int, 8>{});
}

}  // namespace snlm

using namespace snlm;

extern "C" {

int snlm_bf_params(float sigma, float *sigma_s, float *sigma_r)
{
    if (!(sigma >= 0.f) || !std::isfinite(sigma) || !sigma_s || !sigma_r)
        return SNLM_ERR_ARG;
    const double s = sigma, s2 = s * s, s3 = s2 * s;
    *sigma_s = (float)(2.5e-6 * s3 - 3.4e-4 * s2 + 0.021 * s + 0.46);
    *sigma_r = (float)(2.8e-4 * s3 - 0.088 * s2 + 8.0 * s - 24.0);
    return SNLM_OK;
}

int snlm_bilateral(const float *in, int H, int W, int in_pitch, float sigma_s, float sigma_r, float *out,
                   int out_pitch, void *stream)
{
    const int rc = check_bilateral(in, H, W, in_pitch, sigma_s, sigma_r, out, out_pitch);
    if (rc != SNLM_OK)
        return rc;
    return run_bilateral(in, H, W, in_pitch, sigma_s, sigma_r, out, out_pitch, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
