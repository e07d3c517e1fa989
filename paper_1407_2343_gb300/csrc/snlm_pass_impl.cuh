// Fused 1-D NLM pass (Eq. (4), with the divergence of Eq. (24) for SURE) and
// the patch-distance kernel, templated on the patch half-width K.
//
// Work decomposition. A CTA holds kWarpsPerCta consecutive lines (rows for a row
// pass, columns for a column pass) and one tile of T output positions along
// them; each warp owns one line. Lane r owns the M = kRun consecutive positions
// x0(r) = b0 + r*M .. x0(r) + M - 1 of the tile's window, where the first
// HR = ceil(S / M) lanes sit left of the tile and only contribute the pairs whose
// right end falls in the tile.
//
// Search offsets are taken in chunks c of M: s = c*M + sg, sg = 1..M. For each s
// the lane lifts its run into the differences Delta_s(x) = f(x+s) - f(x) (Sec.
// II-A, Eqs. (5)-(7) in difference form), reduces them to patch distances
// d^2(x, x+s) of Eq. (3) without a per-pair loop over K for the box profile, and
// forms w = exp(-d^2/h^2) once per unordered pair: by the band symmetry of Eq. (8),
// w(x+s, -s) = w(x, s). The forward contribution goes to the lane's own
// accumulators. The mirrored one (to pixel x+s) lands at register slot m + sg of a
// 2M-entry buffer whose lower half belongs to lane r + c and upper half to lane
// r + c + 1, so after the chunk two warp shuffles per slot deliver it; a lane below
// r + c (or r + c + 1) receives a wrapped value, but such lanes are halo lanes whose
// own outputs are never stored.
//
// Accumulation is centred: A = sum_j w (f(j) - f(i)), Q = sum_j w, so that
// fhat = f(i) + A/Q; the SURE kernels also keep A2 = sum_j w (f(j) - f(i))^2,
// which gives the P2 - Q fhat^2 term of Alg. 3 as A2 - A^2/Q without cancellation.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "snlm_internal.h"

namespace snlm {

// Symmetric extension of a line of n samples (... f1 f0 | f0 f1 ... f_n-1 | f_n-1 ...),
// for any x: the general case, kept out of line (it only runs for tiny lines).
static __device__ __noinline__ int reflect_index_any(int x, int n)
{
    const int p = 2 * n;
    int y = x % p;
    if (y < 0)
        y += p;
    return y < n ? y : p - 1 - y;
}

__device__ __forceinline__ int reflect_index(int x, int n)
{
    if (x >= 0 && x < n)
        return x;
    if (x >= -n && x < 2 * n)   // one reflection
        return x < 0 ? -x - 1 : 2 * n - 1 - x;
    return reflect_index_any(x, n);
}

__device__ __forceinline__ float load_at(const void *ptr, int dtype, unsigned off)
{
    if (dtype == DT_U8)
        return (float)__ldg(static_cast<const unsigned char *>(ptr) + off);
    if (dtype == DT_F16)
        return __half2float(__ldg(static_cast<const __half *>(ptr) + off));
    return __ldg(static_cast<const float *>(ptr) + off);
}

// Element offsets fit in 31 bits (checked by the host before any launch).
__device__ __forceinline__ float load_sample(const Lines &v, int line, int i)
{
    return load_at(v.ptr, v.dtype, (unsigned)(line * (int)v.line_step + i * (int)v.elem_step));
}

// 2^x with the SFU (MUFU.EX2), flushing denormal results to zero.
__device__ __forceinline__ float exp2_sfu(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two floats in one 64-bit register pair (lo, hi) for the packed FP32x2 forms of
// FFMA/FMUL (sm_100 and later): one issue slot for two lane-operations.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f32x2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float f32x2_lo(f32x2 v)
{
    float lo;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(lo) : "l"(v));
    return lo;
}

__device__ __forceinline__ float f32x2_hi(f32x2 v)
{
    float hi;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(hi) : "l"(v));
    return hi;
}

__device__ __forceinline__ f32x2 f32x2_fma(f32x2 a, f32x2 b, f32x2 c)   // a * b + c, each half rounded once
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 f32x2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 f32x2_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 f32x2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Patch distances D[m] = sum_{k=-K..K} g(k) * dl[m + K + k]^2 for m = 0..M-1,
// where dl holds the lifted differences of M + 2K consecutive positions.
template <int K, int DM, int M>
__device__ __forceinline__ void patch_distances(const float (&dl)[M + 2 * K], float (&D)[M],
                                                const float *__restrict__ g)
{
    constexpr int W = 2 * K + 1;
    if constexpr (DM != DIST_FIR && W >= M - 1) {
        // Box profile, windows at least M - 1 wide: every window [m, m + 2K] contains
        // the split point U = M - 1 or ends right before it, so it is the suffix
        // [m, U - 1] plus the prefix [U, m + 2K]. Both parts are sums of squares that
        // all belong to the window (no cancellation; exact for integer samples) and the
        // cost equals a running sum's, with two short chains instead of one long one.
        constexpr int U = M - 1;
        float suf[U];
        suf[U - 1] = dl[U - 1] * dl[U - 1];
#pragma unroll
        for (int u = U - 2; u >= 0; --u)
            suf[u] = fmaf(dl[u], dl[u], suf[u + 1]);
        float pre[M + 2 * K];
        pre[U] = dl[U] * dl[U];
#pragma unroll
        for (int u = U + 1; u < M + 2 * K; ++u)
            pre[u] = fmaf(dl[u], dl[u], pre[u - 1]);
#pragma unroll
        for (int m = 0; m < M; m += 2) {
            const bool both0 = m < U && m + 2 * K >= U, both1 = m + 1 < U && m + 1 + 2 * K >= U;
            if (both0 && both1) {
                // two windows that are both suffix + prefix: one packed add
                const f32x2 r = f32x2_add(f32x2_pack(suf[m], suf[m + 1]),
                                          f32x2_pack(pre[m + 2 * K], pre[m + 1 + 2 * K]));
                D[m] = f32x2_lo(r);
                D[m + 1] = f32x2_hi(r);
            } else {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int mm = m + e;
                    if (mm >= U)
                        D[mm] = pre[mm + 2 * K];
                    else if (mm + 2 * K < U)
                        D[mm] = suf[mm];
                    else
                        D[mm] = suf[mm] + pre[mm + 2 * K];
                }
            }
        }
    } else if constexpr (DM == DIST_SLIDE) {
        // Running sum (box profile): two updates per step, whatever K is.
        float acc = 0.f;
#pragma unroll
        for (int u = 0; u < W; ++u)
            acc = fmaf(dl[u], dl[u], acc);
        D[0] = acc;
#pragma unroll
        for (int m = 1; m < M; ++m) {
            acc = fmaf(dl[m + 2 * K], dl[m + 2 * K], acc);
            acc = fmaf(-dl[m - 1], dl[m - 1], acc);
            D[m] = acc;
        }
    } else if constexpr (DM == DIST_BLOCK) {
        // Box profile with float samples: split the positions into blocks of W;
        // a window is the suffix of one block plus the prefix of the next, so each
        // distance is a sum of non-negative terms that all belong to its own window.
        float pre[M + 2 * K];
#pragma unroll
        for (int u = 0; u < M + 2 * K; ++u)
            pre[u] = (u % W == 0) ? dl[u] * dl[u] : fmaf(dl[u], dl[u], pre[u - 1]);
        float suf[M];
#pragma unroll
        for (int u = M - 1; u >= 0; --u) {
            const int be = (u / W) * W + W - 1;
            if (u == be) {
                suf[u] = dl[u] * dl[u];
            } else if (u + 1 < M) {
                suf[u] = fmaf(dl[u], dl[u], suf[u + 1]);
            } else {
                float t = 0.f;
#pragma unroll
                for (int v = be; v > u; --v)
                    t = fmaf(dl[v], dl[v], t);
                suf[u] = fmaf(dl[u], dl[u], t);
            }
        }
#pragma unroll
        for (int m = 0; m < M; ++m)
            D[m] = (m % W == 0) ? pre[m + 2 * K] : suf[m] + pre[m + 2 * K];
    } else {
        // Gaussian profile: the truncated (2K+1)-tap weighted sum of Eq. (3).
        float F[M + 2 * K];
#pragma unroll
        for (int u = 0; u < M + 2 * K; ++u)
            F[u] = dl[u] * dl[u];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k)
                acc = fmaf(g[k], F[m + k], acc);
            D[m] = acc;
        }
    }
}

// Gathers of the load phase. Thread (w, q0) of the CTA handles line line0 + w and
// positions q = q0 + 32 b; row-like views (elem_step == 1) give each warp one line
// (consecutive lanes on consecutive samples), column-like views give consecutive
// threads consecutive lines of the same position. Every read of a gather is issued
// before its values are used, so a CTA waits for about one memory round trip.
__device__ __forceinline__ void gather_slot(bool row_like, int &w, int &q0)
{
    w = row_like ? (int)(threadIdx.x >> 5) : (int)(threadIdx.x % kWarpsPerCta);
    q0 = row_like ? (int)(threadIdx.x & 31) : (int)(threadIdx.x / kWarpsPerCta);
}

template <typename T>
__device__ __forceinline__ float to_float(T v) { return (float)v; }
template <>
__device__ __forceinline__ float to_float<__half>(__half v) { return __half2float(v); }

// Window samples: v[b] = sample at position pos0 + q (reflected), q < len.
template <typename T, int NB>
__device__ __forceinline__ void gather_window_t(float (&v)[NB], const T *ptr, unsigned base, int es, int N,
                                                int pos0, int q0, int len)
{
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int q = q0 + 32 * b;
        if (q < len) {
            const int x = pos0 + q;
            const int i = reflect_index(x, N);
            v[b] = to_float(__ldg(ptr + base + (unsigned)(i * es)));
        }
    }
}

template <int NB>
__device__ __forceinline__ void gather_window(float (&v)[NB], const Lines &src, int ln, int N, int pos0, int q0,
                                              int len)
{
    const unsigned base = (unsigned)(ln * (int)src.line_step);
    const int es = (int)src.elem_step;
    if (src.dtype == DT_U8)
        gather_window_t<unsigned char, NB>(v, static_cast<const unsigned char *>(src.ptr), base, es, N, pos0, q0,
                                           len);
    else if (src.dtype == DT_F16)
        gather_window_t<__half, NB>(v, static_cast<const __half *>(src.ptr), base, es, N, pos0, q0, len);
    else
        gather_window_t<float, NB>(v, static_cast<const float *>(src.ptr), base, es, N, pos0, q0, len);
}

// Tile samples of a float image: v[b] = img at position xa + q of the line, q < T;
// `fill` past the end of the line.
template <int NB>
__device__ __forceinline__ void gather_tile(float (&v)[NB], const float *img, long long line_step,
                                            long long elem_step, int ln, int N, int xa, int q0, int T, float fill)
{
    const float *row = img + ln * (int)line_step;
    const int es = (int)elem_step;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int q = q0 + 32 * b;
        v[b] = fill;
        if (q < T && xa + q < N)
            v[b] = __ldg(row + (xa + q) * es);
    }
}

// Same for a strided view of any sample type (zero past the end of the line).
template <typename T, int NB>
__device__ __forceinline__ void gather_tile_t(float (&v)[NB], const T *ptr, unsigned base, int es, int N, int xa,
                                              int q0, int T_)
{
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int q = q0 + 32 * b;
        v[b] = 0.f;
        if (q < T_ && xa + q < N)
            v[b] = to_float(__ldg(ptr + base + (unsigned)((xa + q) * es)));
    }
}

template <int NB>
__device__ __forceinline__ void gather_tile_lines(float (&v)[NB], const Lines &img, int ln, int N, int xa, int q0,
                                                  int T)
{
    const unsigned base = (unsigned)(ln * (int)img.line_step);
    const int es = (int)img.elem_step;
    if (img.dtype == DT_U8)
        gather_tile_t<unsigned char, NB>(v, static_cast<const unsigned char *>(img.ptr), base, es, N, xa, q0, T);
    else if (img.dtype == DT_F16)
        gather_tile_t<__half, NB>(v, static_cast<const __half *>(img.ptr), base, es, N, xa, q0, T);
    else
        gather_tile_t<float, NB>(v, static_cast<const float *>(img.ptr), base, es, N, xa, q0, T);
}

template <int NB>
__device__ __forceinline__ void scatter_padded(float *buf, const float (&v)[NB], int q0, int len)
{
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int q = q0 + 32 * b;
        if (q < len)
            buf[pad_index(q)] = v[b];
    }
}

// Most window samples one thread gathers (S <= kMaxS, K <= kMaxK), and most tile
// positions (T <= 31 M).
constexpr int kWindowSlots = (32 * kRun + kMaxS + 2 * kMaxK + 2 * kRun + 31) / 32;
constexpr int kTileSlots = (31 * kRun + 31) / 32;

// Vector forms of the window and tile loads (16-byte and narrower aligned loads)
// for the common layouts; each returns false, having loaded nothing, when its
// conditions do not hold, and the scalar gathers above run instead. Every load of
// a form is issued before the first shared-memory store.

__device__ __forceinline__ float byte_of(unsigned v, int e) { return (float)((v >> (8 * e)) & 0xffu); }

// Row-like window of line `ln`, positions ws .. ws+len-1 all inside [0, N):
// float samples in 16-byte vectors, 16-bit samples in vectors of 8, 8-bit samples in
// vectors of 16.
__device__ __forceinline__ bool load_window_row_vec(float *buf, const Lines &v, int ln, int N, int ws, int len,
                                                    int lane)
{
    if (v.dtype == DT_F32) {
        const float *row = static_cast<const float *>(v.ptr) + ln * (int)v.line_step;
        const int a = ws & ~3, off = ws - a, nv = (off + len + 3) >> 2;
        if (a < 0 || a + 4 * nv > N || (reinterpret_cast<uintptr_t>(row + a) & 15) != 0)
            return false;
        const float4 *src = reinterpret_cast<const float4 *>(row + a);
        constexpr int J = (kWindowSlots * 32 + 127) / 128 + 1;   // float4 per lane, at most
        float4 r[J];
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (lane + 32 * j < nv)
                r[j] = __ldg(src + lane + 32 * j);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k = lane + 32 * j;
            if (k < nv) {
                const float e4[4] = {r[j].x, r[j].y, r[j].z, r[j].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int q = 4 * k + e - off;
                    if (q >= 0 && q < len)
                        buf[pad_index(q)] = e4[e];
                }
            }
        }
        return true;
    }
    if (v.dtype == DT_U8) {
        const unsigned char *row = static_cast<const unsigned char *>(v.ptr) + ln * (int)v.line_step;
        const int a = ws & ~15, off = ws - a, nv = (off + len + 15) >> 4;
        if (a < 0 || a + 16 * nv > N || (reinterpret_cast<uintptr_t>(row + a) & 15) != 0)
            return false;
        const uint4 *src = reinterpret_cast<const uint4 *>(row + a);
        constexpr int J = (kWindowSlots * 32 + 511) / 512 + 1;
        uint4 r[J];
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (lane + 32 * j < nv)
                r[j] = __ldg(src + lane + 32 * j);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k = lane + 32 * j;
            if (k < nv) {
                const unsigned w4[4] = {r[j].x, r[j].y, r[j].z, r[j].w};
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int q = 16 * k + e - off;
                    if (q >= 0 && q < len)
                        buf[pad_index(q)] = byte_of(w4[e >> 2], e & 3);
                }
            }
        }
        return true;
    }
    if (v.dtype == DT_F16) {
        const __half *row = static_cast<const __half *>(v.ptr) + ln * (int)v.line_step;
        const int a = ws & ~7, off = ws - a, nv = (off + len + 7) >> 3;
        if (a < 0 || a + 8 * nv > N || (reinterpret_cast<uintptr_t>(row + a) & 15) != 0)
            return false;
        const uint4 *src = reinterpret_cast<const uint4 *>(row + a);
        constexpr int J = (kWindowSlots * 32 + 255) / 256 + 1;
        uint4 r[J];
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (lane + 32 * j < nv)
                r[j] = __ldg(src + lane + 32 * j);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k = lane + 32 * j;
            if (k < nv) {
                const unsigned w4[4] = {r[j].x, r[j].y, r[j].z, r[j].w};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int q = 8 * k + e - off;
                    if (q >= 0 && q < len) {
                        const __half2 hh = *reinterpret_cast<const __half2 *>(&w4[e >> 1]);
                        buf[pad_index(q)] = (e & 1) ? __high2float(hh) : __low2float(hh);
                    }
                }
            }
        }
        return true;
    }
    return false;
}

// Column-like window of the CTA's 4 lines (adjacent in memory): one load brings the
// 4 samples of a position (16 bytes of float, 8 of half, 4 of 8-bit samples).
__device__ __forceinline__ bool load_window_col_vec(float *smem, int per_warp, const Lines &v, int n_lines, int N,
                                                    int line0, int ws, int len)
{
    const int es = v.dtype == DT_U8 ? 1 : (v.dtype == DT_F16 ? 2 : 4);
    if (v.line_step != 1 || line0 + kWarpsPerCta > n_lines || (v.elem_step & 3) != 0 ||
        (reinterpret_cast<uintptr_t>(v.ptr) & (uintptr_t)(4 * es - 1)) != 0)
        return false;
    constexpr int J = (kWindowSlots * 32 + 4 * 32 * kWarpsPerCta - 1) / (32 * kWarpsPerCta);
    const int es_step = (int)v.elem_step;
    if (v.dtype == DT_F32) {
        const float *base = static_cast<const float *>(v.ptr) + line0;
        float4 r[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int q = threadIdx.x + blockDim.x * j;
            if (q < len)
                r[j] = __ldg(reinterpret_cast<const float4 *>(base + reflect_index(ws + q, N) * es_step));
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int q = threadIdx.x + blockDim.x * j;
            if (q < len) {
                const int pq = pad_index(q);
                smem[pq] = r[j].x;
                smem[per_warp + pq] = r[j].y;
                smem[2 * per_warp + pq] = r[j].z;
                smem[3 * per_warp + pq] = r[j].w;
            }
        }
        return true;
    }
    if (v.dtype == DT_U8) {
        const unsigned char *base = static_cast<const unsigned char *>(v.ptr) + line0;
        unsigned r[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int q = threadIdx.x + blockDim.x * j;
            if (q < len)
                r[j] = __ldg(reinterpret_cast<const unsigned *>(base + reflect_index(ws + q, N) * es_step));
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int q = threadIdx.x + blockDim.x * j;
            if (q < len) {
                const int pq = pad_index(q);
#pragma unroll
                for (int w = 0; w < kWarpsPerCta; ++w)
                    smem[w * per_warp + pq] = byte_of(r[j], w);
            }
        }
        return true;
    }
    const __half *base = static_cast<const __half *>(v.ptr) + line0;
    uint2 r[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int q = threadIdx.x + blockDim.x * j;
        if (q < len)
            r[j] = __ldg(reinterpret_cast<const uint2 *>(base + reflect_index(ws + q, N) * es_step));
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int q = threadIdx.x + blockDim.x * j;
        if (q < len) {
            const int pq = pad_index(q);
            const __half2 lo = *reinterpret_cast<const __half2 *>(&r[j].x);
            const __half2 hi = *reinterpret_cast<const __half2 *>(&r[j].y);
            smem[pq] = __low2float(lo);
            smem[per_warp + pq] = __high2float(lo);
            smem[2 * per_warp + pq] = __low2float(hi);
            smem[3 * per_warp + pq] = __high2float(hi);
        }
    }
    return true;
}

// A float tile input (positions xa .. xa+T-1 of the CTA's lines, `fill` past N)
// into the padded rows at float offset `row` of each warp. Row-like views: 16-byte
// vectors along each line; column-like views: the 4 lines of a position in one
// 16-byte load. False (nothing loaded) when the layout does not allow it.
__device__ __forceinline__ bool load_tile_vec(float *smem, int per_warp, int row, const float *img,
                                              long long line_step, long long elem_step, int n_lines, int N,
                                              int line0, int xa, int T, float fill)
{
    const int qe = min(T, N - xa);                      // valid positions
    if (elem_step == 1) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int ln = line0 + w;
        const float *src = img + (ln < n_lines ? ln * (int)line_step : 0) + xa;
        if ((reinterpret_cast<uintptr_t>(src) & 15) != 0 || (line_step & 3) != 0)
            return false;
        float *buf = smem + w * per_warp + row;
        constexpr int J = (32 * kRun + 127) / 128;      // float4 per lane (T <= 31 * 8)
        float4 r[J];
        const int nv = qe >> 2;                         // whole vectors inside the line
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (ln < n_lines && lane + 32 * j < nv)
                r[j] = __ldg(reinterpret_cast<const float4 *>(src) + lane + 32 * j);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k = lane + 32 * j;
            if (4 * k < T) {
                const bool whole = ln < n_lines && k < nv;
                const float e4[4] = {r[j].x, r[j].y, r[j].z, r[j].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int q = 4 * k + e;
                    if (q < T)
                        buf[pad_index(q)] = whole ? e4[e] : (ln < n_lines && q < qe ? __ldg(src + q) : fill);
                }
            }
        }
        return true;
    }
    if (line_step != 1 || line0 + kWarpsPerCta > n_lines || (elem_step & 3) != 0 ||
        (reinterpret_cast<uintptr_t>(img + line0) & 15) != 0)
        return false;
    constexpr int J = (32 * kRun + 32 * kWarpsPerCta - 1) / (32 * kWarpsPerCta);
    float4 r[J];
    const int es = (int)elem_step;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int q = threadIdx.x + blockDim.x * j;
        if (q < qe)
            r[j] = __ldg(reinterpret_cast<const float4 *>(img + line0 + (xa + q) * es));
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int q = threadIdx.x + blockDim.x * j;
        if (q < T) {
            const int pq = row + pad_index(q);
            const bool ok = q < qe;
            smem[pq] = ok ? r[j].x : fill;
            smem[per_warp + pq] = ok ? r[j].y : fill;
            smem[2 * per_warp + pq] = ok ? r[j].z : fill;
            smem[3 * per_warp + pq] = ok ? r[j].w : fill;
        }
    }
    return true;
}

// Window load of the distance kernel: buf(w)[pad_index(q)] = sample at position
// pos0 + q of line line0 + w (reflected), q < len.
__device__ __forceinline__ void load_windows(float *smem, int per_warp, const Lines &v, int n_lines,
                                             int N, int line0, int pos0, int len)
{
    int w, q0;
    gather_slot(v.elem_step == 1, w, q0);
    const int ln = line0 + w;
    if (ln >= n_lines)
        return;
    float val[kWindowSlots];
    gather_window(val, v, ln, N, pos0, q0, len);
    scatter_padded(smem + w * per_warp, val, q0, len);
}


// 1/x for x >= 1: the SFU estimate refined by one Newton-Raphson step
// (e = 1 - x r, r' = r + r e), which roughly squares the relative error.
__device__ __forceinline__ float rcp_nr(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.f), r);
}

// One chunk of M search offsets s = c*M + sg, sg = 1..min(M, S - c*M), for the
// lane's run. Every chunk runs the same code (one body, so that the warps of an
// SM share one copy in the instruction cache); the last chunk of a pass may stop
// early. Mirrored contributions wait in slot t = m + sg of a 2M-entry buffer
// whose lower half belongs to lane r + c and upper half to lane r + c + 1, and
// are delivered with warp shuffles at the end of the chunk. The SURE form keeps
// (A, A2) and the mirrored (-A, A2) contributions as float pairs: both take
// (w, w d) x d, one packed FMA each.
template <int K, int DM, bool SURE>
__device__ __forceinline__ void nlm_chunk(const float *__restrict__ fl, int lane, int c, int lim,
                                          const float (&fo)[kRun + 2 * K], float (&A)[kRun], float (&Q)[kRun],
                                          float (&A2)[kRun], float c2, const float *__restrict__ g,
                                          float *wK, int LW)
{
    constexpr int M = kRun;
    constexpr int NF = M + 2 * K;
    constexpr int NG = 2 * M + 2 * K;
    // samples at positions x0 + c*M + 1 - K + j (lanes r + c and r + c + 1)
    float gv[NG];
    const float *gp = fl + 9 * (lane + c);
#pragma unroll
    for (int j = 0; j < NG; ++j)
        gv[j] = gp[(1 + j) + (1 + j) / 8];
    // slots 1..M are first written at sg = 1; the others may stay empty when the
    // chunk stops early
    float BA[2 * M], BQ[2 * M];
    f32x2 AA[M], BB[2 * M];             // SURE: (A, A2) and mirrored (-A, A2)
    if constexpr (SURE) {
#pragma unroll
        for (int m = 0; m < M; ++m)
            AA[m] = f32x2_pack(A[m], A2[m]);
    }
#pragma unroll
    for (int t = M + 1; t < 2 * M; ++t) {
        BQ[t] = 0.f;
        if constexpr (SURE)
            BB[t] = 0ull;
        else
            BA[t] = 0.f;
    }
#pragma unroll
    for (int sg = 1; sg <= M; ++sg) {
        if (sg > lim)
            break;
        // the lift; in the plain passes, for odd sg, two positions per packed subtraction
        // (the sample pairs (gv[2i], gv[2i+1]) against (fo[u], fo[u+1]), u even). The
        // SURE passes keep the scalar form: the pairing constraints cost them spills.
        float dl[NF];
        if (!SURE && (sg & 1)) {
#pragma unroll
            for (int u = 0; u < NF; u += 2) {
                const f32x2 r = f32x2_sub(f32x2_pack(gv[u + sg - 1], gv[u + sg]), f32x2_pack(fo[u], fo[u + 1]));
                dl[u] = f32x2_lo(r);
                dl[u + 1] = f32x2_hi(r);
            }
        } else {
#pragma unroll
            for (int u = 0; u < NF; ++u)
                dl[u] = gv[u + sg - 1] - fo[u];
        }
        float D[M];
        patch_distances<K, DM, M>(dl, D, g);
        float X[M];                     // exponents d^2 * c2, two per packed multiply
#pragma unroll
        for (int m = 0; m < M; m += 2) {
            const f32x2 x = f32x2_mul(f32x2_pack(D[m], D[m + 1]), f32x2_pack(c2, c2));
            X[m] = f32x2_lo(x);
            X[m + 1] = f32x2_hi(x);
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float w = exp2_sfu(X[m]);
            const float d = dl[m + K];
            const int t = m + sg;
            const bool first = (t <= M) && (sg == 1);
            Q[m] += w;
            BQ[t] = first ? w : BQ[t] + w;
            if constexpr (SURE) {
                const f32x2 wv = f32x2_pack(w, w * d);
                const f32x2 dd = f32x2_pack(d, d);
                AA[m] = f32x2_fma(wv, dd, AA[m]);
                BB[t] = first ? f32x2_mul(wv, dd) : f32x2_fma(wv, dd, BB[t]);
                if (sg <= K && c == 0)
                    wK[(sg - 1) * LW + 9 * lane + m] = w;
            } else {
                A[m] = fmaf(w, d, A[m]);
                BA[t] = first ? -w * d : fmaf(-w, d, BA[t]);
            }
        }
    }
    // deliver the mirrored contributions
    const f32x2 sgn = f32x2_pack(-1.f, 1.f);
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const float rq = __shfl_up_sync(0xffffffffu, BQ[M + j], c + 1);
        Q[j] += (j > 0) ? __shfl_up_sync(0xffffffffu, BQ[j], c) + rq : rq;
        if constexpr (SURE) {
            const float n1 = __shfl_up_sync(0xffffffffu, f32x2_lo(BB[M + j]), c + 1);
            const float s1 = __shfl_up_sync(0xffffffffu, f32x2_hi(BB[M + j]), c + 1);
            AA[j] = f32x2_fma(f32x2_pack(n1, s1), sgn, AA[j]);
            if (j > 0) {
                const float n0 = __shfl_up_sync(0xffffffffu, f32x2_lo(BB[j]), c);
                const float s0 = __shfl_up_sync(0xffffffffu, f32x2_hi(BB[j]), c);
                AA[j] = f32x2_fma(f32x2_pack(n0, s0), sgn, AA[j]);
            }
        } else {
            const float ra = __shfl_up_sync(0xffffffffu, BA[M + j], c + 1);
            A[j] += (j > 0) ? __shfl_up_sync(0xffffffffu, BA[j], c) + ra : ra;
        }
    }
    if constexpr (SURE) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            A[m] = f32x2_lo(AA[m]);
            A2[m] = f32x2_hi(AA[m]);
        }
    }
}

// Offsets (in floats) of the per-warp rows of a pass's shared-memory layout: the
// line window (reused for fhat), then blend | SURE: K weight rows, delta_in,
// delta_out, f_rc, f. Tile rows are padded like the window (pad_index).
struct RowOffsets {
    int bl, wk, din, dout, rc, f;
    __device__ __forceinline__ RowOffsets(const WarpLayout &L, int K)
    {
        bl = L.LF;
        wk = bl + L.LT;
        din = wk + L.LK;
        dout = din + L.LT;
        rc = dout + L.LT;
        f = rc + L.LT;
    }
};

// ---- Asynchronous load phase -------------------------------------------------
// The common layouts load through cp.async in short rolled loops: every copy is
// issued before the first wait, nothing is staged in registers, and the code is
// small, so the chunk body of the search stays in the instruction cache (the
// unrolled register gathers below cost ~15 % of a pass's issue slots in cache
// misses alone). float32 samples are copied one by one to their padded slots from
// reflected addresses; 8- and 16-bit samples are copied as raw aligned words into a
// staging area (a region of the warp's rows that is idle during the load phase)
// and converted after the wait.

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ int sample_size(int dtype) { return dtype == DT_U8 ? 1 : (dtype == DT_F16 ? 2 : 4); }

// An 8- or 16-bit sample at byte offset `off` of a staging area.
__device__ __forceinline__ float staged_sample(const unsigned char *raw, int dtype, int off)
{
    if (dtype == DT_U8)
        return (float)raw[off];
    return __half2float(*reinterpret_cast<const __half *>(raw + off));
}

// Samples [lo, hi) of row `ln` of a row-like view as words (and a ragged tail of at
// most 3 bytes) into `stg`; returns the byte offset in the row of stg[0].
__device__ __forceinline__ int stage_row(unsigned char *stg, const Lines &v, int ln, int lo, int hi, int lane)
{
    const int es = sample_size(v.dtype);
    const unsigned char *row = static_cast<const unsigned char *>(v.ptr) + (long long)ln * v.line_step * es;
    const int b0 = (lo * es) & ~3, b1 = hi * es, w1 = b1 & ~3;
#pragma unroll 1
    for (int o = b0 + 4 * lane; o < w1; o += 128)
        cp_async4(stg + (o - b0), row + o);
    if (w1 + lane < b1)
        stg[w1 + lane - b0] = row[w1 + lane];
    return b0;
}

// Positions start .. start+n-1 of the CTA's kWarpsPerCta adjacent lines of a
// column-like view: position q's samples go to stg(q % 4) + (q / 4) * 4 * es, where
// stg(w) = stage + w * pw floats; `reflect` maps positions through the extension.
__device__ __forceinline__ void stage_cols(float *stage, int pw, const Lines &v, int line0, int N, int start, int n,
                                           bool reflect)
{
    const int es = sample_size(v.dtype);
    const unsigned char *base = static_cast<const unsigned char *>(v.ptr) + (long long)line0 * es;
    const long long pstep = v.elem_step * es;
#pragma unroll 1
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int x = reflect ? reflect_index(start + q, N) : min(start + q, N - 1);
        unsigned char *d = reinterpret_cast<unsigned char *>(stage + (q & 3) * pw) + (q >> 2) * 4 * es;
        if (es == 1)
            cp_async4(d, base + x * pstep);
        else
            cp_async8(d, base + x * pstep);
    }
}

// Float32 samples into padded rows: row `row` of line line0 + w holds position
// start + q at pad_index(q), q < n; positions at or past N take `fill` (tiles) or
// are reflected (windows). A thread's slots are 32 positions apart, 36 floats apart
// in the padded row; when every position lies in [0, N) the loop just walks the two
// pointers.
__device__ __forceinline__ void copy_f32(float *smem, int pw, int row, const float *img, long long ls, long long es,
                                         int n_lines, int N, int line0, int start, int n, bool reflect, float fill)
{
    int w, q0;
    gather_slot(es == 1, w, q0);
    const int ln = line0 + w;
    if (ln >= n_lines)
        return;
    const float *src = img + (long long)ln * ls;
    float *buf = smem + w * pw + row;
    if (start >= 0 && start + n <= N) {
        const float *g = src + (long long)(start + q0) * es;
        float *d = buf + pad_index(q0);
        const long long gstep = 32 * es;
#pragma unroll 1
        for (int q = q0; q < n; q += 32, g += gstep, d += 36)
            cp_async4(d, g);
        return;
    }
#pragma unroll 1
    for (int q = q0; q < n; q += 32) {
        const int x = start + q;
        if (reflect)
            cp_async4(buf + pad_index(q), src + (long long)reflect_index(x, N) * es);
        else if (x < N)
            cp_async4(buf + pad_index(q), src + (long long)x * es);
        else
            buf[pad_index(q)] = fill;
    }
}

// Converts a staged view into padded float rows at `row` (windows: reflected
// positions; tiles: zero past N). Each thread walks pointers through its slots (32
// positions apart) when no position needs the extension.
template <typename T>
__device__ __forceinline__ void unstage_walk(float *d, const unsigned char *src, int step, int q, int n)
{
#pragma unroll 1
    for (; q < n; q += 32, src += step, d += 36)
        *d = to_float(*reinterpret_cast<const T *>(src));
}

__device__ __forceinline__ void unstage(float *smem, int pw, int row, const float *stage, const Lines &v, int n_lines,
                                        int N, int line0, int start, int n, int lo, bool reflect)
{
    const int es = sample_size(v.dtype);
    const bool inside = start >= 0 && start + n <= N;
    if (v.elem_step == 1) {
        const int w = threadIdx.x >> 5, ln = line0 + w;
        if (ln >= n_lines)
            return;
        const unsigned char *stg = reinterpret_cast<const unsigned char *>(stage + w * pw);
        const int b0 = (lo * es) & ~3;
        float *buf = smem + w * pw + row;
        const int q0 = threadIdx.x & 31;
        if (inside) {
            const unsigned char *src = stg + (start + q0) * es - b0;
            if (v.dtype == DT_U8)
                unstage_walk<unsigned char>(buf + pad_index(q0), src, 32, q0, n);
            else
                unstage_walk<__half>(buf + pad_index(q0), src, 64, q0, n);
            return;
        }
#pragma unroll 1
        for (int q = q0; q < n; q += 32) {
            const int x = reflect ? reflect_index(start + q, N) : start + q;
            buf[pad_index(q)] = x < N ? staged_sample(stg, v.dtype, x * es - b0) : 0.f;
        }
    } else {
        const int w = threadIdx.x % kWarpsPerCta, q0 = threadIdx.x / kWarpsPerCta;
        if (reflect || inside) {
            // position q's samples sit in area q % 4 at (q / 4) * 4 es; q0 % 4 stays fixed
            const unsigned char *src =
                reinterpret_cast<const unsigned char *>(stage + (q0 & 3) * pw) + (q0 >> 2) * 4 * es + w * es;
            float *d = smem + w * pw + row + pad_index(q0);
            if (v.dtype == DT_U8)
                unstage_walk<unsigned char>(d, src, 32, q0, n);
            else
                unstage_walk<__half>(d, src, 64, q0, n);
            return;
        }
#pragma unroll 1
        for (int q = q0; q < n; q += 32) {
            const unsigned char *src = reinterpret_cast<const unsigned char *>(stage + (q & 3) * pw) + (q >> 2) * 4 * es;
            smem[w * pw + row + pad_index(q)] = start + q < N ? staged_sample(src, v.dtype, w * es) : 0.f;
        }
    }
}

// The load phase through cp.async (see above). The host launches this form only when
// every view's layout allows it (async_layout_ok): float32 views of any layout;
// 8- and 16-bit windows in 4-byte-aligned rows (row-like) or, column-like, in
// aligned groups of kWarpsPerCta lines with n_lines a multiple of kWarpsPerCta; K >= 1
// for a staged window (its staging area is the weight rows). The noisy image f of
// the SURE sums, when it is stored in 8 or 16 bits, is gathered into registers
// while the copies fly.
template <bool SURE, bool STAGED>
__device__ __forceinline__ void load_async(const PassArgs &p, float *smem, int pw, const RowOffsets &R, int line0,
                                           int xa, int T, int ws, int len, int stage_row_off)
{
    const int N = p.N;
    constexpr bool staged_win = STAGED;   // 8- or 16-bit window samples (else float32)
    const bool gathered_f = SURE && p.aux_rc.ptr && p.aux_f.dtype != DT_F32;
    // window samples needed: [lo, hi) covers every reflected index of [ws, ws + len)
    int lo = 0, hi = N;
    if (ws >= -N && ws + len <= 2 * N) {
        lo = max(0, min(ws, 2 * N - ws - len));
        hi = min(N, max(ws + len, -ws));
    }
    float *const stage = smem + stage_row_off;          // warp w's area at stage + w * pw
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- issue every copy
    if constexpr (!staged_win) {
        copy_f32(smem, pw, 0, static_cast<const float *>(p.src.ptr), p.src.line_step, p.src.elem_step, p.n_lines, N,
                 line0, ws, len, true, 0.f);
    } else if (p.src.elem_step == 1) {
        if (line0 + wid < p.n_lines)
            stage_row(reinterpret_cast<unsigned char *>(stage + wid * pw), p.src, line0 + wid, lo, hi, lane);
    } else {
        stage_cols(stage, pw, p.src, line0, N, ws, len, true);
    }
    const long long ols = p.out_line_step, oes = p.out_elem_step;
    if (p.blend)
        copy_f32(smem, pw, R.bl, p.blend, ols, oes, p.n_lines, N, line0, xa, T, false, 0.f);
    if constexpr (SURE) {
        if (p.delta_in)
            copy_f32(smem, pw, R.din, p.delta_in, ols, oes, p.n_lines, N, line0, xa, T, false, 1.f);
        if (p.aux_rc.ptr) {
            copy_f32(smem, pw, R.rc, static_cast<const float *>(p.aux_rc.ptr), p.aux_rc.line_step,
                     p.aux_rc.elem_step, p.n_lines, N, line0, xa, T, false, 0.f);
            if (!gathered_f)
                copy_f32(smem, pw, R.f, static_cast<const float *>(p.aux_f.ptr), p.aux_f.line_step,
                         p.aux_f.elem_step, p.n_lines, N, line0, xa, T, false, 0.f);
        }
        if (!p.delta_in) {
            int dw, dq0;
            gather_slot(p.out_elem_step == 1, dw, dq0);
#pragma unroll 1
            for (int q = dq0; q < T; q += 32)
                smem[dw * pw + R.din + pad_index(q)] = 1.f;
        }
    }
    int ow, oq0;
    gather_slot(p.out_elem_step == 1, ow, oq0);
    const bool oline = line0 + ow < p.n_lines;
    float vf[kTileSlots];
    if (gathered_f && oline)
        gather_tile_lines(vf, p.aux_f, line0 + ow, N, xa, oq0, T);
    cp_async_wait_all();
    if (gathered_f && oline)
        scatter_padded(smem + ow * pw + R.f, vf, oq0, T);
    // ---- the staged window into float rows
    if constexpr (staged_win) {
        __syncthreads();
        unstage(smem, pw, 0, stage, p.src, p.n_lines, N, line0, ws, len, lo, true);
    }
}


__device__ __forceinline__ void st_global_v4(float *p, float a, float b, float c, float d)
{
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// Store the M results of a lane to out[o + m], m < nvalid, with two 16-byte stores
// when the run is whole and aligned.
__device__ __forceinline__ void store_run(float *out, const float (&v)[kRun], int nvalid)
{
    if (nvalid == kRun && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        st_global_v4(out, v[0], v[1], v[2], v[3]);
        st_global_v4(out + 4, v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int m = 0; m < kRun; ++m)
            if (m < nvalid)
                out[m] = v[m];
    }
}

// The end of a unit, after the search: finalise each lane's run in registers
// (fhat = f + A/Q, optionally blended; for SURE the chained derivative of Eq. (24)
// and the sums of its valid pixels), write the results (row-like outputs straight
// from registers; column-like outputs through the warp's rows and 16-byte stores
// across the CTA's 4 lines) and reduce the SURE sums of the unit into its record.
// All threads of the CTA must call it. `pw` is the per-warp stride of smem (floats).
template <int K, int DM, bool SURE>
__device__ __forceinline__ void unit_epilogue(const PassArgs &p, float *smem, int pw, const RowOffsets &R, int LW,
                                              int unit, int line0, int xa, int T, int HR, bool have_line,
                                              const float (&fo)[kRun + 2 * K], const float (&A)[kRun],
                                              const float (&Q)[kRun], const float (&A2)[kRun])
{
    constexpr int M = kRun;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int line = line0 + wid;
    const int N = p.N;
    const int qe = min(T, N - xa);                    // valid positions of the tile
    const bool row_like = p.out_elem_step == 1;
    const int ls = (int)p.out_line_step, es = (int)p.out_elem_step;
    float *const fl = smem + wid * pw;
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (have_line && lane >= HR) {
        const int j = lane - HR;
        const int nvalid = min(M, qe - 8 * j);
        // the run's outputs that enter the SURE sums: valid ones whose image row (the
        // line of a row pass, the position of a column pass) is in [sum_lo, sum_hi)
        int m_lo = 0, m_hi = nvalid;
        if (SURE && p.sum_hi != 0) {
            if (row_like) {
                if (line < p.sum_lo || line >= p.sum_hi)
                    m_hi = 0;
            } else {
                m_lo = max(0, p.sum_lo - (xa + 8 * j));
                m_hi = min(nvalid, p.sum_hi - (xa + 8 * j));
            }
        }
        const float *wf_row = fl + R.wk + 9 * lane;   // w(x, s) of the lane's own positions
        const float ih2 = SURE ? __frcp_rn(p.h2) : 0.f;
        float fh[M], dv[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float Qt = 1.f + Q[m];
            const float r = rcp_nr(Qt);
            const float mu = A[m] * r;
            float v = fo[m + K] + mu;
            if (p.blend)
                v = 0.5f * (v + fl[R.bl + 9 * j + m]);
            fh[m] = v;
            dv[m] = 0.f;
            if constexpr (SURE) {
                // Eq. (24): the patch-overlap term over 0 < |s| <= min(K, S),
                // T = sum_s g(s) [wf (a_s - mu) a_-s + wb (a_-s - mu) a_s] = TA - mu TB
                // with a_s = f(x+s) - f(x), wf = w(x, s), wb = w(x-s, s). Position
                // 8 lane + m - s of the padded weight row is at 9 lane + (m - s) - (m < s).
                float TA = 0.f, TB = 0.f;
#pragma unroll
                for (int sg = 1; sg <= K; ++sg) {
                    if (sg > p.S)
                        break;
                    const float ap = fo[m + K + sg] - fo[m + K];
                    const float am = fo[m + K - sg] - fo[m + K];
                    float wf = wf_row[(sg - 1) * LW + m];
                    float wb = wf_row[(sg - 1) * LW + (m - sg) - (m < sg ? 1 : 0)];
                    if constexpr (DM == DIST_FIR) {
                        wf *= p.g[K + sg];
                        wb *= p.g[K + sg];
                    }
                    TA = fmaf(wf + wb, ap * am, TA);
                    TB = fmaf(wf, am, fmaf(wb, ap, TB));
                }
                const float Tt = fmaf(-mu, TB, TA);
                const float var = A2[m] - mu * A[m];   // sum_j w (f(j) - fhat)^2
                const float num = p.h2 + 2.f * Tt + 2.f * var;
                dv[m] = fl[R.din + 9 * j + m] * (num * r) * ih2;
                if (m >= m_lo && m < m_hi) {
                    s[5] += dv[m];
                    if (p.aux_rc.ptr) {
                        // sums of the SURE system in the basis m = (f_rc + f_cr)/2, d = (f_rc - f_cr)/2
                        const float rc = fl[R.rc + 9 * j + m];
                        const float fv = fl[R.f + 9 * j + m];
                        const float mm = 0.5f * (rc + v), dd = 0.5f * (rc - v);
                        s[0] = fmaf(mm, mm, s[0]);
                        s[1] = fmaf(mm, dd, s[1]);
                        s[2] = fmaf(dd, dd, s[2]);
                        s[3] = fmaf(fv, mm, s[3]);
                        s[4] = fmaf(fv, dd, s[4]);
                    }
                }
            }
        }
        if (row_like) {
            if (nvalid > 0) {
                const unsigned o = (unsigned)(line * ls + xa + 8 * j);
                store_run(p.dst + o, fh, nvalid);
                if (SURE && p.delta_out)
                    store_run(p.delta_out + o, dv, nvalid);
            }
        } else {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                fl[9 * j + m] = fh[m];
                if constexpr (SURE)
                    fl[R.dout + 9 * j + m] = dv[m];
            }
        }
    }
    if (!row_like) {
        // column-like output: position q of the CTA's lines line0..line0+3
        __syncthreads();
        const int nl = min(kWarpsPerCta, p.n_lines - line0);
        const bool packed = ls == 1 && nl == kWarpsPerCta;
        for (int q = threadIdx.x; q < qe; q += blockDim.x) {
            const int pq = pad_index(q);
            const unsigned o = (unsigned)(line0 * ls + (xa + q) * es);
            float v[kWarpsPerCta], d[kWarpsPerCta];
#pragma unroll
            for (int w = 0; w < kWarpsPerCta; ++w) {
                v[w] = smem[w * pw + pq];
                d[w] = SURE ? smem[w * pw + R.dout + pq] : 0.f;
            }
            if (packed && (reinterpret_cast<uintptr_t>(p.dst + o) & 15) == 0) {
                st_global_v4(p.dst + o, v[0], v[1], v[2], v[3]);
                if (SURE && p.delta_out)
                    st_global_v4(p.delta_out + o, d[0], d[1], d[2], d[3]);
            } else {
#pragma unroll
                for (int w = 0; w < kWarpsPerCta; ++w)
                    if (w < nl) {
                        p.dst[o + w * ls] = v[w];
                        if (SURE && p.delta_out)
                            p.delta_out[o + w * ls] = d[w];
                    }
            }
        }
    }
    if constexpr (SURE) {
        if (p.partials) {
            // deterministic reduction: float warp tree, then the warps in order in fp64
            __shared__ float red[kWarpsPerCta][6];
            // without the f_rc input only sum [5] is formed; the others are zero
            const int k0 = p.aux_rc.ptr ? 0 : 5;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (k < k0) {
                    if (lane == 0)
                        red[wid][k] = 0.f;
                    continue;
                }
                float v = s[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0)
                    red[wid][k] = v;
            }
            __syncthreads();
            if (threadIdx.x < kPartials) {
                double t = 0.0;
                if (threadIdx.x < 6)
                    for (int w = 0; w < kWarpsPerCta; ++w)
                        t += (double)red[w][threadIdx.x];
                p.partials[(long long)unit * kPartials + threadIdx.x] = t;
            }
        }
    }
}

// The load phase through register gathers (and 16-byte vector loads where the layout
// allows): the plain passes' path, and the SURE passes' when the asynchronous copies
// do not apply (a separate kernel instantiation, so that neither form's code or
// registers weigh on the other).
template <int K, bool SURE>
__device__ __forceinline__ void load_gather(const PassArgs &p, float *smem, const WarpLayout &L, const RowOffsets &R,
                                         int line0, int xa, int T, int b0, int nch)
{
    constexpr int M = kRun;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int line = line0 + wid;
    const int N = p.N;

        const int len = 32 * M + nch * M + 2 * K + M;
        const int ws = b0 - K;
        // (the vector forms serve the plain passes: measured on GB300 they are slower
        // for the SURE passes, whose several tile inputs then load in separate rounds)
        bool done_win = false, vb_ok = false;
        const bool vd_ok = false, vr_ok = false;
        if constexpr (!SURE) {
            if (p.src.elem_step == 1) {
                done_win = line >= p.n_lines ||
                           load_window_row_vec(smem + wid * L.per_warp, p.src, line, N, ws, len, lane);
                done_win = __syncthreads_and(done_win);
            } else {
                done_win = load_window_col_vec(smem, L.per_warp, p.src, p.n_lines, N, line0, ws, len);
            }
            vb_ok = p.blend && load_tile_vec(smem, L.per_warp, R.bl, p.blend, p.out_line_step, p.out_elem_step,
                                             p.n_lines, N, line0, xa, T, 0.f);
        }
        int w, q0;
        gather_slot(p.src.elem_step == 1, w, q0);
        const int ln = line0 + w;
        float vw[kWindowSlots];
        if (!done_win && ln < p.n_lines)
            gather_window(vw, p.src, ln, N, ws, q0, len);
        int ow, oq0;
        gather_slot(p.out_elem_step == 1, ow, oq0);
        const int oln = line0 + ow;
        const bool oline = oln < p.n_lines;
        float vb[kTileSlots], vd[kTileSlots], vr[kTileSlots], vf[kTileSlots];
        if (p.blend && !vb_ok && oline)
            gather_tile(vb, p.blend, p.out_line_step, p.out_elem_step, oln, N, xa, oq0, T, 0.f);
        if constexpr (SURE) {
            if (oline) {
                if (p.delta_in && !vd_ok)
                    gather_tile(vd, p.delta_in, p.out_line_step, p.out_elem_step, oln, N, xa, oq0, T, 1.f);
                if (p.aux_rc.ptr) {
                    if (!vr_ok)
                        gather_tile(vr, static_cast<const float *>(p.aux_rc.ptr), p.aux_rc.line_step,
                                    p.aux_rc.elem_step, oln, N, xa, oq0, T, 0.f);
                    gather_tile_lines(vf, p.aux_f, oln, N, xa, oq0, T);
                }
            }
        }
        if (!done_win && ln < p.n_lines)
            scatter_padded(smem + w * L.per_warp, vw, q0, len);
        float *const ob = smem + ow * L.per_warp;
        if (p.blend && !vb_ok && oline)
            scatter_padded(ob + R.bl, vb, oq0, T);
        if constexpr (SURE) {
            if (!p.delta_in) {
#pragma unroll
                for (int b = 0; b < kTileSlots; ++b)
                    if (oq0 + 32 * b < T)
                        ob[R.din + pad_index(oq0 + 32 * b)] = 1.f;
            } else if (!vd_ok && oline) {
                scatter_padded(ob + R.din, vd, oq0, T);
            }
            if (p.aux_rc.ptr && oline) {
                if (!vr_ok)
                    scatter_padded(ob + R.rc, vr, oq0, T);
                scatter_padded(ob + R.f, vf, oq0, T);
            }
        }
}

// One CTA-sized unit of a pass: kWarpsPerCta lines x one tile of positions.
// `bid` enumerates the units of the pass (tile fastest). All threads of the CTA
// must call it (it contains CTA barriers); smem must hold the pass's layout.
// How a pass loads its inputs (a template parameter, so that each kernel holds one
// form's code): register gathers and vector loads; asynchronous copies of a float32
// window; asynchronous copies of an 8- or 16-bit window through the staging area.
enum Loader { LOAD_GATHER = 0, LOAD_ASYNC_F32 = 1, LOAD_ASYNC_STAGED = 2 };

template <int K, int DM, bool SURE, int LOADER = LOAD_GATHER>
__device__ __forceinline__ void process_tile(const PassArgs &p, int bid, float *smem)
{
    constexpr int M = kRun;
    constexpr int NF = M + 2 * K;        // lifted positions per run (patch halo K each side)

    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.S;
    const int HR = div_up(S, M), nch = div_up(S, M);
    const int T = tile_positions(S);
    const int tiles = p.tiles;                     // units are numbered tile fastest
    const int grp = bid / tiles;
    const int xa = (bid - grp * tiles) * T;
    const int b0 = xa - HR * M;
    const int line0 = grp * kWarpsPerCta;
    const int line = line0 + wid;
    const WarpLayout L = warp_layout(S, K, SURE, false);
    const RowOffsets R(L, K);
    float *const fl = smem + wid * L.per_warp;     // samples at positions b0 - K + q (padded)
    if constexpr (kSmemGuard > 0) {
        if (lane < kSmemGuard)
            reinterpret_cast<unsigned *>(fl)[L.guard + lane] = kGuardWord ^ (unsigned)lane;
        __syncthreads();
    }

    // ---- load phase: the line windows (with reflection) and every tile input the
    // epilogue reads: asynchronous copies (ASYNC, SURE passes whose layouts allow
    // them; the staging area of 8- and 16-bit windows is the weight rows, idle until
    // the first chunk) or register gathers and vector loads.
    if constexpr (LOADER == LOAD_GATHER)
        load_gather<K, SURE>(p, smem, L, R, line0, xa, T, b0, nch);
    else
        load_async<SURE, LOADER == LOAD_ASYNC_STAGED>(p, smem, L.per_warp, R, line0, xa, T, b0 - K,
                                                      32 * M + nch * M + 2 * K + M, R.wk);
    __syncthreads();

    float fo[NF];
    float A[M], Q[M], A2[M];
    const bool have_line = line < p.n_lines;
    if (have_line) {
        // samples of the own run with the patch halo: positions x0 - K + u
#pragma unroll
        for (int u = 0; u < NF; ++u)
            fo[u] = fl[9 * lane + u + u / 8];
#pragma unroll
        for (int m = 0; m < M; ++m)
            A[m] = Q[m] = A2[m] = 0.f;
        for (int c = 0; c < nch; ++c)
            nlm_chunk<K, DM, SURE>(fl, lane, c, S - c * M, fo, A, Q, A2, p.c2, p.g, fl + R.wk, L.LW);
        __syncwarp();
    }
    unit_epilogue<K, DM, SURE>(p, smem, L.per_warp, R, L.LW, bid, line0, xa, T, HR, have_line, fo, A, Q, A2);
    if constexpr (kSmemGuard > 0) {
        __syncthreads();
        if (lane < kSmemGuard && p.check &&
            reinterpret_cast<const unsigned *>(fl)[L.guard + lane] != (kGuardWord ^ (unsigned)lane))
            atomicExch(p.check, (unsigned)(-SNLM_ERR_CHECK));
        __syncthreads();
    }
}

// CTAs per SM the compiler is held to (registers per thread = 65536 / (128 x this)),
// chosen per variant by measuring 4096^2 passes at S = 10 and 20 on GB300. Plain
// passes: 5 (96 registers) while the variant fits them with few or no spills, else 4
// (128 registers): the running-sum pass up to K = 4 (2-9 % faster than at 4; at K = 5
// 4 is 4 % faster), the float block-sum pass up to K = 3 (up to 8 % faster; 4-36 %
// slower beyond), the Gaussian pass up to K = 5 (1-7 % faster; 3-11 % slower
// beyond). SURE passes: 4 (128 registers; 18 % slower at 3), and 3 (168 registers)
// from K = 7, where 128 registers spill (21 % faster at S = 20).
template <int K, int DM, bool SURE>
constexpr int pass_min_ctas()
{
    if (SURE)
        return K >= 7 ? 3 : 4;
    if (DM == DIST_SLIDE)
        return K <= 4 ? 5 : 4;
    if (DM == DIST_BLOCK)
        return K <= 3 ? 5 : 4;
    return K <= 5 ? 5 : 4;
}

template <int K, int DM, bool SURE, int LOADER>
__global__ void __launch_bounds__(kWarpsPerCta * 32, pass_min_ctas<K, DM, SURE>()) nlm_pass_kernel(const __grid_constant__ PassArgs p)
{
    extern __shared__ __align__(16) float smem[];
    process_tile<K, DM, SURE, LOADER>(p, (int)blockIdx.x, smem);
}

// Patch distances only: the same lift and reduction as the pass kernel, written
// out as d^2(x, x+s) for s in [-S, S] (the mirrored half from the band symmetry).
template <int K, int DM>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 4) patch_dist_kernel(const __grid_constant__ DistArgs p)
{
    constexpr int M = kRun;
    constexpr int NF = M + 2 * K;
    constexpr int NG = 2 * M + 2 * K;
    extern __shared__ __align__(16) float smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.S, N = p.N;
    const int HR = div_up(S, M), nch = div_up(S, M);
    const int T = tile_positions(S);
    const int tiles = div_up(N, T);
    const int xa = (int)(blockIdx.x % tiles) * T;
    const int b0 = xa - HR * M;
    const int line0 = (int)(blockIdx.x / tiles) * kWarpsPerCta;
    const int line = line0 + wid;
    const WarpLayout L = warp_layout(S, K, false, true);
    float *const fl = smem + wid * L.per_warp;

    load_windows(smem, L.per_warp, p.src, p.n_lines, N, line0, b0 - K, 32 * M + nch * M + 2 * K + M);
    __syncthreads();
    if (line >= p.n_lines)
        return;
    const int xe = min(xa + T, N);
    const long long row = 2LL * S + 1;
    const long long base = (long long)line * N * row;
    int *const oi = static_cast<int *>(p.out);
    float *const of = static_cast<float *>(p.out);

    if (lane >= HR) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int x = b0 + lane * M + m;
            if (x < xe) {
                if (p.int_out)
                    oi[base + x * row + S] = 0;
                else
                    of[base + x * row + S] = 0.f;
            }
        }
    }
    float fo[NF];
#pragma unroll
    for (int u = 0; u < NF; ++u)
        fo[u] = fl[9 * lane + u + u / 8];
    for (int c = 0; c < nch; ++c) {
        float g[NG];
        const float *gp = fl + 9 * (lane + c);
#pragma unroll
        for (int j = 0; j < NG; ++j)
            g[j] = gp[(1 + j) + (1 + j) / 8];
#pragma unroll
        for (int sg = 1; sg <= M; ++sg) {
            const int s = c * M + sg;
            if (s > S)
                break;
            float dl[NF];
#pragma unroll
            for (int u = 0; u < NF; ++u)
                dl[u] = g[u + sg - 1] - fo[u];
            float D[M];
            patch_distances<K, DM, M>(dl, D, p.g);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int x = b0 + lane * M + m;
                const int y = x + s;
                if (x >= xa && x < xe) {
                    if (p.int_out)
                        oi[base + x * row + S + s] = __float2int_rn(D[m]);
                    else
                        of[base + x * row + S + s] = D[m];
                }
                if (y >= xa && y < xe) {
                    if (p.int_out)
                        oi[base + y * row + S - s] = __float2int_rn(D[m]);
                    else
                        of[base + y * row + S - s] = D[m];
                }
            }
        }
    }
}

// Whether a view of 8- or 16-bit samples can be copied as aligned 4-byte words by
// every unit of a pass: row-like views (elem_step 1) need 4-byte-aligned rows;
// column-like views (line_step 1) need each position's kWarpsPerCta samples aligned
// (4 or 8 bytes) and every CTA's lines present. float32 views take any layout.
inline bool async_view_ok(const Lines &v, int n_lines)
{
    if (v.dtype == DT_F32)
        return true;
    const long long es = v.dtype == DT_U8 ? 1 : 2;
    const uintptr_t base = reinterpret_cast<uintptr_t>(v.ptr);
    if (v.elem_step == 1)
        return (base & 3) == 0 && ((v.line_step * es) & 3) == 0;
    if (v.line_step == 1)
        return n_lines % kWarpsPerCta == 0 && (base & (uintptr_t)(4 * es - 1)) == 0 &&
               ((v.elem_step * es) & (4 * es - 1)) == 0;
    return false;
}

// The asynchronous load form of a SURE pass applies: its window's layout, and for an
// 8- or 16-bit window a staging area (the K >= 1 weight rows) large enough.
inline bool async_layout_ok(const PassArgs &a, int K)
{
    if (a.src.dtype == DT_F32)
        return true;
    if (K < 1 || !async_view_ok(a.src, a.n_lines))
        return false;
    const WarpLayout L = warp_layout(a.S, K, true, false);
    const int len = 32 * kRun + div_up(a.S, kRun) * kRun + 2 * K + kRun;
    const int es = a.src.dtype == DT_U8 ? 1 : 2;
    const int bytes = a.src.elem_step == 1 ? len * es + 8 : ((len + 3) / 4) * 4 * es;
    return ((bytes + 15) / 16) * 4 <= L.LK;
}

template <int K, int DM, bool SURE, int LOADER>
static cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st)
{
    const WarpLayout L = warp_layout(a.S, K, SURE, false);
    const size_t smem = (size_t)L.per_warp * kWarpsPerCta * sizeof(float);
    auto kern = nlm_pass_kernel<K, DM, SURE, LOADER>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long nb = (long long)div_up(a.N, tile_positions(a.S)) * div_up(a.n_lines, kWarpsPerCta);
    if (nb >= (1LL << 31))
        return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)nb);
    kern<<<grid, kWarpsPerCta * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_pass(const PassArgs &a, int dist_mode, bool sure, cudaStream_t st)
{
    // the SURE passes load asynchronously where the layouts allow (the running-sum
    // passes only ever read 8-bit samples, the block-sum passes 16- or 32-bit ones)
    const int ld = !sure || !async_layout_ok(a, K) ? LOAD_GATHER
                                                   : (a.src.dtype == DT_F32 ? LOAD_ASYNC_F32 : LOAD_ASYNC_STAGED);
    switch (dist_mode) {
    case DIST_SLIDE:
        if (!sure)
            return launch_pass_t<K, DIST_SLIDE, false, LOAD_GATHER>(a, st);
        if (ld == LOAD_ASYNC_STAGED)
            return launch_pass_t<K, DIST_SLIDE, true, LOAD_ASYNC_STAGED>(a, st);
        return launch_pass_t<K, DIST_SLIDE, true, LOAD_GATHER>(a, st);
    case DIST_BLOCK:
        if (!sure)
            return launch_pass_t<K, DIST_BLOCK, false, LOAD_GATHER>(a, st);
        if (ld == LOAD_ASYNC_F32)
            return launch_pass_t<K, DIST_BLOCK, true, LOAD_ASYNC_F32>(a, st);
        if (ld == LOAD_ASYNC_STAGED)
            return launch_pass_t<K, DIST_BLOCK, true, LOAD_ASYNC_STAGED>(a, st);
        return launch_pass_t<K, DIST_BLOCK, true, LOAD_GATHER>(a, st);
    default:
        if (!sure)
            return launch_pass_t<K, DIST_FIR, false, LOAD_GATHER>(a, st);
        if (ld == LOAD_ASYNC_F32)
            return launch_pass_t<K, DIST_FIR, true, LOAD_ASYNC_F32>(a, st);
        if (ld == LOAD_ASYNC_STAGED)
            return launch_pass_t<K, DIST_FIR, true, LOAD_ASYNC_STAGED>(a, st);
        return launch_pass_t<K, DIST_FIR, true, LOAD_GATHER>(a, st);
    }
}

template <int K, int DM>
static cudaError_t launch_dist_t(const DistArgs &a, cudaStream_t st)
{
    const WarpLayout L = warp_layout(a.S, K, false, true);
    const size_t smem = (size_t)L.per_warp * kWarpsPerCta * sizeof(float);
    auto kern = patch_dist_kernel<K, DM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long nb = (long long)div_up(a.N, tile_positions(a.S)) * div_up(a.n_lines, kWarpsPerCta);
    if (nb >= (1LL << 31))
        return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)nb);
    kern<<<grid, kWarpsPerCta * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_dist(const DistArgs &a, int dist_mode, cudaStream_t st)
{
    switch (dist_mode) {
    case DIST_SLIDE:
        return launch_dist_t<K, DIST_SLIDE>(a, st);
    case DIST_BLOCK:
        return launch_dist_t<K, DIST_BLOCK>(a, st);
    default:
        return launch_dist_t<K, DIST_FIR>(a, st);
    }
}

// The kernels launch_pass and launch_dist dispatch to, and no others.
template <int K>
int preload_pass()
{
    const void *f[] = {
        (const void *)nlm_pass_kernel<K, DIST_SLIDE, false, LOAD_GATHER>,
        (const void *)nlm_pass_kernel<K, DIST_SLIDE, true, LOAD_ASYNC_STAGED>,
        (const void *)nlm_pass_kernel<K, DIST_SLIDE, true, LOAD_GATHER>,
        (const void *)nlm_pass_kernel<K, DIST_BLOCK, false, LOAD_GATHER>,
        (const void *)nlm_pass_kernel<K, DIST_BLOCK, true, LOAD_ASYNC_F32>,
        (const void *)nlm_pass_kernel<K, DIST_BLOCK, true, LOAD_ASYNC_STAGED>,
        (const void *)nlm_pass_kernel<K, DIST_BLOCK, true, LOAD_GATHER>,
        (const void *)nlm_pass_kernel<K, DIST_FIR, false, LOAD_GATHER>,
        (const void *)nlm_pass_kernel<K, DIST_FIR, true, LOAD_ASYNC_F32>,
        (const void *)nlm_pass_kernel<K, DIST_FIR, true, LOAD_ASYNC_STAGED>,
        (const void *)nlm_pass_kernel<K, DIST_FIR, true, LOAD_GATHER>,
        (const void *)patch_dist_kernel<K, DIST_SLIDE>,
        (const void *)patch_dist_kernel<K, DIST_BLOCK>,
        (const void *)patch_dist_kernel<K, DIST_FIR>,
    };
    int n = 0;
    for (const void *k : f)
        n += preload_kernel(k);
    return n;
}

}  // namespace snlm

#define SNLM_INSTANTIATE_K(KK)                                                                       \
    template cudaError_t snlm::launch_pass<KK>(const snlm::PassArgs &, int, bool, cudaStream_t);     \
    template cudaError_t snlm::launch_dist<KK>(const snlm::DistArgs &, int, cudaStream_t);           \
    template int snlm::preload_pass<KK>();
