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

__device__ __forceinline__ int reflect_index(int x, int n)
{
    if (x >= 0 && x < n)
        return x;
    const int p = 2 * n;
    int y = x % p;
    if (y < 0)
        y += p;
    return y < n ? y : p - 1 - y;
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

// Patch distances D[m] = sum_{k=-K..K} g(k) * dl[m + K + k]^2 for m = 0..M-1,
// where dl holds the lifted differences of M + 2K consecutive positions.
template <int K, int DM, int M>
__device__ __forceinline__ void patch_distances(const float (&dl)[M + 2 * K], float (&D)[M],
                                                const float *__restrict__ g)
{
    constexpr int W = 2 * K + 1;
    if constexpr (DM == DIST_SLIDE) {
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

// Cooperative load of the CTA's line windows into shared memory:
// buf(w)[pad_index(q)] = sample at position pos0 + q of line line0 + w
// (reflected), q < len. Row-like views (elem_step == 1) are read along the line;
// column-like views across lines, so consecutive threads touch consecutive
// addresses.
__device__ __forceinline__ void load_windows(float *smem, int per_warp, const Lines &v, int n_lines,
                                             int N, int line0, int pos0, int len)
{
    if (v.elem_step == 1) {
        // one warp per line, consecutive lanes on consecutive samples
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int ln = line0 + w;
        float *buf = smem + w * per_warp;
        if (ln >= n_lines)
            return;
        const unsigned base = (unsigned)(ln * (int)v.line_step);
        for (int q = lane; q < len; q += 32) {
            const int x = pos0 + q;
            const int i = (x >= 0 && x < N) ? x : reflect_index(x, N);
            buf[q + (q >> 3)] = load_at(v.ptr, v.dtype, base + (unsigned)i);
        }
    } else {
        // columns: consecutive threads on consecutive lines of the same position
        const int w = threadIdx.x % kWarpsPerCta;
        const int ln = line0 + w;
        if (ln >= n_lines)
            return;
        float *buf = smem + w * per_warp;
        const int es = (int)v.elem_step;
        const unsigned base = (unsigned)(ln * (int)v.line_step);
        for (int q = threadIdx.x / kWarpsPerCta; q < len; q += blockDim.x / kWarpsPerCta) {
            const int x = pos0 + q;
            const int i = (x >= 0 && x < N) ? x : reflect_index(x, N);
            buf[q + (q >> 3)] = load_at(v.ptr, v.dtype, base + (unsigned)(i * es));
        }
    }
}

// Cooperative load of a float image restricted to the tile (positions xa + q,
// q < T), padded like the windows; `fill` where the position is past the line.
__device__ __forceinline__ void load_tile(float *smem, int per_warp, int off, const float *img,
                                          long long line_step, long long elem_step, int n_lines, int N,
                                          int line0, int xa, int T, float fill)
{
    if (elem_step == 1) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int ln = line0 + w;
        float *buf = smem + w * per_warp + off;
        const float *row = img + (ln < n_lines ? ln * (int)line_step : 0);
        for (int q = lane; q < T; q += 32)
            buf[q + (q >> 3)] = (ln < n_lines && xa + q < N) ? __ldg(row + xa + q) : fill;
    } else {
        const int w = threadIdx.x % kWarpsPerCta;
        const int ln = line0 + w;
        float *buf = smem + w * per_warp + off;
        const int es = (int)elem_step;
        const float *col = img + (ln < n_lines ? ln * (int)line_step : 0);
        for (int q = threadIdx.x / kWarpsPerCta; q < T; q += blockDim.x / kWarpsPerCta)
            buf[q + (q >> 3)] = (ln < n_lines && xa + q < N) ? __ldg(col + (xa + q) * es) : fill;
    }
}

// One CTA-sized unit of a pass: kWarpsPerCta lines x one tile of positions.
// `bid` enumerates the units of the pass (tile fastest). All threads of the CTA
// must call it (it contains CTA barriers); smem must hold the pass's layout.
template <int K, int DM, bool SURE>
__device__ __forceinline__ void process_tile(const PassArgs &p, int bid, float *smem)
{
    constexpr int M = kRun;
    constexpr int NF = M + 2 * K;        // lifted positions per run (patch halo K each side)
    constexpr int NG = 2 * M + 2 * K;    // shifted samples needed for one chunk of M offsets

    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.S, N = p.N;
    const int HR = div_up(S, M), nch = div_up(S, M);
    const int T = tile_positions(S);
    const int tiles = div_up(N, T);                // units are numbered tile fastest
    const int xa = (bid % tiles) * T;
    const int b0 = xa - HR * M;
    const int line0 = (bid / tiles) * kWarpsPerCta;
    const int line = line0 + wid;
    const WarpLayout L = warp_layout(S, K, SURE, false);

    float *const fl = smem + wid * L.per_warp;     // samples at positions b0 - K + q (padded)
    float *const wK = fl + L.LF;                   // SURE: w(x, s) for s = 1..K (padded rows)
    float *const din = wK + K * L.LW;              // SURE: delta_in of the tile
    float *const dst_d = din + L.LT;               // SURE: delta_out of the tile

    // ---- load: the line windows (with reflection) and delta_in
    load_windows(smem, L.per_warp, p.src, p.n_lines, N, line0, b0 - K, 32 * M + nch * M + 2 * K + M);
    if constexpr (SURE) {
        if (p.delta_in)
            load_tile(smem, L.per_warp, (int)(din - fl), p.delta_in, p.out_line_step, p.out_elem_step,
                      p.n_lines, N, line0, xa, T, 1.f);
        else
            for (int q = lane; q < T; q += 32)
                din[pad_index(q)] = 1.f;
    }
    __syncthreads();

    if (line < p.n_lines) {
        // samples of the own run with the patch halo: positions x0 - K + u
        float fo[NF];
#pragma unroll
        for (int u = 0; u < NF; ++u)
            fo[u] = fl[9 * lane + u + u / 8];
        float A[M], Q[M], A2[M];
#pragma unroll
        for (int m = 0; m < M; ++m)
            A[m] = Q[m] = A2[m] = 0.f;

        for (int c = 0; c < nch; ++c) {
            // samples at positions x0 + c*M + 1 - K + j (lanes r + c and r + c + 1)
            float g[NG];
            const float *gp = fl + 9 * (lane + c);
#pragma unroll
            for (int j = 0; j < NG; ++j)
                g[j] = gp[(1 + j) + (1 + j) / 8];
            // mirrored contributions: slot t goes to lane r + c (t < M) or r + c + 1
            float BA[2 * M], BQ[2 * M], BA2[2 * M];
#pragma unroll
            for (int t = M + 1; t < 2 * M; ++t)
                BA[t] = BQ[t] = BA2[t] = 0.f;
            BA[0] = BQ[0] = BA2[0] = 0.f;
#pragma unroll
            for (int sg = 1; sg <= M; ++sg) {
                if (c * M + sg > S)
                    break;
                float dl[NF];
#pragma unroll
                for (int u = 0; u < NF; ++u)
                    dl[u] = g[u + sg - 1] - fo[u];
                float D[M];
                patch_distances<K, DM, M>(dl, D, p.g);
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const float w = exp2_sfu(D[m] * p.c2);
                    const float d = dl[m + K];
                    const int t = m + sg;
                    const bool first = (sg == 1);   // slots 1..M are first written at sg = 1
                    A[m] = fmaf(w, d, A[m]);
                    BA[t] = first ? -w * d : fmaf(-w, d, BA[t]);
                    if constexpr (SURE) {
                        const float v = w * d;
                        A2[m] = fmaf(v, d, A2[m]);
                        BA2[t] = first ? v * d : fmaf(v, d, BA2[t]);
                        if (c == 0 && sg <= K)
                            wK[(sg - 1) * L.LW + 9 * lane + m] = w;
                    }
                    Q[m] += w;
                    BQ[t] = first ? w : BQ[t] + w;
                }
            }
            // deliver the mirrored contributions
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const float ra = __shfl_up_sync(0xffffffffu, BA[M + j], c + 1);
                const float rq = __shfl_up_sync(0xffffffffu, BQ[M + j], c + 1);
                if (j > 0) {
                    A[j] += __shfl_up_sync(0xffffffffu, BA[j], c) + ra;
                    Q[j] += __shfl_up_sync(0xffffffffu, BQ[j], c) + rq;
                } else {
                    A[j] += ra;
                    Q[j] += rq;
                }
                if constexpr (SURE) {
                    const float r2 = __shfl_up_sync(0xffffffffu, BA2[M + j], c + 1);
                    A2[j] += (j > 0) ? __shfl_up_sync(0xffffffffu, BA2[j], c) + r2 : r2;
                }
            }
        }
        __syncwarp();

        // ---- finalise own pixels: fhat = f + A/Q (and the chained derivative)
        if (lane >= HR) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int q = 9 * (lane - HR) + m;          // padded tile index
                const float Qt = 1.f + Q[m];
                const float mu = __fdiv_rn(A[m], Qt);
                fl[q] = fo[m + K] + mu;
                if constexpr (SURE) {
                    // Eq. (24): the patch-overlap term over 0 < |s| <= min(K, S),
                    // T = sum_s g(s) [wf (a_s - mu) a_-s + wb (a_-s - mu) a_s] = TA - mu TB
                    // with a_s = f(x+s) - f(x), wf = w(x, s), wb = w(x-s, s).
                    float TA = 0.f, TB = 0.f;
#pragma unroll
                    for (int sg = 1; sg <= K; ++sg) {
                        if (sg > S)
                            break;
                        const float ap = fo[m + K + sg] - fo[m + K];
                        const float am = fo[m + K - sg] - fo[m + K];
                        float wf = wK[(sg - 1) * L.LW + 9 * lane + m];
                        const int pb = 8 * lane + m - sg;   // position of x - s, >= 0
                        float wb = wK[(sg - 1) * L.LW + pb + (pb >> 3)];
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
                    dst_d[q] = din[q] * __fdiv_rn(num, Qt * p.h2);
                }
            }
        }
    }
    __syncthreads();

    // ---- store: fhat (optionally blended), delta_out, partial sums
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    {
        const bool row_like = p.out_elem_step == 1;
        const int w = row_like ? wid : (int)(threadIdx.x % kWarpsPerCta);
        const int q0 = row_like ? lane : (int)(threadIdx.x / kWarpsPerCta);
        const int qs = row_like ? 32 : (int)(blockDim.x / kWarpsPerCta);
        const int ln = line0 + w;
        const float *wb = smem + w * L.per_warp;
        const int qe = (ln < p.n_lines) ? min(T, N - xa) : 0;
        const int ls = (int)p.out_line_step, es = (int)p.out_elem_step;
        for (int q = q0; q < qe; q += qs) {
            const int x = xa + q;
            const unsigned o = (unsigned)(ln * ls + x * es);
            float v = wb[q + (q >> 3)];
            if (p.blend)
                v = 0.5f * (v + __ldg(p.blend + o));
            p.dst[o] = v;
            if constexpr (SURE) {
                const float dv = wb[(int)(dst_d - fl) + q + (q >> 3)];
                if (p.delta_out)
                    p.delta_out[o] = dv;
                s[5] += dv;
                if (p.aux_rc.ptr) {
                    // sums of the SURE system in the basis m = (f_rc + f_cr)/2, d = (f_rc - f_cr)/2
                    const float rc = load_sample(p.aux_rc, ln, x);
                    const float fv = load_sample(p.aux_f, ln, x);
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
    if constexpr (SURE) {
        if (p.partials) {
            // deterministic reduction: float warp tree, then the warps in order in fp64
            const int nk = p.aux_rc.ptr ? 6 : 1;
            __shared__ float red[kWarpsPerCta][6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (k >= 6 - nk) {
                    float v = s[k];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
                        v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0)
                        red[wid][k] = v;
                } else if (lane == 0) {
                    red[wid][k] = 0.f;
                }
            }
            __syncthreads();
            if (threadIdx.x < kPartials) {
                double t = 0.0;
                if (threadIdx.x < 6)
                    for (int w = 0; w < kWarpsPerCta; ++w)
                        t += (double)red[w][threadIdx.x];
                p.partials[(long long)bid * kPartials + threadIdx.x] = t;
            }
        }
    }
}

template <int K, int DM, bool SURE>
__global__ void __launch_bounds__(kWarpsPerCta * 32, SURE ? 4 : 5) nlm_pass_kernel(const __grid_constant__ PassArgs p)
{
    extern __shared__ __align__(16) float smem[];
    process_tile<K, DM, SURE>(p, (int)blockIdx.x, smem);
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

template <int K, int DM, bool SURE>
static cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st)
{
    const WarpLayout L = warp_layout(a.S, K, SURE, false);
    const size_t smem = (size_t)L.per_warp * kWarpsPerCta * sizeof(float);
    auto kern = nlm_pass_kernel<K, DM, SURE>;
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
    switch (dist_mode) {
    case DIST_SLIDE:
        return sure ? launch_pass_t<K, DIST_SLIDE, true>(a, st) : launch_pass_t<K, DIST_SLIDE, false>(a, st);
    case DIST_BLOCK:
        return sure ? launch_pass_t<K, DIST_BLOCK, true>(a, st) : launch_pass_t<K, DIST_BLOCK, false>(a, st);
    default:
        return sure ? launch_pass_t<K, DIST_FIR, true>(a, st) : launch_pass_t<K, DIST_FIR, false>(a, st);
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

}  // namespace snlm

#define SNLM_INSTANTIATE_K(KK)                                                                       \
    template cudaError_t snlm::launch_pass<KK>(const snlm::PassArgs &, int, bool, cudaStream_t);     \
    template cudaError_t snlm::launch_dist<KK>(const snlm::DistArgs &, int, cudaStream_t);
