// Fused 1-D NLM pass (Eq. (4), with the divergence of Eq. (24) for SURE) and
// the patch-distance kernel, templated on the patch half-width K.
//
// Work decomposition. A CTA holds kWarpsPerCta consecutive lines (rows for a row
// pass, columns for a column pass) and one tile of T output positions along
// them; each warp owns one line. Lane r owns the kRun consecutive positions
// b0 + r*kRun .. b0 + r*kRun + kRun - 1 of the tile's window, where the first
// HR = ceil(S / kRun) lanes sit left of the tile: they compute only the pairs
// whose right end falls in the tile.
//
// For every search offset s = 1..S the lane lifts its run into the differences
// Delta_s(x) = f(x+s) - f(x) (Sec. II-A, Eqs. (5)-(7) in difference form), reduces
// them to patch distances d^2(x, x+s) (Eq. (3)) without a per-pair K-loop for the
// box profile, and forms w = exp(-d^2/h^2) once per unordered pair: the band
// symmetry of Eq. (8) gives w(x+s, -s) = w(x, s). The forward contribution goes to
// the lane's own accumulators, the mirrored one (to pixel x+s) into a small
// register buffer that is added to per-warp shared-memory accumulators after each
// chunk of kChunk offsets, in two phases so no two lanes touch the same word.
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

__device__ __forceinline__ float load_sample(const Lines &v, long long line, int i)
{
    const long long off = line * v.line_step + (long long)i * v.elem_step;
    if (v.dtype == DT_U8)
        return (float)__ldg(static_cast<const unsigned char *>(v.ptr) + off);
    if (v.dtype == DT_F16)
        return __half2float(__ldg(static_cast<const __half *>(v.ptr) + off));
    return __ldg(static_cast<const float *>(v.ptr) + off);
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
// buf(w)[q] = sample at position pos0 + q of line line0 + w (reflected), q < len.
// Row-like views (elem_step == 1) are read along the line; column-like views are
// read across lines so consecutive threads touch consecutive addresses.
__device__ __forceinline__ void load_windows(float *smem, int per_warp, const Lines &v, int n_lines,
                                             int N, int line0, int pos0, int len)
{
    if (v.elem_step == 1) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int ln = line0 + w;
        float *buf = smem + w * per_warp;
        for (int q = lane; q < len; q += 32)
            buf[q] = ln < n_lines ? load_sample(v, ln, reflect_index(pos0 + q, N)) : 0.f;
    } else {
        const int total = kWarpsPerCta * len;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int q = e / kWarpsPerCta, w = e % kWarpsPerCta;
            const int ln = line0 + w;
            smem[w * per_warp + q] = ln < n_lines ? load_sample(v, ln, reflect_index(pos0 + q, N)) : 0.f;
        }
    }
}

template <int K, int DM, bool SURE>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 2) nlm_pass_kernel(const __grid_constant__ PassArgs p)
{
    constexpr int M = kRun, SC = kChunk;
    constexpr int NF = M + 2 * K;    // lifted positions per run (patch halo K each side)
    constexpr int NG = NF + SC;      // shifted samples needed for one chunk of offsets
    extern __shared__ __align__(16) float smem[];

    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.S, N = p.N;
    const int HR = div_up(S, M), nch = div_up(S, SC);
    const int T = tile_positions(S);
    const int tiles = div_up(N, T);                // grid is linear: tile fastest
    const int xa = (int)(blockIdx.x % tiles) * T;
    const int b0 = xa - HR * M;
    const int line0 = (int)(blockIdx.x / tiles) * kWarpsPerCta;
    const int line = line0 + wid;
    const WarpLayout L = warp_layout(S, K, SURE, false);

    float *const fl = smem + wid * L.per_warp;     // samples at positions b0 - K + q
    float *const accA = fl + L.LF;
    float *const accQ = accA + L.LA;
    float *const accA2 = accQ + L.LA;              // SURE only
    float *const wK = fl + L.LF + L.kinds * L.LA;  // SURE: w(x, s) for s = 1..K
    float *const din = wK + K * L.LW;              // SURE: delta_in of the tile
    float *const dst_d = din + 32 * M;             // SURE: delta_out of the tile

    // ---- load: the line windows (with reflection), zeroed accumulators, delta_in
    load_windows(smem, L.per_warp, p.src, p.n_lines, N, line0, b0 - K, L.LF);
    for (int q = lane; q < L.kinds * L.LA; q += 32)
        accA[q] = 0.f;
    if constexpr (SURE) {
        if (p.delta_in) {
            const Lines dv{p.delta_in, DT_F32, p.out_line_step, p.out_elem_step};
            // positions past the end of the line are never stored; clamp the read
            if (dv.elem_step == 1) {
                for (int q = lane; q < T; q += 32)
                    din[q] = (line < p.n_lines && xa + q < N) ? load_sample(dv, line, xa + q) : 1.f;
            } else {
                for (int e = threadIdx.x; e < kWarpsPerCta * T; e += blockDim.x) {
                    const int q = e / kWarpsPerCta, w = e % kWarpsPerCta;
                    const int ln = line0 + w;
                    smem[w * L.per_warp + (din - fl) + q] =
                        (ln < p.n_lines && xa + q < N) ? load_sample(dv, ln, xa + q) : 1.f;
                }
            }
        } else {
            for (int q = lane; q < T; q += 32)
                din[q] = 1.f;
        }
    }
    __syncthreads();

    if (line < p.n_lines) {
        float fo[NF];
#pragma unroll
        for (int u = 0; u < NF; ++u)
            fo[u] = fl[lane * M + u];
        float A[M], Q[M], A2[M];
#pragma unroll
        for (int m = 0; m < M; ++m)
            A[m] = Q[m] = A2[m] = 0.f;

        for (int c = 0; c < nch; ++c) {
            float g[NG];
            const float *gp = fl + lane * M + c * SC + 1;
#pragma unroll
            for (int j = 0; j < NG; ++j)
                g[j] = gp[j];
            float BA[M + SC], BQ[M + SC], BA2[M + SC];
#pragma unroll
            for (int j = 0; j < M + SC; ++j)
                BA[j] = BQ[j] = BA2[j] = 0.f;
#pragma unroll
            for (int sg = 1; sg <= SC; ++sg) {
                if (c * SC + sg > S)
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
                    if constexpr (SURE) {
                        const float v = w * d;
                        A[m] += v;
                        BA[m + sg] -= v;
                        A2[m] = fmaf(v, d, A2[m]);
                        BA2[m + sg] = fmaf(v, d, BA2[m + sg]);
                        if (c == 0 && sg <= K)
                            wK[(sg - 1) * L.LW + lane * M + m] = w;
                    } else {
                        A[m] = fmaf(w, d, A[m]);
                        BA[m + sg] = fmaf(-w, d, BA[m + sg]);
                    }
                    Q[m] += w;
                    BQ[m + sg] += w;
                }
            }
            // add the mirrored contributions: targets lane*M + c*SC + j, j = 1..M+SC-1
            __syncwarp();
#pragma unroll
            for (int j = 1; j <= M; ++j) {
                const int q = acc_index(lane * M + c * SC + j);
                accA[q] += BA[j];
                accQ[q] += BQ[j];
                if constexpr (SURE)
                    accA2[q] += BA2[j];
            }
            __syncwarp();
#pragma unroll
            for (int j = M + 1; j < M + SC; ++j) {
                const int q = acc_index(lane * M + c * SC + j);
                accA[q] += BA[j];
                accQ[q] += BQ[j];
                if constexpr (SURE)
                    accA2[q] += BA2[j];
            }
            __syncwarp();
        }

        // ---- finalise own pixels: fhat = f + A/Q (and the chained derivative)
        if (lane >= HR) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int pr = lane * M + m;
                const int q = acc_index(pr);
                const float At = A[m] + accA[q];
                const float Qt = 1.f + Q[m] + accQ[q];
                const float mu = __fdiv_rn(At, Qt);
                fl[pr - HR * M] = fo[m + K] + mu;
                if constexpr (SURE) {
                    // Eq. (24): the patch-overlap term over 0 < |s| <= min(K, S)
                    float Tt = 0.f;
#pragma unroll
                    for (int sg = 1; sg <= K; ++sg) {
                        if (sg > S)
                            break;
                        const float ap = fo[m + K + sg] - fo[m + K];
                        const float am = fo[m + K - sg] - fo[m + K];
                        const float wf = wK[(sg - 1) * L.LW + pr];
                        const float wb = wK[(sg - 1) * L.LW + pr - sg];
                        const float t = wf * (ap - mu) * am + wb * (am - mu) * ap;
                        Tt = (DM == DIST_FIR) ? fmaf(p.g[K + sg], t, Tt) : Tt + t;
                    }
                    const float var = (A2[m] + accA2[q]) - mu * At;   // sum_j w (f(j) - fhat)^2
                    const float num = p.h2 + 2.f * Tt + 2.f * var;
                    dst_d[pr - HR * M] = din[pr - HR * M] * __fdiv_rn(num, Qt * p.h2);
                }
            }
        }
    }
    __syncthreads();

    // ---- store: fhat (optionally blended), delta_out, partial sums
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool row_like = p.out_elem_step == 1;
    const int total = kWarpsPerCta * T;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int q, w;
        if (row_like) {
            w = e / T;
            q = e - w * T;
        } else {
            q = e / kWarpsPerCta;
            w = e % kWarpsPerCta;
        }
        const int ln = line0 + w, x = xa + q;
        if (ln >= p.n_lines || x >= N)
            continue;
        const float *wb = smem + w * L.per_warp;
        const long long o = ln * p.out_line_step + (long long)x * p.out_elem_step;
        float v = wb[q];
        if (p.blend)
            v = 0.5f * (v + p.blend[o]);
        p.dst[o] = v;
        if constexpr (SURE) {
            const float dv = wb[(dst_d - fl) + q];
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
    if constexpr (SURE) {
        if (p.partials) {
            // deterministic reduction: fp64 warp tree, then warps in order
            double d[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                d[k] = s[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    d[k] += __shfl_down_sync(0xffffffffu, d[k], o);
            }
            __shared__ double red[kWarpsPerCta][6];
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    red[wid][k] = d[k];
            __syncthreads();
            if (threadIdx.x < kPartials) {
                double t = 0.0;
                if (threadIdx.x < 6)
                    for (int w = 0; w < kWarpsPerCta; ++w)
                        t += red[w][threadIdx.x];
                p.partials[(long long)blockIdx.x * kPartials + threadIdx.x] = t;
            }
        }
    }
}

// Patch distances only: the same lift and reduction as the pass kernel, written
// out as d^2(x, x+s) for s in [-S, S] (the mirrored half from the band symmetry).
template <int K, int DM>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 2) patch_dist_kernel(const __grid_constant__ DistArgs p)
{
    constexpr int M = kRun, SC = kChunk;
    constexpr int NF = M + 2 * K;
    constexpr int NG = NF + SC;
    extern __shared__ __align__(16) float smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.S, N = p.N;
    const int HR = div_up(S, M), nch = div_up(S, SC);
    const int T = tile_positions(S);
    const int tiles = div_up(N, T);                // grid is linear: tile fastest
    const int xa = (int)(blockIdx.x % tiles) * T;
    const int b0 = xa - HR * M;
    const int line0 = (int)(blockIdx.x / tiles) * kWarpsPerCta;
    const int line = line0 + wid;
    const WarpLayout L = warp_layout(S, K, false, true);
    float *const fl = smem + wid * L.per_warp;

    load_windows(smem, L.per_warp, p.src, p.n_lines, N, line0, b0 - K, L.LF);
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
        fo[u] = fl[lane * M + u];
    for (int c = 0; c < nch; ++c) {
        float g[NG];
        const float *gp = fl + lane * M + c * SC + 1;
#pragma unroll
        for (int j = 0; j < NG; ++j)
            g[j] = gp[j];
#pragma unroll
        for (int sg = 1; sg <= SC; ++sg) {
            const int s = c * SC + sg;
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
