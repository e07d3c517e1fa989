// Persistent form of the fused 1-D NLM pass whose memory traffic is moved by the
// tensor-memory accelerator (TMA): bulk tensor copies into shared memory that
// complete on mbarriers, so a CTA spends no instructions on gathering samples and
// the next unit's line windows arrive while the current unit computes.
//
// Each CTA loops over the units of the pass (unit u, u + gridDim.x, ...). For
// unit i it holds two window stages: at the top of the iteration one thread
// issues the tile inputs of unit i (delta_in, blend, f_rc, f: read only by the
// epilogue, so they land during the search) and the line windows of unit i + 1
// into the other stage. The threads then wait for stage i & 1, convert it into
// the padded float layout of the search (with the symmetric extension at the
// line ends), run the same search, finalise and store code as the gathered
// kernel, and meet at a barrier before the next iteration reuses the buffers.
//
// Every wait is bounded (TmaPass::wait_ns). A CTA whose wait gives up writes NaN
// to every output of its remaining units, records SNLM_ERR_TIMEOUT in *err and
// returns after a bounded wait for its copies still in flight.
#pragma once

#include "../../include/snlm.h"
#include "snlm_pass_impl.cuh"

namespace snlm {

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order earlier generic-proxy accesses of shared memory before later bulk copies.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier to complete, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (globaltimer_ns() - t0 > limit_ns)
            return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ int floor_to(int x, int a)   // largest multiple of a <= x (a > 0)
{
    const int q = x >= 0 ? x / a : -((-x + a - 1) / a);
    return q * a;
}

// Issue the boxes of one view for a unit: lines line0.., positions start..
// (window: b0 - K; tiles: xa). Returns the byte count they deliver.
__device__ __forceinline__ void tma_issue_view(const TmaView &v, const CUtensorMap *map, unsigned char *area,
                                               int line0, int start, unsigned long long *bar)
{
    if (v.mode == TMA_ROWS) {
        const int x0 = floor_to(start, v.align);
        for (int w = 0; w < kWarpsPerCta; ++w)
            for (int b = 0; b < v.nb; ++b)
                tma_load_2d(area + (size_t)(w * v.sw + b * v.bw) * v.esize, map, x0 + b * v.bw, line0 + w, bar);
    } else {
        const int x0 = floor_to(line0, v.align);
        for (int b = 0; b < v.nb; ++b)
            tma_load_2d(area + (size_t)(b * v.bh * v.sq) * v.esize, map, x0, start + b * v.bh, bar);
    }
}

// Element offset o of a unit's landed data (see TmaView).
__device__ __forceinline__ int tma_unit_offset(const TmaView &v, int line0, int start)
{
    return v.mode == TMA_ROWS ? start - floor_to(start, v.align) : line0 - floor_to(line0, v.align);
}

template <typename T>
__device__ __forceinline__ float landed(const unsigned char *area, int idx)
{
    return to_float(reinterpret_cast<const T *>(area)[idx]);
}

// Convert the landed window of line w into the padded float layout of the search:
// fl[pad_index(q)] = f(b0 - K + q), with the symmetric extension at the ends.
template <typename T>
__device__ __forceinline__ void convert_window_t(const TmaView &v, const unsigned char *area, int o, float *smem,
                                                 int per_warp, const PassArgs &p, int line0, int ws, int len)
{
    const int N = p.N;
    const bool rows = v.mode == TMA_ROWS;
    const int w = rows ? (int)(threadIdx.x >> 5) : (int)(threadIdx.x % kWarpsPerCta);
    const int q0 = rows ? (int)(threadIdx.x & 31) : (int)(threadIdx.x / kWarpsPerCta);
    const int ln = line0 + w;
    if (ln >= p.n_lines)
        return;
    float *fl = smem + w * per_warp;
    const int base = w * v.sw + o;
    const bool inner = ws >= 0 && ws + len <= N;        // no position of the window needs the extension
    for (int q = q0; q < len; q += 32) {
        float val;
        if (inner) {
            val = landed<T>(area, base + q * v.sq);
        } else {
            const int x = ws + q;
            const int i = reflect_index(x, N);
            const int rel = i - ws;
            if (rel >= 0 && rel < len)
                val = landed<T>(area, base + rel * v.sq);
            else
                val = load_sample(p.src, ln, i);
        }
        fl[pad_index(q)] = val;
    }
}

__device__ __forceinline__ void convert_window(const TmaView &v, const unsigned char *area, int o, float *smem,
                                               int per_warp, const PassArgs &p, int line0, int ws, int len)
{
    if (v.dtype == DT_U8)
        convert_window_t<unsigned char>(v, area, o, smem, per_warp, p, line0, ws, len);
    else if (v.dtype == DT_F16)
        convert_window_t<__half>(v, area, o, smem, per_warp, p, line0, ws, len);
    else
        convert_window_t<float>(v, area, o, smem, per_warp, p, line0, ws, len);
}

__device__ __forceinline__ float landed_any(const TmaView &v, const unsigned char *area, int idx)
{
    if (v.dtype == DT_U8)
        return landed<unsigned char>(area, idx);
    if (v.dtype == DT_F16)
        return landed<__half>(area, idx);
    return landed<float>(area, idx);
}

// Outputs of a unit the CTA could not compute: NaN, so that no stale value passes.
__device__ __forceinline__ void poison_unit(const PassArgs &p, int u, int tiles, int T)
{
    const float nan = __int_as_float(0x7fc00000);
    const bool row_like = p.out_elem_step == 1;
    const int w = row_like ? (int)(threadIdx.x >> 5) : (int)(threadIdx.x % kWarpsPerCta);
    const int q0 = row_like ? (int)(threadIdx.x & 31) : (int)(threadIdx.x / kWarpsPerCta);
    const int xa = (u % tiles) * T, ln = (u / tiles) * kWarpsPerCta + w;
    const int qe = ln < p.n_lines ? min(T, p.N - xa) : 0;
    for (int q = q0; q < qe; q += 32) {
        const unsigned o = (unsigned)(ln * (int)p.out_line_step + (xa + q) * (int)p.out_elem_step);
        p.dst[o] = nan;
        if (p.delta_out)
            p.delta_out[o] = nan;
    }
    if (p.partials && threadIdx.x < kPartials)
        p.partials[(long long)u * kPartials + threadIdx.x] = (double)nan;
}

template <int K, int DM, bool SURE>
__global__ void __launch_bounds__(kWarpsPerCta * 32, SURE ? 4 : 5)
    nlm_pass_tma_kernel(const __grid_constant__ PassArgs p, const __grid_constant__ TmaPass t)
{
    constexpr int M = kRun;
    constexpr int NF = M + 2 * K;
    extern __shared__ __align__(128) unsigned char sm_dyn[];
    // bulk tensor copies land on 128-byte boundaries: align the base (the host
    // reserves 128 extra bytes)
    unsigned char *const sm = sm_dyn + ((128u - (smem_addr(sm_dyn) & 127u)) & 127u);
    __shared__ __align__(8) unsigned long long bars[3];   // window stage 0, stage 1, tile inputs

    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.S;
    const int HR = div_up(S, M);
    const int T = tile_positions(S);
    const int tiles = p.tiles;
    const int nch = div_up(S, M);
    const int len = t.win_len;
    float *const smem = reinterpret_cast<float *>(sm);    // per-warp float layout at offset 0
    bool has_tile = false;
#pragma unroll
    for (int a = TMA_DIN; a < TMA_ARRAYS; ++a)
        has_tile |= t.v[a].mode != TMA_NONE;
    unsigned tile_bytes = 0;
#pragma unroll
    for (int a = TMA_DIN; a < TMA_ARRAYS; ++a)
        tile_bytes += t.v[a].mode != TMA_NONE ? (unsigned)t.v[a].bytes : 0u;
    const unsigned extra = t.inject ? 16u : 0u;          // test hook: a barrier that never completes

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        fence_mbar_init();
    }
    __syncthreads();

    int u = blockIdx.x;
    if (threadIdx.x == 0 && u < t.units) {
        const int line0 = (u / tiles) * kWarpsPerCta, b0 = (u % tiles) * T - HR * M;
        mbar_arrive_expect_tx(&bars[0], (unsigned)t.v[TMA_SRC].bytes + extra);
        tma_issue_view(t.v[TMA_SRC], &t.map[TMA_SRC], sm + t.v[TMA_SRC].off, line0, b0 - K, &bars[0]);
    }
    int i = 0;
    bool failed = false;
    for (; u < t.units; ++i, u += gridDim.x) {
        const int st = i & 1;
        const int xa = (u % tiles) * T;
        const int b0 = xa - HR * M;
        const int line0 = (u / tiles) * kWarpsPerCta;
        const int line = line0 + wid;
        if (threadIdx.x == 0) {
            fence_proxy_async();
            if (has_tile) {
                mbar_arrive_expect_tx(&bars[2], tile_bytes + extra);
#pragma unroll
                for (int a = TMA_DIN; a < TMA_ARRAYS; ++a)
                    if (t.v[a].mode != TMA_NONE)
                        tma_issue_view(t.v[a], &t.map[a], sm + t.v[a].off, line0, xa, &bars[2]);
            }
            const int un = u + (int)gridDim.x;
            if (un < t.units) {
                const int l1 = (un / tiles) * kWarpsPerCta, c0 = (un % tiles) * T - HR * M;
                mbar_arrive_expect_tx(&bars[st ^ 1], (unsigned)t.v[TMA_SRC].bytes + extra);
                tma_issue_view(t.v[TMA_SRC], &t.map[TMA_SRC], sm + (st ? t.v[TMA_SRC].off : t.win_off1), l1,
                               c0 - K, &bars[st ^ 1]);
            }
        }
        // ---- the unit's windows: wait, then convert to the padded float layout
        const bool ok = mbar_wait_bounded(&bars[st], (unsigned)(i >> 1) & 1u, t.wait_ns);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        {
            const unsigned char *area = sm + (st ? t.win_off1 : t.v[TMA_SRC].off);
            const int o = tma_unit_offset(t.v[TMA_SRC], line0, b0 - K);
            convert_window(t.v[TMA_SRC], area, o, smem, t.per_warp, p, line0, b0 - K, len);
        }
        __syncthreads();

        float *const fl = smem + wid * t.per_warp;
        const WarpLayout L = warp_layout(S, K, SURE, false);
        const RowOffsets R(L, K);
        float fo[NF];
        float A[M], Q[M], A2[M];
        const bool have_line = line < p.n_lines;
        if (have_line) {
#pragma unroll
            for (int uu = 0; uu < NF; ++uu)
                fo[uu] = fl[9 * lane + uu + uu / 8];
#pragma unroll
            for (int m = 0; m < M; ++m)
                A[m] = Q[m] = A2[m] = 0.f;
            for (int c = 0; c < nch; ++c)
                nlm_chunk<K, DM, SURE>(fl, lane, c, S - c * M, fo, A, Q, A2, p.c2, p.g, fl + R.wk, L.LW);
            __syncwarp();
        }
        // ---- tile inputs of the epilogue: wait, then convert into the padded rows
        if (has_tile) {
            const bool okt = mbar_wait_bounded(&bars[2], (unsigned)i & 1u, t.wait_ns);
            if (__syncthreads_or(!okt)) {
                failed = true;
                break;
            }
        }
        {
            int w, q0;
            gather_slot(p.out_elem_step == 1, w, q0);
            float *const ob = smem + w * t.per_warp;
            const int rows[TMA_ARRAYS] = {0, R.din, R.bl, R.rc, R.f};
#pragma unroll
            for (int a = TMA_DIN; a < TMA_ARRAYS; ++a) {
                const TmaView &v = t.v[a];
                if (v.mode == TMA_NONE) {
                    if (SURE && a == TMA_DIN)
                        for (int q = q0; q < T; q += 32)
                            ob[R.din + pad_index(q)] = 1.f;
                    continue;
                }
                const unsigned char *area = sm + v.off;
                const int base = w * v.sw + tma_unit_offset(v, line0, xa);
                for (int q = q0; q < T; q += 32)
                    ob[rows[a] + pad_index(q)] = landed_any(v, area, base + q * v.sq);
            }
        }
        __syncthreads();
        unit_epilogue<K, DM, SURE>(p, smem, t.per_warp, R, L.LW, u, line0, xa, T, HR, have_line, fo, A, Q, A2);
        __syncthreads();   // the per-warp rows and the tile areas are reused by the next unit
    }
    if (failed) {
        for (; u < t.units; u += gridDim.x)
            poison_unit(p, u, tiles, T);
        if (threadIdx.x == 0) {
            if (t.err)
                atomicExch(t.err, (unsigned)(-SNLM_ERR_TIMEOUT));
            // bounded waits for the copies this CTA may still have in flight
            mbar_wait_bounded(&bars[(i & 1) ^ 1], (unsigned)((i + 1) >> 1) & 1u, t.wait_ns);
            if (has_tile)
                mbar_wait_bounded(&bars[2], (unsigned)i & 1u, t.wait_ns);
        }
        __syncthreads();
    }
}

template <int K, int DM, bool SURE>
static cudaError_t launch_pass_tma_t(const PassArgs &a, const TmaPass &t, int grid, cudaStream_t st)
{
    auto kern = nlm_pass_tma_kernel<K, DM, SURE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, kWarpsPerCta * 32, t.smem, st>>>(a, t);
    return cudaGetLastError();
}

template <int K, int DM, bool SURE>
static cudaError_t occupancy_tma_t(int smem, int *n)
{
    auto kern = nlm_pass_tma_kernel<K, DM, SURE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, kWarpsPerCta * 32, smem);
}

template <int K>
cudaError_t launch_pass_tma(const PassArgs &a, const TmaPass &t, int dist_mode, bool sure, int grid, cudaStream_t st)
{
    switch (dist_mode) {
    case DIST_SLIDE:
        return sure ? launch_pass_tma_t<K, DIST_SLIDE, true>(a, t, grid, st)
                    : launch_pass_tma_t<K, DIST_SLIDE, false>(a, t, grid, st);
    case DIST_BLOCK:
        return sure ? launch_pass_tma_t<K, DIST_BLOCK, true>(a, t, grid, st)
                    : launch_pass_tma_t<K, DIST_BLOCK, false>(a, t, grid, st);
    default:
        return sure ? launch_pass_tma_t<K, DIST_FIR, true>(a, t, grid, st)
                    : launch_pass_tma_t<K, DIST_FIR, false>(a, t, grid, st);
    }
}

template <int K>
cudaError_t pass_tma_occupancy(int dist_mode, bool sure, int smem, int *n)
{
    switch (dist_mode) {
    case DIST_SLIDE:
        return sure ? occupancy_tma_t<K, DIST_SLIDE, true>(smem, n) : occupancy_tma_t<K, DIST_SLIDE, false>(smem, n);
    case DIST_BLOCK:
        return sure ? occupancy_tma_t<K, DIST_BLOCK, true>(smem, n) : occupancy_tma_t<K, DIST_BLOCK, false>(smem, n);
    default:
        return sure ? occupancy_tma_t<K, DIST_FIR, true>(smem, n) : occupancy_tma_t<K, DIST_FIR, false>(smem, n);
    }
}

// The kernels launch_pass_tma dispatches to.
template <int K>
int preload_pass_tma()
{
    const void *f[] = {
        (const void *)nlm_pass_tma_kernel<K, DIST_SLIDE, false>, (const void *)nlm_pass_tma_kernel<K, DIST_SLIDE, true>,
        (const void *)nlm_pass_tma_kernel<K, DIST_BLOCK, false>, (const void *)nlm_pass_tma_kernel<K, DIST_BLOCK, true>,
        (const void *)nlm_pass_tma_kernel<K, DIST_FIR, false>,   (const void *)nlm_pass_tma_kernel<K, DIST_FIR, true>,
    };
    int n = 0;
    for (const void *k : f)
        n += preload_kernel(k);
    return n;
}

}  // namespace snlm

#define SNLM_INSTANTIATE_TMA_K(KK)                                                                             \
    template cudaError_t snlm::launch_pass_tma<KK>(const snlm::PassArgs &, const snlm::TmaPass &, int, bool, int, \
                                                   cudaStream_t);                                              \
    template cudaError_t snlm::pass_tma_occupancy<KK>(int, bool, int, int *);                               \
    template int snlm::preload_pass_tma<KK>();
