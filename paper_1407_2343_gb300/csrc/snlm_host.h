// Host-side helpers shared by the libsnlm translation units (validation, pass
// parameters, launch tracing).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/snlm.h"
#include "snlm_iir.h"
#include "snlm_internal.h"

namespace snlm {

inline size_t dtype_size(int dt) { return dt == SNLM_U8 ? 1 : (dt == SNLM_F16 ? 2 : 4); }

inline bool valid_dtype(int dt) { return dt == SNLM_U8 || dt == SNLM_F16 || dt == SNLM_F32; }

// A pointer the device can dereference (device or managed memory of any device).
inline bool is_device_ptr(const void *p)
{
    if (!p)
        return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

inline double beta_or_default(float beta, int K) { return beta > 0.f ? (double)beta : (K > 0 ? K / 2.0 : 1.0); }

// Profile weights g(k), k = -K..K (Sec. II, after Eq. (3)).
inline void fill_profile(float *g, int K, int profile, double beta)
{
    for (int k = -K; k <= K; ++k)
        g[k + K] = profile == SNLM_GAUSS ? (float)exp(-(double)k * k / (2.0 * beta * beta)) : 1.f;
    for (int k = 2 * K + 1; k < 2 * kMaxK + 1; ++k)
        g[k] = 0.f;
}

// exponent scale: w = 2^(c2 * d^2) = exp(-d^2 / h^2); kept finite so that
// d^2 = 0 gives w = 1 even when h^2 underflows.
inline float exp2_scale(double h)
{
    double c = -1.4426950408889634 / (h * h);
    if (!(c > -3.0e38))
        c = -3.0e38;
    return (float)c;
}

inline int dist_mode_for(int dtype, int profile)
{
    if (profile == SNLM_GAUSS_IIR)
        return DIST_IIR;
    if (profile == SNLM_GAUSS)
        return DIST_FIR;
    return dtype == SNLM_U8 ? DIST_SLIDE : DIST_BLOCK;
}

// Number of CTAs of one pass over n_lines lines of length N.
inline long long pass_ctas(int n_lines, int N, int S)
{
    return (long long)div_up(N, tile_positions(S)) * div_up(n_lines, kWarpsPerCta);
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int check_common(int H, int W, int S, int K, float h, int profile, int order, float sigma)
{
    if (H < 1 || W < 1 || (long long)H * W >= (1LL << 31))
        return SNLM_ERR_ARG;
    if (S < 0 || S > kMaxS || K < 0)
        return SNLM_ERR_ARG;
    if (K > kMaxK)
        return SNLM_ERR_UNSUPPORTED;
    if (!(h > 0.f) || !isfinite(h))
        return SNLM_ERR_ARG;
    if (profile == SNLM_GAUSS_IIR)
        return SNLM_ERR_UNSUPPORTED;   // only the entry points that check with check_denoise run it
    if (profile != SNLM_BOX && profile != SNLM_GAUSS)
        return SNLM_ERR_ARG;
    if (order < SNLM_RC || order > SNLM_SURE)
        return SNLM_ERR_ARG;
    if (order == SNLM_SURE) {
        if (!(sigma >= 0.f) || !isfinite(sigma))
            return SNLM_ERR_ARG;
        const double h2 = (double)h * h;
        if (!(h2 > 1e-30 && h2 < 1e30))
            return SNLM_ERR_ARG;
    }
    return SNLM_OK;
}

// check_common for the entry points that also run the recursive Gaussian profile:
// beta (K/2 when beta <= 0) must lie in [kIirBetaMin, kIirBetaMax], and the SURE
// order is not available with it (the divergence of Eq. (24) is not formed).
inline int check_denoise(int H, int W, int S, int K, float h, int profile, int order, float sigma, float beta)
{
    if (profile != SNLM_GAUSS_IIR)
        return check_common(H, W, S, K, h, profile, order, sigma);
    const int rc = check_common(H, W, S, K, h, SNLM_GAUSS, order, sigma);
    if (rc != SNLM_OK)
        return rc;
    return iir_check_beta(beta_or_default(beta, K));
}

// view of a (pitched) image along rows (axis 0) or columns (axis 1)
inline Lines image_lines(const void *p, int dtype, int pitch, int axis)
{
    return axis == 0 ? Lines{p, dtype, (long long)pitch, 1} : Lines{p, dtype, 1, (long long)pitch};
}

inline int status_of(cudaError_t e)
{
    if (e == cudaSuccess)
        return SNLM_OK;
    if (e == cudaErrorMemoryAllocation)
        return SNLM_ERR_NOMEM;
    return SNLM_ERR_CUDA;
}

// Separable 3-D extension (snlm_3d.cu): swap the two outer dimensions of a volume of
// rows (out row (a, b) = in row (b, a), samples converted to float32), and
// out = alpha x + beta out.
cudaError_t launch_swap_outer(const void *in, int dtype, float *out, int A, int B, int W, cudaStream_t st);
cudaError_t launch_axpby(const float *x, float *out, float alpha, float beta, long long n, cudaStream_t st);

// ------------------------------------------------------------------ launch tracing

struct TraceRec {
    int kind;
    cudaEvent_t a, b;
};
struct Trace {
    std::mutex mu;
    bool on = false;
    std::vector<TraceRec> recs;
    std::vector<cudaEvent_t> spare;
};
Trace &trace();   // defined in snlm_api.cu

inline cudaEvent_t trace_event(Trace &t)
{
    if (!t.spare.empty()) {
        cudaEvent_t e = t.spare.back();
        t.spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets one launch with an NVTX range named after its kind (so that profilers
// can select a pass, e.g. ncu --nvtx --nvtx-include "row_pass_sure/block/") and,
// when tracing is on, with events on its stream.
struct TraceScope {
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    bool active = false;
    TraceScope(int k, cudaStream_t s) : kind(k), st(s)
    {
        nvtxRangePushA(snlm_kernel_name(k));
        Trace &t = trace();
        std::lock_guard<std::mutex> g(t.mu);
        if (!t.on)
            return;
        a = trace_event(t);
        b = trace_event(t);
        if (a && b && cudaEventRecord(a, st) == cudaSuccess)
            active = true;
    }
    ~TraceScope()
    {
        nvtxRangePop();
        if (!active)
            return;
        Trace &t = trace();
        std::lock_guard<std::mutex> g(t.mu);
        if (cudaEventRecord(b, st) == cudaSuccess)
            t.recs.push_back({kind, a, b});
    }
};

}  // namespace snlm
