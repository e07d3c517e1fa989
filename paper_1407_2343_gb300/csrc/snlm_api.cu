// C ABI of libsnlm (declared in include/snlm.h): argument validation, scratch
// management and the order of passes of Alg. 4 (Sec. III).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/snlm.h"
#include "snlm_host.h"
#include "snlm_internal.h"
#include "snlm_sure_impl.cuh"

using namespace snlm;

namespace snlm {
Trace &trace()
{
    static Trace t;
    return t;
}
}  // namespace snlm

namespace {

// ------------------------------------------------------------------ helpers

cudaError_t dispatch_pass(int K, const PassArgs &a, int dm, bool sure, cudaStream_t st)
{
    switch (K) {
    case 0: return launch_pass<0>(a, dm, sure, st);
    case 1: return launch_pass<1>(a, dm, sure, st);
    case 2: return launch_pass<2>(a, dm, sure, st);
    case 3: return launch_pass<3>(a, dm, sure, st);
    case 4: return launch_pass<4>(a, dm, sure, st);
    case 5: return launch_pass<5>(a, dm, sure, st);
    case 6: return launch_pass<6>(a, dm, sure, st);
    case 7: return launch_pass<7>(a, dm, sure, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_dist(int K, const DistArgs &a, int dm, cudaStream_t st)
{
    switch (K) {
    case 0: return launch_dist<0>(a, dm, st);
    case 1: return launch_dist<1>(a, dm, st);
    case 2: return launch_dist<2>(a, dm, st);
    case 3: return launch_dist<3>(a, dm, st);
    case 4: return launch_dist<4>(a, dm, st);
    case 5: return launch_dist<5>(a, dm, st);
    case 6: return launch_dist<6>(a, dm, st);
    case 7: return launch_dist<7>(a, dm, st);
    default: return cudaErrorInvalidValue;
    }
}

struct WsLayout {
    size_t tmp, frc, delta, part_rc, part_cr, solve, info, total;
    long long n_part_rc, n_part_cr;
};

// Scratch of one denoise call: the intermediate image of the first pass, f_rc
// (AVG/SURE), the chained derivative (SURE), partial sums (SURE) and info.
WsLayout ws_layout(int H, int W, int S, int order)
{
    WsLayout L;
    const size_t img = align_up((size_t)H * W * sizeof(float), 256);
    size_t off = 0;
    L.tmp = off;
    off += img;
    L.frc = off;
    if (order == SNLM_AVG || order == SNLM_SURE)
        off += img;
    L.delta = off;
    if (order == SNLM_SURE)
        off += img;
    // column pass (RC's second pass) runs over W lines of length H; the row pass
    // over H lines of length W. Size for the worst case S (smallest tiles).
    const int Sw = S < 0 ? kMaxS : S;
    L.n_part_rc = pass_ctas(W, H, Sw);
    L.n_part_cr = pass_ctas(H, W, Sw);
    L.part_rc = off;
    if (order == SNLM_SURE)
        off += align_up((size_t)L.n_part_rc * kPartials * sizeof(double), 256);
    L.part_cr = off;
    if (order == SNLM_SURE)
        off += align_up((size_t)L.n_part_cr * kPartials * sizeof(double), 256);
    L.solve = off;
    if (order == SNLM_SURE)
        off += align_up((size_t)2 * kSolveScratchRecords * kPartials * sizeof(double), 256);
    L.info = off;
    off += 256;
    L.total = off;
    return L;
}


// Per-device scratch pool for the calls that do not take a workspace.
struct Pool {
    std::mutex mu;
    std::vector<void *> ptr;
    std::vector<size_t> bytes;
};
Pool &pool()
{
    static Pool p;
    return p;
}

// Returns scratch of at least `need` bytes on the current device, slot `slot`
// (0: denoise scratch, 1 and 3: host-call inputs, 2 and 4: host-call outputs,
// 5: the output of Alg. 4 before the bilateral post-filter, 6 and 7: the volumes of
// the 3-D extension).
constexpr int kPoolSlots = 8;
void *pool_get(size_t need, int slot)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return nullptr;
    Pool &p = pool();
    std::lock_guard<std::mutex> g(p.mu);
    const size_t idx = (size_t)dev * kPoolSlots + slot;
    if (p.ptr.size() <= idx) {
        p.ptr.resize(idx + 1, nullptr);
        p.bytes.resize(idx + 1, 0);
    }
    if (p.bytes[idx] >= need)
        return p.ptr[idx];
    if (p.ptr[idx]) {
        cudaDeviceSynchronize();
        cudaFree(p.ptr[idx]);
        p.ptr[idx] = nullptr;
        p.bytes[idx] = 0;
    }
    void *q = nullptr;
    if (cudaMalloc(&q, need) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    p.ptr[idx] = q;
    p.bytes[idx] = need;
    return q;
}

// One pass along rows (axis 0) or columns (axis 1) of an H x W image.
struct Pass {
    Lines src;
    float *dst;
    const float *blend = nullptr;
    const float *delta_in = nullptr;
    float *delta_out = nullptr;
    double *partials = nullptr;
    Lines aux_f{nullptr, DT_F32, 0, 0};
    Lines aux_rc{nullptr, DT_F32, 0, 0};
};

cudaError_t run_pass(int axis, int H, int W, const Pass &ps, int S, int K, double h, int profile,
                     double beta, bool sure, cudaStream_t st, int sum_lo = 0, int sum_hi = 0)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.src = ps.src;
    a.n_lines = axis == 0 ? H : W;
    a.N = axis == 0 ? W : H;
    a.S = S;
    a.c2 = exp2_scale(h);
    a.h2 = (float)(h * h);
    fill_profile(a.g, K, profile, beta);
    a.dst = ps.dst;
    a.out_line_step = axis == 0 ? W : 1;
    a.out_elem_step = axis == 0 ? 1 : W;
    a.blend = ps.blend;
    a.delta_in = ps.delta_in;
    a.delta_out = ps.delta_out;
    a.partials = ps.partials;
    a.aux_f = ps.aux_f;
    a.aux_rc = ps.aux_rc;
    a.sum_lo = sum_lo;
    a.sum_hi = sum_hi;
    finish_pass_args(a);
    const int dm = dist_mode_for(ps.src.dtype, profile);
    if (dm == DIST_IIR) {
        TraceScope ts((axis == 0 ? SNLM_K_ROW_PASS : SNLM_K_COL_PASS) | (dm << 8), st);
        return run_iir_pass(a.src, a.n_lines, a.N, S, h, beta, a.dst, a.out_line_step, a.out_elem_step, a.blend,
                            st);
    }
    TmaPass t;
    int grid = 0;
    const bool tma = plan_pass_tma(K, a, dm, sure, &t, &grid);
    TraceScope ts(((axis == 0 ? SNLM_K_ROW_PASS : SNLM_K_COL_PASS) + (sure ? 2 : 0)) | (dm << 8) |
                      (tma ? kTraceTma : 0),
                  st);
    return tma ? launch_planned_tma(K, a, t, dm, sure, grid, st) : dispatch_pass(K, a, dm, sure, st);
}

// The four passes of Alg. 4 with the chained divergences: rows then columns into
// frc (delta_1), columns then rows into fcr (delta_2), with the partial sums of
// the SURE system restricted to image rows [row0, row1) (row1 == 0: all rows).
// *n_rc and *n_cr receive the number of partial records of each order.
cudaError_t run_sure_passes(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h,
                            int profile, double bt, float *frc, float *fcr, const WsLayout &L, char *base,
                            int row0, int row1, cudaStream_t st, int *n_rc, int *n_cr)
{
    float *tmp = reinterpret_cast<float *>(base + L.tmp);
    float *delta = reinterpret_cast<float *>(base + L.delta);
    double *part_rc = reinterpret_cast<double *>(base + L.part_rc);
    double *part_cr = reinterpret_cast<double *>(base + L.part_cr);
    const Lines tmp_rows{tmp, DT_F32, (long long)W, 1};
    const Lines tmp_cols{tmp, DT_F32, 1, (long long)W};
    cudaError_t e;
    if (profile == SNLM_GAUSS_IIR) {
        // The recursive profile's passes form no partial records: each keeps its
        // chained derivative in `delta` (in place), and the sums are taken over the
        // images after the second and the fourth pass.
        const int r0 = row1 == 0 ? 0 : row0, r1 = row1 == 0 ? H : row1;
        *n_rc = (int)std::min<long long>(L.n_part_rc, 1024);
        *n_cr = (int)std::min<long long>(L.n_part_cr, 1024);
        const Lines rows = image_lines(img, dtype, pitch, 0), cols = image_lines(img, dtype, pitch, 1);
        {
            TraceScope ts(SNLM_K_ROW_PASS_SURE | (DIST_IIR << 8), st);
            if ((e = run_iir_pass_sure(rows, H, W, S, h, bt, tmp, W, 1, nullptr, delta, st)) != cudaSuccess)
                return e;
        }
        {
            TraceScope ts(SNLM_K_COL_PASS_SURE | (DIST_IIR << 8), st);
            if ((e = run_iir_pass_sure(tmp_cols, W, H, S, h, bt, frc, 1, W, delta, delta, st)) != cudaSuccess)
                return e;
        }
        {
            TraceScope ts(SNLM_K_SURE_SOLVE, st);
            if ((e = launch_image_sums(nullptr, nullptr, rows, W, r0, r1, delta, part_rc, *n_rc, st)) != cudaSuccess)
                return e;
        }
        {
            TraceScope ts(SNLM_K_COL_PASS_SURE | (DIST_IIR << 8), st);
            if ((e = run_iir_pass_sure(cols, W, H, S, h, bt, tmp, 1, W, nullptr, delta, st)) != cudaSuccess)
                return e;
        }
        {
            TraceScope ts(SNLM_K_ROW_PASS_SURE | (DIST_IIR << 8), st);
            if ((e = run_iir_pass_sure(tmp_rows, H, W, S, h, bt, fcr, W, 1, delta, delta, st)) != cudaSuccess)
                return e;
        }
        TraceScope ts(SNLM_K_SURE_SOLVE, st);
        return launch_image_sums(frc, fcr, rows, W, r0, r1, delta, part_cr, *n_cr, st);
    }
    *n_rc = (int)pass_ctas(W, H, S);
    *n_cr = (int)pass_ctas(H, W, S);
    Pass p1{image_lines(img, dtype, pitch, 0), tmp};
    p1.delta_out = delta;
    if ((e = run_pass(0, H, W, p1, S, K, h, profile, bt, true, st, 0, 0)) != cudaSuccess)
        return e;
    Pass p2{tmp_cols, frc};
    p2.delta_in = delta;
    p2.partials = part_rc;
    if ((e = run_pass(1, H, W, p2, S, K, h, profile, bt, true, st, row0, row1)) != cudaSuccess)
        return e;
    Pass p3{image_lines(img, dtype, pitch, 1), tmp};
    p3.delta_out = delta;
    if ((e = run_pass(1, H, W, p3, S, K, h, profile, bt, true, st, 0, 0)) != cudaSuccess)
        return e;
    Pass p4{tmp_rows, fcr};
    p4.delta_in = delta;
    p4.partials = part_cr;
    p4.aux_f = image_lines(img, dtype, pitch, 0);
    p4.aux_rc = Lines{frc, DT_F32, (long long)W, 1};
    return run_pass(0, H, W, p4, S, K, h, profile, bt, true, st, row0, row1);
}

int denoise_core(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h,
                 int profile, int order, float sigma, float beta, float *out, void *ws,
                 double *info, cudaStream_t st)
{
    const WsLayout L = ws_layout(H, W, S, order);
    char *base = static_cast<char *>(ws);
    float *tmp = reinterpret_cast<float *>(base + L.tmp);
    float *frc = reinterpret_cast<float *>(base + L.frc);
    double *part_rc = reinterpret_cast<double *>(base + L.part_rc);
    double *part_cr = reinterpret_cast<double *>(base + L.part_cr);
    double *winfo = reinterpret_cast<double *>(base + L.info);
    double *wsolve = reinterpret_cast<double *>(base + L.solve);
    const double bt = beta_or_default(beta, K);
    cudaError_t e = cudaSuccess;
#define SNLM_TRY(x)            \
    do {                       \
        e = (x);               \
        if (e != cudaSuccess)  \
            return status_of(e); \
    } while (0)

    const Lines tmp_rows{tmp, DT_F32, (long long)W, 1};
    const Lines tmp_cols{tmp, DT_F32, 1, (long long)W};
    if (order == SNLM_RC) {
        Pass p1{image_lines(img, dtype, pitch, 0), tmp};
        SNLM_TRY(run_pass(0, H, W, p1, S, K, h, profile, bt, false, st));
        Pass p2{tmp_cols, out};
        SNLM_TRY(run_pass(1, H, W, p2, S, K, h, profile, bt, false, st));
        TraceScope ts(SNLM_K_SET_THETA, st);
        SNLM_TRY(launch_set_theta(winfo, 1.0, 0.0, st));
    } else if (order == SNLM_CR) {
        Pass p1{image_lines(img, dtype, pitch, 1), tmp};
        SNLM_TRY(run_pass(1, H, W, p1, S, K, h, profile, bt, false, st));
        Pass p2{tmp_rows, out};
        SNLM_TRY(run_pass(0, H, W, p2, S, K, h, profile, bt, false, st));
        TraceScope ts(SNLM_K_SET_THETA, st);
        SNLM_TRY(launch_set_theta(winfo, 0.0, 1.0, st));
    } else if (order == SNLM_AVG) {
        Pass p1{image_lines(img, dtype, pitch, 0), tmp};
        SNLM_TRY(run_pass(0, H, W, p1, S, K, h, profile, bt, false, st));
        Pass p2{tmp_cols, frc};
        SNLM_TRY(run_pass(1, H, W, p2, S, K, h, profile, bt, false, st));
        Pass p3{image_lines(img, dtype, pitch, 1), tmp};
        SNLM_TRY(run_pass(1, H, W, p3, S, K, h, profile, bt, false, st));
        Pass p4{tmp_rows, out};
        p4.blend = frc;
        SNLM_TRY(run_pass(0, H, W, p4, S, K, h, profile, bt, false, st));
        TraceScope ts(SNLM_K_SET_THETA, st);
        SNLM_TRY(launch_set_theta(winfo, 0.5, 0.5, st));
    } else {
        // Alg. 4: rows then columns with delta_1, columns then rows with delta_2
        int n_rc = 0, n_cr = 0;
        SNLM_TRY(run_sure_passes(img, dtype, H, W, pitch, S, K, h, profile, bt, frc, out, L, base, 0, 0, st, &n_rc,
                                 &n_cr));
        {
            TraceScope ts(SNLM_K_SURE_SOLVE, st);
            // the reduction's ticket word sits in the info area's spare tail (info uses 10
            // of its 32 doubles)
            unsigned *ticket = reinterpret_cast<unsigned *>(winfo + 16);
            SNLM_TRY(launch_sure_solve(part_rc, n_rc, part_cr, n_cr, (double)sigma * sigma, winfo, wsolve, ticket,
                                       st));
        }
        {
            TraceScope ts(SNLM_K_COMBINE, st);
            SNLM_TRY(launch_combine(frc, out, winfo, (long long)H * W, st));
        }
    }
    if (info)
        SNLM_TRY(cudaMemcpyAsync(info, winfo, 10 * sizeof(double), cudaMemcpyDeviceToDevice, st));
#undef SNLM_TRY
    return SNLM_OK;
}

}  // namespace

extern "C" {

const char *snlm_status_str(int status)
{
    switch (status) {
    case SNLM_OK: return "SNLM_OK";
    case SNLM_ERR_ARG: return "SNLM_ERR_ARG: invalid argument";
    case SNLM_ERR_CUDA: return "SNLM_ERR_CUDA: a CUDA call failed";
    case SNLM_ERR_NOMEM: return "SNLM_ERR_NOMEM: out of memory";
    case SNLM_ERR_TIMEOUT: return "SNLM_ERR_TIMEOUT: a bounded device wait gave up";
    case SNLM_ERR_UNSUPPORTED: return "SNLM_ERR_UNSUPPORTED: configuration not compiled";
    case SNLM_ERR_CHECK: return "SNLM_ERR_CHECK: a shared-memory guard was overwritten (checked build)";
    default: return "SNLM: unknown status";
    }
}

int snlm_version(void) { return 100; }

int snlm_preload(int *n_loaded)
{
    const int n = preload_pass<0>() + preload_pass<1>() + preload_pass<2>() + preload_pass<3>() +
                  preload_pass<4>() + preload_pass<5>() + preload_pass<6>() + preload_pass<7>() +
                  preload_pass_tma<0>() + preload_pass_tma<1>() + preload_pass_tma<2>() + preload_pass_tma<3>() +
                  preload_pass_tma<4>() + preload_pass_tma<5>() + preload_pass_tma<6>() + preload_pass_tma<7>() +
                  preload_batch() + preload_iir() + preload_sure() + preload_bilateral() + preload_nlm2d() +
                  preload_3d();
    if (n_loaded)
        *n_loaded = n;
    return n == SNLM_KERNEL_COUNT ? SNLM_OK : SNLM_ERR_CUDA;
}

float snlm_default_h(float sigma, int K, int profile, float beta)
{
    if (!(sigma >= 0.f) || K < 0 || K > 64)
        return -1.f;
    const double bt = beta_or_default(beta, K);
    if (profile == SNLM_GAUSS_IIR)   // unit DC gain times beta sqrt(2 pi)
        return iir_check_beta(bt) == SNLM_OK ? (float)(sigma * sqrt(bt * sqrt(2.0 * 3.14159265358979323846)))
                                             : -1.f;
    if (profile != SNLM_BOX && profile != SNLM_GAUSS)
        return -1.f;
    double s = 0.0;
    for (int k = -K; k <= K; ++k)
        s += profile == SNLM_GAUSS ? exp(-(double)k * k / (2.0 * bt * bt)) : 1.0;
    return (float)(sigma * sqrt(s));
}

size_t snlm_workspace_bytes(int H, int W, int order)
{
    if (H < 1 || W < 1 || (long long)H * W >= (1LL << 31) || order < SNLM_RC || order > SNLM_SURE)
        return 0;
    return ws_layout(H, W, -1, order).total;
}

int snlm_denoise_ws(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h,
                    int profile, int order, float sigma, float beta, float *out, void *workspace,
                    size_t workspace_bytes, double *info, void *stream)
{
    int rc = check_denoise(H, W, S, K, h, profile, order, sigma, beta);
    if (rc != SNLM_OK)
        return rc;
    if (!valid_dtype(dtype) || pitch < W || (long long)H * pitch >= (1LL << 31))
        return SNLM_ERR_ARG;
    if (!is_device_ptr(img) || !is_device_ptr(out) || !is_device_ptr(workspace))
        return SNLM_ERR_ARG;
    if (info && !is_device_ptr(info))
        return SNLM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & 15) != 0)
        return SNLM_ERR_ARG;
    if (workspace_bytes < ws_layout(H, W, S, order).total)
        return SNLM_ERR_ARG;
    return denoise_core(img, dtype, H, W, pitch, S, K, h, profile, order, sigma, beta, out, workspace,
                        info, static_cast<cudaStream_t>(stream));
}

int snlm_sure_band(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h, int profile,
                   float beta, int row0, int row1, float *f_rc, float *f_cr, double *sums, void *workspace,
                   size_t workspace_bytes, void *stream)
{
    int rc = check_denoise(H, W, S, K, h, profile, SNLM_SURE, 0.f, beta);
    if (rc != SNLM_OK)
        return rc;
    if (!valid_dtype(dtype) || pitch < W || (long long)H * pitch >= (1LL << 31))
        return SNLM_ERR_ARG;
    if (row0 < 0 || row1 <= row0 || row1 > H)
        return SNLM_ERR_ARG;
    if (!is_device_ptr(img) || !is_device_ptr(f_rc) || !is_device_ptr(f_cr) || !is_device_ptr(sums) ||
        !is_device_ptr(workspace) || f_rc == f_cr)
        return SNLM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & 15) != 0 || (reinterpret_cast<uintptr_t>(sums) & 7) != 0)
        return SNLM_ERR_ARG;
    const WsLayout L = ws_layout(H, W, S, SNLM_SURE);
    if (workspace_bytes < L.total)
        return SNLM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(workspace);
    const double bt = beta_or_default(beta, K);
    int n_rc = 0, n_cr = 0;
    cudaError_t e = run_sure_passes(img, dtype, H, W, pitch, S, K, h, profile, bt, f_rc, f_cr, L, base, row0, row1,
                                    st, &n_rc, &n_cr);
    if (e != cudaSuccess)
        return status_of(e);
    TraceScope ts(SNLM_K_SURE_SOLVE, st);
    e = launch_sure_sums(reinterpret_cast<double *>(base + L.part_rc), n_rc,
                         reinterpret_cast<double *>(base + L.part_cr), n_cr, sums,
                         reinterpret_cast<double *>(base + L.solve), st);
    return status_of(e);
}

int snlm_sure_theta(const double *sums, float sigma, double *theta)
{
    if (!sums || !theta || !(sigma >= 0.f) || !std::isfinite(sigma))
        return SNLM_ERR_ARG;
    for (int k = 0; k < 7; ++k)
        if (!std::isfinite(sums[k]))
            return SNLM_ERR_ARG;
    sure_theta(sums, (double)sigma * sigma, &theta[0], &theta[1]);
    return SNLM_OK;
}

int snlm_sure_combine(const float *f_rc, const float *f_cr, long long n, double theta1, double theta2, float *out,
                      void *stream)
{
    if (n < 0 || !std::isfinite(theta1) || !std::isfinite(theta2))
        return SNLM_ERR_ARG;
    if (n == 0)
        return SNLM_OK;
    if (!is_device_ptr(f_rc) || !is_device_ptr(f_cr) || !is_device_ptr(out))
        return SNLM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TraceScope ts(SNLM_K_COMBINE, st);
    return status_of(launch_combine_theta(f_rc, f_cr, out, n, theta1, theta2, st));
}

int snlm_denoise(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h,
                 int profile, int order, float sigma, float beta, float *out, void *stream)
{
    int rc = check_denoise(H, W, S, K, h, profile, order, sigma, beta);
    if (rc != SNLM_OK)
        return rc;
    if (!valid_dtype(dtype) || pitch < W || (long long)H * pitch >= (1LL << 31))
        return SNLM_ERR_ARG;
    if (!is_device_ptr(img) || !is_device_ptr(out))
        return SNLM_ERR_ARG;
    const size_t need = ws_layout(H, W, S, order).total;
    void *ws = pool_get(need, 0);
    if (!ws)
        return SNLM_ERR_NOMEM;
    return denoise_core(img, dtype, H, W, pitch, S, K, h, profile, order, sigma, beta, out, ws, nullptr,
                        static_cast<cudaStream_t>(stream));
}

int snlm_denoise_bf(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h, int profile,
                    int order, float sigma, float beta, float sigma_s, float sigma_r, float *out, void *stream)
{
    if (!(sigma_s > 0.f) || !(sigma_r > 0.f)) {
        if (snlm_bf_params(sigma, &sigma_s, &sigma_r) != SNLM_OK || !(sigma_r > 0.f) || !(sigma_s > 0.f))
            return SNLM_ERR_ARG;
    }
    int rc = check_denoise(H, W, S, K, h, profile, order, sigma, beta);
    if (rc != SNLM_OK)
        return rc;
    if (!valid_dtype(dtype) || pitch < W || (long long)H * pitch >= (1LL << 31) || !is_device_ptr(img))
        return SNLM_ERR_ARG;
    if (!std::isfinite(sigma_s) || !std::isfinite(sigma_r) || !is_device_ptr(out))
        return SNLM_ERR_ARG;
    if (bilateral_radius(sigma_s) > kBfMaxR)
        return SNLM_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *mid = static_cast<float *>(pool_get((size_t)H * W * sizeof(float), 5));
    void *ws = pool_get(ws_layout(H, W, S, order).total, 0);
    if (!mid || !ws)
        return SNLM_ERR_NOMEM;
    rc = denoise_core(img, dtype, H, W, pitch, S, K, h, profile, order, sigma, beta, mid, ws, nullptr, st);
    if (rc != SNLM_OK)
        return rc;
    return run_bilateral(mid, H, W, W, sigma_s, sigma_r, out, W, st);
}

int snlm_denoise_host(const void *img_host, int dtype, int H, int W, int pitch, int S, int K,
                      float h, int profile, int order, float sigma, float beta, float *out_host,
                      void *stream)
{
    int rc = check_denoise(H, W, S, K, h, profile, order, sigma, beta);
    if (rc != SNLM_OK)
        return rc;
    if (!valid_dtype(dtype) || pitch < W || (long long)H * pitch >= (1LL << 31) || !img_host || !out_host)
        return SNLM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t in_bytes = (size_t)H * pitch * dtype_size(dtype);
    const size_t out_bytes = (size_t)H * W * sizeof(float);
    void *din = pool_get(in_bytes, 1);
    void *dout = pool_get(out_bytes, 2);
    void *ws = pool_get(ws_layout(H, W, S, order).total, 0);
    if (!din || !dout || !ws)
        return SNLM_ERR_NOMEM;
    cudaError_t e = cudaMemcpyAsync(din, img_host, in_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return status_of(e);
    rc = denoise_core(din, dtype, H, W, pitch, S, K, h, profile, order, sigma, beta,
                      static_cast<float *>(dout), ws, nullptr, st);
    if (rc != SNLM_OK)
        return rc;
    e = cudaMemcpyAsync(out_host, dout, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess)
        return status_of(e);
    rc = status_of(cudaStreamSynchronize(st));
    if (rc != SNLM_OK)
        return rc;
    return snlm_device_error(st);
}

int snlm_denoise_host_many(const void *const *imgs_host, float *const *outs_host, int n, int dtype, int H,
                           int W, int pitch, int S, int K, float h, int profile, int order, float sigma,
                           float beta, void *stream)
{
    int rc = check_denoise(H, W, S, K, h, profile, order, sigma, beta);
    if (rc != SNLM_OK)
        return rc;
    if (n < 0 || (n > 0 && (!imgs_host || !outs_host)) || !valid_dtype(dtype) || pitch < W ||
        (long long)H * pitch >= (1LL << 31))
        return SNLM_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!imgs_host[i] || !outs_host[i])
            return SNLM_ERR_ARG;
    if (n == 0)
        return SNLM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t in_bytes = (size_t)H * pitch * dtype_size(dtype);
    const size_t out_bytes = (size_t)H * W * sizeof(float);
    void *din[2] = {pool_get(in_bytes, 1), pool_get(in_bytes, 3)};
    void *dout[2] = {pool_get(out_bytes, 2), pool_get(out_bytes, 4)};
    void *ws = pool_get(ws_layout(H, W, S, order).total, 0);
    if (!din[0] || !din[1] || !dout[0] || !dout[1] || !ws)
        return SNLM_ERR_NOMEM;
    // copies in on `cin`, computation on `st`, copies out on `cout`; buffer b = i & 1
    // is reused by image i + 2 once image i's computation (input) and copy out
    // (output) are done. Every wait names the latest record of its event.
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t in_done[2] = {}, comp_done[2] = {}, out_done[2] = {};
    cudaError_t e = cudaStreamCreateWithFlags(&cin, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&cout, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&in_done[b], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&comp_done[b], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&out_done[b], cudaEventDisableTiming);
    }
    rc = status_of(e);
    for (int i = 0; i < n && rc == SNLM_OK; ++i) {
        const int b = i & 1;
        if (i >= 2)
            e = cudaStreamWaitEvent(cin, comp_done[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(din[b], imgs_host[i], in_bytes, cudaMemcpyHostToDevice, cin);
        if (e == cudaSuccess)
            e = cudaEventRecord(in_done[b], cin);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(st, in_done[b], 0);
        if (e == cudaSuccess && i >= 2)
            e = cudaStreamWaitEvent(st, out_done[b], 0);
        rc = status_of(e);
        if (rc != SNLM_OK)
            break;
        rc = denoise_core(din[b], dtype, H, W, pitch, S, K, h, profile, order, sigma, beta,
                          static_cast<float *>(dout[b]), ws, nullptr, st);
        if (rc != SNLM_OK)
            break;
        e = cudaEventRecord(comp_done[b], st);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(cout, comp_done[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(outs_host[i], dout[b], out_bytes, cudaMemcpyDeviceToHost, cout);
        if (e == cudaSuccess)
            e = cudaEventRecord(out_done[b], cout);
        rc = status_of(e);
    }
    // drain all three streams whatever happened, then release the call's objects
    const int r1 = cin ? status_of(cudaStreamSynchronize(cin)) : SNLM_OK;
    const int r2 = status_of(cudaStreamSynchronize(st));
    const int r3 = cout ? status_of(cudaStreamSynchronize(cout)) : SNLM_OK;
    for (int b = 0; b < 2; ++b) {
        if (in_done[b])
            cudaEventDestroy(in_done[b]);
        if (comp_done[b])
            cudaEventDestroy(comp_done[b]);
        if (out_done[b])
            cudaEventDestroy(out_done[b]);
    }
    if (cin)
        cudaStreamDestroy(cin);
    if (cout)
        cudaStreamDestroy(cout);
    if (rc == SNLM_OK)
        rc = r1 != SNLM_OK ? r1 : (r2 != SNLM_OK ? r2 : r3);
    if (rc != SNLM_OK)
        return rc;
    return snlm_device_error(st);
}

// One 1-D pass of the 3-D extension along `axis` (0: x, 1: y, 2: z) of a D x H x W
// volume; dst has src's layout. Along x both orders of the volume, (z, y, x) and
// (y, z, x), have lines of one stride; y needs the order (y, z, x) and z (z, y, x).
static int pass_3d(const void *src, int dtype, float *dst, int D, int H, int W, int axis, int S, int K, float h,
                   int profile, float beta, cudaStream_t st)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    long long ls, es;
    int n, N;
    if (axis == 0) {
        n = D * H, N = W, ls = W, es = 1;
    } else if (axis == 1) {
        n = D * W, N = H, ls = 1, es = (long long)D * W;       // order (y, z, x)
    } else {
        n = H * W, N = D, ls = 1, es = (long long)H * W;       // order (z, y, x)
    }
    a.src = Lines{src, dtype, ls, es};
    a.n_lines = n;
    a.N = N;
    a.S = S;
    a.c2 = exp2_scale(h);
    a.h2 = (float)((double)h * h);
    fill_profile(a.g, K, profile, beta_or_default(beta, K));
    a.dst = dst;
    a.out_line_step = ls;
    a.out_elem_step = es;
    a.aux_f = Lines{nullptr, DT_F32, 0, 0};
    a.aux_rc = Lines{nullptr, DT_F32, 0, 0};
    finish_pass_args(a);
    const int dm = dist_mode_for(dtype, profile);
    TraceScope ts(SNLM_K_LINE_PASS_3D | (dm << 8), st);
    return status_of(dispatch_pass(K, a, dm, false, st));
}

int snlm_denoise_3d(const void *vol, int dtype, int D, int H, int W, int S, int K, float h, int profile,
                    float beta, int order3, float *out, void *stream)
{
    if (D < 1 || H < 1 || W < 1 || (long long)D * H * W >= (1LL << 31))
        return SNLM_ERR_ARG;
    if (profile == SNLM_GAUSS_IIR)
        return SNLM_ERR_UNSUPPORTED;
    if (S < 0 || S > kMaxS || K < 0 || !valid_dtype(dtype) || (profile != SNLM_BOX && profile != SNLM_GAUSS))
        return SNLM_ERR_ARG;
    if (!(h > 0.f) || !std::isfinite(h) || (order3 != SNLM3_XYZ && order3 != SNLM3_AVG6))
        return SNLM_ERR_ARG;
    if (K > kMaxK)
        return SNLM_ERR_UNSUPPORTED;
    if (!is_device_ptr(vol) || !is_device_ptr(out))
        return SNLM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n = (long long)D * H * W;
    float *buf[2] = {static_cast<float *>(pool_get((size_t)n * sizeof(float), 6)),
                     static_cast<float *>(pool_get((size_t)n * sizeof(float), 7))};
    if (!buf[0] || !buf[1])
        return SNLM_ERR_NOMEM;
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int n_orders = order3 == SNLM3_XYZ ? 1 : 6;
    for (int o = 0; o < n_orders; ++o) {
        // the samples in hand: the input itself (order (z, y, x), its own type) or a
        // float32 volume in one of the two buffers
        const void *cur = vol;
        int cur_dt = dtype, lay = 0, cur_buf = -1;
        auto next_buf = [&]() { return cur_buf == 0 ? 1 : 0; };
        auto relayout = [&](int to) -> int {
            const int b = next_buf();
            // order 0 = D x H rows, order 1 = H x D rows (rows of W samples)
            const cudaError_t e = to == 1 ? launch_swap_outer(cur, cur_dt, buf[b], H, D, W, st)
                                          : launch_swap_outer(cur, cur_dt, buf[b], D, H, W, st);
            cur = buf[b], cur_dt = DT_F32, lay = to, cur_buf = b;
            return status_of(e);
        };
        for (int k = 0; k < 3; ++k) {
            const int axis = perms[order3 == SNLM3_XYZ ? 0 : o][k];
            int rc = SNLM_OK;
            if (axis == 1 && lay != 1) {
                TraceScope ts(SNLM_K_RELAYOUT_3D, st);
                rc = relayout(1);
            } else if (axis == 2 && lay != 0) {
                TraceScope ts(SNLM_K_RELAYOUT_3D, st);
                rc = relayout(0);
            }
            if (rc != SNLM_OK)
                return rc;
            // the last pass of the single order in order (z, y, x) writes the result
            const bool last = k == 2 && n_orders == 1 && lay == 0;
            const int b = next_buf();
            float *dst = last ? out : buf[b];
            rc = pass_3d(cur, cur_dt, dst, D, H, W, axis, S, K, h, profile, beta, st);
            if (rc != SNLM_OK)
                return rc;
            if (last)
                return SNLM_OK;
            cur = dst, cur_dt = DT_F32, cur_buf = b;
        }
        if (lay == 1) {
            TraceScope ts(SNLM_K_RELAYOUT_3D, st);
            const int rc = n_orders == 1 ? status_of(launch_swap_outer(cur, DT_F32, out, D, H, W, st)) : relayout(0);
            if (rc != SNLM_OK)
                return rc;
            if (n_orders == 1)
                return SNLM_OK;
        }
        TraceScope ts(SNLM_K_RELAYOUT_3D, st);
        const int rc = status_of(launch_axpby(static_cast<const float *>(cur), out, 1.f / 6.f, o == 0 ? 0.f : 1.f,
                                              n, st));
        if (rc != SNLM_OK)
            return rc;
    }
    return SNLM_OK;
}

int snlm_nlm_1d(const void *x, int dtype, int n_lines, int N, long long line_step,
                long long elem_step, int S, int K, float h, int profile, float beta, float *fhat,
                long long out_line_step, long long out_elem_step, const float *delta_in,
                float *delta_out, void *stream)
{
    if (n_lines < 1 || N < 1 || (long long)n_lines * N >= (1LL << 31) || S < 0 || S > kMaxS || K < 0)
        return SNLM_ERR_ARG;
    if (K > kMaxK)
        return SNLM_ERR_UNSUPPORTED;
    if (!valid_dtype(dtype) || !(h > 0.f) || !isfinite(h) ||
        (profile != SNLM_BOX && profile != SNLM_GAUSS && profile != SNLM_GAUSS_IIR))
        return SNLM_ERR_ARG;
    if (profile == SNLM_GAUSS_IIR && (delta_in || delta_out))
        return SNLM_ERR_UNSUPPORTED;
    if (profile == SNLM_GAUSS_IIR && iir_check_beta(beta_or_default(beta, K)) != SNLM_OK)
        return SNLM_ERR_ARG;
    if (!is_device_ptr(x) || !is_device_ptr(fhat))
        return SNLM_ERR_ARG;
    if ((delta_in && !is_device_ptr(delta_in)) || (delta_out && !is_device_ptr(delta_out)))
        return SNLM_ERR_ARG;
    // strides are positive and every element offset fits in 31 bits
    if (line_step < 1 || elem_step < 1 || out_line_step < 1 || out_elem_step < 1)
        return SNLM_ERR_ARG;
    if ((n_lines - 1) * line_step + (long long)(N - 1) * elem_step >= (1LL << 31) ||
        (n_lines - 1) * out_line_step + (long long)(N - 1) * out_elem_step >= (1LL << 31))
        return SNLM_ERR_ARG;
    const bool sure = delta_out != nullptr;
    if (sure) {
        const double h2 = (double)h * h;
        if (!(h2 > 1e-30 && h2 < 1e30))
            return SNLM_ERR_ARG;
    }
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.src = Lines{x, dtype, line_step, elem_step};
    a.n_lines = n_lines;
    a.N = N;
    a.S = S;
    a.c2 = exp2_scale(h);
    a.h2 = (float)((double)h * h);
    fill_profile(a.g, K, profile, beta_or_default(beta, K));
    a.dst = fhat;
    a.out_line_step = out_line_step;
    a.out_elem_step = out_elem_step;
    a.delta_in = delta_in;
    a.delta_out = delta_out;
    a.aux_f = Lines{nullptr, DT_F32, 0, 0};
    a.aux_rc = Lines{nullptr, DT_F32, 0, 0};
    finish_pass_args(a);
    const int dm = dist_mode_for(dtype, profile);
    TraceScope ts(SNLM_K_LINE_PASS | (dm << 8), static_cast<cudaStream_t>(stream));
    if (dm == DIST_IIR)
        return status_of(run_iir_pass(a.src, n_lines, N, S, h, beta_or_default(beta, K), fhat, out_line_step,
                                      out_elem_step, nullptr, static_cast<cudaStream_t>(stream)));
    return status_of(dispatch_pass(K, a, dm, sure, static_cast<cudaStream_t>(stream)));
}

int snlm_patch_dist_1d(const void *x, int dtype, int n_lines, int N, int stride, int S, int K,
                       int profile, float beta, void *out, void *stream)
{
    if (n_lines < 1 || N < 1 || stride < N || S < 0 || S > kMaxS || K < 0)
        return SNLM_ERR_ARG;
    if ((long long)n_lines * stride >= (1LL << 31))
        return SNLM_ERR_ARG;
    if ((long long)n_lines * N * (2LL * S + 1) >= (1LL << 40))
        return SNLM_ERR_ARG;
    if (K > kMaxK)
        return SNLM_ERR_UNSUPPORTED;
    if (!valid_dtype(dtype) || (profile != SNLM_BOX && profile != SNLM_GAUSS && profile != SNLM_GAUSS_IIR))
        return SNLM_ERR_ARG;
    if (profile == SNLM_GAUSS_IIR && iir_check_beta(beta_or_default(beta, K)) != SNLM_OK)
        return SNLM_ERR_ARG;
    if (!is_device_ptr(x) || !is_device_ptr(out))
        return SNLM_ERR_ARG;
    if (profile == SNLM_GAUSS_IIR) {
        TraceScope ts(SNLM_K_PATCH_DIST | (DIST_IIR << 8), static_cast<cudaStream_t>(stream));
        return status_of(run_iir_dist(Lines{x, dtype, (long long)stride, 1}, n_lines, N, S, beta_or_default(beta, K),
                                      static_cast<float *>(out), static_cast<cudaStream_t>(stream)));
    }
    DistArgs a;
    memset(&a, 0, sizeof(a));
    a.src = Lines{x, dtype, (long long)stride, 1};
    a.n_lines = n_lines;
    a.N = N;
    a.S = S;
    fill_profile(a.g, K, profile, beta_or_default(beta, K));
    a.out = out;
    a.int_out = (dtype == SNLM_U8 && profile == SNLM_BOX) ? 1 : 0;
    const int dm = dist_mode_for(dtype, profile);
    TraceScope ts(SNLM_K_PATCH_DIST | (dm << 8), static_cast<cudaStream_t>(stream));
    return status_of(dispatch_dist(K, a, dm, static_cast<cudaStream_t>(stream)));
}

int snlm_trace_enable(int enable)
{
    Trace &t = trace();
    std::lock_guard<std::mutex> g(t.mu);
    const int prev = t.on ? 1 : 0;
    t.on = enable != 0;
    return prev;
}

int snlm_trace_read(int *kinds, float *ms, int max_records, int *n_records)
{
    if (max_records < 0 || (max_records > 0 && (!kinds || !ms)) || !n_records)
        return SNLM_ERR_ARG;
    Trace &t = trace();
    std::lock_guard<std::mutex> g(t.mu);
    int n = 0;
    int rc = SNLM_OK;
    for (const TraceRec &r : t.recs) {
        if (n < max_records) {
            float v = -1.f;
            if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&v, r.a, r.b) != cudaSuccess) {
                cudaGetLastError();
                rc = SNLM_ERR_CUDA;
            }
            kinds[n] = r.kind;
            ms[n] = v;
            ++n;
        }
        t.spare.push_back(r.a);
        t.spare.push_back(r.b);
    }
    t.recs.clear();
    *n_records = n;
    return rc;
}

const char *snlm_kernel_name(int kind)
{
    // low byte: snlm_kernel_kind; bits 8..11: how the patch distances were
    // reduced; bit 12: the pass moved its data with TMA bulk tensor copies
    static const char *names[14][5] = {
        {"row_pass", "row_pass/slide", "row_pass/block", "row_pass/fir", "row_pass/iir"},
        {"col_pass", "col_pass/slide", "col_pass/block", "col_pass/fir", "col_pass/iir"},
        {"row_pass_sure", "row_pass_sure/slide", "row_pass_sure/block", "row_pass_sure/fir", "row_pass_sure/iir"},
        {"col_pass_sure", "col_pass_sure/slide", "col_pass_sure/block", "col_pass_sure/fir", "col_pass_sure/iir"},
        {"sure_solve", "sure_solve", "sure_solve", "sure_solve", "sure_solve"},
        {"combine", "combine", "combine", "combine", "combine"},
        {"set_theta", "set_theta", "set_theta", "set_theta", "set_theta"},
        {"patch_dist", "patch_dist/slide", "patch_dist/block", "patch_dist/fir", "patch_dist/iir"},
        {"line_pass", "line_pass/slide", "line_pass/block", "line_pass/fir", "line_pass/iir"},
        {"batch", "batch", "batch", "batch", "batch"},
        {"bilateral", "bilateral", "bilateral", "bilateral", "bilateral"},
        {"nlm_2d", "nlm_2d", "nlm_2d", "nlm_2d", "nlm_2d"},
        {"line_pass_3d", "line_pass_3d/slide", "line_pass_3d/block", "line_pass_3d/fir", "unknown"},
        {"relayout_3d", "relayout_3d", "relayout_3d", "relayout_3d", "relayout_3d"},
    };
    static const char *tma_names[4][3] = {
        {"row_pass/slide/tma", "row_pass/block/tma", "row_pass/fir/tma"},
        {"col_pass/slide/tma", "col_pass/block/tma", "col_pass/fir/tma"},
        {"row_pass_sure/slide/tma", "row_pass_sure/block/tma", "row_pass_sure/fir/tma"},
        {"col_pass_sure/slide/tma", "col_pass_sure/block/tma", "col_pass_sure/fir/tma"},
    };
    const int base = kind & 0xff, dm = (kind >> 8) & 0xf, tma = (kind >> 12) & 1;
    if (kind < 0 || base > 13 || dm > 3 || (kind >> 13) != 0)
        return "unknown";
    if (tma)
        return base <= 3 && dm <= 2 ? tma_names[base][dm] : "unknown";
    const bool has_dm = base <= 3 || base == 7 || base == 8 || base == 12;
    return names[base][has_dm ? dm + 1 : 0];
}

}  // extern "C"
