/*
 * snlm.h - C ABI of libsnlm, a GB300 (sm_103a) implementation of the separable
 * non-local means filter of Ghosh & Chaudhury, "Fast Separable Non-Local Means"
 * (arXiv:1407.2343).
 *
 * Conventions shared by every entry point
 *  - Every call returns an snlm_status (0 = success). No exception crosses the
 *    ABI and nothing aborts the process.
 *  - Arguments are validated before any work is queued; on an argument error the
 *    outputs are left untouched.
 *  - Pointers documented as DEVICE must point to memory of the current CUDA
 *    device (cudaMalloc, cudaMallocAsync, or any allocator that hands out such
 *    memory, e.g. a PyTorch CUDA tensor). The caller owns all memory passed in;
 *    the library never frees it.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Device work is queued asynchronously on it; the call returns
 *    before the work finishes unless stated otherwise.
 *  - Images are row-major. `pitch` is the distance between consecutive rows in
 *    ELEMENTS of the input type (pitch >= W).
 *  - Boundaries use half-sample symmetric extension (f(-1) = f(0),
 *    f(N) = f(N-1)), repeated with period 2N when S + K >= N; it applies to the
 *    samples of a patch and to search positions alike.
 *  - Limits: 0 <= K <= SNLM_MAX_K, 0 <= S <= SNLM_MAX_S, H, W >= 1,
 *    H * W < 2^31 and H * pitch < 2^31 (element offsets are 32-bit), h > 0 and
 *    finite. Strides are positive.
 */
#ifndef SNLM_H
#define SNLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNLM_MAX_K 7
#define SNLM_MAX_S 128

typedef enum {
    SNLM_OK = 0,
    SNLM_ERR_ARG = -1,         /* an argument is out of range or a pointer is null */
    SNLM_ERR_CUDA = -2,        /* a CUDA call failed (launch, copy, or a sticky device error) */
    SNLM_ERR_NOMEM = -3,       /* device or host memory could not be obtained */
    SNLM_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    SNLM_ERR_UNSUPPORTED = -5, /* valid request outside the compiled configurations */
    SNLM_ERR_CHECK = -6        /* checked builds only: a kernel wrote past its shared-memory rows */
} snlm_status;

typedef enum { SNLM_U8 = 0, SNLM_F16 = 1, SNLM_F32 = 2 } snlm_dtype;

/* Patch profile g_beta (Sec. II, Eq. (3)): box (g = 1) or Gaussian
 * g(k) = exp(-k^2 / (2 beta^2)), both truncated to k in [-K, K].
 * SNLM_GAUSS_IIR is the recursive Gaussian that Sec. II-B names for computing the
 * Gaussian distances in constant time per pair (the third-order filter of Young
 * and van Vliet, 1995): the lifted squares (f(x) - f(x+s))^2 along each line go
 * through its causal and anti-causal passes and are scaled by beta sqrt(2 pi), which
 * approximates g_beta with infinite support (K then only sets the default beta =
 * K/2). It needs 0.5 <= beta <= 3.5; results are float32 (not bit-exact). The plain
 * entry points (snlm_denoise, _ws, _host, _host_many, _bf, _noalloc) accept it
 * with the RC, CR and AVG orders; SURE, the batch plans, the server, the 2-D NLM and
 * the 3-D extension return SNLM_ERR_UNSUPPORTED for it, and snlm_nlm_1d does when
 * a derivative is asked. */
typedef enum { SNLM_BOX = 0, SNLM_GAUSS = 1, SNLM_GAUSS_IIR = 2 } snlm_profile;

/* How the row-then-column (RC) and column-then-row (CR) results are combined
 * (Sec. III, Eq. (14)): RC alone, CR alone, their average, or the SURE-optimal
 * weights of Sec. III-A (Eqs. (17), (19), (25); Alg. 4). */
typedef enum { SNLM_RC = 0, SNLM_CR = 1, SNLM_AVG = 2, SNLM_SURE = 3 } snlm_order;

/* Human-readable name of a status code (static storage; never NULL). */
const char *snlm_status_str(int status);

/* Library version as 10000*major + 100*minor + patch. */
int snlm_version(void);

/* Default smoothing parameter h = sigma * sqrt(sum_{k=-K..K} g(k)); for the
 * box profile this is sigma * sqrt(2K+1), for the recursive Gaussian
 * sigma * sqrt(beta sqrt(2 pi)) (its whole response). beta <= 0 selects beta = K/2.
 * Returns -1 on an invalid argument. Host-only; no device work. */
float snlm_default_h(float sigma, int K, int profile, float beta);

/* Bytes of device scratch that snlm_denoise_ws needs for an H x W image with the
 * given order. Returns 0 on an invalid argument. Host-only. */
size_t snlm_workspace_bytes(int H, int W, int order);

/*
 * Separable NLM of one image: Alg. 4 of the paper without the bilateral
 * post-filter of Sec. III-B. Each 1-D pass is the NLM of Eq. (4) along rows or
 * columns, with patch distances of Eq. (3) and weights w = exp(-d^2/h^2).
 *   img    DEVICE, H rows of `pitch` elements of type `dtype` (u8, f16 or f32).
 *   out    DEVICE, H*W float32, dense row-major; receives
 *          RC: f_rc, CR: f_cr, AVG: (f_rc + f_cr)/2,
 *          SURE: theta1 f_rc + theta2 f_cr with theta solving Eq. (19)/(25).
 *   S, K   search half-width and patch half-width.
 *   h      smoothing parameter (> 0); see snlm_default_h.
 *   profile, beta   patch profile; beta <= 0 selects K/2 (ignored for box).
 *   order  snlm_order.
 *   sigma  noise standard deviation, used only by SNLM_SURE (>= 0).
 * Scratch comes from a per-device pool inside the library (grown on demand with
 * cudaMalloc, kept until process exit); calls on one device must therefore not
 * run concurrently from several host threads. Use snlm_denoise_ws to supply
 * scratch instead.
 */
int snlm_denoise(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h,
                 int profile, int order, float sigma, float beta, float *out, void *stream);

/*
 * As snlm_denoise, with caller-provided DEVICE scratch of at least
 * snlm_workspace_bytes(H, W, order) bytes (16-byte aligned), and an optional
 * DEVICE pointer `info` (NULL allowed) that receives 10 doubles:
 *   theta1, theta2, A11, A12, A22, sum f*f_rc, sum f*f_cr, sum delta1,
 *   sum delta2, sigma^2   (A and the sums of Eqs. (19) and (25); theta of Eq. (14)).
 * The sums are filled only for SNLM_SURE; theta is always filled.
 */
int snlm_denoise_ws(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h,
                    int profile, int order, float sigma, float beta, float *out, void *workspace,
                    size_t workspace_bytes, double *info, void *stream);

/*
 * End-to-end variant for HOST buffers: copies `img_host` (H rows of `pitch`
 * elements) to the device, runs snlm_denoise, and copies the H*W float32 result
 * into `out_host`, all on `stream`; returns after the result is in `out_host`.
 * Pinned (page-locked) host memory gives asynchronous copies; pageable memory
 * works but is slower. Device buffers come from the library's pool.
 */
int snlm_denoise_host(const void *img_host, int dtype, int H, int W, int pitch, int S, int K,
                      float h, int profile, int order, float sigma, float beta, float *out_host,
                      void *stream);

/*
 * Pipelined end-to-end variant for n same-shaped HOST images: image i is copied
 * from imgs_host[i], denoised and copied into outs_host[i] (H*W float32) exactly
 * as snlm_denoise_host would do it, but the copies run on two streams of the
 * call's own, overlapped with the computation of the neighbouring images (two
 * device input and two output buffers; the computations run one after another
 * on `stream`). Returns after every result is in its buffer. The overlap needs
 * pinned host memory; pageable memory works without it. Device buffers come from
 * the library's pool. Arguments are validated as in snlm_denoise_host, plus:
 * n >= 0 (n == 0 does nothing) and every imgs_host[i] and outs_host[i] non-NULL.
 * Results are identical to n calls of snlm_denoise_host.
 */
int snlm_denoise_host_many(const void *const *imgs_host, float *const *outs_host, int n, int dtype, int H,
                           int W, int pitch, int S, int K, float h, int profile, int order, float sigma,
                           float beta, void *stream);

/*
 * Bilateral post-filter of Sec. III-B, Eq. (BF): out(i) is the average of in(i - j)
 * over the integer offsets j of [-R, R]^2, R = floor(3 sigma_s), with weights
 * exp(-|j|^2 / (2 sigma_s^2)) * exp(-(in(i - j) - in(i))^2 / (2 sigma_r^2));
 * samples outside the image are read through the half-sample symmetric extension.
 * Computed exactly (direct sum, FP32, one ex2 per tap), not through an
 * approximation of the range kernel.
 *   in   DEVICE float32, H rows of in_pitch >= W elements.
 *   out  DEVICE float32, H rows of out_pitch >= W elements; must not overlap in.
 *   sigma_s > 0, sigma_r > 0, both finite; R <= 8 (sigma_s < 3) and H <= 2,097,120,
 *   else SNLM_ERR_UNSUPPORTED. Asynchronous on `stream`.
 */
int snlm_bilateral(const float *in, int H, int W, int in_pitch, float sigma_s, float sigma_r, float *out,
                   int out_pitch, void *stream);

/*
 * The post-filter's parameters as functions of the noise level sigma >= 0: the
 * cubic rules learnt in Sec. IV-A,
 *   sigma_s = 2.5e-6 sigma^3 - 3.4e-4 sigma^2 + 0.021 sigma + 0.46,
 *   sigma_r = 2.8e-4 sigma^3 - 0.088 sigma^2 + 8 sigma - 24
 * (evaluated in double, returned as float). SNLM_ERR_ARG for a negative or
 * non-finite sigma or a NULL output.
 */
int snlm_bf_params(float sigma, float *sigma_s, float *sigma_r);

/*
 * SNLM[f] of Sec. III-B: snlm_denoise followed by snlm_bilateral. Arguments as in
 * snlm_denoise, plus the post-filter's sigma_s and sigma_r; when either is <= 0
 * both come from snlm_bf_params(sigma) (which needs sigma > ~3.2 for sigma_r > 0).
 * The intermediate image comes from the library's pool. Asynchronous on `stream`.
 */
int snlm_denoise_bf(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h, int profile,
                    int order, float sigma, float beta, float sigma_s, float sigma_r, float *out, void *stream);

/*
 * The 2-D non-local means of Eqs. (1)-(2) (Sec. I), the workload the run-time
 * tables of Sec. IV-B compare separable NLM against: at pixel i the average of
 * f(j) over the (2S+1)^2 window centred at i with weights
 * exp(-(1/h^2) sum_{k in [-K,K]^2} G(k) (f(i+k) - f(j+k))^2), G(k1,k2) = g(k1) g(k2)
 * (box: 1; Gaussian: exp(-|k|^2 / (2 alpha^2)), alpha <= 0 selects K/2); samples
 * through the half-sample symmetric extension along each axis. Evaluated exactly
 * (every offset of the window, the patch sum as two 1-D filters), FP32.
 *   img  DEVICE, H rows of `pitch` elements of `dtype`; out DEVICE float32 H x W.
 *   S <= 32, K <= 7 and H <= 1,048,560 (else SNLM_ERR_UNSUPPORTED). Asynchronous on `stream`.
 */
int snlm_nlm_2d(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h, int profile,
                float alpha, float *out, void *stream);

/*
 * Separable 3-D extension (the paper's conclusion: separable NLM extends directly to
 * video and volume data): the 1-D pass of Eq. (4) along x, y and z in turn.
 *   vol   DEVICE, D x H x W samples of `dtype`, dense (x fastest, then y, then z).
 *   out   DEVICE float32, D x H x W dense.
 *   order3  SNLM3_XYZ: x, then y, then z; SNLM3_AVG6: the average of the six orders.
 * S, K, h, profile, beta as in snlm_denoise (h > 0 required); D*H*W < 2^31.
 * Scratch: two float32 volumes from the library's pool. Asynchronous on `stream`.
 */
typedef enum { SNLM3_XYZ = 0, SNLM3_AVG6 = 1 } snlm_order3;
int snlm_denoise_3d(const void *vol, int dtype, int D, int H, int W, int S, int K, float h, int profile,
                    float beta, int order3, float *out, void *stream);

/*
 * One 1-D NLM pass (Eq. (4)) over n_lines signals, with the derivative chain of
 * Eq. (24) when delta_out is given (the computation of Alg. 3).
 *   x          DEVICE, samples of type dtype; sample i of line l is at
 *              x[l*line_step + i*elem_step] (elements).
 *   fhat       DEVICE float32, same indexing with (out_line_step, out_elem_step).
 *   delta_in   DEVICE float32 or NULL (all ones), same indexing as fhat.
 *   delta_out  DEVICE float32 or NULL (not computed), same indexing as fhat; may
 *              alias delta_in.
 * fhat must not overlap x.
 */
int snlm_nlm_1d(const void *x, int dtype, int n_lines, int N, long long line_step,
                long long elem_step, int S, int K, float h, int profile, float beta,
                float *fhat, long long out_line_step, long long out_elem_step,
                const float *delta_in, float *delta_out, void *stream);

/*
 * Patch distances of Eq. (3) for n_lines 1-D signals of length N.
 *   x     DEVICE; sample i of line l at x[l*stride + i] (elements of dtype).
 *   out   DEVICE; out[(l*N + i)*(2S+1) + (s+S)] = d^2(i, i+s), s in [-S, S].
 *         int32 when dtype == SNLM_U8 and profile == SNLM_BOX (exact integers),
 *         float32 otherwise.
 * Computed by the same device code as the fused passes: lifted squared
 * differences reduced by running sums (box), the (2K+1)-tap profile (Gaussian) or
 * the recursive filter (SNLM_GAUSS_IIR, which writes d^2(i, i-s) from the filter
 * of offset s by the band symmetry of Eq. (8)).
 */
int snlm_patch_dist_1d(const void *x, int dtype, int n_lines, int N, int stride, int S, int K,
                       int profile, float beta, void *out, void *stream);


/*
 * SURE over row bands: the one exchange step when an image is split into bands of
 * rows (across GPUs or ranks). Alg. 4's divergence and the seven sums of Eqs. (19)
 * and (25) are sums over pixels, so each band forms its own sums over the rows it
 * owns, the sums of all bands are added (an all-reduce), and every band solves the
 * same 2x2 system and combines its own rows.
 *
 * snlm_sure_band runs the four passes of Alg. 4 on `img` (a band of a larger image
 * together with its halo rows, S + K on each side; or any whole image) like
 * snlm_denoise_ws in the SURE order, but keeps the two orders apart: f_rc (rows then
 * columns) and f_cr (columns then rows), device float32 H x W (dense, row-major),
 * and writes to `sums` (device, 7 doubles, 8-byte aligned) the seven sums over the
 * image rows [row0, row1) only, in the basis m = (f_rc + f_cr)/2,
 * d = (f_rc - f_cr)/2:
 *   sums = {sum m^2, sum m d, sum d^2, sum f m, sum f d, sum delta_1, sum delta_2}
 * (f the stored input samples, delta_1 and delta_2 the chained derivatives of
 * Eq. (24) of the two orders). The sums of disjoint row sets add. The workspace is
 * snlm_workspace_bytes(H, W, SNLM_SURE) bytes (16-byte aligned). Errors as
 * snlm_denoise_ws; SNLM_ERR_ARG also for 0 <= row0 < row1 <= H violated or
 * f_rc == f_cr. The recursive profile returns SNLM_ERR_UNSUPPORTED.
 *
 * snlm_sure_theta solves Eqs. (19), (25) for theta from seven such sums (HOST
 * arrays; theta: 2 doubles): the minimiser of Eq. (17) in the basis m, d, the
 * minimum-norm solution when the system is singular (det <= 1e-12 trace^2). It
 * runs on the host and touches no device.
 *
 * snlm_sure_combine writes out = theta1 f_rc + theta2 f_cr over n floats (device
 * pointers; out may alias f_cr), asynchronously on `stream`.
 */
int snlm_sure_band(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h, int profile,
                   float beta, int row0, int row1, float *f_rc, float *f_cr, double *sums, void *workspace,
                   size_t workspace_bytes, void *stream);
int snlm_sure_theta(const double *sums, float sigma, double *theta);
int snlm_sure_combine(const float *f_rc, const float *f_cr, long long n, double theta1, double theta2, float *out,
                      void *stream);

/*
 * Separable NLM without any device allocation (no counterpart in the paper).
 * Same computation, arguments and results as snlm_denoise, for callers that may
 * not call cudaMalloc or cudaFree at run time: real-time loops (an allocation can
 * synchronise the device and take an unbounded time), plug-ins whose host
 * application owns all device memory, programs that must keep a fixed footprint.
 * The caller passes the input and output buffers; the intermediate images use a
 * fixed scratch area of SNLM_NOALLOC_SCRATCH_BYTES compiled into the library
 * (held by every device that loads the library until the process exits).
 *  - Images that need more scratch are rejected with SNLM_ERR_ARG before any work
 *    is queued; snlm_workspace_bytes(H, W, order) <= SNLM_NOALLOC_SCRATCH_BYTES is
 *    a sufficient condition. The largest square images it admits for every S are
 *    1654 x 1654 (SURE), 2047 x 2047 (AVG) and 2896 x 2896 (RC, CR).
 *  - Every call looks up the scratch area's device address in the context that is
 *    current (a host-side query, so a reset device or another context on the same
 *    device is handled). The first call in a context may load the library's device
 *    code, unless snlm_preload loaded it beforehand.
 *  - All calls in the process share the scratch area. Calls whose device work can
 *    overlap in time (several streams, or several host threads without ordering)
 *    race on it and corrupt each other's results: serialise them.
 */
#define SNLM_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int snlm_denoise_noalloc(const void *img, int dtype, int H, int W, int pitch, int S, int K, float h,
                         int profile, int order, float sigma, float beta, float *out, void *stream);

/*
 * Batched denoising of many independent images (uneven sizes, per-image S, K, h,
 * profile, order) in a few launches over a tile work queue.
 *
 * A plan turns the requests into jobs (one per 1-D pass of an image, plus the
 * SURE solve and combination) and jobs into CTA-sized units (4 lines x one tile).
 * Jobs are grouped into classes by dependency level (all first passes, then all
 * second passes, ...) and kernel (a pass variant and K, or the solve or the
 * combination), one launch each with one CTA per unit, run in level order, so a
 * unit's dependencies are complete when it starts. Each CTA still checks them on
 * per-job completion counters with a bounded wait (snlm_batch_config.spin_limit_us);
 * when a bound is hit (only an injected fault does that) the kernel records it, the
 * CTAs after it do no work, and snlm_batch_plan_status returns SNLM_ERR_TIMEOUT. Each image's result equals snlm_denoise's bit for bit for the
 * RC, CR and AVG orders (same per-unit code); for SURE the per-image sums are
 * reduced in a different fixed order, so theta may differ in the last bits.
 */
typedef struct {
    const void *img;   /* DEVICE input, H rows of `pitch` elements of `dtype` */
    float *out;        /* DEVICE output, H*W float32 */
    int dtype, H, W, pitch;
    int S, K;
    float h;
    int profile, order;
    float sigma, beta; /* as in snlm_denoise */
} snlm_request;

typedef struct {
    int ctas_per_sm;   /* cap on resident CTAs per SM (applied through each CTA's
                          share of shared memory); <= 0: as many as fit */
    int queue_order;   /* 0: as given, 1: largest images first, 2: smallest first */
    int spin_limit_us; /* bound of one dependency wait; <= 0: 2 000 000 */
    int fail_job;      /* testing aid: >= 0 makes that job's first dependency
                          unsatisfiable (host-side fault injection); -1 normally.
                          Jobs are numbered in the plan's order (by dependency
                          level); the last job always has a dependency, a job
                          without one gives SNLM_ERR_ARG */
} snlm_batch_config;

typedef struct snlm_batch_plan snlm_batch_plan;

/* Builds a plan (host only). Every request is validated as in snlm_denoise;
 * K must be >= 1 in a batch. cfg may be NULL (defaults). */
int snlm_batch_plan_create(const snlm_request *reqs, int n, const snlm_batch_config *cfg,
                           snlm_batch_plan **plan);
/* DEVICE scratch the plan needs (job table, counters, intermediate images). */
size_t snlm_batch_plan_workspace_bytes(const snlm_batch_plan *plan);
/* Copies the job table into `workspace` (16-byte aligned, >= the bytes above) on
 * `stream` and binds the plan to it. */
int snlm_batch_plan_upload(snlm_batch_plan *plan, void *workspace, size_t workspace_bytes, void *stream);
/* Queues one run of the whole batch on `stream` (counter reset + one kernel per
 * class, in dependency-level order, one CTA per unit); replays the captured graph
 * if snlm_batch_plan_capture was called. */
int snlm_batch_plan_launch(snlm_batch_plan *plan, void *stream);
/* Records one run into a CUDA graph (stream capture on `stream`, thread-local
 * mode) and instantiates it; later launches replay the graph. */
int snlm_batch_plan_capture(snlm_batch_plan *plan, void *stream);
/* Waits for `stream`, then reports whether a bounded wait gave up in the last run
 * (SNLM_ERR_TIMEOUT) and clears the flag. */
int snlm_batch_plan_status(snlm_batch_plan *plan, void *stream);
/* The same report without waiting: enqueues on `stream` a copy of the plan's
 * failure word into *host_word and returns. Once the stream has passed that point
 * (an event recorded after this call has completed), *host_word != 0 means a
 * bounded wait of the runs enqueued before it gave up. host_word should be pinned
 * host memory (cudaHostAlloc); with pageable memory CUDA performs the copy
 * synchronously. SNLM_ERR_ARG for a NULL plan, a plan without workspace or a NULL
 * host_word. */
int snlm_batch_plan_status_async(snlm_batch_plan *plan, int *host_word, void *stream);
/* Number of jobs, units and K classes of the plan (any pointer may be NULL). */
int snlm_batch_plan_info(const snlm_batch_plan *plan, int *jobs, int *units, int *classes);
void snlm_batch_plan_destroy(snlm_batch_plan *plan);

/*
 * Launch tracing (no counterpart in the paper; for profiling). When enabled,
 * every kernel the library launches is bracketed by two CUDA events recorded on
 * the launching stream, and snlm_trace_read returns one record per launch:
 * kinds[i] (an snlm_kernel_kind) and ms[i] (device time between the events).
 * The low byte of a kind is an snlm_kernel_kind; bits 8 and up tell how the
 * patch distances were reduced in that launch (0 running sum, 1 block sums,
 * 2 weighted taps), and bit 12 is set when the pass ran the TMA kernel;
 * snlm_kernel_name spells them out (e.g. "row_pass/slide", "col_pass_sure/block/tma").
 * Tracing is process-wide; do not enable it while a stream is being captured
 * into a CUDA graph. snlm_trace_read waits for the recorded events, copies at
 * most max_records records (oldest first), sets *n_records to the number copied
 * and clears the trace. snlm_trace_enable returns the previous setting.
 */
typedef enum {
    SNLM_K_ROW_PASS = 0,       /* 1-D NLM pass along rows (Eq. (4)) */
    SNLM_K_COL_PASS = 1,       /* 1-D NLM pass along columns */
    SNLM_K_ROW_PASS_SURE = 2,  /* row pass with the divergence of Eq. (24) */
    SNLM_K_COL_PASS_SURE = 3,  /* column pass with the divergence of Eq. (24) */
    SNLM_K_SURE_SOLVE = 4,     /* reduction of the sums of Eqs. (19), (25) and the 2x2 solve */
    SNLM_K_COMBINE = 5,        /* theta1 f_rc + theta2 f_cr (Eq. (14)) */
    SNLM_K_SET_THETA = 6,      /* writes the fixed weights of the RC / CR / AVG orders */
    SNLM_K_PATCH_DIST = 7,     /* patch distances of Eq. (3) */
    SNLM_K_LINE_PASS = 8,      /* snlm_nlm_1d pass over arbitrary strided lines */
    SNLM_K_BATCH = 9,          /* one batch class kernel (a pass variant and K, or the solve and combination) */
    SNLM_K_BILATERAL = 10,     /* bilateral post-filter of Sec. III-B (Eq. (BF)) */
    SNLM_K_NLM_2D = 11,        /* the 2-D NLM of Eqs. (1)-(2) (comparison workload) */
    SNLM_K_LINE_PASS_3D = 12,  /* a 1-D pass of the separable 3-D extension */
    SNLM_K_RELAYOUT_3D = 13    /* the 3-D extension's outer-dimension swaps and averaging */
} snlm_kernel_kind;

int snlm_trace_enable(int enable);
int snlm_trace_read(int *kinds, float *ms, int max_records, int *n_records);
const char *snlm_kernel_name(int kind);

/*
 * Measured arithmetic peaks of the current device (no counterpart in the paper; a
 * measurement aid for the roofline of the 1-D passes, which are bound by FP32
 * issue). Runs three short kernels on `stream` (cudaStream_t as void*, NULL for the
 * default stream), each of independent dependency chains in every thread of a grid
 * of 8 CTAs of 256 threads per SM, timed with CUDA events over 3 launches after
 * one warm-up launch, and waits for them. On return rates[0] = FP32 lane-operations
 * per second issued as packed FP32x2 FMAs, rates[1] = the same through scalar FMAs
 * (an FMA counts as one lane-operation, as in the roofline's operation count),
 * rates[2] = MUFU.EX2 results per second. `rates` is a HOST array of 3 doubles.
 * Takes a few tens of milliseconds. Returns SNLM_ERR_ARG for a NULL `rates`,
 * SNLM_ERR_CUDA when a launch or an event fails.
 */
int snlm_probe_peaks(double *rates, void *stream);

/*
 * Serving loop (no counterpart in the paper): continuous batching of requests
 * that arrive over time. Submit requests whose images and result buffers are in
 * HOST memory (pinned memory lets the copies overlap), each with an arrival time
 * in seconds on the server's clock (which starts at the first snlm_server_drain),
 * then drain: the calling thread runs the loop until every submitted request is
 * served, and returns.
 *
 * SNLM_SERVE_BATCHED: requests are admitted from a FIFO queue as device memory
 * (a slab of mem_budget bytes allocated at creation; <= 0: half the free memory)
 * and one of `streams` streams free up. A request of at least solo_pixels pixels,
 * or a lone request on an idle GPU, runs alone through the per-image path; the
 * consecutive smaller requests at the front of the queue (at most max_batch) run
 * as one batch plan (snlm_batch_plan_*). Each launch
 * copies its inputs in, runs, and copies its results out on its own stream, so
 * launches overlap on the device; half of the streams (at least one) have the
 * device's highest priority and carry the launches of requests below solo_pixels,
 * so that their blocks are dispatched ahead of those of a large request's pass
 * already in flight. SNLM_SERVE_PLAIN serves one request at a time
 * through the per-image path and waits for each (the per-request baseline).
 * Results are those of snlm_denoise (bitwise for RC/CR/AVG; SURE within the float
 * rounding of its sums).
 */
typedef enum { SNLM_SERVE_BATCHED = 0, SNLM_SERVE_PLAIN = 1 } snlm_serve_mode;

typedef struct {
    const void *img;   /* HOST input, H rows of `pitch` elements of `dtype` */
    float *out;        /* HOST output, H*W float32 */
    int dtype, H, W, pitch;
    int S, K;
    float h;
    int profile, order;
    float sigma, beta; /* as in snlm_denoise */
    double t_arrival;  /* seconds on the server clock, >= 0 */
} snlm_serve_request;

typedef struct {
    int mode;               /* snlm_serve_mode */
    long long mem_budget;   /* device bytes for admitted requests; <= 0: half the free memory */
    int streams;            /* launches in flight (1..64; plain mode uses 1) */
    int max_batch;          /* requests per batch launch */
    long long solo_pixels;  /* requests of at least this many pixels run alone */
    int ctas_per_sm;        /* batch kernels; <= 0: as many as fit */
} snlm_server_config;

typedef struct {
    int launches;             /* solo and batch launches made */
    int max_batch;            /* most requests in one launch */
    int max_inflight;         /* most launches in flight at once */
    int images;               /* requests served */
    long long max_used_bytes; /* peak of the admitted requests' device memory */
    long long budget_bytes;   /* the slab */
    double wall_s;            /* server clock at the end of the last drain */
    double host_busy_s;       /* time the loop spent not sleeping */
    double max_yield_s;       /* longest single yield of the core while idle (host scheduling) */
    double max_iter_s;        /* longest pass of the loop's own work (admission, launch, retire) */
    int yields_over_1ms;      /* yields that kept the loop away for more than 1 ms */
} snlm_server_stats;

typedef struct snlm_server snlm_server;

/* cfg may be NULL (defaults: batched, half the free memory, 4 streams, 256 per batch,
 * 1<<20 solo pixels). Loads every kernel first (snlm_preload): SNLM_ERR_CUDA if that
 * fails. SNLM_ERR_NOMEM if the slab cannot be allocated. */
int snlm_server_create(const snlm_server_config *cfg, snlm_server **server);
/* Validates and queues n requests (host pointers stay owned by the caller and must
 * stay valid until the drain that serves them returns); ids[i] (may be NULL)
 * receives each request's id. SNLM_ERR_NOMEM for a request larger than the slab. */
int snlm_server_submit(snlm_server *server, const snlm_serve_request *reqs, int n, int *ids);
/* Runs the loop until every submitted request has its result in host memory. */
int snlm_server_drain(snlm_server *server);
/* Completion time (server clock, -1 if not served yet) and launch index of a request. */
int snlm_server_result(const snlm_server *server, int id, double *t_done, int *launch);
int snlm_server_get_stats(const snlm_server *server, snlm_server_stats *stats);
double snlm_server_clock(const snlm_server *server);
/* Waits for work in flight and frees the slab and streams. */
void snlm_server_destroy(snlm_server *server);

/*
 * Process-wide options (no counterpart in the paper).
 *
 * SNLM_OPT_TMA (default 0): 1 makes the per-image passes (snlm_denoise*, SURE
 *   order included) run the persistent kernel that moves line windows and tile
 *   inputs with TMA bulk tensor copies whenever every array a pass reads allows
 *   it: a 16-byte-aligned base address, unit stride along the lines or across
 *   them, and the other stride a multiple of 16 bytes (e.g. an 8-bit image whose
 *   pitch is a multiple of 16, float intermediates of width a multiple of 4).
 *   Other passes, snlm_nlm_1d and the batch kernels always gather their samples
 *   with loads. Both kernels give the same results (the tests hold both to the
 *   oracle's tolerance); the gathering kernel is the faster one on GB300 today.
 * SNLM_OPT_WAIT_LIMIT_US (default 2,000,000): bound of every device-side wait of
 *   the TMA passes, in microseconds (1 .. 60,000,000).
 * SNLM_OPT_INJECT_WAIT_TIMEOUT (default 0): fault injection for tests: the next
 *   `value` TMA pass launches wait for bytes that never arrive, so their waits run
 *   out (no device fault); their outputs are NaN and snlm_device_error reports it.
 *
 * snlm_set_option returns SNLM_OK or SNLM_ERR_ARG; snlm_get_option returns the
 * value, or -1 for an unknown option.
 */
typedef enum {
    SNLM_OPT_TMA = 0,
    SNLM_OPT_WAIT_LIMIT_US = 1,
    SNLM_OPT_INJECT_WAIT_TIMEOUT = 2
} snlm_option;

int snlm_set_option(int option, long long value);
long long snlm_get_option(int option);

/*
 * Device-side failure record of the current device. Waits for the work queued on
 * `stream` (NULL: the legacy default stream), then returns SNLM_ERR_TIMEOUT if a
 * bounded wait of a TMA pass gave up since the last call (every output of the
 * units it could not finish was set to NaN), SNLM_ERR_CUDA if the stream failed,
 * else SNLM_OK; the record is cleared. snlm_denoise_host checks it itself.
 */
int snlm_device_error(void *stream);

/*
 * Loads the device code of every kernel the library launches, on the current device
 * (no counterpart in the paper). Under lazy module loading, CUDA's default, a kernel
 * is otherwise loaded by its first launch, inside the caller's launch sequence, which
 * then holds the calling thread for the load. Call it once per context before
 * latency-sensitive work (a serving loop, the first snlm_denoise_noalloc of a
 * real-time loop); snlm_server_create calls it. A kernel
 * that is already loaded costs a lookup, so repeated calls are cheap. *n_loaded (may
 * be NULL) receives the number of kernels loaded, SNLM_KERNEL_COUNT when all were.
 * Returns SNLM_OK, or SNLM_ERR_CUDA if some kernel could not be loaded.
 */
#define SNLM_KERNEL_COUNT 234
int snlm_preload(int *n_loaded);

#ifdef __cplusplus
}
#endif

#endif /* SNLM_H */
