// Internal declarations shared by the libsnlm translation units (host + device).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace snlm {

constexpr int kMaxK = 7;           // largest patch half-width compiled
constexpr int kMaxS = 128;         // largest search half-width accepted
constexpr int kBfMaxR = 8;         // largest bilateral half-width floor(3 sigma_s) compiled
constexpr int kMaxS2d = 32;        // largest search half-width of the 2-D NLM
constexpr int kRun = 8;            // consecutive positions a lane owns (M)
constexpr int kWarpsPerCta = 4;    // lines per CTA (one warp per line tile)
constexpr int kPartials = 8;       // doubles per CTA in the SURE partial-sum records
#ifdef SNLM_CHECKED
// Checked builds: guard words after each warp's shared-memory rows, written before a
// unit's first store and verified after its last (SNLM_ERR_CHECK when damaged).
constexpr int kSmemGuard = 8;
#else
constexpr int kSmemGuard = 0;
#endif
constexpr unsigned kGuardWord = 0x5a17c0deu;

enum DType { DT_U8 = 0, DT_F16 = 1, DT_F32 = 2 };
// How the patch distance of Eq. (3) is reduced along the line:
//  SLIDE  running window sum (two updates per step) - exact for integer samples
//  BLOCK  prefix/suffix sums inside blocks of 2K+1 samples (no long drift; float samples)
//  FIR    the (2K+1)-tap weighted sum of the Gaussian profile
enum DistMode { DIST_SLIDE = 0, DIST_BLOCK = 1, DIST_FIR = 2 };

// Strided view of a set of 1-D signals: sample i of line l is at
// ptr[l * line_step + i * elem_step] (elements of dtype).
struct Lines {
    const void *ptr;
    int dtype;
    long long line_step;
    long long elem_step;
};

struct PassArgs {
    Lines src;                  // input samples of the pass
    int n_lines, N, S;
    int tiles;                  // tiles per line: div_up(N, tile_positions(S)) (set by finish_pass_args)
    float c2;                   // -log2(e) / h^2, so w = 2^(c2 * d^2)
    float h2;                   // h^2 (divergence only)
    float g[2 * kMaxK + 1];     // patch profile g(k), k = -K..K
    float *dst;                 // fhat, float32
    long long out_line_step, out_elem_step;
    const float *blend;         // optional: dst = (fhat + blend) / 2, same indexing as dst
    const float *delta_in;      // optional (SURE kernels): chained derivative in (NULL = 1)
    float *delta_out;           // optional (SURE kernels): chained derivative out
    double *partials;           // optional: kPartials sums per CTA (see below)
    unsigned *check;            // checked builds: the device word a damaged guard is recorded in
    Lines aux_f;                // the noisy input image f, viewed like dst
    Lines aux_rc;               // f_rc (float32), viewed like dst: when given, the SURE sums below are formed
    int sum_lo, sum_hi;         // only outputs in image rows [sum_lo, sum_hi) enter the sums (sum_hi == 0: all)
    // Per-CTA partial sums (SURE). With m = (f_rc + fhat)/2 and d = (f_rc - fhat)/2
    // (fhat = f_cr in the last pass of the CR order):
    //   [0] sum m^2  [1] sum m d  [2] sum d^2  [3] sum f m  [4] sum f d  [5] sum delta_out
};

struct DistArgs {
    Lines src;
    int n_lines, N, S;
    float g[2 * kMaxK + 1];
    void *out;                  // (n_lines, N, 2S+1), int32 when int_out else float32
    int int_out;
};

// Per-warp shared-memory layout of the pass and distance kernels (in floats).
// Every array indexed by position uses pad_index: one pad word after every kRun
// words, so the 32 lanes (which own runs of kRun consecutive positions) hit 32
// distinct banks.
struct WarpLayout {
    int LF;        // line samples (padded)
    int LW;        // one stored-weight row (SURE, padded)
    int LK;        // SURE: the K stored-weight rows of offsets 1..K
    int LT;        // one tile-sized row (blend, SURE delta in / out, f_rc, f; padded)
    int per_warp;  // total, multiple of 4
    int guard;     // first of the kSmemGuard guard words (checked builds)
};

__host__ __device__ inline int div_up(int a, int b) { return (a + b - 1) / b; }

__host__ __device__ inline int pad_index(int p) { return p + p / kRun; }

__host__ __device__ inline WarpLayout warp_layout(int S, int K, bool sure, bool dist_only)
{
    WarpLayout L;
    L.LK = 0;
    const int nch = div_up(S, kRun);
    // samples at positions b0 - K + q for q < 32*kRun + nch*kRun + 2K + kRun
    const int nf = 32 * kRun + nch * kRun + 2 * K + kRun;
    L.LF = (pad_index(nf) + 4) & ~3;
    L.LW = (pad_index(32 * kRun) + 4) & ~3;
    L.LT = L.LW;
    int n = L.LF;
    if (!dist_only) {
        n += L.LT;                  // the blend input of the tile
        L.LK = sure ? K * L.LW : 0;
        if (sure)                   // stored weights for |s| <= K; delta in, delta out; f_rc and f
            n += L.LK + 4 * L.LT;
    }
    L.guard = n;
    L.per_warp = (n + kSmemGuard + 3) & ~3;
    return L;
}

// Output positions per line tile: 32 lanes minus the halo lanes that only
// contribute mirrored pairs to the tile's first positions.
__host__ __device__ inline int tile_positions(int S)
{
    return (32 - div_up(S, kRun)) * kRun;
}

// Fills the derived fields of a pass's arguments (after n_lines, N and S).
// The device word of device-side failure records (snlm_tma_host.cu; read and
// cleared by snlm_device_error).
unsigned *device_error_word();

inline void finish_pass_args(PassArgs &a)
{
    a.tiles = div_up(a.N, tile_positions(a.S));
    a.check = kSmemGuard > 0 ? device_error_word() : nullptr;
}

template <int K> cudaError_t launch_pass(const PassArgs &a, int dist_mode, bool sure, cudaStream_t st);

// Bilateral post-filter (snlm_bilateral.cu): argument checks (an snlm_status) and
// the launch on validated arguments.
int bilateral_radius(float sigma_s);
int check_bilateral(const float *in, int H, int W, long long in_pitch, float sigma_s, float sigma_r,
                    const float *out, long long out_pitch);
int run_bilateral(const float *in, int H, int W, long long in_pitch, float sigma_s, float sigma_r, float *out,
                  long long out_pitch, cudaStream_t st);
// ---- Tensor-memory-accelerator (TMA) movement of a pass (sm_90+ bulk tensor copies).
// Each array a pass reads (the line windows and the tile inputs of the epilogue)
// gets a 2-D tensor map over (dim0, dim1) = (positions, lines) for row-like views
// (TMA_ROWS) or (lines, positions) for column-like views (TMA_COLS), and a unit
// loads boxes whose dim0 start is a multiple of 16 bytes. The landed element
// (line w, position q) of a unit sits at element w*sw + q*sq + o of the view's
// shared-memory area, o being the unit's alignment offset.
enum TmaMode { TMA_NONE = 0, TMA_ROWS = 1, TMA_COLS = 2 };
enum TmaArray { TMA_SRC = 0, TMA_DIN = 1, TMA_BLEND = 2, TMA_RC = 3, TMA_F = 4, TMA_ARRAYS = 5 };

struct TmaView {
    int mode;       // TmaMode
    int dtype;      // DType of the elements
    int esize;      // bytes per element
    int align;      // elements per 16 bytes (dim0 coordinates are multiples of it)
    int nb;         // boxes per line (ROWS) or along the positions (COLS)
    int bw, bh;     // box extents along dim0 and dim1 (elements)
    int sw, sq;     // element strides of the landed data between lines and positions
    int bytes;      // bytes a unit's boxes deliver
    int smem;       // shared-memory bytes reserved for them (multiple of 128)
    int off;        // byte offset of that area in the CTA's dynamic shared memory
};

struct TmaPass {
    CUtensorMap map[TMA_ARRAYS];    // src, delta_in, blend, aux_rc, aux_f
    TmaView v[TMA_ARRAYS];          // v[TMA_SRC].off is window stage 0
    int win_off1;                   // byte offset of window stage 1
    int win_len;                    // window samples per line and unit
    int units;                      // units of the pass (tile fastest)
    int per_warp, LF, LW, LT;       // per-warp float layout: window, K weight rows, delta_out
    int smem;                       // dynamic shared-memory bytes per CTA
    unsigned long long wait_ns;     // bound of every barrier wait
    unsigned *err;                  // receives SNLM_ERR_TIMEOUT when a wait gives up (may be NULL)
    int inject;                     // test hook: units expect bytes that never arrive
};

template <int K> cudaError_t launch_pass_tma(const PassArgs &a, const TmaPass &t, int dist_mode, bool sure, int grid,
                                             cudaStream_t st);
template <int K> cudaError_t pass_tma_occupancy(int dist_mode, bool sure, int smem, int *ctas_per_sm);

// Host side (snlm_tma_host.cu).
bool plan_pass_tma(int K, const PassArgs &a, int dist_mode, bool sure, TmaPass *t, int *grid);
cudaError_t launch_planned_tma(int K, const PassArgs &a, const TmaPass &t, int dist_mode, bool sure, int grid,
                               cudaStream_t st);
constexpr int kTraceTma = 1 << 12;   // trace-kind flag: the launch used the TMA kernel

template <int K> cudaError_t launch_dist(const DistArgs &a, int dist_mode, cudaStream_t st);

// scratch: 2 * kSolveScratchRecords * kPartials doubles; ticket: one word of device
// memory (zeroed on the stream by the launch)
constexpr int kSolveScratchRecords = 128;
cudaError_t launch_sure_solve(const double *part_rc, int n_rc, const double *part_cr, int n_cr,
                              double sigma2, double *info, double *scratch, unsigned *ticket, cudaStream_t st);
cudaError_t launch_combine(const float *frc, float *out_fcr, const double *info, long long n,
                           cudaStream_t st);
cudaError_t launch_set_theta(double *info, double t1, double t2, cudaStream_t st);
// The seven sums of a SURE band (snlm_sure_band) from the partial-sum records of the
// last pass of each order, in the basis m = (f_rc + f_cr)/2, d = (f_rc - f_cr)/2:
// sums = {sum m^2, sum m d, sum d^2, sum f m, sum f d, sum delta_1, sum delta_2}.
cudaError_t launch_sure_sums(const double *part_rc, int n_rc, const double *part_cr, int n_cr, double *sums,
                             double *scratch, cudaStream_t st);
// Records of the SURE sums over rows [r0, r1) of dense W-wide images (frc == NULL:
// the delta sum only), n_records blocks: for the passes without records of their own.
cudaError_t launch_image_sums(const float *frc, const float *fcr, const Lines &f, int W, int r0, int r1,
                              const float *delta, double *records, int n_records, cudaStream_t st);
// out = theta1 frc + theta2 fcr over n floats (out may alias fcr).
cudaError_t launch_combine_theta(const float *frc, const float *fcr, float *out, long long n, double theta1,
                                 double theta2, cudaStream_t st);

// ---- Loading the device code up front (snlm_preload). Under lazy module loading,
// CUDA's default, a kernel is loaded by its first launch, inside the caller's launch
// sequence, where the load holds the calling thread. Each preload_* loads every
// kernel its file launches on the current
// device and returns how many it loaded; a kernel that is already loaded costs a
// lookup.
inline int preload_kernel(const void *f)
{
    cudaFuncAttributes attr;
    if (cudaFuncGetAttributes(&attr, f) == cudaSuccess)
        return 1;
    cudaGetLastError();
    return 0;
}
template <int K> int preload_pass();       // snlm_pass_k<K>.cu: pass and distance kernels
template <int K> int preload_pass_tma();   // snlm_pass_k<K>.cu: TMA pass kernels
int preload_batch();                       // snlm_batch.cu
int preload_iir();                         // snlm_iir.cu
int preload_sure();                        // snlm_sure.cu
int preload_bilateral();                   // snlm_bilateral.cu
int preload_nlm2d();                       // snlm_nlm2d.cu
int preload_3d();                          // snlm_3d.cu

}  // namespace snlm
