// Recursive Gaussian patch profile: the constant-time route to the Gaussian
// distances of Eq. (3) that Sec. II-B names (the third-order recursive filter of
// Young and van Vliet, 1995).
//
// For an offset s the distances d^2(x, x+s) along a line are the lifted squares
// F(x) = (f(x+s) - f(x))^2 of the extended line, filtered by a causal pass
//   w(x) = B F(x) + a1 w(x-1) + a2 w(x-2) + a3 w(x-3)
// and then the same recursion run anti-causally on w, times beta sqrt(2 pi). The
// filter has unit DC gain and approximates the normalised Gaussian of standard
// deviation beta, so the product approximates the profile g_beta of Eq. (3) with
// infinite support, at a cost per pair that does not depend on the patch width.
//
// Work decomposition. A CTA holds kIirWarps lines and one tile of output positions,
// one warp per line; lane r owns the kIirRun = 16 consecutive positions
// b0 + 16 r .. b0 + 16 r + 15 of a 512-position window. A recursion along the
// window is spread over the lanes as a scan of affine maps (the parallel evaluation
// of a linear recurrence): each lane runs the recursion over its own run from a zero
// state, which gives the run's end state v (its last three outputs); the state
// entering lane r is sum_j A^(16 j) v_(r-1-j), formed by a
// Kogge-Stone scan of warp shuffles with the 3x3 companion matrix A of the
// recursion; the lane then runs its recursion again from that state. The
// anti-causal pass does the same from right to left.
//
// The impulse response decays geometrically, so a position needs a bounded history:
// the host sets `warm`, the number of samples after which the causal response stays
// below 1e-9 of its peak, and the scan runs the rounds that reach that far
// (16 * 2^rounds >= warm). Only positions with `warm` samples of the window on both
// sides have exact distances; the S positions after the first of them only feed
// mirrored pairs (below), so a tile has 512 - 2 warm - S output positions.
//
// Band symmetry (Eq. (8)): for the filter over the extended line,
// d^2(x+s, -s) = d^2(x, s), so only s = 1..S are filtered. The weight w of the pair
// (x, x+s) goes to pixel x with the difference f(x+s) - f(x) and to pixel x+s with
// the opposite one: each lane pushes w and w (f(x+s) - f(x)) into two per-warp
// shared-memory rows at position x+s (the index it read f(x+s) from), and after a
// warp barrier every lane reads its own positions back. Accumulation is centred as in
// the running-sum passes: fhat = f(x) + A / (1 + Q), A = sum w (f(j) - f(x)), Q = sum w.
#include "snlm_host.h"
#include "snlm_iir.h"
#include "snlm_internal.h"

#include <cuda_fp16.h>

#include <vector>

namespace snlm {

namespace {

constexpr int kIirRun = 16;                      // positions per lane
constexpr int kIirSpan = 32 * kIirRun;           // positions per warp window
constexpr int kIirWarps = 4;                     // lines per CTA
constexpr int kIirMaxWarm = 64;                  // history a position may need (58 at beta = 3.5)
constexpr int kIirMaxRounds = 2;                 // scan rounds (16 * 2^rounds >= warm)

__host__ __device__ constexpr int iir_pad(int p) { return p + (p >> 4); }   // 32 lanes -> 32 banks

// Floats of one per-warp row indexed by window position (padded), for a window of
// 512 + S <= 640 samples; a warp holds the samples, and for the NLM pass the pushed
// weights and weighted differences as well, at fixed offsets from the samples.
constexpr int kIirRow = (iir_pad(kIirSpan + kMaxS) + 4) & ~3;

struct IirArgs {
    Lines src;
    int n_lines, N, S;
    int warm, rounds;            // history samples a position needs, scan rounds
    int T;                       // output positions per tile
    float a1, a2, a3;            // the recursion (its gain B is folded into c2 and scale)
    float P[kIirMaxRounds][9];   // A^(16 * 2^d), row-major
    float c2;                    // -log2(e) beta sqrt(2 pi) B^2 / h^2: w = 2^(c2 * y)
    float scale;                 // beta sqrt(2 pi) B^2: distance = scale * y
    float *dst;                  // fhat (pass) ...
    long long out_line_step, out_elem_step;
    const float *blend;          // optional: dst = (fhat + blend) / 2, indexed like dst
    float *dist;                 // ... or the distances (n_lines, N, 2S+1), float32
    // divergence of Eq. (24) (SURE passes): the profile's weight at each lag, its
    // centre weight and h^2; delta in (NULL = 1) and out, indexed like dst
    float geff[kMaxS + 1];
    float g0, h2;
    const float *delta_in;
    float *delta_out;
};

constexpr int kIirPass = 0, kIirDist = 1, kIirSure = 2;   // what iir_pass_kernel computes

// Half-sample symmetric extension of any x onto [0, n).
__device__ __forceinline__ int iir_reflect(int x, int n)
{
    if (x >= 0 && x < n)
        return x;
    const int p = 2 * n;
    int y = x % p;
    if (y < 0)
        y += p;
    return y < n ? y : p - 1 - y;
}

// A warp's window into its shared-memory row: fs[pad(q)] = sample at line position
// b0 + q (through the extension), q < nf, lane q of every 32. The loads go out in
// batches of five, each issued before its first value is stored (five slots at a time
// keep the pass kernels within their register budget). Element offsets fit in 31 bits
// (checked by the host before any launch).
constexpr int kIirLoadSlots = (kIirSpan + kMaxS + 31) / 32;

template <typename T>
__device__ __forceinline__ void iir_gather_t(float *fs, const T *p, unsigned base, int es, int N,
                                             int b0, int lane, int nf)
{
#pragma unroll 1
    for (int j0 = 0; j0 < kIirLoadSlots; j0 += 5) {
        float v[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int q = lane + 32 * (j0 + j);
            if (q < nf) {
                const T t = __ldg(p + base + (unsigned)(iir_reflect(b0 + q, N) * es));
                if constexpr (sizeof(T) == 2)
                    v[j] = __half2float(t);
                else
                    v[j] = (float)t;
            }
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int q = lane + 32 * (j0 + j);
            if (q < nf)
                fs[iir_pad(q)] = v[j];
        }
    }
}

__device__ __forceinline__ void iir_gather(float *fs, const Lines &src, int ln, int N, int b0,
                                           int lane, int nf)
{
    const unsigned base = (unsigned)(ln * (int)src.line_step);
    const int es = (int)src.elem_step;
    if (src.dtype == DT_U8)
        iir_gather_t(fs, static_cast<const unsigned char *>(src.ptr), base, es, N, b0, lane, nf);
    else if (src.dtype == DT_F16)
        iir_gather_t(fs, static_cast<const __half *>(src.ptr), base, es, N, b0, lane, nf);
    else
        iir_gather_t(fs, static_cast<const float *>(src.ptr), base, es, N, b0, lane, nf);
}

__device__ __forceinline__ float iir_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// State entering each lane: the lanes' own end states (v0, v1, v2) combined over the
// preceding lanes (UP) or the following lanes (down) by the Kogge-Stone scan
// S_r <- S_r + A^(16 d) S_(r -+ d); the lane's entering state is its neighbour's S.
template <bool UP>
__device__ __forceinline__ void scan_state(float v0, float v1, float v2, const IirArgs &a, int lane, float &e0,
                                           float &e1, float &e2)
{
    constexpr unsigned kAll = 0xffffffffu;
    float s0 = v0, s1 = v1, s2 = v2;
#pragma unroll
    for (int d = 0; d < kIirMaxRounds; ++d) {
        if (d < a.rounds) {
            const int sh = 1 << d;
            const float t0 = UP ? __shfl_up_sync(kAll, s0, sh) : __shfl_down_sync(kAll, s0, sh);
            const float t1 = UP ? __shfl_up_sync(kAll, s1, sh) : __shfl_down_sync(kAll, s1, sh);
            const float t2 = UP ? __shfl_up_sync(kAll, s2, sh) : __shfl_down_sync(kAll, s2, sh);
            const bool has = UP ? lane >= sh : lane + sh < 32;
            if (has) {
                const float *P = a.P[d];
                s0 = fmaf(P[0], t0, fmaf(P[1], t1, fmaf(P[2], t2, s0)));
                s1 = fmaf(P[3], t0, fmaf(P[4], t1, fmaf(P[5], t2, s1)));
                s2 = fmaf(P[6], t0, fmaf(P[7], t1, fmaf(P[8], t2, s2)));
            }
        }
    }
    e0 = UP ? __shfl_up_sync(kAll, s0, 1) : __shfl_down_sync(kAll, s0, 1);
    e1 = UP ? __shfl_up_sync(kAll, s1, 1) : __shfl_down_sync(kAll, s1, 1);
    e2 = UP ? __shfl_up_sync(kAll, s2, 1) : __shfl_down_sync(kAll, s2, 1);
    if (UP ? lane == 0 : lane == 31)
        e0 = e1 = e2 = 0.f;
}

// The recursive Gaussian of the lifted squares of one offset over the warp's window:
// y[m] = filter output at position b0 + 16 lane + m divided by B^2. The gain B of
// each pass is taken out of the recursions (u = w / B runs u(x) = F(x) + a1 u(x-1) +
// a2 u(x-2) + a3 u(x-3), and y / B^2 the same recursion on u) and folded into the
// host's distance scale and exponent factor, which saves one multiply per pass.
// Each pass runs twice over the lane's run: from rest, for the run's end state that
// the scan combines, then from the state entering the run. (Adding the entering
// state's response afterwards takes as many operations but a table of 48 responses
// that costs the kernel its registers.)
__device__ __forceinline__ void iir_filter_run(const float (&dl)[kIirRun], float (&y)[kIirRun], const IirArgs &a,
                                               int lane)
{
    float w[kIirRun];
    float w1 = 0.f, w2 = 0.f, w3 = 0.f;
#pragma unroll
    for (int m = 0; m < kIirRun; ++m) {          // from rest: the run's end state
        float v = fmaf(dl[m], dl[m], a.a3 * w3);
        v = fmaf(a.a2, w2, v);
        v = fmaf(a.a1, w1, v);
        w3 = w2;
        w2 = w1;
        w1 = v;
    }
    float e0, e1, e2;
    scan_state<true>(w1, w2, w3, a, lane, e0, e1, e2);
    w1 = e0;
    w2 = e1;
    w3 = e2;
#pragma unroll
    for (int m = 0; m < kIirRun; ++m) {          // from the state entering the run
        float v = fmaf(dl[m], dl[m], a.a3 * w3);
        v = fmaf(a.a2, w2, v);
        v = fmaf(a.a1, w1, v);
        w[m] = v;
        w3 = w2;
        w2 = w1;
        w1 = v;
    }
    float y1 = 0.f, y2 = 0.f, y3 = 0.f;
#pragma unroll
    for (int m = kIirRun - 1; m >= 0; --m) {     // anti-causal, from rest
        float v = fmaf(a.a3, y3, w[m]);
        v = fmaf(a.a2, y2, v);
        v = fmaf(a.a1, y1, v);
        y3 = y2;
        y2 = y1;
        y1 = v;
    }
    scan_state<false>(y1, y2, y3, a, lane, e0, e1, e2);
    y1 = e0;
    y2 = e1;
    y3 = e2;
#pragma unroll
    for (int m = kIirRun - 1; m >= 0; --m) {     // and from the state entering from the right
        float v = fmaf(a.a3, y3, w[m]);
        v = fmaf(a.a2, y2, v);
        v = fmaf(a.a1, y1, v);
        y[m] = v;
        y3 = y2;
        y2 = y1;
        y1 = v;
    }
}

// MODE kIirPass: the 1-D NLM pass of Eq. (4) with the recursive profile.
// MODE kIirDist: the distances d^2(x, x+s), s in [-S, S], written to a.dist.
// MODE kIirSure: the pass and the divergence of Eq. (24) with the profile's weight at
// each lag (reading R17): per pixel x and offset s the patch term takes
// w(x, s) g(s) (a_s - mu) a_-s + w(x-s, s) g(s) (a_-s - mu) a_s, a_s = f(x+s) - f(x),
// kept as TA - mu TB; the owner of x reads f(x-s) from the window row and w(x-s, s)
// from the pushed weights. Occupancy: CTAs of 4 warps (warps work independently,
// so small CTAs fill the SMs evenly); 4 per SM for the plain passes (128 registers),
// 3 for SURE (168 registers: its three more accumulators per position spill a few
// words there, and 16 warps at 128 registers spill ~0.5 KB; 12 warps measured 13 %
// faster than 8 at 255 registers).
template <int MODE>
__global__ void __launch_bounds__(kIirWarps * 32, MODE == kIirSure ? 3 : 4) iir_pass_kernel(const IirArgs a)
{
    constexpr bool DIST = MODE == kIirDist;
    constexpr bool SURE = MODE == kIirSure;
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *fs = smem + warp * (DIST ? 1 : 3) * kIirRow;  // f(b0 + q), q < kIirSpan + S
    float *pw = fs + kIirRow;                    // pushed weights of the current offset
    float *pd = pw + kIirRow;                    // pushed weighted differences
    const int q0 = a.warm + a.S;                 // window index of the tile's first output
    const int b0 = blockIdx.x * a.T - q0;        // line position of window index 0
    const int base = lane * kIirRun;
    const int nf = kIirSpan + a.S;
    const int n_groups = div_up(a.n_lines, kIirWarps);
    for (int grp = blockIdx.y; grp < n_groups; grp += gridDim.y) {
        const int ln = grp * kIirWarps + warp;
        if (ln >= a.n_lines)
            continue;                            // warps work independently (no CTA barrier)
        __syncwarp();
        iir_gather(fs, a.src, ln, a.N, b0, lane, nf);
        __syncwarp();
        float fo[kIirRun], accA[kIirRun], accQ[kIirRun];
        float accA2[SURE ? kIirRun : 1], accTA[SURE ? kIirRun : 1], accTB[SURE ? kIirRun : 1];
#pragma unroll
        for (int m = 0; m < kIirRun; ++m) {
            fo[m] = fs[iir_pad(base + m)];
            accA[m] = 0.f;
            accQ[m] = 0.f;
            if constexpr (SURE)
                accA2[m] = accTA[m] = accTB[m] = 0.f;
        }
        for (int s = 1; s <= a.S; ++s) {
            float dl[kIirRun], y[kIirRun];
            const int ib = base + s;
#pragma unroll
            for (int m = 0; m < kIirRun; ++m)
                dl[m] = fs[iir_pad(ib + m)] - fo[m];
            iir_filter_run(dl, y, a, lane);
            if constexpr (DIST) {
                const long long row = (long long)ln * a.N;
                const int stride = 2 * a.S + 1;
#pragma unroll
                for (int m = 0; m < kIirRun; ++m) {
                    const int q = base + m, x = b0 + q;
                    const float d = a.scale * fmaxf(y[m], 0.f);   // the response is non-negative
                    if (q >= q0 && q < q0 + a.T && x < a.N)
                        a.dist[(row + x) * stride + a.S + s] = d;          // d^2(x, x+s)
                    if (q + s >= q0 && q + s < q0 + a.T && x + s < a.N)
                        a.dist[(row + x + s) * stride + a.S - s] = d;      // d^2(x+s, x)
                }
            } else {
                float am[SURE ? kIirRun : 1];            // SURE: a_-s = f(x-s) - f(x)
                const float gs = SURE ? a.geff[s] : 0.f;
#pragma unroll
                for (int m = 0; m < kIirRun; ++m) {
                    // the filter's response is non-negative, so a negative output is
                    // float rounding of a zero distance (weight 1)
                    const float wt = iir_ex2(fminf(a.c2 * y[m], 0.f));
                    const float wd = wt * dl[m];
                    accA[m] += wd;
                    accQ[m] += wt;
                    pw[iir_pad(ib + m)] = wt;            // the pair's share of pixel x + s
                    pd[iir_pad(ib + m)] = wd;
                    if constexpr (SURE) {
                        // positions below s (only before the tile's first output) read a
                        // clamped, unused sample
                        am[m] = fs[iir_pad(max(base + m - s, 0))] - fo[m];
                        const float wg = gs * wt;
                        accA2[m] = fmaf(wd, dl[m], accA2[m]);
                        accTA[m] = fmaf(wg, dl[m] * am[m], accTA[m]);
                        accTB[m] = fmaf(wg, am[m], accTB[m]);
                    }
                }
                __syncwarp();
                // every position q >= s received the push of q - s, whose difference
                // has the opposite sign; positions below s (stale values) lie before the
                // tile's first output
#pragma unroll
                for (int m = 0; m < kIirRun; ++m) {
                    const float db = pd[iir_pad(base + m)], wb = pw[iir_pad(base + m)];
                    accA[m] -= db;
                    accQ[m] += wb;
                    if constexpr (SURE) {
                        // the pair (x-s, x): weight wb, difference f(x-s) - f(x) = a_-s, and
                        // db = wb (f(x) - f(x-s)), so wb a_-s^2 = -db a_-s
                        const float wg = gs * wb;
                        accA2[m] = fmaf(-db, am[m], accA2[m]);
                        accTA[m] = fmaf(wg, dl[m] * am[m], accTA[m]);
                        accTB[m] = fmaf(wg, dl[m], accTB[m]);
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int m = 0; m < kIirRun; ++m) {
            const int q = base + m, x = b0 + q;
            if (q < q0 || q >= q0 + a.T || x >= a.N)
                continue;
            if constexpr (DIST) {
                a.dist[((long long)ln * a.N + x) * (2 * a.S + 1) + a.S] = 0.f;
            } else {
                const float Wt = 1.f + accQ[m];
                const float mu = accA[m] / Wt;
                float v = fo[m] + mu;
                const long long o = (long long)ln * a.out_line_step + (long long)x * a.out_elem_step;
                if (a.blend)
                    v = 0.5f * (v + a.blend[o]);
                a.dst[o] = v;
                if constexpr (SURE) {
                    // Eq. (24) with the profile's centre weight g0 (reading R17):
                    // delta_out = delta_in (h^2 + 2 g0 var + 2 T) / (W h^2),
                    // var = sum_j w (f(j) - fhat)^2 = A2 - mu A, T = TA - mu TB
                    const float var = fmaf(-mu, accA[m], accA2[m]);
                    const float T = fmaf(-mu, accTB[m], accTA[m]);
                    const float num = fmaf(2.f * a.g0, var, fmaf(2.f, T, a.h2));
                    const float din = a.delta_in ? a.delta_in[o] : 1.f;
                    a.delta_out[o] = din * num / (Wt * a.h2);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- host side

// Young and van Vliet's design rules for standard deviation beta (0.5 <= beta):
//   q  = 0.98711 beta - 0.96330 (beta >= 2.5), 3.97156 - 4.14554 sqrt(1 - 0.26891 beta) (below),
//   b0 = 1.57825 + 2.44413 q + 1.4281 q^2 + 0.422205 q^3,  b1 = 2.44413 q + 2.85619 q^2 + 1.26661 q^3,
//   b2 = -(1.4281 q^2 + 1.26661 q^3),  b3 = 0.422205 q^3,  B = 1 - (b1 + b2 + b3) / b0;
// the recursion coefficients are a_k = b_k / b0.
struct IirDesign {
    double B, a[3];
};

IirDesign iir_design(double beta)
{
    const double q = beta >= 2.5 ? 0.98711 * beta - 0.96330 : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * beta);
    const double b0 = 1.57825 + q * (2.44413 + q * (1.4281 + q * 0.422205));
    const double b1 = q * (2.44413 + q * (2.85619 + q * 1.26661));
    const double b2 = -q * q * (1.4281 + q * 1.26661);
    const double b3 = 0.422205 * q * q * q;
    IirDesign d;
    d.a[0] = b1 / b0;
    d.a[1] = b2 / b0;
    d.a[2] = b3 / b0;
    d.B = 1.0 - (b1 + b2 + b3) / b0;
    return d;
}

void mat3_mul(const double *x, const double *y, double *z)
{
    double t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            t[3 * i + j] = x[3 * i] * y[j] + x[3 * i + 1] * y[3 + j] + x[3 * i + 2] * y[6 + j];
    memcpy(z, t, sizeof(t));
}

// Recursion, window geometry and scan tables of one call; SNLM_ERR_ARG when beta
// is outside [kIirBetaMin, kIirBetaMax].
int iir_plan(double beta, int S, IirArgs &a)
{
    if (!(beta >= kIirBetaMin && beta <= kIirBetaMax))
        return SNLM_ERR_ARG;
    const IirDesign d = iir_design(beta);
    // samples after which the causal impulse response stays below 1e-9 of its peak:
    // the truncated tail then moves an exponent d^2 / h^2 by at most about
    // 1e-9 * 255^2 / sigma^2 (h^2 = sigma^2 beta sqrt(2 pi), the default rule)
    int warm = 0;
    {
        double w1 = 0, w2 = 0, w3 = 0, peak = 0;
        for (int n = 0; n < 4096; ++n) {
            const double v = (n == 0 ? d.B : 0.0) + d.a[0] * w1 + d.a[1] * w2 + d.a[2] * w3;
            peak = fmax(peak, fabs(v));
            if (fabs(v) > 1e-9 * peak)
                warm = n + 1;
            w3 = w2;
            w2 = w1;
            w1 = v;
        }
    }
    if (warm > kIirMaxWarm)
        return SNLM_ERR_ARG;
    a.warm = warm;
    a.rounds = 0;
    while ((kIirRun << a.rounds) < warm)
        ++a.rounds;
    a.T = kIirSpan - 2 * warm - S;
    a.a1 = (float)d.a[0];
    a.a2 = (float)d.a[1];
    a.a3 = (float)d.a[2];
    // companion matrix of the recursion: state (w(x), w(x-1), w(x-2))
    const double A[9] = {d.a[0], d.a[1], d.a[2], 1, 0, 0, 0, 1, 0};
    double R[9];
    memcpy(R, A, sizeof(R));
    for (int m = 1; m < kIirRun; ++m)            // A^16: the transfer over one lane's run
        mat3_mul(R, A, R);
    for (int r = 0; r < kIirMaxRounds; ++r) {    // A^(16 * 2^r)
        for (int c = 0; c < 9; ++c)
            a.P[r][c] = (float)R[c];
        mat3_mul(R, R, R);
    }
    a.scale = (float)(beta * sqrt(2.0 * 3.14159265358979323846) * d.B * d.B);
    return SNLM_OK;
}

template <int MODE>
cudaError_t launch_iir_t(const IirArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(iir_pass_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        iir_pass_kernel<MODE><<<grid, kIirWarps * 32, smem, st>>>(a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_iir(const IirArgs &a, int mode, cudaStream_t st)
{
    const int tiles = div_up(a.N, a.T);
    const int groups = div_up(a.n_lines, kIirWarps);
    const dim3 grid((unsigned)tiles, (unsigned)(groups < 65535 ? groups : 65535));
    const bool dist = mode == kIirDist;
    const int smem = kIirWarps * (dist ? 1 : 3) * kIirRow * (int)sizeof(float);   // 33 KB (pass), 11 KB
    if (mode == kIirDist)
        return launch_iir_t<kIirDist>(a, grid, smem, st);
    if (mode == kIirSure)
        return launch_iir_t<kIirSure>(a, grid, smem, st);
    return launch_iir_t<kIirPass>(a, grid, smem, st);
}

// The profile's weight at the lags 0..S: beta sqrt(2 pi) times the two-pass impulse
// response (the weight of the lifted square at x + s in d^2(x, .)), from the same
// recursion run in double on a unit impulse far from both ends.
void iir_lag_weights(double beta, int S, float *geff)
{
    const IirDesign d = iir_design(beta);
    const int L = 4096 + S, n = 2 * L + 1;
    std::vector<double> w((size_t)n, 0.0), y((size_t)n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double x = i == L ? d.B : 0.0;
        w[i] = x + (i >= 1 ? d.a[0] * w[i - 1] : 0.0) + (i >= 2 ? d.a[1] * w[i - 2] : 0.0) +
               (i >= 3 ? d.a[2] * w[i - 3] : 0.0);
    }
    for (int i = n - 1; i >= 0; --i)
        y[i] = d.B * w[i] + (i + 1 < n ? d.a[0] * y[i + 1] : 0.0) + (i + 2 < n ? d.a[1] * y[i + 2] : 0.0) +
               (i + 3 < n ? d.a[2] * y[i + 3] : 0.0);
    const double scale = beta * sqrt(2.0 * 3.14159265358979323846);
    for (int s = 0; s <= S; ++s)
        geff[s] = (float)(scale * y[L + s]);
}

}  // namespace

int preload_iir()
{
    return preload_kernel((const void *)iir_pass_kernel<kIirPass>) +
           preload_kernel((const void *)iir_pass_kernel<kIirDist>) +
           preload_kernel((const void *)iir_pass_kernel<kIirSure>);
}

int iir_check_beta(double beta)
{
    IirArgs a;
    return iir_plan(beta, 0, a);
}

cudaError_t run_iir_pass(const Lines &src, int n_lines, int N, int S, double h, double beta, float *dst,
                         long long out_line_step, long long out_elem_step, const float *blend, cudaStream_t st)
{
    IirArgs a;
    memset(&a, 0, sizeof(a));
    if (iir_plan(beta, S, a) != SNLM_OK)
        return cudaErrorInvalidValue;
    a.src = src;
    a.n_lines = n_lines;
    a.N = N;
    a.S = S;
    const IirDesign d = iir_design(beta);
    double c = -1.4426950408889634 * beta * sqrt(2.0 * 3.14159265358979323846) * d.B * d.B / (h * h);
    if (!(c > -3.0e38))
        c = -3.0e38;
    a.c2 = (float)c;
    a.dst = dst;
    a.out_line_step = out_line_step;
    a.out_elem_step = out_elem_step;
    a.blend = blend;
    return launch_iir(a, kIirPass, st);
}

cudaError_t run_iir_pass_sure(const Lines &src, int n_lines, int N, int S, double h, double beta, float *dst,
                              long long out_line_step, long long out_elem_step, const float *delta_in,
                              float *delta_out, cudaStream_t st)
{
    IirArgs a;
    memset(&a, 0, sizeof(a));
    if (S > kMaxS || iir_plan(beta, S, a) != SNLM_OK)
        return cudaErrorInvalidValue;
    a.src = src;
    a.n_lines = n_lines;
    a.N = N;
    a.S = S;
    const IirDesign d = iir_design(beta);
    double c = -1.4426950408889634 * beta * sqrt(2.0 * 3.14159265358979323846) * d.B * d.B / (h * h);
    if (!(c > -3.0e38))
        c = -3.0e38;
    a.c2 = (float)c;
    a.dst = dst;
    a.out_line_step = out_line_step;
    a.out_elem_step = out_elem_step;
    iir_lag_weights(beta, S, a.geff);
    a.g0 = a.geff[0];
    a.h2 = (float)(h * h);
    a.delta_in = delta_in;
    a.delta_out = delta_out;
    return launch_iir(a, kIirSure, st);
}

cudaError_t run_iir_dist(const Lines &src, int n_lines, int N, int S, double beta, float *out, cudaStream_t st)
{
    IirArgs a;
    memset(&a, 0, sizeof(a));
    if (iir_plan(beta, S, a) != SNLM_OK)
        return cudaErrorInvalidValue;
    a.src = src;
    a.n_lines = n_lines;
    a.N = N;
    a.S = S;
    a.dist = out;
    return launch_iir(a, kIirDist, st);
}

}  // namespace snlm
