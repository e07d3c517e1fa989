/*
 * FP64 CPU oracle for separable non-local means (Ghosh & Chaudhury,
 * "Fast Separable Non-Local Means", arXiv:1407.2343).
 *
 * TEST INFRASTRUCTURE ONLY. This file is used by tests/, by the smoke check
 * and by the benchmark's CPU-baseline / reference leg. The product path (the
 * CUDA library under paper_1407_2343_gb300/) never links, imports or calls it,
 * and it shares no code, header, table or helper with that path.
 *
 * What it computes is the plain definition, one pixel at a time, in double
 * precision, with explicit (2K+1)-tap patch sums: no lifting, no running sums,
 * no symmetry reuse. Each function names the passage it follows.
 *
 * Readings of points the paper leaves open:
 *  - Boundary: half-sample symmetric extension, applied to patch samples and
 *    to search positions alike, repeated with period 2N when the reach S+K
 *    exceeds the signal (the paper comments the extension sentence out in
 *    Sec. II; Alg. 2/3 index f(j) and f(2i-j) outside [1,N]).
 *  - Gaussian profile: the truncated (2K+1)-tap g_beta on [-K,K] exactly as in
 *    Eq. (3), not a recursive approximation.
 *  - Divergence: Eq. (24) taken literally, with every sample read through the
 *    extension; its patch term runs over the offsets of the search window that
 *    also satisfy |j-i| <= K (the Appendix sums over the window only).
 *  - SURE solve: A theta = b with A from Eq. (19) and b from Eq. (25); when A is
 *    (numerically) singular the minimum-norm pseudo-inverse solution is used.
 *  - Recursive Gaussian profile (the constant-time route to Eq. (3) that Sec. II-B
 *    points to): the third-order recursive filter of Young and van Vliet (1995),
 *    a causal pass followed by an anti-causal pass with the same coefficients,
 *    applied along i to the lifted squares (f(i) - f(i+s))^2 of the extended
 *    signal. That filter has unit DC gain and approximates the sampled Gaussian
 *    of standard deviation beta divided by its integral, so the distance is its
 *    output times beta*sqrt(2 pi), the integral of g_beta. Its support is
 *    infinite: both passes start from a zero state far enough outside [0, N)
 *    (iir_margin) that the truncated tail is below double rounding.
 *    Its divergence is Eq. (24) with the profile's own centre weight g(0) (not 1)
 *    and the patch term over every offset of the window, weighted by the profile
 *    at that lag (its support is unbounded).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BOX 0
#define ORC_GAUSS 1
#define ORC_GAUSS_IIR 2

#define ORC_RC 0
#define ORC_CR 1
#define ORC_AVG 2
#define ORC_SURE 3

/* Half-sample symmetric extension of an index into [0, N): the extended
 * signal satisfies fe(-1) = f(0), fe(N) = f(N-1), and is 2N-periodic. */
int64_t orc_ext(int64_t x, int64_t N)
{
    int64_t p = 2 * N;
    int64_t y = x % p;
    if (y < 0)
        y += p;
    if (y >= N)
        y = p - 1 - y;
    return y;
}

/* Patch profile g_beta(k), k in [-K, K] (Sec. II, after Eq. (3)): the box
 * profile is 1 everywhere; the Gaussian is exp(-k^2 / (2 beta^2)). */
void orc_profile(int K, int profile, double beta, double *g)
{
    for (int k = -K; k <= K; ++k)
        g[k + K] = (profile == ORC_GAUSS) ? exp(-((double)k * k) / (2.0 * beta * beta)) : 1.0;
}

/* Coefficients of the recursive Gaussian of Young and van Vliet (1995) for the
 * standard deviation beta, from their design rules (q from beta, then the
 * normalised denominator b1/b0, b2/b0, b3/b0 and the gain B that makes the DC
 * gain of each pass exactly one):
 *   q  = 0.98711 beta - 0.96330                    for beta >= 2.5,
 *   q  = 3.97156 - 4.14554 sqrt(1 - 0.26891 beta)  for 0.5 <= beta < 2.5,
 *   b0 = 1.57825 + 2.44413 q + 1.4281 q^2 + 0.422205 q^3,
 *   b1 = 2.44413 q + 2.85619 q^2 + 1.26661 q^3,
 *   b2 = -(1.4281 q^2 + 1.26661 q^3),
 *   b3 = 0.422205 q^3,
 *   B  = 1 - (b1 + b2 + b3) / b0.
 * c receives {B, b1/b0, b2/b0, b3/b0, q}. Returns -1 outside [0.5, 64]. */
int orc_iir_coeffs(double beta, double *c)
{
    if (!(beta >= 0.5) || !(beta <= 64.0))
        return -1;
    const double q = beta >= 2.5 ? 0.98711 * beta - 0.96330 : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * beta);
    const double q2 = q * q, q3 = q2 * q;
    const double b0 = 1.57825 + 2.44413 * q + 1.4281 * q2 + 0.422205 * q3;
    const double b1 = 2.44413 * q + 2.85619 * q2 + 1.26661 * q3;
    const double b2 = -(1.4281 * q2 + 1.26661 * q3);
    const double b3 = 0.422205 * q3;
    c[0] = 1.0 - (b1 + b2 + b3) / b0;
    c[1] = b1 / b0;
    c[2] = b2 / b0;
    c[3] = b3 / b0;
    c[4] = q;
    return 0;
}

/* Number of samples before (after) the first (last) output at which the causal
 * (anti-causal) pass starts from a zero state. For every beta in [0.5, 64] the
 * largest pole modulus rho of the filter satisfies rho^(80 q + 64) < exp(-89), so
 * the truncated tail lies far under double rounding. */
int64_t orc_iir_margin(double beta)
{
    double c[5];
    if (orc_iir_coeffs(beta, c) != 0)
        return -1;
    return (int64_t)ceil(80.0 * c[4]) + 64;
}

/* The Young-van Vliet filter of a finite sequence x[0..n) with a zero state
 * before x[0] and after x[n-1]:
 *   causal       w(m) = B x(m) + a1 w(m-1) + a2 w(m-2) + a3 w(m-3),
 *   anti-causal  y(m) = B w(m) + a1 y(m+1) + a2 y(m+2) + a3 y(m+3),
 * with (a1, a2, a3) = (b1, b2, b3) / b0. y may not alias x. */
int orc_iir_filter(const double *x, int64_t n, double beta, double *y)
{
    double c[5];
    if (n < 0 || orc_iir_coeffs(beta, c) != 0)
        return -1;
    const double B = c[0], a1 = c[1], a2 = c[2], a3 = c[3];
    double w1 = 0.0, w2 = 0.0, w3 = 0.0;
    for (int64_t m = 0; m < n; ++m) {
        const double w = B * x[m] + a1 * w1 + a2 * w2 + a3 * w3;
        y[m] = w;
        w3 = w2;
        w2 = w1;
        w1 = w;
    }
    double y1 = 0.0, y2 = 0.0, y3 = 0.0;
    for (int64_t m = n - 1; m >= 0; --m) {
        const double v = B * y[m] + a1 * y1 + a2 * y2 + a3 * y3;
        y[m] = v;
        y3 = y2;
        y2 = y1;
        y1 = v;
    }
    return 0;
}

/* Scale that turns the unit-gain recursive filter into the profile g_beta of
 * Eq. (3): the integral of exp(-x^2 / (2 beta^2)), beta sqrt(2 pi). */
static double iir_scale(double beta) { return beta * sqrt(2.0 * acos(-1.0)); }

/* Smoothing parameter rule used when the caller gives none:
 * h = sigma * sqrt(sum_k g(k)), which is sigma*sqrt(2K+1) for the box and
 * sigma*sqrt(beta sqrt(2 pi)) for the recursive Gaussian (unit DC gain times
 * the scale above). */
double orc_default_h(double sigma, int K, int profile, double beta)
{
    double g[2 * 64 + 1];
    if (profile == ORC_GAUSS_IIR) {
        double c[5];
        return orc_iir_coeffs(beta, c) == 0 ? sigma * sqrt(iir_scale(beta)) : -1.0;
    }
    if (K > 64)
        return -1.0;
    orc_profile(K, profile, beta, g);
    double s = 0.0;
    for (int k = 0; k <= 2 * K; ++k)
        s += g[k];
    return sigma * sqrt(s);
}

/* Copy one line (n samples, element stride `stride`) into the extended signal
 * fe[0 .. n + 2R), where fe[R + x] = f(ext(x)) for x in [-R, n + R). */
static void extend_line(const double *f, int64_t n, int64_t stride, int64_t R, double *fe)
{
    for (int64_t x = -R; x < n + R; ++x)
        fe[R + x] = f[orc_ext(x, n) * stride];
}

/* Eq. (3): squared patch distance between the patches centred at i and j of
 * the extended signal (fe is indexed with the offset R already added). */
static double patch_dist2(const double *fe, int64_t i, int64_t j, int K, const double *g)
{
    double d = 0.0;
    for (int k = -K; k <= K; ++k) {
        double a = fe[i + k] - fe[j + k];
        d += g[k + K] * a * a;
    }
    return d;
}

/* Distances of the recursive Gaussian profile for one line (n samples, element
 * stride `stride`): dtab[i*(2S+1) + (s+S)], i in [0, n), s in [-S, S], is
 * beta sqrt(2 pi) times the Young-van Vliet filter, along m, of the lifted
 * sequence (fe(m) - fe(m+s))^2 of the extended signal, both passes started
 * iir_margin(beta) samples outside [0, n). Returns -1 on a bad beta, -3 when out
 * of memory. */
static int iir_dist_table(const double *f, int64_t n, int64_t stride, int S, double beta, double *dtab)
{
    const int64_t M = orc_iir_margin(beta);
    if (M < 0)
        return -1;
    const int64_t R = M + S, L = n + 2 * M;
    double *fe = (double *)malloc(sizeof(double) * (size_t)(n + 2 * R));
    double *xs = (double *)malloc(sizeof(double) * (size_t)L);
    double *ys = (double *)malloc(sizeof(double) * (size_t)L);
    if (!fe || !xs || !ys) {
        free(fe); free(xs); free(ys);
        return -3;
    }
    extend_line(f, n, stride, R, fe);
    const double scale = iir_scale(beta);
    for (int s = -S; s <= S; ++s) {
        for (int64_t m = -M; m < n + M; ++m) {
            const double a = fe[R + m] - fe[R + m + s];
            xs[M + m] = a * a;
        }
        orc_iir_filter(xs, L, beta, ys);
        for (int64_t i = 0; i < n; ++i)
            dtab[i * (2 * S + 1) + (s + S)] = scale * ys[M + i];
    }
    free(fe); free(xs); free(ys);
    return 0;
}

/* Weights of the recursive profile at the lags s in [-S, S]: geff[s + S] =
 * beta sqrt(2 pi) times the two-pass impulse response at lag s, i.e. the weight of
 * the lifted square at i + s in d^2(i, .). Returns -1 on a bad beta, -3 when out of
 * memory. */
static int iir_lag_weights(double beta, int S, double *geff)
{
    const int64_t M = orc_iir_margin(beta);
    if (M < 0)
        return -1;
    const int64_t L = M + S, n = 2 * L + 1;
    double *x = (double *)calloc((size_t)n, sizeof(double));
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    if (!x || !y) {
        free(x); free(y);
        return -3;
    }
    x[L] = 1.0;
    orc_iir_filter(x, n, beta, y);
    for (int s = -S; s <= S; ++s)
        geff[s + S] = iir_scale(beta) * y[L + s];
    free(x); free(y);
    return 0;
}

/* Patch distances of n_lines signals of length N (row-major, line after line):
 * out[(line*N + i)*(2S+1) + (s+S)] = d^2(i, i+s) of Eq. (3), s in [-S, S]. */
int orc_patch_dist_1d(const double *x, int64_t n_lines, int64_t N, int S, int K, int profile,
                      double beta, double *out, int nthreads)
{
    if (profile == ORC_GAUSS_IIR) {
        if (N < 1 || S < 0 || n_lines < 0 || orc_iir_margin(beta) < 0)
            return -1;
        int rc = 0;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(min : rc)
        for (int64_t ln = 0; ln < n_lines; ++ln) {
            int r = iir_dist_table(x + ln * N, N, 1, S, beta, out + ln * N * (2 * S + 1));
            rc = r < rc ? r : rc;
        }
        return rc;
    }
    if (N < 1 || S < 0 || K < 0 || K > 64 || n_lines < 0)
        return -1;
    double g[2 * 64 + 1];
    orc_profile(K, profile, beta, g);
    const int64_t R = (int64_t)S + K;
    const int64_t L = N + 2 * R;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t ln = 0; ln < n_lines; ++ln) {
        double *fe = (double *)malloc(sizeof(double) * (size_t)L);
        extend_line(x + ln * N, N, 1, R, fe);
        for (int64_t i = 0; i < N; ++i)
            for (int s = -S; s <= S; ++s)
                out[(ln * N + i) * (2 * S + 1) + (s + S)] = patch_dist2(fe, R + i, R + i + s, K, g);
        free(fe);
    }
    return 0;
}

/* One-dimensional NLM of Eq. (4) with the divergence of Eq. (24) (the pair
 * that Alg. 3 computes), for one line with element strides:
 *   fhat(i)  = sum_j w_ij f(j) / W_i,   w_ij = exp(-d^2_ij / h^2),  |j-i| <= S
 *   dout(i)  = din(i) * dfhat(i)/df(i)   (the chaining used by Alg. 4)
 * with d^2 from Eq. (3). `din` may alias `dout`; either may be NULL together. */
static void nlm_line(const double *f, int64_t N, int64_t stride, const double *din, double *fhat,
                     double *dout, int64_t ostride, int S, int K, double h, const double *g,
                     const double *dtab, const double *geff, double *fe /* scratch, N + 2(S+K) */)
{
    /* dtab, geff (recursive Gaussian profile only): the distances of iir_dist_table,
     * used in place of the (2K+1)-tap sums, and the profile's weight at each lag
     * s in [-S, S] (geff[s + S]), which Eq. (24) needs in place of g. */
    const int64_t R = (int64_t)S + K;
    extend_line(f, N, stride, R, fe);
    const double h2 = h * h;
    /* patch-overlap offsets that lie in the window: |s| <= K for the (2K+1)-tap
     * profiles, the whole window for the recursive one (its support is unbounded) */
    const int KT = geff ? S : (K < S ? K : S);
    /* weight of the centre tap: g(0) = 1 for the tap profiles */
    const double g0 = geff ? geff[S] : 1.0;
    for (int64_t i = 0; i < N; ++i) {
        const int64_t ci = R + i;
        double W = 0.0, P1 = 0.0, P2 = 0.0;
        for (int s = -S; s <= S; ++s) {
            const double d2 = dtab ? dtab[i * (2 * S + 1) + (s + S)] : patch_dist2(fe, ci, ci + s, K, g);
            double w = exp(-d2 / h2);
            double fj = fe[ci + s];
            W += w;
            P1 += w * fj;
            P2 += w * fj * fj;
        }
        const double fh = P1 / W;
        fhat[i * ostride] = fh;
        if (dout) {
            /* Last term of Eq. (24): sum over the offsets where the patches of i and j
             * share the sample f(i) of w_ij g(i-j) (f(j) - fhat(i)) (f(2i-j) - f(i)). */
            double T = 0.0;
            for (int s = -KT; s <= KT; ++s) {
                const double d2 = dtab ? dtab[i * (2 * S + 1) + (s + S)] : patch_dist2(fe, ci, ci + s, K, g);
                const double gs = geff ? geff[-s + S] : g[-s + K];
                T += exp(-d2 / h2) * gs * (fe[ci + s] - fh) * (fe[ci - s] - fe[ci]);
            }
            /* Eq. (24); its first terms carry the centre weight g(0), which is 1 for the
             * tap profiles (the general form of d d^2_ij / d f(i) = 2 g(0) (f(i) - f(j))
             * - 2 g(i-j) (f(2i-j) - f(i))) */
            double div = 2.0 * g0 / (h2 * W) * P2 + 1.0 / W - 2.0 * g0 / h2 * fh * fh + 2.0 / (W * h2) * T;
            double d0 = din ? din[i * ostride] : 1.0;
            dout[i * ostride] = d0 * div;
        }
    }
}

/* Eq. (4) (+ Eq. (24)) applied to n_lines contiguous signals of length N.
 * delta_in may be NULL (taken as ones); delta_out may be NULL (not computed). */
int orc_nlm_1d(const double *x, int64_t n_lines, int64_t N, int S, int K, double h, int profile,
               double beta, const double *delta_in, double *fhat, double *delta_out, int nthreads)
{
    if (N < 1 || S < 0 || K < 0 || K > 64 || !(h > 0.0) || n_lines < 0)
        return -1;
    const int iir = profile == ORC_GAUSS_IIR;
    if (iir && orc_iir_margin(beta) < 0)
        return -1;
    double g[2 * 64 + 1];
    orc_profile(K, profile, beta, g);
    double *geff = iir ? (double *)malloc(sizeof(double) * (size_t)(2 * S + 1)) : NULL;
    if (iir && (!geff || iir_lag_weights(beta, S, geff) != 0)) {
        free(geff);
        return -3;
    }
    const int64_t L = N + 2 * ((int64_t)S + K);
    int rc = 0;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(min : rc)
    for (int64_t ln = 0; ln < n_lines; ++ln) {
        double *fe = (double *)malloc(sizeof(double) * (size_t)L);
        double *dtab = iir ? (double *)malloc(sizeof(double) * (size_t)(N * (2 * S + 1))) : NULL;
        int r = (!fe || (iir && !dtab)) ? -3 : 0;
        if (r == 0 && iir)
            r = iir_dist_table(x + ln * N, N, 1, S, beta, dtab);
        if (r == 0)
            nlm_line(x + ln * N, N, 1, delta_in ? delta_in + ln * N : NULL, fhat + ln * N,
                     delta_out ? delta_out + ln * N : NULL, 1, S, K, h, g, dtab, geff, fe);
        rc = r < rc ? r : rc;
        free(fe);
        free(dtab);
    }
    free(geff);
    return rc;
}

/* Apply the 1-D map to every row (axis 0) or every column (axis 1) of an H x W
 * row-major image; the derivative sequence is chained in place (Alg. 4). */
static int sweep(const double *src, double *dst, double *delta, int64_t H, int64_t W, int axis,
                 int S, int K, double h, const double *g, int profile, double beta, int nthreads)
{
    const int64_t n_lines = axis == 0 ? H : W;
    const int64_t N = axis == 0 ? W : H;
    const int64_t line_step = axis == 0 ? W : 1;
    const int64_t elem_step = axis == 0 ? 1 : W;
    const int64_t L = N + 2 * ((int64_t)S + K);
    const int iir = profile == ORC_GAUSS_IIR;
    double *geff = iir ? (double *)malloc(sizeof(double) * (size_t)(2 * S + 1)) : NULL;
    if (iir && (!geff || iir_lag_weights(beta, S, geff) != 0)) {
        free(geff);
        return -3;
    }
    int rc = 0;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(min : rc)
    for (int64_t ln = 0; ln < n_lines; ++ln) {
        double *fe = (double *)malloc(sizeof(double) * (size_t)L);
        double *dtab = iir ? (double *)malloc(sizeof(double) * (size_t)(N * (2 * S + 1))) : NULL;
        int r = (!fe || (iir && !dtab)) ? -3 : 0;
        if (r == 0 && iir)
            r = iir_dist_table(src + ln * line_step, N, elem_step, S, beta, dtab);
        if (r == 0)
            nlm_line(src + ln * line_step, N, elem_step, delta ? delta + ln * line_step : NULL,
                     dst + ln * line_step, delta ? delta + ln * line_step : NULL, elem_step, S, K, h, g,
                     dtab, geff, fe);
        rc = r < rc ? r : rc;
        free(fe);
        free(dtab);
    }
    free(geff);
    return rc;
}

/* Minimum-norm solution of the symmetric 2x2 system [a c; c e] t = b.
 * Regular case: Cramer's rule. Singular case (det <= 1e-12 * trace^2): the
 * pseudo-inverse, i.e. the projection on the dominant eigenvector. */
static void solve2_sym(double a, double c, double e, const double *b, double *t)
{
    double det = a * e - c * c;
    double tr = a + e;
    if (det > 1e-12 * tr * tr) {
        t[0] = (e * b[0] - c * b[1]) / det;
        t[1] = (a * b[1] - c * b[0]) / det;
        return;
    }
    double half = 0.5 * (a - e);
    double lam = 0.5 * tr + sqrt(half * half + c * c);
    if (!(lam > 0.0)) {
        t[0] = t[1] = 0.0;
        return;
    }
    /* eigenvector of the largest eigenvalue */
    double v0, v1;
    if (fabs(c) > 0.0) {
        v0 = c;
        v1 = lam - a;
    } else if (a >= e) {
        v0 = 1.0;
        v1 = 0.0;
    } else {
        v0 = 0.0;
        v1 = 1.0;
    }
    double nv = sqrt(v0 * v0 + v1 * v1);
    v0 /= nv;
    v1 /= nv;
    double coef = (v0 * b[0] + v1 * b[1]) / lam;
    t[0] = coef * v0;
    t[1] = coef * v1;
}

/* Separable NLM, Alg. 4 (Sec. III):
 *   f_r  = rows(f),  f_rc = cols(f_r)   with delta_1 chained (Eq. (21))
 *   f_c  = cols(f),  f_cr = rows(f_c)   with delta_2 chained (Eq. (22))
 *   out  = theta_1 f_rc + theta_2 f_cr  (Eq. (14))
 * order RC: theta = (1,0); CR: (0,1); AVG: (1/2,1/2); SURE: A theta = b with
 * A from Eq. (19) and b from Eq. (25).
 * info (may be NULL) receives 10 doubles:
 *   theta1, theta2, A11, A12, A22, sum(f f_rc), sum(f f_cr), sum d1, sum d2, sigma^2. */
int orc_snlm(const double *img, int64_t H, int64_t W, int S, int K, double h, int profile,
             double beta, int order, double sigma, double *out, double *info, int nthreads)
{
    if (H < 1 || W < 1 || S < 0 || K < 0 || K > 64 || !(h > 0.0) || order < 0 || order > 3)
        return -1;
    if (order == ORC_SURE && !(sigma >= 0.0))
        return -1;
    if (profile == ORC_GAUSS_IIR && orc_iir_margin(beta) < 0)
        return -1;
    double g[2 * 64 + 1];
    orc_profile(K, profile, beta, g);
    const int64_t n = H * W;
    const int need_rc = order != ORC_CR;
    const int need_cr = order != ORC_RC;
    const int need_div = order == ORC_SURE;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    double *frc = need_rc ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    double *fcr = need_cr ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    double *d1 = need_div ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    double *d2 = need_div ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    if (!tmp || (need_rc && !frc) || (need_cr && !fcr) || (need_div && (!d1 || !d2))) {
        free(tmp); free(frc); free(fcr); free(d1); free(d2);
        return -3;
    }
    if (need_div)
        for (int64_t p = 0; p < n; ++p)
            d1[p] = d2[p] = 1.0;
    int rc = 0;
    if (need_rc) {
        rc = sweep(img, tmp, d1, H, W, 0, S, K, h, g, profile, beta, nthreads); /* f_r  */
        if (rc == 0)
            rc = sweep(tmp, frc, d1, H, W, 1, S, K, h, g, profile, beta, nthreads); /* f_rc */
    }
    if (need_cr && rc == 0) {
        rc = sweep(img, tmp, d2, H, W, 1, S, K, h, g, profile, beta, nthreads); /* f_c  */
        if (rc == 0)
            rc = sweep(tmp, fcr, d2, H, W, 0, S, K, h, g, profile, beta, nthreads); /* f_cr */
    }
    if (rc != 0) {
        free(tmp); free(frc); free(fcr); free(d1); free(d2);
        return rc;
    }
    double th[2] = {0.0, 0.0};
    double A11 = 0, A12 = 0, A22 = 0, Bf1 = 0, Bf2 = 0, Sd1 = 0, Sd2 = 0;
    if (order == ORC_RC) {
        th[0] = 1.0;
    } else if (order == ORC_CR) {
        th[1] = 1.0;
    } else if (order == ORC_AVG) {
        th[0] = th[1] = 0.5;
    } else {
        for (int64_t p = 0; p < n; ++p) {
            A11 += frc[p] * frc[p];
            A12 += frc[p] * fcr[p];
            A22 += fcr[p] * fcr[p];
            Bf1 += img[p] * frc[p];
            Bf2 += img[p] * fcr[p];
            Sd1 += d1[p];
            Sd2 += d2[p];
        }
        double b[2] = {Bf1 - sigma * sigma * Sd1, Bf2 - sigma * sigma * Sd2};
        solve2_sym(A11, A12, A22, b, th);
    }
    for (int64_t p = 0; p < n; ++p) {
        double v = 0.0;
        if (need_rc)
            v += th[0] * frc[p];
        if (need_cr)
            v += th[1] * fcr[p];
        out[p] = v;
    }
    if (info) {
        info[0] = th[0]; info[1] = th[1];
        info[2] = A11; info[3] = A12; info[4] = A22;
        info[5] = Bf1; info[6] = Bf2; info[7] = Sd1; info[8] = Sd2;
        info[9] = sigma * sigma;
    }
    free(tmp); free(frc); free(fcr); free(d1); free(d2);
    return 0;
}

/* Intermediate images of Alg. 4 for tests: f_r, f_rc, f_c, f_cr and the two
 * chained derivative maps delta_1, delta_2 (each H*W, any may be NULL). */
int orc_snlm_parts(const double *img, int64_t H, int64_t W, int S, int K, double h, int profile,
                   double beta, double *fr, double *frc, double *fc, double *fcr, double *d1,
                   double *d2, int nthreads)
{
    if (H < 1 || W < 1 || S < 0 || K < 0 || K > 64 || !(h > 0.0))
        return -1;
    if (profile == ORC_GAUSS_IIR && orc_iir_margin(beta) < 0)
        return -1;
    double g[2 * 64 + 1];
    orc_profile(K, profile, beta, g);
    const int64_t n = H * W;
    double *a = (double *)malloc(sizeof(double) * (size_t)n);
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    double *da = (double *)malloc(sizeof(double) * (size_t)n);
    double *db = (double *)malloc(sizeof(double) * (size_t)n);
    if (!a || !b || !da || !db) {
        free(a); free(b); free(da); free(db);
        return -3;
    }
    for (int64_t p = 0; p < n; ++p)
        da[p] = db[p] = 1.0;
    int rc = sweep(img, a, da, H, W, 0, S, K, h, g, profile, beta, nthreads);
    if (fr) memcpy(fr, a, sizeof(double) * (size_t)n);
    if (rc == 0) rc = sweep(a, b, da, H, W, 1, S, K, h, g, profile, beta, nthreads);
    if (frc) memcpy(frc, b, sizeof(double) * (size_t)n);
    if (d1) memcpy(d1, da, sizeof(double) * (size_t)n);
    if (rc == 0) rc = sweep(img, a, db, H, W, 1, S, K, h, g, profile, beta, nthreads);
    if (fc) memcpy(fc, a, sizeof(double) * (size_t)n);
    if (rc == 0) rc = sweep(a, b, db, H, W, 0, S, K, h, g, profile, beta, nthreads);
    if (fcr) memcpy(fcr, b, sizeof(double) * (size_t)n);
    if (d2) memcpy(d2, db, sizeof(double) * (size_t)n);
    free(a); free(b); free(da); free(db);
    return rc;
}

/* Non-local means of Eqs. (1)-(2) (Sec. I), the comparison workload of the run-time
 * tables of Sec. IV-B: at pixel i, the average of f(j) over the (2Sy+1) x (2Sx+1)
 * window centred at i, weighted by exp(-(1/h^2) sum_{k in P} G(k) (f(i+k) - f(j+k))^2)
 * with P = [-Ky, Ky] x [-Kx, Kx] and G(k1, k2) = g(k1) g(k2) (box: 1; Gaussian:
 * exp(-(k1^2 + k2^2) / (2 alpha^2)), the product of the 1-D profiles). Samples are
 * read through the symmetric extension (the boundary reading of the 1-D passes,
 * applied along each axis). Direct evaluation, O(S^2 K^2) per pixel. */
int orc_nlm_2d(const double *img, int64_t H, int64_t W, int Sy, int Sx, int Ky, int Kx, double h, int profile,
               double alpha, double *out, int nthreads)
{
    if (H < 1 || W < 1 || Sy < 0 || Sx < 0 || Ky < 0 || Kx < 0 || Ky > 64 || Kx > 64 || !(h > 0.0) ||
        (profile != ORC_BOX && profile != ORC_GAUSS))
        return -1;
    double gy[2 * 64 + 1], gx[2 * 64 + 1];
    orc_profile(Ky, profile, alpha, gy);
    orc_profile(Kx, profile, alpha, gx);
    const double ih2 = 1.0 / (h * h);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t y = 0; y < H; ++y) {
        for (int64_t x = 0; x < W; ++x) {
            double num = 0.0, den = 0.0;
            for (int64_t sy = -Sy; sy <= Sy; ++sy) {
                for (int64_t sx = -Sx; sx <= Sx; ++sx) {
                    double d = 0.0;
                    for (int64_t k1 = -Ky; k1 <= Ky; ++k1) {
                        const int64_t ri = orc_ext(y + k1, H), rj = orc_ext(y + sy + k1, H);
                        for (int64_t k2 = -Kx; k2 <= Kx; ++k2) {
                            const double a = img[ri * W + orc_ext(x + k2, W)];
                            const double b = img[rj * W + orc_ext(x + sx + k2, W)];
                            d += gy[k1 + Ky] * gx[k2 + Kx] * (a - b) * (a - b);
                        }
                    }
                    const double w = exp(-d * ih2);
                    num += w * img[orc_ext(y + sy, H) * W + orc_ext(x + sx, W)];
                    den += w;
                }
            }
            out[y * W + x] = num / den;
        }
    }
    return 0;
}

/* Parameters of the bilateral post-filter as functions of the noise level: the
 * cubic rules learnt in the parameter study (Sec. IV-A). */
void orc_bf_params(double sigma, double *sigma_s, double *sigma_r)
{
    const double s2 = sigma * sigma, s3 = s2 * sigma;
    *sigma_s = 2.5e-6 * s3 - 3.4e-4 * s2 + 0.021 * sigma + 0.46;
    *sigma_r = 2.8e-4 * s3 - 0.088 * s2 + 8.0 * sigma - 24.0;
}

/* Bilateral post-filter of Sec. III-B, Eq. (BF): at pixel i, the average of the
 * samples f(i - j) over the integer offsets j of Omega = [-3 sigma_s, 3 sigma_s]^2,
 * weighted by exp(-|j|^2 / (2 sigma_s^2)) * exp(-(f(i - j) - f(i))^2 / (2 sigma_r^2)).
 * Samples outside the image are read through the symmetric extension (the same
 * boundary reading as the NLM passes). Direct summation, one pixel at a time. */
int orc_bilateral(const double *img, int64_t H, int64_t W, double sigma_s, double sigma_r, double *out,
                  int nthreads)
{
    if (H < 1 || W < 1 || !(sigma_s > 0.0) || !(sigma_r > 0.0) || !isfinite(sigma_s))
        return -1;
    const int64_t R = (int64_t)floor(3.0 * sigma_s);
    if (R > 64)
        return -1;
    const double two_ss = 2.0 * sigma_s * sigma_s, two_sr = 2.0 * sigma_r * sigma_r;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t y = 0; y < H; ++y) {
        for (int64_t x = 0; x < W; ++x) {
            const double c = img[y * W + x];
            double num = 0.0, den = 0.0;
            for (int64_t jy = -R; jy <= R; ++jy) {
                for (int64_t jx = -R; jx <= R; ++jx) {
                    const double v = img[orc_ext(y - jy, H) * W + orc_ext(x - jx, W)];
                    const double ws = exp(-(double)(jx * jx + jy * jy) / two_ss);
                    const double gr = exp(-(v - c) * (v - c) / two_sr);
                    num += ws * gr * v;
                    den += ws * gr;
                }
            }
            out[y * W + x] = num / den;
        }
    }
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
