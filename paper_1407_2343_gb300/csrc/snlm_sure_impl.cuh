// Device helpers of the SURE combination (Sec. III-A, Alg. 4) shared by the
// single-image launches (snlm_sure.cu) and the batched persistent kernel.
#pragma once

#include "snlm_internal.h"

namespace snlm {

// Sum `n` records of kPartials doubles in a fixed order: thread t takes records
// t, t + 256, ... in sequence, then a fixed binary tree over threads.
__device__ __forceinline__ void reduce_records(const double *part, int n, double *sh, double out[kPartials])
{
    const int nt = blockDim.x;   // a power of two; sh holds kPartials * nt doubles
    double a[kPartials];
    for (int k = 0; k < kPartials; ++k)
        a[k] = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = 0; k < kPartials; ++k)
            a[k] += part[(long long)i * kPartials + k];
    for (int k = 0; k < kPartials; ++k)
        sh[k * nt + threadIdx.x] = a[k];
    __syncthreads();
    for (int stride = nt / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride)
            for (int k = 0; k < kPartials; ++k)
                sh[k * nt + threadIdx.x] += sh[k * nt + threadIdx.x + stride];
        __syncthreads();
    }
    for (int k = 0; k < kPartials; ++k)
        out[k] = sh[k * nt];
    __syncthreads();
}

// Minimum-norm solution of the symmetric 2x2 system [a c; c e] t = b: Cramer's
// rule when det > 1e-12 trace^2, else the projection on the dominant eigenvector.
__host__ __device__ inline void solve2_sym(double a, double c, double e, double b0, double b1, double *t0, double *t1)
{
    const double det = a * e - c * c, tr = a + e;
    if (det > 1e-12 * tr * tr) {
        *t0 = (e * b0 - c * b1) / det;
        *t1 = (a * b1 - c * b0) / det;
        return;
    }
    const double half = 0.5 * (a - e);
    const double lam = 0.5 * tr + sqrt(half * half + c * c);
    if (!(lam > 0.0)) {
        *t0 = *t1 = 0.0;
        return;
    }
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
    const double nv = sqrt(v0 * v0 + v1 * v1);
    v0 /= nv;
    v1 /= nv;
    const double coef = (v0 * b0 + v1 * b1) / lam;
    *t0 = coef * v0;
    *t1 = coef * v1;
}

// The SURE objective of Eq. (17) is minimised over f~ = theta1 f_rc + theta2 f_cr
// (Eq. (14)). It is solved here in the basis m = (f_rc + f_cr)/2, d = (f_rc - f_cr)/2,
// f~ = alpha m + beta d, theta1 = (alpha + beta)/2, theta2 = (alpha - beta)/2: the
// same minimiser (a linear change of variables; det/trace^2 is unchanged), but the
// sums that fix the nearly singular direction (beta) are made of the small
// differences d, so float32 per-pixel products keep them accurate.
// theta and the reported sums from the reduced records of the last pass of each
// order, solved in the basis m = (f_rc + f_cr)/2, d = (f_rc - f_cr)/2 (see the
// solve kernel in snlm_sure.cu for why).
// theta of Eqs. (19), (25) from the seven sums in the basis m, d:
// {sum m^2, sum m d, sum d^2, sum f m, sum f d, sum delta_1, sum delta_2}.
__host__ __device__ inline void sure_theta(const double *sums, double sigma2, double *t0, double *t1)
{
    const double smm = sums[0], smd = sums[1], sdd = sums[2], sfm = sums[3], sfd = sums[4];
    const double sd1 = sums[5], sd2 = sums[6];
    const double b0 = sfm - sigma2 * 0.5 * (sd1 + sd2);
    const double b1 = sfd - sigma2 * 0.5 * (sd1 - sd2);
    double al, be;
    solve2_sym(smm, smd, sdd, b0, b1, &al, &be);
    *t0 = 0.5 * (al + be);
    *t1 = 0.5 * (al - be);
}

__device__ __forceinline__ void sure_finish(const double rc[kPartials], const double cr[kPartials], double sigma2,
                                            double *info)
{
    const double smm = cr[0], smd = cr[1], sdd = cr[2], sfm = cr[3], sfd = cr[4];
    const double sd1 = rc[5], sd2 = cr[5];
    const double sums[7] = {smm, smd, sdd, sfm, sfd, sd1, sd2};
    sure_theta(sums, sigma2, &info[0], &info[1]);
    info[2] = smm + 2.0 * smd + sdd;   // sum f_rc^2       (A11 of Eq. (19))
    info[3] = smm - sdd;               // sum f_rc f_cr    (A12)
    info[4] = smm - 2.0 * smd + sdd;   // sum f_cr^2       (A22)
    info[5] = sfm + sfd;               // sum f f_rc       (Eq. (25))
    info[6] = sfm - sfd;               // sum f f_cr
    info[7] = sd1;                     // sum delta_1
    info[8] = sd2;                     // sum delta_2
    info[9] = sigma2;
}

// out[i] = theta1 frc[i] + theta2 out[i] for i in [lo, hi), theta split into float
// hi + lo parts so the weights keep ~48 bits.
__device__ __forceinline__ void combine_range(const float *__restrict__ frc, float *__restrict__ out,
                                              const double *__restrict__ info, long long lo, long long hi)
{
    const double t0 = info[0], t1 = info[1];
    const float h0 = (float)t0, h1 = (float)t1;
    const float l0 = (float)(t0 - (double)h0), l1 = (float)(t1 - (double)h1);
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
        out[i] = fmaf(h0, frc[i], fmaf(h1, out[i], fmaf(l0, frc[i], l1 * out[i])));
}

}  // namespace snlm
