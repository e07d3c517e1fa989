// Recursive Gaussian profile (snlm_iir.cu): the declarations the API layer uses.
#pragma once

#include <cuda_runtime.h>

#include "snlm_internal.h"

namespace snlm {

// Distance mode of the recursive profile in launch-trace kinds (bits 8..11), next
// to DIST_SLIDE, DIST_BLOCK and DIST_FIR; its passes run in their own kernels.
constexpr int DIST_IIR = 3;

// Widths of the recursive Gaussian profile the library accepts: Young and van
// Vliet's rule for q holds from 0.5, and up to 3.5 (K = 7 at beta = K/2) the
// filter's history (58 samples at 3.5) fits the scan of one warp window (at most 64).
constexpr double kIirBetaMin = 0.5;
constexpr double kIirBetaMax = 3.5;

// iir_check_beta: SNLM_OK or SNLM_ERR_ARG.
// run_iir_pass: the 1-D NLM of Eq. (4) over n_lines lines of `src` into dst (fhat,
// or (fhat + blend) / 2 when blend is given).
// run_iir_dist: the distances d^2(x, x+s), s in [-S, S], as (n_lines, N, 2S+1) float32.
int iir_check_beta(double beta);
cudaError_t run_iir_pass(const Lines &src, int n_lines, int N, int S, double h, double beta, float *dst,
                         long long out_line_step, long long out_elem_step, const float *blend, cudaStream_t st);
cudaError_t run_iir_dist(const Lines &src, int n_lines, int N, int S, double beta, float *out, cudaStream_t st);
// run_iir_pass_sure: the pass with the divergence of Eq. (24) for the recursive
// profile (reading R17): delta_out = delta_in (NULL = 1) times the derivative of the
// pass, both indexed like dst (delta_in may alias delta_out).
cudaError_t run_iir_pass_sure(const Lines &src, int n_lines, int N, int S, double h, double beta, float *dst,
                              long long out_line_step, long long out_elem_step, const float *delta_in,
                              float *delta_out, cudaStream_t st);

}  // namespace snlm
