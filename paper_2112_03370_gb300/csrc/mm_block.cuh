// Block conjugate-gradient kernels (k_block.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

constexpr int kMaxBlk = 64;   // largest block width

// G (ta x tb, FP64) = A^T B over n pixels; A float32 block, B float32 or float64 block; idx_a / idx_b
// select block columns (null: identity); part holds nblk * kMaxBlk^2 doubles.
cudaError_t launch_bgram(const float* A, int ta, const int* idx_a, const void* B, int b_is_fp64,
                         int tb, const int* idx_b, int64_t n, double* part, int nblk, double* G,
                         cudaStream_t s);
// out_j (+)= sign * sum_i A_i C[i * ldc + j]; norms[j] = ||out_j||^2 when norm_part != null (FP64 out)
cudaError_t launch_bcombine(void* out, int out_is_fp64, const int* idx_out, int v, const float* A, int t,
                            const double* C, int ldc, double sign, int mode, int64_t n, double* norm_part,
                            int nblk, double* norms, cudaStream_t s);
// W_j = M_BD R_{idx[j]} (float32 out)
cudaError_t launch_bprecond(const double* minv, const double* R, const int* idx, int v, int64_t n,
                            float* W, cudaStream_t s);
// W_j = M_BD R_j (float32 block in and out, j < v)
cudaError_t launch_bprecond32(const double* minv, const float* R, int v, int64_t n, float* W, cudaStream_t s);
// enlarged CG: split of r (FP64 [n][4]) into t columns over contiguous pixel ranges (FP64 [t][n][4])
cudaError_t launch_bsplit(const double* r4, int t, int64_t n, double* R, cudaStream_t s);
// s = sum of the t columns of X; out (+)= s when out != null; *norm = ||s||^2
cudaError_t launch_bsum(const double* X, int t, int64_t n, double* out, int accumulate, double* norm_part,
                        int nblk, double* norm, cudaStream_t s);
// pivoted Cholesky of the t x t Gram matrix and the inverse of its factor (one CTA)
cudaError_t launch_bchol(const double* G, int t, double rank_tol, double* Linv, int* piv, int* rank,
                         cudaStream_t s);
// combine coefficients that turn a block Z into P = Z[piv] L^-T
cudaError_t launch_linv_coef(const double* Linv, const int* piv, const int* rank, int t, double* Cmb,
                             cudaStream_t s);

// R_j = B_j - AX_j and norms[j] = ||R_j||^2 (FP64 blocks)
cudaError_t launch_bresid(const double* B, const double* AX, int v, int64_t n, double* R,
                          double* norm_part, int nblk, double* norms, cudaStream_t s);

}  // namespace mm
