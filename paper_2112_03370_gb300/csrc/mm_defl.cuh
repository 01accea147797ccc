// Two-level a-posteriori preconditioner (k_defl.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mm_cg.cuh"

namespace mm {

constexpr int kMaxDefl = 64;   // largest deflation space

struct DeflWork {
  int k;                 // columns of Z
  const float* Z;        // [k][n][4]
  const float* Zp;       // A Z, [k][n][4]
  const double* Einv;    // [k][k] pseudo-inverse of Z^T A Z
  double* y;             // [nrhs][kMaxDefl]
  double* part;          // [nrhs][n_blocks][kMaxDefl]
  double* part2;         // [nrhs][n_blocks]
  unsigned* counters;    // [nrhs]
  unsigned* counters2;   // [nrhs]
  int restart;           // 1: beta = 0 (restart from p = z), used after a residual replacement
};

// dot product of two FP64 vectors of n4 doubles into out[0] (deterministic)
cudaError_t launch_ldot(const double* a, const double* b, int64_t n4, double* part, int nblk,
                        double* out, cudaStream_t s);
// y = a x + b y
cudaError_t launch_laxpby(double a, const double* x, double b, double* y, int64_t n4, cudaStream_t s);
// eigen-decomposition of the Lanczos tridiagonal matrix (X row-major, columns = Ritz vectors)
cudaError_t launch_tridiag_eig(const double* alpha, const double* beta, int m, double* work, double* theta,
                               double* X, cudaStream_t s);
// symmetric pseudo-inverse (eigenvalues below rcond * max |w| dropped)
// 2lvl a-priori space: Z [n_int][n][4] float32 from the kept hits per time interval (hits:
// scratch int32 [n_int][n]); block_off: device [n_blocks + 1]
cudaError_t launch_apriori_z(const int32_t* lpix, const int64_t* block_off, int n_blocks, int n_int, int64_t n,
                             int32_t* hits, float* Z, cudaStream_t s);
cudaError_t launch_pinv_sym(const double* E, int k, double rcond, double* work, double* U, double* w,
                            double* Einv, cudaStream_t s);
// z = M_2lvl r for every column not halted, then <r, z> and beta (PCG scalars)
cudaError_t launch_defl_step(const DeflWork& d, const CgWork& w, cudaStream_t s);

}  // namespace mm
