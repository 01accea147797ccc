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
// A (k x k, symmetric, row-major, destroyed) = U diag(w) U^T; U row-major [k][k] (columns = vectors)
__device__ inline void jacobi_eig(double* A, int k, double* w, double* U) {
  for (int i = 0; i < k; i++)
    for (int j = 0; j < k; j++) U[i * k + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < k; i++)
      for (int j = 0; j < k; j++) {
        tot += A[i * k + j] * A[i * k + j];
        if (i != j) off += A[i * k + j] * A[i * k + j];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < k - 1; p++)
      for (int q = p + 1; q < k; q++) {
        const double apq = A[p * k + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * k + q] - A[p * k + p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < k; r++) {   // A <- A J (columns p, q)
          const double arp = A[r * k + p], arq = A[r * k + q];
          A[r * k + p] = c * arp - s * arq;
          A[r * k + q] = s * arp + c * arq;
        }
        for (int r = 0; r < k; r++) {   // A <- J^T A (rows p, q)
          const double apr = A[p * k + r], aqr = A[q * k + r];
          A[p * k + r] = c * apr - s * aqr;
          A[q * k + r] = s * apr + c * aqr;
        }
        for (int r = 0; r < k; r++) {   // U <- U J
          const double urp = U[r * k + p], urq = U[r * k + q];
          U[r * k + p] = c * urp - s * urq;
          U[r * k + q] = s * urp + c * urq;
        }
      }
  }
  for (int i = 0; i < k; i++) w[i] = A[i * k + i];
}

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
