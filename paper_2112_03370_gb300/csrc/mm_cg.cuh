// Device state of the PCG loop (Algorithm 1), shared by the CG kernels and the host driver.
#pragma once

#include <stdint.h>

#include <cuda_runtime.h>

namespace mm {

// Scalars of one right-hand side, resident on the device so the loop needs no host round trip.
struct CgScalars {
  double bnorm2;    // ||b||^2
  double rz;        // <r_k, z_k>
  double rz_prev;   // <r_{k-1}, z_{k-1}>
  double pq;        // <p_k, A p_k>
  double alpha;
  double beta;
  double rr;        // ||r||^2 (recursive, or true after a replacement)
  double rr_true;   // ||b - A x||^2 from an FP64 A-application
  int32_t halt;     // skip all work of this column (done or paused)
  int32_t done;     // finished (converged or failed)
  int32_t paused;   // FP32 path: recursive residual below tol, waiting for the FP64 check
  int32_t status;   // mm_status
  int32_t iters;
  int32_t n_true;   // FP64 true-residual evaluations
  int32_t since_rep;
  int32_t restart_req;   // FP32 path: the next residual replacement restarts from p = z
};
static_assert(sizeof(CgScalars) == 96, "layout");
constexpr int kScalStrideInts = (int)(sizeof(CgScalars) / sizeof(int32_t));
constexpr int kHaltOffsetInts = 16;   // offsetof(CgScalars, halt) / 4
constexpr int kDoneOffsetInts = 17;

struct CgWork {
  int64_t n;          // pixels (n_obs)
  int32_t nrhs;
  int32_t n_blocks;   // CTAs per column of the reduction kernels
  int32_t fp32;       // mixed-precision path
  double tol2;        // eps^2
  int32_t max_iter;   // a column stops with MM_ENOTCONV after this many iterations
  const double* minv; // [n][6]
  const double* b;    // [nrhs][n][4]
  double* x;
  double* r;
  double* z;
  double* p;
  double* q;          // A p (FP64 path) or A x (replacement / true residual)
  float* p32;         // [nrhs][n][4] (FP32 path)
  float* q32;
  double* partials;   // [nrhs][n_blocks][4]
  unsigned* counters; // [nrhs]
  CgScalars* scal;    // [nrhs]
};

enum CgKernel { CG_INIT, CG_PUPDATE, CG_DOT_PQ, CG_UPDATE, CG_REPLACE, CG_TRUE_RES };

cudaError_t launch_cg(CgKernel k, const CgWork& w, cudaStream_t s);
int cg_blocks_for(int64_t n);

}  // namespace mm
