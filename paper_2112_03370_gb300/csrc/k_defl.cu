// Two-level a-posteriori preconditioner (Sect. 3.2): Lanczos vector updates (Algorithm 3), the
// small symmetric eigenproblems, and the per-iteration application of Eq. 2lvlDef0
//     M_2lvl r = M_BD r - M_BD Z' E^-1 Z^T r + Z E^-1 Z^T r = M_BD (r - Z' y) + Z y,
//     y = E^-1 Z^T r,  Z' = A Z,  E = Z^T Z'.
// Z and Z' are float32 [k][n][4] blocks; r, z and the PCG scalars are float64.
#include "mm_cg.cuh"
#include "mm_defl.cuh"
#include "mm_internal.cuh"

namespace mm {

namespace {
constexpr int kNT = 256;

__device__ __forceinline__ double block_reduce(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kNT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}
}  // namespace

// ---------------------------------------------------------------------------------------------
// Lanczos (Algorithm 3) vector steps, FP64 vectors [n][4]
// ---------------------------------------------------------------------------------------------

// part[blk] = sum over this CTA of <a, b>
__global__ void k_ldot(const double* __restrict__ a, const double* __restrict__ b, int64_t n4,
                       double* __restrict__ part) {
  __shared__ double sh[kNT];
  double v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kNT)
    v += a[i] * b[i];
  v = block_reduce(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// out[0] = sum of part[0..nblk) (fixed order)
__global__ void k_lsum(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  __shared__ double sh[kNT];
  double v = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kNT) v += part[i];
  v = block_reduce(v, sh);
  if (threadIdx.x == 0) out[0] = v;
}

cudaError_t launch_ldot(const double* a, const double* b, int64_t n4, double* part, int nblk,
                        double* out, cudaStream_t s) {
  k_ldot<<<nblk, kNT, 0, s>>>(a, b, n4, part);
  k_lsum<<<1, kNT, 0, s>>>(part, nblk, out);
  return cudaGetLastError();
}

// y = a x + b y (FP64)
__global__ void k_laxpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n4) {
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kNT)
    y[i] = a * x[i] + b * y[i];
}

cudaError_t launch_laxpby(double a, const double* x, double b, double* y, int64_t n4, cudaStream_t s) {
  k_laxpby<<<4 * sm_count(), kNT, 0, s>>>(a, x, b, y, n4);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// small symmetric eigenproblems: cyclic Jacobi rotations (Golub & Van Loan, Sect. 8.5), one thread
// ---------------------------------------------------------------------------------------------

// T_m = tridiag(beta, alpha, beta) -> Ritz values theta and vectors X (row-major [m][m])
__global__ void k_tridiag_eig(const double* __restrict__ alpha, const double* __restrict__ beta, int m,
                              double* __restrict__ work, double* __restrict__ theta, double* __restrict__ X) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < m * m; i++) work[i] = 0.0;
  for (int i = 0; i < m; i++) {
    work[i * m + i] = alpha[i];
    if (i + 1 < m) {
      work[i * m + i + 1] = beta[i];
      work[(i + 1) * m + i] = beta[i];
    }
  }
  jacobi_eig(work, m, theta, X);
}

// Einv = pseudo-inverse of the symmetrised E (k x k): eigenvalues below rcond * max |w| dropped
__global__ void k_pinv_sym(const double* __restrict__ E, int k, double rcond, double* __restrict__ work,
                           double* __restrict__ U, double* __restrict__ w, double* __restrict__ Einv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < k; i++)
    for (int j = 0; j < k; j++) work[i * k + j] = 0.5 * (E[i * k + j] + E[j * k + i]);
  jacobi_eig(work, k, w, U);
  double mx = 0.0;
  for (int i = 0; i < k; i++) mx = fmax(mx, fabs(w[i]));
  for (int i = 0; i < k; i++)
    for (int j = 0; j < k; j++) {
      double s = 0.0;
      for (int l = 0; l < k; l++)
        if (fabs(w[l]) > rcond * mx) s += U[i * k + l] * U[j * k + l] / w[l];
      Einv[i * k + j] = s;
    }
}

cudaError_t launch_tridiag_eig(const double* alpha, const double* beta, int m, double* work, double* theta,
                               double* X, cudaStream_t s) {
  k_tridiag_eig<<<1, 32, 0, s>>>(alpha, beta, m, work, theta, X);
  return cudaGetLastError();
}

cudaError_t launch_pinv_sym(const double* E, int k, double rcond, double* work, double* U, double* w,
                            double* Einv, cudaStream_t s) {
  k_pinv_sym<<<1, 32, 0, s>>>(E, k, rcond, work, U, w, Einv);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// per-iteration application inside PCG
// ---------------------------------------------------------------------------------------------

// s = Z^T r per column (k dots) with deterministic partials; the last CTA forms y = E^-1 s.
__global__ void k_defl_dots(DeflWork d, CgWork w) {
  __shared__ double sh[kNT];
  __shared__ bool last;
  const int col = blockIdx.y;
  if (w.scal[col].halt) return;
  const double* r = w.r + (int64_t)col * w.n * 4;
  double* part = d.part + ((int64_t)col * gridDim.x + blockIdx.x) * kMaxDefl;
  for (int j = 0; j < d.k; j++) {
    const float4* z = reinterpret_cast<const float4*>(d.Z) + (int64_t)j * w.n;
    double v = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < w.n; p += (int64_t)gridDim.x * kNT) {
      const float4 zz = __ldg(z + p);
      v += (double)zz.x * r[4 * p] + (double)zz.y * r[4 * p + 1] + (double)zz.z * r[4 * p + 2];
    }
    v = block_reduce(v, sh);
    if (threadIdx.x == 0) part[j] = v;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(d.counters + col, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double sv[kMaxDefl];
  for (int j = threadIdx.x; j < d.k; j += kNT) {
    double acc = 0.0;
    for (unsigned b = 0; b < gridDim.x; b++)
      acc += reinterpret_cast<volatile double*>(d.part)[((int64_t)col * gridDim.x + b) * kMaxDefl + j];
    sv[j] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d.k; i += kNT) {
    double acc = 0.0;
    for (int j = 0; j < d.k; j++) acc += d.Einv[i * d.k + j] * sv[j];
    d.y[col * kMaxDefl + i] = acc;
  }
  if (threadIdx.x == 0) d.counters[col] = 0;
}

// z = M_BD (r - Z' y) + Z y; <r, z>; the last CTA sets rz and beta of the column.
__global__ void k_defl_apply(DeflWork d, CgWork w) {
  __shared__ double sh[kNT];
  __shared__ float ys[kMaxDefl];
  __shared__ bool last;
  const int col = blockIdx.y;
  if (w.scal[col].halt) return;
  for (int j = threadIdx.x; j < d.k; j += kNT) ys[j] = (float)d.y[col * kMaxDefl + j];
  __syncthreads();
  const double* r = w.r + (int64_t)col * w.n * 4;
  double* z = w.z + (int64_t)col * w.n * 4;
  double v = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < w.n; p += (int64_t)gridDim.x * kNT) {
    float zx = 0.f, zy = 0.f, zz = 0.f, qx = 0.f, qy = 0.f, qz = 0.f;
    for (int j = 0; j < d.k; j++) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(d.Z) + (int64_t)j * w.n + p);
      const float4 b = __ldg(reinterpret_cast<const float4*>(d.Zp) + (int64_t)j * w.n + p);
      zx = fmaf(a.x, ys[j], zx); zy = fmaf(a.y, ys[j], zy); zz = fmaf(a.z, ys[j], zz);
      qx = fmaf(b.x, ys[j], qx); qy = fmaf(b.y, ys[j], qy); qz = fmaf(b.z, ys[j], qz);
    }
    const double r0 = r[4 * p], r1 = r[4 * p + 1], r2 = r[4 * p + 2];
    const double u0 = r0 - qx, u1 = r1 - qy, u2 = r2 - qz;
    const double* m = w.minv + 6 * p;
    const double z0 = m[0] * u0 + m[1] * u1 + m[2] * u2 + zx;
    const double z1 = m[1] * u0 + m[3] * u1 + m[4] * u2 + zy;
    const double z2 = m[2] * u0 + m[4] * u1 + m[5] * u2 + zz;
    z[4 * p] = z0; z[4 * p + 1] = z1; z[4 * p + 2] = z2; z[4 * p + 3] = 0.0;
    v += r0 * z0 + r1 * z1 + r2 * z2;
  }
  v = block_reduce(v, sh);
  double* part = d.part2 + (int64_t)col * gridDim.x;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(d.counters2 + col, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kNT) acc += reinterpret_cast<volatile double*>(part)[b];
  acc = block_reduce(acc, sh);
  if (threadIdx.x == 0) {
    CgScalars& s = w.scal[col];
    s.rz = acc;
    // A-DEF1 is not symmetric: after a residual replacement the old direction is dropped
    s.beta = d.restart ? 0.0 : acc / s.rz_prev;
    d.counters2[col] = 0;
  }
}

// 2lvl a-priori space (Sect. 3.2): hits[j][p] += 1 for every kept sample of pixel p in time interval
// j = block mod n_int (blocks are detector-major); one grid row per block
__global__ void k_interval_hits(const int32_t* __restrict__ lpix, const int64_t* __restrict__ block_off,
                                int n_int, int64_t n, int32_t* __restrict__ hits) {
  const int b = blockIdx.y;
  const int64_t lo = block_off[b], hi = block_off[b + 1];
  int32_t* h = hits + (int64_t)(b % n_int) * n;
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = __ldg(lpix + i);
    if (p >= 0) atomicAdd(h + p, 1);
  }
}

// Z_j[p] = (s_p^j / s_p, 0, 0, 0): the fraction of pixel p's kept hits in interval j (I rows only)
__global__ void k_apriori_z(const int32_t* __restrict__ hits, int k, int64_t n, float4* __restrict__ Z) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t tot = 0;
    for (int j = 0; j < k; j++) tot += hits[(int64_t)j * n + p];
    const double inv = tot > 0 ? 1.0 / (double)tot : 0.0;
    for (int j = 0; j < k; j++) Z[(int64_t)j * n + p] = make_float4((float)(hits[(int64_t)j * n + p] * inv), 0.f, 0.f, 0.f);
  }
}

cudaError_t launch_apriori_z(const int32_t* lpix, const int64_t* block_off, int n_blocks, int n_int, int64_t n,
                             int32_t* hits, float* Z, cudaStream_t s) {
  if (n_blocks <= 0 || n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(hits, 0, (size_t)n_int * n * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  for (int b0 = 0; b0 < n_blocks; b0 += 65535) {   // gridDim.y limit
    const int nb = n_blocks - b0 < 65535 ? n_blocks - b0 : 65535;
    k_interval_hits<<<dim3(32, nb), 256, 0, s>>>(lpix, block_off + b0, n_int, n, hits);
  }
  int64_t g = (n + 255) / 256;
  if (g > 16 * sm_count()) g = 16 * sm_count();
  k_apriori_z<<<(unsigned)g, 256, 0, s>>>(hits, n_int, n, reinterpret_cast<float4*>(Z));
  return cudaGetLastError();
}

cudaError_t launch_defl_step(const DeflWork& d, const CgWork& w, cudaStream_t s) {
  dim3 grid(w.n_blocks, w.nrhs);
  k_defl_dots<<<grid, kNT, 0, s>>>(d, w);
  k_defl_apply<<<grid, kNT, 0, s>>>(d, w);
  return cudaGetLastError();
}

}  // namespace mm
