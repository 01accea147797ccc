// Pixel-domain and time-domain elementwise kernels: P / P^T in FP64, the banded Toeplitz product by
// its definition, block-Jacobi apply, layout conversions and the fused CG kernels of Algorithm 1.
#include "mm_internal.cuh"
#include "mm_cg.cuh"

namespace mm {

namespace {
constexpr int kNT = 256;
inline unsigned grid_for(int64_t n, int per = kNT, unsigned cap = 0) {
  if (cap == 0) cap = 32u * (unsigned)sm_count();
  int64_t g = (n + per - 1) / per;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}
}  // namespace

// ---------------------------------------------------------------------------------------------
// N^-1 by the definition (stbmm): y_i = sum_{j in block(i), |i-j| <= lambda} c_|i-j| t_j.
// O(lambda) per sample; used for checks and tiny bands.
// ---------------------------------------------------------------------------------------------
__global__ void k_toeplitz_direct(const double* __restrict__ band, const int64_t* __restrict__ off,
                                  int32_t n_blocks, int32_t lambda, int64_t N,
                                  const double* __restrict__ t, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_blocks;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
    }
    const int b = lo;
    const int64_t b0 = off[b], b1 = off[b + 1];
    const double* c = band + (int64_t)b * (lambda + 1);
    double acc = c[0] * t[i];
    const int64_t kmax_l = min((int64_t)lambda, i - b0);
    const int64_t kmax_r = min((int64_t)lambda, b1 - 1 - i);
    for (int64_t k = 1; k <= kmax_l; k++) acc = fma(c[k], t[i - k], acc);
    for (int64_t k = 1; k <= kmax_r; k++) acc = fma(c[k], t[i + k], acc);
    y[i] = acc;
  }
}

cudaError_t launch_toeplitz_direct(const double* band, const int64_t* block_off, int32_t n_blocks,
                                   int32_t lambda, int64_t N, const double* t, double* y,
                                   cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_toeplitz_direct<<<grid_for(N), kNT, 0, s>>>(band, block_off, n_blocks, lambda, N, t, y);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// P and P^T (Sect. 3.1 un-pointing / pointing), FP64, map in the padded [n_obs][4] layout.
// ---------------------------------------------------------------------------------------------
__global__ void k_unpoint64(const int32_t* __restrict__ lpix, const double2* __restrict__ w64, int64_t N,
                            const double* __restrict__ x4, double* __restrict__ t) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = lpix[i];
    double v = 0.0;
    if (p >= 0) {
      const double2 w = w64[i];
      const double* m = x4 + 4 * (int64_t)p;
      v = m[0] + w.x * m[1] + w.y * m[2];
    }
    t[i] = v;
  }
}

__global__ void k_point64(const int32_t* __restrict__ lpix, const double2* __restrict__ w64, int64_t N,
                          const double* __restrict__ t, double* __restrict__ y4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = lpix[i];
    if (p < 0) continue;
    const double2 w = w64[i];
    const double v = t[i];
    double* m = y4 + 4 * (int64_t)p;
    atomicAdd(m, v);
    atomicAdd(m + 1, w.x * v);
    atomicAdd(m + 2, w.y * v);
  }
}

cudaError_t launch_unpoint64(const int32_t* lpix, const double2* w64, int64_t N, const double* x4,
                             double* t, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_unpoint64<<<grid_for(N), kNT, 0, s>>>(lpix, w64, N, x4, t);
  return cudaGetLastError();
}

cudaError_t launch_point64(const int32_t* lpix, const double2* w64, int64_t N, const double* t,
                           double* y4, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_point64<<<grid_for(N), kNT, 0, s>>>(lpix, w64, N, t, y4);
  return cudaGetLastError();
}

__global__ void k_mask_d(const int32_t* __restrict__ lpix, const void* __restrict__ d, int is32,
                         int64_t N, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = is32 ? (double)reinterpret_cast<const float*>(d)[i]
                          : reinterpret_cast<const double*>(d)[i];
    out[i] = lpix[i] >= 0 ? v : 0.0;
  }
}

cudaError_t launch_mask_d(const int32_t* lpix, const void* d, int d_is_fp32, int64_t N, double* out,
                          cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_mask_d<<<grid_for(N), kNT, 0, s>>>(lpix, d, d_is_fp32, N, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// layout conversions: ABI [nrhs][n][3] <-> internal padded [nrhs][n][4]; FP64 <-> FP32
// ---------------------------------------------------------------------------------------------
__global__ void k_pack3to4(const double* __restrict__ x3, int64_t n_tot, double* __restrict__ x4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    x4[4 * i] = x3[3 * i];
    x4[4 * i + 1] = x3[3 * i + 1];
    x4[4 * i + 2] = x3[3 * i + 2];
    x4[4 * i + 3] = 0.0;
  }
}

__global__ void k_unpack4to3(const double* __restrict__ x4, int64_t n_tot, double* __restrict__ x3) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    x3[3 * i] = x4[4 * i];
    x3[3 * i + 1] = x4[4 * i + 1];
    x3[3 * i + 2] = x4[4 * i + 2];
  }
}

cudaError_t launch_pack3to4(const double* x3, int64_t n, int nrhs, double* x4, cudaStream_t s) {
  const int64_t tot = n * nrhs;
  if (tot == 0) return cudaSuccess;
  k_pack3to4<<<grid_for(tot), kNT, 0, s>>>(x3, tot, x4);
  return cudaGetLastError();
}

cudaError_t launch_unpack4to3(const double* x4, int64_t n, int nrhs, double* x3, cudaStream_t s) {
  const int64_t tot = n * nrhs;
  if (tot == 0) return cudaSuccess;
  k_unpack4to3<<<grid_for(tot), kNT, 0, s>>>(x4, tot, x3);
  return cudaGetLastError();
}

__global__ void k_to32(const double* __restrict__ x, int64_t n4, float* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = reinterpret_cast<const double2*>(x)[2 * i];
    const double2 b = reinterpret_cast<const double2*>(x)[2 * i + 1];
    reinterpret_cast<float4*>(y)[i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}

__global__ void k_to64(const float* __restrict__ x, int64_t n4, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = reinterpret_cast<const float4*>(x)[i];
    reinterpret_cast<double2*>(y)[2 * i] = make_double2(a.x, a.y);
    reinterpret_cast<double2*>(y)[2 * i + 1] = make_double2(a.z, a.w);
  }
}

cudaError_t launch_to32(const double* x4, int64_t n4, float* y4, cudaStream_t s) {
  if (n4 == 0) return cudaSuccess;
  k_to32<<<grid_for(n4), kNT, 0, s>>>(x4, n4, y4);
  return cudaGetLastError();
}

cudaError_t launch_to64(const float* x4, int64_t n4, double* y4, cudaStream_t s) {
  if (n4 == 0) return cudaSuccess;
  k_to64<<<grid_for(n4), kNT, 0, s>>>(x4, n4, y4);
  return cudaGetLastError();
}

// map [n_pix][3] (pre-zeroed) at obs_to_global[i] <- x [n_obs][4]
__global__ void k_to_global(const double* __restrict__ x4, const int32_t* __restrict__ o2g, int64_t n,
                            double* __restrict__ map3) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = o2g[i];
    map3[3 * p] = x4[4 * i];
    map3[3 * p + 1] = x4[4 * i + 1];
    map3[3 * p + 2] = x4[4 * i + 2];
  }
}

cudaError_t launch_to_global(const double* x4, const int32_t* o2g, int64_t n, double* map3, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_to_global<<<grid_for(n), kNT, 0, s>>>(x4, o2g, n, map3);
  return cudaGetLastError();
}

// z = M_BD r per pixel (symmetric 3x3 stored as 00 01 02 11 12 22)
__device__ __forceinline__ void bd3(const double* __restrict__ m, double r0, double r1, double r2,
                                    double& z0, double& z1, double& z2) {
  const double a00 = m[0], a01 = m[1], a02 = m[2], a11 = m[3], a12 = m[4], a22 = m[5];
  z0 = a00 * r0 + a01 * r1 + a02 * r2;
  z1 = a01 * r0 + a11 * r1 + a12 * r2;
  z2 = a02 * r0 + a12 * r1 + a22 * r2;
}

__global__ void k_bd_apply(const double* __restrict__ minv, int64_t n, int nrhs,
                           const double* __restrict__ r4, double* __restrict__ z4) {
  const int64_t tot = n * nrhs;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % n;
    const double* r = r4 + 4 * i;
    double z0, z1, z2;
    bd3(minv + 6 * p, r[0], r[1], r[2], z0, z1, z2);
    double* z = z4 + 4 * i;
    z[0] = z0; z[1] = z1; z[2] = z2; z[3] = 0.0;
  }
}

cudaError_t launch_bd_apply(const double* minv, int64_t n, int nrhs, const double* r4, double* z4,
                            cudaStream_t s) {
  if (n * nrhs == 0) return cudaSuccess;
  k_bd_apply<<<grid_for(n * nrhs), kNT, 0, s>>>(minv, n, nrhs, r4, z4);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Algorithm 1 (PCG), one column per blockIdx.y.  Dot products are reduced deterministically:
// fixed per-thread order, a fixed shared-memory tree per CTA, and the last CTA to finish sums
// the CTA partials in index order and updates the column's scalars on the device.
// ---------------------------------------------------------------------------------------------
namespace {

template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double (*sh)[kNT]) {
#pragma unroll
  for (int k = 0; k < K; k++) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int s = kNT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < K; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < K; k++) v[k] = sh[k][0];
}

// Writes this CTA's K partial sums; returns true in exactly one CTA per column (the last one),
// in which `tot` then holds the column totals.
template <int K>
__device__ bool grid_sum(double (&v)[K], const CgWork& w, int col, double (&tot)[K]) {
  __shared__ double sh[K][kNT];
  __shared__ bool last;
  block_sum<K>(v, sh);
  double* part = w.partials + ((int64_t)col * gridDim.x) * 4;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) part[4 * blockIdx.x + k] = v[k];
    __threadfence();
    const unsigned prev = atomicAdd(w.counters + col, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; k++) acc[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kNT) {
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] += reinterpret_cast<volatile double*>(part)[4 * b + k];
  }
  block_sum<K>(acc, sh);
#pragma unroll
  for (int k = 0; k < K; k++) tot[k] = acc[k];
  if (threadIdx.x == 0) w.counters[col] = 0;
  return true;
}

__device__ __forceinline__ const double* col4(const double* base, const CgWork& w, int col) {
  return base + (int64_t)col * w.n * 4;
}
__device__ __forceinline__ double* col4(double* base, const CgWork& w, int col) {
  return base + (int64_t)col * w.n * 4;
}

}  // namespace

// r = b, z = M r, x = 0, p = 0, beta = 0; ||b||^2 and <r, z>.
__global__ void k_cg_init(CgWork w) {
  const int col = blockIdx.y;
  const double* b = col4(w.b, w, col);
  double* x = col4(w.x, w, col);
  double* r = col4(w.r, w, col);
  double* z = col4(w.z, w, col);
  double* p = col4(w.p, w, col);
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * kNT) {
    const double r0 = b[4 * i], r1 = b[4 * i + 1], r2 = b[4 * i + 2];
    double z0, z1, z2;
    bd3(w.minv + 6 * i, r0, r1, r2, z0, z1, z2);
    r[4 * i] = r0; r[4 * i + 1] = r1; r[4 * i + 2] = r2; r[4 * i + 3] = 0.0;
    z[4 * i] = z0; z[4 * i + 1] = z1; z[4 * i + 2] = z2; z[4 * i + 3] = 0.0;
    x[4 * i] = 0.0; x[4 * i + 1] = 0.0; x[4 * i + 2] = 0.0; x[4 * i + 3] = 0.0;
    p[4 * i] = 0.0; p[4 * i + 1] = 0.0; p[4 * i + 2] = 0.0; p[4 * i + 3] = 0.0;
    v[0] += r0 * r0 + r1 * r1 + r2 * r2;
    v[1] += r0 * z0 + r1 * z1 + r2 * z2;
  }
  double t[2];
  if (grid_sum<2>(v, w, col, t) && threadIdx.x == 0) {
    CgScalars& s = w.scal[col];
    s.bnorm2 = t[0];
    s.halt = 0;
    s.rr = t[0];
    s.rz = t[1];
    s.rz_prev = t[1];
    s.beta = 0.0;
    s.alpha = 0.0;
    s.pq = 0.0;
    s.rr_true = t[0];
    s.iters = 0;
    s.n_true = 0;
    s.since_rep = 0;
    s.restart_req = 0;
    s.status = MM_OK;
    s.paused = 0;
    s.done = (t[0] == 0.0) ? 1 : 0;
    if (!s.done && w.max_iter <= 0) {
      s.status = MM_ENOTCONV;
      s.done = 1;
    }
    s.halt = s.done;
  }
}

// p = z + beta p; zero the A-apply accumulator (q, or q32 and p32 = (float) p on the FP32 path).
__global__ void k_cg_pupdate(CgWork w) {
  const int col = blockIdx.y;
  const CgScalars& s = w.scal[col];
  if (s.halt) return;
  const double beta = s.beta;
  const double* z = col4(w.z, w, col);
  double* p = col4(w.p, w, col);
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * kNT) {
    const double2 z01 = reinterpret_cast<const double2*>(z)[2 * i];
    const double z2 = z[4 * i + 2];
    double2 p01 = reinterpret_cast<double2*>(p)[2 * i];
    double p2 = p[4 * i + 2];
    p01.x = z01.x + beta * p01.x;
    p01.y = z01.y + beta * p01.y;
    p2 = z2 + beta * p2;
    reinterpret_cast<double2*>(p)[2 * i] = p01;
    reinterpret_cast<double2*>(p)[2 * i + 1] = make_double2(p2, 0.0);
    if (w.fp32) {
      reinterpret_cast<float4*>(w.p32)[(int64_t)col * w.n + i] =
          make_float4((float)p01.x, (float)p01.y, (float)p2, 0.f);
      reinterpret_cast<float4*>(w.q32)[(int64_t)col * w.n + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      double* q = col4(w.q, w, col);
      reinterpret_cast<double2*>(q)[2 * i] = make_double2(0.0, 0.0);
      reinterpret_cast<double2*>(q)[2 * i + 1] = make_double2(0.0, 0.0);
    }
  }
}

__device__ __forceinline__ void load_q(const CgWork& w, int col, int64_t i, double& q0, double& q1,
                                       double& q2) {
  if (w.fp32) {
    const float4 v = reinterpret_cast<const float4*>(w.q32)[(int64_t)col * w.n + i];
    q0 = v.x; q1 = v.y; q2 = v.z;
  } else {
    const double* q = col4(w.q, w, col) + 4 * i;
    q0 = q[0]; q1 = q[1]; q2 = q[2];
  }
}

// <p, A p> and alpha = <r, z> / <p, A p>
__global__ void k_cg_dot_pq(CgWork w) {
  const int col = blockIdx.y;
  if (w.scal[col].halt) return;
  const double* p = col4(w.p, w, col);
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * kNT) {
    double q0, q1, q2;
    load_q(w, col, i, q0, q1, q2);
    v[0] += p[4 * i] * q0 + p[4 * i + 1] * q1 + p[4 * i + 2] * q2;
  }
  double t[1];
  if (grid_sum<1>(v, w, col, t) && threadIdx.x == 0) {
    CgScalars& s = w.scal[col];
    s.pq = t[0];
    const double alpha = s.rz / t[0];
    if (!(t[0] > 0.0) || !isfinite(alpha)) {
      s.alpha = 0.0;
      if (w.fp32 && s.since_rep > 0 && isfinite(t[0])) {
        // FP32 operator noise along a (near-)null direction of a semi-definite A (e.g. a map offset
        // degenerate with templates): restart from the FP64-class true residual instead of failing
        s.paused = 1;
        s.restart_req = 1;
        s.halt = 1;
      } else {
        s.status = MM_EBREAKDOWN;
        s.done = 1;
        s.halt = 1;
      }
    } else {
      s.alpha = alpha;
    }
  }
}

// x += alpha p; r -= alpha A p; z = M r; ||r||^2, <r, z>; stop rule and beta.
__global__ void k_cg_update(CgWork w) {
  const int col = blockIdx.y;
  if (w.scal[col].halt) return;
  const double alpha = w.scal[col].alpha;
  const double* p = col4(w.p, w, col);
  double* x = col4(w.x, w, col);
  double* r = col4(w.r, w, col);
  double* z = col4(w.z, w, col);
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * kNT) {
    double q0, q1, q2;
    load_q(w, col, i, q0, q1, q2);
    const double p0 = p[4 * i], p1 = p[4 * i + 1], p2 = p[4 * i + 2];
    x[4 * i] += alpha * p0;
    x[4 * i + 1] += alpha * p1;
    x[4 * i + 2] += alpha * p2;
    const double r0 = r[4 * i] - alpha * q0, r1 = r[4 * i + 1] - alpha * q1,
                 r2 = r[4 * i + 2] - alpha * q2;
    r[4 * i] = r0; r[4 * i + 1] = r1; r[4 * i + 2] = r2;
    double z0, z1, z2;
    bd3(w.minv + 6 * i, r0, r1, r2, z0, z1, z2);
    z[4 * i] = z0; z[4 * i + 1] = z1; z[4 * i + 2] = z2;
    v[0] += r0 * r0 + r1 * r1 + r2 * r2;
    v[1] += r0 * z0 + r1 * z1 + r2 * z2;
  }
  double t[2];
  if (grid_sum<2>(v, w, col, t) && threadIdx.x == 0) {
    CgScalars& s = w.scal[col];
    s.iters += 1;
    s.since_rep += 1;
    s.rr = t[0];
    s.rz_prev = s.rz;
    s.rz = t[1];
    s.beta = t[1] / s.rz_prev;
    // FP32 path: pause at half the tolerance so that the FP64 check that follows usually
    // confirms convergence at once (the recursive FP32 residual drifts from the true one)
    if (t[0] < (w.fp32 ? 0.25 : 1.0) * w.tol2 * s.bnorm2) {
      if (w.fp32) {
        s.paused = 1;   // confirm with the FP64 true residual before stopping
      } else {
        s.done = 1;
      }
      s.halt = 1;
    } else if (!isfinite(t[0]) || !isfinite(s.beta)) {
      s.status = MM_EBREAKDOWN;
      s.done = 1;
      s.halt = 1;
    } else if (s.iters >= w.max_iter) {
      s.status = MM_ENOTCONV;
      s.done = 1;
      s.halt = 1;
    }
  }
}

// Residual replacement (FP32 path): r = b - A x with A x in FP64 (in q), z = M r, new beta.
__global__ void k_cg_replace(CgWork w) {
  const int col = blockIdx.y;
  if (w.scal[col].done) return;
  const double* b = col4(w.b, w, col);
  const double* ax = col4(w.q, w, col);
  double* r = col4(w.r, w, col);
  double* z = col4(w.z, w, col);
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * kNT) {
    const double r0 = b[4 * i] - ax[4 * i], r1 = b[4 * i + 1] - ax[4 * i + 1],
                 r2 = b[4 * i + 2] - ax[4 * i + 2];
    r[4 * i] = r0; r[4 * i + 1] = r1; r[4 * i + 2] = r2;
    double z0, z1, z2;
    bd3(w.minv + 6 * i, r0, r1, r2, z0, z1, z2);
    z[4 * i] = z0; z[4 * i + 1] = z1; z[4 * i + 2] = z2;
    v[0] += r0 * r0 + r1 * r1 + r2 * r2;
    v[1] += r0 * z0 + r1 * z1 + r2 * z2;
  }
  double t[2];
  if (grid_sum<2>(v, w, col, t) && threadIdx.x == 0) {
    CgScalars& s = w.scal[col];
    s.n_true += 1;
    s.since_rep = 0;
    // Keep the search direction (reliable update) while the true residual is close to the
    // recursive one; when it is more than twice as large in norm (the recursion has run below the
    // FP32 operator's accuracy) p was built for a residual that no longer exists, and CG restarts
    // from p = z.
    const bool restart = t[0] > 4.0 * s.rr || s.restart_req != 0;
    s.restart_req = 0;
    s.rr = t[0];
    s.rr_true = t[0];
    s.rz = t[1];
    s.beta = restart ? 0.0 : t[1] / s.rz_prev;
    s.paused = 0;
    if (t[0] < w.tol2 * s.bnorm2) {
      s.done = 1;
      s.halt = 1;
    } else if (s.iters >= w.max_iter) {
      s.status = MM_ENOTCONV;
      s.done = 1;
      s.halt = 1;
    } else if (!isfinite(t[0]) || !isfinite(s.beta)) {
      s.status = MM_EBREAKDOWN;
      s.done = 1;
      s.halt = 1;
    } else {
      s.halt = 0;
    }
  }
}

// ||b - A x||^2 for reporting (A x in q).
__global__ void k_cg_true_res(CgWork w) {
  const int col = blockIdx.y;
  const double* b = col4(w.b, w, col);
  const double* ax = col4(w.q, w, col);
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < w.n; i += (int64_t)gridDim.x * kNT) {
    const double r0 = b[4 * i] - ax[4 * i], r1 = b[4 * i + 1] - ax[4 * i + 1],
                 r2 = b[4 * i + 2] - ax[4 * i + 2];
    v[0] += r0 * r0 + r1 * r1 + r2 * r2;
  }
  double t[1];
  if (grid_sum<1>(v, w, col, t) && threadIdx.x == 0) w.scal[col].rr_true = t[0];
}

cudaError_t launch_cg(CgKernel k, const CgWork& w, cudaStream_t s) {
  dim3 grid(w.n_blocks, w.nrhs);
  switch (k) {
    case CG_INIT: k_cg_init<<<grid, kNT, 0, s>>>(w); break;
    case CG_PUPDATE: k_cg_pupdate<<<grid, kNT, 0, s>>>(w); break;
    case CG_DOT_PQ: k_cg_dot_pq<<<grid, kNT, 0, s>>>(w); break;
    case CG_UPDATE: k_cg_update<<<grid, kNT, 0, s>>>(w); break;
    case CG_REPLACE: k_cg_replace<<<grid, kNT, 0, s>>>(w); break;
    case CG_TRUE_RES: k_cg_true_res<<<grid, kNT, 0, s>>>(w); break;
  }
  return cudaGetLastError();
}

int cg_blocks_for(int64_t n) {
  int64_t g = (n + kNT - 1) / kNT;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace mm
