// Block conjugate gradients on s right-hand sides (Algorithm 2 in its block Orthomin form with
// R_0 = [b_1 .. b_s]): tall-skinny block products and the small dense steps.
//
// Layouts: a block of t pixel-domain vectors is [t][n][4] (IQU + pad per pixel, pad = 0).
// Search blocks (Z, A Z, P, A P, M R) are float32; X, R and every t x t matrix are float64.
// Tall-skinny products run on the FP32 units (GB300's FP64 rate is 1/64 of FP32) with FP64
// accumulation across CTAs; the solver's accuracy is restored by FP64 residual checks.
#include "mm_block.cuh"
#include "mm_internal.cuh"

namespace mm {

namespace {
constexpr int kNT = 256;
}  // namespace

// Partial Gram products: out_part[blk][i tb + j] = sum over this CTA's contiguous range of pixels
// of <A_i, B_j> (3 components), FP32 products and sums, FP64 per-CTA totals.  ta, tb <= kMaxBlk.
// A is a float4 block, B a float4 or float64 block (R); columns selected through idx_a / idx_b
// (identity when null).

// The same partial Gram products for small blocks (ta <= MA, tb <= MB): every thread streams its
// pixels (grid-stride, coalesced) and keeps the ta tb dot products in registers; then a block
// reduction in FP64.  (The staged kernel above keeps most threads idle when t is small.)
template <typename TB, int MA, int MB>
__global__ void __launch_bounds__(kNT) k_bgram_small(const float4* __restrict__ A, int ta,
                                                      const int* __restrict__ idx_a,
                                                      const TB* __restrict__ B, int tb,
                                                      const int* __restrict__ idx_b, int64_t n,
                                                      double* __restrict__ out_part) {
  __shared__ double red[kNT / 32][MA * MB];
  float acc[MA][MB];
#pragma unroll
  for (int i = 0; i < MA; i++)
#pragma unroll
    for (int j = 0; j < MB; j++) acc[i][j] = 0.f;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += (int64_t)gridDim.x * kNT) {
    float bx[MB], by[MB], bz[MB];
#pragma unroll
    for (int j = 0; j < MB; j++) {
      bx[j] = by[j] = bz[j] = 0.f;
      if (j < tb) {
        const int64_t col = idx_b ? idx_b[j] : j;
        if constexpr (sizeof(TB) == sizeof(float4)) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(B) + col * n + p);
          bx[j] = v.x; by[j] = v.y; bz[j] = v.z;
        } else {
          const double* v = reinterpret_cast<const double*>(B) + 4 * (col * n + p);
          bx[j] = (float)v[0]; by[j] = (float)v[1]; bz[j] = (float)v[2];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < MA; i++) {
      if (i < ta) {
        const float4 a = __ldg(A + (int64_t)(idx_a ? idx_a[i] : i) * n + p);
#pragma unroll
        for (int j = 0; j < MB; j++) acc[i][j] += a.x * bx[j] + a.y * by[j] + a.z * bz[j];
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MA; i++)
#pragma unroll
    for (int j = 0; j < MB; j++) {
      double v = (double)acc[i][j];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][i * MB + j] = v;
    }
  __syncthreads();
  if (threadIdx.x < MA * MB) {
    const int i = threadIdx.x / MB, j = threadIdx.x % MB;
    if (i < ta && j < tb) {
      double v = 0.0;
      for (int w = 0; w < kNT / 32; w++) v += red[w][threadIdx.x];
      out_part[(int64_t)blockIdx.x * kMaxBlk * kMaxBlk + i * tb + j] = v;
    }
  }
}

template <int MA, int MB>
static void bgram_small(const float* A, int ta, const int* idx_a, const void* B, int b_is_fp64, int tb,
                        const int* idx_b, int64_t n, double* part, int nblk, cudaStream_t s) {
  if (b_is_fp64)
    k_bgram_small<double4_16a, MA, MB><<<nblk, kNT, 0, s>>>(reinterpret_cast<const float4*>(A), ta, idx_a,
                                                            reinterpret_cast<const double4_16a*>(B), tb, idx_b, n,
                                                            part);
  else
    k_bgram_small<float4, MA, MB><<<nblk, kNT, 0, s>>>(reinterpret_cast<const float4*>(A), ta, idx_a,
                                                       reinterpret_cast<const float4*>(B), tb, idx_b, n, part);
}

// The same partial Gram products for wide blocks: 64 x 64 pairs over 256 threads, each thread a
// 4 x 4 tile of (i, j) in registers; kGR pixels of both blocks staged per step as
// [pixel][component][column] (rows padded to keep 16-byte alignment and spread the staging stores
// over banks), so a thread's four a values and four b values of one pixel component are two
// 16-byte shared loads for 16 FMAs.
constexpr int kGR = 24;   // 2 x 19.6 KB of static shared memory
constexpr int kGRow = kMaxBlk + 4;
template <typename TB>
__global__ void __launch_bounds__(kNT) k_bgram_tiled(const float4* __restrict__ A, int ta,
                                                      const int* __restrict__ idx_a,
                                                      const TB* __restrict__ B, int tb,
                                                      const int* __restrict__ idx_b, int64_t n,
                                                      double* __restrict__ out_part) {
  static_assert(kNT == 256 && kMaxBlk == 64, "16 x 16 threads of 4 x 4 pairs");
  __shared__ __align__(16) float sa[kGR][3][kGRow];
  __shared__ __align__(16) float sb[kGR][3][kGRow];
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  double tot[4][4];   // FP64 totals of the per-chunk FP32 sums (two-level summation)
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) tot[u][v] = 0.0;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = (int64_t)blockIdx.x * per, p1 = min(n, p0 + per);
  for (int64_t base = p0; base < p1; base += kGR) {
    const int cnt = (int)min((int64_t)kGR, p1 - base);
    // staging: consecutive threads take consecutive pixels of one column (coalesced loads)
    for (int e = threadIdx.x; e < kGR * kMaxBlk; e += kNT) {
      const int r = e % kGR, i = e / kGR;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < cnt && i < ta) v = __ldg(A + (int64_t)(idx_a ? idx_a[i] : i) * n + base + r);
      sa[r][0][i] = v.x; sa[r][1][i] = v.y; sa[r][2][i] = v.z;
      float x = 0.f, y = 0.f, z = 0.f;
      if (r < cnt && i < tb) {
        const int64_t col = idx_b ? idx_b[i] : i;
        if constexpr (sizeof(TB) == sizeof(float4)) {
          const float4 w = __ldg(reinterpret_cast<const float4*>(B) + col * n + base + r);
          x = w.x; y = w.y; z = w.z;
        } else {
          const double* w = reinterpret_cast<const double*>(B) + 4 * (col * n + base + r);
          x = (float)w[0]; y = (float)w[1]; z = (float)w[2];
        }
      }
      sb[r][0][i] = x; sb[r][1][i] = y; sb[r][2][i] = z;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int v = 0; v < 4; v++) acc[u][v] = 0.f;
    for (int r = 0; r < cnt; r++) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float4 a = *reinterpret_cast<const float4*>(&sa[r][c][4 * ti]);
        const float4 b = *reinterpret_cast<const float4*>(&sb[r][c][4 * tj]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
          for (int v = 0; v < 4; v++) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int v = 0; v < 4; v++) tot[u][v] += (double)acc[u][v];
    __syncthreads();
  }
  double* o = out_part + (int64_t)blockIdx.x * kMaxBlk * kMaxBlk;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int i = 4 * ti + u, j = 4 * tj + v;
      if (i < ta && j < tb) o[i * tb + j] = tot[u][v];
    }
}

// G[i][j] = sum over CTAs of out_part (fixed order: deterministic)
// One warp per output: lane l sums partials l, l + 32, ... in order, then a fixed shuffle tree
// (deterministic, and 32 loads in flight instead of one serial chain over all CTAs).
__device__ __forceinline__ double warp_sum_strided(const double* __restrict__ part, int64_t stride, int nblk) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * stride];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__global__ void k_bgram_reduce(const double* __restrict__ part, int nblk, int npair,
                               double* __restrict__ G) {
  const int pr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (pr >= npair) return;
  const double s = warp_sum_strided(part + pr, (int64_t)kMaxBlk * kMaxBlk, nblk);
  if ((threadIdx.x & 31) == 0) G[pr] = s;
}

cudaError_t launch_bgram(const float* A, int ta, const int* idx_a, const void* B, int b_is_fp64,
                         int tb, const int* idx_b, int64_t n, double* part, int nblk, double* G,
                         cudaStream_t s) {
  if (ta <= 0 || tb <= 0) return cudaSuccess;
  if (ta > kMaxBlk || tb > kMaxBlk) return cudaErrorInvalidValue;
  if (ta <= 4 && tb <= 4) {
    bgram_small<4, 4>(A, ta, idx_a, B, b_is_fp64, tb, idx_b, n, part, nblk, s);
  } else if (ta == 1 && tb <= 16) {
    bgram_small<1, 16>(A, ta, idx_a, B, b_is_fp64, tb, idx_b, n, part, nblk, s);
  } else if (b_is_fp64) {
    k_bgram_tiled<double4_16a><<<nblk, kNT, 0, s>>>(reinterpret_cast<const float4*>(A), ta, idx_a,
                                                    reinterpret_cast<const double4_16a*>(B), tb, idx_b, n, part);
  } else {
    k_bgram_tiled<float4><<<nblk, kNT, 0, s>>>(reinterpret_cast<const float4*>(A), ta, idx_a,
                                               reinterpret_cast<const float4*>(B), tb, idx_b, n, part);
  }
  k_bgram_reduce<<<(ta * tb + 7) / 8, 256, 0, s>>>(part, nblk, ta * tb, G);
  return cudaGetLastError();
}

// out_j (+)= sign * sum_i A_i C[i][j] for j < v (A: float32 [t][n]; C: FP64 [t][v] row-major with
// leading dimension ldc; out: FP64 or FP32 block, column j stored at idx_out[j] (or j)).  mode 0:
// out = sign * sum, mode 1: out += sign * sum.  A CTA stages kCP pixels of every input column and
// the coefficients in shared memory, then each thread forms 8 output columns of one pixel (warp w
// takes columns 8 w .. 8 w + 7, its lanes consecutive pixels, so the stores coalesce and each
// warp owns its columns' norm partials).  With norm_part != null (FP64 outputs), per-CTA partials
// of ||out_j||^2 are written.
constexpr int kCP = 32;
template <typename TO>
__global__ void __launch_bounds__(kNT) k_bcombine(TO* __restrict__ out, const int* __restrict__ idx_out,
                                                   int v, const float4* __restrict__ A, int t,
                                                   const double* __restrict__ C, int ldc, double sign,
                                                   int mode, int64_t n, double* __restrict__ norm_part) {
  static_assert(kNT == 256 && kMaxBlk == 64 && kCP == 32, "8 warps x 8 columns, 32 pixels per step");
  __shared__ __align__(16) float4 sA[kMaxBlk][kCP];     // 32 KB
  __shared__ __align__(16) float cs[kMaxBlk][kMaxBlk];  // 16 KB
  for (int e = threadIdx.x; e < t * v; e += kNT) cs[e / v][e % v] = (float)(sign * C[(e / v) * ldc + (e % v)]);
  const int r = threadIdx.x & 31, g = threadIdx.x >> 5;   // pixel in the chunk, column group
  const int j0 = 8 * g;
  const int nj = max(0, min(8, v - j0));
  double nrm[8];
#pragma unroll
  for (int jj = 0; jj < 8; jj++) nrm[jj] = 0.0;
  const int64_t n_chunks = (n + kCP - 1) / kCP;
  for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int64_t base = ch * kCP;
    const int cnt = (int)min((int64_t)kCP, n - base);
    __syncthreads();   // the previous chunk is no longer read (and the coefficients are staged)
    for (int e = threadIdx.x; e < t * kCP; e += kNT) {
      const int i = e / kCP, q = e % kCP;
      sA[i][q] = (q < cnt) ? __ldg(A + (int64_t)i * n + base + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (nj == 0 || r >= cnt) continue;
    float ax[8], ay[8], az[8];
#pragma unroll
    for (int jj = 0; jj < 8; jj++) ax[jj] = ay[jj] = az[jj] = 0.f;
    for (int i = 0; i < t; i++) {
      const float4 a = sA[i][r];
      const float4 c0 = *reinterpret_cast<const float4*>(&cs[i][j0]);
      const float4 c1 = *reinterpret_cast<const float4*>(&cs[i][j0 + 4]);
      const float c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
      for (int jj = 0; jj < 8; jj++) {
        ax[jj] = fmaf(a.x, c[jj], ax[jj]);
        ay[jj] = fmaf(a.y, c[jj], ay[jj]);
        az[jj] = fmaf(a.z, c[jj], az[jj]);
      }
    }
    const int64_t p = base + r;
#pragma unroll
    for (int jj = 0; jj < 8; jj++) {
      if (jj >= nj) break;
      const int64_t col = idx_out ? idx_out[j0 + jj] : (j0 + jj);
      if constexpr (sizeof(TO) == sizeof(float4)) {
        float4* o = reinterpret_cast<float4*>(out) + col * n + p;
        float4 cur = mode ? *o : make_float4(0.f, 0.f, 0.f, 0.f);
        cur.x += ax[jj]; cur.y += ay[jj]; cur.z += az[jj];
        cur.w = 0.f;
        *o = cur;
      } else {
        double* o = reinterpret_cast<double*>(out) + 4 * (col * n + p);
        double x0 = mode ? o[0] : 0.0, x1 = mode ? o[1] : 0.0, x2 = mode ? o[2] : 0.0;
        x0 += (double)ax[jj]; x1 += (double)ay[jj]; x2 += (double)az[jj];
        o[0] = x0; o[1] = x1; o[2] = x2; o[3] = 0.0;
        nrm[jj] += x0 * x0 + x1 * x1 + x2 * x2;
      }
    }
  }
  if (norm_part) {
#pragma unroll
    for (int jj = 0; jj < 8; jj++) {
      double v2 = nrm[jj];
      for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
      if (r == 0 && jj < nj) norm_part[(int64_t)(j0 + jj) * gridDim.x + blockIdx.x] = v2;
    }
  }
}

// Narrow blocks (v, t <= kCombJ): each thread streams pixels (grid-stride) and forms all v outputs
// of its pixel in registers; no staging, so a column or two costs one pass over A.
constexpr int kCombJ = 16;
template <typename TO, int J>
__global__ void __launch_bounds__(kNT) k_bcombine_stream(TO* __restrict__ out, const int* __restrict__ idx_out,
                                                   int v, const float4* __restrict__ A, int t,
                                                   const double* __restrict__ C, int ldc, double sign,
                                                   int mode, int64_t n, double* __restrict__ norm_part) {
  __shared__ float cs[kMaxBlk * kMaxBlk];
  __shared__ double red[kNT];
  for (int e = threadIdx.x; e < t * v; e += kNT) cs[e] = (float)(sign * C[(e / v) * ldc + (e % v)]);
  __syncthreads();
  for (int j0 = 0; j0 < v; j0 += J) {
    const int nj = min(J, v - j0);
    double nrm[J];
#pragma unroll
    for (int jj = 0; jj < J; jj++) nrm[jj] = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += (int64_t)gridDim.x * kNT) {
      float ax[J], ay[J], az[J];
#pragma unroll
      for (int jj = 0; jj < J; jj++) ax[jj] = ay[jj] = az[jj] = 0.f;
      for (int i = 0; i < t; i++) {
        const float4 a = __ldg(A + (int64_t)i * n + p);
#pragma unroll
        for (int jj = 0; jj < J; jj++) {
          const float c = (jj < nj) ? cs[i * v + j0 + jj] : 0.f;
          ax[jj] = fmaf(a.x, c, ax[jj]);
          ay[jj] = fmaf(a.y, c, ay[jj]);
          az[jj] = fmaf(a.z, c, az[jj]);
        }
      }
#pragma unroll
      for (int jj = 0; jj < J; jj++) {
        if (jj >= nj) break;
        const int64_t col = idx_out ? idx_out[j0 + jj] : (j0 + jj);
        if constexpr (sizeof(TO) == sizeof(float4)) {
          float4* o = reinterpret_cast<float4*>(out) + col * n + p;
          float4 cur = mode ? *o : make_float4(0.f, 0.f, 0.f, 0.f);
          cur.x += ax[jj]; cur.y += ay[jj]; cur.z += az[jj];
          cur.w = 0.f;
          *o = cur;
        } else {
          // 16-byte accesses to the pixel's 32 bytes
          double2* o = reinterpret_cast<double2*>(out) + 2 * (col * n + p);
          double2 xy = mode ? o[0] : make_double2(0.0, 0.0);
          double2 zw = mode ? o[1] : make_double2(0.0, 0.0);
          xy.x += (double)ax[jj]; xy.y += (double)ay[jj]; zw.x += (double)az[jj];
          zw.y = 0.0;
          o[0] = xy;
          o[1] = zw;
          nrm[jj] += xy.x * xy.x + xy.y * xy.y + zw.x * zw.x;
        }
      }
    }
    if (norm_part) {
      for (int jj = 0; jj < nj; jj++) {
        red[threadIdx.x] = nrm[jj];
        __syncthreads();
        for (int sh = kNT / 2; sh > 0; sh >>= 1) {
          if (threadIdx.x < sh) red[threadIdx.x] += red[threadIdx.x + sh];
          __syncthreads();
        }
        if (threadIdx.x == 0) norm_part[(int64_t)(j0 + jj) * gridDim.x + blockIdx.x] = red[0];
        __syncthreads();
      }
    }
  }
}

__global__ void k_norm_reduce(const double* __restrict__ part, int nblk, int v, double* __restrict__ out) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= v) return;
  const double s = warp_sum_strided(part + (int64_t)j * nblk, 1, nblk);
  if ((threadIdx.x & 31) == 0) out[j] = s;
}

cudaError_t launch_bcombine(void* out, int out_is_fp64, const int* idx_out, int v, const float* A, int t,
                            const double* C, int ldc, double sign, int mode, int64_t n, double* norm_part,
                            int nblk, double* norms, cudaStream_t s) {
  if (v <= 0) return cudaSuccess;
  if (t > kMaxBlk || v > kMaxBlk) return cudaErrorInvalidValue;
  const bool narrow = v <= kCombJ && t <= kCombJ;
  if (out_is_fp64) {
    if (narrow && v <= 4)   // few outputs: fewer registers, more resident warps
      k_bcombine_stream<double4_16a, 4><<<nblk, kNT, 0, s>>>(reinterpret_cast<double4_16a*>(out), idx_out, v,
                                                             reinterpret_cast<const float4*>(A), t, C, ldc, sign,
                                                             mode, n, norm_part);
    else if (narrow)
      k_bcombine_stream<double4_16a, kCombJ><<<nblk, kNT, 0, s>>>(reinterpret_cast<double4_16a*>(out), idx_out, v,
                                                                  reinterpret_cast<const float4*>(A), t, C, ldc,
                                                                  sign, mode, n, norm_part);
    else
      k_bcombine<double4_16a><<<nblk, kNT, 0, s>>>(reinterpret_cast<double4_16a*>(out), idx_out, v,
                                                   reinterpret_cast<const float4*>(A), t, C, ldc, sign, mode,
                                                   n, norm_part);
  } else {
    if (narrow && v <= 4)
      k_bcombine_stream<float4, 4><<<nblk, kNT, 0, s>>>(reinterpret_cast<float4*>(out), idx_out, v,
                                                        reinterpret_cast<const float4*>(A), t, C, ldc, sign, mode, n,
                                                        nullptr);
    else if (narrow)
      k_bcombine_stream<float4, kCombJ><<<nblk, kNT, 0, s>>>(reinterpret_cast<float4*>(out), idx_out, v,
                                                             reinterpret_cast<const float4*>(A), t, C, ldc, sign, mode,
                                                             n, nullptr);
    else
      k_bcombine<float4><<<nblk, kNT, 0, s>>>(reinterpret_cast<float4*>(out), idx_out, v,
                                              reinterpret_cast<const float4*>(A), t, C, ldc, sign, mode, n,
                                              nullptr);
  }
  if (norm_part && out_is_fp64) k_norm_reduce<<<(v + 7) / 8, 256, 0, s>>>(norm_part, nblk, v, norms);
  return cudaGetLastError();
}

// W_j = M_BD R_{idx_j} in FP32 (j < v; idx null = identity); R float64 [.][n][4] or float4
template <typename TR>
__global__ void k_bprecond(const double* __restrict__ minv, const TR* __restrict__ R,
                           const int* __restrict__ idx, int v, int64_t n, float4* __restrict__ W) {
  const int64_t tot = (int64_t)v * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n);
    const int64_t p = e - (int64_t)j * n;
    const int64_t o = (int64_t)(idx ? idx[j] : j) * n + p;
    double r0, r1, r2;
    if constexpr (sizeof(TR) == sizeof(float4)) {
      const float4 f = R[o];
      r0 = f.x; r1 = f.y; r2 = f.z;
    } else {
      const double* r = reinterpret_cast<const double*>(R) + 4 * o;
      r0 = r[0]; r1 = r[1]; r2 = r[2];
    }
    const double* m = minv + 6 * p;
    const double z0 = m[0] * r0 + m[1] * r1 + m[2] * r2;
    const double z1 = m[1] * r0 + m[3] * r1 + m[4] * r2;
    const double z2 = m[2] * r0 + m[4] * r1 + m[5] * r2;
    W[e] = make_float4((float)z0, (float)z1, (float)z2, 0.f);
  }
}

static unsigned precond_grid(int64_t tot) {
  int64_t g = (tot + 255) / 256;
  if (g > 32 * sm_count()) g = 32 * sm_count();
  return (unsigned)g;
}

cudaError_t launch_bprecond(const double* minv, const double* R, const int* idx, int v, int64_t n,
                            float* W, cudaStream_t s) {
  if (v <= 0) return cudaSuccess;
  k_bprecond<double><<<precond_grid((int64_t)v * n), 256, 0, s>>>(minv, R, idx, v, n, reinterpret_cast<float4*>(W));
  return cudaGetLastError();
}

cudaError_t launch_bprecond32(const double* minv, const float* R, int v, int64_t n, float* W, cudaStream_t s) {
  if (v <= 0) return cudaSuccess;
  k_bprecond<float4><<<precond_grid((int64_t)v * n), 256, 0, s>>>(
      minv, reinterpret_cast<const float4*>(R), nullptr, v, n, reinterpret_cast<float4*>(W));
  return cudaGetLastError();
}

// Enlarged CG (Sect. 3.2, ECG): the split of one residual r [n][4] into t columns over contiguous
// ranges of pixels (column i keeps the pixels p with floor(p t / n) = i, zero elsewhere).
__global__ void k_bsplit(const double* __restrict__ r, int t, int64_t n, double* __restrict__ R) {
  const int64_t tot = (int64_t)t * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n);
    const int64_t p = e - (int64_t)i * n;
    const bool own = (p * t) / n == i;
    const double2* src = reinterpret_cast<const double2*>(r + 4 * p);
    double2* dst = reinterpret_cast<double2*>(R + 4 * e);
    dst[0] = own ? src[0] : make_double2(0.0, 0.0);
    dst[1] = own ? make_double2(src[1].x, 0.0) : make_double2(0.0, 0.0);
  }
}

cudaError_t launch_bsplit(const double* r4, int t, int64_t n, double* R, cudaStream_t s) {
  if (t <= 0 || n <= 0) return cudaSuccess;
  k_bsplit<<<precond_grid((int64_t)t * n), 256, 0, s>>>(r4, t, n, R);
  return cudaGetLastError();
}

// s_p = sum_i X_i[p] over the t columns of a FP64 block; out (+)= s when out != null, and per-CTA
// partials of ||s||^2 (norm of the summed residual of ECG, or of x = X 1).
__global__ void k_bsum(const double* __restrict__ X, int t, int64_t n, double* __restrict__ out, int accumulate,
                       double* __restrict__ norm_part) {
  __shared__ double red[kNT];
  double nrm = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += (int64_t)gridDim.x * kNT) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < t; i++) {
      const double* x = X + 4 * ((int64_t)i * n + p);
      s0 += x[0]; s1 += x[1]; s2 += x[2];
    }
    if (out) {
      double* o = out + 4 * p;
      if (accumulate) { s0 += o[0]; s1 += o[1]; s2 += o[2]; }
      o[0] = s0; o[1] = s1; o[2] = s2; o[3] = 0.0;
    }
    nrm += s0 * s0 + s1 * s1 + s2 * s2;
  }
  red[threadIdx.x] = nrm;
  __syncthreads();
  for (int sh = kNT / 2; sh > 0; sh >>= 1) {
    if (threadIdx.x < sh) red[threadIdx.x] += red[threadIdx.x + sh];
    __syncthreads();
  }
  if (threadIdx.x == 0) norm_part[blockIdx.x] = red[0];
}

cudaError_t launch_bsum(const double* X, int t, int64_t n, double* out, int accumulate, double* norm_part,
                        int nblk, double* norm, cudaStream_t s) {
  if (t <= 0 || t > kMaxBlk) return cudaErrorInvalidValue;
  k_bsum<<<nblk, kNT, 0, s>>>(X, t, n, out, accumulate, norm_part);
  k_norm_reduce<<<1, 32, 0, s>>>(norm_part, nblk, 1, norm);
  return cudaGetLastError();
}

// Small dense step of one iteration, one CTA, FP64:
//   G (t x t, symmetrised) = L L^T by a pivoted Cholesky with relative tolerance rank_tol;
//   Linv = L^-1 (rank x rank, lower); piv[0..rank) = pivoted columns; *rank_out = rank.
// The caller forms P = Linv Z[piv] and A P = Linv (A Z)[piv] (rows are block columns).
__global__ void k_bchol(const double* __restrict__ G, int t, double rank_tol, double* __restrict__ Linv_out,
                        int* __restrict__ piv_out, int* __restrict__ rank_out) {
  // The factorisation is O(t^3) <= ~90K flops: one thread does it, with explicit indexing.
  extern __shared__ double dsm[];      // g [kMaxBlk * kLd] then L [kMaxBlk * kLd]
  constexpr int kLd = kMaxBlk + 1;
  double* g = dsm;
  double* L = dsm + kMaxBlk * kLd;
  if (threadIdx.x != 0) return;
  int piv[kMaxBlk];
  double mx = 0.0;
  for (int i = 0; i < t; i++) {
    piv[i] = i;
    for (int j = 0; j < t; j++) {
      g[i * kLd + j] = 0.5 * (G[i * t + j] + G[j * t + i]);
      L[i * kLd + j] = 0.0;
    }
    mx = fmax(mx, fabs(g[i * kLd + i]));
  }
  const double scale = mx > 0.0 ? mx : 1e-300;
  int r = t;
  for (int k = 0; k < t; k++) {
    int best = k;
    double bd = -1.0;
    for (int i = k; i < t; i++) {
      double d = g[i * kLd + i];
      for (int m = 0; m < k; m++) d -= L[i * kLd + m] * L[i * kLd + m];
      if (d > bd) { bd = d; best = i; }
    }
    if (!(bd > rank_tol * scale)) { r = k; break; }
    if (best != k) {   // symmetric swap of rows/columns k and best, and of the computed rows of L
      for (int j = 0; j < t; j++) { const double tmp = g[k * kLd + j]; g[k * kLd + j] = g[best * kLd + j]; g[best * kLd + j] = tmp; }
      for (int j = 0; j < t; j++) { const double tmp = g[j * kLd + k]; g[j * kLd + k] = g[j * kLd + best]; g[j * kLd + best] = tmp; }
      for (int m = 0; m < k; m++) { const double tmp = L[k * kLd + m]; L[k * kLd + m] = L[best * kLd + m]; L[best * kLd + m] = tmp; }
      const int tp = piv[k]; piv[k] = piv[best]; piv[best] = tp;
    }
    L[k * kLd + k] = sqrt(bd);
    for (int i = k + 1; i < t; i++) {
      double sacc = g[i * kLd + k];
      for (int m = 0; m < k; m++) sacc -= L[i * kLd + m] * L[k * kLd + m];
      L[i * kLd + k] = sacc / L[k * kLd + k];
    }
  }
  // Linv = L^-1 (r x r, lower) by forward substitution, column by column
  for (int e = 0; e < kMaxBlk * kMaxBlk; e++) Linv_out[e] = 0.0;
  for (int c = 0; c < r; c++) {
    for (int i = c; i < r; i++) {
      double sacc = (i == c) ? 1.0 : 0.0;
      for (int m = c; m < i; m++) sacc -= L[i * kLd + m] * Linv_out[m * kMaxBlk + c];
      Linv_out[i * kMaxBlk + c] = sacc / L[i * kLd + i];
    }
  }
  for (int i = 0; i < t; i++) piv_out[i] = piv[i];
  *rank_out = r;
}

cudaError_t launch_bchol(const double* G, int t, double rank_tol, double* Linv, int* piv, int* rank,
                         cudaStream_t s) {
  if (t > kMaxBlk) return cudaErrorInvalidValue;
  const size_t smem = 2 * kMaxBlk * (kMaxBlk + 1) * sizeof(double);
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_bchol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_bchol<<<1, 32, smem, s>>>(G, t, rank_tol, Linv, piv, rank);
  return cudaGetLastError();
}

// Linv as a [t][t] coefficient matrix for the combine kernel: Cmb[k][i] = Linv[i][pos(k)] where
// block column k = piv[pos]; rows/cols beyond the rank are zero.  out_i = sum_k Z_k Cmb[k][i].
__global__ void k_linv_coef(const double* __restrict__ Linv, const int* __restrict__ piv,
                            const int* __restrict__ rank, int t, double* __restrict__ Cmb) {
  const int r = *rank;
  for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
    const int k = e / t, i = e % t;
    double c = 0.0;
    if (i < r) {
      for (int pos = 0; pos < r; pos++)
        if (piv[pos] == k) c = Linv[i * kMaxBlk + pos];
    }
    Cmb[k * t + i] = c;
  }
}

cudaError_t launch_linv_coef(const double* Linv, const int* piv, const int* rank, int t, double* Cmb,
                             cudaStream_t s) {
  k_linv_coef<<<1, 256, 0, s>>>(Linv, piv, rank, t, Cmb);
  return cudaGetLastError();
}

// R_j = B_j - AX_j (FP64) and norms_part of ||R_j||^2 (j < v); grid (nblk, v)
__global__ void k_bresid(const double* __restrict__ B, const double* __restrict__ AX, int64_t n,
                         double* __restrict__ R, double* __restrict__ norm_part) {
  __shared__ double red[kNT];
  const int j = blockIdx.y;
  double nrm = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += (int64_t)gridDim.x * kNT) {
    const int64_t o = 4 * ((int64_t)j * n + p);
    const double r0 = B[o] - AX[o], r1 = B[o + 1] - AX[o + 1], r2 = B[o + 2] - AX[o + 2];
    R[o] = r0; R[o + 1] = r1; R[o + 2] = r2; R[o + 3] = 0.0;
    nrm += r0 * r0 + r1 * r1 + r2 * r2;
  }
  red[threadIdx.x] = nrm;
  __syncthreads();
  for (int sh = kNT / 2; sh > 0; sh >>= 1) {
    if (threadIdx.x < sh) red[threadIdx.x] += red[threadIdx.x + sh];
    __syncthreads();
  }
  if (threadIdx.x == 0) norm_part[(int64_t)j * gridDim.x + blockIdx.x] = red[0];
}

cudaError_t launch_bresid(const double* B, const double* AX, int v, int64_t n, double* R,
                          double* norm_part, int nblk, double* norms, cudaStream_t s) {
  if (v <= 0) return cudaSuccess;
  k_bresid<<<dim3(nblk, v), kNT, 0, s>>>(B, AX, n, R, norm_part);
  k_norm_reduce<<<(v + 7) / 8, 256, 0, s>>>(norm_part, nblk, v, norms);
  return cudaGetLastError();
}

}  // namespace mm
