// Plan-time kernels: input validation, block-Jacobi blocks, pixel excision and compaction.
//
// Block-Jacobi preconditioner (Sect. 3.2): B_p = sum_{t: p_t = p} c_0,b(t) w_t w_t^T with
// w_t = (1, cos 2psi_t, sin 2psi_t); the diagonal of N^-1 on sample t is its block's c_0.
// Excision (Sect. 2.4): a pixel with fewer than 3 hits or cond_2(B_p) > cond_max is dropped with
// all its samples.  Local pixel ids are assigned in ascending global order over kept pixels
// (Sect. 3.1 local indexation).
#include "df64.cuh"
#include "mm_internal.cuh"

namespace mm {

__global__ void k_validate(const int32_t* __restrict__ pix, const float* __restrict__ psi, int64_t N,
                           int64_t n_pix, int32_t* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = pix[i];
    const float a = psi[i];
    if (p < -1 || (int64_t)p >= n_pix) atomicOr(bad, 1);
    if (!isfinite(a)) atomicOr(bad, 2);
  }
}

cudaError_t launch_validate(const int32_t* pix, const float* psi, int64_t N, int64_t n_pix,
                            int32_t* bad, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_validate<<<4 * sm_count(), 256, 0, s>>>(pix, psi, N, n_pix, bad);
  return cudaGetLastError();
}

// Block index of sample i (block_off has n_blocks + 1 entries).
__device__ __forceinline__ int block_of(const int64_t* __restrict__ off, int32_t n_blocks, int64_t i) {
  int lo = 0, hi = n_blocks;   // find the last b with off[b] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Each CTA takes a contiguous chunk of the samples and its warps stride through it, lane l of a
// warp on sample base + l, so a lane's block index is found once and only moves forward; the
// weights are the plan's FP64 (cos 2psi, sin 2psi).  Consecutive samples of a slow scan often
// fall on the same pixel: in a warp that holds such a run, the lanes of each run of equal pixels
// are summed by a segmented scan across the warp and the run's last lane adds the sums with one
// set of atomics.
__global__ void k_bd_accum(const int32_t* __restrict__ pix, const double2* __restrict__ w64,
                           const int64_t* __restrict__ off, const double* __restrict__ c0_blk,
                           int32_t n_blocks, int64_t N, double* __restrict__ B6,
                           int32_t* __restrict__ hits) {
  const int64_t chunk = (N + gridDim.x - 1) / gridDim.x;
  const int64_t c_lo = (int64_t)blockIdx.x * chunk, c_hi = min(N, c_lo + chunk);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = c_lo + (threadIdx.x - lane);
  if (warp0 >= c_hi) return;   // whole warps leave together
  int bi = block_of(off, n_blocks, min(warp0 + lane, c_hi - 1));
  for (int64_t base = warp0; base < c_hi; base += blockDim.x) {
    const int64_t i = base + lane;
    int32_t p = -1;
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < c_hi) {
      while (__ldg(off + bi + 1) <= i) bi++;
      p = pix[i];
      if (p >= 0) {
        const double c0 = c0_blk[bi];
        const double2 w = w64[i];
        const double c = w.x, sn = w.y;
        v[0] = c0;
        v[1] = c0 * c;
        v[2] = c0 * sn;
        v[3] = c0 * c * c;
        v[4] = c0 * c * sn;
        v[5] = c0 * sn * sn;
      }
    }
    const int32_t p_prev = __shfl_up_sync(0xffffffffu, p, 1);
    // FP64 arithmetic runs at 1/64 of the FP32 rate on GB300: the segmented scan runs only in
    // warps that hold a run of equal pixels; elsewhere every lane adds its own sample
    if (!__any_sync(0xffffffffu, lane > 0 && p >= 0 && p == p_prev)) {
      if (p >= 0) {
        double* b = B6 + 6 * (int64_t)p;
#pragma unroll
        for (int k = 0; k < 6; k++) atomicAdd(b + k, v[k]);
        atomicAdd(hits + p, 1);
      }
      continue;
    }
    // first lane of this lane's run of equal pixels (a max-scan of the run heads)
    int head = (lane == 0 || p_prev != p) ? lane : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int h = __shfl_up_sync(0xffffffffu, head, o);
      if (lane >= o) head = max(head, h);
    }
    // segmented inclusive sums: the run's last lane holds the run's totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
      for (int k = 0; k < 6; k++) {
        const double t = __shfl_up_sync(0xffffffffu, v[k], o);
        if (lane - o >= head) v[k] += t;
      }
    }
    const int32_t p_next = __shfl_down_sync(0xffffffffu, p, 1);
    if (p >= 0 && (lane == 31 || p_next != p)) {
      double* b = B6 + 6 * (int64_t)p;
#pragma unroll
      for (int k = 0; k < 6; k++) atomicAdd(b + k, v[k]);
      atomicAdd(hits + p, lane - head + 1);
    }
  }
}

cudaError_t launch_bd_accum(const int32_t* pix, const double2* w64, const int64_t* block_off,
                            const double* c0_blk, int32_t n_blocks, int64_t N, double* B6,
                            int32_t* hits, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_bd_accum<<<8 * sm_count(), 256, 0, s>>>(pix, w64, block_off, c0_blk, n_blocks, N, B6, hits);
  return cudaGetLastError();
}

// Eigenvalues of a symmetric 3x3 matrix (closed form, trigonometric solution of the
// characteristic cubic; Smith, Comm. ACM 4, 1961).  Returns lo <= hi.
__device__ void sym3_eig_range(const double a[6], double& lo, double& hi) {
  const double a00 = a[0], a01 = a[1], a02 = a[2], a11 = a[3], a12 = a[4], a22 = a[5];
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const double q = (a00 + a11 + a22) / 3.0;
  if (p1 == 0.0) {
    lo = fmin(a00, fmin(a11, a22));
    hi = fmax(a00, fmax(a11, a22));
    return;
  }
  const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
  const double p = sqrt(p2 / 6.0);
  const double ip = 1.0 / p;
  const double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip;
  const double c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
  const double det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) +
                     c02 * (c01 * c12 - c11 * c02);
  double r = 0.5 * det;
  r = fmin(1.0, fmax(-1.0, r));
  const double phi = acos(r) / 3.0;
  const double two_pi_3 = 2.0943951023931954923;
  const double e1 = q + 2.0 * p * cos(phi);
  const double e3 = q + 2.0 * p * cos(phi + two_pi_3);
  const double e2 = 3.0 * q - e1 - e3;
  hi = fmax(e1, fmax(e2, e3));
  lo = fmin(e1, fmin(e2, e3));
}

__global__ void k_bd_finalize(const double* __restrict__ B6, const int32_t* __restrict__ hits,
                              int64_t n_pix, double cond_max, int32_t* __restrict__ keep,
                              double* __restrict__ inv6) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  double a[6];
#pragma unroll
  for (int i = 0; i < 6; i++) a[i] = B6[6 * p + i];
  int ok = hits[p] >= 3;
  if (ok) {
    double lo, hi;
    sym3_eig_range(a, lo, hi);
    ok = (lo > 0.0) && (hi <= cond_max * lo);
  }
  keep[p] = ok;
  if (!ok) return;
  // inverse of the symmetric block by cofactors
  const double a00 = a[0], a01 = a[1], a02 = a[2], a11 = a[3], a12 = a[4], a22 = a[5];
  const double c00 = a11 * a22 - a12 * a12;
  const double c01 = a02 * a12 - a01 * a22;
  const double c02 = a01 * a12 - a02 * a11;
  const double c11 = a00 * a22 - a02 * a02;
  const double c12 = a01 * a02 - a00 * a12;
  const double c22 = a00 * a11 - a01 * a01;
  const double det = a00 * c00 + a01 * c01 + a02 * c02;
  const double id = 1.0 / det;
  double* o = inv6 + 6 * p;
  o[0] = c00 * id; o[1] = c01 * id; o[2] = c02 * id;
  o[3] = c11 * id; o[4] = c12 * id; o[5] = c22 * id;
}

cudaError_t launch_bd_finalize(const double* B6, const int32_t* hits, int64_t n_pix, double cond_max,
                               int32_t* keep, double* inv6, cudaStream_t s) {
  if (n_pix == 0) return cudaSuccess;
  k_bd_finalize<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(B6, hits, n_pix, cond_max, keep, inv6);
  return cudaGetLastError();
}

// ---- exclusive scan of the keep flags (three passes: tile sums, scan of sums, tile scans) ----
constexpr int kScanTile = 1024;   // elements per CTA (256 threads x 4)

__global__ void k_scan_tile_sums(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
  __shared__ int32_t red[256];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t v = 0;
  for (int i = threadIdx.x; i < kScanTile; i += 256) {
    const int64_t g = base + i;
    if (g < n) v += in[g] != 0;
  }
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

// single CTA: exclusive scan of the tile sums in place; total written to *total
__global__ void k_scan_sums(int32_t* sums, int64_t n_tiles, int32_t* total) {
  __shared__ int32_t buf[1024];
  int32_t carry = 0;
  for (int64_t base = 0; base < n_tiles; base += 1024) {
    const int64_t g = base + threadIdx.x;
    const int32_t v = g < n_tiles ? sums[g] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int32_t t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (g < n_tiles) sums[g] = carry + buf[threadIdx.x] - v;
    const int32_t tile_total = buf[1023];
    __syncthreads();
    carry += tile_total;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_tiles(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ sums,
                             int32_t* __restrict__ out) {
  __shared__ int32_t buf[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += 256) {
    const int64_t g = base + i;
    buf[i] = (g < n && in[g] != 0) ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // 1024 adds: negligible next to the rest of the plan
    int32_t acc = sums[blockIdx.x];
    for (int i = 0; i < kScanTile; i++) {
      const int32_t v = buf[i];
      buf[i] = acc;
      acc += v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kScanTile; i += 256) {
    const int64_t g = base + i;
    if (g < n) out[g] = buf[i];
  }
}

size_t scan_scratch_len(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

cudaError_t launch_scan_keep(const int32_t* keep, int64_t n, int32_t* lid, int32_t* total,
                             int32_t* scratch, int64_t scratch_len, cudaStream_t s) {
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt + 1 > scratch_len) return cudaErrorInvalidValue;
  if (n == 0) return cudaMemsetAsync(total, 0, sizeof(int32_t), s);
  k_scan_tile_sums<<<(unsigned)nt, 256, 0, s>>>(keep, n, scratch);
  k_scan_sums<<<1, 1024, 0, s>>>(scratch, nt, total);
  k_scan_tiles<<<(unsigned)nt, 256, 0, s>>>(keep, n, scratch, lid);
  return cudaGetLastError();
}

__global__ void k_compact(const int32_t* __restrict__ keep, const int32_t* __restrict__ lid,
                          const double* __restrict__ inv6_glob, int64_t n_pix,
                          int32_t* __restrict__ obs_to_global, double* __restrict__ minv) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix || !keep[p]) return;
  const int32_t l = lid[p];
  obs_to_global[l] = (int32_t)p;
#pragma unroll
  for (int i = 0; i < 6; i++) minv[6 * (int64_t)l + i] = inv6_glob[6 * p + i];
}

cudaError_t launch_compact(const int32_t* keep, const int32_t* lid, const double* inv6_glob,
                           int64_t n_pix, int32_t* obs_to_global, double* minv, cudaStream_t s) {
  if (n_pix == 0) return cudaSuccess;
  k_compact<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(keep, lid, inv6_glob, n_pix,
                                                             obs_to_global, minv);
  return cudaGetLastError();
}

__global__ void k_localize(const int32_t* __restrict__ pix, const int32_t* __restrict__ keep,
                           const int32_t* __restrict__ lid, int64_t N, int32_t* __restrict__ lpix) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = pix[i];
    lpix[i] = (p >= 0 && keep[p]) ? lid[p] : -1;
  }
}

cudaError_t launch_localize(const int32_t* pix, const int32_t* keep, const int32_t* lid, int64_t N,
                            int32_t* lpix, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_localize<<<8 * sm_count(), 256, 0, s>>>(pix, keep, lid, N, lpix);
  return cudaGetLastError();
}

// (cos 2psi, sin 2psi) once per sample in FP64 (the FP64 pipe runs at 1/64 of the FP32 rate, so the
// sine and cosine are taken once): w64 as is, w32 as their FP32 roundings, wdf (if non-null) split
// into df64 (hi, lo) pairs
// One FP64 sincos of 2 psi per sample: the FP64 weights, their FP32 roundings, (wdf non-null) their
// df64 split, and the angle 2 psi reduced to [-pi, pi] in FP64 and rounded once to FP32 (the FP32
// window kernels evaluate the weights from it in registers).
// cos(k pi/32), sin(k pi/32), k = 0 .. 63 (values of the circular functions rounded to FP64)
__device__ const double2 kSinCosPi32[64] = {
    {1.0, 0.0}, {0.9951847266721969, 0.0980171403295606},
    {0.9807852804032304, 0.19509032201612828}, {0.9569403357322088, 0.2902846772544624},
    {0.9238795325112867, 0.3826834323650898}, {0.881921264348355, 0.47139673682599764},
    {0.8314696123025452, 0.5555702330196022}, {0.773010453362737, 0.6343932841636455},
    {0.7071067811865476, 0.7071067811865476}, {0.6343932841636455, 0.773010453362737},
    {0.5555702330196022, 0.8314696123025452}, {0.47139673682599764, 0.881921264348355},
    {0.3826834323650898, 0.9238795325112867}, {0.2902846772544624, 0.9569403357322088},
    {0.19509032201612828, 0.9807852804032304}, {0.0980171403295606, 0.9951847266721969},
    {0.0, 1.0}, {-0.0980171403295606, 0.9951847266721969},
    {-0.19509032201612828, 0.9807852804032304}, {-0.2902846772544624, 0.9569403357322088},
    {-0.3826834323650898, 0.9238795325112867}, {-0.47139673682599764, 0.881921264348355},
    {-0.5555702330196022, 0.8314696123025452}, {-0.6343932841636455, 0.773010453362737},
    {-0.7071067811865476, 0.7071067811865476}, {-0.773010453362737, 0.6343932841636455},
    {-0.8314696123025452, 0.5555702330196022}, {-0.881921264348355, 0.47139673682599764},
    {-0.9238795325112867, 0.3826834323650898}, {-0.9569403357322088, 0.2902846772544624},
    {-0.9807852804032304, 0.19509032201612828}, {-0.9951847266721969, 0.0980171403295606},
    {-1.0, 0.0}, {-0.9951847266721969, -0.0980171403295606},
    {-0.9807852804032304, -0.19509032201612828}, {-0.9569403357322088, -0.2902846772544624},
    {-0.9238795325112867, -0.3826834323650898}, {-0.881921264348355, -0.47139673682599764},
    {-0.8314696123025452, -0.5555702330196022}, {-0.773010453362737, -0.6343932841636455},
    {-0.7071067811865476, -0.7071067811865476}, {-0.6343932841636455, -0.773010453362737},
    {-0.5555702330196022, -0.8314696123025452}, {-0.47139673682599764, -0.881921264348355},
    {-0.3826834323650898, -0.9238795325112867}, {-0.2902846772544624, -0.9569403357322088},
    {-0.19509032201612828, -0.9807852804032304}, {-0.0980171403295606, -0.9951847266721969},
    {0.0, -1.0}, {0.0980171403295606, -0.9951847266721969},
    {0.19509032201612828, -0.9807852804032304}, {0.2902846772544624, -0.9569403357322088},
    {0.3826834323650898, -0.9238795325112867}, {0.47139673682599764, -0.881921264348355},
    {0.5555702330196022, -0.8314696123025452}, {0.6343932841636455, -0.773010453362737},
    {0.7071067811865476, -0.7071067811865476}, {0.773010453362737, -0.6343932841636455},
    {0.8314696123025452, -0.5555702330196022}, {0.881921264348355, -0.47139673682599764},
    {0.9238795325112867, -0.3826834323650898}, {0.9569403357322088, -0.2902846772544624},
    {0.9807852804032304, -0.19509032201612828}, {0.9951847266721969, -0.0980171403295606}};

// (cos x, sin x) in FP64 by table lookup and angle addition (the table-driven method of
// P. T. P. Tang, ACM TOMS 1989-91): x = k pi/32 + r with k = rint(32 x / pi) and r = x - k pi/32
// by a two-constant Cody-Waite reduction (pi/32 = H + L, H = fl64(pi/32): k H is taken exactly
// inside one FMA, k L has an error far below 1e-30 for |k| < 2^40); |r| <= pi/64, where the Taylor
// series of sin r to r^9 and of cos r to r^8 leave truncation errors below 1e-19; then
//   cos x = C_k cos r - S_k sin r,  sin x = S_k cos r + C_k sin r,  (C_k, S_k) = table[k mod 64].
// About 20 FP64 operations instead of a general sincos (on GB300 FP64 runs at 1/64 of the FP32
// rate, and the plan spends most of this kernel's time there).
__device__ __forceinline__ void sincos_tab(double x, double& sn, double& cs) {
  if (!(fabs(x) < 1e9)) {   // far outside any angle a scan produces: the general routine
    sincos(x, &sn, &cs);
    return;
  }
  constexpr double kH = 0.09817477042468103;       // fl64(pi / 32)
  constexpr double kL = 3.827021247335479e-18;     // pi / 32 - kH
  constexpr double k32OverPi = 10.185916357881302;  // 32 / pi
  const double kd = rint(x * k32OverPi);
  double r = fma(-kd, kH, x);
  r = fma(-kd, kL, r);
  const double z = r * r;
  const double sr = r * fma(z, fma(z, fma(z, fma(z, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0), -1.0 / 6.0), 1.0);
  const double cr =
      fma(z, fma(z, fma(z, fma(z, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5), 1.0);
  const double2 t = kSinCosPi32[(int)((long long)kd & 63)];
  cs = fma(t.x, cr, -t.y * sr);
  sn = fma(t.y, cr, t.x * sr);
}

__global__ void k_weights(const float* __restrict__ psi, int64_t N, double2* __restrict__ w64,
                          float2* __restrict__ w32, float4* __restrict__ wdf, float* __restrict__ ang2) {
  constexpr double kTwoPi = 6.283185307179586476925;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = 2.0 * (double)psi[i];
    double s, c;
    sincos_tab(a, s, c);
    w64[i] = make_double2(c, s);
    w32[i] = make_float2((float)c, (float)s);
    if (wdf) {
      const df dc(c), ds(s);
      wdf[i] = make_float4(dc.hi, dc.lo, ds.hi, ds.lo);
    }
    if (ang2) {
      ang2[i] = (float)fma(-rint(a * (1.0 / kTwoPi)), kTwoPi, a);
    }
  }
}

cudaError_t launch_weights(const float* psi, int64_t N, double2* w64, float2* w32, float4* wdf, float* ang2,
                           cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_weights<<<8 * sm_count(), 256, 0, s>>>(psi, N, w64, w32, wdf, ang2);
  return cudaGetLastError();
}

}  // namespace mm
