// Template map-making with diagonal weights (Sect. 2, Eq. genMapEstimator with the filtering operator
// F_T = W - W T (T^T W T)^+ T^T W; the templates of Appendix A), one interval per block:
//   Legendre P_k(x), k < n_poly, x = 2 tau / (n - 1) - 1, rescaled by sqrt((2k + 1) / n);
//   azimuth bins over the block's azimuth range (value 1), or linear interpolation between n_az nodes;
//   cos(k phi), sin(k phi) of the HWP angle, k = 1..n_hwp.
// W = diag(w_b) on the kept samples of block b (w_b = the band's c_0 of a lambda = 0 plan), 0 on masked
// ones.  The kernel T^T W T of every block is built in FP64 and pseudo-inverted (eigenvalues below
// 1e-12 of the largest dropped) when the templates are attached; the filter then costs two passes over
// the block's samples per application.  Azimuth bins and interpolation fractions are decided once, in
// FP64, so the FP32 and FP64 operators use the same templates.
#include <math.h>

#include <vector>

#include "mm_defl.cuh"
#include "mm_internal.cuh"
#include "mm_tmpl.cuh"

namespace mm {

namespace {

constexpr int kTNT = 256;

// Legendre values P_k(x) sqrt((2k + 1) / n), k < n_poly (<= kMaxPoly), into constant-indexed p[]
template <typename T>
__device__ __forceinline__ void legendre(const TmplDev& d, int b, int64_t tau, T (&p)[kMaxPoly]) {
  T x;
  if constexpr (sizeof(T) == 4) x = (float)tau * (float)d.xscale[b] - (float)d.xoff[b];
  else x = (double)tau * d.xscale[b] - d.xoff[b];
  T pm = T(1), pc = x;
#pragma unroll
  for (int k = 0; k < kMaxPoly; k++) {
    if (k >= d.n_poly) break;
    T v;
    if (k == 0) {
      v = T(1);
    } else if (k == 1) {
      v = x;
    } else {
      v = ((T)(2 * k - 1) * x * pc - (T)(k - 1) * pm) / (T)k;
      pm = pc;
      pc = v;
    }
    p[k] = v * (T)d.pscale[b * d.n_poly + k];
  }
}

// cos(k phi), sin(k phi), k = 1..n_hwp (<= kMaxHwp), by the angle-addition recurrence
template <typename T>
__device__ __forceinline__ void harmonics(const TmplDev& d, int64_t g, T (&hc)[kMaxHwp], T (&hs)[kMaxHwp]) {
  T s1, c1;
  if constexpr (sizeof(T) == 4) sincosf(d.hwp[g], &s1, &c1);
  else sincos((double)d.hwp[g], &s1, &c1);
  T ck = c1, sk = s1;
#pragma unroll
  for (int k = 0; k < kMaxHwp; k++) {
    if (k >= d.n_hwp) break;
    hc[k] = ck;
    hs[k] = sk;
    const T cn = ck * c1 - sk * s1, sn = sk * c1 + ck * s1;
    ck = cn;
    sk = sn;
  }
}

// per block: lo/hi of az over kept samples, then bins / interpolation fractions of every sample (FP64)
__global__ void k_tmpl_bins(const int32_t* __restrict__ lpix, const float* __restrict__ az,
                            const int64_t* __restrict__ off, int n_az, int interp, int32_t* __restrict__ bin,
                            double* __restrict__ frac) {
  __shared__ double slo[kTNT], shi[kTNT];
  const int b = blockIdx.x;
  const int64_t lo = off[b], hi = off[b + 1];
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t g = lo + threadIdx.x; g < hi; g += kTNT) {
    if (lpix[g] >= 0) {
      const double a = az[g];
      mn = fmin(mn, a);
      mx = fmax(mx, a);
    }
  }
  slo[threadIdx.x] = mn;
  shi[threadIdx.x] = mx;
  __syncthreads();
  for (int sh = kTNT / 2; sh > 0; sh >>= 1) {
    if (threadIdx.x < sh) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + sh]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + sh]);
    }
    __syncthreads();
  }
  double a_lo = slo[0], a_hi = shi[0];
  if (!(a_lo <= a_hi)) a_lo = a_hi = 0.0;   // no kept sample
  for (int64_t g = lo + threadIdx.x; g < hi; g += kTNT) {
    const double a = az[g];
    if (interp) {
      if (a_hi > a_lo && n_az > 1) {
        const double step = (a_hi - a_lo) / (double)(n_az - 1);
        const double pos = fmin(fmax((a - a_lo) / step, 0.0), (double)(n_az - 1));
        const int i = min((int)floor(pos), n_az - 2);
        bin[g] = i;
        frac[g] = pos - (double)i;
      } else {
        bin[g] = 0;
        frac[g] = 0.0;
      }
    } else {
      int i = 0;
      if (a_hi > a_lo) {
        i = (int)floor((a - a_lo) / (a_hi - a_lo) * (double)n_az);
        i = min(max(i, 0), n_az - 1);
      }
      bin[g] = i;
    }
  }
}

// K_b = T^T W T in FP64: 32-sample tiles staged in shared memory, each thread owns a few (i <= j)
constexpr int kGramTile = 32;
constexpr int kGramPairs = (kMaxTmpl * (kMaxTmpl + 1) / 2 + kTNT - 1) / kTNT;
__global__ void __launch_bounds__(kTNT) k_tmpl_gram(TmplDev d, double* __restrict__ K) {
  __shared__ double rows[kGramTile][kMaxTmpl + 1];
  __shared__ double wsm[kGramTile];
  const int b = blockIdx.x;
  const int k = d.k;
  const int64_t lo = d.off[b], hi = d.off[b + 1];
  const double wb = d.w[b];
  const int npairs = k * (k + 1) / 2;
  int pi[kGramPairs], pj[kGramPairs];
  double acc[kGramPairs];
#pragma unroll
  for (int r = 0; r < kGramPairs; r++) {
    acc[r] = 0.0;
    int p = threadIdx.x + r * kTNT, i = 0;
    if (p < npairs) {
      while (p >= k - i) {   // row i of the upper triangle holds k - i pairs
        p -= k - i;
        i++;
      }
    }
    pi[r] = i;
    pj[r] = i + p;
  }
  for (int64_t base = lo; base < hi; base += kGramTile) {
    if (threadIdx.x < kGramTile) {
      const int64_t g = base + threadIdx.x;
      double* row = rows[threadIdx.x];
      for (int j = 0; j < k; j++) row[j] = 0.0;
      if (g < hi) {
        if (d.n_poly > 0) {
          double p[kMaxPoly];
          legendre<double>(d, b, g - lo, p);
#pragma unroll
          for (int q = 0; q < kMaxPoly; q++)
            if (q < d.n_poly) row[q] = p[q];
        }
        if (d.n_az > 0) {
          const int i = d.az_bin[g];
          if (d.interp) {
            const double fr = d.az_frac[g];
            row[d.n_poly + i] = 1.0 - fr;
            if (i + 1 < d.n_az) row[d.n_poly + i + 1] = fr;
          } else {
            row[d.n_poly + i] = 1.0;
          }
        }
        if (d.n_hwp > 0) {
          double hc[kMaxHwp], hs[kMaxHwp];
          harmonics<double>(d, g, hc, hs);
          const int h0 = d.n_poly + d.n_az;
#pragma unroll
          for (int q = 0; q < kMaxHwp; q++)
            if (q < d.n_hwp) {
              row[h0 + 2 * q] = hc[q];
              row[h0 + 2 * q + 1] = hs[q];
            }
        }
        wsm[threadIdx.x] = d.lpix[g] >= 0 ? wb : 0.0;
      } else {
        wsm[threadIdx.x] = 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kGramPairs; r++) {
      if (threadIdx.x + r * kTNT < npairs) {
        double s = acc[r];
        for (int t = 0; t < kGramTile; t++) s += wsm[t] * rows[t][pi[r]] * rows[t][pj[r]];
        acc[r] = s;
      }
    }
    __syncthreads();
  }
  double* Kb = K + (int64_t)b * k * k;
#pragma unroll
  for (int r = 0; r < kGramPairs; r++) {
    if (threadIdx.x + r * kTNT < npairs) {
      Kb[pi[r] * k + pj[r]] = acc[r];
      Kb[pj[r] * k + pi[r]] = acc[r];
    }
  }
}

// per block (one thread): Kinv_b = pseudo-inverse of K_b, eigenvalues below rcond * max |w| dropped
__global__ void k_tmpl_pinv(const double* __restrict__ K, int k, int nb, double rcond, double* __restrict__ work,
                            double* __restrict__ U, double* __restrict__ w, double* __restrict__ Kinv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double* Kb = K + (int64_t)b * k * k;
  double* A = work + (int64_t)b * k * k;
  double* Ub = U + (int64_t)b * k * k;
  double* wb = w + (int64_t)b * k;
  double* out = Kinv + (int64_t)b * k * k;
  for (int i = 0; i < k * k; i++) A[i] = Kb[i];
  jacobi_eig(A, k, wb, Ub);
  double mx = 0.0;
  for (int i = 0; i < k; i++) mx = fmax(mx, fabs(wb[i]));
  for (int i = 0; i < k; i++)
    for (int j = 0; j < k; j++) {
      double s = 0.0;
      for (int l = 0; l < k; l++)
        if (fabs(wb[l]) > rcond * mx) s += Ub[i * k + l] * Ub[j * k + l] / wb[l];
      out[i * k + j] = s;
    }
}

// t <- F_T t block by block, in place (T = float: the CG operator; double: the FP64 operator).
// Pass 1 forms a = T^T W t (Legendre and HWP terms in registers, azimuth bins through FP64
// shared-memory atomics), c = Kinv a; pass 2 writes w (t - T c), 0 at masked samples.
template <typename T>
__global__ void __launch_bounds__(kTNT) k_tmpl_filter(TmplDev d, T* __restrict__ t, int64_t t_stride,
                                                     const int32_t* __restrict__ done, int done_stride) {
  __shared__ double red[kTNT];
  __shared__ double a_sm[kMaxTmpl], c_sm[kMaxTmpl];
  const int b = blockIdx.x, rhs = blockIdx.y;
  if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) return;
  T* tr = t + rhs * t_stride;
  const int k = d.k, c0 = d.n_poly, h0 = d.n_poly + d.n_az;
  const int64_t lo = d.off[b], hi = d.off[b + 1];
  const T wb = (T)d.w[b];
  for (int j = threadIdx.x; j < kMaxTmpl; j += kTNT) a_sm[j] = 0.0;
  __syncthreads();
  T ap[kMaxPoly], ahc[kMaxHwp], ahs[kMaxHwp];
#pragma unroll
  for (int q = 0; q < kMaxPoly; q++) ap[q] = T(0);
#pragma unroll
  for (int q = 0; q < kMaxHwp; q++) ahc[q] = ahs[q] = T(0);
  for (int64_t g = lo + threadIdx.x; g < hi; g += kTNT) {
    if (d.lpix[g] < 0) continue;
    const T v = wb * tr[g];
    if (d.n_poly > 0) {
      T p[kMaxPoly];
      legendre<T>(d, b, g - lo, p);
#pragma unroll
      for (int q = 0; q < kMaxPoly; q++)
        if (q < d.n_poly) ap[q] += p[q] * v;
    }
    if (d.n_az > 0) {
      const int i = d.az_bin[g];
      if (d.interp) {
        const double fr = d.az_frac[g];
        atomicAdd(&a_sm[c0 + i], (1.0 - fr) * (double)v);
        if (i + 1 < d.n_az) atomicAdd(&a_sm[c0 + i + 1], fr * (double)v);
      } else {
        atomicAdd(&a_sm[c0 + i], (double)v);
      }
    }
    if (d.n_hwp > 0) {
      T hc[kMaxHwp], hs[kMaxHwp];
      harmonics<T>(d, g, hc, hs);
#pragma unroll
      for (int q = 0; q < kMaxHwp; q++)
        if (q < d.n_hwp) {
          ahc[q] += hc[q] * v;
          ahs[q] += hs[q] * v;
        }
    }
  }
  __syncthreads();   // every azimuth atomic is in a_sm before it is read
  // block sums of the register terms (FP64 across threads)
  for (int j = 0; j < k; j++) {
    if (j >= c0 && j < h0) continue;   // azimuth terms are already in a_sm
    double x = 0.0;
#pragma unroll
    for (int q = 0; q < kMaxPoly; q++)
      if (j == q) x = (double)ap[q];
#pragma unroll
    for (int q = 0; q < kMaxHwp; q++) {
      if (j == h0 + 2 * q) x = (double)ahc[q];
      if (j == h0 + 2 * q + 1) x = (double)ahs[q];
    }
    red[threadIdx.x] = x;
    __syncthreads();
    for (int sh = kTNT / 2; sh > 0; sh >>= 1) {
      if (threadIdx.x < sh) red[threadIdx.x] += red[threadIdx.x + sh];
      __syncthreads();
    }
    if (threadIdx.x == 0) a_sm[j] = red[0];
    __syncthreads();
  }
  if (threadIdx.x < k) {
    const double* Ki = d.kinv + ((int64_t)b * k + threadIdx.x) * k;
    double s = 0.0;
    for (int l = 0; l < k; l++) s += Ki[l] * a_sm[l];
    c_sm[threadIdx.x] = s;
  }
  __syncthreads();
  T cp[kMaxPoly], chc[kMaxHwp], chs[kMaxHwp];
#pragma unroll
  for (int q = 0; q < kMaxPoly; q++) cp[q] = q < d.n_poly ? (T)c_sm[q] : T(0);
#pragma unroll
  for (int q = 0; q < kMaxHwp; q++) {
    chc[q] = q < d.n_hwp ? (T)c_sm[h0 + 2 * q] : T(0);
    chs[q] = q < d.n_hwp ? (T)c_sm[h0 + 2 * q + 1] : T(0);
  }
  for (int64_t g = lo + threadIdx.x; g < hi; g += kTNT) {
    if (d.lpix[g] < 0) {
      tr[g] = T(0);
      continue;
    }
    T s = T(0);
    if (d.n_poly > 0) {
      T p[kMaxPoly];
      legendre<T>(d, b, g - lo, p);
#pragma unroll
      for (int q = 0; q < kMaxPoly; q++)
        if (q < d.n_poly) s += cp[q] * p[q];
    }
    if (d.n_az > 0) {
      const int i = d.az_bin[g];
      if (d.interp) {
        const double fr = d.az_frac[g];
        s += (T)((1.0 - fr) * c_sm[c0 + i] + (i + 1 < d.n_az ? fr * c_sm[c0 + i + 1] : 0.0));
      } else {
        s += (T)c_sm[c0 + i];
      }
    }
    if (d.n_hwp > 0) {
      T hc[kMaxHwp], hs[kMaxHwp];
      harmonics<T>(d, g, hc, hs);
#pragma unroll
      for (int q = 0; q < kMaxHwp; q++)
        if (q < d.n_hwp) s += chc[q] * hc[q] + chs[q] * hs[q];
    }
    tr[g] = wb * (tr[g] - s);
  }
}

// y (FP32 float4 map, accumulated) += P^T t for the samples of every block
__global__ void k_point32t(const int32_t* __restrict__ lpix, const float2* __restrict__ w32, int64_t N,
                           const float* __restrict__ t, int64_t t_stride, float4* __restrict__ y, int64_t y_stride4,
                           const int32_t* __restrict__ done, int done_stride) {
  const int rhs = blockIdx.y;
  if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) return;
  const float* tr = t + rhs * t_stride;
  float4* yr = y + rhs * y_stride4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = lpix[i];
    if (p < 0) continue;
    const float v = tr[i];
    const float2 cs = w32[i];
    atomicAdd(yr + p, make_float4(v, cs.x * v, cs.y * v, 0.f));
  }
}

template <typename T>
cudaError_t filter_launch(const TmplDev& d, int nb, T* t, int64_t t_stride, int nrhs, const int32_t* done,
                          int done_stride, cudaStream_t s) {
  if (nb <= 0 || nrhs <= 0) return cudaSuccess;
  k_tmpl_filter<T><<<dim3(nb, nrhs), kTNT, 0, s>>>(d, t, t_stride, done, done_stride);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tmpl_setup(TmplDev& d, int nb, double* K, double* work, double* U, double* w, cudaStream_t s) {
  if (d.n_az > 0) k_tmpl_bins<<<nb, kTNT, 0, s>>>(d.lpix, d.az, d.off, d.n_az, d.interp, d.az_bin_w, d.az_frac_w);
  k_tmpl_gram<<<nb, kTNT, 0, s>>>(d, K);
  k_tmpl_pinv<<<(nb + 31) / 32, 32, 0, s>>>(K, d.k, nb, 1e-12, work, U, w, d.kinv_w);
  return cudaGetLastError();
}

cudaError_t launch_tmpl_filter32(const TmplDev& d, int nb, float* t, int64_t t_stride, int nrhs, const int32_t* done,
                                 int done_stride, cudaStream_t s) {
  return filter_launch<float>(d, nb, t, t_stride, nrhs, done, done_stride, s);
}

cudaError_t launch_tmpl_filter64(const TmplDev& d, int nb, double* t, int64_t t_stride, int nrhs, cudaStream_t s) {
  return filter_launch<double>(d, nb, t, t_stride, nrhs, nullptr, 0, s);
}

cudaError_t launch_point32t(const int32_t* lpix, const float2* w32, int64_t N, const float* t, int64_t t_stride,
                            float* y4, int64_t y_stride, int nrhs, const int32_t* done, int done_stride,
                            cudaStream_t s) {
  if (N == 0 || nrhs <= 0) return cudaSuccess;
  int64_t g = (N + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_point32t<<<dim3((unsigned)g, nrhs), 256, 0, s>>>(lpix, w32, N, t, t_stride, reinterpret_cast<float4*>(y4),
                                                      y_stride / 4, done, done_stride);
  return cudaGetLastError();
}

}  // namespace mm
