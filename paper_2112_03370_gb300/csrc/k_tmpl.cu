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

#include <cooperative_groups.h>

#include <vector>

#include "df64.cuh"
#include "mm_defl.cuh"
#include "mm_internal.cuh"
#include "mm_tmpl.cuh"

namespace mm {

namespace {

namespace cg = cooperative_groups;

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
                            double* __restrict__ frac, uint8_t* __restrict__ bin8, float* __restrict__ frac32) {
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
        bin8[g] = (uint8_t)i;
        frac[g] = pos - (double)i;
        frac32[g] = (float)(pos - (double)i);
      } else {
        bin[g] = 0;
        bin8[g] = 0;
        frac[g] = 0.0;
        frac32[g] = 0.f;
      }
    } else {
      int i = 0;
      if (a_hi > a_lo) {
        i = (int)floor((a - a_lo) / (a_hi - a_lo) * (double)n_az);
        i = min(max(i, 0), n_az - 1);
      }
      bin[g] = i;
      bin8[g] = (uint8_t)i;
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

// ---- fused FP32 template operator -------------------------------------------------------------
// One cluster of kTC CTAs per block; CTA r streams the r-th contiguous slice of the block twice.
// Pass 1 un-points x (t = P x, the map gathered from L2), forms v = w_b t and accumulates the slice's
// T^T v: Legendre and HWP terms in registers, azimuth bins as one shared-memory atomic per run of
// equal bins within a warp.  The slices' sums meet over distributed shared memory, every CTA forms
// c = Kinv a from them in the same order, and pass 2 recomputes t and scatters w_b (t - T c) into y.
constexpr int kTC = 8;     // CTAs per block
constexpr int kTA = 256;   // threads per CTA

// unscaled Legendre P_0..P_{n-1}(x) by k P_k = (2k - 1) x P_{k-1} - (k - 1) P_{k-2}
template <int NP>
__device__ __forceinline__ void legendre_raw(float x, int n, float (&p)[NP]) {
  float pm = 1.f, pc = x;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    if (k >= n) break;
    if (k == 0) {
      p[k] = 1.f;
    } else if (k == 1) {
      p[k] = x;
    } else {
      const float v = ((float)(2 * k - 1) / (float)k) * x * pc - ((float)(k - 1) / (float)k) * pm;
      pm = pc;
      pc = v;
      p[k] = v;
    }
  }
}

template <int NH>
__device__ __forceinline__ void harmonics32(float phi, int n, float (&hc)[NH], float (&hs)[NH]) {
  float s1, c1;
  sincosf(phi, &s1, &c1);
  float ck = c1, sk = s1;
#pragma unroll
  for (int k = 0; k < NH; k++) {
    if (k >= n) break;
    hc[k] = ck;
    hs[k] = sk;
    const float cn = ck * c1 - sk * s1, sn = sk * c1 + ck * s1;
    ck = cn;
    sk = sn;
  }
}

// Warp-collective: the lanes' (bin, value) pairs summed per run of equal bins (lanes are consecutive
// samples, so a run is a stretch of constant azimuth bin); the run's first lane adds the sum to a[bin]
// (and the right-node share to a[bin + 1] when interpolating).  bin < 0 marks a lane with no sample.
__device__ __forceinline__ void az_run_sums(double* a, int bin, float v, float fr, int interp, int n_az,
                                            int lane) {
  const int prev = __shfl_up_sync(0xffffffffu, bin, 1);
  const int next = __shfl_down_sync(0xffffffffu, bin, 1);
  const bool head = lane == 0 || prev != bin;
  const unsigned tails = __ballot_sync(0xffffffffu, lane == 31 || next != bin);
  const int end = lane + __ffs(tails >> lane) - 1;   // last lane of this lane's run (bit 31 is set)
  float s0 = interp ? (1.f - fr) * v : v;
  float s1 = interp ? fr * v : 0.f;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float u0 = __shfl_down_sync(0xffffffffu, s0, off);
    if (lane + off <= end) s0 += u0;
  }
  if (interp) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float u1 = __shfl_down_sync(0xffffffffu, s1, off);
      if (lane + off <= end) s1 += u1;
    }
  }
  if (head && bin >= 0) {
    atomicAdd(a + bin, (double)s0);
    if (interp && bin + 1 < n_az) atomicAdd(a + bin + 1, (double)s1);
  }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

template <int NP, int NH>
__global__ void __cluster_dims__(kTC, 1, 1) __launch_bounds__(kTA)
    k_tmpl_apply32(TmplDev d, const float2* __restrict__ w32, const float4* __restrict__ x, int64_t x_stride4,
                   float4* __restrict__ y, int64_t y_stride4, const int32_t* __restrict__ done, int done_stride) {
  constexpr int kW = kTA / 32;
  __shared__ double a_sm[kMaxTmpl];              // this slice's T^T W t
  __shared__ double red[kW][NP + 2 * NH];        // per-warp sums of the register terms
  __shared__ double c_sm[kMaxTmpl];              // c = Kinv a (the whole block's a)
  __shared__ float caz[kMaxTmpl + 1];            // azimuth part of c in FP32 (+1: a zero right node)
  const int rhs = blockIdx.y;
  // every CTA of a cluster reads the same flag, so the cluster leaves together
  if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) return;
  cg::cluster_group cl = cg::this_cluster();
  const int b = blockIdx.x / kTC, rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = d.k, np = d.n_poly, naz = d.n_az, nh = d.n_hwp, c0 = np, h0 = np + naz;
  const int64_t lo = d.off[b], n = d.off[b + 1] - lo;
  const int64_t per = (n + kTC - 1) / kTC;
  const int64_t s_lo = lo + min(n, per * rank), s_hi = lo + min(n, per * (rank + 1));
  const float wb = (float)d.w[b];
  const float xs = (float)d.xscale[b], xo = (float)d.xoff[b];
  const float4* xr = x + rhs * x_stride4;
  for (int j = tid; j < kMaxTmpl; j += kTA) a_sm[j] = 0.0;
  __syncthreads();

  // ---- pass 1: a = T^T W P x over the slice ----
  float ap[NP], ahc[NH], ahs[NH];
#pragma unroll
  for (int q = 0; q < NP; q++) ap[q] = 0.f;
#pragma unroll
  for (int q = 0; q < NH; q++) ahc[q] = ahs[q] = 0.f;
  for (int64_t g0 = s_lo + (tid - lane); g0 < s_hi; g0 += kTA) {   // warp-uniform trip count
    const int64_t g = g0 + lane;
    float v = 0.f, fr = 0.f;
    int bin = -1;
    if (g < s_hi) {
      const int32_t p = d.lpix[g];
      if (p >= 0) {
        const float2 cs = w32[g];
        const float4 m = xr[p];
        v = wb * (m.x + cs.x * m.y + cs.y * m.z);
        if (np > 0) {
          float pl[NP];
          legendre_raw<NP>((float)(g - lo) * xs - xo, np, pl);
#pragma unroll
          for (int q = 0; q < NP; q++)
            if (q < np) ap[q] += pl[q] * v;
        }
        if (nh > 0) {
          float hc[NH], hs[NH];
          harmonics32<NH>(d.hwp[g], nh, hc, hs);
#pragma unroll
          for (int q = 0; q < NH; q++)
            if (q < nh) {
              ahc[q] += hc[q] * v;
              ahs[q] += hs[q] * v;
            }
        }
        if (naz > 0) {
          bin = d.bin8[g];
          if (d.interp) fr = d.frac32[g];
        }
      }
    }
    if (naz > 0) az_run_sums(a_sm + c0, bin, v, fr, d.interp, naz, lane);
  }
  // register terms: warp sums in FP64, then across warps
#pragma unroll
  for (int q = 0; q < NP; q++)
    if (q < np) {
      const double t = warp_sum((double)ap[q]);
      if (lane == 0) red[warp][q] = t;
    }
#pragma unroll
  for (int q = 0; q < NH; q++)
    if (q < nh) {
      const double tc = warp_sum((double)ahc[q]), ts = warp_sum((double)ahs[q]);
      if (lane == 0) {
        red[warp][NP + 2 * q] = tc;
        red[warp][NP + 2 * q + 1] = ts;
      }
    }
  __syncthreads();   // azimuth atomics and warp sums are in shared memory
  if (tid < np) {
    double t = 0.0;
    for (int w = 0; w < kW; w++) t += red[w][tid];
    a_sm[tid] = t * d.pscale[(int64_t)b * np + tid];
  } else if (tid >= NP && tid < NP + 2 * nh) {
    double t = 0.0;
    for (int w = 0; w < kW; w++) t += red[w][tid];
    a_sm[h0 + (tid - NP)] = t;
  }
  // ---- the block's a over the cluster, c = Kinv a ----
  cl.sync();
  double* atot = c_sm;   // reused: a of the whole block, then c
  __shared__ double a_all[kMaxTmpl];
  if (tid < k) {
    double t = 0.0;
    for (int r = 0; r < kTC; r++) t += cl.map_shared_rank(a_sm, r)[tid];
    a_all[tid] = t;
  }
  // remote reads are done: arrive now, wait before leaving (no CTA's shared memory goes away while
  // another CTA may still read it)
  asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
  __syncthreads();
  if (tid < k) {
    const double* Ki = d.kinv + ((int64_t)b * k + tid) * k;
    double t = 0.0;
    for (int l = 0; l < k; l++) t += Ki[l] * a_all[l];
    atot[tid] = t;
  }
  __syncthreads();
  float cp[NP], chc[NH], chs[NH];
#pragma unroll
  for (int q = 0; q < NP; q++) cp[q] = q < np ? (float)(c_sm[q] * d.pscale[(int64_t)b * np + q]) : 0.f;
#pragma unroll
  for (int q = 0; q < NH; q++) {
    chc[q] = q < nh ? (float)c_sm[h0 + 2 * q] : 0.f;
    chs[q] = q < nh ? (float)c_sm[h0 + 2 * q + 1] : 0.f;
  }
  for (int j = tid; j <= naz; j += kTA) caz[j] = j < naz ? (float)c_sm[c0 + j] : 0.f;
  __syncthreads();

  // ---- pass 2: y += P^T w_b (t - T c) ----
  float4* yr = y + rhs * y_stride4;
  for (int64_t g = s_lo + tid; g < s_hi; g += kTA) {
    const int32_t p = d.lpix[g];
    if (p < 0) continue;
    const float2 cs = w32[g];
    const float4 m = xr[p];
    const float t = m.x + cs.x * m.y + cs.y * m.z;
    float sv = 0.f;
    if (np > 0) {
      float pl[NP];
      legendre_raw<NP>((float)(g - lo) * xs - xo, np, pl);
#pragma unroll
      for (int q = 0; q < NP; q++)
        if (q < np) sv += cp[q] * pl[q];
    }
    if (naz > 0) {
      const int i = d.bin8[g];
      if (d.interp) {
        const float fr = d.frac32[g];
        sv += (1.f - fr) * caz[i] + fr * caz[i + 1];   // caz[naz] = 0 covers i + 1 = naz
      } else {
        sv += caz[i];
      }
    }
    if (nh > 0) {
      float hc[NH], hs[NH];
      harmonics32<NH>(d.hwp[g], nh, hc, hs);
#pragma unroll
      for (int q = 0; q < NH; q++)
        if (q < nh) sv += chc[q] * hc[q] + chs[q] * hs[q];
    }
    const float yv = wb * (t - sv);
    atomicAdd(yr + p, make_float4(yv, cs.x * yv, cs.y * yv, 0.f));
  }
  asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

// ---- fused FP64-class (df64) template operator ---------------------------------------------------
// The same two-pass cluster scheme as the FP32 operator with every per-sample quantity in df64 on the
// FP32 pipes (GB300 runs FP64 at 1/64 of the FP32 rate): the pointing weights and cos/sin of the HWP
// angle come precomputed as df64, the Legendre values from the integer-coefficient recurrence of
// Q_k = k! P_k (exact multipliers), the HWP harmonics by complex multiplication.  Per-thread sums stay
// in df64; block, cluster and kernel-inverse arithmetic is FP64.  The result is scattered into the FP64
// map with FP64 atomics after an exact integer widening of each df64 part.

// a b + c with one renormalisation (error a small multiple of 2^-48 (|a b| + |c|))
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  float sum, e2;
  two_sum(p, c.hi, sum, e2);
  float t = __fadd_rn(e, e2);
  t = __fadd_rn(t, c.lo);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  return fast_two_sum(sum, t);
}

// a m for an FP32 m
__device__ __forceinline__ df df_mul_f(df a, float m) {
  const float p = __fmul_rn(a.hi, m);
  float e = __fmaf_rn(a.hi, m, -p);
  e = __fmaf_rn(a.lo, m, e);
  return fast_two_sum(p, e);
}

// Q_k(x) = k! P_k(x), k < n: Q_k = (2k - 1) x Q_{k-1} - (k - 1)^2 Q_{k-2}
template <int NP>
__device__ __forceinline__ void legendre_q_df(df x, int n, df (&q)[NP]) {
  df qm = df_make(1.f, 0.f), qc = x;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    if (k >= n) break;
    if (k == 0) {
      q[k] = df_make(1.f, 0.f);
    } else if (k == 1) {
      q[k] = x;
    } else {
      const df v = df_prod_sum(df_mul_f(x, (float)(2 * k - 1)), qc, df_make(-(float)((k - 1) * (k - 1)), 0.f), qm);
      qm = qc;
      qc = v;
      q[k] = v;
    }
  }
}

// cos(k phi), sin(k phi), k = 1..n, from cos(phi), sin(phi) by complex multiplication
template <int NH>
__device__ __forceinline__ void harmonics_df(float4 cs1, int n, df (&hc)[NH], df (&hs)[NH]) {
  const df c1 = df_make(cs1.x, cs1.y), s1 = df_make(cs1.z, cs1.w);
  df ck = c1, sk = s1;
#pragma unroll
  for (int k = 0; k < NH; k++) {
    if (k >= n) break;
    hc[k] = ck;
    hs[k] = sk;
    if (k + 1 < n) {
      const df cn = df_prod_sum(ck, c1, -sk, s1), sn = df_prod_sum(sk, c1, ck, s1);
      ck = cn;
      sk = sn;
    }
  }
}

__device__ __forceinline__ df shfl_down_df(df v, int off) {
  return df_make(__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off));
}

// az_run_sums in df64 (the run's first lane adds the FP64 value of its sums)
__device__ __forceinline__ void az_run_sums_df(double* a, int bin, df v, df fr, int interp, int n_az, int lane) {
  const int prev = __shfl_up_sync(0xffffffffu, bin, 1);
  const int next = __shfl_down_sync(0xffffffffu, bin, 1);
  const bool head = lane == 0 || prev != bin;
  const unsigned tails = __ballot_sync(0xffffffffu, lane == 31 || next != bin);
  const int end = lane + __ffs(tails >> lane) - 1;
  df s1 = interp ? fr * v : df_make(0.f, 0.f);
  df s0 = interp ? v - s1 : v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const df u0 = shfl_down_df(s0, off);
    if (lane + off <= end) s0 = s0 + u0;
  }
  if (interp) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const df u1 = shfl_down_df(s1, off);
      if (lane + off <= end) s1 = s1 + u1;
    }
  }
  if (head && bin >= 0) {
    atomicAdd(a + bin, df_to_double(s0));
    if (interp && bin + 1 < n_az) atomicAdd(a + bin + 1, df_to_double(s1));
  }
}

// the Legendre abscissa (2 tau - (n - 1)) / (n - 1) in df64 from an exactly split numerator
__device__ __forceinline__ df legendre_x(int64_t tau, int64_t nm1, df inv) {
  const int64_t num = 2 * tau - nm1;
  const float h = (float)num;
  return df_make(h, (float)(num - (int64_t)h)) * inv;
}

template <int NP, int NH, bool TOD>
__global__ void __cluster_dims__(kTC, 1, 1) __launch_bounds__(kTA)
    k_tmpl_apply_df(TmplDev d, const float4* __restrict__ wdf, const float4* __restrict__ mdf, int64_t m_stride4,
                    const float2* __restrict__ tdf, int64_t t_stride, double* __restrict__ y, int64_t y_stride,
                    const int32_t* __restrict__ done, int done_stride) {
  constexpr int kW = kTA / 32;
  __shared__ double a_sm[kMaxTmpl];
  __shared__ double red[kW][NP + 2 * NH];
  __shared__ double a_all[kMaxTmpl];
  __shared__ double c_sm[kMaxTmpl];
  __shared__ df caz[kMaxTmpl + 1];
  const int rhs = blockIdx.y;
  if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) return;
  cg::cluster_group cl = cg::this_cluster();
  const int b = blockIdx.x / kTC, rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = d.k, np = d.n_poly, naz = d.n_az, nh = d.n_hwp, c0 = np, h0 = np + naz;
  const int64_t lo = d.off[b], n = d.off[b + 1] - lo;
  const int64_t per = (n + kTC - 1) / kTC;
  const int64_t s_lo = lo + min(n, per * rank), s_hi = lo + min(n, per * (rank + 1));
  const df wb(d.w[b]);
  const int64_t nm1 = n > 1 ? n - 1 : 0;
  const df inv = n > 1 ? df(1.0 / (double)nm1) : df_make(0.f, 0.f);
  const float4* mr = TOD ? nullptr : mdf + rhs * m_stride4;
  const float2* tr = TOD ? tdf + rhs * t_stride : nullptr;
  for (int j = tid; j < kMaxTmpl; j += kTA) a_sm[j] = 0.0;
  __syncthreads();

  auto tod = [&](int64_t g, int32_t p, float4 w4) -> df {
    if constexpr (TOD) {
      const float2 v = tr[g];
      return df_make(v.x, v.y);
    } else {
      const float4 iq = mr[2 * (int64_t)p], u4 = mr[2 * (int64_t)p + 1];
      return df_make(iq.x, iq.y) +
             df_prod_sum(df_make(w4.x, w4.y), df_make(iq.z, iq.w), df_make(w4.z, w4.w), df_make(u4.x, u4.y));
    }
  };

  // ---- pass 1 ----
  df aq[NP], ahc[NH], ahs[NH];
#pragma unroll
  for (int q = 0; q < NP; q++) aq[q] = df_make(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < NH; q++) ahc[q] = ahs[q] = df_make(0.f, 0.f);
  for (int64_t g0 = s_lo + (tid - lane); g0 < s_hi; g0 += kTA) {
    const int64_t g = g0 + lane;
    df v = df_make(0.f, 0.f), fr = df_make(0.f, 0.f);
    int bin = -1;
    if (g < s_hi) {
      const int32_t p = d.lpix[g];
      if (p >= 0) {
        const float4 w4 = TOD ? make_float4(0.f, 0.f, 0.f, 0.f) : wdf[g];
        v = wb * tod(g, p, w4);
        if (np > 0) {
          df ql[NP];
          legendre_q_df<NP>(legendre_x(g - lo, nm1, inv), np, ql);
#pragma unroll
          for (int q = 0; q < NP; q++)
            if (q < np) aq[q] = df_fma(ql[q], v, aq[q]);
        }
        if (nh > 0) {
          df hc[NH], hs[NH];
          harmonics_df<NH>(d.hwpdf[g], nh, hc, hs);
#pragma unroll
          for (int q = 0; q < NH; q++)
            if (q < nh) {
              ahc[q] = df_fma(hc[q], v, ahc[q]);
              ahs[q] = df_fma(hs[q], v, ahs[q]);
            }
        }
        if (naz > 0) {
          bin = d.bin8[g];
          if (d.interp) {
            const float2 f = d.fracdf[g];
            fr = df_make(f.x, f.y);
          }
        }
      }
    }
    if (naz > 0) az_run_sums_df(a_sm + c0, bin, v, fr, d.interp, naz, lane);
  }
#pragma unroll
  for (int q = 0; q < NP; q++)
    if (q < np) {
      const double t = warp_sum(df_to_double(aq[q]));
      if (lane == 0) red[warp][q] = t;
    }
#pragma unroll
  for (int q = 0; q < NH; q++)
    if (q < nh) {
      const double tc = warp_sum(df_to_double(ahc[q])), ts = warp_sum(df_to_double(ahs[q]));
      if (lane == 0) {
        red[warp][NP + 2 * q] = tc;
        red[warp][NP + 2 * q + 1] = ts;
      }
    }
  __syncthreads();
  if (tid < np) {
    double t = 0.0, fact = 1.0;
    for (int w = 0; w < kW; w++) t += red[w][tid];
    for (int j = 2; j <= tid; j++) fact *= (double)j;
    a_sm[tid] = t * (d.pscale[(int64_t)b * np + tid] / fact);
  } else if (tid >= NP && tid < NP + 2 * nh) {
    double t = 0.0;
    for (int w = 0; w < kW; w++) t += red[w][tid];
    a_sm[h0 + (tid - NP)] = t;
  }
  cl.sync();
  if (tid < k) {
    double t = 0.0;
    for (int r = 0; r < kTC; r++) t += cl.map_shared_rank(a_sm, r)[tid];
    a_all[tid] = t;
  }
  asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
  __syncthreads();
  if (tid < k) {
    const double* Ki = d.kinv + ((int64_t)b * k + tid) * k;
    double t = 0.0;
    for (int l = 0; l < k; l++) t += Ki[l] * a_all[l];
    c_sm[tid] = t;
  }
  __syncthreads();
  df cq[NP], chc[NH], chs[NH];
#pragma unroll
  for (int q = 0; q < NP; q++) {
    double fact = 1.0;
    for (int j = 2; j <= q; j++) fact *= (double)j;
    cq[q] = q < np ? df(c_sm[q] * (d.pscale[(int64_t)b * np + q] / fact)) : df_make(0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < NH; q++) {
    chc[q] = q < nh ? df(c_sm[h0 + 2 * q]) : df_make(0.f, 0.f);
    chs[q] = q < nh ? df(c_sm[h0 + 2 * q + 1]) : df_make(0.f, 0.f);
  }
  for (int j = tid; j <= naz; j += kTA) caz[j] = j < naz ? df(c_sm[c0 + j]) : df_make(0.f, 0.f);
  __syncthreads();

  // ---- pass 2 ----
  double* yr = y + rhs * y_stride;
  for (int64_t g = s_lo + tid; g < s_hi; g += kTA) {
    const int32_t p = d.lpix[g];
    if (p < 0) continue;
    const float4 w4 = wdf[g];
    const df t = tod(g, p, w4);
    df sv = df_make(0.f, 0.f);
    if (np > 0) {
      df ql[NP];
      legendre_q_df<NP>(legendre_x(g - lo, nm1, inv), np, ql);
#pragma unroll
      for (int q = 0; q < NP; q++)
        if (q < np) sv = df_fma(cq[q], ql[q], sv);
    }
    if (naz > 0) {
      const int i = d.bin8[g];
      if (d.interp) {
        const float2 f = d.fracdf[g];
        const df ci = caz[i];
        sv = df_fma(df_make(f.x, f.y), caz[i + 1] - ci, sv + ci);
      } else {
        sv = sv + caz[i];
      }
    }
    if (nh > 0) {
      df hc[NH], hs[NH];
      harmonics_df<NH>(d.hwpdf[g], nh, hc, hs);
#pragma unroll
      for (int q = 0; q < NH; q++)
        if (q < nh) sv = sv + df_prod_sum(chc[q], hc[q], chs[q], hs[q]);
    }
    const df yv = wb * (t - sv);
    double* yp = yr + 4 * (int64_t)p;
    atomicAdd(yp, df_to_double(yv));
    atomicAdd(yp + 1, df_to_double(df_make(w4.x, w4.y) * yv));
    atomicAdd(yp + 2, df_to_double(df_make(w4.z, w4.w) * yv));
  }
  asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

// df64 copies of cos/sin of the HWP angle and of the interpolation fractions (setup)
__global__ void k_tmpl_df_tables(const float* __restrict__ hwp, const double* __restrict__ frac, int64_t N,
                                 float4* __restrict__ hwpdf, float2* __restrict__ fracdf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    if (hwpdf) {
      double sn, cs;
      sincos((double)hwp[i], &sn, &cs);
      const df c(cs), s(sn);
      hwpdf[i] = make_float4(c.hi, c.lo, s.hi, s.lo);
    }
    if (fracdf) {
      const df f(frac[i]);
      fracdf[i] = make_float2(f.hi, f.lo);
    }
  }
}

}  // namespace

cudaError_t launch_tmpl_setup(TmplDev& d, int nb, double* K, double* work, double* U, double* w, cudaStream_t s) {
  if (d.n_az > 0)
    k_tmpl_bins<<<nb, kTNT, 0, s>>>(d.lpix, d.az, d.off, d.n_az, d.interp, d.az_bin_w, d.az_frac_w, d.bin8_w,
                                    d.frac32_w);
  if (d.hwpdf_w || d.fracdf_w) k_tmpl_df_tables<<<152 * 8, 256, 0, s>>>(d.hwp, d.az_frac, d.n_total, d.hwpdf_w, d.fracdf_w);
  k_tmpl_gram<<<nb, kTNT, 0, s>>>(d, K);
  k_tmpl_pinv<<<(nb + 31) / 32, 32, 0, s>>>(K, d.k, nb, 1e-12, work, U, w, d.kinv_w);
  return cudaGetLastError();
}

cudaError_t launch_tmpl_apply32(const TmplDev& d, int nb, const float2* w32, const float* x32, int64_t x_stride,
                                float* y32, int64_t y_stride, int nrhs, const int32_t* done, int done_stride,
                                cudaStream_t s) {
  if (nb <= 0 || nrhs <= 0) return cudaSuccess;
  if ((int64_t)nb * kTC > 0x7fffffffLL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)(nb * kTC), (unsigned)nrhs);
  const float4* x = reinterpret_cast<const float4*>(x32);
  float4* y = reinterpret_cast<float4*>(y32);
  if (d.n_poly <= 4 && d.n_hwp <= 4)
    k_tmpl_apply32<4, 4><<<grid, kTA, 0, s>>>(d, w32, x, x_stride / 4, y, y_stride / 4, done, done_stride);
  else if (d.n_poly <= 4)
    k_tmpl_apply32<4, kMaxHwp><<<grid, kTA, 0, s>>>(d, w32, x, x_stride / 4, y, y_stride / 4, done, done_stride);
  else
    k_tmpl_apply32<kMaxPoly, kMaxHwp><<<grid, kTA, 0, s>>>(d, w32, x, x_stride / 4, y, y_stride / 4, done,
                                                            done_stride);
  return cudaGetLastError();
}

cudaError_t launch_tmpl_apply_df(const TmplDev& d, int nb, const float4* wdf, const float4* mdf, int64_t m_stride4,
                                 const float2* tdf, int64_t t_stride, double* y, int64_t y_stride, int nrhs,
                                 const int32_t* done, int done_stride, cudaStream_t s) {
  if (nb <= 0 || nrhs <= 0) return cudaSuccess;
  if ((int64_t)nb * kTC > 0x7fffffffLL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)(nb * kTC), (unsigned)nrhs);
#define MM_TMPL_DF(NP, NH)                                                                                   \
  do {                                                                                                       \
    if (tdf)                                                                                                 \
      k_tmpl_apply_df<NP, NH, true><<<grid, kTA, 0, s>>>(d, wdf, mdf, m_stride4, tdf, t_stride, y, y_stride, \
                                                         done, done_stride);                                 \
    else                                                                                                     \
      k_tmpl_apply_df<NP, NH, false><<<grid, kTA, 0, s>>>(d, wdf, mdf, m_stride4, tdf, t_stride, y, y_stride,\
                                                          done, done_stride);                                \
  } while (0)
  if (d.n_poly <= 4 && d.n_hwp <= 4) MM_TMPL_DF(4, 4);
  else if (d.n_poly <= 4) MM_TMPL_DF(4, kMaxHwp);
  else MM_TMPL_DF(kMaxPoly, kMaxHwp);
#undef MM_TMPL_DF
  return cudaGetLastError();
}

}  // namespace mm
