// Template map-making with diagonal weights (Sect. 2, Eq. genMapEstimator with the filtering operator
// F_T = W - W T (T^T W T)^+ T^T W; the templates of Appendix A), one interval per block:
//   Legendre P_k(x), k < n_poly, x = 2 tau / (n - 1) - 1, rescaled by sqrt((2k + 1) / n);
//   azimuth bins over the block's azimuth range (value 1), or linear interpolation between n_az nodes;
//   cos(k phi), sin(k phi) of the HWP angle, k = 1..n_hwp.
// W = diag(w_b) on the kept samples of block b (w_b = the band's c_0 of a lambda = 0 plan), 0 on masked
// ones.  When the templates are attached, the setup decides the azimuth bins and interpolation
// fractions once in FP64 (so every operator uses the same templates), tabulates cos/sin of the HWP
// angle in FP32 and df64, builds T^T W T of every block in df64 and pseudo-inverts it (eigenvalues
// below 1e-12 of the largest dropped).  An application A x = P^T F_T P x = M x - P^T W T c, with
// M = P^T W P per pixel and c = (T^T W T)^+ T^T W P x, then costs one fused kernel that streams each
// block twice (FP32 for the iterations, df64 for the FP64-class operator and the right-hand side).
#include <math.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "df64.cuh"
#include "mm_defl.cuh"
#include "mm_internal.cuh"
#include "mm_tmpl.cuh"

namespace mm {

namespace {

namespace cg = cooperative_groups;

constexpr int kTNT = 256;

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

// ---- fused FP32 template operator -------------------------------------------------------------
// One cluster of kTC CTAs per block; CTA r streams the r-th contiguous slice of the block twice.
// Pass 1 un-points x (t = P x, the map gathered from L2), forms v = w_b t and accumulates the slice's
// T^T v: Legendre and HWP terms in registers, azimuth bins as one shared-memory atomic per run of
// equal bins within a warp.  The slices' sums meet over distributed shared memory, every CTA forms
// c = Kinv a from them in the same order, and pass 2 scatters -w_b T c into y.  The diagonal part
// P^T W P x of the operator is added per pixel (k_tmpl_mx32), so pass 2 needs no map gather.
constexpr int kTC = 8;     // CTAs per block
constexpr int kTA = 256;   // threads per CTA
constexpr int kU = 4;      // samples per thread and step of the FP32 operator (loads in flight)
constexpr int kUdf = 2;    // the same for the df64 operator

// Unscaled Legendre P_k(x), k < n, by k P_k = (2k - 1) x P_{k-1} - (k - 1) P_{k-2}, generated and
// consumed on the fly: acc[k] += P_k(x) v (pass 1), or the dot product sum_k c[k] P_k(x) (pass 2).
template <int NP>
__device__ __forceinline__ void legendre_acc(float x, int n, float v, float (&acc)[NP]) {
  float pm = 1.f, pc = x;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    if (k >= n) break;
    if (k == 0) {
      acc[k] += v;
    } else if (k == 1) {
      acc[k] += x * v;
    } else {
      const float pn = ((float)(2 * k - 1) / (float)k) * x * pc - ((float)(k - 1) / (float)k) * pm;
      pm = pc;
      pc = pn;
      acc[k] += pn * v;
    }
  }
}
template <int NP>
__device__ __forceinline__ float legendre_dot(float x, int n, const float (&c)[NP]) {
  float pm = 1.f, pc = x, s = 0.f;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    if (k >= n) break;
    if (k == 0) {
      s = c[0];
    } else if (k == 1) {
      s += c[1] * x;
    } else {
      const float pn = ((float)(2 * k - 1) / (float)k) * x * pc - ((float)(k - 1) / (float)k) * pm;
      pm = pc;
      pc = pn;
      s += c[k] * pn;
    }
  }
  return s;
}

// cos(k phi), sin(k phi), k = 1..n, by the angle-addition recurrence from cos(phi), sin(phi) (FP32
// roundings of the FP64 values, precomputed), generated and consumed on the fly:
// ac[k-1] += cos(k phi) v and as[k-1] += sin(k phi) v, or sum_k cc[k-1] cos(k phi) + cs[k-1] sin(k phi)
template <int NH>
__device__ __forceinline__ void harmonics_acc(float2 cs1, int n, float v, float (&ac)[NH], float (&as)[NH]) {
  const float c1 = cs1.x, s1 = cs1.y;
  float ck = c1, sk = s1;
#pragma unroll
  for (int k = 0; k < NH; k++) {
    if (k >= n) break;
    ac[k] += ck * v;
    as[k] += sk * v;
    const float cn = ck * c1 - sk * s1, sn = sk * c1 + ck * s1;
    ck = cn;
    sk = sn;
  }
}
template <int NH>
__device__ __forceinline__ float harmonics_dot(float2 cs1, int n, const float (&cc)[NH], const float (&cs)[NH]) {
  const float c1 = cs1.x, s1 = cs1.y;
  float ck = c1, sk = s1, s = 0.f;
#pragma unroll
  for (int k = 0; k < NH; k++) {
    if (k >= n) break;
    s += cc[k] * ck + cs[k] * sk;
    const float cn = ck * c1 - sk * s1, sn = sk * c1 + ck * s1;
    ck = cn;
    sk = sn;
  }
  return s;
}

// Warp-collective: the lanes' (bin, value) pairs summed per run of equal bins (lanes are consecutive
// samples, so a run is a stretch of constant azimuth bin); the run's first lane adds the sum to the
// warp's own FP32 accumulator a[bin] (and the right-node share to a[bin + 1] when interpolating) with a
// native shared-memory atomic.  bin < 0 marks a lane with no sample.
__device__ __forceinline__ void az_run_sums(float* a, int bin, float v, float fr, int interp, int n_az,
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
    atomicAdd(a + bin, s0);
    if (interp && bin + 1 < n_az) atomicAdd(a + bin + 1, s1);
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
  __shared__ float az_w[kW][kMaxTmpl];           // per-warp azimuth sums of pass 1
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
  // slice-relative 32-bit indexing (blocks are shorter than 2^31 samples)
  const int m = (int)(s_hi - s_lo), tau0 = (int)(s_lo - lo);
  const int32_t* lp = d.lpix + s_lo;
  const float2* wp = w32 + s_lo;
  const float2* hp = nh > 0 ? d.hwp32 + s_lo : nullptr;
  const uint8_t* bp = naz > 0 ? d.bin8 + s_lo : nullptr;
  const float* fp = (naz > 0 && d.interp) ? d.frac32 + s_lo : nullptr;
  for (int j = tid; j < kMaxTmpl; j += kTA) a_sm[j] = 0.0;
  for (int j = tid; j < kW * kMaxTmpl; j += kTA) (&az_w[0][0])[j] = 0.f;
  __syncthreads();

  // ---- pass 1: a = T^T W P x over the slice ----
  float ap[NP], ahc[NH], ahs[NH];
#pragma unroll
  for (int q = 0; q < NP; q++) ap[q] = 0.f;
#pragma unroll
  for (int q = 0; q < NH; q++) ahc[q] = ahs[q] = 0.f;
  // warp w takes kU runs of 32 consecutive samples per step (warp-uniform trip count); the loads of
  // all kU samples are issued before their map gathers, and those before any arithmetic
  for (int i0 = warp * 32 * kU; i0 < m; i0 += kTA * kU) {
    int32_t pp[kU];
    float2 cs[kU], hw[kU];
    float fr[kU];
    int bn[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const int i = i0 + u * 32 + lane;
      const bool in = i < m;
      pp[u] = in ? lp[i] : -1;
      cs[u] = in ? wp[i] : make_float2(0.f, 0.f);
      hw[u] = (in && nh > 0) ? hp[i] : make_float2(1.f, 0.f);
      bn[u] = (in && naz > 0) ? (int)bp[i] : -1;
      fr[u] = (in && naz > 0 && d.interp) ? fp[i] : 0.f;
    }
    float4 m[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) m[u] = pp[u] >= 0 ? xr[pp[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const int i = i0 + u * 32 + lane;
      float v = 0.f;
      int bin = -1;
      if (pp[u] >= 0) {
        v = wb * (m[u].x + cs[u].x * m[u].y + cs[u].y * m[u].z);
        if (np > 0) legendre_acc<NP>((float)(tau0 + i) * xs - xo, np, v, ap);
        if (nh > 0) harmonics_acc<NH>(hw[u], nh, v, ahc, ahs);
        bin = bn[u];
      }
      if (naz > 0) az_run_sums(az_w[warp], bin, v, fr[u], d.interp, naz, lane);
    }
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
  if (tid >= kTA - kMaxTmpl && tid - (kTA - kMaxTmpl) < naz) {   // azimuth bins: the warps' sums
    const int j = tid - (kTA - kMaxTmpl);
    double t = 0.0;
    for (int w = 0; w < kW; w++) t += (double)az_w[w][j];
    a_sm[c0 + j] = t;
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

  // ---- pass 2: y -= P^T w_b T c (the diagonal part M x is added per pixel) ----
  float4* yr = y + rhs * y_stride4;
  for (int i0 = warp * 32 * kU; i0 < m; i0 += kTA * kU) {
    int32_t pp[kU];
    float2 cs[kU], hw[kU];
    float fr[kU];
    int bn[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const int i = i0 + u * 32 + lane;
      const bool in = i < m;
      pp[u] = in ? lp[i] : -1;
      cs[u] = in ? wp[i] : make_float2(0.f, 0.f);
      hw[u] = (in && nh > 0) ? hp[i] : make_float2(1.f, 0.f);
      bn[u] = (in && naz > 0) ? (int)bp[i] : 0;
      fr[u] = (in && naz > 0 && d.interp) ? fp[i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kU; u++) {
      if (pp[u] < 0) continue;
      const int i = i0 + u * 32 + lane;
      float sv = 0.f;
      if (np > 0) sv += legendre_dot<NP>((float)(tau0 + i) * xs - xo, np, cp);
      if (naz > 0) {
        const int j = bn[u];
        if (d.interp) sv += (1.f - fr[u]) * caz[j] + fr[u] * caz[j + 1];   // caz[naz] = 0 covers j + 1 = naz
        else sv += caz[j];
      }
      if (nh > 0) sv += harmonics_dot<NH>(hw[u], nh, chc, chs);
      const float yv = -wb * sv;
      atomicAdd(yr + pp[u], make_float4(yv, cs[u].x * yv, cs[u].y * yv, 0.f));
    }
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

// Q_k(x) = k! P_k(x), k < n, by Q_k = (2k - 1) x Q_{k-1} - (k - 1)^2 Q_{k-2} (exact FP32 multipliers),
// generated and consumed on the fly: acc[k] += Q_k v, or sum_k c[k] Q_k
template <int NP>
__device__ __forceinline__ void legendre_q_acc(df x, int n, df v, df (&acc)[NP]) {
  df qm = df_make(1.f, 0.f), qc = x;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    if (k >= n) break;
    if (k == 0) {
      acc[k] = acc[k] + v;
    } else if (k == 1) {
      acc[k] = df_fma(x, v, acc[k]);
    } else {
      const df qn = df_prod_sum(df_mul_f(x, (float)(2 * k - 1)), qc, df_make(-(float)((k - 1) * (k - 1)), 0.f), qm);
      qm = qc;
      qc = qn;
      acc[k] = df_fma(qn, v, acc[k]);
    }
  }
}
template <int NP>
__device__ __forceinline__ df legendre_q_dot(df x, int n, const df (&c)[NP], df s) {
  df qm = df_make(1.f, 0.f), qc = x;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    if (k >= n) break;
    if (k == 0) {
      s = s + c[0];
    } else if (k == 1) {
      s = df_fma(c[1], x, s);
    } else {
      const df qn = df_prod_sum(df_mul_f(x, (float)(2 * k - 1)), qc, df_make(-(float)((k - 1) * (k - 1)), 0.f), qm);
      qm = qc;
      qc = qn;
      s = df_fma(c[k], qn, s);
    }
  }
  return s;
}

// cos(k phi), sin(k phi), k = 1..n, from cos(phi), sin(phi) by complex multiplication, generated and
// consumed on the fly
template <int NH>
__device__ __forceinline__ void harmonics_df_acc(float4 cs1, int n, df v, df (&ac)[NH], df (&as)[NH]) {
  const df c1 = df_make(cs1.x, cs1.y), s1 = df_make(cs1.z, cs1.w);
  df ck = c1, sk = s1;
#pragma unroll
  for (int k = 0; k < NH; k++) {
    if (k >= n) break;
    ac[k] = df_fma(ck, v, ac[k]);
    as[k] = df_fma(sk, v, as[k]);
    if (k + 1 < n) {
      const df cn = df_prod_sum(ck, c1, -sk, s1), sn = df_prod_sum(sk, c1, ck, s1);
      ck = cn;
      sk = sn;
    }
  }
}
template <int NH>
__device__ __forceinline__ df harmonics_df_dot(float4 cs1, int n, const df (&cc)[NH], const df (&cs)[NH], df s) {
  const df c1 = df_make(cs1.x, cs1.y), s1 = df_make(cs1.z, cs1.w);
  df ck = c1, sk = s1;
#pragma unroll
  for (int k = 0; k < NH; k++) {
    if (k >= n) break;
    s = s + df_prod_sum(cc[k], ck, cs[k], sk);
    if (k + 1 < n) {
      const df cn = df_prod_sum(ck, c1, -sk, s1), sn = df_prod_sum(sk, c1, ck, s1);
      ck = cn;
      sk = sn;
    }
  }
  return s;
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

  // the un-pointed value of sample g from its loaded parts: the df64 TOD (TOD mode) or the map's I, Q,
  // U at p with the pointing weights w4
  auto unpoint = [&](float2 tv, float4 w4, float4 iq, float4 u4) -> df {
    if constexpr (TOD) {
      return df_make(tv.x, tv.y);
    } else {
      return df_make(iq.x, iq.y) +
             df_prod_sum(df_make(w4.x, w4.y), df_make(iq.z, iq.w), df_make(w4.z, w4.w), df_make(u4.x, u4.y));
    }
  };
  // loads of kUdf samples of the warp's step (sample g0 + u 32 + lane), then their map gathers
  struct Ld {
    int32_t p;
    float4 w4, h4, iq, u4;
    float2 tv, fr;
    int bin;
  };
  auto load = [&](int64_t g0, Ld (&L)[kUdf], bool need_w, bool gather) {
#pragma unroll
    for (int u = 0; u < kUdf; u++) {
      const int64_t g = g0 + u * 32 + lane;
      const bool in = g < s_hi;
      L[u].p = in ? d.lpix[g] : -1;
      L[u].w4 = (in && need_w) ? wdf[g] : make_float4(0.f, 0.f, 0.f, 0.f);
      L[u].h4 = (in && nh > 0) ? d.hwpdf[g] : make_float4(0.f, 0.f, 0.f, 0.f);
      L[u].bin = (in && naz > 0) ? (int)d.bin8[g] : 0;
      L[u].fr = (in && naz > 0 && d.interp) ? d.fracdf[g] : make_float2(0.f, 0.f);
      if constexpr (TOD) L[u].tv = in ? tr[g] : make_float2(0.f, 0.f);
    }
    if constexpr (!TOD) {
      if (gather) {
#pragma unroll
        for (int u = 0; u < kUdf; u++) {
          const int32_t p = L[u].p;
          L[u].iq = p >= 0 ? mr[2 * (int64_t)p] : make_float4(0.f, 0.f, 0.f, 0.f);
          L[u].u4 = p >= 0 ? mr[2 * (int64_t)p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
  };

  // ---- pass 1 ----
  df aq[NP], ahc[NH], ahs[NH];
#pragma unroll
  for (int q = 0; q < NP; q++) aq[q] = df_make(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < NH; q++) ahc[q] = ahs[q] = df_make(0.f, 0.f);
  for (int64_t g0 = s_lo + (int64_t)warp * 32 * kUdf; g0 < s_hi; g0 += (int64_t)kTA * kUdf) {
    Ld L[kUdf];
    load(g0, L, !TOD, true);
#pragma unroll
    for (int u = 0; u < kUdf; u++) {
      const int64_t g = g0 + u * 32 + lane;
      df v = df_make(0.f, 0.f);
      int bin = -1;
      if (L[u].p >= 0) {
        v = wb * unpoint(L[u].tv, L[u].w4, L[u].iq, L[u].u4);
        if (np > 0) legendre_q_acc<NP>(legendre_x(g - lo, nm1, inv), np, v, aq);
        if (nh > 0) harmonics_df_acc<NH>(L[u].h4, nh, v, ahc, ahs);
        bin = L[u].bin;
      }
      if (naz > 0) az_run_sums_df(a_sm + c0, bin, v, df_make(L[u].fr.x, L[u].fr.y), d.interp, naz, lane);
    }
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
  for (int64_t g0 = s_lo + (int64_t)warp * 32 * kUdf; g0 < s_hi; g0 += (int64_t)kTA * kUdf) {
    Ld L[kUdf];
    load(g0, L, true, false);
#pragma unroll
    for (int u = 0; u < kUdf; u++) {
      const int32_t p = L[u].p;
      if (p < 0) continue;
      const int64_t g = g0 + u * 32 + lane;
      const float4 w4 = L[u].w4;
      df sv = df_make(0.f, 0.f);
      if (np > 0) sv = legendre_q_dot<NP>(legendre_x(g - lo, nm1, inv), np, cq, sv);
      if (naz > 0) {
        const int i = L[u].bin;
        if (d.interp) {
          const df ci = caz[i];
          sv = df_fma(df_make(L[u].fr.x, L[u].fr.y), caz[i + 1] - ci, sv + ci);
        } else {
          sv = sv + caz[i];
        }
      }
      if (nh > 0) sv = harmonics_df_dot<NH>(L[u].h4, nh, chc, chs, sv);
      // TOD mode: w_b (t - T c); map mode: -w_b T c (the diagonal part M x is added per pixel)
      df yv;
      if constexpr (TOD) yv = wb * (df_make(L[u].tv.x, L[u].tv.y) - sv);
      else yv = -(wb * sv);
      double* yp = yr + 4 * (int64_t)p;
      atomicAdd(yp, df_to_double(yv));
      atomicAdd(yp + 1, df_to_double(df_make(w4.x, w4.y) * yv));
      atomicAdd(yp + 2, df_to_double(df_make(w4.z, w4.w) * yv));
    }
  }
  asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

// ---- T^T W T per block (setup) --------------------------------------------------------------------
// One 8-CTA cluster per block, each CTA a slice.  The dense templates (Legendre, HWP) of a 64-sample
// tile are generated once in df64 into shared memory; threads owning a (dense, dense) pair accumulate
// its products over the tile (df64, folded into FP64 per tile).  The azimuth rows come from sweeps of
// short sample segments that sum each run of one bin (df64) and add it to the bin's entry; the
// azimuth-azimuth block is the kept-sample count per bin (binned) or the three interpolation weight
// products.  The slices meet over distributed shared memory and rank 0 writes K_b = w_b (...), the
// Legendre columns carrying their scale sqrt((2q + 1) / n) / q!.
constexpr int kGT = 64;                                   // samples per tile
constexpr int kGSeg = 8;                                  // azimuth sweep segments per tile
constexpr int kMaxDense = kMaxPoly + 2 * kMaxHwp;
constexpr int kMaxPairs = kMaxDense * (kMaxDense + 1) / 2;
constexpr int kGP = (kMaxPairs + kTA - 1) / kTA;          // pairs per thread when they outnumber threads

__device__ __forceinline__ int dense_pair(int i, int j, int D) { return i * D - i * (i - 1) / 2 + (j - i); }

__global__ void __cluster_dims__(kTC, 1, 1) __launch_bounds__(kTA) k_tmpl_gram(TmplDev d, double* __restrict__ K) {
  __shared__ df Td[kMaxDense][kGT];
  __shared__ int sbin[kGT];
  __shared__ df sfr[kGT];
  __shared__ double Sd[kMaxPairs];
  __shared__ double Saz[kMaxDense][kMaxTmpl + 1];
  __shared__ double Sdiag[kMaxTmpl + 1], Soff[kMaxTmpl + 1];
  cg::cluster_group cl = cg::this_cluster();
  const int b = blockIdx.x / kTC, rank = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int k = d.k, np = d.n_poly, naz = d.n_az, nh = d.n_hwp, c0 = np, h0 = np + naz;
  const int D = np + 2 * nh, NP2 = D * (D + 1) / 2;
  const int64_t lo = d.off[b], n = d.off[b + 1] - lo;
  const int64_t per = (n + kTC - 1) / kTC;
  const int64_t s_lo = lo + min(n, per * rank), s_hi = lo + min(n, per * (rank + 1));
  const int64_t nm1 = n > 1 ? n - 1 : 0;
  const df inv = n > 1 ? df(1.0 / (double)nm1) : df_make(0.f, 0.f);
  for (int j = tid; j < kMaxPairs; j += kTA) Sd[j] = 0.0;
  for (int j = tid; j < kMaxDense * (kMaxTmpl + 1); j += kTA) (&Saz[0][0])[j] = 0.0;
  for (int j = tid; j <= kMaxTmpl; j += kTA) Sdiag[j] = Soff[j] = 0.0;
  // pair ownership: H sample phases per pair when pairs are few, else up to kGP pairs per thread
  const int H = NP2 > 0 && NP2 <= kTA ? min(8, kTA / NP2) : 1;
  int pi[kGP], pj[kGP], np_own = 0, phase = 0;
  if (NP2 > 0 && NP2 <= kTA) {
    if (tid < NP2 * H) {
      int p = tid % NP2, i = 0;
      while (p >= D - i) { p -= D - i; i++; }
      pi[0] = i;
      pj[0] = i + p;
      np_own = 1;
      phase = tid / NP2;
    }
  } else {
#pragma unroll
    for (int r = 0; r < kGP; r++) {
      int p = tid + r * kTA, i = 0;
      if (p < NP2) {
        while (p >= D - i) { p -= D - i; i++; }
        pi[r] = i;
        pj[r] = i + p;
        np_own = r + 1;
      }
    }
  }
  double acc[kGP];
#pragma unroll
  for (int r = 0; r < kGP; r++) acc[r] = 0.0;
  __syncthreads();

  for (int64_t base = s_lo; base < s_hi; base += kGT) {
    // ---- phase A: the tile's dense template values, bins and fractions ----
    if (tid < kGT) {
      const int64_t g = base + tid;
      const bool kept = g < s_hi && d.lpix[g] >= 0;
      if (kept) {
        if (np > 0) {
          const df x = legendre_x(g - lo, nm1, inv);
          df qm = df_make(1.f, 0.f), qc = x;
          for (int q = 0; q < np; q++) {
            df v;
            if (q == 0) v = df_make(1.f, 0.f);
            else if (q == 1) v = x;
            else {
              v = df_prod_sum(df_mul_f(x, (float)(2 * q - 1)), qc, df_make(-(float)((q - 1) * (q - 1)), 0.f), qm);
              qm = qc;
              qc = v;
            }
            Td[q][tid] = v;
          }
        }
        if (nh > 0) {
          const float4 h4 = d.hwpdf[g];
          const df c1 = df_make(h4.x, h4.y), s1 = df_make(h4.z, h4.w);
          df ck = c1, sk = s1;
          for (int q = 0; q < nh; q++) {
            Td[np + 2 * q][tid] = ck;
            Td[np + 2 * q + 1][tid] = sk;
            const df cn = df_prod_sum(ck, c1, -sk, s1), sn = df_prod_sum(sk, c1, ck, s1);
            ck = cn;
            sk = sn;
          }
        }
        sbin[tid] = naz > 0 ? (int)d.bin8[g] : -1;
        if (naz > 0 && d.interp) {
          const float2 f = d.fracdf[g];
          sfr[tid] = df_make(f.x, f.y);
        } else {
          sfr[tid] = df_make(0.f, 0.f);
        }
      } else {
        for (int q = 0; q < D; q++) Td[q][tid] = df_make(0.f, 0.f);
        sbin[tid] = -1;
        sfr[tid] = df_make(0.f, 0.f);
      }
    }
    __syncthreads();
    // ---- phase B: dense x dense ----
#pragma unroll
    for (int r = 0; r < kGP; r++) {
      if (r < np_own) {
        const df* ti = Td[pi[r]];
        const df* tj = Td[pj[r]];
        df t = df_make(0.f, 0.f);
        for (int q = phase; q < kGT; q += H) t = df_fma(ti[q], tj[q], t);
        acc[r] += df_to_double(t);
      }
    }
    // ---- phase C: azimuth rows (column c < D: dense c; c == D: azimuth x azimuth) ----
    if (naz > 0) {
      constexpr int seg = kGT / kGSeg;
      for (int item = tid; item < (D + 1) * kGSeg; item += kTA) {
        const int c = item / kGSeg, q0 = (item % kGSeg) * seg;
        int cur = -1;
        df r0 = df_make(0.f, 0.f), r1 = df_make(0.f, 0.f), r2 = df_make(0.f, 0.f);
        int cnt = 0;
        auto flush = [&]() {
          if (cur < 0) return;
          if (c < D) {
            atomicAdd(&Saz[c][cur], df_to_double(r0));
            if (d.interp && cur + 1 < naz) atomicAdd(&Saz[c][cur + 1], df_to_double(r1));
          } else if (!d.interp) {
            atomicAdd(&Sdiag[cur], (double)cnt);
          } else {
            atomicAdd(&Sdiag[cur], df_to_double(r0));
            if (cur + 1 < naz) {
              atomicAdd(&Sdiag[cur + 1], df_to_double(r1));
              atomicAdd(&Soff[cur], df_to_double(r2));
            }
          }
          r0 = r1 = r2 = df_make(0.f, 0.f);
          cnt = 0;
        };
        for (int q = q0; q < q0 + seg; q++) {
          const int bq = sbin[q];
          if (bq < 0) continue;
          if (bq != cur) {
            flush();
            cur = bq;
          }
          if (c < D) {
            const df v = Td[c][q];
            if (d.interp) {
              r1 = df_fma(sfr[q], v, r1);
              r0 = r0 + (v - sfr[q] * v);
            } else {
              r0 = r0 + v;
            }
          } else if (!d.interp) {
            cnt++;
          } else {
            const df f = sfr[q], omf = df_make(1.f, 0.f) - f;
            r0 = df_fma(omf, omf, r0);
            r1 = df_fma(f, f, r1);
            r2 = df_fma(omf, f, r2);
          }
        }
        flush();
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kGP; r++)
    if (r < np_own) atomicAdd(&Sd[dense_pair(pi[r], pj[r], D)], acc[r]);
  cl.sync();
  if (rank == 0) {
    const double wb = d.w[b];
    double* Kb = K + (int64_t)b * k * k;
    for (int e = tid; e < k * k; e += kTA) {
      const int i = e / k, j = e % k;
      const bool ai = i >= c0 && i < h0, aj = j >= c0 && j < h0;
      double v = 0.0;
      auto sc = [&](int t) -> double {   // scale of template t (dense)
        if (t < np) {
          double f = 1.0;
          for (int m = 2; m <= t; m++) f *= (double)m;
          return d.pscale[(int64_t)b * np + t] / f;
        }
        return 1.0;
      };
      auto di = [&](int t) { return t < np ? t : np + (t - h0); };
      if (!ai && !aj) {
        const int x = min(di(i), di(j)), y = max(di(i), di(j));
        const int pidx = dense_pair(x, y, D);
        for (int r = 0; r < kTC; r++) v += cl.map_shared_rank(Sd, r)[pidx];
        v *= sc(i) * sc(j);
      } else if (ai != aj) {
        const int t = ai ? j : i, bz = (ai ? i : j) - c0;
        for (int r = 0; r < kTC; r++) v += cl.map_shared_rank(&Saz[0][0], r)[di(t) * (kMaxTmpl + 1) + bz];
        v *= sc(t);
      } else {
        const int bi = i - c0, bj = j - c0;
        if (bi == bj) {
          for (int r = 0; r < kTC; r++) v += cl.map_shared_rank(Sdiag, r)[bi];
        } else if (d.interp && (bi - bj == 1 || bj - bi == 1)) {
          for (int r = 0; r < kTC; r++) v += cl.map_shared_rank(Soff, r)[min(bi, bj)];
        }
      }
      Kb[e] = wb * v;
    }
  }
  cl.sync();   // rank 0 has read every slice's shared memory
}

// Kinv_b = pseudo-inverse of K_b (eigenvalues below rcond * max |w| dropped): cyclic Jacobi with the
// round-robin ordering of disjoint rotation pairs (each round's rotations commute and are applied at
// once), one CTA per block, A and the eigenvectors U in shared memory.
constexpr int kPinvThreads = 256;
__global__ void __launch_bounds__(kPinvThreads) k_tmpl_pinv(const double* __restrict__ K, int k, double rcond,
                                                            double* __restrict__ Kinv) {
  extern __shared__ double pv_sm[];
  const int ld = k + 1, kk = k + (k & 1), npair = kk / 2;
  double* A = pv_sm;
  double* U = A + k * ld;
  double* cs = U + k * ld;        // [npair][2]
  double* red = cs + 2 * 32;      // [kPinvThreads][2]
  __shared__ int pp[32], qq[32];
  __shared__ int stop;
  const int b = blockIdx.x, tid = threadIdx.x;
  const double* Kb = K + (int64_t)b * k * k;
  for (int e = tid; e < k * k; e += kPinvThreads) {
    const int i = e / k, j = e % k;
    A[i * ld + j] = Kb[e];
    U[i * ld + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < k * k; e += kPinvThreads) {
      const int i = e / k, j = e % k;
      const double a2 = A[i * ld + j] * A[i * ld + j];
      tot += a2;
      if (i != j) off += a2;
    }
    red[2 * tid] = off;
    red[2 * tid + 1] = tot;
    __syncthreads();
    for (int sh = kPinvThreads / 2; sh > 0; sh >>= 1) {
      if (tid < sh) {
        red[2 * tid] += red[2 * (tid + sh)];
        red[2 * tid + 1] += red[2 * (tid + sh) + 1];
      }
      __syncthreads();
    }
    if (tid == 0) stop = (red[0] <= 1e-30 * red[1] || red[0] == 0.0) ? 1 : 0;
    __syncthreads();
    if (stop) break;
    for (int r = 0; r < kk - 1; r++) {
      if (tid < npair) {
        int p, q;
        if (tid == 0) {
          p = r;
          q = kk - 1;
        } else {
          p = (r + tid) % (kk - 1);
          q = (r - tid + kk - 1) % (kk - 1);
        }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, sn = 0.0;
        if (q < k) {
          const double apq = A[p * ld + q];
          if (apq != 0.0) {
            const double theta = (A[q * ld + q] - A[p * ld + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sn = t * c;
          }
        }
        pp[tid] = p;
        qq[tid] = q < k ? q : -1;
        cs[2 * tid] = c;
        cs[2 * tid + 1] = sn;
      }
      __syncthreads();
      for (int it = tid; it < k * npair; it += kPinvThreads) {   // A <- A J, U <- U J (columns p, q)
        const int i = it / npair, m = it % npair, p = pp[m], q = qq[m];
        if (q < 0) continue;
        const double c = cs[2 * m], sn = cs[2 * m + 1];
        const double arp = A[i * ld + p], arq = A[i * ld + q];
        A[i * ld + p] = c * arp - sn * arq;
        A[i * ld + q] = sn * arp + c * arq;
        const double urp = U[i * ld + p], urq = U[i * ld + q];
        U[i * ld + p] = c * urp - sn * urq;
        U[i * ld + q] = sn * urp + c * urq;
      }
      __syncthreads();
      for (int it = tid; it < npair * k; it += kPinvThreads) {   // A <- J^T A (rows p, q)
        const int m = it / k, j = it % k, p = pp[m], q = qq[m];
        if (q < 0) continue;
        const double c = cs[2 * m], sn = cs[2 * m + 1];
        const double apj = A[p * ld + j], aqj = A[q * ld + j];
        A[p * ld + j] = c * apj - sn * aqj;
        A[q * ld + j] = sn * apj + c * aqj;
      }
      __syncthreads();
    }
  }
  // pseudo-inverse from the eigen-decomposition
  double mx = 0.0;
  for (int i = 0; i < k; i++) mx = fmax(mx, fabs(A[i * ld + i]));
  double* out = Kinv + (int64_t)b * k * k;
  for (int e = tid; e < k * k; e += kPinvThreads) {
    const int i = e / k, j = e % k;
    double sum = 0.0;
    for (int l = 0; l < k; l++) {
      const double wl = A[l * ld + l];
      if (fabs(wl) > rcond * mx) sum += U[i * ld + l] * U[j * ld + l] / wl;
    }
    out[e] = sum;
  }
}

// df64 copies of cos/sin of the HWP angle and of the interpolation fractions (setup)
__global__ void k_tmpl_df_tables(const float* __restrict__ hwp, const double* __restrict__ frac, int64_t N,
                                 float4* __restrict__ hwpdf, float2* __restrict__ hwp32, float2* __restrict__ fracdf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    if (hwpdf) {
      double sn, cs;
      sincos((double)hwp[i], &sn, &cs);
      const df c(cs), s(sn);
      hwpdf[i] = make_float4(c.hi, c.lo, s.hi, s.lo);
      hwp32[i] = make_float2(c.hi, s.hi);
    }
    if (fracdf) {
      const df f(frac[i]);
      fracdf[i] = make_float2(f.hi, f.lo);
    }
  }
}

// y += M x per pixel, M = P^T W P (symmetric 3 x 3: m00 m01 m02 m11 m12 m22)
__global__ void k_tmpl_mx32(const float4* __restrict__ M, int64_t n, const float4* __restrict__ x,
                            float4* __restrict__ y, const int32_t* __restrict__ done, int done_stride) {
  const int rhs = blockIdx.y;
  if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) return;
  const float4* xr = x + rhs * n;
  float4* yr = y + rhs * n;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = M[2 * p], c = M[2 * p + 1], v = xr[p];
    float4 o = yr[p];
    o.x += a.x * v.x + a.y * v.y + a.z * v.z;
    o.y += a.y * v.x + a.w * v.y + c.x * v.z;
    o.z += a.z * v.x + c.x * v.y + c.y * v.z;
    yr[p] = o;
  }
}
__global__ void k_tmpl_mx64(const double* __restrict__ M, int64_t n, const double* __restrict__ x,
                            double* __restrict__ y, const int32_t* __restrict__ done, int done_stride) {
  const int rhs = blockIdx.y;
  if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) return;
  const double* xr = x + rhs * n * 4;
  double* yr = y + rhs * n * 4;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double* m = M + 6 * p;
    const double v0 = xr[4 * p], v1 = xr[4 * p + 1], v2 = xr[4 * p + 2];
    yr[4 * p] += m[0] * v0 + m[1] * v1 + m[2] * v2;
    yr[4 * p + 1] += m[1] * v0 + m[3] * v1 + m[4] * v2;
    yr[4 * p + 2] += m[2] * v0 + m[4] * v1 + m[5] * v2;
  }
}
__global__ void k_m64_to_32(const double* __restrict__ M, int64_t n, float4* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double* m = M + 6 * p;
    out[2 * p] = make_float4((float)m[0], (float)m[1], (float)m[2], (float)m[3]);
    out[2 * p + 1] = make_float4((float)m[4], (float)m[5], 0.f, 0.f);
  }
}

}  // namespace

cudaError_t launch_tmpl_setup(TmplDev& d, int nb, double* K, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (d.n_az > 0)
    k_tmpl_bins<<<nb, kTNT, 0, s>>>(d.lpix, d.az, d.off, d.n_az, d.interp, d.az_bin_w, d.az_frac_w, d.bin8_w,
                                    d.frac32_w);
  if (d.hwpdf_w || d.fracdf_w)
    k_tmpl_df_tables<<<8 * sm_count(), 256, 0, s>>>(d.hwp, d.az_frac, d.n_total, d.hwpdf_w, d.hwp32_w, d.fracdf_w);
  k_tmpl_gram<<<nb * kTC, kTA, 0, s>>>(d, K);
  const int k = d.k;
  const size_t smem = (size_t)(2 * k * (k + 1) + 2 * 32 + 2 * kPinvThreads) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_tmpl_pinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tmpl_pinv<<<nb, kPinvThreads, smem, s>>>(K, k, 1e-12, d.kinv_w);
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

cudaError_t launch_tmpl_mx32(const float4* M32, int64_t n_obs, const float* x, float* y, int nrhs, const int32_t* done,
                             int done_stride, cudaStream_t s) {
  if (n_obs == 0 || nrhs <= 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<int64_t>((n_obs + 255) / 256, 8 * (int64_t)sm_count());
  k_tmpl_mx32<<<dim3(g, nrhs), 256, 0, s>>>(M32, n_obs, reinterpret_cast<const float4*>(x),
                                            reinterpret_cast<float4*>(y), done, done_stride);
  return cudaGetLastError();
}

cudaError_t launch_tmpl_mx64(const double* M64, int64_t n_obs, const double* x, double* y, int nrhs,
                             const int32_t* done, int done_stride, cudaStream_t s) {
  if (n_obs == 0 || nrhs <= 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<int64_t>((n_obs + 255) / 256, 8 * (int64_t)sm_count());
  k_tmpl_mx64<<<dim3(g, nrhs), 256, 0, s>>>(M64, n_obs, x, y, done, done_stride);
  return cudaGetLastError();
}

cudaError_t launch_m64_to_32(const double* M64, int64_t n_obs, float4* M32, cudaStream_t s) {
  if (n_obs == 0) return cudaSuccess;
  k_m64_to_32<<<(unsigned)std::min<int64_t>((n_obs + 255) / 256, 8 * (int64_t)sm_count()), 256, 0, s>>>(M64, n_obs, M32);
  return cudaGetLastError();
}

}  // namespace mm
