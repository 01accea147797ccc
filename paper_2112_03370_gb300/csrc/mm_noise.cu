// Noise weights estimated from the data (Sect. 2.2, the paragraph on how the weights are computed,
// with the PSD model of Eq. noisepowermodel at f_0 = 0): the averaged periodogram of each block's
// gap-masked TOD, a fit of log P(f) = log sigma^2 (1 + (f_knee / f)^alpha), and the inverse-noise
// Toeplitz row from the fitted PSD (inverse transform, Gaussian window N(0, lambda/2), cut at
// lambda).
//
// Both transforms are real DFTs of 32768 points, done as a 16384-point complex FFT in shared memory
// (the tiles' FFT) of the packed sequence z_j = x_{2j} + i x_{2j+1}, followed by the split
//   X_k = E_k + W_L^k O_k,  E_k = (Z_k + conj Z_{M-k}) / 2,  O_k = (Z_k - conj Z_{M-k}) / (2i),
// k = 0..M (Z_M = Z_0), W_L = exp(-2 pi i / L).  FP32 transforms, FP64 accumulation and fit.
#include <math.h>

#include <vector>

#include "fft_smem.cuh"
#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kSeg = kL;          // 32768 samples per segment and inverse-transform length
constexpr int kBins = kM + 1;     // k = 0..kSeg/2
constexpr int kFitThreads = 256;
using NoiseFFT = SmemFFT<kLogM, kM, kTileThreads>;
constexpr size_t kNoiseSmem =
    (size_t)(smem_pad(kM) + twiddle_tab_entries(kM) + NoiseFFT::kPassTabEntries) * sizeof(float2) + 64;

__global__ void k_noise_twiddles(float2* tw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kM) return;
  double s, c;
  sincospi(2.0 * (double)k / (double)kM, &s, &c);   // W_M^k = exp(-2 pi i k / M)
  tw[k] = make_float2((float)c, (float)-s);
}

// X_k of the real sequence packed in sm (after the forward transform), k = 0..M
__device__ __forceinline__ float2 real_spectrum(const float2* sm, int k) {
  const int kk = k & (kM - 1);
  const float2 a = sm[smem_pad(NoiseFFT::storage_of(kk))];
  const float2 bz = sm[smem_pad(NoiseFFT::storage_of((kM - kk) & (kM - 1)))];
  const float er = 0.5f * (a.x + bz.x), ei = 0.5f * (a.y - bz.y);     // E_k
  const float orr = 0.5f * (a.y + bz.y), oi = -0.5f * (a.x - bz.x);   // O_k
  float s, c;
  sincospif((float)k / (float)kM, &s, &c);                            // W_L^k = c - i s
  return make_float2(er + c * orr + s * oi, ei + c * oi - s * orr);
}

// One CTA per block: the block's segments one after the other; P[b][k] += |X_k|^2 / n_kept in FP64
// (the row belongs to this CTA), then divided by the number of segments used.
__global__ void __launch_bounds__(kTileThreads, 1)
k_periodogram(const int32_t* __restrict__ pix, const double* __restrict__ d, const int64_t* __restrict__ off,
              const float2* __restrict__ tw_g, double* __restrict__ P, int32_t* __restrict__ nseg_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* tw_sm = sm + smem_pad(kM);
  float2* ptab = tw_sm + twiddle_tab_entries(kM);
  int* kept_sm = reinterpret_cast<int*>(ptab + NoiseFFT::kPassTabEntries);
  const int b = blockIdx.x;
  const int64_t lo = off[b], n = off[b + 1] - lo;
  const TwiddleTab<float2> tw = load_twiddle_tab<float2, kM, kTileThreads>(tw_sm, tw_g);
  double* Pb = P + (int64_t)b * kBins;
  for (int k = threadIdx.x; k < kBins; k += kTileThreads) Pb[k] = 0.0;
  __syncthreads();
  NoiseFFT::build_pass_tables(ptab, tw);
  const int64_t count = n > 0 ? (n / kSeg > 1 ? n / kSeg : 1) : 0;
  int used = 0;
  for (int64_t s = 0; s < count; s++) {
    const int64_t base = lo + s * kSeg;
    const int64_t m = (n - s * kSeg) < kSeg ? (n - s * kSeg) : kSeg;
    if (threadIdx.x == 0) *kept_sm = 0;
    __syncthreads();
    int kept = 0;
    // the pixel and data loads of NB sample pairs per thread are issued before any is used (the data
    // load does not wait for the mask), then G d is packed as complex pairs
    constexpr int NB = 8;
    for (int j0 = threadIdx.x; j0 < kM; j0 += NB * kTileThreads) {
      int32_t pv[NB][2];
      double dv[NB][2];
#pragma unroll
      for (int u = 0; u < NB; u++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int64_t t = 2 * (int64_t)(j0 + u * kTileThreads) + h;
          const bool in = j0 + u * kTileThreads < kM && t < m;
          pv[u][h] = in ? __ldg(pix + base + t) : -1;
          dv[u][h] = in ? __ldg(d + base + t) : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < NB; u++) {
        const int j = j0 + u * kTileThreads;
        if (j >= kM) continue;
        const bool ok0 = pv[u][0] >= 0, ok1 = pv[u][1] >= 0;
        kept += (ok0 ? 1 : 0) + (ok1 ? 1 : 0);
        sm[smem_pad(j)] = make_float2(ok0 ? (float)dv[u][0] : 0.f, ok1 ? (float)dv[u][1] : 0.f);
      }
    }
    atomicAdd(kept_sm, kept);
    __syncthreads();
    const int n_kept = *kept_sm;
    __syncthreads();             // every thread has read the count before it is reset
    if (n_kept == 0) continue;   // uniform across the CTA
    used += 1;
    NoiseFFT::forward(sm, tw, ptab);
    const double inv = 1.0 / (double)n_kept;
    // NB bins per thread: their row entries are read before any is updated (independent round trips)
    for (int k0 = threadIdx.x; k0 < kBins; k0 += NB * kTileThreads) {
      double acc[NB];
#pragma unroll
      for (int u = 0; u < NB; u++) acc[u] = k0 + u * kTileThreads < kBins ? Pb[k0 + u * kTileThreads] : 0.0;
#pragma unroll
      for (int u = 0; u < NB; u++) {
        const int k = k0 + u * kTileThreads;
        if (k >= kBins) continue;
        const float2 X = real_spectrum(sm, k);
        Pb[k] = acc[u] + ((double)X.x * X.x + (double)X.y * X.y) * inv;
      }
    }
    __syncthreads();   // the next segment overwrites sm
  }
  if (used > 0) {
    const double inv = 1.0 / (double)used;
    for (int k = threadIdx.x; k < kBins; k += kTileThreads) Pb[k] *= inv;
  }
  if (threadIdx.x == 0) nseg_out[b] = used;
}

// block-wide FP64 sums of NV values per thread (kFitThreads threads)
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
#pragma unroll
  for (int q = 0; q < NV; q++) red[q * kFitThreads + threadIdx.x] = v[q];
  __syncthreads();
  for (int sh = kFitThreads / 2; sh > 0; sh >>= 1) {
    if (threadIdx.x < sh)
#pragma unroll
      for (int q = 0; q < NV; q++) red[q * kFitThreads + threadIdx.x] += red[q * kFitThreads + threadIdx.x + sh];
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NV; q++) v[q] = red[q * kFitThreads];
  __syncthreads();
}

// cost, J^T J (6) and J^T r (3) of log P_k - log m_k over k = 1..M at theta.  The per-bin terms
// and each thread's partial sums (64 bins) are FP32 (GB300's FP64 rate is 1/64 of FP32); the sums
// across threads are FP64.
__device__ void fit_sums(const float* xs, const float* ys, const double th[3], double out[10], double* red) {
  float v[10];
#pragma unroll
  for (int q = 0; q < 10; q++) v[q] = 0.f;
  const float t0 = (float)th[0], t1 = (float)th[1], t2 = (float)th[2];
  for (int k = 1 + threadIdx.x; k < kBins; k += kFitThreads) {
    const float e = t1 - xs[k];
    const float u = expf(t2 * e);
    const float g = u / (1.f + u);
    const float r = ys[k] - (t0 + log1pf(u));
    const float j1 = t2 * g, j2 = e * g;   // d log m / d theta = (1, alpha g, (log f_knee - log f) g)
    v[0] += r * r;
    v[1] += 1.f; v[2] += j1; v[3] += j2; v[4] += j1 * j1; v[5] += j1 * j2; v[6] += j2 * j2;
    v[7] += r; v[8] += j1 * r; v[9] += j2 * r;
  }
  double w[10];
#pragma unroll
  for (int q = 0; q < 10; q++) w[q] = v[q];
  block_sum<10>(w, red);
#pragma unroll
  for (int q = 0; q < 10; q++) out[q] = w[q];
}

// One CTA per block: the closed-form start of the fit, then Levenberg-Marquardt on
// theta = (log sigma^2, log f_knee, alpha).
__global__ void __launch_bounds__(kFitThreads) k_psd_fit(const double* __restrict__ P, const int32_t* __restrict__ nseg,
                                                         double* __restrict__ theta_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* xs = reinterpret_cast<float*>(smem_raw);   // log f_k
  float* ys = xs + kBins;                           // log P_k
  double* red = reinterpret_cast<double*>(xs + 2 * kBins);   // 2 kBins floats: 8-byte aligned
  __shared__ double th_s[3];
  __shared__ int stop_s;
  const int b = blockIdx.x;
  double* out = theta_out + 3 * (int64_t)b;
  if (nseg[b] == 0) {
    if (threadIdx.x < 3) out[threadIdx.x] = 0.0;
    return;
  }
  const double* Pb = P + (int64_t)b * kBins;
  for (int k = threadIdx.x; k < kBins; k += kFitThreads) {
    xs[k] = logf((float)k / (float)kSeg);
    ys[k] = logf((float)Pb[k]);
  }
  // start: sigma^2 = mean over k >= seg/4; a line through log(P/s2 - 1) vs log f over P > 3 s2
  double v1[1] = {0.0};
  for (int k = kSeg / 4 + threadIdx.x; k < kBins; k += kFitThreads) v1[0] += Pb[k];
  block_sum<1>(v1, red);
  const double s2 = v1[0] / (double)(kBins - kSeg / 4);
  double v5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int k = 1 + threadIdx.x; k < kBins; k += kFitThreads) {
    if (Pb[k] > 3.0 * s2) {
      const double x = log((double)k / (double)kSeg), y = log(Pb[k] / s2 - 1.0);
      v5[0] += 1.0; v5[1] += x; v5[2] += y; v5[3] += x * x; v5[4] += x * y;
    }
  }
  block_sum<5>(v5, red);
  if (threadIdx.x == 0) {
    double a = 1.0, lfk = log(1.0 / (double)kSeg);
    if (v5[0] >= 3.0) {
      const double nn = v5[0];
      const double slope = (nn * v5[4] - v5[1] * v5[2]) / (nn * v5[3] - v5[1] * v5[1]);
      const double icpt = (v5[2] - slope * v5[1]) / nn;
      a = fmin(fmax(-slope, 0.2), 5.0);
      lfk = icpt / a;
    }
    th_s[0] = log(s2); th_s[1] = lfk; th_s[2] = a;
    stop_s = 0;
  }
  __syncthreads();
  double th[3] = {th_s[0], th_s[1], th_s[2]};
  double cur[10];
  fit_sums(xs, ys, th, cur, red);
  double mu = 1e-3;
  for (int it = 0; it < 400; it++) {
    // (J^T J + mu diag(J^T J)) delta = J^T r  (thread 0), then the trial cost (all threads)
    if (threadIdx.x == 0) {
      double A[3][3] = {{cur[1], cur[2], cur[3]}, {cur[2], cur[4], cur[5]}, {cur[3], cur[5], cur[6]}};
      double g[3] = {cur[7], cur[8], cur[9]};
      for (int i = 0; i < 3; i++) A[i][i] *= (1.0 + mu);
      // Cramer's rule on the 3x3 system
      const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
      double dl[3];
      for (int c = 0; c < 3; c++) {
        double M_[3][3];
        for (int i = 0; i < 3; i++)
          for (int j = 0; j < 3; j++) M_[i][j] = (j == c) ? g[i] : A[i][j];
        dl[c] = (M_[0][0] * (M_[1][1] * M_[2][2] - M_[1][2] * M_[2][1]) -
                 M_[0][1] * (M_[1][0] * M_[2][2] - M_[1][2] * M_[2][0]) +
                 M_[0][2] * (M_[1][0] * M_[2][1] - M_[1][1] * M_[2][0])) / det;
      }
      // at most 1 per parameter and step (log sigma^2, log f_knee, alpha): from a poor start an
      // unbounded step can land on the plateau where the 1/f term vanishes and stay there
      double mx = 0.0;
      for (int c = 0; c < 3; c++) {
        if (!isfinite(dl[c])) dl[c] = 0.0;
        mx = fmax(mx, fabs(dl[c]));
      }
      const double sc = mx > 1.0 ? 1.0 / mx : 1.0;
      for (int c = 0; c < 3; c++) th_s[c] = th[c] + sc * dl[c];
    }
    __syncthreads();
    double tr[3] = {th_s[0], th_s[1], th_s[2]};
    double nxt[10];
    fit_sums(xs, ys, tr, nxt, red);
    if (threadIdx.x == 0) {
      const double step = fmax(fabs(tr[0] - th[0]), fmax(fabs(tr[1] - th[1]), fabs(tr[2] - th[2])));
      // an accepted step below 1e-6 (far inside the fit's statistical error, and near the FP32
      // resolution of the cost) ends the fit
      stop_s = (nxt[0] <= cur[0] && step <= 1e-6) ? 1 : 0;
    }
    __syncthreads();
    if (nxt[0] <= cur[0]) {   // accept (every thread holds the same sums)
      for (int c = 0; c < 3; c++) th[c] = tr[c];
      for (int q = 0; q < 10; q++) cur[q] = nxt[q];
      mu = fmax(mu / 3.0, 1e-12);
    } else {
      mu *= 4.0;
    }
    if (stop_s || mu > 1e12) break;
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = th[threadIdx.x];
}

// One CTA per block: S_k = 1 / P(k / seg) (S_0 = 0, S_{seg-k} = S_k) transformed forward as a real
// sequence (S is even, so the DFT is real and equals seg c), then window and cut.
__global__ void __launch_bounds__(kTileThreads, 1)
k_band_from_fit(const double* __restrict__ theta, const int32_t* __restrict__ nseg, const float2* __restrict__ tw_g,
                int lam, double* __restrict__ band) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* tw_sm = sm + smem_pad(kM);
  float2* ptab = tw_sm + twiddle_tab_entries(kM);
  const int b = blockIdx.x;
  double* out = band + (int64_t)b * (lam + 1);
  if (nseg[b] == 0) {
    for (int t = threadIdx.x; t <= lam; t += kTileThreads) out[t] = 0.0;
    return;
  }
  const TwiddleTab<float2> tw = load_twiddle_tab<float2, kM, kTileThreads>(tw_sm, tw_g);
  const float inv_s2 = (float)exp(-theta[3 * b]), lfk = (float)theta[3 * b + 1], a = (float)theta[3 * b + 2];
  for (int j = threadIdx.x; j < kM; j += kTileThreads) {
    float x[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      int k = 2 * j + h;
      if (k > kM) k = kSeg - k;   // S_{seg-k} = S_k
      x[h] = (k == 0) ? 0.f : inv_s2 / (1.f + expf(a * (lfk - logf((float)k / (float)kSeg))));
    }
    sm[smem_pad(j)] = make_float2(x[0], x[1]);
  }
  __syncthreads();
  NoiseFFT::build_pass_tables(ptab, tw);
  __syncthreads();
  NoiseFFT::forward(sm, tw, ptab);
  const double sig = lam / 2.0;
  for (int t = threadIdx.x; t <= lam; t += kTileThreads) {
    const float2 X = real_spectrum(sm, t);
    const double w = lam > 0 ? exp(-0.5 * ((double)t / sig) * ((double)t / sig)) : 1.0;
    out[t] = (double)X.x / (double)kSeg * w;
  }
}

}  // namespace

}  // namespace mm

using namespace mm;

extern "C" int mm_estimate_bands(int32_t n_det, int32_t n_int, const int64_t* block_len, const int32_t* pix,
                                 const double* d, int32_t lambda, double* band, double* params, void* stream) {
  if (n_det <= 0 || n_int <= 0 || !block_len || !pix || !d || !band)
    return fail(MM_EINVAL, "mm_estimate_bands: bad argument");
  if (lambda < 0 || lambda > kMaxLambda) return fail(MM_EINVAL, "mm_estimate_bands: lambda out of range");
  const int nb = n_det * n_int;
  std::vector<int64_t> off(nb + 1, 0);
  for (int b = 0; b < nb; b++) {
    if (block_len[b] < 0) return fail(MM_EINVAL, "mm_estimate_bands: negative block length");
    off[b + 1] = off[b] + block_len[b];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  static int attr_done = 0;
  if (!attr_done) {
    MM_CUDA(cudaFuncSetAttribute(k_periodogram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNoiseSmem));
    MM_CUDA(cudaFuncSetAttribute(k_band_from_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNoiseSmem));
    MM_CUDA(cudaFuncSetAttribute(k_psd_fit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * (kBins + 1) * sizeof(float) + 10 * kFitThreads * sizeof(double))));
    attr_done = 1;
  }
  int64_t* off_d = nullptr;
  float2* tw = nullptr;
  double *P = nullptr, *theta = nullptr;
  int32_t* nseg = nullptr;
  auto release = [&]() {
    cudaFree(off_d); cudaFree(tw); cudaFree(P); cudaFree(theta); cudaFree(nseg);
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc((void**)&off_d, (nb + 1) * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&tw, kM * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&P, (size_t)nb * kBins * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&theta, (size_t)nb * 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&nseg, nb * sizeof(int32_t));
  if (e != cudaSuccess) {
    release();
    return fail(MM_ENOMEM, std::string("mm_estimate_bands: cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(off_d, off.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_noise_twiddles<<<(kM + 255) / 256, 256, 0, s>>>(tw);
    k_periodogram<<<nb, kTileThreads, kNoiseSmem, s>>>(pix, d, off_d, tw, P, nseg);
    k_psd_fit<<<nb, kFitThreads, 2 * (kBins + 1) * sizeof(float) + 10 * kFitThreads * sizeof(double), s>>>(
        P, nseg, theta);
    k_band_from_fit<<<nb, kTileThreads, kNoiseSmem, s>>>(theta, nseg, tw, lambda, band);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && params) e = cudaMemcpyAsync(params, theta, (size_t)nb * 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return cuda_fail(e, "mm_estimate_bands");
  return MM_OK;
}
