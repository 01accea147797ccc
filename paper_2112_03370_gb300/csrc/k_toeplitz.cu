// Fused A-apply tiles: un-point -> banded block-Toeplitz product -> point, one overlap-save tile
// per CTA (FP32) or per 2-CTA cluster (FP64).
//
// The block-Toeplitz product y = T(c_b) t (Eq. MADCAP, stbmm of Sect. 3.1) is a linear
// convolution of each block with the symmetric kernel h = (c_lam..c_1, c_0, c_1..c_lam).
// Following the shift-and-overlap approach of Sect. 3.1, a block is cut into overlapping tiles
// of L = 32768 samples; each tile is transformed, multiplied by the kernel's spectrum on the
// L-point circulant, transformed back, and only the outputs whose whole band lies inside the
// tile are kept (L - 2 lam per tile).  Samples outside the block read as zero, so there is no
// wrap-around and no coupling between blocks.
//
// Real-input packing: the L real samples are packed as M = L/2 complex values
// z[n] = t[2n] + i t[2n+1].  Because the kernel is real and even, its spectrum H is real and the
// whole "unpack, multiply by H, repack" step reduces to a per-frequency pair update
//     Z'[k] = a_k Z[k] + i b_k conj(Z[M-k]),
//     a_k = (S_k - D_k sin th_k) / M,  b_k = D_k cos th_k / M,
//     S_k = (H_k + H_{M-k}) / 2,  D_k = (H_k - H_{M-k}) / 2,  th_k = 2 pi k / L,
// which is precomputed per band (in the FFT's storage order) at plan time.
//
// FP64: a 16384-point complex tile needs 256 KB, more than one CTA's shared memory.  The tile is
// split by one radix-2 decimation-in-frequency step done while gathering: CTA 0 transforms
// e[n] = z[n] + z[n+M/2] (the even frequencies), CTA 1 transforms o[n] = (z[n] - z[n+M/2]) W_M^n
// (the odd ones).  The pair update stays inside each CTA (k and M-k have the same parity), and
// the final radix-2 decimation-in-time step reads the partner CTA's half once through
// distributed shared memory.
#include <cooperative_groups.h>

#include "fft_smem.cuh"
#include "mm_internal.cuh"

namespace cg = cooperative_groups;

namespace mm {

namespace {

template <typename T> struct Map4;
template <> struct Map4<float> {
  // FP32 map: float4 per pixel (I, Q, U, 0)
  static __device__ __forceinline__ void load(const void* base, int64_t off, int32_t p, float& I,
                                              float& Q, float& U) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(base) + off / 4 + p);
    I = v.x; Q = v.y; U = v.z;
  }
  static __device__ __forceinline__ void add(void* base, int64_t off, int32_t p, float a, float b,
                                             float c) {
    atomicAdd(reinterpret_cast<float4*>(base) + off / 4 + p, make_float4(a, b, c, 0.f));
  }
};
template <> struct Map4<double> {
  static __device__ __forceinline__ void load(const void* base, int64_t off, int32_t p, double& I,
                                              double& Q, double& U) {
    const double2* b = reinterpret_cast<const double2*>(reinterpret_cast<const double*>(base) + off) +
                       2 * (int64_t)p;
    const double2 v0 = __ldg(b), v1 = __ldg(b + 1);
    I = v0.x; Q = v0.y; U = v1.x;
  }
  static __device__ __forceinline__ void add(void* base, int64_t off, int32_t p, double a, double b,
                                             double c) {
    double* q = reinterpret_cast<double*>(base) + off + 4 * (int64_t)p;
    atomicAdd(q, a);
    atomicAdd(q + 1, b);
    atomicAdd(q + 2, c);
  }
};

// Pointing weights (cos 2psi, sin 2psi) of sample g.
template <typename T> struct Weights;
template <> struct Weights<float> {
  static __device__ __forceinline__ void get(const TileArgs& a, int64_t g, float& c, float& s) {
    const float psi = __ldg(a.psi + g);
    sincosf(2.f * psi, &s, &c);
  }
};
template <> struct Weights<double> {
  static __device__ __forceinline__ void get(const TileArgs& a, int64_t g, double& c, double& s) {
    const double2 w = __ldg(a.w64 + g);
    c = w.x;
    s = w.y;
  }
};

// Time-domain input value of sample g for the tile's mode (0 outside the block).
template <typename T, int MODE>
__device__ __forceinline__ T sample_in(const TileArgs& a, int rhs, int64_t g, int64_t lo, int64_t hi) {
  if (g < lo || g >= hi) return T(0);
  if (MODE == MODE_NINV) {
    return (T)__ldg(reinterpret_cast<const double*>(a.x) + rhs * a.x_stride + g);
  }
  const int32_t p = __ldg(a.lpix + g);
  if (p < 0) return T(0);
  if (MODE == MODE_RHS) {
    if (a.x_is_fp32) return (T)__ldg(reinterpret_cast<const float*>(a.x) + rhs * a.x_stride + g);
    return (T)__ldg(reinterpret_cast<const double*>(a.x) + rhs * a.x_stride + g);
  }
  T c, s, I, Q, U;
  Weights<T>::get(a, g, c, s);
  Map4<T>::load(a.x, rhs * a.x_stride, p, I, Q, U);
  return I + c * Q + s * U;
}

// Output of sample g: accumulate into the map (APPLY / RHS) or store (NINV).
template <typename T, int MODE>
__device__ __forceinline__ void sample_out(const TileArgs& a, int rhs, int64_t g, T y) {
  if (MODE == MODE_NINV) {
    reinterpret_cast<double*>(a.y)[rhs * a.y_stride + g] = (double)y;
    return;
  }
  const int32_t p = __ldg(a.lpix + g);
  if (p < 0) return;
  T c, s;
  Weights<T>::get(a, g, c, s);
  Map4<T>::add(a.y, rhs * a.y_stride, p, y, c * y, s * y);
}

// Same for the two samples of one packed complex value, merging them when they hit one pixel.
template <typename T, int MODE>
__device__ __forceinline__ void pair_out(const TileArgs& a, int rhs, int64_t g, bool e0, bool e1,
                                         T y0, T y1) {
  if (MODE == MODE_NINV) {
    if (e0) sample_out<T, MODE>(a, rhs, g, y0);
    if (e1) sample_out<T, MODE>(a, rhs, g + 1, y1);
    return;
  }
  const int32_t p0 = e0 ? __ldg(a.lpix + g) : -1;
  const int32_t p1 = e1 ? __ldg(a.lpix + g + 1) : -1;
  T c0 = 0, s0 = 0, c1 = 0, s1 = 0;
  if (p0 >= 0) Weights<T>::get(a, g, c0, s0);
  if (p1 >= 0) Weights<T>::get(a, g + 1, c1, s1);
  if (p0 >= 0 && p0 == p1) {
    Map4<T>::add(a.y, rhs * a.y_stride, p0, y0 + y1, c0 * y0 + c1 * y1, s0 * y0 + s1 * y1);
    return;
  }
  if (p0 >= 0) Map4<T>::add(a.y, rhs * a.y_stride, p0, y0, c0 * y0, s0 * y0);
  if (p1 >= 0) Map4<T>::add(a.y, rhs * a.y_stride, p1, y1, c1 * y1, s1 * y1);
}

}  // namespace

// One overlap-save tile (CL = 1) or half a tile (CL = 2) per CTA.
template <typename T, int CL, int MODE>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile(const TileArgs a) {
  using C = typename V2<T>::t;
  constexpr int LOGMS = kLogM - (CL == 2 ? 1 : 0);
  constexpr int MS = 1 << LOGMS;
  using FFT = SmemFFT<LOGMS, kM, kTileThreads>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);

  const int64_t unit = blockIdx.x / CL;
  const int rank = (CL == 2) ? (int)(blockIdx.x % CL) : 0;
  const int rhs = (int)(unit % a.nrhs);
  // both CTAs of a cluster read the same flag, so they leave together
  if (a.done != nullptr && a.done[(int64_t)rhs * a.done_stride] != 0) return;
  const int64_t tile_id = unit / a.nrhs;
  const TileDesc td = a.tiles[tile_id];
  const C* __restrict__ tw = reinterpret_cast<const C*>(a.tw);

  // ---- gather: packed complex input (CL = 2: with the first radix-2 DIF step) ----
  for (int n = threadIdx.x; n < MS; n += kTileThreads) {
    const int64_t g = td.in0 + 2 * (int64_t)n;
    C z{sample_in<T, MODE>(a, rhs, g, td.blk_lo, td.blk_hi),
        sample_in<T, MODE>(a, rhs, g + 1, td.blk_lo, td.blk_hi)};
    if (CL == 2) {
      const int64_t g2 = g + 2 * (int64_t)MS;
      const C z2{sample_in<T, MODE>(a, rhs, g2, td.blk_lo, td.blk_hi),
                 sample_in<T, MODE>(a, rhs, g2 + 1, td.blk_lo, td.blk_hi)};
      z = (rank == 0) ? c_add(z, z2) : c_mul(c_sub(z, z2), __ldg(tw + n));
    }
    sm[smem_pad(n)] = z;
  }
  __syncthreads();

  FFT::forward(sm, tw);

  // ---- pair update with the band's precomputed (a_k, b_k) in storage order ----
  {
    const C* __restrict__ tab =
        reinterpret_cast<const C*>(a.tab) + ((int64_t)td.tab * CL + rank) * MS;
    const T sc = (T)td.scale;
    for (int j = threadIdx.x; j < MS; j += kTileThreads) {
      const int k = FFT::freq_of(j);
      const int kp = (CL == 2 && rank == 1) ? (MS - 1 - k) : ((MS - k) & (MS - 1));
      const int jp = FFT::storage_of(kp);
      if (j > jp) continue;
      const C ab = __ldg(tab + j);
      const C z = sm[smem_pad(j)];
      if (j == jp) {
        sm[smem_pad(j)] = C{sc * (ab.x * z.x + ab.y * z.y), sc * (ab.x * z.y + ab.y * z.x)};
      } else {
        const C abp = __ldg(tab + jp);
        const C zp = sm[smem_pad(jp)];
        // a Z + i b conj(Zp) = (a x + b yp, a y + b xp)
        sm[smem_pad(j)] = C{sc * (ab.x * z.x + ab.y * zp.y), sc * (ab.x * z.y + ab.y * zp.x)};
        sm[smem_pad(jp)] = C{sc * (abp.x * zp.x + abp.y * z.y), sc * (abp.x * zp.y + abp.y * z.x)};
      }
    }
  }
  __syncthreads();

  FFT::inverse(sm, tw);

  // ---- scatter of the tile's valid outputs ----
  const int64_t r_lo = td.out_lo - td.in0, r_hi = td.out_hi - td.in0;   // real offsets
  if constexpr (CL == 1) {
    const int n_lo = (int)(r_lo >> 1), n_hi = (int)((r_hi + 1) >> 1);
    for (int n = n_lo + threadIdx.x; n < n_hi; n += kTileThreads) {
      const C z = sm[smem_pad(n)];
      const int64_t g = td.in0 + 2 * (int64_t)n;
      pair_out<T, MODE>(a, rhs, g, g >= td.out_lo && g < td.out_hi,
                        g + 1 >= td.out_lo && g + 1 < td.out_hi, z.x, z.y);
    }
  } else {
    cg::cluster_group cl = cg::this_cluster();
    if (rank == 1) {
      for (int n = threadIdx.x; n < MS; n += kTileThreads) {
        sm[smem_pad(n)] = c_mulc(sm[smem_pad(n)], __ldg(tw + n));   // W_M^{-n} O'[n]
      }
    }
    cl.sync();
    const C* other = cl.map_shared_rank(sm, rank ^ 1);
    // complex outputs [n_lo, n_hi): rank 0 owns [0, MS), rank 1 owns [MS, 2 MS)
    const int n_lo = (int)(r_lo >> 1), n_hi = (int)((r_hi + 1) >> 1);
    const int lo = max(n_lo - rank * MS, 0), hi = min(n_hi - rank * MS, MS);
    for (int n = lo + threadIdx.x; n < hi; n += kTileThreads) {
      const C mine = sm[smem_pad(n)];
      const C theirs = other[smem_pad(n)];
      const C z = (rank == 0) ? c_add(mine, theirs) : c_sub(theirs, mine);
      const int64_t g = td.in0 + 2 * ((int64_t)n + rank * MS);
      pair_out<T, MODE>(a, rhs, g, g >= td.out_lo && g < td.out_hi,
                        g + 1 >= td.out_lo && g + 1 < td.out_hi, z.x, z.y);
    }
    cl.sync();
  }
}

constexpr size_t kSmemBytes32 = (size_t)smem_pad(kM) * sizeof(float2);
constexpr size_t kSmemBytes64 = (size_t)smem_pad(kM / 2) * sizeof(double2);

int tile_kernels_init() {
  static int done = 0;
  static int status = MM_OK;
  if (done) return status;
  done = 1;
  cudaError_t e = cudaSuccess;
#define MM_SET(K, B)                                                                       \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(B));
  MM_SET((k_tile<float, 1, MODE_APPLY>), kSmemBytes32);
  MM_SET((k_tile<float, 1, MODE_RHS>), kSmemBytes32);
  MM_SET((k_tile<double, 2, MODE_APPLY>), kSmemBytes64);
  MM_SET((k_tile<double, 2, MODE_RHS>), kSmemBytes64);
  MM_SET((k_tile<double, 2, MODE_NINV>), kSmemBytes64);
#undef MM_SET
  if (e == cudaSuccess) {
    // 2-CTA clusters with 136 KB of dynamic shared memory each are a non-portable size only in
    // CTA count terms; allow it explicitly.
    e = cudaFuncSetAttribute((k_tile<double, 2, MODE_APPLY>), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  if (e != cudaSuccess) status = cuda_fail(e, "tile kernel attributes");
  return status;
}

template <typename T, int CL, int MODE>
static cudaError_t launch_tiles(const TileArgs& a, size_t smem, cudaStream_t s) {
  const int64_t n_cta = a.n_tiles * a.nrhs * CL;
  if (n_cta == 0) return cudaSuccess;
  if (n_cta > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_cta);
  cfg.blockDim = dim3(kTileThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  int na = 0;
  if (CL > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    na = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, k_tile<T, CL, MODE>, a);
}

cudaError_t launch_tiles_fp32(int mode, const TileArgs& a, cudaStream_t s) {
  if (mode == MODE_APPLY) return launch_tiles<float, 1, MODE_APPLY>(a, kSmemBytes32, s);
  if (mode == MODE_RHS) return launch_tiles<float, 1, MODE_RHS>(a, kSmemBytes32, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tiles_fp64(int mode, const TileArgs& a, cudaStream_t s) {
  if (mode == MODE_APPLY) return launch_tiles<double, 2, MODE_APPLY>(a, kSmemBytes64, s);
  if (mode == MODE_RHS) return launch_tiles<double, 2, MODE_RHS>(a, kSmemBytes64, s);
  if (mode == MODE_NINV) return launch_tiles<double, 2, MODE_NINV>(a, kSmemBytes64, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// plan-time tables
// ---------------------------------------------------------------------------------------------

// H_j = c_0 + 2 sum_{tau=1}^{lam} c_tau cos(2 pi tau j / L), j = 0..M: the L-point circulant
// spectrum of the band (real and even because the kernel is symmetric).
__global__ void k_spectra(const double* __restrict__ band_rows, int32_t lambda,
                          const double* __restrict__ costab, double* __restrict__ H) {
  extern __shared__ double c_s[];
  const int tab = blockIdx.y;
  const double* c = band_rows + (int64_t)tab * (lambda + 1);
  for (int i = threadIdx.x; i <= lambda; i += blockDim.x) c_s[i] = c[i];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > kM) return;
  double acc = 0.0;
  for (int tau = 1; tau <= lambda; tau++) {
    acc = fma(c_s[tau], __ldg(costab + (((int64_t)tau * j) & (kL - 1))), acc);
  }
  H[(int64_t)tab * (kM + 1) + j] = c_s[0] + 2.0 * acc;
}

cudaError_t launch_spectra(const double* band_rows, int32_t n_tab, int32_t lambda, double* H,
                           const double* costab, cudaStream_t s) {
  if (n_tab == 0) return cudaSuccess;
  const int nt = 256;
  const size_t sm = (size_t)(lambda + 1) * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (sm > 48 * 1024) e = cudaFuncSetAttribute(k_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  for (int32_t t0 = 0; t0 < n_tab; t0 += 65535) {   // gridDim.y limit
    const int32_t nt_y = (n_tab - t0) < 65535 ? (n_tab - t0) : 65535;
    dim3 grid((kM + 1 + nt - 1) / nt, nt_y);
    k_spectra<<<grid, nt, sm, s>>>(band_rows + (int64_t)t0 * (lambda + 1), lambda, costab,
                                   H + (int64_t)t0 * (kM + 1));
  }
  return cudaGetLastError();
}

// (a_k, b_k) of the pair update for every storage position of both layouts.
template <int CL>
__global__ void k_pair_table(const double* __restrict__ H, const double* __restrict__ costab,
                             int32_t n_tab, void* __restrict__ out, int fp32) {
  constexpr int LOGMS = kLogM - (CL == 2 ? 1 : 0);
  constexpr int MS = 1 << LOGMS;
  using FFT = SmemFFT<LOGMS, kM, kTileThreads>;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_tab * kM) return;
  const int tab = (int)(idx / kM);
  const int rem = (int)(idx % kM);
  const int rank = rem / MS, j = rem % MS;
  const int k = CL * FFT::freq_of(j) + rank;       // global frequency, 0 <= k < M
  const double* h = H + (int64_t)tab * (kM + 1);
  const double S = 0.5 * (h[k] + h[kM - k]);
  const double D = 0.5 * (h[k] - h[kM - k]);
  const double cth = costab[k];
  const double sth = costab[(k - kL / 4) & (kL - 1)];
  const double inv_m = 1.0 / (double)kM;
  const double av = (S - D * sth) * inv_m;
  const double bv = D * cth * inv_m;
  if (fp32) reinterpret_cast<float2*>(out)[idx] = make_float2((float)av, (float)bv);
  else reinterpret_cast<double2*>(out)[idx] = make_double2(av, bv);
}

cudaError_t launch_pair_tables(const double* H, int32_t n_tab, const double* costab, double2* tab64,
                               float2* tab32, cudaStream_t s) {
  if (n_tab == 0) return cudaSuccess;
  const int64_t n = (int64_t)n_tab * kM;
  const int nt = 256;
  const unsigned nb = (unsigned)((n + nt - 1) / nt);
  k_pair_table<kCl64><<<nb, nt, 0, s>>>(H, costab, n_tab, tab64, 0);
  k_pair_table<kCl32><<<nb, nt, 0, s>>>(H, costab, n_tab, tab32, 1);
  return cudaGetLastError();
}

// tw[k] = W_M^k = exp(-2 pi i k / M) = cos(2 pi 2k / L) - i sin(2 pi 2k / L)
__global__ void k_twiddles(double2* tw64, float2* tw32, const double* __restrict__ costab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kM) return;
  const double c = costab[(2 * k) & (kL - 1)];
  const double s = costab[(2 * k - kL / 4) & (kL - 1)];
  tw64[k] = make_double2(c, -s);
  tw32[k] = make_float2((float)c, (float)-s);
}

cudaError_t launch_twiddles(double2* tw64, float2* tw32, const double* costab, cudaStream_t s) {
  k_twiddles<<<(kM + 255) / 256, 256, 0, s>>>(tw64, tw32, costab);
  return cudaGetLastError();
}

}  // namespace mm
