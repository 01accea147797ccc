// Data preparation of the df64 (double-float) A-application and right-hand side.
//
// The df64 tiles (k_tile<df, 2, MODE_APPLY_T> in k_toeplitz.cu) read an un-pointed time stream
// of (hi, lo) float pairs and accumulate P^T N^-1 of it into the FP64 map.  The kernels here
// produce that stream at full occupancy: t = P x (Eq. 1's pointing with weights
// (1, cos 2psi, sin 2psi), Sect. 2) from a df64 copy of the map, or the gap-masked TOD G d of the
// right-hand side.  Plan-time kernels split the FP64 weights, pair tables and twiddles into
// df64 form once.
#include "df64.cuh"
#include "mm_internal.cuh"

namespace mm {

namespace {

__device__ __forceinline__ float4 split4(double a, double b) {
  const df x(a), y(b);
  return make_float4(x.hi, x.lo, y.hi, y.lo);
}

// (cos 2psi, sin 2psi) in FP64, split into df64
__global__ void k_weights_df(const float* __restrict__ psi, int64_t N, float4* __restrict__ w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincos(2.0 * (double)psi[i], &s, &c);
    w[i] = split4(c, s);
  }
}

__global__ void k_c64_to_df(const double2* __restrict__ in, int64_t n, float4* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = split4(v.x, v.y);
  }
}

// FP64 map [nrhs][n_obs][4] -> df64 map [nrhs][n_obs][2] float4
__global__ void k_map_to_df(const double2* __restrict__ m, int64_t n, float4* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 iq = m[2 * i], u = m[2 * i + 1];
    out[2 * i] = split4(iq.x, iq.y);
    out[2 * i + 1] = split4(u.x, 0.0);
  }
}

// t_i = I_p + cos 2psi_i Q_p + sin 2psi_i U_p (p = lpix_i), 0 at gaps and excised pixels; with the
// TOD (d_kind 1: float32, 2: float64) t_i = that - d_i, the time-domain residual.  Lane = sample,
// so the pointing and weight loads coalesce and the map gathers of a scan fall on a few cache
// lines per warp.
__global__ void __launch_bounds__(256) k_unpoint_df(const int32_t* __restrict__ lpix,
                                                    const float4* __restrict__ w, int64_t N,
                                                    const float4* __restrict__ m, int64_t m_stride,
                                                    const int32_t* __restrict__ done, int done_stride,
                                                    const void* __restrict__ d, int d_kind, int64_t d_stride,
                                                    float2* __restrict__ t, int64_t t_stride) {
  const int rhs = blockIdx.y;
  if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) return;
  const float4* mr = m + rhs * m_stride;
  float2* tr = t + rhs * t_stride;
  const float* d32 = reinterpret_cast<const float*>(d) + rhs * d_stride;
  const double* d64 = reinterpret_cast<const double*>(d) + rhs * d_stride;
  constexpr int U = 4;
  for (int64_t i0 = (int64_t)blockIdx.x * 256 * U + threadIdx.x; i0 < N; i0 += (int64_t)gridDim.x * 256 * U) {
    int32_t p[U];
    float4 wv[U], iq[U], u0[U];
    df dv[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = i0 + u * 256;
      p[u] = (i < N) ? __ldg(lpix + i) : -1;
      wv[u] = (i < N) ? __ldg(w + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      dv[u] = df_make(0.f, 0.f);
      if (p[u] >= 0 && d_kind == 1) dv[u] = df_make(__ldcs(d32 + i), 0.f);
      if (p[u] >= 0 && d_kind == 2) dv[u] = df(__ldcs(d64 + i));
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (p[u] >= 0) {
        iq[u] = __ldg(mr + 2 * (int64_t)p[u]);
        u0[u] = __ldg(mr + 2 * (int64_t)p[u] + 1);
      } else {
        iq[u] = u0[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = i0 + u * 256;
      if (i < N) {
        df v = df_make(iq[u].x, iq[u].y) + df_make(wv[u].x, wv[u].y) * df_make(iq[u].z, iq[u].w) +
               df_make(wv[u].z, wv[u].w) * df_make(u0[u].x, u0[u].y);
        if (d_kind != 0) v = v - dv[u];
        tr[i] = (p[u] >= 0) ? make_float2(v.hi, v.lo) : make_float2(0.f, 0.f);
      }
    }
  }
}

// G d in df64: d (float32 or float64) where the sample is kept, 0 elsewhere
template <typename D>
__global__ void k_d_to_df(const int32_t* __restrict__ lpix, const D* __restrict__ d, int64_t N,
                          int64_t d_stride, float2* __restrict__ t, int64_t t_stride) {
  const int rhs = blockIdx.y;
  const D* dr = d + rhs * d_stride;
  float2* tr = t + rhs * t_stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    df v;
    if constexpr (sizeof(D) == 4) v = df_make(dr[i], 0.f);
    else v = df((double)dr[i]);
    tr[i] = (__ldg(lpix + i) >= 0) ? make_float2(v.hi, v.lo) : make_float2(0.f, 0.f);
  }
}

unsigned grid_for(int64_t n, int per_block) {
  int64_t g = (n + per_block - 1) / per_block;
  if (g > 16 * sm_count()) g = 16 * sm_count();
  return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_weights_df(const float* psi, int64_t N, float4* wdf, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_weights_df<<<8 * sm_count(), 256, 0, s>>>(psi, N, wdf);
  return cudaGetLastError();
}

cudaError_t launch_c64_to_df(const double2* in, int64_t n, float4* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_c64_to_df<<<grid_for(n, 256), 256, 0, s>>>(in, n, out);
  return cudaGetLastError();
}

cudaError_t launch_map_to_df(const double* m4, int64_t n_pix4, float4* out, cudaStream_t s) {
  if (n_pix4 == 0) return cudaSuccess;
  k_map_to_df<<<grid_for(n_pix4, 256), 256, 0, s>>>(reinterpret_cast<const double2*>(m4), n_pix4, out);
  return cudaGetLastError();
}

cudaError_t launch_unpoint_df(const int32_t* lpix, const float4* wdf, int64_t N, const float4* mapdf,
                              int64_t n_obs, int nrhs, const int32_t* done, int done_stride, float2* t,
                              int64_t t_stride, cudaStream_t s, const void* d, int d_is_fp32) {
  if (N == 0 || nrhs <= 0) return cudaSuccess;
  const int d_kind = d == nullptr ? 0 : (d_is_fp32 ? 1 : 2);
  k_unpoint_df<<<dim3(grid_for(N, 1024), nrhs), 256, 0, s>>>(lpix, wdf, N, mapdf, 2 * n_obs, done,
                                                             done_stride, d, d_kind, N, t, t_stride);
  return cudaGetLastError();
}

cudaError_t launch_d_to_df(const int32_t* lpix, const void* d, int d_is_fp32, int64_t N, int nrhs,
                           float2* t, int64_t t_stride, cudaStream_t s) {
  if (N == 0 || nrhs <= 0) return cudaSuccess;
  const dim3 grid(grid_for(N, 256), nrhs);
  if (d_is_fp32)
    k_d_to_df<float><<<grid, 256, 0, s>>>(lpix, reinterpret_cast<const float*>(d), N, N, t, t_stride);
  else
    k_d_to_df<double><<<grid, 256, 0, s>>>(lpix, reinterpret_cast<const double*>(d), N, N, t, t_stride);
  return cudaGetLastError();
}

}  // namespace mm
