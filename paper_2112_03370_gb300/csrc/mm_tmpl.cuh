// Template map-making state and kernels (k_tmpl.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

constexpr int kMaxTmpl = 64;   // templates per block: n_poly + n_az + 2 n_hwp
constexpr int kMaxPoly = 16;
constexpr int kMaxHwp = 8;

// What the template kernels read (device pointers).
struct TmplDev {
  int n_poly, n_az, n_hwp, interp, k;
  int64_t n_total;           // samples of the plan (N)
  const int64_t* off;        // [n_blocks + 1] block offsets
  const int32_t* lpix;       // [N] (masked samples have weight 0)
  const double* w;           // [n_blocks] diagonal weight w_b (the band's c_0)
  const double* xscale;      // [n_blocks] 2 / (n_b - 1), and the offset: x = tau xscale - xoff
  const double* xoff;        // [n_blocks] 1 (0 when n_b <= 1, where x = 0)
  const double* pscale;      // [n_blocks][n_poly] sqrt((2k + 1) / n_b)
  const float* az;           // [N] azimuth (setup only)
  const float* hwp;          // [N] HWP angle (setup only)
  const int32_t* az_bin;     // [N] bin, or left interpolation node (setup only)
  const double* az_frac;     // [N] weight of the right node (interpolation; setup only)
  const uint8_t* bin8;       // [N] the same bin as uint8 (n_az <= 64), for the fused operators
  const float* frac32;       // [N] az_frac rounded to FP32 (interpolation)
  const float2* fracdf;      // [N] az_frac as df64 (interpolation)
  const float4* hwpdf;       // [N] cos(phi), sin(phi) of the HWP angle as df64 (hi, lo, hi, lo)
  const float2* hwp32;       // [N] cos(phi), sin(phi) rounded to FP32
  const double* kinv;        // [n_blocks][k][k] pseudo-inverse of T^T W T
  int32_t* az_bin_w;         // writable aliases used by the setup kernels
  double* az_frac_w;
  uint8_t* bin8_w;
  float* frac32_w;
  float2* fracdf_w;
  float4* hwpdf_w;
  float2* hwp32_w;
  double* kinv_w;
};

// Host-side state owned by a plan.
struct TmplState {
  TmplDev dev{};
  uint8_t* bin8 = nullptr;
  float* frac32 = nullptr;
  float2* fracdf = nullptr;
  float4* hwpdf = nullptr;
  float2* hwp32 = nullptr;
  double* M64 = nullptr;     // [n_obs][6] P^T W P per pixel (m00 m01 m02 m11 m12 m22)
  float4* M32 = nullptr;     // [n_obs][2] the same in FP32 (m00 m01 m02 m11 | m12 m22 0 0)
  double* xscale = nullptr;
  double* xoff = nullptr;
  double* pscale = nullptr;
  double* kinv = nullptr;
};

// bins, df64 tables, T^T W T and its pseudo-inverse (scratch K: [nb][k][k])
cudaError_t launch_tmpl_setup(TmplDev& d, int nb, double* K, cudaStream_t s);
// y += M x per pixel (M = P^T W P, the diagonal-weight part of the template operator): FP32 float4 maps
// and FP64 maps [nrhs][n_obs][4], columns with a nonzero done flag skipped
cudaError_t launch_tmpl_mx32(const float4* M32, int64_t n_obs, const float* x, float* y, int nrhs, const int32_t* done,
                             int done_stride, cudaStream_t s);
cudaError_t launch_tmpl_mx64(const double* M64, int64_t n_obs, const double* x, double* y, int nrhs,
                             const int32_t* done, int done_stride, cudaStream_t s);
cudaError_t launch_m64_to_32(const double* M64, int64_t n_obs, float4* M32, cudaStream_t s);
// Fused FP32 template operator, the template part: y -= P^T W T c with c = Kinv T^T W P x, for nrhs
// float4 maps ([nrhs][n_obs][4], stride in floats), columns with a nonzero done flag skipped: one 8-CTA
// cluster per block, no TOD buffer.  With launch_tmpl_mx32 it forms y += P^T F_T P x.
cudaError_t launch_tmpl_apply32(const TmplDev& d, int nb, const float2* w32, const float* x32, int64_t x_stride,
                                float* y32, int64_t y_stride, int nrhs, const int32_t* done, int done_stride,
                                cudaStream_t s);
// Fused FP64-class (df64) template operator into FP64 maps y [nrhs][n_obs][4] (accumulated, stride in
// doubles), columns with a nonzero done flag skipped.  wdf: (cos 2psi, sin 2psi) as df64 per sample.
// Map mode (tdf == nullptr): y += P^T F_T P x with x as the df64 map mdf [nrhs][n_obs][2] float4
// (I, Q | U, 0), m_stride4 float4 per column.  TOD mode: y += P^T F_T t with t the df64 TOD tdf
// [nrhs][t_stride] float2 (the right-hand side P^T F_T G d).
cudaError_t launch_tmpl_apply_df(const TmplDev& d, int nb, const float4* wdf, const float4* mdf, int64_t m_stride4,
                                 const float2* tdf, int64_t t_stride, double* y, int64_t y_stride, int nrhs,
                                 const int32_t* done, int done_stride, cudaStream_t s);

}  // namespace mm
