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
  const int64_t* off;        // [n_blocks + 1] block offsets
  const int32_t* lpix;       // [N] (masked samples have weight 0)
  const double* w;           // [n_blocks] diagonal weight w_b (the band's c_0)
  const double* xscale;      // [n_blocks] 2 / (n_b - 1), and the offset: x = tau xscale - xoff
  const double* xoff;        // [n_blocks] 1 (0 when n_b <= 1, where x = 0)
  const double* pscale;      // [n_blocks][n_poly] sqrt((2k + 1) / n_b)
  const float* az;           // [N] azimuth (setup only)
  const float* hwp;          // [N] HWP angle
  const int32_t* az_bin;     // [N] bin, or left interpolation node
  const double* az_frac;     // [N] weight of the right node (interpolation)
  const double* kinv;        // [n_blocks][k][k] pseudo-inverse of T^T W T
  int32_t* az_bin_w;         // writable aliases used by the setup kernels
  double* az_frac_w;
  double* kinv_w;
};

// Host-side state owned by a plan.
struct TmplState {
  TmplDev dev{};
  float* az = nullptr;
  float* hwp = nullptr;
  int32_t* az_bin = nullptr;
  double* az_frac = nullptr;
  double* xscale = nullptr;
  double* xoff = nullptr;
  double* pscale = nullptr;
  double* kinv = nullptr;
};

// bins, T^T W T and its pseudo-inverse (scratch K, work, U: [nb][k][k]; w: [nb][k])
cudaError_t launch_tmpl_setup(TmplDev& d, int nb, double* K, double* work, double* U, double* w, cudaStream_t s);
// t <- F_T t for nrhs columns of stride t_stride (FP32 honours per-column done flags)
cudaError_t launch_tmpl_filter32(const TmplDev& d, int nb, float* t, int64_t t_stride, int nrhs, const int32_t* done,
                                 int done_stride, cudaStream_t s);
cudaError_t launch_tmpl_filter64(const TmplDev& d, int nb, double* t, int64_t t_stride, int nrhs, cudaStream_t s);
// y (FP32 float4 maps [nrhs][n_obs][4], accumulated) += P^T t
cudaError_t launch_point32t(const int32_t* lpix, const float2* w32, int64_t N, const float* t, int64_t t_stride,
                            float* y4, int64_t y_stride, int nrhs, const int32_t* done, int done_stride,
                            cudaStream_t s);

}  // namespace mm
