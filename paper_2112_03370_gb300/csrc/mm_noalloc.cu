// mm_apply_A_noalloc: y = A x for callers that cannot allocate device memory.
//
// mm_apply_A keeps its padded working copies of x and y in buffers that the plan allocates with
// cudaMalloc the first time they are needed.  Some callers cannot let a library allocate at that
// point: code running inside a memory pool or arena it must not grow, real-time loops where an
// allocation (and the device synchronisation cudaMalloc/cudaFree can imply) is not allowed,
// embedding hosts that account for every byte of device memory themselves.  This entry point
// does the same computation but takes its working space from one fixed array compiled into the
// library (kScratchBytes below), so it calls no cudaMalloc, cudaFree or allocating routine.
//
// Costs and rules of that choice:
//   - every GPU that loads the library holds the array (kScratchBytes) until the process exits;
//   - the working set is limited: nrhs * n_obs padded pixels must fit (checked, MM_EINVAL);
//   - all calls share the one array, so calls whose work overlaps on the GPU (different
//     streams, or different host threads) race and must be serialised by the caller;
//   - the first call on a device looks up the array's device address (cudaGetSymbolAddress);
//     make that first call before any stream capture is under way on the device.
#include <mutex>

#include "mm_internal.cuh"

namespace mm {
namespace {

// Working space: [nrhs][n_obs][4] input map followed by the [nrhs][n_obs][4] accumulated output
// (float64 elements on the FP64 path, float32 on the FP32 path).
constexpr size_t kScratchBytes = 32u << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(MM_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MM_OK;
}

// x [tot][3] float64 -> [tot][4] (float64 or float32), padding element 0
__global__ void k_na_pack(const double* __restrict__ x3, int64_t tot, int fp32, void* __restrict__ x4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = x3[3 * i], b = x3[3 * i + 1], c = x3[3 * i + 2];
    if (fp32) {
      reinterpret_cast<float4*>(x4)[i] = make_float4((float)a, (float)b, (float)c, 0.f);
    } else {
      reinterpret_cast<double2*>(x4)[2 * i] = make_double2(a, b);
      reinterpret_cast<double2*>(x4)[2 * i + 1] = make_double2(c, 0.0);
    }
  }
}

// [tot][4] (float64 or float32) -> y [tot][3] float64
__global__ void k_na_unpack(const void* __restrict__ y4, int64_t tot, int fp32, double* __restrict__ y3) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (fp32) {
      const float4 v = reinterpret_cast<const float4*>(y4)[i];
      y3[3 * i] = v.x; y3[3 * i + 1] = v.y; y3[3 * i + 2] = v.z;
    } else {
      const double* v = reinterpret_cast<const double*>(y4) + 4 * i;
      y3[3 * i] = v[0]; y3[3 * i + 1] = v[1]; y3[3 * i + 2] = v[2];
    }
  }
}

unsigned grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  const int64_t cap = 32 * (int64_t)sm_count();
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" int mm_apply_A_noalloc(mm_plan_t plan, const double* x, double* y, int nrhs, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !x || !y || nrhs <= 0) return fail(MM_EINVAL, "bad argument");
  if (P->algo == MM_TPLZ_DIRECT)
    return fail(MM_EINVAL, "mm_apply_A_noalloc needs an FFT plan (the direct band sum needs a "
                           "time-domain buffer of N samples)");
  if (P->tmpl)
    return fail(MM_EINVAL, "mm_apply_A_noalloc does not apply template filters (they need a "
                           "time-domain buffer of N samples)");
  // MM_DF64 plans: mm_apply_A runs the double-float tiles, which read an N-sample un-pointed
  // buffer; this entry point has no room for it and does not substitute other arithmetic
  if (P->df64 && P->precision != MM_FP32)
    return fail(MM_EINVAL, "mm_apply_A_noalloc does not run MM_DF64 plans (their double-float "
                           "operator needs a time-domain buffer of N samples); use an MM_FP64, "
                           "MM_FP32 or MM_FP32_DF64 plan");
  const bool fp32 = P->precision == MM_FP32;
  const size_t elem = fp32 ? sizeof(float) : sizeof(double);
  const size_t tot = (size_t)nrhs * (size_t)P->n_obs;
  const size_t half = tot * 4 * elem;
  const size_t half_aligned = (half + 255) & ~(size_t)255;
  if (half_aligned + half > kScratchBytes)
    return fail(MM_EINVAL, "mm_apply_A_noalloc: nrhs * n_obs = " + std::to_string(tot) +
                               " padded pixels need " + std::to_string(half_aligned + half) +
                               " bytes of working space; the fixed array holds " +
                               std::to_string(kScratchBytes));
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != P->device) return fail(MM_EINVAL, "the plan's device must be current");
  void* base = nullptr;
  const int st = scratch_address(cur, &base);
  if (st != MM_OK) return st;
  unsigned char* in4 = reinterpret_cast<unsigned char*>(base);
  unsigned char* out4 = in4 + half_aligned;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  k_na_pack<<<grid_of((int64_t)tot), 256, 0, s>>>(x, (int64_t)tot, fp32 ? 1 : 0, in4);
  MM_CUDA(cudaGetLastError());
  // the output is accumulated by atomics: clear what the previous call left in the array
  MM_CUDA(cudaMemsetAsync(out4, 0, half, s));
  TileArgs a{};
  a.nrhs = nrhs;
  a.N = P->N;
  a.lpix = P->lpix;
  a.w32 = P->w32;
  a.w64 = P->w64;
  a.x = in4;
  a.x_stride = P->n_obs * 4;
  a.y = out4;
  a.y_stride = P->n_obs * 4;
  if (fp32) {
    a.tiles = P->segs;
    a.n_tiles = P->n_segs;
    a.tab = P->tab32;
    a.tw = P->tw32;
    MM_CUDA(launch_tiles_fp32(MODE_APPLY, a, P->seg_halo, s));
  } else {
    a.tiles = P->tiles;
    a.n_tiles = P->n_tiles;
    a.tab = P->tab64;
    a.tw = P->tw64;
    MM_CUDA(launch_tiles_fp64(MODE_APPLY, a, s));
  }
  k_na_unpack<<<grid_of((int64_t)tot), 256, 0, s>>>(out4, (int64_t)tot, fp32 ? 1 : 0, y);
  MM_CUDA(cudaGetLastError());
  return MM_OK;
}
