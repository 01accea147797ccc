// Pixel windows of time-aligned detector groups: the un-pointing P and pointing P^T of the FP32
// A-application (Sect. 3.1, MAPMAT and the local pixel indexation).
//
// Detectors of one focal plane observe nearly the same sky at the same time, so the samples of a
// group of detectors over a short window of time fall on few distinct pixels (ground raster, all
// detectors x 64 samples: 9.6 samples per pixel; satellite spin scan: 3.4), while one detector's
// own samples almost never repeat a pixel within a tile.  The plan gives each sample the rank of
// its pixel among the sorted distinct pixels of its group (a uint16 slot), so
//   P:   a CTA loads the group's map entries once into shared memory and every sample reads its
//        (I, Q, U) from there;
//   P^T: a CTA sums the group's samples per slot in shared memory and then adds each pixel's sum
//        to the global map with one vector atomic, instead of one global atomic per sample (the
//        local reduction before the global one of Sect. 3.1).
// The weights (cos 2psi, sin 2psi) are evaluated in registers from the angle 2psi reduced to
// [-pi, pi] once at plan time in FP64, so the kernels stream 6 bytes of pointing per sample
// (slot + angle) instead of a pixel index and two precomputed weights.
#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kHashBits = 13;
constexpr int kHash = 1 << kHashBits;   // open-addressing set, twice the window capacity
static_assert(kHash >= 2 * kWinCap, "hash set must be sparse");
constexpr int kWarps = kWinThreads / 32;

__device__ __forceinline__ uint32_t hash_of(int32_t p) {
  return ((uint32_t)p * 2654435761u) >> (32 - kHashBits);   // Knuth's multiplicative hash
}

// The chunk of block b that belongs to a group: samples [lo, lo + len) of the global order.
__device__ __forceinline__ void group_chunk(const PGroup& G, const int64_t* __restrict__ block_off, int c,
                                            int64_t& lo, int& len) {
  const int b = G.b0 + c * G.b_stride;
  const int64_t blo = __ldg(block_off + b), bhi = __ldg(block_off + b + 1);
  const int64_t start = blo + G.w0;
  const int64_t n = min(bhi - start, (int64_t)1 << G.log_w);
  lo = start;
  len = n > 0 ? (int)n : 0;
}

// Insert p into the set (bounded probing); returns the position, or -1 when the set is full.
__device__ __forceinline__ int set_insert(int32_t* keys, int32_t p, int* count) {
  uint32_t h = hash_of(p);
  for (int probe = 0; probe < kHash; probe++) {
    const int32_t prev = atomicCAS(keys + h, -1, p);
    if (prev == -1) {
      atomicAdd(count, 1);
      return (int)h;
    }
    if (prev == p) return (int)h;
    h = (h + 1) & (kHash - 1);
  }
  return -1;
}

__device__ __forceinline__ int set_find(const int32_t* keys, int32_t p) {
  uint32_t h = hash_of(p);
  for (int probe = 0; probe < kHash; probe++) {
    const int32_t k = keys[h];
    if (k == p) return (int)h;
    if (k == -1) return -1;
    h = (h + 1) & (kHash - 1);
  }
  return -1;
}

// (cos x, sin x) for x in [-pi, pi] (the plan's reduced 2 psi)
__device__ __forceinline__ void weights_of_angle(float x, float& c, float& s) { __sincosf(x, &s, &c); }

}  // namespace

// One CTA per group.  Count mode (slot == nullptr): n_slots_out[g] = distinct kept pixels of the
// group, or -1 above kWinCap.  Fill mode: the pixel-sorted slot table and every sample's slot.
__global__ void __launch_bounds__(kWinThreads) k_win_build(const PGroup* __restrict__ groups,
                                                           const int64_t* __restrict__ block_off,
                                                           const int32_t* __restrict__ lpix,
                                                           int32_t* __restrict__ n_slots_out,
                                                           uint16_t* __restrict__ slot,
                                                           int32_t* __restrict__ slot_pix) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t* keys = reinterpret_cast<int32_t*>(smem_raw);                 // [kHash]
  int32_t* sorted = keys + kHash;                                       // [kWinCap]
  uint16_t* rank_of = reinterpret_cast<uint16_t*>(sorted + kWinCap);    // [kHash]
  __shared__ int s_count, s_n;
  const PGroup G = groups[blockIdx.x];
  for (int i = threadIdx.x; i < kHash; i += kWinThreads) keys[i] = -1;
  if (threadIdx.x == 0) {
    s_count = 0;
    s_n = 0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < G.n_blk; c += kWarps) {
    int64_t lo;
    int len;
    group_chunk(G, block_off, c, lo, len);
    for (int o = lane; o < len; o += 32) {
      const int32_t p = __ldg(lpix + lo + o);
      if (p < 0) continue;
      if (*(volatile int*)&s_count > kWinCap) break;
      set_insert(keys, p, &s_count);
    }
  }
  __syncthreads();
  const int n = s_count;
  if (slot == nullptr) {
    if (threadIdx.x == 0) n_slots_out[blockIdx.x] = (n > kWinCap) ? -1 : n;
    return;
  }
  if (n != G.n_slots) {   // the host counted with the same kernel; a mismatch is a bug
    if (threadIdx.x == 0) atomicOr(n_slots_out, 1);
    return;
  }
  // compact the set and sort it (bitonic, padded to a power of two with INT_MAX)
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = threadIdx.x; i < kHash; i += kWinThreads)
    if (keys[i] != -1) sorted[atomicAdd(&s_n, 1)] = keys[i];
  __syncthreads();
  for (int i = n + threadIdx.x; i < n2; i += kWinThreads) sorted[i] = 0x7fffffff;
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += kWinThreads) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t a = sorted[i], b = sorted[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            sorted[i] = b;
            sorted[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int k = threadIdx.x; k < n; k += kWinThreads) {
    const int32_t p = sorted[k];
    slot_pix[G.slot_off + k] = p;
    const int h = set_find(keys, p);
    if (h >= 0) rank_of[h] = (uint16_t)k;
  }
  __syncthreads();
  for (int c = warp; c < G.n_blk; c += kWarps) {
    int64_t lo;
    int len;
    group_chunk(G, block_off, c, lo, len);
    for (int o = lane; o < len; o += 32) {
      const int32_t p = __ldg(lpix + lo + o);
      uint16_t r = kNoSlot;
      if (p >= 0) {
        const int h = set_find(keys, p);
        if (h >= 0) r = rank_of[h];
      }
      slot[lo + o] = r;
    }
  }
}

constexpr size_t kBuildSmem = (size_t)kHash * 4 + (size_t)kWinCap * 4 + (size_t)kHash * 2;
constexpr size_t kUnpointSmem = (size_t)kWinCap * sizeof(float4);

#define MM_TRY_CUDA(expr)             \
  do {                                \
    const cudaError_t e_ = (expr);    \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

// dynamic shared-memory limit of a kernel, set once per process
template <typename K>
static cudaError_t smem_limit_once(K kernel, size_t bytes, cudaError_t& status, bool& done) {
  if (!done) {
    status = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done = true;
  }
  return status;
}

cudaError_t launch_win_build(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                             const int32_t* lpix, int32_t* n_slots_out, uint16_t* slot, int32_t* slot_pix,
                             cudaStream_t s) {
  if (n_groups == 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_win_build, kBuildSmem, st, set));
  k_win_build<<<(unsigned)n_groups, kWinThreads, kBuildSmem, s>>>(groups, block_off, lpix, n_slots_out, slot,
                                                                   slot_pix);
  return cudaGetLastError();
}

// t = P x over the windows: one CTA per group, the group's map entries of column r in shared
// memory, then one coalesced pass over the group's samples.  Unroll U keeps U independent
// (slot, angle) load pairs in flight per lane.
__global__ void __launch_bounds__(kWinThreads, 3) k_unpoint_win32(
    const PGroup* __restrict__ groups, const int64_t* __restrict__ block_off,
    const uint16_t* __restrict__ slot, const int32_t* __restrict__ slot_pix, const float* __restrict__ ang2,
    const float4* __restrict__ x4, int64_t x_stride4, int nrhs, const int32_t* __restrict__ done,
    int done_stride, float* __restrict__ t, int64_t t_stride) {
  extern __shared__ float4 win[];   // [kWinCap]
  const PGroup G = groups[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int U = 4;
  for (int r = 0; r < nrhs; r++) {
    if (done != nullptr && done[(int64_t)r * done_stride] != 0) continue;
    const float4* x = x4 + r * x_stride4;
    float* tr = t + r * t_stride;
    __syncthreads();   // the previous column's window is no longer read
    for (int k = threadIdx.x; k < G.n_slots; k += kWinThreads) win[k] = __ldg(x + __ldg(slot_pix + G.slot_off + k));
    __syncthreads();
    for (int c = warp; c < G.n_blk; c += kWarps) {
      int64_t lo;
      int len;
      group_chunk(G, block_off, c, lo, len);
      for (int o0 = lane; o0 < len; o0 += 32 * U) {
        uint16_t sl[U];
        float a[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int o = o0 + 32 * u;
          sl[u] = (o < len) ? __ldg(slot + lo + o) : kNoSlot;
          a[u] = (o < len) ? __ldg(ang2 + lo + o) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int o = o0 + 32 * u;
          if (o < len) {
            float v = 0.f;
            if (sl[u] != kNoSlot) {
              float cs, sn;
              weights_of_angle(a[u], cs, sn);
              const float4 m = win[sl[u]];
              v = m.x + cs * m.y + sn * m.z;
            }
            tr[lo + o] = v;
          }
        }
      }
    }
  }
}

cudaError_t launch_unpoint_win32(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                                 const uint16_t* slot, const int32_t* slot_pix, const float* ang2,
                                 const float* x4, int64_t x_stride, int nrhs, const int32_t* done,
                                 int done_stride, float* t, int64_t t_stride, cudaStream_t s) {
  if (n_groups == 0 || nrhs <= 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_unpoint_win32, kUnpointSmem, st, set));
  k_unpoint_win32<<<(unsigned)n_groups, kWinThreads, kUnpointSmem, s>>>(groups, block_off, slot, slot_pix, ang2,
                                                             reinterpret_cast<const float4*>(x4), x_stride / 4, nrhs,
                                                             done, done_stride, t, t_stride);
  return cudaGetLastError();
}

// y += P^T u over the windows: one CTA per group and column, samples summed per slot in shared
// memory (three FP32 shared-memory atomics per sample), then one float4 global atomic per
// distinct pixel of the group.
__global__ void __launch_bounds__(kWinThreads, 3) k_point_win32(
    const PGroup* __restrict__ groups, const int64_t* __restrict__ block_off,
    const uint16_t* __restrict__ slot, const int32_t* __restrict__ slot_pix, const float* __restrict__ ang2,
    const float* __restrict__ u, int64_t u_stride, int nrhs, const int32_t* __restrict__ done, int done_stride,
    float4* __restrict__ y4, int64_t y_stride4) {
  __shared__ float acc[3][kWinCap];
  const PGroup G = groups[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int U = 4;
  for (int r = 0; r < nrhs; r++) {
    if (done != nullptr && done[(int64_t)r * done_stride] != 0) continue;
    const float* ur = u + r * u_stride;
    for (int k = threadIdx.x; k < G.n_slots; k += kWinThreads) acc[0][k] = acc[1][k] = acc[2][k] = 0.f;
    __syncthreads();
    for (int c = warp; c < G.n_blk; c += kWarps) {
      int64_t lo;
      int len;
      group_chunk(G, block_off, c, lo, len);
      for (int o0 = lane; o0 < len; o0 += 32 * U) {
        uint16_t sl[U];
        float a[U], yv[U];
#pragma unroll
        for (int q = 0; q < U; q++) {
          const int o = o0 + 32 * q;
          sl[q] = (o < len) ? __ldg(slot + lo + o) : kNoSlot;
          a[q] = (o < len) ? __ldg(ang2 + lo + o) : 0.f;
          yv[q] = (o < len) ? __ldg(ur + lo + o) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < U; q++) {
          if (sl[q] != kNoSlot) {
            float cs, sn;
            weights_of_angle(a[q], cs, sn);
            atomicAdd(&acc[0][sl[q]], yv[q]);
            atomicAdd(&acc[1][sl[q]], cs * yv[q]);
            atomicAdd(&acc[2][sl[q]], sn * yv[q]);
          }
        }
      }
    }
    __syncthreads();
    float4* yr = y4 + r * y_stride4;
    for (int k = threadIdx.x; k < G.n_slots; k += kWinThreads) {
      const int32_t p = __ldg(slot_pix + G.slot_off + k);
      atomicAdd(yr + p, make_float4(acc[0][k], acc[1][k], acc[2][k], 0.f));
    }
    __syncthreads();   // the next column clears the sums
  }
}

cudaError_t launch_point_win32(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                               const uint16_t* slot, const int32_t* slot_pix, const float* ang2,
                               const float* u, int64_t u_stride, int nrhs, const int32_t* done,
                               int done_stride, float* y4, int64_t y_stride, cudaStream_t s) {
  if (n_groups == 0 || nrhs <= 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_point_win32<<<(unsigned)n_groups, kWinThreads, 0, s>>>(groups, block_off, slot, slot_pix, ang2, u, u_stride,
                                                           nrhs, done, done_stride, reinterpret_cast<float4*>(y4),
                                                           y_stride / 4);
  return cudaGetLastError();
}

}  // namespace mm
