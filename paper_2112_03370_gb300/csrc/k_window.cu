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
#include <algorithm>

#include "df64.cuh"
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

// Streaming arrays (slot, angle, TOD) are read and written with the evict-first cache policy
// (__ldcs / __stcs) so that they do not push the map, which the window gathers and the per-pixel
// atomics reuse, out of L2.

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
constexpr size_t kUnpointSmem = (size_t)(kWinCap + kWinCap / 8) * sizeof(float4);

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

// ---- chunk walking shared by the un-point and point kernels ------------------------------------
// A warp takes CPI = 32 / LPC chunks at a time, LPC = min(32, W / 4) lanes per chunk.  Inside a
// chunk [lo, lo + len) the lanes walk aligned quads of 4 samples [a0, a1) (a0 = lo rounded up to
// 4) with vector loads; the at most 3 + 3 samples before a0 and after a1 go one per lane.
struct ChunkWalk {
  int lpc, cpi, sub, ql;
};
__device__ __forceinline__ ChunkWalk chunk_walk(const PGroup& G, int lane) {
  ChunkWalk w;
  w.lpc = G.log_w >= 7 ? 32 : (1 << (G.log_w - 2));
  w.cpi = 32 / w.lpc;
  w.sub = lane / w.lpc;
  w.ql = lane % w.lpc;
  return w;
}

// Visit every sample of chunk c: f_quad(base, q4) for aligned quads (samples base + 4 q4 .. + 3),
// f_one(i) for the single samples of the ragged ends.  Global sample indices are 64-bit.
template <typename FQ, typename F1>
__device__ __forceinline__ void visit_chunk(const PGroup& G, const int64_t* __restrict__ block_off, int c,
                                            const ChunkWalk& w, FQ f_quad, F1 f_one) {
  int64_t lo;
  int len;
  group_chunk(G, block_off, c, lo, len);
  if (len <= 0) return;
  const int64_t a0 = (lo + 3) & ~(int64_t)3;
  const int head = (int)min((int64_t)len, a0 - lo);
  const int nq = (len - head) >> 2;
  const int tail = len - head - 4 * nq;
  const int64_t a1 = a0 + 4 * (int64_t)nq;
  if (w.ql < head) f_one(lo + w.ql);
  if (w.ql < tail) f_one(a1 + w.ql);
  for (int q = w.ql; q < nq; q += w.lpc) f_quad(a0, q);
}

// L2 prefetch of the lines of samples [lo, lo + len) of one array, spread over the LPC lanes of a
// chunk: elements lo + k (128 / sizeof(T)) and the last one touch every line of the range, and
// every address stays inside it.  A warp issues it for the chunk of its next iteration, so that
// iteration's loads find their lines in L2 while this one waits on DRAM.  Used by the un-point
// kernel and the double-float point kernel (the FP32 point kernel measured slower with it: its
// shared-memory adds, not its loads, set its pace).
template <typename T>
__device__ __forceinline__ void prefetch_chunk(const T* base, int64_t lo, int len, const ChunkWalk& w) {
  constexpr int kPerLine = 128 / (int)sizeof(T);
  for (int o = w.ql * kPerLine; o < len; o += w.lpc * kPerLine)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(base + lo + o)));
  if (w.ql == 0 && len > 0)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(base + lo + len - 1)));
}

// Pointing loads (slot, angle): evict-first when a pass has one column; with several columns the
// CTA reads the same group's pointing once per column, so it is kept in L2 for the later ones.
template <typename T>
__device__ __forceinline__ T ld_point(const T* p, bool keep) { return keep ? __ldg(p) : __ldcs(p); }

// Padded shared-memory indices of slot k.  A lane holds 4 consecutive samples, so one warp-wide
// access touches slots about 4 x (pixels per sample) apart; one padding word per 32 scalar slots
// (accumulators) or one padding float4 per 8 slots (map window) keeps strides of 1, 2, 4 and 8
// slots in distinct banks.
__device__ __forceinline__ int acc_index(int k) { return k + (k >> 5); }
__device__ __forceinline__ int win_index(int k) { return k + (k >> 3); }
constexpr int kAccStride = kWinCap + kWinCap / 32;
constexpr int kWinEntries = kWinCap + kWinCap / 8;

// t = P x over the windows: one CTA per group, the group's map entries of column r in shared
// memory, then one coalesced pass over the group's samples.  MULTI: the group's problem (one
// column) comes from probs[G.prob].
template <bool MULTI>
__global__ void __launch_bounds__(kWinThreads, 3) k_unpoint_win32(
    const PGroup* __restrict__ groups, const int64_t* __restrict__ block_off,
    const uint16_t* __restrict__ slot, const int32_t* __restrict__ slot_pix, const float* __restrict__ ang2,
    const float4* __restrict__ x4, int64_t x_stride4, int nrhs, const int32_t* __restrict__ done,
    int done_stride, float* __restrict__ t, int64_t t_stride, const WinProb* __restrict__ probs) {
  extern __shared__ float4 win[];   // [kWinEntries], slot k at win_index(k)
  const PGroup G = groups[blockIdx.x];
  if constexpr (MULTI) {
    const WinProb& pp = probs[G.prob];
    block_off = pp.block_off;
    slot = pp.slot;
    slot_pix = pp.slot_pix;
    ang2 = pp.ang2;
    x4 = reinterpret_cast<const float4*>(pp.x);
    t = pp.t;
    done = pp.done;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ChunkWalk cw = chunk_walk(G, lane);
  const bool keep = nrhs > 1;
  for (int r = 0; r < nrhs; r++) {
    if (done != nullptr && done[(int64_t)r * done_stride] != 0) continue;
    const float4* x = x4 + r * x_stride4;
    float* tr = t + r * t_stride;
    __syncthreads();   // the previous column's window is no longer read
    for (int k = threadIdx.x; k < G.n_slots; k += kWinThreads)
      win[win_index(k)] = __ldg(x + __ldg(slot_pix + G.slot_off + k));
    __syncthreads();
    auto value = [&](uint32_t sl, float a) -> float {
      if (sl == kNoSlot) return 0.f;
      float cs, sn;
      weights_of_angle(a, cs, sn);
      const float4 m = win[win_index((int)sl)];
      return m.x + cs * m.y + sn * m.z;
    };
    for (int c0 = warp * cw.cpi; c0 < G.n_blk; c0 += kWarps * cw.cpi) {
      const int c = c0 + cw.sub;
      if (c >= G.n_blk) continue;
      if (c + kWarps * cw.cpi < G.n_blk) {
        int64_t lo;
        int len;
        group_chunk(G, block_off, c + kWarps * cw.cpi, lo, len);
        prefetch_chunk(slot, lo, len, cw);
        prefetch_chunk(ang2, lo, len, cw);
      }
      visit_chunk(
          G, block_off, c, cw,
          [&](int64_t a0, int q) {
            const int64_t i = a0 + 4 * (int64_t)q;
            const uint2 s2 = ld_point(reinterpret_cast<const uint2*>(slot + i), keep);
            const float4 a = ld_point(reinterpret_cast<const float4*>(ang2 + i), keep);
            float4 v;
            v.x = value(s2.x & 0xFFFFu, a.x);
            v.y = value(s2.x >> 16, a.y);
            v.z = value(s2.y & 0xFFFFu, a.z);
            v.w = value(s2.y >> 16, a.w);
            __stcs(reinterpret_cast<float4*>(tr + i), v);
          },
          [&](int64_t i) { __stcs(tr + i, value(ld_point(slot + i, keep), ld_point(ang2 + i, keep))); });
    }
  }
}

cudaError_t launch_unpoint_win32(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                                 const uint16_t* slot, const int32_t* slot_pix, const float* ang2,
                                 const float* x4, int64_t x_stride, int nrhs, const int32_t* done,
                                 int done_stride, float* t, int64_t t_stride, cudaStream_t s) {
  if (n_groups == 0 || nrhs <= 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL || t_stride % 4 != 0) return cudaErrorInvalidValue;
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_unpoint_win32<false>, kUnpointSmem, st, set));
  k_unpoint_win32<false><<<(unsigned)n_groups, kWinThreads, kUnpointSmem, s>>>(
      groups, block_off, slot, slot_pix, ang2, reinterpret_cast<const float4*>(x4), x_stride / 4, nrhs, done,
      done_stride, t, t_stride, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_unpoint_win32_multi(const PGroup* groups, int64_t n_groups, const WinProb* probs,
                                       cudaStream_t s) {
  if (n_groups == 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL || probs == nullptr) return cudaErrorInvalidValue;
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_unpoint_win32<true>, kUnpointSmem, st, set));
  k_unpoint_win32<true><<<(unsigned)n_groups, kWinThreads, kUnpointSmem, s>>>(
      groups, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 1, nullptr, 0, nullptr, 0, probs);
  return cudaGetLastError();
}

// y += P^T u over the windows: one CTA per group and column, samples summed per slot in shared
// memory (three FP32 shared-memory adds per sample), then one float4 global atomic per distinct
// pixel of the group.
constexpr size_t kPointSmem = (size_t)3 * kAccStride * sizeof(float);
template <bool MULTI>
__global__ void __launch_bounds__(kWinThreads, 3) k_point_win32(
    const PGroup* __restrict__ groups, const int64_t* __restrict__ block_off,
    const uint16_t* __restrict__ slot, const int32_t* __restrict__ slot_pix, const float* __restrict__ ang2,
    const float* __restrict__ u, int64_t u_stride, int nrhs, const int32_t* __restrict__ done, int done_stride,
    float4* __restrict__ y4, int64_t y_stride4, const WinProb* __restrict__ probs) {
  extern __shared__ float acc[];   // [3][kAccStride]
  const PGroup G = groups[blockIdx.x];
  if constexpr (MULTI) {
    const WinProb& pp = probs[G.prob];
    block_off = pp.block_off;
    slot = pp.slot;
    slot_pix = pp.slot_pix;
    ang2 = pp.ang2;
    u = pp.u;
    y4 = reinterpret_cast<float4*>(pp.y);
    done = pp.done;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ChunkWalk cw = chunk_walk(G, lane);
  const int n_pad = acc_index(G.n_slots);
  const bool keep = nrhs > 1;
  for (int r = 0; r < nrhs; r++) {
    if (done != nullptr && done[(int64_t)r * done_stride] != 0) continue;
    const float* ur = u + r * u_stride;
    for (int k = threadIdx.x; k < n_pad; k += kWinThreads) {
      acc[k] = 0.f;
      acc[kAccStride + k] = 0.f;
      acc[2 * kAccStride + k] = 0.f;
    }
    __syncthreads();
    auto add = [&](uint32_t sl, float a, float y) {
      if (sl == kNoSlot) return;
      float cs, sn;
      weights_of_angle(a, cs, sn);
      const int k = acc_index((int)sl);
      atomicAdd(acc + k, y);
      atomicAdd(acc + kAccStride + k, cs * y);
      atomicAdd(acc + 2 * kAccStride + k, sn * y);
    };
    // warps take contiguous ranges of the group's chunks (detectors), so warps running at the
    // same time sit far apart on the focal plane and rarely add to the same pixel at once
    const int n_it = (G.n_blk + cw.cpi - 1) / cw.cpi;
    const int per = (n_it + kWarps - 1) / kWarps;
    for (int it = warp * per; it < min(n_it, (warp + 1) * per); it++) {
      const int c = it * cw.cpi + cw.sub;
      if (c >= G.n_blk) continue;
      visit_chunk(
          G, block_off, c, cw,
          [&](int64_t a0, int q) {
            const int64_t i = a0 + 4 * (int64_t)q;
            const uint2 s2 = ld_point(reinterpret_cast<const uint2*>(slot + i), keep);
            const float4 a = ld_point(reinterpret_cast<const float4*>(ang2 + i), keep);
            const float4 y = __ldcs(reinterpret_cast<const float4*>(ur + i));
            add(s2.x & 0xFFFFu, a.x, y.x);
            add(s2.x >> 16, a.y, y.y);
            add(s2.y & 0xFFFFu, a.z, y.z);
            add(s2.y >> 16, a.w, y.w);
          },
          [&](int64_t i) { add(ld_point(slot + i, keep), ld_point(ang2 + i, keep), __ldcs(ur + i)); });
    }
    __syncthreads();
    float4* yr = y4 + r * y_stride4;
    for (int k = threadIdx.x; k < G.n_slots; k += kWinThreads) {
      const int32_t p = __ldg(slot_pix + G.slot_off + k);
      const int j = acc_index(k);
      atomicAdd(yr + p, make_float4(acc[j], acc[kAccStride + j], acc[2 * kAccStride + j], 0.f));
    }
    __syncthreads();   // the next column clears the sums
  }
}

cudaError_t launch_point_win32(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                               const uint16_t* slot, const int32_t* slot_pix, const float* ang2,
                               const float* u, int64_t u_stride, int nrhs, const int32_t* done,
                               int done_stride, float* y4, int64_t y_stride, cudaStream_t s) {
  if (n_groups == 0 || nrhs <= 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL || u_stride % 4 != 0) return cudaErrorInvalidValue;
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_point_win32<false>, kPointSmem, st, set));
  k_point_win32<false><<<(unsigned)n_groups, kWinThreads, kPointSmem, s>>>(
      groups, block_off, slot, slot_pix, ang2, u, u_stride, nrhs, done, done_stride, reinterpret_cast<float4*>(y4),
      y_stride / 4, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_point_win32_multi(const PGroup* groups, int64_t n_groups, const WinProb* probs,
                                     cudaStream_t s) {
  if (n_groups == 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL || probs == nullptr) return cudaErrorInvalidValue;
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_point_win32<true>, kPointSmem, st, set));
  k_point_win32<true><<<(unsigned)n_groups, kWinThreads, kPointSmem, s>>>(
      groups, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 1, nullptr, 0, nullptr, 0, probs);
  return cudaGetLastError();
}

// ---- P^T by segment reduction over pixel-sorted sub-windows ----------------------------------
// Sample l = c 2^log_s + o of sub-window sw: global index, false past its chunk's end.
__device__ __forceinline__ bool sub_sample(const PGroup& G, const int64_t* __restrict__ block_off, int sw,
                                           int log_s, int l, int64_t& i) {
  int64_t lo;
  int len;
  group_chunk(G, block_off, l >> log_s, lo, len);
  const int o = (sw << log_s) + (l & ((1 << log_s) - 1));
  i = lo + o;
  return o < len;
}

// One CTA per group: for each sub-window, the keys (slot << 16 | l) of its samples (masked ones
// with slot kNoSlot) sorted ascending in shared memory (bitonic, padded with 0xFFFFFFFF), so equal
// slots form runs ordered by l, then written out with each kept entry's angle.
__global__ void __launch_bounds__(kWinThreads) k_seg_build(const PGroup* __restrict__ groups,
                                                           const int64_t* __restrict__ block_off,
                                                           const uint16_t* __restrict__ slot,
                                                           const float* __restrict__ ang2, int sub_cap,
                                                           uint32_t* __restrict__ ent,
                                                           float* __restrict__ ent_ang,
                                                           int32_t* __restrict__ kept) {
  extern __shared__ __align__(16) uint32_t keys[];   // [next power of two >= sub_cap]
  __shared__ int s_kept;
  const PGroup G = groups[blockIdx.x];
  const int ls = seg_log_s(G.n_blk, G.log_w, sub_cap);
  const int n_sub = 1 << (G.log_w - ls);
  const int64_t stride = seg_stride(G.n_blk, ls);
  const int n_l = G.n_blk << ls;
  int n2 = 1;
  while (n2 < n_l) n2 <<= 1;
  for (int sw = 0; sw < n_sub; sw++) {
    if (threadIdx.x == 0) s_kept = 0;
    __syncthreads();
    int my_kept = 0;
    for (int l = threadIdx.x; l < n2; l += kWinThreads) {
      uint32_t key = 0xFFFFFFFFu;
      if (l < n_l) {
        int64_t i;
        uint32_t sl = kNoSlot;
        if (sub_sample(G, block_off, sw, ls, l, i)) sl = slot[i];
        key = (sl << 16) | (uint32_t)l;
        my_kept += sl != kNoSlot;
      }
      keys[l] = key;
    }
    atomicAdd(&s_kept, my_kept);
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < n2; i += kWinThreads) {
          const int l = i ^ j;
          if (l > i) {
            const uint32_t a = keys[i], b = keys[l];
            if ((a > b) == ((i & k) == 0)) {
              keys[i] = b;
              keys[l] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    const int nk = s_kept;
    const int64_t base = G.ent_off + (int64_t)sw * stride;
    for (int j = threadIdx.x; j < stride; j += kWinThreads) {
      uint32_t e = (uint32_t)kNoSlot << 16;
      float a = 0.f;
      if (j < nk) {
        e = keys[j];
        int64_t i;
        sub_sample(G, block_off, sw, ls, (int)(e & 0xFFFFu), i);
        a = __ldg(ang2 + i);
      }
      ent[base + j] = e;
      ent_ang[base + j] = a;
    }
    if (threadIdx.x == 0) kept[G.sub0 + sw] = nk;
    __syncthreads();   // the keys are rewritten by the next sub-window
  }
}

constexpr int kSegSubMax = 16384;
constexpr size_t kSegBuildSmemMax = (size_t)kSegSubMax * sizeof(uint32_t);
constexpr size_t kPointSegSmemMax = (size_t)3 * kAccStride * sizeof(float) + (size_t)kSegSubMax * sizeof(float);

static int pow2_at_least(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

cudaError_t launch_seg_build(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                             const uint16_t* slot, const float* ang2, int sub_cap, uint32_t* ent,
                             float* ent_ang, int32_t* kept, cudaStream_t s) {
  if (n_groups == 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL || sub_cap < 32 || sub_cap > kSegSubMax) return cudaErrorInvalidValue;
  const size_t smem = (size_t)pow2_at_least(sub_cap) * sizeof(uint32_t);
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_seg_build, kSegBuildSmemMax, st, set));
  k_seg_build<<<(unsigned)n_groups, kWinThreads, smem, s>>>(groups, block_off, slot, ang2, sub_cap, ent, ent_ang,
                                                           kept);
  return cudaGetLastError();
}

// One CTA per group and column.  Per sub-window: the sub-window's u into shared memory (one
// coalesced pass over its chunks), then each thread reduces kSegRange consecutive sorted entries:
// it sums (u, cos 2psi u, sin 2psi u) in registers along each run of equal slots and adds a run's
// sums to the group's per-slot totals once, with a shared-memory atomic for the first and last run
// of its range (which other threads may share) and a plain update for the runs between them (which
// lie wholly in its range).  Last, one float4 global atomic per distinct pixel of the group.
__global__ void __launch_bounds__(kWinThreads, 2) k_point_seg32(
    const PGroup* __restrict__ groups, const int64_t* __restrict__ block_off, const uint32_t* __restrict__ ent,
    const float* __restrict__ ent_ang, const int32_t* __restrict__ kept, const int32_t* __restrict__ slot_pix,
    int sub_cap, const float* __restrict__ u, int64_t u_stride, int nrhs, const int32_t* __restrict__ done,
    int done_stride, float4* __restrict__ y4, int64_t y_stride4) {
  extern __shared__ __align__(16) float smem_f[];
  float* acc = smem_f;                   // [3][kAccStride]
  float* us = smem_f + 3 * kAccStride;   // [sub_cap] u of the sub-window, sample l at us[l]
  const PGroup G = groups[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ls = seg_log_s(G.n_blk, G.log_w, sub_cap);
  const int n_sub = 1 << (G.log_w - ls);
  const int64_t stride = seg_stride(G.n_blk, ls);
  PGroup S = G;   // the current sub-window as a group of window 2^log_s
  S.log_w = ls;
  const ChunkWalk cw = chunk_walk(S, lane);
  const int n_pad = acc_index(G.n_slots);
  for (int r = 0; r < nrhs; r++) {
    if (done != nullptr && done[(int64_t)r * done_stride] != 0) continue;
    const float* ur = u + r * u_stride;
    for (int k = threadIdx.x; k < n_pad; k += kWinThreads) {
      acc[k] = 0.f;
      acc[kAccStride + k] = 0.f;
      acc[2 * kAccStride + k] = 0.f;
    }
    for (int sw = 0; sw < n_sub; sw++) {
      S.w0 = G.w0 + ((int64_t)sw << ls);
      const int nk = __ldg(kept + G.sub0 + sw);
      const int64_t base = G.ent_off + (int64_t)sw * stride;
      const int n_rng = (nk + kSegRange - 1) / kSegRange;
      // this thread's first range, loaded before the staging pass so both latencies overlap
      uint4 pe[kSegRange / 4];
      float4 pa[kSegRange / 4];
      if ((int)threadIdx.x < n_rng) {
        const uint4* ep = reinterpret_cast<const uint4*>(ent + base + (int64_t)threadIdx.x * kSegRange);
        const float4* ap = reinterpret_cast<const float4*>(ent_ang + base + (int64_t)threadIdx.x * kSegRange);
#pragma unroll
        for (int v = 0; v < kSegRange / 4; v++) {
          pe[v] = __ldcs(ep + v);
          pa[v] = __ldcs(ap + v);
        }
      }
      __syncthreads();   // the previous sub-window's u is no longer read (and the sums are cleared)
      for (int c0 = warp * cw.cpi; c0 < S.n_blk; c0 += kWarps * cw.cpi) {
        const int c = c0 + cw.sub;
        if (c >= S.n_blk) continue;
        int64_t lo;
        int len;
        group_chunk(S, block_off, c, lo, len);
        const int l0 = c << ls;
        visit_chunk(
            S, block_off, c, cw,
            [&](int64_t a0, int q) {
              const int64_t i = a0 + 4 * (int64_t)q;
              const float4 v = __ldcs(reinterpret_cast<const float4*>(ur + i));
              const int l = l0 + (int)(i - lo);
              us[l] = v.x;
              us[l + 1] = v.y;
              us[l + 2] = v.z;
              us[l + 3] = v.w;
            },
            [&](int64_t i) { us[l0 + (int)(i - lo)] = __ldcs(ur + i); });
      }
      __syncthreads();
      for (int g = threadIdx.x; g < n_rng; g += kWinThreads) {
        if (g != (int)threadIdx.x) {
          const uint4* ep = reinterpret_cast<const uint4*>(ent + base + (int64_t)g * kSegRange);
          const float4* ap = reinterpret_cast<const float4*>(ent_ang + base + (int64_t)g * kSegRange);
#pragma unroll
          for (int v = 0; v < kSegRange / 4; v++) {
            pe[v] = __ldcs(ep + v);
            pa[v] = __ldcs(ap + v);
          }
        }
        uint32_t cur = pe[0].x >> 16;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        bool first = true;
        auto flush = [&](bool shared_run) {
          if (cur == kNoSlot) return;
          const int k = acc_index((int)cur);
          if (shared_run) {
            atomicAdd(acc + k, s0);
            atomicAdd(acc + kAccStride + k, s1);
            atomicAdd(acc + 2 * kAccStride + k, s2);
          } else {
            acc[k] += s0;
            acc[kAccStride + k] += s1;
            acc[2 * kAccStride + k] += s2;
          }
        };
#pragma unroll
        for (int i = 0; i < kSegRange; i++) {
          const uint4& e4 = pe[i / 4];
          const float4& a4 = pa[i / 4];
          const uint32_t e = (i % 4 == 0) ? e4.x : (i % 4 == 1) ? e4.y : (i % 4 == 2) ? e4.z : e4.w;
          const float ang = (i % 4 == 0) ? a4.x : (i % 4 == 1) ? a4.y : (i % 4 == 2) ? a4.z : a4.w;
          const uint32_t sl = e >> 16;
          if (sl != cur) {
            flush(first);
            first = false;
            cur = sl;
            s0 = s1 = s2 = 0.f;
          }
          if (sl != kNoSlot) {
            float cs, sn;
            weights_of_angle(ang, cs, sn);
            const float y = us[e & 0xFFFFu];
            s0 += y;
            s1 = fmaf(cs, y, s1);
            s2 = fmaf(sn, y, s2);
          }
        }
        flush(true);
      }
    }
    __syncthreads();
    float4* yr = y4 + r * y_stride4;
    for (int k = threadIdx.x; k < G.n_slots; k += kWinThreads) {
      const int32_t p = __ldg(slot_pix + G.slot_off + k);
      const int j = acc_index(k);
      atomicAdd(yr + p, make_float4(acc[j], acc[kAccStride + j], acc[2 * kAccStride + j], 0.f));
    }
    __syncthreads();   // the next column clears the sums
  }
}

cudaError_t launch_point_seg32(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                               const uint32_t* ent, const float* ent_ang, const int32_t* kept,
                               const int32_t* slot_pix, int sub_cap, const float* u, int64_t u_stride,
                               int nrhs, const int32_t* done, int done_stride, float* y4, int64_t y_stride,
                               cudaStream_t s) {
  if (n_groups == 0 || nrhs <= 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL || u_stride % 4 != 0 || sub_cap < 32 || sub_cap > kSegSubMax)
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)3 * kAccStride * sizeof(float) + (size_t)sub_cap * sizeof(float);
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_point_seg32, kPointSegSmemMax, st, set));
  k_point_seg32<<<(unsigned)n_groups, kWinThreads, smem, s>>>(groups, block_off, ent, ent_ang, kept, slot_pix,
                                                               sub_cap, u, u_stride, nrhs, done, done_stride,
                                                               reinterpret_cast<float4*>(y4), y_stride / 4);
  return cudaGetLastError();
}

// ---- FP32 right-hand side input: t = G d rounded to FP32 (0 at flagged and excised samples) ----
template <typename D>
__global__ void k_d_to_t32(const int32_t* __restrict__ lpix, const D* __restrict__ d, int64_t N, int64_t d_stride,
                           float* __restrict__ t, int64_t t_stride) {
  const D* dr = d + blockIdx.y * d_stride;
  float* tr = t + blockIdx.y * t_stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    __stcs(tr + i, (__ldg(lpix + i) >= 0) ? (float)__ldcs(dr + i) : 0.f);
}

cudaError_t launch_d_to_t32(const int32_t* lpix, const void* d, int d_is_fp32, int64_t N, int nrhs, float* t,
                            int64_t t_stride, cudaStream_t s) {
  if (N == 0 || nrhs <= 0) return cudaSuccess;
  const int64_t g = std::min<int64_t>((N + 255) / 256, 16 * (int64_t)sm_count());
  const dim3 grid((unsigned)g, nrhs);
  if (d_is_fp32)
    k_d_to_t32<float><<<grid, 256, 0, s>>>(lpix, reinterpret_cast<const float*>(d), N, N, t, t_stride);
  else
    k_d_to_t32<double><<<grid, 256, 0, s>>>(lpix, reinterpret_cast<const double*>(d), N, N, t, t_stride);
  return cudaGetLastError();
}

// ---- the FP64-class (double-float) P^T over the windows ------------------------------------------
// Each group's sums are 64-bit fixed-point integers in shared memory: integer shared-memory
// atomics are native, and integer sums do not depend on the order of the additions.  The column's
// u values are bounded by umax (the df64 N^-1 tiles record max |u|), the weights by 1 and a slot
// receives at most 2^15 samples, so with 2^k, k = 45 - floor(log2 umax), a slot's sum stays below
// 2^61 while one unit is about 2^-46 umax, under the double-float operator's own relative error.

// round(f 2^k) as a 64-bit integer with integer instructions only (the FP32 -> 64-bit conversion
// instruction runs on the FP64 pipe); zero and subnormal f give 0
__device__ __forceinline__ long long fixed_of(float f, int k) {
  const uint32_t b = __float_as_uint(f);
  const int e = (int)((b >> 23) & 0xffu);
  if (e == 0) return 0;
  const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 150 + k;
  long long v;
  if (sh >= 0) v = m << min(sh, 39);
  else if (sh > -40) v = (m + (1ll << (-sh - 1))) >> (-sh);
  else v = 0;
  return (b >> 31) ? -v : v;
}
__device__ __forceinline__ long long fixed_of(df v, int k) { return fixed_of(v.hi, k) + fixed_of(v.lo, k); }

// round(f 2^(32 + e)) with sc = 2^e (a normal float) and |f sc| < 2^30, rounding the magnitude:
// x = |f| sc (exact), its integer part and its fraction (x - floor(x), exact for x >= 0) times 2^32
// as two 32-bit conversions, then the sign.
__device__ __forceinline__ long long fixed_fast(float f, float sc) {
  const float x = fabsf(f) * sc;
  const float h = floorf(x);
  const unsigned long long m =
      ((unsigned long long)__float2uint_rn(h) << 32) + __float2uint_rn((x - h) * 4294967296.f);
  return f < 0.f ? -(long long)m : (long long)m;
}
__device__ __forceinline__ long long fixed_fast(df v, float sc) { return fixed_fast(v.hi, sc) + fixed_fast(v.lo, sc); }

constexpr size_t kPointDfSmem = (size_t)3 * kAccStride * sizeof(unsigned long long);

__global__ void __launch_bounds__(kWinThreads, 2) k_point_win_df(
    const PGroup* __restrict__ groups, const int64_t* __restrict__ block_off,
    const uint16_t* __restrict__ slot, const int32_t* __restrict__ slot_pix, const float4* __restrict__ wdf,
    const float2* __restrict__ u, int64_t u_stride, const uint32_t* __restrict__ amax, int nrhs,
    const int32_t* __restrict__ done, int done_stride, double* __restrict__ y4, int64_t y_stride) {
  extern __shared__ unsigned long long acc64[];   // [3][kAccStride]
  const PGroup G = groups[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ChunkWalk cw = chunk_walk(G, lane);
  const int n_pad = acc_index(G.n_slots);
  for (int r = 0; r < nrhs; r++) {
    if (done != nullptr && done[(int64_t)r * done_stride] != 0) continue;
    const uint32_t ub = __ldg(amax + r);
    if (ub == 0u) continue;   // u = 0: nothing to add
    double* yr = y4 + r * y_stride;
    if (ub >= 0x7f800000u) {   // a non-finite u: poison the outputs so the solver sees it
      for (int k = threadIdx.x; k < G.n_slots; k += kWinThreads)
        atomicAdd(yr + 4 * (int64_t)__ldg(slot_pix + G.slot_off + k), __longlong_as_double(0x7ff8000000000000ll));
      continue;
    }
    const int e_u = (int)((ub >> 23) & 0xffu) - 127;   // umax in [2^e_u, 2^(e_u + 1)) (subnormal: e_u = -127)
    const int ks = 45 - e_u;
    // sums in units of 2^-ks: |y| < 2^(e_u + 1) gives |y 2^(ks - 32)| < 2^14; the fast conversion
    // takes the scale 2^(ks - 32) as a normal float (all but umax below 2^-114)
    const bool fast = ks - 32 <= 126;
    const float sc = fast ? __int_as_float((ks - 32 + 127) << 23) : 0.f;
    const double unit = __longlong_as_double((long long)(1023 - ks) << 52);   // 2^-ks
    const float2* ur = u + r * u_stride;
    for (int k = threadIdx.x; k < n_pad; k += kWinThreads) {
      acc64[k] = 0ull;
      acc64[kAccStride + k] = 0ull;
      acc64[2 * kAccStride + k] = 0ull;
    }
    __syncthreads();
    auto add = [&](uint32_t sl, float4 w, float2 y2) {
      if (sl == kNoSlot) return;
      const df y = df_make(y2.x, y2.y);
      const df cy = df_make(w.x, w.y) * y, sy = df_make(w.z, w.w) * y;
      const int k = acc_index((int)sl);
      if (fast) {
        atomicAdd(acc64 + k, (unsigned long long)fixed_fast(y, sc));
        atomicAdd(acc64 + kAccStride + k, (unsigned long long)fixed_fast(cy, sc));
        atomicAdd(acc64 + 2 * kAccStride + k, (unsigned long long)fixed_fast(sy, sc));
      } else {
        atomicAdd(acc64 + k, (unsigned long long)fixed_of(y, ks));
        atomicAdd(acc64 + kAccStride + k, (unsigned long long)fixed_of(cy, ks));
        atomicAdd(acc64 + 2 * kAccStride + k, (unsigned long long)fixed_of(sy, ks));
      }
    };
    const int n_it = (G.n_blk + cw.cpi - 1) / cw.cpi;
    const int per = (n_it + kWarps - 1) / kWarps;
    const int it_end = min(n_it, (warp + 1) * per);
    for (int it = warp * per; it < it_end; it++) {
      const int c = it * cw.cpi + cw.sub;
      if (c >= G.n_blk) continue;
      if (it + 1 < it_end && c + cw.cpi < G.n_blk) {
        int64_t lo;
        int len;
        group_chunk(G, block_off, c + cw.cpi, lo, len);
        prefetch_chunk(slot, lo, len, cw);
        prefetch_chunk(wdf, lo, len, cw);
        prefetch_chunk(ur, lo, len, cw);
      }
      visit_chunk(
          G, block_off, c, cw,
          [&](int64_t a0, int q) {
            const int64_t i = a0 + 4 * (int64_t)q;
            const uint2 s2 = __ldcs(reinterpret_cast<const uint2*>(slot + i));
            add(s2.x & 0xFFFFu, __ldcs(wdf + i), __ldcs(ur + i));
            add(s2.x >> 16, __ldcs(wdf + i + 1), __ldcs(ur + i + 1));
            add(s2.y & 0xFFFFu, __ldcs(wdf + i + 2), __ldcs(ur + i + 2));
            add(s2.y >> 16, __ldcs(wdf + i + 3), __ldcs(ur + i + 3));
          },
          [&](int64_t i) { add(__ldcs(slot + i), __ldcs(wdf + i), __ldcs(ur + i)); });
    }
    __syncthreads();
    for (int k = threadIdx.x; k < G.n_slots; k += kWinThreads) {
      const int64_t p = __ldg(slot_pix + G.slot_off + k);
      const int j = acc_index(k);
      atomicAdd(yr + 4 * p, (double)(long long)acc64[j] * unit);
      atomicAdd(yr + 4 * p + 1, (double)(long long)acc64[kAccStride + j] * unit);
      atomicAdd(yr + 4 * p + 2, (double)(long long)acc64[2 * kAccStride + j] * unit);
    }
    __syncthreads();   // the next column clears the sums
  }
}

cudaError_t launch_point_win_df(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                                const uint16_t* slot, const int32_t* slot_pix, const float4* wdf,
                                const float2* u, int64_t u_stride, const uint32_t* amax, int nrhs,
                                const int32_t* done, int done_stride, double* y4, int64_t y_stride,
                                cudaStream_t s) {
  if (n_groups == 0 || nrhs <= 0) return cudaSuccess;
  if (n_groups > 0x7fffffffLL || u_stride % 4 != 0 || y_stride % 4 != 0) return cudaErrorInvalidValue;
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  MM_TRY_CUDA(smem_limit_once(k_point_win_df, kPointDfSmem, st, set));
  k_point_win_df<<<(unsigned)n_groups, kWinThreads, kPointDfSmem, s>>>(groups, block_off, slot, slot_pix, wdf, u,
                                                                         u_stride, amax, nrhs, done, done_stride, y4,
                                                                         y_stride);
  return cudaGetLastError();
}

}  // namespace mm
