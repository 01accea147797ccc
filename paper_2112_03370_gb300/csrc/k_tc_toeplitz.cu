// Banded block-Toeplitz product u = T(c_b) t (Eq. MADCAP; stbmm of Sect. 3.1) as a GEMM on the
// fifth-generation tensor cores (tcgen05), in 3xTF32: the alternative to the overlap-save FFT for
// small half-bandwidths, chosen by measurement (MM_TPLZ_GEMM, and MM_TPLZ_AUTO below the measured
// crossover).
//
// A block's samples are cut into rows of B = 32 (row k holds samples 32k .. 32k + 31 of the block).
// With T_J[i][r] = c_{|32 J + r - i|} (0 beyond lambda), output row k is
//     u[32 k + i] = sum_{J = -J0..J0} sum_{r < 32} T_J[i][r] t[32 (k + J) + r],   J0 = ceil(lambda / 32),
// i.e. one GEMM per shift J of the row block X_J (rows k + J, M x 32) with T_J (32 x 32), all
// accumulated into one 128 x 32 FP32 tile in tensor memory.  3xTF32: every FP32 operand is split
// into hi = tf32(x) and lo = tf32(x - hi), and the products hi.hi + hi.lo + lo.hi restore FP32
// accuracy.  Rows outside the block read as zero, so there is no wrap and no coupling across blocks.
//
// Shared-memory operands use the no-swizzle K-major layout: a 16-byte core-matrix row holds 4 TF32
// values of one row; for each group of 4 columns (k-group) all rows are stored contiguously
// (stride-dimension offset 128 bytes between groups of 8 rows), and k-groups lie `lbo` bytes apart.
// Because rows are contiguous, the shifted operand X_J of the tile is the same smem tile read from a
// start address 16 (J0 + J) bytes further on.  T_J (hi and lo) of each band table is precomputed at
// plan time in exactly this layout and copied in once per table.
//
// One elected thread issues the MMAs and commits them to an mbarrier; every wait on it is bounded:
// after the bound the kernel records an error, waits once more (bounded) for its own MMAs, frees its
// tensor memory and leaves.
#include <algorithm>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kTcB = 32;                          // samples per row = GEMM N = K per shift
constexpr int kTcM = 128;                         // rows per tile = GEMM M (TMEM lanes)
constexpr int kTcKg = kTcB / 4;                   // k-groups of 4 TF32 values (16 bytes)
constexpr int kTcRowStride = kTcM + 2 * kTcMaxJ0 + 1;   // 137: A rows per k-group (odd: bank spread)
constexpr int kTcLboA = kTcRowStride * 16;        // bytes between k-groups of A
constexpr int kTcLboB = kTcB * 16;                // bytes between k-groups of T_J
constexpr int kTcASize = kTcKg * kTcLboA;         // one A operand (hi or lo)
constexpr int kTcBShift = kTcKg * kTcLboB;        // one T_J (hi or lo)
constexpr int kTcMaxShifts = 2 * kTcMaxJ0 + 1;
constexpr int kTcBSize = kTcMaxShifts * kTcBShift;
constexpr int kTcGuard = 4096;                    // keeps every descriptor-reachable byte inside
// dynamic shared memory for 2 j0 + 1 shifts: A hi/lo, T_J hi/lo, guard
__host__ __device__ constexpr size_t tc_smem_bytes(int j0) {
  return 2 * (size_t)kTcASize + 2 * (size_t)(2 * j0 + 1) * kTcBShift + kTcGuard;
}
constexpr size_t kTcSmem = tc_smem_bytes(kTcMaxJ0);
constexpr int kTcThreads = 128;
constexpr uint32_t kTcSpin = 1u << 22;            // bound of an mbarrier wait (iterations)

static_assert(kTcASize % 16 == 0 && kTcBSize % 16 == 0, "16-byte aligned operands");

// tcgen05 instruction descriptor: dense, D FP32, A and B TF32, both K-major, N = 32, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcB >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

// shared-memory matrix descriptor, no swizzle (start, leading and stride byte offsets in 16-byte
// units; descriptor version 1)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (uint32_t i = 0; i < kTcSpin; i++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(mbar), "r"(phase));
    if (ok) return true;
  }
  return false;
}

// 32 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// One persistent CTA per SM slot; each walks (tile, column) items.  Tile = 128 rows of one block.
__global__ void __launch_bounds__(kTcThreads) k_tplz_tc(const TcTile* __restrict__ tiles, int64_t n_tiles,
                                                        const int64_t* __restrict__ block_off,
                                                        const int32_t* __restrict__ blk_tab,
                                                        const float* __restrict__ blk_scale,
                                                        const uint4* __restrict__ bmat, int j0,
                                                        const float* __restrict__ t, int64_t t_stride,
                                                        float* __restrict__ u, int64_t u_stride, int nrhs,
                                                        const int32_t* __restrict__ done, int done_stride,
                                                        int32_t* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ uint32_t taddr_s;
  __shared__ __align__(8) uint64_t mbar;
  const int n_shift = 2 * j0 + 1;
  unsigned char* a_hi = tc_smem;
  unsigned char* a_lo = a_hi + kTcASize;
  unsigned char* b_hi = a_lo + kTcASize;
  unsigned char* b_lo = b_hi + n_shift * kTcBShift;
  const uint32_t s_ahi = (uint32_t)__cvta_generic_to_shared(a_hi);
  const uint32_t s_alo = (uint32_t)__cvta_generic_to_shared(a_lo);
  const uint32_t s_bhi = (uint32_t)__cvta_generic_to_shared(b_hi);
  const uint32_t s_blo = (uint32_t)__cvta_generic_to_shared(b_lo);
  const uint32_t s_mbar = (uint32_t)__cvta_generic_to_shared(&mbar);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = kTcM + 2 * j0;

  // guard bytes are zero: a mis-read can never see stale values
  for (int i = threadIdx.x; i < (int)(tc_smem_bytes(j0) / 16); i += kTcThreads)
    reinterpret_cast<uint4*>(tc_smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&taddr_s);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(dst));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_mbar));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = taddr_s;

  int loaded_tab = -1;
  uint32_t phase = 0;
  bool ok = true;
  // Operand prefetch: item e = threadIdx.x + 128 p (p < kPf) is k-group e % 8 of stored row e / 8;
  // the next tile's items are loaded into registers while the current tile's MMAs and epilogue run.
  constexpr int kPf = (kTcM + 2 * kTcMaxJ0) * kTcKg / kTcThreads + 1;   // 9 items per thread
  float4 pf[kPf];
  auto fetch = [&](int64_t item) {
    if (item >= n_tiles * nrhs) return;
    const int rhs = (int)(item % nrhs);
    const TcTile tl = tiles[item / nrhs];
    const int64_t lo = __ldg(block_off + tl.blk), hi = __ldg(block_off + tl.blk + 1);
    const float* tr = t + rhs * t_stride;
    const bool al4 = ((lo | t_stride) & 3) == 0 && (((uintptr_t)tr) & 15) == 0;
#pragma unroll
    for (int p = 0; p < kPf; p++) {
      const int e = threadIdx.x + kTcThreads * p;
      const int r = e >> 3, kg = e & 7;
      const int64_t g = lo + (int64_t)kTcB * (tl.k0 - j0 + r) + 4 * kg;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) {
        if (al4 && g >= lo && g + 4 <= hi) {
          x = __ldg(reinterpret_cast<const float4*>(tr + g));
        } else {
          x.x = (g >= lo && g < hi) ? __ldg(tr + g) : 0.f;
          x.y = (g + 1 >= lo && g + 1 < hi) ? __ldg(tr + g + 1) : 0.f;
          x.z = (g + 2 >= lo && g + 2 < hi) ? __ldg(tr + g + 2) : 0.f;
          x.w = (g + 3 >= lo && g + 3 < hi) ? __ldg(tr + g + 3) : 0.f;
        }
      }
      pf[p] = x;
    }
  };
  fetch(blockIdx.x);
  for (int64_t it = blockIdx.x; it < n_tiles * nrhs && ok; it += gridDim.x) {
    const int rhs = (int)(it % nrhs);
    const int64_t ti = it / nrhs;
    if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) {
      fetch(it + gridDim.x);
      continue;
    }
    const TcTile tl = tiles[ti];
    const int64_t lo = __ldg(block_off + tl.blk), hi = __ldg(block_off + tl.blk + 1);
    const int tab = __ldg(blk_tab + tl.blk);
    const float sc = __ldg(blk_scale + tl.blk);
    if (tab != loaded_tab) {   // T_J hi and lo of this band table (n_shift shifts)
      const uint4* src = bmat + (int64_t)tab * (2 * kTcBSize / 16);
      for (int i = threadIdx.x; i < n_shift * kTcBShift / 16; i += kTcThreads) {
        reinterpret_cast<uint4*>(b_hi)[i] = __ldg(src + i);
        reinterpret_cast<uint4*>(b_lo)[i] = __ldg(src + kTcBSize / 16 + i);
      }
      loaded_tab = tab;
    }
    // A (hi and lo TF32 split) from the prefetched registers: one 16-byte store per operand and
    // item (k-groups lie 2192 bytes apart, so 8 consecutive items hit 8 distinct bank groups)
#pragma unroll
    for (int p = 0; p < kPf; p++) {
      const int e = threadIdx.x + kTcThreads * p;
      const int r = e >> 3, kg = e & 7;
      if (r < rows) {
        const float4 x = pf[p];
        uint4 h, l;
        h.x = tf32_rna(x.x); l.x = tf32_rna(x.x - __uint_as_float(h.x));
        h.y = tf32_rna(x.y); l.y = tf32_rna(x.y - __uint_as_float(h.y));
        h.z = tf32_rna(x.z); l.z = tf32_rna(x.z - __uint_as_float(h.z));
        h.w = tf32_rna(x.w); l.w = tf32_rna(x.w - __uint_as_float(h.w));
        const int off = kg * kTcLboA + r * 16;
        *reinterpret_cast<uint4*>(a_hi + off) = h;
        *reinterpret_cast<uint4*>(a_lo + off) = l;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");   // generic-proxy writes -> tensor-core reads
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t acc = 0;
      for (int js = 0; js < n_shift; js++) {        // shift J = js - j0
        for (int ks = 0; ks < kTcKg / 2; ks++) {    // K = 8 per instruction: two k-groups
          const uint32_t ao = (uint32_t)(ks * 2 * kTcLboA + js * 16);
          const uint32_t bo = (uint32_t)(js * kTcBShift + ks * 2 * kTcLboB);
          const uint64_t dah = smem_desc(s_ahi + ao, kTcLboA, 128), dal = smem_desc(s_alo + ao, kTcLboA, 128);
          const uint64_t dbh = smem_desc(s_bhi + bo, kTcLboB, 128), dbl = smem_desc(s_blo + bo, kTcLboB, 128);
          mma_tf32(tmem, dah, dbh, acc);
          acc = 1;
          mma_tf32(tmem, dah, dbl, 1);
          mma_tf32(tmem, dal, dbh, 1);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_mbar));
    }
    fetch(it + gridDim.x);   // the next tile's operand loads overlap the MMAs and the epilogue
    // every thread must take the same branch (the TMEM load below is warp-collective)
    if (!__syncthreads_and(mbar_wait(s_mbar, phase) ? 1 : 0)) {
      ok = false;
      if (threadIdx.x == 0) atomicExch(err, 1);
      mbar_wait(s_mbar, phase);   // give the MMAs one more bounded wait before the memory is freed
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w holds rows 32 w .. 32 w + 31 (TMEM lanes), this thread one row of 32 outputs;
    // the rows go through shared memory (the A operand is free once the MMAs completed) so that the
    // tile's output, one contiguous range of 4096 samples, is stored with coalesced vector stores
    {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
      float* stage = reinterpret_cast<float*>(a_hi);   // [128][33]: padded rows, no bank conflicts
      const int row = 32 * warp + lane;
#pragma unroll
      for (int i = 0; i < kTcB; i++) stage[row * (kTcB + 1) + i] = sc * v[i];
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    {
      float* ur = u + rhs * u_stride;
      const float* stage = reinterpret_cast<const float*>(a_hi);
      const int64_t base = lo + (int64_t)kTcB * tl.k0;
      const bool v4 = ((base | u_stride) & 3) == 0 && (((uintptr_t)ur) & 15) == 0;
      for (int q = threadIdx.x; q < kTcM * kTcB / 4; q += kTcThreads) {
        const int row = q >> 3, c = 4 * (q & 7);
        const int64_t g = base + 4 * (int64_t)q;
        const float* sv = stage + row * (kTcB + 1) + c;
        if (v4 && g + 4 <= hi) {
          *reinterpret_cast<float4*>(ur + g) = make_float4(sv[0], sv[1], sv[2], sv[3]);
        } else {
#pragma unroll
          for (int e = 0; e < 4; e++)
            if (g + e < hi) ur[g + e] = sv[e];
        }
      }
    }
    __syncthreads();   // the staging rows and A consumed before the next tile overwrites them
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// T_J hi / lo of each table in the shared-memory image layout: bmat [n_tab][2][kTcBSize bytes]
__global__ void k_tc_bmat(const double* __restrict__ rows, int32_t lambda, int j0, int32_t n_tab,
                          uint32_t* __restrict__ bmat) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int per = kTcMaxShifts * kTcB * kTcB;
  if (idx >= (int64_t)n_tab * per) return;
  const int tab = (int)(idx / per);
  const int rem = (int)(idx % per);
  const int js = rem / (kTcB * kTcB), i = (rem / kTcB) % kTcB, r = rem % kTcB;
  const int lag = abs(kTcB * (js - j0) + r - i);
  const double c = (js <= 2 * j0 && lag <= lambda) ? rows[(int64_t)tab * (lambda + 1) + lag] : 0.0;
  const float h = __uint_as_float(tf32_rna((float)c));
  const float l = __uint_as_float(tf32_rna((float)(c - (double)h)));
  const int off = js * kTcBShift + (r >> 2) * kTcLboB + i * 16 + (r & 3) * 4;   // bytes
  uint32_t* base = bmat + (int64_t)tab * (2 * kTcBSize / 4);
  base[off / 4] = __float_as_uint(h);
  base[kTcBSize / 4 + off / 4] = __float_as_uint(l);
}

size_t tc_bmat_bytes(int32_t n_tab) { return (size_t)n_tab * 2 * kTcBSize; }

cudaError_t launch_tc_bmat(const double* rows, int32_t lambda, int32_t n_tab, void* bmat, cudaStream_t s) {
  if (lambda > kTcMaxJ0 * kTcB) return cudaErrorInvalidValue;
  const int j0 = (lambda + kTcB - 1) / kTcB;
  const int64_t n = (int64_t)n_tab * kTcMaxShifts * kTcB * kTcB;
  cudaError_t e = cudaMemsetAsync(bmat, 0, tc_bmat_bytes(n_tab), s);
  if (e != cudaSuccess) return e;
  k_tc_bmat<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rows, lambda, j0, n_tab, reinterpret_cast<uint32_t*>(bmat));
  return cudaGetLastError();
}

std::vector<TcTile> tc_tiles(const std::vector<int64_t>& block_off) {
  std::vector<TcTile> out;
  for (size_t b = 0; b + 1 < block_off.size(); b++) {
    const int64_t n = block_off[b + 1] - block_off[b];
    const int64_t rows = (n + kTcB - 1) / kTcB;
    for (int64_t k0 = 0; k0 < rows; k0 += kTcM) out.push_back(TcTile{(int32_t)b, (int32_t)k0});
  }
  return out;
}

cudaError_t launch_tplz_tc(const TcTile* tiles, int64_t n_tiles, const int64_t* block_off, const int32_t* blk_tab,
                           const float* blk_scale, const void* bmat, int32_t lambda, const float* t,
                           int64_t t_stride, float* u, int64_t u_stride, int nrhs, const int32_t* done,
                           int done_stride, int32_t* err, cudaStream_t s) {
  if (n_tiles == 0 || nrhs <= 0) return cudaSuccess;
  if (lambda > kTcMaxJ0 * kTcB) return cudaErrorInvalidValue;
  static cudaError_t st = cudaSuccess;
  static bool set = false;
  if (!set) {
    st = cudaFuncSetAttribute(k_tplz_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    set = true;
  }
  if (st != cudaSuccess) return st;
  const int j0 = (lambda + kTcB - 1) / kTcB;
  const size_t smem = tc_smem_bytes(j0);
  const int per_sm = std::max(1, std::min(4, (int)((227u * 1024u) / (smem + 1024))));
  const int64_t items = n_tiles * nrhs;
  const int64_t grid = std::min<int64_t>(items, (int64_t)per_sm * sm_count());
  k_tplz_tc<<<(unsigned)grid, kTcThreads, smem, s>>>(tiles, n_tiles, block_off, blk_tab, blk_scale,
                                                         reinterpret_cast<const uint4*>(bmat), j0, t, t_stride, u,
                                                         u_stride, nrhs, done, done_stride, err);
  return cudaGetLastError();
}

}  // namespace mm
