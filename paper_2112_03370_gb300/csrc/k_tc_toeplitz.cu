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
// The input rows of a tile are one contiguous range of the block's samples: one elected thread
// brings the next two tiles' ranges into a two-stage shared-memory ring with 1D bulk copies
// (cp.async.bulk, completion counted on an mbarrier per stage), so the loads of later tiles run
// under the current tile's split, MMAs and epilogue.  The same thread issues the MMAs and commits
// them to an mbarrier.  Every wait is bounded: after the bound the kernel records an error, waits
// once more (bounded) for its own copies and MMAs in flight, frees its tensor memory and leaves.
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
// one ring stage: the tile's 128 + 2 j0 rows of input plus up to 8 samples of 16-byte alignment
__host__ __device__ constexpr size_t tc_stage_bytes(int j0) {
  return (((size_t)(kTcM + 2 * j0) * kTcB + 8) * 4 + 15) / 16 * 16;
}
// dynamic shared memory for 2 j0 + 1 shifts: A hi/lo, T_J hi/lo, two input stages, guard
__host__ __device__ constexpr size_t tc_smem_bytes(int j0) {
  return 2 * (size_t)kTcASize + 2 * (size_t)(2 * j0 + 1) * kTcBShift + 2 * tc_stage_bytes(j0) + kTcGuard;
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

// Expect `bytes` on the mbarrier and start the 1D bulk copy of [src, src + bytes) into shared
// memory at dst (both 16-byte aligned, bytes a multiple of 16; none when bytes is 0).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  if (bytes > 0)
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(mbar)
                 : "memory");
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
  __shared__ __align__(8) uint64_t mbar_ld[2];
  __shared__ int64_t stage_c0[2];   // first staged sample (in-column index) of each stage
  __shared__ int stage_busy[2];     // a copy was issued into the stage and not yet waited for
  const int n_shift = 2 * j0 + 1;
  unsigned char* a_hi = tc_smem;
  unsigned char* a_lo = a_hi + kTcASize;
  unsigned char* b_hi = a_lo + kTcASize;
  unsigned char* b_lo = b_hi + n_shift * kTcBShift;
  unsigned char* stg0 = b_lo + n_shift * kTcBShift;
  const size_t stage_bytes = tc_stage_bytes(j0);
  const uint32_t s_ahi = (uint32_t)__cvta_generic_to_shared(a_hi);
  const uint32_t s_alo = (uint32_t)__cvta_generic_to_shared(a_lo);
  const uint32_t s_bhi = (uint32_t)__cvta_generic_to_shared(b_hi);
  const uint32_t s_blo = (uint32_t)__cvta_generic_to_shared(b_lo);
  const uint32_t s_stg0 = (uint32_t)__cvta_generic_to_shared(stg0);
  const uint32_t s_mbar = (uint32_t)__cvta_generic_to_shared(&mbar);
  const uint32_t s_mld0 = (uint32_t)__cvta_generic_to_shared(&mbar_ld[0]);   // stage st: + 8 st
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = kTcM + 2 * j0;
  const int64_t total = n_tiles * nrhs;

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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_mld0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_mld0 + 8));
    asm volatile("fence.mbarrier_init.release.cluster;");
    stage_busy[0] = stage_busy[1] = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = taddr_s;

  // thread 0: start the copy of item `item`'s input range into stage st.  The range is the tile's
  // rows k0 - j0 .. k0 + 127 + j0 of its block, clipped to the column [0, t_stride) and widened to
  // 16-byte boundaries; samples outside the block are masked when the stage is read.
  auto issue = [&](int64_t item, int st) {
    if (item >= total) return;
    const int rhs = (int)(item % nrhs);
    const TcTile tl = tiles[item / nrhs];
    const int64_t lo = __ldg(block_off + tl.blk);
    const int64_t start = lo + (int64_t)kTcB * (tl.k0 - j0), end = start + (int64_t)kTcB * rows;
    const int64_t c0 = max(start, (int64_t)0) & ~(int64_t)3;
    const int64_t c1 = min((end + 3) & ~(int64_t)3, t_stride);
    const uint32_t bytes = c1 > c0 ? (uint32_t)((c1 - c0) * 4) : 0u;
    stage_c0[st] = c0;
    stage_busy[st] = 1;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the stage first
    bulk_load(s_stg0 + (uint32_t)(st * stage_bytes), t + rhs * t_stride + c0, bytes, s_mld0 + 8 * st);
  };
  if (threadIdx.x == 0) {
    issue(blockIdx.x, 0);
    issue((int64_t)blockIdx.x + gridDim.x, 1);
  }
  __syncthreads();

  int loaded_tab = -1;
  uint32_t phase = 0, ld_phase = 0;   // ld_phase bit st: the parity stage st waits for next
  bool ok = true;
  int k = 0;
  for (int64_t it = blockIdx.x; it < total && ok; it += gridDim.x, k++) {
    const int st = k & 1;
    // this tile's input has arrived (every thread takes the same branch)
    if (!__syncthreads_and(mbar_wait(s_mld0 + 8 * st, (ld_phase >> st) & 1u) ? 1 : 0)) {
      ok = false;
      if (threadIdx.x == 0) atomicExch(err, 1);
      break;
    }
    ld_phase ^= 1u << st;
    if (threadIdx.x == 0) stage_busy[st] = 0;
    const int rhs = (int)(it % nrhs);
    const TcTile tl = tiles[it / nrhs];
    const int64_t lo = __ldg(block_off + tl.blk), hi = __ldg(block_off + tl.blk + 1);
    const float* stage = reinterpret_cast<const float*>(stg0 + st * stage_bytes);
    const int64_t c0 = stage_c0[st];
    if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) {
      __syncthreads();
      if (threadIdx.x == 0) issue(it + 2 * (int64_t)gridDim.x, st);
      continue;
    }
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
    // A (hi and lo TF32 split) from the stage: item e is k-group e % 8 of stored row e / 8, one
    // 16-byte store per operand (k-groups lie 2192 bytes apart: 8 consecutive items, 8 bank groups)
    for (int e = threadIdx.x; e < rows * kTcKg; e += kTcThreads) {
      const int r = e >> 3, kg = e & 7;
      const int64_t g = lo + (int64_t)kTcB * (tl.k0 - j0 + r) + 4 * kg;
      float x[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const bool in = g + q >= lo && g + q < hi;   // inside the block: inside the staged range
        x[q] = in ? stage[in ? g + q - c0 : 0] : 0.f;
      }
      uint4 h, l;
      h.x = tf32_rna(x[0]); l.x = tf32_rna(x[0] - __uint_as_float(h.x));
      h.y = tf32_rna(x[1]); l.y = tf32_rna(x[1] - __uint_as_float(h.y));
      h.z = tf32_rna(x[2]); l.z = tf32_rna(x[2] - __uint_as_float(h.z));
      h.w = tf32_rna(x[3]); l.w = tf32_rna(x[3] - __uint_as_float(h.w));
      const int off = kg * kTcLboA + r * 16;
      *reinterpret_cast<uint4*>(a_hi + off) = h;
      *reinterpret_cast<uint4*>(a_lo + off) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;");   // generic-proxy writes -> tensor-core reads
    __syncthreads();
    if (threadIdx.x == 0) {
      issue(it + 2 * (int64_t)gridDim.x, st);   // the stage is free: the tile after next
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
      float* stg = reinterpret_cast<float*>(a_hi);   // [128][33]: padded rows, no bank conflicts
      const int row = 32 * warp + lane;
#pragma unroll
      for (int i = 0; i < kTcB; i++) stg[row * (kTcB + 1) + i] = sc * v[i];
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    {
      float* ur = u + rhs * u_stride;
      const float* stg = reinterpret_cast<const float*>(a_hi);
      const int64_t base = lo + (int64_t)kTcB * tl.k0;
      const bool v4 = ((base | u_stride) & 3) == 0 && (((uintptr_t)ur) & 15) == 0;
      for (int q = threadIdx.x; q < kTcM * kTcB / 4; q += kTcThreads) {
        const int row = q >> 3, c = 4 * (q & 7);
        const int64_t g = base + 4 * (int64_t)q;
        const float* sv = stg + row * (kTcB + 1) + c;
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
  // copies still in flight (issued ahead, or a wait that ran out) land before the memory is reused
  if (threadIdx.x == 0) {
    for (int st = 0; st < 2; st++)
      if (stage_busy[st]) mbar_wait(s_mld0 + 8 * st, (ld_phase >> st) & 1u);
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
