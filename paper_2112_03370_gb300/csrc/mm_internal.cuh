// Internal declarations of libmm shared by its translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mm.h"

namespace mm {

// ---------------------------------------------------------------------------------------------
// Toeplitz tile geometry.  One tile = L = 2M real samples gathered into M packed complex values
// (z[n] = t[2n] + i t[2n+1]); the tile's output range holds the samples whose whole band
// [g - lambda, g + lambda] lies inside the tile (overlap-save, Sect. 3.1 shift-and-overlap).
// ---------------------------------------------------------------------------------------------
constexpr int kLogM = 14;                 // complex points per tile (both precisions)
constexpr int kM = 1 << kLogM;            // 16384 complex = 32768 real samples
constexpr int kL = 2 * kM;
constexpr int kMaxLambda = 12288;         // keeps >= 8192 valid outputs per tile
constexpr int kBigTileLambda = 6144;      // FP32 operators can use 65536-sample tiles above this lambda
constexpr int kCl32 = 1;                  // FP32: one CTA holds the whole tile (128 KB smem)
constexpr int kCl64 = 2;                  // FP64: a 2-CTA cluster holds it (2 x 128 KB smem)
constexpr int kTileThreads = 512;

// A segment of n_steps consecutive overlap-save tiles of one block.  Tile k of the segment reads
// input samples [in0 + k vstep, in0 + k vstep + L) and writes outputs
// [out_lo + k vstep, min(out_lo + (k + 1) vstep, out_hi)).  Consecutive tiles overlap by
// L - vstep input samples, which the FP32 kernel keeps in shared memory instead of gathering
// them again.
struct TileDesc {
  int64_t in0;      // global sample index of the first tile's first input sample (multiple of 4)
  int64_t out_lo;   // output range [out_lo, out_hi) of the whole segment
  int64_t out_hi;
  int64_t blk_lo;   // the block's sample range: samples outside read as 0
  int64_t blk_hi;
  int32_t tab;      // spectrum table id
  int32_t n_steps;  // tiles in the segment (1 on the FP64 path)
  double scale;     // block band / table band
  int32_t vstep;    // output samples per tile (multiple of 4)
  int32_t prob;     // problem index of a multi-problem launch (0 otherwise)
};

// Per-problem pointers of a launch that batches the tiles of several plans (serving).
struct ProbPtrs {
  const int32_t* lpix;
  const float2* w32;
  const double2* w64;
  const void* tab;
  const void* x;
  void* y;
  const int32_t* done;
};

// MODE_APPLY_T: A-application whose un-pointed input t = P x was written beforehand (FP32
// tiles: float t; df64 tiles: (hi, lo) float pairs, also used for the masked TOD of the RHS)
// MODE_NINV_T: FP32 y = N^-1 t on the segments, float t in and float y out (the pointing is
// applied by the window kernels around it)
enum Mode { MODE_APPLY = 0, MODE_RHS = 1, MODE_NINV = 2, MODE_APPLY_T = 3, MODE_NINV_T = 4 };

// ---------------------------------------------------------------------------------------------
// Pixel windows of time-aligned detector groups (P and P^T of the FP32 A-application).
// A group is the same window [w0, w0 + W) of relative time in n_blk blocks b0, b0 + b_stride, ...
// (the detectors of one stationary interval).  Its kept samples see n_slots distinct pixels; slot
// k of the group is the k-th smallest of them (slot_pix[slot_off + k]), and every sample stores
// the slot of its pixel (uint16, kNoSlot at masked samples): a pixel-sorted local index, so the
// un-point kernel reads the group's map entries once into shared memory and the point kernel
// sums the group's samples per pixel in shared memory before one global update per pixel.
// ---------------------------------------------------------------------------------------------
constexpr int kWinCap = 4096;              // most distinct pixels of a group (shared-memory window)
constexpr int kWinThreads = 512;
constexpr uint16_t kNoSlot = 0xFFFF;
struct PGroup {
  int32_t b0;        // first block of the group
  int32_t n_blk;     // blocks in the group
  int32_t b_stride;  // block index step (n_int: the same interval of consecutive detectors)
  int32_t log_w;     // window length W = 2^log_w
  int32_t n_slots;   // distinct kept pixels (0 .. kWinCap)
  int32_t sub0;      // first sub-window of the group in the plan's sub-window list
  int32_t prob;      // multi-problem launches: the group's problem (index into the WinProb list)
  int64_t w0;        // window start, samples from each block's start
  int64_t slot_off;  // first entry of the group's pixel-sorted slot table
  int64_t ent_off;   // first pixel-sorted entry of the group's sub-windows
};

// Per-problem pointers of the multi-problem window launches of a server step (every running
// FP32 request's groups in one launch; group g belongs to problem groups[g].prob): its plan's
// block offsets, slots, slot tables and reduced angles, the map x read by P, the un-pointed t it
// writes, the u = N^-1 t read by P^T, the map y it accumulates into and the column's halt flag.
struct WinProb {
  const int64_t* block_off;
  const uint16_t* slot;
  const int32_t* slot_pix;
  const float* ang2;
  const float* x;    // [n_obs][4]
  float* t;          // [N]
  const float* u;    // [N]
  float* y;          // [n_obs][4]
  const int32_t* done;
};

// Pixel-sorted sub-windows (P^T by segment reduction).  Sub-window s of a group is the window
// [w0 + s 2^log_s, w0 + (s + 1) 2^log_s) of every block of the group, log_s the largest with
// n_blk 2^log_s <= sub_cap; its samples are numbered l = c 2^log_s + o (chunk c, offset o).  The
// plan stores, per sub-window, its entries (slot << 16 | l) sorted ascending, so every slot's
// samples form one run, masked samples (slot kNoSlot) and padding last, with each entry's angle
// beside it; a sub-window holds seg_stride(n_blk, log_s) entries (a multiple of 16).
constexpr int kSegRange = 16;              // entries one thread reduces at a time
__host__ __device__ inline int seg_log_s(int n_blk, int log_w, int sub_cap) {
  int ls = log_w;
  while (ls > 0 && ((int64_t)n_blk << ls) > sub_cap) ls--;
  return ls;
}
__host__ __device__ inline int64_t seg_stride(int n_blk, int log_s) {
  return ((((int64_t)n_blk << log_s) + kSegRange - 1) / kSegRange) * kSegRange;
}

// ---------------------------------------------------------------------------------------------
// Tensor-core banded Toeplitz product (k_tc_toeplitz.cu): tiles of 128 rows x 32 samples of one
// block, 3xTF32 tcgen05 MMAs over the 2 J0 + 1 row shifts, J0 = ceil(lambda / 32) <= kTcMaxJ0.
// ---------------------------------------------------------------------------------------------
constexpr int kTcMaxJ0 = 4;                 // lambda <= 128
constexpr int kTcAutoLambda = 64;           // MM_TPLZ_AUTO picks the tensor cores up to this lambda
                                            // (measured crossover against the FFT tiles)
struct TcTile {
  int32_t blk;   // block
  int32_t k0;    // first 32-sample row of the tile within the block
};
std::vector<TcTile> tc_tiles(const std::vector<int64_t>& block_off);
size_t tc_bmat_bytes(int32_t n_tab);
// T_J (hi, lo) of each band table in the kernel's shared-memory image layout
cudaError_t launch_tc_bmat(const double* rows, int32_t lambda, int32_t n_tab, void* bmat, cudaStream_t s);
// u = N^-1 t (FP32, 3xTF32 on the tensor cores), t and u [nrhs][stride]; err set on a timed-out wait
cudaError_t launch_tplz_tc(const TcTile* tiles, int64_t n_tiles, const int64_t* block_off, const int32_t* blk_tab,
                           const float* blk_scale, const void* bmat, int32_t lambda, const float* t,
                           int64_t t_stride, float* u, int64_t u_stride, int nrhs, const int32_t* done,
                           int done_stride, int32_t* err, cudaStream_t s);

// Arguments of the fused Toeplitz-tile kernels.
struct TileArgs {
  const TileDesc* tiles;
  int64_t n_tiles;
  int32_t nrhs;
  int64_t N;
  const int32_t* lpix;      // [N] local pixel or -1
  const float2* w32;        // [N] (cos, sin) (FP32 path)
  const double2* w64;       // [N] (cos, sin) (FP64 path)
  const float4* wdf;        // [N] (cos hi, cos lo, sin hi, sin lo) (df64 path)
  const void* tab;          // [n_tab][cl][M/cl] (a, b) of float2 / double2
  const void* tw;           // [M] twiddles W_M^k (float2 / double2)
  const void* x;            // APPLY: map in, [nrhs][n_obs][4]; RHS: d [nrhs][N]; NINV: t [N]
  int32_t x_is_fp32;        // RHS only: d in float32
  int64_t x_stride;         // elements between right-hand sides of x
  void* y;                  // APPLY/RHS: map out [nrhs][n_obs][4] (accumulated); NINV: y [N]
  int64_t y_stride;
  const int32_t* done;      // optional: skip the work of column r when done[r * done_stride] != 0
  int32_t done_stride;
  const ProbPtrs* probs;    // multi-problem launches: per-tile pointers (tile.prob), else null
  uint32_t* amax;           // MODE_NINV_T df64 tiles (optional): per column, the bits of max |u|
};

// ---------------------------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------------------------
struct Plan {
  int device = 0;
  int32_t n_det = 0, n_int = 0, n_blocks = 0;
  int64_t N = 0, n_pix = 0, n_obs = 0;
  int32_t lambda = 0, precision = MM_FP64, algo = MM_TPLZ_FFT;
  double cond_max = 1e3;
  std::vector<int64_t> block_off;      // host [n_blocks + 1]

  // device state
  int32_t* lpix = nullptr;             // [N]
  float* psi = nullptr;                // [N]
  float2* w32 = nullptr;               // [N] cos 2psi, sin 2psi in FP32 (FP32 operators)
  double2* w64 = nullptr;              // [N] cos 2psi, sin 2psi in FP64 (FP64 operators)
  bool df64 = false;                   // FP64-class operators run in df64 arithmetic
  float4* wdf = nullptr;               // [N] df64 weights (df64 plans)
  float* ang2 = nullptr;               // [N] 2 psi reduced to [-pi, pi] (FP32 window kernels)
  int32_t* obs_to_global = nullptr;    // [n_obs]
  double* minv = nullptr;              // [n_obs][6] symmetric inverse BD blocks (00 01 02 11 12 22)
  double* band = nullptr;              // [n_blocks][lambda + 1]
  int64_t* block_off_dev = nullptr;    // [n_blocks + 1]
  double* c0_blk = nullptr;            // [n_blocks]

  // Toeplitz FFT state
  int32_t n_tab = 0;
  float2* tab32 = nullptr;             // [n_tab][M]
  double2* tab64 = nullptr;            // [n_tab][M]
  float2* tw32 = nullptr;              // [M]
  double2* tw64 = nullptr;             // [M]
  float4* tabdf = nullptr;             // [n_tab][M] df64 pair tables (df64 plans)
  float4* twdf = nullptr;              // [M] df64 twiddles
  float2* tdf = nullptr;               // [nrhs][N4] un-pointed df64 input, N4 = N rounded up to 4
  size_t tdf_cap = 0;
  float4* mapdf = nullptr;             // [nrhs][n_obs][2] df64 map: (I hi, I lo, Q hi, Q lo), (U hi, U lo, 0, 0)
  size_t mapdf_cap = 0;
  TileDesc* tiles = nullptr;           // FP64 tiles (one per descriptor)
  int64_t n_tiles = 0;
  TileDesc* segs = nullptr;            // FP32 segments (several tiles per descriptor)
  int64_t n_segs = 0;
  std::vector<TileDesc> segs_host;     // host copy (multi-problem launches)
  std::vector<int32_t> blk_tab;        // host: spectrum table of each block
  std::vector<double> blk_scale;       // host: band scale of each block against its table
  int32_t tile_steps = 0;              // FP32 tiles walked per segment
  int32_t win_samples = 32768;         // target samples per pixel-window group
  int32_t tuned_width = 0;             // block width chosen by mm_autotune (0: not tuned)

  // tensor-core Toeplitz product (MM_TPLZ_GEMM plans)
  bool tc = false;                     // the FP32 N^-1 runs on the tensor cores
  TcTile* tc_tiles = nullptr;          // [n_tc_tiles]
  int64_t n_tc_tiles = 0;
  void* tc_bmat = nullptr;             // T_J images of every table
  int32_t* tc_tab = nullptr;           // [n_blocks] table of each block
  float* tc_scale = nullptr;           // [n_blocks] band scale of each block
  int32_t* tc_err = nullptr;           // set by a timed-out wait of the tensor-core kernel
  // FP32 N^-1 on 65536-sample tiles (2-CTA clusters) for large lambda: the tables are built for
  // lambda > kBigTileLambda, the path is used when mm_autotune measured it faster (use_big)
  bool big = false;
  bool use_big = false;
  TileDesc* segs_big = nullptr;        // one 65536-sample tile per descriptor
  int64_t n_segs_big = 0;
  float2* tab32_big = nullptr;         // [n_tab][2 kM] pair tables of the 32768-point transform
  float2* tw32_big = nullptr;          // [2 kM] twiddles W_{2 kM}^k
  float* t32 = nullptr;                // [nrhs][N4] un-pointed FP32 input of the tiles (N4 = N
                                       // rounded up to 4)
  size_t t32_cap = 0;
  int32_t seg_halo = 0;                // largest L - vstep over the segments (samples)

  // pixel windows of detector groups (FP32 operators); skipped by FP64-class server requests, whose
  // plans never run the FP32 operators
  bool no_windows = false;
  bool no_big = false;                 // skip the 65536-sample tile tables (server requests)
  PGroup* groups = nullptr;            // [n_groups]
  std::vector<PGroup> groups_host;     // host copy (multi-problem window launches)
  int64_t n_groups = 0;
  uint16_t* slot = nullptr;            // [N] pixel-sorted local index of each sample in its group
  int32_t* slot_pix = nullptr;         // [n_slots_total] compacted pixel of each slot
  int64_t n_slots_total = 0;
  float* u32 = nullptr;                // [nrhs][N4] FP32 u = N^-1 t of the windowed A-application
  size_t u32_cap = 0;
  float2* udf = nullptr;               // [nrhs][N4] df64 u = N^-1 t of the windowed df64 operator
  size_t udf_cap = 0;
  uint32_t* amax = nullptr;            // [amax_cap] per column: bits of max |u| of the df64 tiles
  size_t amax_cap = 0;
  double win_repeat = 0.0;             // kept samples per (group, pixel) pair: the P^T reduction factor
  // pixel-sorted sub-windows of the groups (P^T by segment reduction; FP32 operators)
  bool use_seg = false;                // the FP32 P^T reduces pixel-sorted runs (else per-sample
                                       // shared-memory atomics over the windows)
  int32_t seg_sub = 8192;              // most samples of a sub-window
  uint32_t* seg_ent = nullptr;         // [n_ent] sorted entries (slot << 16 | l)
  float* seg_ang = nullptr;            // [n_ent] 2 psi of each entry
  int32_t* seg_kept = nullptr;         // [n_sub_total] kept samples of each sub-window
  int64_t n_ent = 0;
  int64_t n_sub_total = 0;

  // work buffers (grown on demand)
  float* map32_in = nullptr;  size_t map32_in_cap = 0;
  float* map32_out = nullptr; size_t map32_out_cap = 0;
  double* map64_in = nullptr; size_t map64_in_cap = 0;
  double* map64_out = nullptr; size_t map64_out_cap = 0;

  // time-domain scratch of the direct path and of the P / P^T / N^-1 entry points
  double* td_a = nullptr;
  double* td_b = nullptr;
  size_t td_cap = 0;

  // staging of host TOD in mm_rhs: two device buffers filled on a copy stream
  void* stage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  cudaStream_t copy_stream = nullptr;
  void* tod_buf = nullptr;             // device copy of a host TOD handed to mm_solve_tod
  size_t tod_cap = 0;
  cudaEvent_t stage_ev[4] = {nullptr, nullptr, nullptr, nullptr};   // copied[0..1], consumed[0..1]

  cudaStream_t stream = nullptr;       // plan-owned stream (graph capture)
  void* cg = nullptr;                  // solver workspace (mm_api.cu)
  void* blk = nullptr;                 // block-CG workspace (mm_api.cu)
  void* defl = nullptr;                // two-level deflation space (mm_api.cu)
  void* tmpl = nullptr;                // template map-making state (TmplState, mm_tmpl.cuh)
  uint64_t buf_gen = 0;                // bumped whenever a buffer a captured graph may read is reallocated

  size_t bytes = 0;
};

// error state
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define MM_CUDA(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ::mm::cuda_fail(e_, #call);      \
  } while (0)

template <typename T>
int dalloc(Plan* p, T** ptr, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)ptr, n * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return fail(MM_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  p->bytes += n * sizeof(T);
  return MM_OK;
}

// ---------------------------------------------------------------------------------------------
// launchers (each returns a cudaError_t of its launch)
// ---------------------------------------------------------------------------------------------
// plan kernels (k_plan.cu)
cudaError_t launch_bd_accum(const int32_t* pix, const double2* w64, const int64_t* block_off,
                            const double* c0_blk, int32_t n_blocks, int64_t N, double* B6,
                            int32_t* hits, cudaStream_t s);
cudaError_t launch_bd_finalize(const double* B6, const int32_t* hits, int64_t n_pix,
                               double cond_max, int32_t* keep, double* inv6, cudaStream_t s);
cudaError_t launch_scan_keep(const int32_t* keep, int64_t n, int32_t* lid, int32_t* total,
                             int32_t* scratch, int64_t scratch_len, cudaStream_t s);
size_t scan_scratch_len(int64_t n);
cudaError_t launch_compact(const int32_t* keep, const int32_t* lid, const double* inv6_glob,
                           int64_t n_pix, int32_t* obs_to_global, double* minv, cudaStream_t s);
cudaError_t launch_localize(const int32_t* pix, const int32_t* keep, const int32_t* lid,
                            int64_t N, int32_t* lpix, cudaStream_t s);
// (cos 2psi, sin 2psi) in FP64, their FP32 roundings, (wdf non-null) their df64 split and (ang2
// non-null) 2 psi reduced to [-pi, pi], one sincos per sample
cudaError_t launch_weights(const float* psi, int64_t N, double2* w64, float2* w32, float4* wdf, float* ang2,
                           cudaStream_t s);
cudaError_t launch_validate(const int32_t* pix, const float* psi, int64_t N, int64_t n_pix,
                            int32_t* bad, cudaStream_t s);
// spectra of the L-point circulants, L = 2^(logm + 1): H [n_tab][M + 1], costab [L]
cudaError_t launch_spectra(const double* band_rows, int32_t n_tab, int32_t lambda,
                           double* H /* [n_tab][M+1] */, const double* costab /* [L] */,
                           cudaStream_t s, int logm = kLogM);
cudaError_t launch_pair_tables(const double* H, int32_t n_tab, const double* costab,
                               double2* tab64, float2* tab32, cudaStream_t s);
// FP32 pair tables of the 65536-sample 2-CTA tiles: tab32 [n_tab][2 kM]
cudaError_t launch_pair_table32_big(const double* H, int32_t n_tab, const double* costab, float2* tab32,
                                    cudaStream_t s);
// W_M^k, k < M = 2^logm (tw64 may be null)
cudaError_t launch_twiddles(double2* tw64, float2* tw32, const double* costab, cudaStream_t s,
                            int logm = kLogM);
// FP32 u = N^-1 t over 65536-sample 2-CTA tiles
cudaError_t launch_ninv32_big(const TileArgs& a, cudaStream_t s);

// Toeplitz-tile kernels (k_toeplitz.cu)
cudaError_t launch_tiles_fp32(int mode, const TileArgs& a, int halo_samples, cudaStream_t s);
// FP32 A-application over the tiles of several plans at once (a.probs set, nrhs = 1)
cudaError_t launch_tiles_fp32_multi(const TileArgs& a, int halo_samples, cudaStream_t s);
// u = N^-1 t of several problems' segments in one launch (a.probs: x = t, y = u, tab, done of
// each problem; nrhs 1)
cudaError_t launch_ninv32_multi(const TileArgs& a, int halo_samples, cudaStream_t s);
// t [nrhs][t_stride] float32 = P x for every sample (0 at masked samples), x float4 maps
// [nrhs][n_obs]
cudaError_t launch_unpoint32(const int32_t* lpix, const float2* w32, int64_t N, const float* x4,
                             int64_t x_stride, int nrhs, const int32_t* done, int done_stride, float* t,
                             int64_t t_stride, cudaStream_t s);
cudaError_t launch_tiles_fp64(int mode, const TileArgs& a, cudaStream_t s);

// pixel windows (k_window.cu)
// count (slot_tab == nullptr: n_slots of every group, -1 when over kWinCap) or fill (slots and
// tables of groups whose n_slots and slot_off are set)
cudaError_t launch_win_build(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                             const int32_t* lpix, int32_t* n_slots_out, uint16_t* slot, int32_t* slot_pix,
                             cudaStream_t s);
// t [nrhs][t_stride] = P x (FP32, weights from psi in registers) over the windows
cudaError_t launch_unpoint_win32(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                                 const uint16_t* slot, const int32_t* slot_pix, const float* psi,
                                 const float* x4, int64_t x_stride, int nrhs, const int32_t* done,
                                 int done_stride, float* t, int64_t t_stride, cudaStream_t s);
// y4 [nrhs][y_stride] (FP64 map) += P^T u for df64 u ((hi, lo) pairs [nrhs][u_stride]) over the
// windows: per group, 64-bit fixed-point sums in shared memory scaled by amax[r] (bits of the
// column's max |u|), then one FP64 atomic per pixel and component
cudaError_t launch_point_win_df(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                                const uint16_t* slot, const int32_t* slot_pix, const float4* wdf,
                                const float2* u, int64_t u_stride, const uint32_t* amax, int nrhs,
                                const int32_t* done, int done_stride, double* y4, int64_t y_stride,
                                cudaStream_t s);
// pixel-sorted entries of every sub-window of the groups (groups' sub0 and ent_off set)
cudaError_t launch_seg_build(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                             const uint16_t* slot, const float* ang2, int sub_cap, uint32_t* ent,
                             float* ent_ang, int32_t* kept, cudaStream_t s);
// y4 [nrhs][y_stride] += P^T u (FP32) by segment reduction over the pixel-sorted sub-windows
cudaError_t launch_point_seg32(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                               const uint32_t* ent, const float* ent_ang, const int32_t* kept,
                               const int32_t* slot_pix, int sub_cap, const float* u, int64_t u_stride,
                               int nrhs, const int32_t* done, int done_stride, float* y4, int64_t y_stride,
                               cudaStream_t s);
// y4 [nrhs][y_stride] += P^T u (FP32) over the windows, u [nrhs][u_stride]
cudaError_t launch_point_win32(const PGroup* groups, int64_t n_groups, const int64_t* block_off,
                               const uint16_t* slot, const int32_t* slot_pix, const float* psi,
                               const float* u, int64_t u_stride, int nrhs, const int32_t* done,
                               int done_stride, float* y4, int64_t y_stride, cudaStream_t s);
// the same two operators for several problems in one launch (continuous batching): groups from
// every problem's plan, each with its prob index into probs (one column per problem)
cudaError_t launch_unpoint_win32_multi(const PGroup* groups, int64_t n_groups, const WinProb* probs,
                                       cudaStream_t s);
cudaError_t launch_point_win32_multi(const PGroup* groups, int64_t n_groups, const WinProb* probs,
                                     cudaStream_t s);
// multiprocessors of the current device (cached per device)
int sm_count();
// df64 tiles and their data preparation (k_df64.cu)
cudaError_t launch_tiles_df(const TileArgs& a, cudaStream_t s);
// df64 u = N^-1 t (pairs in, pairs out), per-column max |u| into a.amax
cudaError_t launch_ninv_df(const TileArgs& a, cudaStream_t s);
cudaError_t launch_weights_df(const float* psi, int64_t N, float4* wdf, cudaStream_t s);
cudaError_t launch_c64_to_df(const double2* in, int64_t n, float4* out, cudaStream_t s);
cudaError_t launch_map_to_df(const double* m4, int64_t n_pix4, float4* out, cudaStream_t s);
cudaError_t launch_unpoint_df(const int32_t* lpix, const float4* wdf, int64_t N, const float4* mapdf,
                              int64_t n_obs, int nrhs, const int32_t* done, int done_stride, float2* t,
                              int64_t t_stride, cudaStream_t s, const void* d = nullptr, int d_is_fp32 = 0);
cudaError_t launch_d_to_df(const int32_t* lpix, const void* d, int d_is_fp32, int64_t N, int nrhs,
                           float2* t, int64_t t_stride, cudaStream_t s);
// t [nrhs][t_stride] = G d rounded to FP32
cudaError_t launch_d_to_t32(const int32_t* lpix, const void* d, int d_is_fp32, int64_t N, int nrhs, float* t,
                            int64_t t_stride, cudaStream_t s);
int tile_kernels_init();   // sets smem attributes once per process
int fp32_max_halo_samples();   // largest halo the FP32 segment kernel can keep in shared memory

// direct / elementwise kernels (k_vec.cu)
cudaError_t launch_toeplitz_direct(const double* band, const int64_t* block_off, int32_t n_blocks,
                                   int32_t lambda, int64_t N, const double* t, double* y,
                                   cudaStream_t s);
cudaError_t launch_unpoint64(const int32_t* lpix, const double2* w64, int64_t N,
                             const double* x4, double* t, cudaStream_t s);
cudaError_t launch_point64(const int32_t* lpix, const double2* w64, int64_t N, const double* t,
                           double* y4, cudaStream_t s);
cudaError_t launch_mask_d(const int32_t* lpix, const void* d, int d_is_fp32, int64_t N,
                          double* out, cudaStream_t s);
cudaError_t launch_pack3to4(const double* x3, int64_t n, int nrhs, double* x4, cudaStream_t s);
cudaError_t launch_unpack4to3(const double* x4, int64_t n, int nrhs, double* x3, cudaStream_t s);
cudaError_t launch_to32(const double* x4, int64_t n4, float* y4, cudaStream_t s);
cudaError_t launch_to64(const float* x4, int64_t n4, double* y4, cudaStream_t s);
cudaError_t launch_to_global(const double* x4, const int32_t* o2g, int64_t n, double* map3, cudaStream_t s);
cudaError_t launch_bd_apply(const double* minv, int64_t n, int nrhs, const double* r4, double* z4,
                            cudaStream_t s);

// CG kernels (k_vec.cu)
struct CgScalars;   // defined in k_vec.cu
}  // namespace mm
