// C ABI of libmm: plan construction, the operators of the map-making system and the PCG driver.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "mm_block.cuh"
#include "mm_cg.cuh"
#include "mm_defl.cuh"
#include "mm_internal.cuh"
#include "mm_tmpl.cuh"

namespace mm {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
// multiprocessors of the current device, cached per device (the GB300's 152 only if the query fails)
int sm_count() {
  constexpr int kFallbackSms = 152;
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return kFallbackSms;
  int n = 0;
  if (dev >= 64)
    return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : kFallbackSms;
  if (cached[dev] == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return kFallbackSms;
    cached[dev] = n;
  }
  return cached[dev];
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return MM_ECUDA;
}

namespace {

// Solver workspace, grown on demand and kept with the plan.
struct CgState {
  int64_t n = 0;
  int nrhs_cap = 0;
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  float *p32 = nullptr, *q32 = nullptr;
  double* partials = nullptr;
  unsigned* counters = nullptr;
  CgScalars* scal = nullptr;
  CgScalars* scal_host = nullptr;   // pinned
  // cached graph of `chunk` iterations
  cudaGraphExec_t exec = nullptr;
  int g_nrhs = -1, g_fp32 = -1, g_chunk = -1, g_maxit = -1, g_prec = -1;
  double g_tol2 = -1.0;
  uint64_t g_buf_gen = ~0ull;       // plan buffer generation the graph's pointers belong to
};

// Block-CG workspace, grown on demand and kept with the plan.
struct BlkState {
  int64_t n = 0;
  int s_cap = 0;
  double *X = nullptr, *R = nullptr, *B = nullptr, *AX = nullptr;   // [s][n][4] FP64
  float *Z = nullptr, *AZ = nullptr, *P = nullptr, *AP = nullptr;   // [s][n][4] FP32
  double *part = nullptr, *G = nullptr, *Linv = nullptr, *Cmb = nullptr, *alpha = nullptr,
         *C2 = nullptr, *norms = nullptr, *norm_part = nullptr;
  int *piv = nullptr, *rank = nullptr, *idx = nullptr;
  double* T64 = nullptr;    // [s][n][4] FP64 apply output (FP64 operator path)
  double* host = nullptr;   // pinned: norms
  int* host_i = nullptr;    // pinned: rank
  // enlarged CG: previous search block (Orthodir), accumulated solution, residual, A x
  float *Pp = nullptr, *APp = nullptr;                               // [s][n][4] FP32
  double *xe = nullptr, *re = nullptr, *ax = nullptr;                // [n][4] FP64
  // captured parts of a block iteration (FP32 operators), by shape; they hold raw pointers into
  // this state and the plan, valid while neither is reallocated (graph_gen = the plan's buf_gen)
  std::unordered_map<uint64_t, cudaGraphExec_t> graphs;
  uint64_t graph_gen = 0;
};

// Two-level deflation space and its per-solve work buffers.
struct DeflState {
  int k = 0;
  int64_t n = 0;
  float *Z = nullptr, *Zp = nullptr;            // [k][n][4]
  double* Einv = nullptr;                      // [k][k]
  std::vector<double> theta;                   // Ritz values (host copy)
  int nrhs_cap = 0;
  double *y = nullptr, *part = nullptr, *part2 = nullptr;
  unsigned *counters = nullptr, *counters2 = nullptr;
};

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

int grow(Plan* P, double** buf, size_t* cap, size_t n) {
  if (*cap >= n && *buf) return MM_OK;
  dfree(*buf);
  *cap = 0;
  int st = dalloc(P, buf, n);
  if (st == MM_OK) *cap = n;
  return st;
}
int grow32(Plan* P, float** buf, size_t* cap, size_t n) {
  if (*cap >= n && *buf) return MM_OK;
  dfree(*buf);
  *cap = 0;
  int st = dalloc(P, buf, n);
  if (st == MM_OK) *cap = n;
  return st;
}

void free_cg(CgState* c) {
  if (!c) return;
  dfree(c->b); dfree(c->x); dfree(c->r); dfree(c->z); dfree(c->p); dfree(c->q);
  dfree(c->p32); dfree(c->q32); dfree(c->partials); dfree(c->counters); dfree(c->scal);
  if (c->scal_host) cudaFreeHost(c->scal_host);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  delete c;
}

void free_blk(BlkState* b) {
  if (!b) return;
  dfree(b->X); dfree(b->R); dfree(b->B); dfree(b->AX); dfree(b->Z); dfree(b->AZ); dfree(b->P);
  dfree(b->AP); dfree(b->part); dfree(b->G); dfree(b->Linv); dfree(b->Cmb); dfree(b->alpha);
  dfree(b->C2); dfree(b->norms); dfree(b->norm_part); dfree(b->piv); dfree(b->rank); dfree(b->idx);
  dfree(b->T64); dfree(b->Pp); dfree(b->APp); dfree(b->xe); dfree(b->re); dfree(b->ax);
  if (b->host) cudaFreeHost(b->host);
  if (b->host_i) cudaFreeHost(b->host_i);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  delete b;
}

// Replay on s the captured graph of `key` (bits 60-63: 1, 2 the two parts of a block CG iteration,
// 3, 4 those of an enlarged-CG iteration; below: the shape), capturing enqueue() into it first when it is absent
// or when the plan's buffers were reallocated since the graphs were captured.
template <typename F>
int blk_graph(Plan* P, BlkState* b, uint64_t key, cudaStream_t s, F&& enqueue) {
  if (b->graph_gen != P->buf_gen) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->graph_gen = P->buf_gen;
  }
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaGraph_t g = nullptr;
    MM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int st = enqueue();
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (st != MM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    MM_CUDA(ce);
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    MM_CUDA(ie);
    it = b->graphs.emplace(key, ex).first;
  }
  MM_CUDA(cudaGraphLaunch(it->second, s));
  return MM_OK;
}

void free_defl(DeflState* d) {
  if (!d) return;
  dfree(d->Z); dfree(d->Zp); dfree(d->Einv); dfree(d->y); dfree(d->part); dfree(d->part2);
  dfree(d->counters); dfree(d->counters2);
  delete d;
}

void free_tmpl(TmplState* t) {
  if (!t) return;
  dfree(t->bin8); dfree(t->frac32); dfree(t->fracdf); dfree(t->hwpdf); dfree(t->hwp32); dfree(t->M64);
  dfree(t->M32);
  dfree(t->xscale); dfree(t->xoff);
  dfree(t->pscale);
  dfree(t->kinv);
  delete t;
}

void free_plan(Plan* P) {
  if (!P) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  dfree(P->lpix); dfree(P->psi); dfree(P->w32); dfree(P->w64); dfree(P->obs_to_global); dfree(P->minv);
  dfree(P->band); dfree(P->block_off_dev); dfree(P->c0_blk); dfree(P->tab32); dfree(P->tab64);
  dfree(P->tw32); dfree(P->tw64); dfree(P->tiles); dfree(P->segs); dfree(P->map32_in); dfree(P->map32_out);
  dfree(P->map64_in); dfree(P->map64_out); dfree(P->td_a); dfree(P->td_b); dfree(P->t32);
  dfree(P->wdf); dfree(P->tabdf); dfree(P->twdf); dfree(P->tdf); dfree(P->mapdf);
  dfree(P->ang2); dfree(P->groups); dfree(P->slot); dfree(P->slot_pix); dfree(P->u32);
  dfree(P->seg_ent); dfree(P->seg_ang); dfree(P->seg_kept);
  dfree(P->udf); dfree(P->amax);
  dfree(P->tc_tiles); dfree(P->tc_tab); dfree(P->tc_scale); dfree(P->tc_err);
  dfree(P->segs_big); dfree(P->tab32_big); dfree(P->tw32_big);
  if (P->tc_bmat) { cudaFree(P->tc_bmat); P->tc_bmat = nullptr; }
  for (void*& b : P->stage) if (b) { cudaFree(b); b = nullptr; }
  for (cudaEvent_t& e : P->stage_ev) if (e) { cudaEventDestroy(e); e = nullptr; }
  if (P->copy_stream) cudaStreamDestroy(P->copy_stream);
  if (P->tod_buf) cudaFree(P->tod_buf);
  free_cg(reinterpret_cast<CgState*>(P->cg));
  free_blk(reinterpret_cast<BlkState*>(P->blk));
  free_defl(reinterpret_cast<DeflState*>(P->defl));
  free_tmpl(reinterpret_cast<TmplState*>(P->tmpl));
  if (P->stream) cudaStreamDestroy(P->stream);
  cudaSetDevice(cur);
  delete P;
}

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

// ---- band de-duplication: blocks whose rows are scalar multiples share one spectrum table ----
struct BandTables {
  std::vector<int32_t> blk_tab;     // [n_blocks]
  std::vector<double> blk_scale;    // [n_blocks]
  std::vector<int32_t> tab_src;     // block whose row defines the table
};

uint64_t row_key(const double* c, int lam) {
  uint64_t h = 1469598103934665603ull;
  const int idx[3] = {std::min(1, lam), lam / 2, lam};
  for (int k = 0; k < 3; k++) {
    const double v = c[idx[k]] / c[0];
    const long long q = (long long)std::llround(v * 1e9);
    h ^= (uint64_t)q;
    h *= 1099511628211ull;
  }
  return h;
}

bool rows_match(const double* a, const double* b, int lam) {
  const double a0 = a[0], b0 = b[0];
  double amax = 0.0;
  for (int k = 0; k <= lam; k++) amax = std::max(amax, std::fabs(b[k] / b0));
  for (int k = 0; k <= lam; k++) {
    if (std::fabs(a[k] / a0 - b[k] / b0) > 1e-14 * amax) return false;
  }
  return true;
}

BandTables dedupe_bands(const std::vector<double>& band, int nb, int lam) {
  BandTables t;
  t.blk_tab.resize(nb);
  t.blk_scale.resize(nb);
  std::unordered_map<uint64_t, std::vector<int32_t>> buckets;
  for (int b = 0; b < nb; b++) {
    const double* row = band.data() + (size_t)b * (lam + 1);
    const uint64_t key = row_key(row, lam);
    int found = -1;
    auto it = buckets.find(key);
    if (it != buckets.end()) {
      for (int32_t tab : it->second) {
        const double* ref = band.data() + (size_t)t.tab_src[tab] * (lam + 1);
        if (rows_match(row, ref, lam)) {
          found = tab;
          break;
        }
      }
    }
    if (found < 0) {
      found = (int)t.tab_src.size();
      t.tab_src.push_back(b);
      buckets[key].push_back(found);
    }
    t.blk_tab[b] = found;
    t.blk_scale[b] = row[0] / band[(size_t)t.tab_src[found] * (lam + 1)];
  }
  return t;
}

// Overlap-save tiles of every block.  A block of n samples gets t = ceil(n / vmax) tiles with
// vmax = L - 2 lambda - a rounded down to a multiple of 4, a = (block start - lambda) mod 4, all
// with the same output step vstep = ceil(n / t) rounded up to a multiple of 4 (so no tile is
// nearly empty).  Each tile's input window starts at the multiple of 4 a samples before
// (first output - lambda), so its L inputs cover every output's band.
// Tiles are grouped into segments of up to `max_steps` consecutive tiles (one CTA walks a
// segment and keeps the overlap of consecutive windows); max_steps = 1 gives single tiles.
std::vector<TileDesc> make_tiles(const std::vector<int64_t>& off, const BandTables& bt, int lam,
                                 int max_steps, int max_halo, int32_t* halo_out, int64_t L = kL) {
  std::vector<TileDesc> tiles;
  const int nb = (int)off.size() - 1;
  int32_t halo_used = 0;
  for (int b = 0; b < nb; b++) {
    const int64_t lo = off[b], hi = off[b + 1], n = hi - lo;
    if (n <= 0) continue;
    // a tile's input starts at out_lo - lam rounded down to a multiple of 4 (a samples earlier),
    // and its L inputs must reach out_hi + lam: vstep <= L - 2 lam - a (a multiple of 4)
    const int64_t a = (((lo - lam) % 4) + 4) % 4;
    const int64_t vmax = (L - 2 * (int64_t)lam - a) & ~(int64_t)3;
    const int64_t nt = (n + vmax - 1) / vmax;
    const int64_t vstep = (((n + nt - 1) / nt) + 3) & ~(int64_t)3;
    const int64_t halo = L - vstep;
    const int64_t steps_cap = (halo <= max_halo) ? max_steps : 1;
    const int64_t nseg = (nt + steps_cap - 1) / steps_cap;
    const int64_t per = (nt + nseg - 1) / nseg;
    for (int64_t t0 = 0; t0 < nt; t0 += per) {
      const int64_t t1 = std::min(t0 + per, nt);
      TileDesc td{};
      td.out_lo = lo + t0 * vstep;
      td.out_hi = std::min(lo + t1 * vstep, hi);
      const int64_t start = td.out_lo - lam;
      td.in0 = (start >= 0) ? (start & ~(int64_t)3) : -((-start + 3) & ~(int64_t)3);
      td.blk_lo = lo;
      td.blk_hi = hi;
      td.tab = bt.blk_tab[b];
      td.scale = bt.blk_scale[b];
      td.n_steps = (int32_t)(t1 - t0);
      td.vstep = (int32_t)vstep;
      if (td.n_steps > 1) halo_used = std::max(halo_used, (int32_t)halo);
      tiles.push_back(td);
    }
  }
  if (halo_out) *halo_out = halo_used;
  return tiles;
}

int validate_desc(const mm_problem_desc* d) {
  if (!d) return fail(MM_EINVAL, "desc is NULL");
  if (d->n_det <= 0 || d->n_int <= 0) return fail(MM_EINVAL, "n_det and n_int must be >= 1");
  if (!d->block_len) return fail(MM_EINVAL, "block_len is NULL");
  if (d->n_pix <= 0 || d->n_pix >= (int64_t)0x7fffffff) return fail(MM_EINVAL, "n_pix out of range");
  if (d->lambda < 0 || d->lambda > kMaxLambda)
    return fail(MM_EINVAL, "lambda must lie in [0, " + std::to_string(kMaxLambda) + "]");
  if (!d->pix || !d->psi || !d->band) return fail(MM_EINVAL, "pix, psi and band must be non-NULL");
  if (d->tile_steps < 0) return fail(MM_EINVAL, "tile_steps must be >= 0");
  if (d->pt_sub != 0 && d->pt_sub != 4096 && d->pt_sub != 8192 && d->pt_sub != 16384)
    return fail(MM_EINVAL, "pt_sub must be 0, 4096, 8192 or 16384");
  if (d->precision != MM_FP64 && d->precision != MM_FP32 && d->precision != MM_DF64 &&
      d->precision != MM_FP32_DF64)
    return fail(MM_EINVAL, "bad precision");
  if (d->toeplitz_algo != MM_TPLZ_AUTO && d->toeplitz_algo != MM_TPLZ_FFT &&
      d->toeplitz_algo != MM_TPLZ_GEMM && d->toeplitz_algo != MM_TPLZ_DIRECT)
    return fail(MM_EINVAL, "bad toeplitz_algo");
  if (d->toeplitz_algo == MM_TPLZ_GEMM) {
    if (d->lambda > kTcMaxJ0 * 32)
      return fail(MM_EINVAL, "MM_TPLZ_GEMM needs lambda <= " + std::to_string(kTcMaxJ0 * 32));
    if (d->precision != MM_FP32 && d->precision != MM_FP32_DF64)
      return fail(MM_EINVAL, "MM_TPLZ_GEMM runs the FP32 operators: use MM_FP32 or MM_FP32_DF64");
  }
  return MM_OK;
}

#define MM_TRY(expr)              \
  do {                            \
    int st_ = (expr);             \
    if (st_ != MM_OK) return st_; \
  } while (0)

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// largest time-domain working set (t, and u = N^-1 t with pixel windows, for the columns of one
// pass) the split A-applications may allocate per precision
constexpr size_t kSplitTBytes = (size_t)48 << 30;

// Plan-time scratch: freed when the plan build returns, on every path.
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  int alloc(T** p, size_t n) {
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
      *p = nullptr;
      return fail(MM_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    ptrs.push_back((void*)*p);
    return MM_OK;
  }
};

// FP32 segments of up to `steps` consecutive tiles (replacing previous ones: captured graphs
// must be captured again)
int build_segments(Plan* P, int steps, cudaStream_t s) {
  BandTables bt;
  bt.blk_tab = P->blk_tab;
  bt.blk_scale = P->blk_scale;
  std::vector<TileDesc> segs = make_tiles(P->block_off, bt, P->lambda, std::max(1, steps), fp32_max_halo_samples(),
                                          &P->seg_halo);
  if (P->segs) {
    P->buf_gen++;
    dfree(P->segs);
  }
  P->n_segs = (int64_t)segs.size();
  P->segs_host = segs;
  P->tile_steps = std::max(1, steps);
  MM_TRY(dalloc(P, &P->segs, segs.size()));
  MM_CUDA(cudaMemcpyAsync(P->segs, segs.data(), segs.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, s));
  return MM_OK;
}

// Pixel windows of time-aligned detector groups for the FP32 operators (P and P^T of the FP32
// A-application; Sect. 3.1 local pixel indexation applied per group of samples).  The detectors of
// every stationary interval are taken in groups of up to kWinDets, over windows of W = 2^k samples
// of relative time (about win_samples samples per group, W >= 32).  A group whose kept samples see
// more than kWinCap distinct pixels is split, its window halved down to 32 samples and then its
// detectors halved, until every group fits; then each group's pixel-sorted slot table and every
// sample's slot are written.
int build_windows(Plan* P, cudaStream_t s) {
  constexpr int kWinDets = 512;
  const int64_t kWinSamples = P->win_samples;
  constexpr int kMinLogW = 5;
  // a rebuild (autotuning) replaces the previous windows; captured graphs must be captured again
  if (P->groups) {
    P->buf_gen++;
    P->bytes -= (size_t)P->n_groups * sizeof(PGroup) + (size_t)P->N * sizeof(uint16_t) +
                (size_t)std::max<int64_t>(P->n_slots_total, 1) * sizeof(int32_t);
    dfree(P->groups);
    dfree(P->slot);
    dfree(P->slot_pix);
    P->n_groups = 0;
    P->groups_host.clear();
  }
  if (P->seg_ent) {
    P->bytes -= (size_t)P->n_ent * (sizeof(uint32_t) + sizeof(float)) + (size_t)P->n_sub_total * sizeof(int32_t);
    dfree(P->seg_ent);
    dfree(P->seg_ang);
    dfree(P->seg_kept);
    P->n_ent = P->n_sub_total = 0;
  }
  const std::vector<int64_t>& off = P->block_off;
  for (int b = 0; b < P->n_blocks; b++)
    if (off[b + 1] - off[b] > ((int64_t)1 << 30)) return MM_OK;   // blocks that long keep the fused tiles
  std::vector<PGroup> pending, done;
  for (int i = 0; i < P->n_int; i++) {
    for (int d0 = 0; d0 < P->n_det; d0 += kWinDets) {
      const int nd = std::min(kWinDets, P->n_det - d0);
      int64_t maxlen = 0;
      for (int d = d0; d < d0 + nd; d++) {
        const int b = d * P->n_int + i;
        maxlen = std::max(maxlen, off[b + 1] - off[b]);
      }
      int log_w = kMinLogW;
      while (log_w < 30 && ((int64_t)nd << (log_w + 1)) <= kWinSamples) log_w++;
      for (int64_t w0 = 0; w0 < maxlen; w0 += (int64_t)1 << log_w) {
        PGroup g{};
        g.b0 = d0 * P->n_int + i;
        g.n_blk = nd;
        g.b_stride = P->n_int;
        g.log_w = log_w;
        g.w0 = w0;
        pending.push_back(g);
      }
    }
  }
  Scratch scr;
  for (int round = 0; !pending.empty(); round++) {
    if (round > 64) return fail(MM_EINVAL, "pixel windows: splitting did not converge");
    PGroup* gd = nullptr;
    int32_t* cnt = nullptr;
    MM_TRY(scr.alloc(&gd, pending.size()));
    MM_TRY(scr.alloc(&cnt, pending.size()));
    MM_CUDA(cudaMemcpyAsync(gd, pending.data(), pending.size() * sizeof(PGroup), cudaMemcpyHostToDevice, s));
    MM_CUDA(launch_win_build(gd, (int64_t)pending.size(), P->block_off_dev, P->lpix, cnt, nullptr, nullptr, s));
    std::vector<int32_t> hc(pending.size());
    MM_CUDA(cudaMemcpyAsync(hc.data(), cnt, hc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    std::vector<PGroup> next;
    for (size_t k = 0; k < pending.size(); k++) {
      PGroup g = pending[k];
      if (hc[k] >= 0) {
        g.n_slots = hc[k];
        done.push_back(g);
      } else if (g.log_w > kMinLogW) {
        g.log_w--;
        PGroup h = g;
        h.w0 += (int64_t)1 << g.log_w;
        next.push_back(g);
        next.push_back(h);
      } else if (g.n_blk > 1) {
        const int half = g.n_blk / 2;
        PGroup h = g;
        g.n_blk = half;
        h.b0 += half * g.b_stride;
        h.n_blk -= half;
        next.push_back(g);
        next.push_back(h);
      } else {
        return fail(MM_EINVAL, "pixel windows: a single detector chunk exceeds the window capacity");
      }
    }
    pending.swap(next);
  }
  // process groups interval by interval, in time order, detectors ascending
  std::sort(done.begin(), done.end(), [&](const PGroup& a, const PGroup& b) {
    const int ia = a.b0 % P->n_int, ib = b.b0 % P->n_int;
    if (ia != ib) return ia < ib;
    if (a.w0 != b.w0) return a.w0 < b.w0;
    return a.b0 < b.b0;
  });
  int64_t total = 0;
  const bool seg = P->precision == MM_FP32 && P->use_seg;   // pixel-sorted sub-windows (FP32 P^T)
  int64_t n_ent = 0, n_sub = 0;
  for (PGroup& g : done) {
    g.slot_off = total;
    total += g.n_slots;
    const int ls = seg_log_s(g.n_blk, g.log_w, P->seg_sub);
    g.sub0 = (int32_t)n_sub;
    g.ent_off = n_ent;
    n_sub += (int64_t)1 << (g.log_w - ls);
    n_ent += ((int64_t)1 << (g.log_w - ls)) * seg_stride(g.n_blk, ls);
  }
  if (seg && n_sub > 0x7fffffffLL) return fail(MM_EINVAL, "pixel windows: too many sub-windows");
  P->n_groups = (int64_t)done.size();
  P->n_slots_total = total;
  P->win_repeat = total > 0 ? (double)P->N / (double)total : 0.0;
  MM_TRY(dalloc(P, &P->groups, done.size()));
  MM_TRY(dalloc(P, &P->slot, P->N));
  MM_TRY(dalloc(P, &P->slot_pix, (size_t)std::max<int64_t>(total, 1)));
  int32_t* err = nullptr;
  MM_TRY(scr.alloc(&err, 1));
  MM_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
  MM_CUDA(cudaMemcpyAsync(P->groups, done.data(), done.size() * sizeof(PGroup), cudaMemcpyHostToDevice, s));
  MM_CUDA(launch_win_build(P->groups, P->n_groups, P->block_off_dev, P->lpix, err, P->slot, P->slot_pix, s));
  int32_t herr = 0;
  MM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  if (herr != 0) return fail(MM_ECUDA, "pixel windows: slot tables do not match the counts");
  P->groups_host = std::move(done);
  if (seg) {
    MM_TRY(dalloc(P, &P->seg_ent, (size_t)n_ent));
    MM_TRY(dalloc(P, &P->seg_ang, (size_t)n_ent));
    MM_TRY(dalloc(P, &P->seg_kept, (size_t)n_sub));
    P->n_ent = n_ent;
    P->n_sub_total = n_sub;
    MM_CUDA(launch_seg_build(P->groups, P->n_groups, P->block_off_dev, P->slot, P->ang2, P->seg_sub, P->seg_ent,
                             P->seg_ang, P->seg_kept, s));
  }
  return MM_OK;
}

int build_plan(const mm_problem_desc* d, cudaStream_t us, Plan* P) {
  MM_CUDA(cudaGetDevice(&P->device));
  MM_TRY(tile_kernels_init());
  P->n_det = d->n_det;
  P->n_int = d->n_int;
  P->n_blocks = d->n_det * d->n_int;
  P->n_pix = d->n_pix;
  P->lambda = d->lambda;
  // P->precision: arithmetic of the CG-iteration operators; P->df64: FP64-class ones in df64
  P->precision = (d->precision == MM_FP32 || d->precision == MM_FP32_DF64) ? MM_FP32 : MM_FP64;
  P->algo = (d->toeplitz_algo == MM_TPLZ_DIRECT) ? MM_TPLZ_DIRECT : MM_TPLZ_FFT;
  P->tc = P->precision == MM_FP32 && P->algo == MM_TPLZ_FFT && d->lambda <= kTcMaxJ0 * 32 &&
          (d->toeplitz_algo == MM_TPLZ_GEMM || (d->toeplitz_algo == MM_TPLZ_AUTO && d->lambda <= kTcAutoLambda));
  P->df64 = (d->precision == MM_DF64 || d->precision == MM_FP32_DF64) && P->algo == MM_TPLZ_FFT;
  P->cond_max = d->cond_max > 0 ? d->cond_max : 1e3;
  P->use_seg = d->pt_sub > 0;
  if (d->pt_sub > 0) P->seg_sub = d->pt_sub;
  const int nb = P->n_blocks, lam = P->lambda;
  P->block_off.assign(nb + 1, 0);
  for (int b = 0; b < nb; b++) {
    if (d->block_len[b] < 0) return fail(MM_EINVAL, "negative block length");
    P->block_off[b + 1] = P->block_off[b] + d->block_len[b];
  }
  P->N = P->block_off[nb];
  if (P->N <= 0) return fail(MM_EINVAL, "no samples");
  MM_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
  cudaStream_t s = P->stream;
  // order after the caller's stream (inputs may be produced there)
  cudaEvent_t ev;
  MM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MM_CUDA(cudaEventRecord(ev, us));
  MM_CUDA(cudaStreamWaitEvent(s, ev, 0));
  cudaEventDestroy(ev);

  const cudaMemcpyKind kind = d->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // band rows on the host for checks and de-duplication
  std::vector<double> band((size_t)nb * (lam + 1));
  if (d->inputs_on_device) {
    MM_CUDA(cudaMemcpyAsync(band.data(), d->band, band.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(band.data(), d->band, band.size() * sizeof(double));
  }
  std::vector<double> c0(nb);
  for (int b = 0; b < nb; b++) {
    for (int k = 0; k <= lam; k++)
      if (!std::isfinite(band[(size_t)b * (lam + 1) + k])) return fail(MM_EINVAL, "non-finite band");
    c0[b] = band[(size_t)b * (lam + 1)];
    if (!(c0[b] > 0.0)) return fail(MM_ENOTSPD, "band c_0 must be positive (block " + std::to_string(b) + ")");
  }

  Scratch scr;
  // inputs
  int32_t* pix = nullptr;
  MM_TRY(scr.alloc(&pix, P->N));
  MM_TRY(dalloc(P, &P->psi, P->N));
  MM_CUDA(cudaMemcpyAsync(pix, d->pix, P->N * sizeof(int32_t), kind, s));
  MM_CUDA(cudaMemcpyAsync(P->psi, d->psi, P->N * sizeof(float), kind, s));
  MM_TRY(dalloc(P, &P->block_off_dev, nb + 1));
  MM_TRY(dalloc(P, &P->c0_blk, nb));
  MM_TRY(dalloc(P, &P->band, (size_t)nb * (lam + 1)));
  MM_CUDA(cudaMemcpyAsync(P->block_off_dev, P->block_off.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemcpyAsync(P->c0_blk, c0.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemcpyAsync(P->band, band.data(), band.size() * sizeof(double), cudaMemcpyHostToDevice, s));

  // validation
  int32_t* flag = nullptr;
  MM_TRY(scr.alloc(&flag, 4));
  MM_CUDA(cudaMemsetAsync(flag, 0, 4 * sizeof(int32_t), s));
  MM_CUDA(launch_validate(pix, P->psi, P->N, P->n_pix, flag, s));
  int32_t hflag[4] = {0, 0, 0, 0};
  MM_CUDA(cudaMemcpyAsync(hflag, flag, sizeof(hflag), cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  if (hflag[0] & 1) return fail(MM_EINVAL, "pix values must lie in [-1, n_pix)");
  if (hflag[0] & 2) return fail(MM_EINVAL, "psi has non-finite values");

  // block-Jacobi blocks, excision, compaction
  double* B6 = nullptr;
  double* inv6 = nullptr;
  int32_t *hits = nullptr, *keep = nullptr, *lid = nullptr, *scan_scratch = nullptr;
  const size_t sl = scan_scratch_len(P->n_pix);
  MM_TRY(scr.alloc(&B6, 6 * P->n_pix));
  MM_TRY(scr.alloc(&inv6, 6 * P->n_pix));
  MM_TRY(scr.alloc(&hits, P->n_pix));
  MM_TRY(scr.alloc(&keep, P->n_pix));
  MM_TRY(scr.alloc(&lid, P->n_pix));
  MM_TRY(scr.alloc(&scan_scratch, sl));
  MM_CUDA(cudaMemsetAsync(B6, 0, 6 * P->n_pix * sizeof(double), s));
  MM_CUDA(cudaMemsetAsync(hits, 0, P->n_pix * sizeof(int32_t), s));
  // pointing weights first (one FP64 sincos per sample), then the BD blocks from them
  MM_TRY(dalloc(P, &P->w64, P->N));
  MM_TRY(dalloc(P, &P->w32, P->N));
  if (P->df64) MM_TRY(dalloc(P, &P->wdf, P->N));
  const bool windows = (P->precision == MM_FP32 || P->df64) && P->algo == MM_TPLZ_FFT && !P->no_windows;
  if (windows && P->precision == MM_FP32) MM_TRY(dalloc(P, &P->ang2, P->N));
  MM_CUDA(launch_weights(P->psi, P->N, P->w64, P->w32, P->df64 ? P->wdf : nullptr, P->ang2, s));
  MM_CUDA(launch_bd_accum(pix, P->w64, P->block_off_dev, P->c0_blk, nb, P->N, B6, hits, s));
  MM_CUDA(launch_bd_finalize(B6, hits, P->n_pix, P->cond_max, keep, inv6, s));
  MM_CUDA(launch_scan_keep(keep, P->n_pix, lid, flag + 1, scan_scratch, (int64_t)sl, s));
  MM_CUDA(cudaMemcpyAsync(hflag, flag, sizeof(hflag), cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  P->n_obs = hflag[1];
  if (P->n_obs == 0) return fail(MM_ENOTSPD, "no pixel survives excision");
  MM_TRY(dalloc(P, &P->obs_to_global, P->n_obs));
  MM_TRY(dalloc(P, &P->minv, 6 * P->n_obs));
  MM_TRY(dalloc(P, &P->lpix, P->N));
  MM_CUDA(launch_compact(keep, lid, inv6, P->n_pix, P->obs_to_global, P->minv, s));
  MM_CUDA(launch_localize(pix, keep, lid, P->N, P->lpix, s));
  if (windows) MM_TRY(build_windows(P, s));

  // Toeplitz spectra: L-point circulant spectrum of each distinct band, then the pair tables
  BandTables bt = dedupe_bands(band, nb, lam);
  P->n_tab = (int32_t)bt.tab_src.size();
  std::vector<double> rows((size_t)P->n_tab * (lam + 1));
  for (int t = 0; t < P->n_tab; t++)
    std::memcpy(rows.data() + (size_t)t * (lam + 1), band.data() + (size_t)bt.tab_src[t] * (lam + 1),
                (lam + 1) * sizeof(double));
  std::vector<double> costab(kL);
  for (int i = 0; i < kL; i++) costab[i] = std::cos(2.0 * M_PI * (double)i / (double)kL);
  double *rows_d = nullptr, *costab_d = nullptr, *H = nullptr;
  MM_TRY(scr.alloc(&rows_d, rows.size()));
  MM_TRY(scr.alloc(&costab_d, kL));
  MM_TRY(scr.alloc(&H, (size_t)P->n_tab * (kM + 1)));
  MM_TRY(dalloc(P, &P->tab32, (size_t)P->n_tab * kM));
  MM_TRY(dalloc(P, &P->tab64, (size_t)P->n_tab * kM));
  MM_TRY(dalloc(P, &P->tw32, kM));
  MM_TRY(dalloc(P, &P->tw64, kM));
  MM_CUDA(cudaMemcpyAsync(rows_d, rows.data(), rows.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemcpyAsync(costab_d, costab.data(), kL * sizeof(double), cudaMemcpyHostToDevice, s));
  MM_CUDA(launch_spectra(rows_d, P->n_tab, lam, H, costab_d, s));
  MM_CUDA(launch_pair_tables(H, P->n_tab, costab_d, P->tab64, P->tab32, s));
  MM_CUDA(launch_twiddles(P->tw64, P->tw32, costab_d, s));
  // FP32 N^-1 on 65536-sample tiles (2-CTA clusters) when a 32768-sample tile would keep less than
  // 5/8 of its outputs: tables built here, used when mm_autotune measures them faster
  P->big = P->precision == MM_FP32 && P->algo == MM_TPLZ_FFT && !P->tc && !P->no_windows && !P->no_big &&
           lam > kBigTileLambda;
  if (P->big) {
    const int lb = 2 * kL, mb = 2 * kM;
    std::vector<double> cb(lb);
    for (int i = 0; i < lb; i++) cb[i] = std::cos(2.0 * M_PI * (double)i / (double)lb);
    double *cb_d = nullptr, *Hb = nullptr;
    MM_TRY(scr.alloc(&cb_d, lb));
    MM_TRY(scr.alloc(&Hb, (size_t)P->n_tab * (mb + 1)));
    MM_TRY(dalloc(P, &P->tab32_big, (size_t)P->n_tab * mb));
    MM_TRY(dalloc(P, &P->tw32_big, mb));
    MM_CUDA(cudaMemcpyAsync(cb_d, cb.data(), lb * sizeof(double), cudaMemcpyHostToDevice, s));
    MM_CUDA(launch_spectra(rows_d, P->n_tab, lam, Hb, cb_d, s, kLogM + 1));
    MM_CUDA(launch_pair_table32_big(Hb, P->n_tab, cb_d, P->tab32_big, s));
    MM_CUDA(launch_twiddles(nullptr, P->tw32_big, cb_d, s, kLogM + 1));
    const std::vector<TileDesc> sb = make_tiles(P->block_off, bt, lam, 1, 0, nullptr, lb);
    P->n_segs_big = (int64_t)sb.size();
    MM_TRY(dalloc(P, &P->segs_big, sb.size()));
    MM_CUDA(cudaMemcpyAsync(P->segs_big, sb.data(), sb.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
  }
  if (P->tc) {   // tensor-core Toeplitz product: T_J images, tiles, per-block table and scale
    unsigned char* bm = nullptr;
    MM_TRY(dalloc(P, &bm, tc_bmat_bytes(P->n_tab)));
    P->tc_bmat = bm;
    MM_CUDA(launch_tc_bmat(rows_d, lam, P->n_tab, P->tc_bmat, s));
    const std::vector<TcTile> tt = tc_tiles(P->block_off);
    P->n_tc_tiles = (int64_t)tt.size();
    MM_TRY(dalloc(P, &P->tc_tiles, tt.size()));
    MM_TRY(dalloc(P, &P->tc_tab, nb));
    MM_TRY(dalloc(P, &P->tc_scale, nb));
    MM_TRY(dalloc(P, &P->tc_err, 1));
    std::vector<float> scf(bt.blk_scale.begin(), bt.blk_scale.end());
    MM_CUDA(cudaMemcpyAsync(P->tc_tiles, tt.data(), tt.size() * sizeof(TcTile), cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(P->tc_tab, bt.blk_tab.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(P->tc_scale, scf.data(), nb * sizeof(float), cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemsetAsync(P->tc_err, 0, sizeof(int32_t), s));
    MM_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
  }
  if (P->df64) {
    MM_TRY(dalloc(P, &P->tabdf, (size_t)P->n_tab * kM));
    MM_TRY(dalloc(P, &P->twdf, kM));
    MM_CUDA(launch_c64_to_df(P->tab64, (int64_t)P->n_tab * kM, P->tabdf, s));
    MM_CUDA(launch_c64_to_df(P->tw64, kM, P->twdf, s));
  }
  std::vector<double> Hh((size_t)P->n_tab * (kM + 1));
  MM_CUDA(cudaMemcpyAsync(Hh.data(), H, Hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));

  std::vector<TileDesc> tiles = make_tiles(P->block_off, bt, lam, 1, 0, nullptr);
  P->n_tiles = (int64_t)tiles.size();
  MM_TRY(dalloc(P, &P->tiles, tiles.size()));
  MM_CUDA(cudaMemcpyAsync(P->tiles, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, s));
  P->blk_tab = bt.blk_tab;
  P->blk_scale = bt.blk_scale;
  // FP32 segments: enough of them to keep every SM busy (about 8 per SM), at most 16 tiles each
  const int64_t steps = d->tile_steps > 0 ? d->tile_steps
                                           : std::max<int64_t>(1, std::min<int64_t>(16, P->n_tiles / (8 * sm_count())));
  MM_TRY(build_segments(P, (int)steps, s));
  MM_CUDA(cudaStreamSynchronize(s));

  // the band's symbol sampled on the tile's circulant must be positive (A is then SPD)
  for (int t = 0; t < P->n_tab; t++) {
    double mn = Hh[(size_t)t * (kM + 1)];
    for (int j = 0; j <= kM; j++) mn = std::min(mn, Hh[(size_t)t * (kM + 1) + j]);
    if (!(mn > 0.0))
      return fail(MM_ENOTSPD, "a band's Fourier symbol is not positive (min " + std::to_string(mn) + ")");
  }
  MM_CUDA(cudaGetLastError());
  return MM_OK;
}

// internal map buffers [nrhs][n_obs][4]
int ensure_maps(Plan* P, int nrhs, bool need32) {
  const size_t n4 = (size_t)nrhs * P->n_obs * 4;
  MM_TRY(grow(P, &P->map64_in, &P->map64_in_cap, n4));
  MM_TRY(grow(P, &P->map64_out, &P->map64_out_cap, n4));
  if (need32) {
    MM_TRY(grow32(P, &P->map32_in, &P->map32_in_cap, n4));
    MM_TRY(grow32(P, &P->map32_out, &P->map32_out_cap, n4));
  }
  return MM_OK;
}

int ensure_td(Plan* P) {
  if (P->td_cap >= (size_t)P->N && P->td_a && P->td_b) return MM_OK;
  P->buf_gen++;
  dfree(P->td_a);
  dfree(P->td_b);
  P->td_cap = 0;
  MM_TRY(dalloc(P, &P->td_a, P->N));
  MM_TRY(dalloc(P, &P->td_b, P->N));
  P->td_cap = P->N;
  return MM_OK;
}

TileArgs base_args(const Plan* P, bool fp32) {
  TileArgs a{};
  a.tiles = P->tiles;
  a.n_tiles = P->n_tiles;
  a.nrhs = 1;
  a.N = P->N;
  a.lpix = P->lpix;
  a.w32 = P->w32;
  a.w64 = P->w64;
  a.tab = fp32 ? (const void*)P->tab32 : (const void*)P->tab64;
  a.tw = fp32 ? (const void*)P->tw32 : (const void*)P->tw64;
  a.done = nullptr;
  a.done_stride = 0;
  return a;
}

// df64 path: samples per right-hand side of the un-pointed buffer (N rounded up to 4, so every
// column starts 16-byte aligned), and how many columns one pass of it holds
int64_t df_stride(const Plan* P) { return (P->N + 3) / 4 * 4; }
int df_cols(const Plan* P, int nrhs) {
  const int64_t per = df_stride(P) * (int64_t)sizeof(float2) * (P->groups && !P->tmpl ? 2 : 1);
  const int64_t k = std::max<int64_t>(1, (int64_t)kSplitTBytes / per);
  return (int)std::min<int64_t>(nrhs, k);
}

// df64 TOD buffer for ncols columns and df64 maps for ncols columns (allocated outside graph capture)
int ensure_tdf(Plan* P, int ncols) {
  const size_t t_elems = (size_t)ncols * (size_t)df_stride(P);
  if (P->tdf_cap < t_elems) {
    P->buf_gen++;
    dfree(P->tdf);
    P->tdf_cap = 0;
    MM_TRY(dalloc(P, &P->tdf, t_elems));
    P->tdf_cap = t_elems;
  }
  return MM_OK;
}
int ensure_mapdf(Plan* P, int ncols) {
  const size_t m_elems = (size_t)ncols * (size_t)P->n_obs * 2;
  if (P->mapdf_cap < m_elems) {
    P->buf_gen++;
    dfree(P->mapdf);
    P->mapdf_cap = 0;
    MM_TRY(dalloc(P, &P->mapdf, m_elems));
    P->mapdf_cap = m_elems;
  }
  return MM_OK;
}
// N^-1 t of the windowed df64 operator and the per-column max |u| (allocated outside graph capture)
int ensure_udf(Plan* P, int ncols) {
  const size_t t_elems = (size_t)ncols * (size_t)df_stride(P);
  if (P->udf_cap < t_elems) {
    P->buf_gen++;
    dfree(P->udf);
    P->udf_cap = 0;
    MM_TRY(dalloc(P, &P->udf, t_elems));
    P->udf_cap = t_elems;
  }
  if (P->amax_cap < (size_t)ncols) {
    P->buf_gen++;
    dfree(P->amax);
    P->amax_cap = 0;
    MM_TRY(dalloc(P, &P->amax, (size_t)ncols));
    P->amax_cap = (size_t)ncols;
  }
  return MM_OK;
}

// df64 working buffers of the df64 Toeplitz operator for nrhs columns
int ensure_df(Plan* P, int nrhs) {
  if (P->tmpl) return ensure_mapdf(P, nrhs);
  if (!P->df64) return MM_OK;
  MM_TRY(ensure_tdf(P, df_cols(P, nrhs)));
  if (P->groups) MM_TRY(ensure_udf(P, df_cols(P, nrhs)));
  return ensure_mapdf(P, df_cols(P, nrhs));
}

bool df_ready(const Plan* P, int nrhs) {
  const int k = df_cols(P, nrhs);
  return P->tdf_cap >= (size_t)k * df_stride(P) && P->mapdf_cap >= (size_t)k * P->n_obs * 2 &&
         (!P->groups || (P->udf_cap >= (size_t)k * df_stride(P) && P->amax_cap >= (size_t)k));
}

TileArgs df_args(const Plan* P) {
  TileArgs a = base_args(P, false);
  a.wdf = P->wdf;
  a.tab = P->tabdf;
  a.tw = P->twdf;
  a.x_stride = df_stride(P);
  a.y_stride = P->n_obs * 4;
  return a;
}

// y4 (FP64 map [g][n_obs][4], accumulated) += P^T N^-1 of the g df64 columns in P->tdf: with pixel
// windows, u = N^-1 t into P->udf, then P^T over the windows; otherwise the tiles scatter P^T
int df_ninv_point(Plan* P, int g, const int32_t* done, int done_stride, double* y4, cudaStream_t s) {
  TileArgs a = df_args(P);
  a.nrhs = g;
  a.x = P->tdf;
  a.done = done;
  a.done_stride = done_stride;
  if (!P->groups) {
    a.y = y4;
    MM_CUDA(launch_tiles_df(a, s));
    return MM_OK;
  }
  MM_CUDA(cudaMemsetAsync(P->amax, 0, (size_t)g * sizeof(uint32_t), s));
  a.y = P->udf;
  a.y_stride = df_stride(P);
  a.amax = P->amax;
  MM_CUDA(launch_ninv_df(a, s));
  MM_CUDA(launch_point_win_df(P->groups, P->n_groups, P->block_off_dev, P->slot, P->slot_pix, P->wdf, P->udf,
                              df_stride(P), P->amax, g, done, done_stride, y4, P->n_obs * 4, s));
  return MM_OK;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// TOD of a solve that evaluates its residuals from the data: d [nrhs][N] device, float32 or float64
struct TodSrc {
  const void* d;
  int d_is_fp32;
};

// y4 (accumulated, pre-zeroed by the caller) += A x4 with the FP64-class operators, [nrhs][n_obs][4].
// With tod (double-float plans with pixel windows): y4 += P^T N^-1 (P x - G d) = A x - b instead.
int apply64_internal(Plan* P, const double* x4, double* y4, int nrhs, cudaStream_t s,
                     const int32_t* done = nullptr, int done_stride = 0, const TodSrc* tod = nullptr) {
  if (P->tmpl) {   // template map-making: P^T F_T P in one fused df64 kernel, from the df64 map
    const TmplState* ts = reinterpret_cast<const TmplState*>(P->tmpl);
    const size_t m_elems = (size_t)nrhs * P->n_obs * 2;
    if (capturing(s) && P->mapdf_cap < m_elems) return fail(MM_EINVAL, "df64 buffers must be allocated before graph capture");
    MM_TRY(ensure_mapdf(P, nrhs));
    MM_CUDA(launch_map_to_df(x4, (int64_t)nrhs * P->n_obs, P->mapdf, s));
    MM_CUDA(launch_tmpl_mx64(ts->M64, P->n_obs, x4, y4, nrhs, done, done_stride, s));
    MM_CUDA(launch_tmpl_apply_df(ts->dev, P->n_blocks, P->wdf, P->mapdf, P->n_obs * 2, nullptr, 0, y4, P->n_obs * 4,
                                 nrhs, done, done_stride, s));
    return MM_OK;
  }
  if (P->df64) {
    const int k = df_cols(P, nrhs);
    if (capturing(s) && !df_ready(P, nrhs))
      return fail(MM_EINVAL, "df64 buffers must be allocated before graph capture");
    MM_TRY(ensure_df(P, nrhs));
    for (int r0 = 0; r0 < nrhs; r0 += k) {
      const int g = std::min(k, nrhs - r0);
      const int32_t* dn = done ? done + (int64_t)r0 * done_stride : nullptr;
      MM_CUDA(launch_map_to_df(x4 + (size_t)r0 * P->n_obs * 4, (int64_t)g * P->n_obs, P->mapdf, s));
      // t = P x, or with the TOD t = P x - G d (the time-domain residual: N^-1 and P^T of it give
      // A x - b) in one pass
      const size_t esz = (tod && tod->d_is_fp32) ? sizeof(float) : sizeof(double);
      MM_CUDA(launch_unpoint_df(P->lpix, P->wdf, P->N, P->mapdf, P->n_obs, g, dn, done_stride, P->tdf,
                                df_stride(P), s,
                                tod ? reinterpret_cast<const char*>(tod->d) + (size_t)r0 * P->N * esz : nullptr,
                                tod ? tod->d_is_fp32 : 0));
      MM_TRY(df_ninv_point(P, g, dn, done_stride, y4 + (size_t)r0 * P->n_obs * 4, s));
    }
    return MM_OK;
  }
  if (P->algo == MM_TPLZ_DIRECT) {
    MM_TRY(ensure_td(P));
    for (int r = 0; r < nrhs; r++) {
      MM_CUDA(launch_unpoint64(P->lpix, P->w64, P->N, x4 + (size_t)r * P->n_obs * 4, P->td_a, s));
      MM_CUDA(launch_toeplitz_direct(P->band, P->block_off_dev, P->n_blocks, P->lambda, P->N,
                                     P->td_a, P->td_b, s));
      MM_CUDA(launch_point64(P->lpix, P->w64, P->N, P->td_b, y4 + (size_t)r * P->n_obs * 4, s));
    }
    return MM_OK;
  }
  TileArgs a = base_args(P, false);
  a.nrhs = nrhs;
  a.x = x4;
  a.x_stride = P->n_obs * 4;
  a.y = y4;
  a.y_stride = P->n_obs * 4;
  a.done = done;
  a.done_stride = done_stride;
  MM_CUDA(launch_tiles_fp64(MODE_APPLY, a, s));
  return MM_OK;
}

// plan-owned un-pointed buffer of the split FP32 A-application (allocated outside graph capture)
int64_t t32_stride(const Plan* P) { return (P->N + 3) / 4 * 4; }

// u = N^-1 t for g FP32 columns (t, u [g][ts]): tensor-core GEMM tiles on MM_TPLZ_GEMM plans,
// overlap-save FFT segments otherwise
int ninv32(Plan* P, const float* t, float* u, int64_t ts, int g, const int32_t* done, int done_stride,
           cudaStream_t s) {
  if (P->tc) {
    MM_CUDA(launch_tplz_tc(P->tc_tiles, P->n_tc_tiles, P->block_off_dev, P->tc_tab, P->tc_scale, P->tc_bmat,
                           P->lambda, t, ts, u, ts, g, done, done_stride, P->tc_err, s));
    return MM_OK;
  }
  TileArgs a = base_args(P, true);
  if (P->big && P->use_big) {
    a.tiles = P->segs_big;
    a.n_tiles = P->n_segs_big;
    a.tab = P->tab32_big;
    a.tw = P->tw32_big;
    a.nrhs = g;
    a.x = t;
    a.x_stride = ts;
    a.y = u;
    a.y_stride = ts;
    a.done = done;
    a.done_stride = done_stride;
    MM_CUDA(launch_ninv32_big(a, s));
    return MM_OK;
  }
  a.tiles = P->segs;
  a.n_tiles = P->n_segs;
  a.nrhs = g;
  a.x = t;
  a.x_stride = ts;
  a.y = u;
  a.y_stride = ts;
  a.done = done;
  a.done_stride = done_stride;
  MM_CUDA(launch_tiles_fp32(MODE_NINV_T, a, P->seg_halo, s));
  return MM_OK;
}

// The split FP32 A-application keeps t = P x (and, with pixel windows, u = N^-1 t) for the
// columns of one pass; a pass holds as many columns as fit in kSplitTBytes (at least one), and
// more columns run in several passes.  Only when a single column does not fit do the fused tiles
// run instead.
int split32_cols(const Plan* P, int nrhs) {
  const size_t per = (size_t)t32_stride(P) * sizeof(float) * (P->groups ? 2 : 1);
  return (int)std::min<size_t>((size_t)nrhs, kSplitTBytes / per);
}

int ensure_t32(Plan* P, int nrhs) {
  const int k = split32_cols(P, nrhs);
  if (k == 0) return MM_OK;
  const size_t t_elems = (size_t)k * (size_t)t32_stride(P);
  if (P->t32_cap < t_elems) {
    dfree(P->t32);
    P->t32_cap = 0;
    P->buf_gen++;
    MM_TRY(dalloc(P, &P->t32, t_elems));
    P->t32_cap = t_elems;
  }
  if (P->groups && P->u32_cap < t_elems) {
    dfree(P->u32);
    P->u32_cap = 0;
    P->buf_gen++;
    MM_TRY(dalloc(P, &P->u32, t_elems));
    P->u32_cap = t_elems;
  }
  return MM_OK;
}

// y4 += P^T u (FP32) of a plan with pixel windows: segment reduction over the pixel-sorted
// sub-windows, or per-sample shared-memory sums over the windows
cudaError_t point32(Plan* P, const float* u, int64_t u_stride, int nrhs, const int32_t* done, int done_stride,
                    float* y4, int64_t y_stride, cudaStream_t s) {
  if (P->use_seg && P->seg_ent)
    return launch_point_seg32(P->groups, P->n_groups, P->block_off_dev, P->seg_ent, P->seg_ang, P->seg_kept,
                              P->slot_pix, P->seg_sub, u, u_stride, nrhs, done, done_stride, y4, y_stride, s);
  return launch_point_win32(P->groups, P->n_groups, P->block_off_dev, P->slot, P->slot_pix, P->ang2, u, u_stride,
                            nrhs, done, done_stride, y4, y_stride, s);
}

// y32 (accumulated, pre-zeroed) += A x32 in FP32, [nrhs][n_obs][4] float.  Profiling events: mid
// after P (t = P x), mid2 after N^-1 (pixel windows only).
int apply32_internal(Plan* P, const float* x32, float* y32, int nrhs, cudaStream_t s,
                     const int32_t* done = nullptr, int done_stride = 0, cudaEvent_t mid = nullptr,
                     cudaEvent_t mid2 = nullptr) {
  TileArgs a = base_args(P, true);
  a.tiles = P->segs;
  a.n_tiles = P->n_segs;
  a.nrhs = nrhs;
  a.y = y32;
  a.y_stride = P->n_obs * 4;
  a.done = done;
  a.done_stride = done_stride;
  if (P->tmpl) {   // template map-making: y += P^T F_T P x in one fused kernel (FP32), no TOD buffer
    const TmplState* ts = reinterpret_cast<const TmplState*>(P->tmpl);
    if (mid) MM_CUDA(cudaEventRecord(mid, s));
    MM_CUDA(launch_tmpl_mx32(ts->M32, P->n_obs, x32, y32, nrhs, done, done_stride, s));
    MM_CUDA(launch_tmpl_apply32(ts->dev, P->n_blocks, P->w32, x32, P->n_obs * 4, y32, P->n_obs * 4, nrhs, done,
                                done_stride, s));
    if (mid2) MM_CUDA(cudaEventRecord(mid2, s));
    return MM_OK;
  }
  const int kc = split32_cols(P, nrhs);
  if (kc > 0 && P->groups) {
    if (capturing(s) && P->u32_cap < (size_t)kc * t32_stride(P))
      return fail(MM_EINVAL, "FP32 buffers must be allocated before graph capture");
    MM_TRY(ensure_t32(P, nrhs));
    const int64_t ts = t32_stride(P);
    const int64_t ms = P->n_obs * 4;
    // P over the pixel windows, u = N^-1 t on the segments, P^T over the windows; kc columns per
    // pass (the window kernels read a group's pointing once per pass and reuse it from L2 for
    // every column of the pass)
    for (int r0 = 0; r0 < nrhs; r0 += kc) {
      const int g = std::min(kc, nrhs - r0);
      const int32_t* dn = done ? done + (int64_t)r0 * done_stride : nullptr;
      MM_CUDA(launch_unpoint_win32(P->groups, P->n_groups, P->block_off_dev, P->slot, P->slot_pix, P->ang2,
                                   x32 + (size_t)r0 * ms, ms, g, dn, done_stride, P->t32, ts, s));
      if (mid && r0 == 0) MM_CUDA(cudaEventRecord(mid, s));
      MM_TRY(ninv32(P, P->t32, P->u32, ts, g, dn, done_stride, s));
      if (mid2 && r0 + kc >= nrhs) MM_CUDA(cudaEventRecord(mid2, s));
      MM_CUDA(point32(P, P->u32, ts, g, dn, done_stride, y32 + (size_t)r0 * ms, ms, s));
    }
    return MM_OK;
  }
  if (kc >= nrhs) {
    MM_TRY(ensure_t32(P, nrhs));
    const int64_t ts = t32_stride(P);
    // un-point first at full occupancy, then the tiles stream t and scatter P^T themselves
    MM_CUDA(launch_unpoint32(P->lpix, P->w32, P->N, x32, P->n_obs * 4, nrhs, done, done_stride, P->t32, ts, s));
    if (mid) MM_CUDA(cudaEventRecord(mid, s));
    a.x = P->t32;
    a.x_stride = ts;
    MM_CUDA(launch_tiles_fp32(MODE_APPLY_T, a, P->seg_halo, s));
    if (mid2) MM_CUDA(cudaEventRecord(mid2, s));
  } else {
    if (mid) MM_CUDA(cudaEventRecord(mid, s));
    a.x = x32;
    a.x_stride = P->n_obs * 4;
    MM_CUDA(launch_tiles_fp32(MODE_APPLY, a, P->seg_halo, s));
    if (mid2) MM_CUDA(cudaEventRecord(mid2, s));
  }
  return MM_OK;
}

// b4 [nrhs][n_obs][4] (FP64) = P^T N^-1 G d with the FP32 operators over the pixel windows (the
// start of a solve whose true residuals come from the TOD); needs an FP32 plan with windows
int rhs32_internal(Plan* P, const void* d, int d_is_fp32, int nrhs, double* b4, cudaStream_t s) {
  MM_TRY(ensure_maps(P, nrhs, true));
  MM_TRY(ensure_t32(P, nrhs));
  const int kc = split32_cols(P, nrhs);
  if (kc == 0 || !P->groups) return fail(MM_EINVAL, "the FP32 right-hand side needs pixel windows");
  const int64_t ts = t32_stride(P), ms = P->n_obs * 4;
  const size_t esz = d_is_fp32 ? sizeof(float) : sizeof(double);
  MM_CUDA(cudaMemsetAsync(P->map32_out, 0, (size_t)nrhs * ms * sizeof(float), s));
  for (int r0 = 0; r0 < nrhs; r0 += kc) {
    const int g = std::min(kc, nrhs - r0);
    MM_CUDA(launch_d_to_t32(P->lpix, reinterpret_cast<const char*>(d) + (size_t)r0 * P->N * esz, d_is_fp32, P->N, g,
                            P->t32, ts, s));
    MM_TRY(ninv32(P, P->t32, P->u32, ts, g, nullptr, 0, s));
    MM_CUDA(point32(P, P->u32, ts, g, nullptr, 0, P->map32_out + (size_t)r0 * ms, ms, s));
  }
  MM_CUDA(launch_to64(P->map32_out, (int64_t)nrhs * P->n_obs, b4, s));
  return MM_OK;
}

// CG state for nrhs columns; its reduction counters are zeroed on stream s, the stream of the CG
// kernels that first use them (a memset on the legacy default stream is not ordered before work
// on the non-blocking streams of the server's planner threads)
int ensure_cg(Plan* P, int nrhs, bool fp32, CgState** out, cudaStream_t s) {
  CgState* c = reinterpret_cast<CgState*>(P->cg);
  if (!c) {
    c = new CgState();
    P->cg = c;
  }
  if (c->nrhs_cap < nrhs || c->n != P->n_obs) {
    if (c->exec) {
      cudaGraphExecDestroy(c->exec);
      c->exec = nullptr;
    }
    dfree(c->b); dfree(c->x); dfree(c->r); dfree(c->z); dfree(c->p); dfree(c->q);
    dfree(c->p32); dfree(c->q32); dfree(c->partials); dfree(c->counters); dfree(c->scal);
    if (c->scal_host) { cudaFreeHost(c->scal_host); c->scal_host = nullptr; }
    const size_t n4 = (size_t)nrhs * P->n_obs * 4;
    MM_TRY(dalloc(P, &c->b, n4)); MM_TRY(dalloc(P, &c->x, n4)); MM_TRY(dalloc(P, &c->r, n4));
    MM_TRY(dalloc(P, &c->z, n4)); MM_TRY(dalloc(P, &c->p, n4)); MM_TRY(dalloc(P, &c->q, n4));
    MM_TRY(dalloc(P, &c->p32, n4)); MM_TRY(dalloc(P, &c->q32, n4));
    MM_TRY(dalloc(P, &c->partials, (size_t)nrhs * 1024 * 4));
    MM_TRY(dalloc(P, &c->counters, nrhs));
    MM_TRY(dalloc(P, &c->scal, nrhs));
    MM_CUDA(cudaMemsetAsync(c->counters, 0, nrhs * sizeof(unsigned), s));
    MM_CUDA(cudaMallocHost((void**)&c->scal_host, nrhs * sizeof(CgScalars)));
    c->nrhs_cap = nrhs;
    c->n = P->n_obs;
  }
  (void)fp32;
  *out = c;
  return MM_OK;
}

CgWork make_work(Plan* P, CgState* c, int nrhs, bool fp32, double tol, int max_iter) {
  CgWork w{};
  w.n = P->n_obs;
  w.nrhs = nrhs;
  w.n_blocks = cg_blocks_for(P->n_obs);
  w.fp32 = fp32 ? 1 : 0;
  w.tol2 = tol * tol;
  w.max_iter = max_iter;
  w.minv = P->minv;
  w.b = c->b; w.x = c->x; w.r = c->r; w.z = c->z; w.p = c->p; w.q = c->q;
  w.p32 = c->p32; w.q32 = c->q32;
  w.partials = c->partials;
  w.counters = c->counters;
  w.scal = c->scal;
  return w;
}

// One PCG iteration: p = z + beta p; q = A p; alpha; x, r, z, beta (z = M_2lvl r when dw != null).
int enqueue_iteration(Plan* P, const CgWork& w, int nrhs, bool fp32, cudaStream_t s,
                      const DeflWork* dw = nullptr) {
  MM_CUDA(launch_cg(CG_PUPDATE, w, s));
  const int32_t* halt = reinterpret_cast<const int32_t*>(w.scal) + kHaltOffsetInts;
  if (fp32) {
    MM_TRY(apply32_internal(P, w.p32, w.q32, nrhs, s, halt, kScalStrideInts));
  } else {
    MM_TRY(apply64_internal(P, w.p, w.q, nrhs, s, halt, kScalStrideInts));
  }
  MM_CUDA(launch_cg(CG_DOT_PQ, w, s));
  MM_CUDA(launch_cg(CG_UPDATE, w, s));
  if (dw) MM_CUDA(launch_defl_step(*dw, w, s));
  return MM_OK;
}

// per-solve buffers of the deflated preconditioner for nrhs columns
int ensure_defl_work(Plan* P, DeflState* d, int nrhs, int n_blocks, DeflWork* out, cudaStream_t s) {
  if (d->nrhs_cap < nrhs) {
    P->buf_gen++;
    dfree(d->y); dfree(d->part); dfree(d->part2); dfree(d->counters); dfree(d->counters2);
    d->nrhs_cap = 0;
    MM_TRY(dalloc(P, &d->y, (size_t)nrhs * kMaxDefl));
    MM_TRY(dalloc(P, &d->part, (size_t)nrhs * 1024 * kMaxDefl));
    MM_TRY(dalloc(P, &d->part2, (size_t)nrhs * 1024));
    MM_TRY(dalloc(P, &d->counters, nrhs));
    MM_TRY(dalloc(P, &d->counters2, nrhs));
    MM_CUDA(cudaMemsetAsync(d->counters, 0, nrhs * sizeof(unsigned), s));
    MM_CUDA(cudaMemsetAsync(d->counters2, 0, nrhs * sizeof(unsigned), s));
    d->nrhs_cap = nrhs;
  }
  (void)n_blocks;
  out->k = d->k;
  out->Z = d->Z;
  out->Zp = d->Zp;
  out->Einv = d->Einv;
  out->y = d->y;
  out->part = d->part;
  out->part2 = d->part2;
  out->counters = d->counters;
  out->counters2 = d->counters2;
  return MM_OK;
}

// CTAs (and partial sums) of the block reductions: two per SM
int blk_ctas() { return 2 * sm_count(); }

int ensure_blk(Plan* P, int s, BlkState** out) {
  BlkState* b = reinterpret_cast<BlkState*>(P->blk);
  if (!b) {
    b = new BlkState();
    P->blk = b;
  }
  if (b->s_cap < s || b->n != P->n_obs) {
    BlkState fresh;
    std::swap(*b, fresh);
    free_blk(new BlkState(fresh));   // releases the old buffers
    const size_t n4 = (size_t)s * P->n_obs * 4;
    MM_TRY(dalloc(P, &b->X, n4)); MM_TRY(dalloc(P, &b->R, n4)); MM_TRY(dalloc(P, &b->B, n4));
    MM_TRY(dalloc(P, &b->AX, n4)); MM_TRY(dalloc(P, &b->T64, n4));
    MM_TRY(dalloc(P, &b->Z, n4)); MM_TRY(dalloc(P, &b->AZ, n4)); MM_TRY(dalloc(P, &b->P, n4));
    MM_TRY(dalloc(P, &b->AP, n4));
    MM_TRY(dalloc(P, &b->part, (size_t)blk_ctas() * kMaxBlk * kMaxBlk));
    MM_TRY(dalloc(P, &b->G, kMaxBlk * kMaxBlk)); MM_TRY(dalloc(P, &b->Linv, kMaxBlk * kMaxBlk));
    MM_TRY(dalloc(P, &b->Cmb, kMaxBlk * kMaxBlk)); MM_TRY(dalloc(P, &b->alpha, kMaxBlk * kMaxBlk));
    MM_TRY(dalloc(P, &b->C2, kMaxBlk * kMaxBlk)); MM_TRY(dalloc(P, &b->norms, kMaxBlk));
    MM_TRY(dalloc(P, &b->norm_part, (size_t)kMaxBlk * blk_ctas()));
    MM_TRY(dalloc(P, &b->piv, kMaxBlk)); MM_TRY(dalloc(P, &b->rank, 4)); MM_TRY(dalloc(P, &b->idx, kMaxBlk));
    MM_CUDA(cudaMallocHost((void**)&b->host, kMaxBlk * sizeof(double)));
    MM_CUDA(cudaMallocHost((void**)&b->host_i, 4 * sizeof(int)));
    b->s_cap = s;
    b->n = P->n_obs;
  }
  *out = b;
  return MM_OK;
}

// enlarged-CG buffers on top of a block state of s_cap columns
int ensure_ecg(Plan* P, BlkState* b) {
  if (b->Pp && b->APp && b->xe && b->re && b->ax) return MM_OK;
  const size_t n4 = (size_t)b->s_cap * P->n_obs * 4;
  MM_TRY(dalloc(P, &b->Pp, n4)); MM_TRY(dalloc(P, &b->APp, n4));
  MM_TRY(dalloc(P, &b->xe, (size_t)P->n_obs * 4)); MM_TRY(dalloc(P, &b->re, (size_t)P->n_obs * 4));
  MM_TRY(dalloc(P, &b->ax, (size_t)P->n_obs * 4));
  return MM_OK;
}

// A Z for t FP32 columns (AZ zeroed and accumulated), with the plan's FP32 or FP64 operator.
int blk_apply(Plan* P, BlkState* b, int t, bool fp32, cudaStream_t s) {
  const size_t n4 = (size_t)t * P->n_obs * 4;
  if (fp32) {
    MM_CUDA(cudaMemsetAsync(b->AZ, 0, n4 * sizeof(float), s));
    return apply32_internal(P, b->Z, b->AZ, t, s);
  }
  MM_CUDA(launch_to64(b->Z, (int64_t)(n4 / 4), b->AX, s));
  MM_CUDA(cudaMemsetAsync(b->T64, 0, n4 * sizeof(double), s));
  MM_TRY(apply64_internal(P, b->AX, b->T64, t, s));
  MM_CUDA(launch_to32(b->T64, (int64_t)(n4 / 4), b->AZ, s));
  return MM_OK;
}


// ---------------------------------------------------------------------------------------------
// serving: continuous batching of PCG solves
// ---------------------------------------------------------------------------------------------
using Clock = std::chrono::steady_clock;

// Copy n bytes with up to 8 threads.  mm_submit copies a request's pointing and TOD (16 bytes per
// sample with an FP64 TOD: hundreds of MB) before it returns; one thread copying into fresh pages
// (each first touch a page fault) takes tens of ms per request and would bound the rate at which
// a client can submit.
void par_copy(void* dst, const void* src, size_t n) {
  constexpr size_t kChunk = (size_t)32 << 20;
  const int nt = (int)std::min<size_t>(8, (n + kChunk - 1) / kChunk);
  if (nt <= 1) {
    if (n) std::memcpy(dst, src, n);
    return;
  }
  const size_t per = (n + nt - 1) / nt;
  std::vector<std::thread> th;
  for (int i = 1; i < nt; i++) {
    const size_t lo = (size_t)i * per, hi = std::min(n, lo + per);
    if (lo < hi)
      th.emplace_back([=] { std::memcpy((char*)dst + lo, (const char*)src + lo, hi - lo); });
  }
  std::memcpy(dst, src, std::min(per, n));
  for (std::thread& t : th) t.join();
}

// Owning host array whose elements are left uninitialised until par_copy writes them (a
// std::vector would first zero-fill every page on the calling thread).
template <typename T>
struct HostArray {
  std::unique_ptr<T[]> p;
  size_t n = 0;
  void copy_from(const T* src, size_t count) {
    p.reset(count ? new T[count] : nullptr);
    n = count;
    par_copy(p.get(), src, count * sizeof(T));
  }
  T* data() { return p.get(); }
  size_t size() const { return n; }
  void release() {
    p.reset();
    n = 0;
  }
};

struct Request {
  mm_req_t id = 0;
  mm_problem_desc desc{};
  std::vector<int64_t> block_len;
  HostArray<int32_t> pix;
  HostArray<float> psi;
  std::vector<double> band;
  HostArray<unsigned char> d;     // the TOD, float64 or float32 (d_is_fp32)
  int d_is_fp32 = 0;
  bool fp32 = true;               // FP32 iterations (batched) or FP64-class iterations (own launches)
  mm_solve_opts opts{};
  size_t footprint = 0;
  int state = 0;                  // 0 queued, 1 running, 2 finished
  Plan* plan = nullptr;
  CgState* cg = nullptr;
  CgWork w{};
  double* d_dev = nullptr;
  double* b_dev = nullptr;
  CgScalars* scal_host = nullptr; // pinned
  std::vector<double> map;        // [n_pix][3]
  mm_solve_info info{};
  int batch = 1;
  int launched = 0;
  Clock::time_point t_submit, t_admit;
};

struct Server {
  size_t budget = 0;
  int max_slots = 1;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_plan;
  std::deque<Request*> queue;
  std::vector<Request*> running;   // touched by the server thread only
  // planner threads build admitted requests' plans, right-hand sides and CG state on their own
  // streams while the server thread iterates the running ones (under mu: ready, planning, n_running)
  std::vector<std::thread> planners;
  std::vector<Request*> ready;     // planned, joining the running set at the next step
  int planning = 0;                // requests being planned
  int n_running = 0;               // running.size() as the planners see it
  std::unordered_map<mm_req_t, Request*> all;
  size_t used = 0;
  bool stop = false;
  mm_req_t next_id = 1;
  std::thread th;
  // one server step's launches: requests with pixel windows run P, N^-1 and P^T over all their
  // groups and segments in three launches (wgroups / wprobs, ntiles / nprobs); requests whose plan
  // has no windows run the fused tiles (un-pointing in the gather, per-sample scatter) in one
  TileDesc* tiles_dev = nullptr;
  size_t tiles_cap = 0;
  ProbPtrs* probs_dev = nullptr;
  size_t probs_cap = 0;
  int64_t n_tiles = 0;
  int halo = 0;
  PGroup* wgroups_dev = nullptr;
  size_t wgroups_cap = 0;
  int64_t n_wgroups = 0;
  WinProb* wprobs_dev = nullptr;
  size_t wprobs_cap = 0;
  TileDesc* ntiles_dev = nullptr;
  size_t ntiles_cap = 0;
  int64_t n_ntiles = 0;
  ProbPtrs* nprobs_dev = nullptr;
  size_t nprobs_cap = 0;
  int nhalo = 0;
  const float2* tw32 = nullptr;    // twiddles of a running request's plan (the same in every plan)
  bool dirty = true;
};

size_t estimate_footprint(const Request& r) {
  int64_t N = 0;
  for (int64_t v : r.block_len) N += v;
  // pointing (pixel, angle, reduced angle, window slot), FP32, FP64 and df64 weights, un-pointed
  // FP32 and df64 buffers, N^-1 t in FP32 and df64 and the TOD: 100 bytes per sample
  return (size_t)N * 100 + (size_t)r.desc.n_pix * 480 + ((size_t)64 << 20);
}

void finish_request(Server* S, Request* r, int status) {
  if (r->plan) {
    free_plan(r->plan);
    r->plan = nullptr;
  }
  if (r->d_dev) cudaFree(r->d_dev);
  if (r->b_dev) cudaFree(r->b_dev);
  r->d_dev = r->b_dev = nullptr;
  if (r->scal_host) cudaFreeHost(r->scal_host);
  r->scal_host = nullptr;
  r->info.status = status;
  r->info.batch = r->batch;
  std::lock_guard<std::mutex> lock(S->mu);
  r->state = 2;
  S->used -= std::min(S->used, r->footprint);
  r->pix.release();
  r->psi.release();
  r->d.release();
  S->cv_done.notify_all();
  S->cv_plan.notify_all();   // memory and a slot are free for the next plan
}

// plan + right-hand side + PCG initialisation of an admitted request.  FP32 requests get an
// MM_FP32_DF64 plan (FP32 iterations, double-float right-hand side and replacements); FP64-class
// requests keep the plan precision they asked for, whose FP64-class operator (IEEE FP64 for
// MM_FP64 / MM_FP32, double-float for MM_DF64 / MM_FP32_DF64) runs in every iteration.
int start_request(Server* S, Request* r, cudaStream_t ps) {
  r->desc.block_len = r->block_len.data();
  r->desc.pix = r->pix.data();
  r->desc.psi = r->psi.data();
  r->desc.band = r->band.data();
  r->desc.inputs_on_device = 0;
  if (r->fp32) r->desc.precision = MM_FP32_DF64;
  r->desc.toeplitz_algo = MM_TPLZ_FFT;   // the multi-problem launches run the FFT tiles
  r->plan = new Plan();
  r->plan->no_windows = !r->fp32;        // FP64-class requests never run the FP32 operators
  r->plan->no_big = true;
  int st = build_plan(&r->desc, ps, r->plan);
  if (st != MM_OK) return st;
  Plan* P = r->plan;
  if (r->fp32 && P->groups) MM_TRY(ensure_t32(P, 1));   // t = P x and u = N^-1 t of the window path
  const size_t esz = r->d_is_fp32 ? sizeof(float) : sizeof(double);
  MM_CUDA(cudaMalloc((void**)&r->d_dev, P->N * esz));
  MM_CUDA(cudaMalloc((void**)&r->b_dev, P->n_obs * 3 * sizeof(double)));
  MM_CUDA(cudaMemcpyAsync(r->d_dev, r->d.data(), P->N * esz, cudaMemcpyHostToDevice, ps));
  st = mm_rhs(reinterpret_cast<mm_plan_t>(P), r->d_dev, r->d_is_fp32, 1, r->b_dev, ps);
  if (st != MM_OK) return st;
  MM_TRY(ensure_cg(P, 1, r->fp32, &r->cg, ps));
  if (!r->fp32) MM_TRY(ensure_df(P, 1));
  r->w = make_work(P, r->cg, 1, r->fp32, r->opts.tol, r->opts.max_iter);
  MM_CUDA(cudaMallocHost((void**)&r->scal_host, sizeof(CgScalars)));
  MM_CUDA(launch_pack3to4(r->b_dev, P->n_obs, 1, r->cg->b, ps));
  MM_CUDA(launch_cg(CG_INIT, r->w, ps));
  MM_CUDA(cudaStreamSynchronize(ps));   // the server thread uses the state on its own stream
  r->t_admit = Clock::now();
  return MM_OK;
}

// Planner thread: takes queued requests while slots and the HBM budget allow (counting the ones
// being planned, planned and running; a request is always taken when none is active), builds
// each on its own stream and hands it to the server thread.
void planner_loop(Server* S) {
  cudaSetDevice(S->device);
  cudaStream_t ps = nullptr;
  if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess) ps = nullptr;
  while (true) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      auto admissible = [&] {
        if (S->queue.empty()) return false;
        const int active = S->n_running + S->planning + (int)S->ready.size();
        if (active >= S->max_slots) return false;
        return active == 0 || S->used + S->queue.front()->footprint <= S->budget;
      };
      S->cv_plan.wait(lock, [&] { return S->stop || admissible(); });
      if (S->stop) break;
      r = S->queue.front();
      S->queue.pop_front();
      S->used += r->footprint;
      S->planning += 1;
      r->state = 1;
    }
    const int st = ps ? start_request(S, r, ps) : cuda_fail(cudaErrorInvalidResourceHandle, "planner stream");
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->planning -= 1;
      if (st == MM_OK) S->ready.push_back(r);
    }
    if (st != MM_OK) finish_request(S, r, st);
    S->cv_work.notify_all();
    S->cv_plan.notify_all();
  }
  if (ps) cudaStreamDestroy(ps);
}

// grow (after the stream's work that reads it) and fill one device list of a server step
template <typename T>
static int upload_list(const std::vector<T>& v, T*& dev, size_t& cap, cudaStream_t s) {
  if (v.size() > cap) {
    MM_CUDA(cudaStreamSynchronize(s));
    if (dev) cudaFree(dev);
    dev = nullptr;
    cap = 0;
    MM_CUDA(cudaMalloc((void**)&dev, (v.size() * 2 + 4) * sizeof(T)));
    cap = v.size() * 2 + 4;
  }
  if (!v.empty()) MM_CUDA(cudaMemcpyAsync(dev, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return MM_OK;
}

// combined launch lists and per-problem pointers of the running FP32 requests
int rebuild_launch(Server* S) {
  std::vector<TileDesc> tiles, ntiles;
  std::vector<ProbPtrs> probs, nprobs;
  std::vector<PGroup> wgroups;
  std::vector<WinProb> wprobs;
  int halo = 0, nhalo = 0;
  S->tw32 = nullptr;
  for (size_t i = 0; i < S->running.size(); i++) {
    Request* r = S->running[i];
    if (!r->fp32) continue;   // FP64-class requests run their own iterations
    Plan* P = r->plan;
    const int32_t* halt = reinterpret_cast<const int32_t*>(r->cg->scal) + kHaltOffsetInts;
    if (!S->tw32) S->tw32 = P->tw32;
    ProbPtrs pp{};
    pp.lpix = P->lpix;
    pp.w32 = P->w32;
    pp.w64 = P->w64;
    pp.tab = P->tab32;
    pp.done = halt;
    if (P->groups && P->t32 && P->u32) {
      // P over the windows (x = p32 -> t), N^-1 on the segments (t -> u), P^T over the windows
      // (u -> q32)
      for (PGroup g : P->groups_host) {
        g.prob = (int32_t)wprobs.size();
        wgroups.push_back(g);
      }
      wprobs.push_back(WinProb{P->block_off_dev, P->slot, P->slot_pix, P->ang2, r->cg->p32, P->t32, P->u32,
                               r->cg->q32, halt});
      for (TileDesc td : P->segs_host) {
        td.prob = (int32_t)nprobs.size();
        ntiles.push_back(td);
      }
      nhalo = std::max(nhalo, (int)P->seg_halo);
      pp.x = P->t32;
      pp.y = P->u32;
      nprobs.push_back(pp);
    } else {
      for (TileDesc td : P->segs_host) {
        td.prob = (int32_t)probs.size();
        tiles.push_back(td);
      }
      halo = std::max(halo, (int)P->seg_halo);
      pp.x = r->cg->p32;
      pp.y = r->cg->q32;
      probs.push_back(pp);
    }
  }
  MM_TRY(upload_list(tiles, S->tiles_dev, S->tiles_cap, S->stream));
  MM_TRY(upload_list(probs, S->probs_dev, S->probs_cap, S->stream));
  MM_TRY(upload_list(ntiles, S->ntiles_dev, S->ntiles_cap, S->stream));
  MM_TRY(upload_list(nprobs, S->nprobs_dev, S->nprobs_cap, S->stream));
  MM_TRY(upload_list(wgroups, S->wgroups_dev, S->wgroups_cap, S->stream));
  MM_TRY(upload_list(wprobs, S->wprobs_dev, S->wprobs_cap, S->stream));
  MM_CUDA(cudaStreamSynchronize(S->stream));   // host vectors go out of scope
  S->n_tiles = (int64_t)tiles.size();
  S->halo = halo;
  S->n_ntiles = (int64_t)ntiles.size();
  S->nhalo = nhalo;
  S->n_wgroups = (int64_t)wgroups.size();
  S->dirty = false;
  return MM_OK;
}

// one A-application of every running FP32 request (accumulated into its zeroed q32)
int enqueue_multi_apply(Server* S, cudaStream_t s) {
  if (S->n_wgroups > 0) {
    MM_CUDA(launch_unpoint_win32_multi(S->wgroups_dev, S->n_wgroups, S->wprobs_dev, s));
    TileArgs a{};
    a.tiles = S->ntiles_dev;
    a.n_tiles = S->n_ntiles;
    a.nrhs = 1;
    a.tw = S->tw32;
    a.probs = S->nprobs_dev;
    MM_CUDA(launch_ninv32_multi(a, S->nhalo, s));
    MM_CUDA(launch_point_win32_multi(S->wgroups_dev, S->n_wgroups, S->wprobs_dev, s));
  }
  if (S->n_tiles > 0) {
    TileArgs a{};
    a.tiles = S->tiles_dev;
    a.n_tiles = S->n_tiles;
    a.nrhs = 1;
    a.tw = S->tw32;
    a.probs = S->probs_dev;
    MM_CUDA(launch_tiles_fp32_multi(a, S->halo, s));
  }
  return MM_OK;
}

// map in global pixel order
int collect_map(Server* S, Request* r) {
  Plan* P = r->plan;
  double* gmap = nullptr;
  MM_CUDA(cudaMalloc((void**)&gmap, (size_t)P->n_pix * 3 * sizeof(double)));
  MM_CUDA(cudaMemsetAsync(gmap, 0, (size_t)P->n_pix * 3 * sizeof(double), S->stream));
  MM_CUDA(launch_to_global(r->cg->x, P->obs_to_global, P->n_obs, gmap, S->stream));
  r->map.resize((size_t)P->n_pix * 3);
  MM_CUDA(cudaMemcpyAsync(r->map.data(), gmap, r->map.size() * sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  MM_CUDA(cudaStreamSynchronize(S->stream));
  cudaFree(gmap);
  return MM_OK;
}

void server_loop(Server* S) {
  cudaSetDevice(S->device);
  int step = 0;
  while (true) {
    // admission: requests the planner threads finished join the running set
    {
      std::unique_lock<std::mutex> lock(S->mu);
      if (S->running.empty() && S->ready.empty() && !S->stop)
        S->cv_work.wait_for(lock, std::chrono::milliseconds(50));
      if (S->stop) break;
      if (!S->ready.empty()) {
        for (Request* r : S->ready) S->running.push_back(r);
        S->ready.clear();
        S->dirty = true;
      }
      S->n_running = (int)S->running.size();
    }
    if (S->running.empty()) continue;
    // a failed launch or copy ends every running request with MM_ECUDA (no result is read from a
    // state the device did not write); the server goes on with the next requests
    auto abort_running = [&] {
      cudaGetLastError();   // a launch error is not sticky: clear it
      for (Request* r : S->running) finish_request(S, r, MM_ECUDA);
      S->running.clear();
      S->dirty = true;
      std::lock_guard<std::mutex> lock(S->mu);
      S->n_running = 0;
    };
    if (S->dirty && rebuild_launch(S) != MM_OK) {
      abort_running();
      continue;
    }
    const int nb = (int)S->running.size();
    for (Request* r : S->running) r->batch = std::max(r->batch, nb);
    // one PCG iteration of every running request: the FP32 requests' A-applications in shared
    // launches (three over the pixel windows and segments, one of fused tiles for plans without
    // windows), the FP64-class requests' own operator launches after them
    cudaStream_t s = S->stream;
    bool ok = true;
    for (Request* r : S->running)
      if (r->fp32) ok = ok && launch_cg(CG_PUPDATE, r->w, s) == cudaSuccess;
    ok = ok && enqueue_multi_apply(S, s) == MM_OK;
    for (Request* r : S->running) {
      if (r->fp32) {
        ok = ok && launch_cg(CG_DOT_PQ, r->w, s) == cudaSuccess;
        ok = ok && launch_cg(CG_UPDATE, r->w, s) == cudaSuccess;
      } else {
        ok = ok && enqueue_iteration(r->plan, r->w, 1, false, s) == MM_OK;
      }
      r->launched += 1;
    }
    if (!ok) {
      abort_running();
      continue;
    }
    step += 1;
    if (step % 4 != 0) continue;
    for (Request* r : S->running)
      ok = ok && cudaMemcpyAsync(r->scal_host, r->cg->scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, s) ==
                     cudaSuccess;
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) {
      abort_running();
      continue;
    }
    // FP64-class work of this check, enqueued for every request that needs it before one wait:
    // the residual replacement of FP32 requests, the true residual of finished FP64-class ones
    std::vector<char> enq_ok(S->running.size(), 1);
    bool any = false;
    for (size_t k = 0; k < S->running.size(); k++) {
      Request* r = S->running[k];
      const CgScalars sc = *r->scal_host;
      const int rel_every = r->opts.reliable_every > 0 ? r->opts.reliable_every : 50;
      const bool replace = r->fp32 && !sc.done && (sc.paused || sc.since_rep >= rel_every);
      const bool report = !r->fp32 && sc.done;
      if (!replace && !report) continue;
      Plan* P = r->plan;
      any = true;
      enq_ok[k] = cudaMemsetAsync(r->cg->q, 0, P->n_obs * 4 * sizeof(double), s) == cudaSuccess &&
                  (replace ? apply64_internal(P, r->cg->x, r->cg->q, 1, s,
                                              reinterpret_cast<const int32_t*>(r->cg->scal) + kDoneOffsetInts,
                                              kScalStrideInts)
                           : apply64_internal(P, r->cg->x, r->cg->q, 1, s)) == MM_OK &&
                  launch_cg(replace ? CG_REPLACE : CG_TRUE_RES, r->w, s) == cudaSuccess &&
                  cudaMemcpyAsync(r->scal_host, r->cg->scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, s) ==
                      cudaSuccess;
    }
    if (any && cudaStreamSynchronize(s) != cudaSuccess) {
      abort_running();
      continue;
    }
    std::vector<Request*> still;
    for (size_t k = 0; k < S->running.size(); k++) {
      Request* r = S->running[k];
      if (!enq_ok[k]) {
        cudaGetLastError();
        finish_request(S, r, MM_ECUDA);
        S->dirty = true;
        continue;
      }
      const CgScalars sc2 = *r->scal_host;
      const double el = std::chrono::duration<double, std::micro>(Clock::now() - r->t_admit).count();
      const bool late = r->opts.deadline_us > 0 && el > (double)r->opts.deadline_us;
      if (sc2.done || late) {
        mm_solve_info& in = r->info;
        in.iters = sc2.iters;
        in.rel_res = sc2.bnorm2 > 0 ? std::sqrt(sc2.rr / sc2.bnorm2) : 0.0;
        in.true_rel_res = sc2.bnorm2 > 0 ? std::sqrt(sc2.rr_true / sc2.bnorm2) : 0.0;
        in.n_true_res = sc2.n_true;
        in.t_queue_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
        in.t_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_admit).count();
        in.n_apply32 = r->fp32 ? r->launched : 0;
        in.n_apply64 = r->fp32 ? sc2.n_true : r->launched;
        int st = sc2.done ? sc2.status : MM_ETIMEOUT;
        if (st == MM_OK && !sc2.done) st = MM_ENOTCONV;
        if (collect_map(S, r) != MM_OK && st == MM_OK) st = MM_ECUDA;
        finish_request(S, r, st);
        S->dirty = true;
      } else {
        still.push_back(r);
      }
    }
    S->running.swap(still);
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->n_running = (int)S->running.size();
    }
    S->cv_plan.notify_all();
  }
  // abandoned requests
  for (Request* r : S->running) finish_request(S, r, MM_ECUDA);
  S->running.clear();
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" {

const char* mm_last_error(void) { return g_err.c_str(); }

int mm_plan(const mm_problem_desc* desc, void* stream, mm_plan_t* out) {
  if (!out) return fail(MM_EINVAL, "out is NULL");
  *out = nullptr;
  MM_TRY(validate_desc(desc));
  Plan* P = new Plan();
  const int st = build_plan(desc, as_stream(stream), P);
  if (st != MM_OK) {
    free_plan(P);
    return st;
  }
  *out = reinterpret_cast<mm_plan_t>(P);
  return MM_OK;
}

int mm_plan_query(mm_plan_t plan, int64_t* n_obs, const int32_t** obs_to_global_dev, int64_t* n_samples,
                  size_t* bytes) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P) return fail(MM_EINVAL, "plan is NULL");
  if (n_obs) *n_obs = P->n_obs;
  if (obs_to_global_dev) *obs_to_global_dev = P->obs_to_global;
  if (n_samples) *n_samples = P->N;
  if (bytes) *bytes = P->bytes;
  return MM_OK;
}

void mm_plan_destroy(mm_plan_t plan) { free_plan(reinterpret_cast<Plan*>(plan)); }

int mm_apply_P(mm_plan_t plan, const double* x, double* t, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !x || !t) return fail(MM_EINVAL, "NULL argument");
  DeviceGuard g(P->device);
  cudaStream_t s = as_stream(stream);
  MM_TRY(ensure_maps(P, 1, false));
  MM_CUDA(launch_pack3to4(x, P->n_obs, 1, P->map64_in, s));
  MM_CUDA(launch_unpoint64(P->lpix, P->w64, P->N, P->map64_in, t, s));
  return MM_OK;
}

int mm_apply_Pt(mm_plan_t plan, const double* t, double* y, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !t || !y) return fail(MM_EINVAL, "NULL argument");
  DeviceGuard g(P->device);
  cudaStream_t s = as_stream(stream);
  MM_TRY(ensure_maps(P, 1, false));
  MM_CUDA(cudaMemsetAsync(P->map64_out, 0, P->n_obs * 4 * sizeof(double), s));
  MM_CUDA(launch_point64(P->lpix, P->w64, P->N, t, P->map64_out, s));
  MM_CUDA(launch_unpack4to3(P->map64_out, P->n_obs, 1, y, s));
  return MM_OK;
}

int mm_apply_Ninv(mm_plan_t plan, const double* t, double* y, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !t || !y) return fail(MM_EINVAL, "NULL argument");
  if (t == y) return fail(MM_EINVAL, "mm_apply_Ninv cannot run in place");
  DeviceGuard g(P->device);
  cudaStream_t s = as_stream(stream);
  if (P->algo == MM_TPLZ_DIRECT) {
    MM_CUDA(launch_toeplitz_direct(P->band, P->block_off_dev, P->n_blocks, P->lambda, P->N, t, y, s));
    return MM_OK;
  }
  TileArgs a = base_args(P, false);
  a.x = t;
  a.x_stride = P->N;
  a.y = y;
  a.y_stride = P->N;
  MM_CUDA(launch_tiles_fp64(MODE_NINV, a, s));
  return MM_OK;
}

// Is p host memory (pinned or pageable) rather than device or managed memory?
static bool is_host_pointer(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();   // older drivers report unregistered host memory as an error
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

constexpr size_t kStageBytes = (size_t)64 << 20;

// Host TOD -> the df64 input buffer: chunks of one column go through two staging buffers, the
// copy of chunk k + 1 (copy stream) overlapping the split of chunk k (stream s).
static int stage_d_to_df(Plan* P, const void* d, int d_is_fp32, int r0, int g, cudaStream_t s) {
  if (!P->stage[0]) {
    for (int i = 0; i < 2; i++) MM_TRY(dalloc(P, reinterpret_cast<unsigned char**>(&P->stage[i]), kStageBytes));
    P->stage_bytes = kStageBytes;
    MM_CUDA(cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : P->stage_ev) MM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  const size_t esz = d_is_fp32 ? sizeof(float) : sizeof(double);
  const int64_t chunk = (int64_t)(P->stage_bytes / esz) & ~(int64_t)1023;
  cudaStream_t cs = P->copy_stream;
  MM_CUDA(cudaEventRecord(P->stage_ev[2], s));   // the buffers are free once earlier work on s is
  MM_CUDA(cudaEventRecord(P->stage_ev[3], s));
  int k = 0;
  for (int r = r0; r < r0 + g; r++) {
    const unsigned char* col = reinterpret_cast<const unsigned char*>(d) + (size_t)r * P->N * esz;
    for (int64_t c0 = 0; c0 < P->N; c0 += chunk, k ^= 1) {
      const int64_t n = std::min(chunk, P->N - c0);
      MM_CUDA(cudaStreamWaitEvent(cs, P->stage_ev[2 + k], 0));
      MM_CUDA(cudaMemcpyAsync(P->stage[k], col + (size_t)c0 * esz, (size_t)n * esz, cudaMemcpyHostToDevice, cs));
      MM_CUDA(cudaEventRecord(P->stage_ev[k], cs));
      MM_CUDA(cudaStreamWaitEvent(s, P->stage_ev[k], 0));
      MM_CUDA(launch_d_to_df(P->lpix + c0, P->stage[k], d_is_fp32, n, 1,
                             P->tdf + (size_t)(r - r0) * df_stride(P) + c0, df_stride(P), s));
      MM_CUDA(cudaEventRecord(P->stage_ev[2 + k], s));
    }
  }
  return MM_OK;
}

int mm_rhs(mm_plan_t plan, const void* d, int d_is_fp32, int nrhs, double* b, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !d || !b || nrhs <= 0) return fail(MM_EINVAL, "bad argument");
  DeviceGuard g(P->device);
  cudaStream_t s = as_stream(stream);
  const bool host_d = is_host_pointer(d);
  MM_TRY(ensure_maps(P, nrhs, false));
  const size_t n4 = (size_t)nrhs * P->n_obs * 4;
  const size_t esz = d_is_fp32 ? sizeof(float) : sizeof(double);
  MM_CUDA(cudaMemsetAsync(P->map64_out, 0, n4 * sizeof(double), s));
  if (P->tmpl || P->df64) {   // the TOD split to df64 pairs (G d), then the df64 operator
    const int k = df_cols(P, nrhs);
    MM_TRY(P->tmpl ? ensure_tdf(P, k) : ensure_df(P, nrhs));
    for (int r0 = 0; r0 < nrhs; r0 += k) {
      const int g = std::min(k, nrhs - r0);
      if (host_d) {
        MM_TRY(stage_d_to_df(P, d, d_is_fp32, r0, g, s));
      } else {
        MM_CUDA(launch_d_to_df(P->lpix, reinterpret_cast<const char*>(d) + (size_t)r0 * P->N * esz, d_is_fp32,
                               P->N, g, P->tdf, df_stride(P), s));
      }
      double* out = P->map64_out + (size_t)r0 * P->n_obs * 4;
      if (P->tmpl) {   // template map-making: b = P^T F_T G d in one fused kernel
        const TmplState* ts = reinterpret_cast<const TmplState*>(P->tmpl);
        MM_CUDA(launch_tmpl_apply_df(ts->dev, P->n_blocks, P->wdf, nullptr, 0, P->tdf, df_stride(P), out,
                                     P->n_obs * 4, g, nullptr, 0, s));
      } else {
        MM_TRY(df_ninv_point(P, g, nullptr, 0, out, s));
      }
    }
  } else if (P->algo == MM_TPLZ_DIRECT) {
    MM_TRY(ensure_td(P));
    for (int r = 0; r < nrhs; r++) {
      const void* dr = reinterpret_cast<const char*>(d) + (size_t)r * P->N * esz;
      if (host_d) {   // the column into td_b, masked into td_a
        MM_CUDA(cudaMemcpyAsync(P->td_b, dr, P->N * esz, cudaMemcpyHostToDevice, s));
        dr = P->td_b;
      }
      MM_CUDA(launch_mask_d(P->lpix, dr, d_is_fp32, P->N, P->td_a, s));
      MM_CUDA(launch_toeplitz_direct(P->band, P->block_off_dev, P->n_blocks, P->lambda, P->N,
                                     P->td_a, P->td_b, s));
      MM_CUDA(launch_point64(P->lpix, P->w64, P->N, P->td_b, P->map64_out + (size_t)r * P->n_obs * 4, s));
    }
  } else {
    TileArgs a = base_args(P, false);
    a.x_is_fp32 = d_is_fp32 ? 1 : 0;
    a.x_stride = P->N;
    a.y_stride = P->n_obs * 4;
    if (!host_d) {
      a.nrhs = nrhs;
      a.x = d;
      a.y = P->map64_out;
      MM_CUDA(launch_tiles_fp64(MODE_RHS, a, s));
    } else {   // one column at a time through the plan's N-sample FP64 buffer
      MM_TRY(ensure_td(P));
      for (int r = 0; r < nrhs; r++) {
        MM_CUDA(cudaMemcpyAsync(P->td_a, reinterpret_cast<const char*>(d) + (size_t)r * P->N * esz, P->N * esz,
                                cudaMemcpyHostToDevice, s));
        a.nrhs = 1;
        a.x = P->td_a;
        a.y = P->map64_out + (size_t)r * P->n_obs * 4;
        MM_CUDA(launch_tiles_fp64(MODE_RHS, a, s));
      }
    }
  }
  MM_CUDA(launch_unpack4to3(P->map64_out, P->n_obs, nrhs, b, s));
  // a host TOD may be reused once the call returns
  if (host_d) MM_CUDA(cudaStreamSynchronize(s));
  return MM_OK;
}

int mm_apply_A(mm_plan_t plan, const double* x, double* y, int nrhs, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !x || !y || nrhs <= 0) return fail(MM_EINVAL, "bad argument");
  DeviceGuard g(P->device);
  cudaStream_t s = as_stream(stream);
  const bool fp32 = P->precision == MM_FP32 && P->algo != MM_TPLZ_DIRECT;
  MM_TRY(ensure_maps(P, nrhs, fp32));
  const size_t n4 = (size_t)nrhs * P->n_obs * 4;
  MM_CUDA(launch_pack3to4(x, P->n_obs, nrhs, P->map64_in, s));
  if (fp32) {
    MM_CUDA(launch_to32(P->map64_in, (int64_t)(n4 / 4), P->map32_in, s));
    MM_CUDA(cudaMemsetAsync(P->map32_out, 0, n4 * sizeof(float), s));
    MM_TRY(apply32_internal(P, P->map32_in, P->map32_out, nrhs, s));
    MM_CUDA(launch_to64(P->map32_out, (int64_t)(n4 / 4), P->map64_out, s));
  } else {
    MM_CUDA(cudaMemsetAsync(P->map64_out, 0, n4 * sizeof(double), s));
    MM_TRY(apply64_internal(P, P->map64_in, P->map64_out, nrhs, s));
  }
  MM_CUDA(launch_unpack4to3(P->map64_out, P->n_obs, nrhs, y, s));
  return MM_OK;
}

int mm_precond(mm_plan_t plan, const double* r, double* z, int nrhs, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !r || !z || nrhs <= 0) return fail(MM_EINVAL, "bad argument");
  DeviceGuard g(P->device);
  cudaStream_t s = as_stream(stream);
  MM_TRY(ensure_maps(P, nrhs, false));
  MM_CUDA(launch_pack3to4(r, P->n_obs, nrhs, P->map64_in, s));
  MM_CUDA(launch_bd_apply(P->minv, P->n_obs, nrhs, P->map64_in, P->map64_out, s));
  MM_CUDA(launch_unpack4to3(P->map64_out, P->n_obs, nrhs, z, s));
  return MM_OK;
}

// PCG (Algorithm 1) from b, or, with tod (FP32 iterations on a double-float plan with pixel
// windows), from the TOD: b is formed with the FP32 operators and every true residual is
// evaluated as P^T N^-1 G (d - P x) with the double-float operator, one FP64-class pass for the
// right-hand side and the final check together.
static int pcg_solve_impl(Plan* P, const double* b, const TodSrc* tod, double* x, int nrhs, const mm_solve_opts* opts,
                   mm_solve_info* info, void* stream) {
  if (!P || (!b && !tod) || !x || !opts || !info || nrhs <= 0) return fail(MM_EINVAL, "bad argument");
  if (!(opts->tol > 0.0) || opts->max_iter < 0) return fail(MM_EINVAL, "bad tol / max_iter");
  if (opts->precond != MM_PREC_BD && opts->precond != MM_PREC_2LVL_POST)
    return fail(MM_EINVAL, "unsupported preconditioner");
  DeflState* dst = reinterpret_cast<DeflState*>(P->defl);
  if (opts->precond == MM_PREC_2LVL_POST && (!dst || dst->k == 0))
    return fail(MM_EINVAL, "MM_PREC_2LVL_POST needs mm_deflation_build on the plan");
  if (opts->precision != MM_FP64 && opts->precision != MM_FP32) return fail(MM_EINVAL, "bad precision");
  DeviceGuard g(P->device);
  const auto t0 = std::chrono::steady_clock::now();
  const bool fp32 = opts->precision == MM_FP32 && P->algo != MM_TPLZ_DIRECT;
  // profiling launches one iteration per host check, so no halted launch is timed or counted
  const int chunk = opts->profile ? 1 : (opts->check_every > 0 ? opts->check_every : 8);
  const int rel_every = opts->reliable_every > 0 ? opts->reliable_every : 50;
  cudaStream_t us = as_stream(stream);
  cudaStream_t s = P->stream;
  CgState* c = nullptr;
  MM_TRY(ensure_cg(P, nrhs, fp32, &c, s));
  CgWork w = make_work(P, c, nrhs, fp32, opts->tol, opts->max_iter);
  if (P->algo == MM_TPLZ_DIRECT) MM_TRY(ensure_td(P));
  if (fp32) MM_TRY(ensure_t32(P, nrhs));
  MM_TRY(ensure_df(P, nrhs));
  DeflWork dw{};
  const DeflWork* dwp = nullptr;
  if (opts->precond == MM_PREC_2LVL_POST) {
    MM_TRY(ensure_defl_work(P, dst, nrhs, w.n_blocks, &dw, s));
    dwp = &dw;
  }

  cudaEvent_t ev;
  MM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MM_CUDA(cudaEventRecord(ev, us));
  MM_CUDA(cudaStreamWaitEvent(s, ev, 0));

  if (tod) {
    MM_TRY(rhs32_internal(P, tod->d, tod->d_is_fp32, nrhs, c->b, s));
  } else {
    MM_CUDA(launch_pack3to4(b, P->n_obs, nrhs, c->b, s));
  }
  MM_CUDA(launch_cg(CG_INIT, w, s));
  if (dwp) MM_CUDA(launch_defl_step(dw, w, s));

  // graph of `chunk` iterations, cached on the plan
  // A captured graph holds raw pointers: it is replayed only while none of the plan buffers it
  // reads (t, df64 and direct-path scratch, deflation space and its work arrays) was reallocated.
  if (opts->profile == 0 && (!c->exec || c->g_nrhs != nrhs || c->g_fp32 != (int)fp32 || c->g_chunk != chunk ||
      c->g_tol2 != w.tol2 || c->g_maxit != opts->max_iter || c->g_prec != opts->precond ||
      c->g_buf_gen != P->buf_gen)) {
    if (c->exec) {
      cudaGraphExecDestroy(c->exec);
      c->exec = nullptr;
    }
    cudaGraph_t graph;
    MM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int st = MM_OK;
    for (int k = 0; k < chunk && st == MM_OK; k++) st = enqueue_iteration(P, w, nrhs, fp32, s, dwp);
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != MM_OK) return st;
    MM_CUDA(ce);
    ce = cudaGraphInstantiate(&c->exec, graph, 0);
    cudaGraphDestroy(graph);
    MM_CUDA(ce);
    c->g_nrhs = nrhs;
    c->g_fp32 = fp32;
    c->g_chunk = chunk;
    c->g_tol2 = w.tol2;
    c->g_maxit = opts->max_iter;
    c->g_prec = opts->precond;
    c->g_buf_gen = P->buf_gen;
  }

  std::vector<int> timed_out(nrhs, 0);
  const bool profile = opts->profile != 0;
  int64_t n_kernels = 2;   // pack + init
  // profile mode: event pairs around every tile launch, summed at each host sync
  struct EvPair { cudaEvent_t a, b, m, m2; int is64; };
  std::vector<EvPair> pool, pending;
  double t32 = 0.0, t64 = 0.0, tup = 0.0, tpt = 0.0;
  int n32 = 0, n64 = 0;
  auto take_pair = [&](int is64, EvPair* out) -> int {
    if (pool.empty()) {
      EvPair e{};
      MM_CUDA(cudaEventCreate(&e.a));
      MM_CUDA(cudaEventCreate(&e.b));
      MM_CUDA(cudaEventCreate(&e.m));
      MM_CUDA(cudaEventCreate(&e.m2));
      pool.push_back(e);
    }
    *out = pool.back();
    pool.pop_back();
    out->is64 = is64;
    return MM_OK;
  };
  auto drain = [&]() -> int {
    for (EvPair& e : pending) {
      float ms = 0.f;
      MM_CUDA(cudaEventElapsedTime(&ms, e.a, e.b));
      if (e.is64) { t64 += ms; n64++; } else {
        t32 += ms;
        n32++;
        float mu = 0.f, mp = 0.f;
        MM_CUDA(cudaEventElapsedTime(&mu, e.a, e.m));
        MM_CUDA(cudaEventElapsedTime(&mp, e.m2, e.b));
        tup += mu;
        tpt += mp;
      }
      pool.push_back(e);
    }
    pending.clear();
    return MM_OK;
  };
  // q before an FP64-class A x: 0, or b for the TOD form (q = b + P^T N^-1 (P x - G d), r = b - q)
  auto clear_q = [&]() -> int {
    const size_t bytes = (size_t)nrhs * P->n_obs * 4 * sizeof(double);
    if (tod) MM_CUDA(cudaMemcpyAsync(c->q, c->b, bytes, cudaMemcpyDeviceToDevice, s));
    else MM_CUDA(cudaMemsetAsync(c->q, 0, bytes, s));
    return MM_OK;
  };
  auto timed_apply64 = [&](const int32_t* done_flags) -> int {
    EvPair e{};
    if (profile) {
      MM_TRY(take_pair(1, &e));
      MM_CUDA(cudaEventRecord(e.a, s));
    }
    MM_TRY(apply64_internal(P, c->x, c->q, nrhs, s, done_flags, done_flags ? kScalStrideInts : 0, tod));
    if (profile) {
      MM_CUDA(cudaEventRecord(e.b, s));
      pending.push_back(e);
    } else {
      n64++;
    }
    n_kernels += (P->algo == MM_TPLZ_DIRECT) ? 3 * nrhs : 1;
    return MM_OK;
  };
  const int32_t* halt = reinterpret_cast<const int32_t*>(c->scal) + kHaltOffsetInts;
  while (true) {
    MM_CUDA(cudaMemcpyAsync(c->scal_host, c->scal, nrhs * sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    MM_TRY(drain());
    bool all_done = true, need_rep = false;
    for (int r = 0; r < nrhs; r++) {
      const CgScalars& sc = c->scal_host[r];
      if (!sc.done) all_done = false;
      if (!sc.done && fp32 && (sc.paused || sc.since_rep >= rel_every)) need_rep = true;
    }
    if (all_done) break;
    const double el_us =
        std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    if (opts->deadline_us > 0 && el_us > (double)opts->deadline_us) {
      for (int r = 0; r < nrhs; r++) timed_out[r] = !c->scal_host[r].done;
      break;
    }
    if (need_rep) {
      // residual replacement: r = b - A x with A in FP64 (from the TOD: q = b + A x - b_exact)
      MM_TRY(clear_q());
      MM_TRY(timed_apply64(reinterpret_cast<const int32_t*>(c->scal) + kDoneOffsetInts));
      MM_CUDA(launch_cg(CG_REPLACE, w, s));
      n_kernels += 1;
      if (dwp) {
        DeflWork dr = dw;
        dr.restart = 1;
        MM_CUDA(launch_defl_step(dr, w, s));
        n_kernels += 2;
      }
      continue;
    }
    if (!profile) {
      MM_CUDA(cudaGraphLaunch(c->exec, s));
      n_kernels += (int64_t)chunk * ((fp32 || P->algo != MM_TPLZ_DIRECT ? 4 : 3 + 3 * nrhs) + (dwp ? 2 : 0));
      if (fp32) n32 += chunk; else n64 += chunk;
    } else {
      for (int k = 0; k < chunk; k++) {
        MM_CUDA(launch_cg(CG_PUPDATE, w, s));
        EvPair e{};
        MM_TRY(take_pair(fp32 ? 0 : 1, &e));
        MM_CUDA(cudaEventRecord(e.a, s));
        if (fp32) {
          MM_TRY(apply32_internal(P, w.p32, w.q32, nrhs, s, halt, kScalStrideInts, e.m, e.m2));
        } else {
          MM_TRY(apply64_internal(P, w.p, w.q, nrhs, s, halt, kScalStrideInts));
        }
        MM_CUDA(cudaEventRecord(e.b, s));
        pending.push_back(e);
        MM_CUDA(launch_cg(CG_DOT_PQ, w, s));
        MM_CUDA(launch_cg(CG_UPDATE, w, s));
        n_kernels += (fp32 || P->algo != MM_TPLZ_DIRECT) ? 4 : 3 + 3 * nrhs;
        if (dwp) {
          MM_CUDA(launch_defl_step(dw, w, s));
          n_kernels += 2;
        }
      }
    }
  }

  // true residual ||b - A x|| in FP64 for the report.  On the FP32 path a column can only
  // finish with MM_OK through a residual replacement, which already measured it at the final x.
  bool need_true = !fp32;
  for (int r = 0; r < nrhs; r++)
    if (!(c->scal_host[r].done && c->scal_host[r].status == MM_OK)) need_true = true;
  if (need_true) {
    MM_TRY(clear_q());
    MM_TRY(timed_apply64(nullptr));
    MM_CUDA(launch_cg(CG_TRUE_RES, w, s));
    n_kernels += 1;
  }
  MM_CUDA(launch_unpack4to3(c->x, P->n_obs, nrhs, x, s));
  n_kernels += 1;
  MM_CUDA(cudaMemcpyAsync(c->scal_host, c->scal, nrhs * sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  MM_TRY(drain());
  if (P->tc) {   // a timed-out tensor-core wait leaves its tile unwritten: the solve cannot be trusted
    int32_t e = 0;
    MM_CUDA(cudaMemcpy(&e, P->tc_err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e != 0) return fail(MM_ECUDA, "a tensor-core Toeplitz tile timed out waiting for its MMAs");
  }
  for (EvPair& e : pool) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
    cudaEventDestroy(e.m);
    cudaEventDestroy(e.m2);
  }
  MM_CUDA(cudaEventRecord(ev, s));
  MM_CUDA(cudaStreamWaitEvent(us, ev, 0));
  cudaEventDestroy(ev);
  const double t_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int worst = MM_OK;
  for (int r = 0; r < nrhs; r++) {
    const CgScalars& sc = c->scal_host[r];
    mm_solve_info& in = info[r];
    in.iters = sc.iters;
    in.rel_res = sc.bnorm2 > 0 ? std::sqrt(sc.rr / sc.bnorm2) : 0.0;
    in.true_rel_res = sc.bnorm2 > 0 ? std::sqrt(sc.rr_true / sc.bnorm2) : 0.0;
    in.t_ms = t_ms;
    in.n_true_res = sc.n_true;
    in.batch = 1;
    in.t_queue_ms = 0.0;
    in.t_apply32_ms = t32;
    in.t_unpoint32_ms = tup;
    in.t_point32_ms = tpt;
    in.t_apply64_ms = t64;
    in.n_apply32 = n32;
    in.n_apply64 = n64;
    in.n_kernels = n_kernels;
    int st = sc.status;
    if (st == MM_OK && !sc.done) st = timed_out[r] ? MM_ETIMEOUT : MM_ENOTCONV;
    in.status = st;
    if (st != MM_OK && (worst == MM_OK || st < worst)) worst = st;
  }
  if (worst != MM_OK) set_error("solve did not converge for every right-hand side");
  return worst;
}

// median device time (ms) of one FP32 A-application of `ncols` columns on the plan's stream
static int time_apply32(Plan* P, int ncols, int reps, double* ms_out) {
  cudaStream_t s = P->stream;
  MM_TRY(ensure_maps(P, ncols, true));
  MM_TRY(ensure_t32(P, ncols));
  const size_t bytes = (size_t)ncols * P->n_obs * 4 * sizeof(float);
  MM_CUDA(cudaMemsetAsync(P->map32_in, 0x3f, bytes, s));   // every value 0.747: timing only
  MM_CUDA(cudaMemsetAsync(P->map32_out, 0, bytes, s));
  MM_TRY(apply32_internal(P, P->map32_in, P->map32_out, ncols, s));   // warm-up
  std::vector<float> t(reps);
  cudaEvent_t a, b;
  MM_CUDA(cudaEventCreate(&a));
  MM_CUDA(cudaEventCreate(&b));
  int st = MM_OK;
  for (int k = 0; k < reps && st == MM_OK; k++) {
    cudaEventRecord(a, s);
    st = apply32_internal(P, P->map32_in, P->map32_out, ncols, s);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&t[k], a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != MM_OK) return st;
  MM_CUDA(cudaGetLastError());
  std::sort(t.begin(), t.end());
  *ms_out = t[reps / 2];
  return MM_OK;
}

int mm_autotune(mm_plan_t plan, int max_width, mm_tune_info* out, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !out || max_width < 0 || max_width > kMaxBlk) return fail(MM_EINVAL, "bad argument");
  if (P->precision != MM_FP32 || P->algo != MM_TPLZ_FFT || !P->groups || P->tmpl)
    return fail(MM_EINVAL, "mm_autotune tunes the FP32 operators of an FFT plan with pixel windows "
                           "(MM_FP32 or MM_FP32_DF64, no templates)");
  DeviceGuard g(P->device);
  cudaEvent_t ev;
  MM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MM_CUDA(cudaEventRecord(ev, as_stream(stream)));
  MM_CUDA(cudaStreamWaitEvent(P->stream, ev, 0));
  cudaEventDestroy(ev);
  std::memset(out, 0, sizeof(*out));
  constexpr int kReps = 3;
  // every candidate's A x (of the same filled input) is checked against the first one's
  std::vector<float> ref, cur;
  auto check = [&](bool* pass) -> int {
    const size_t n = (size_t)P->n_obs * 4;
    std::vector<float>& dst = ref.empty() ? ref : cur;
    dst.resize(n);
    MM_CUDA(cudaMemcpyAsync(dst.data(), P->map32_out, n * sizeof(float), cudaMemcpyDeviceToHost, P->stream));
    MM_CUDA(cudaStreamSynchronize(P->stream));
    *pass = true;
    if (&dst == &ref) return MM_OK;
    double mx = 0.0, dv = 0.0;
    for (size_t i = 0; i < n; i++) {
      mx = std::max(mx, (double)std::fabs(ref[i]));
      dv = std::max(dv, (double)std::fabs(cur[i] - ref[i]));
    }
    const double rel = mx > 0.0 ? dv / mx : dv;
    out->max_rel_dev = std::max(out->max_rel_dev, rel);
    *pass = std::isfinite(rel) && rel < 1e-4;
    if (!*pass) out->n_rejected++;
    return MM_OK;
  };
  // 1. tiles per segment: more tiles per CTA re-read less of the overlap, fewer leave SMs idle
  const int steps_c[] = {1, 2, 4, 8, 16, 32};
  double best = 1e300;
  int best_steps = P->tile_steps;
  for (int v : steps_c) {
    if (v > 1 && P->n_tiles / v < sm_count()) continue;   // fewer segments than SMs
    MM_TRY(build_segments(P, v, P->stream));
    double ms = 0.0;
    bool pass = false;
    MM_TRY(time_apply32(P, 1, kReps, &ms));
    MM_TRY(check(&pass));
    out->steps_cand[out->n_steps] = v;
    out->steps_ms[out->n_steps++] = ms;
    if (pass && ms < best) {
      best = ms;
      best_steps = v;
    }
  }
  MM_TRY(build_segments(P, best_steps, P->stream));
  // 1b. 65536-sample tiles over 2-CTA clusters (large lambda): kept when faster
  out->big_tiles = -1;
  if (P->big) {
    P->use_big = true;
    double ms = 0.0;
    bool pass = false;
    MM_TRY(time_apply32(P, 1, kReps, &ms));
    MM_TRY(check(&pass));
    out->big_tiles_ms = ms;
    P->use_big = pass && ms < best;
    if (P->use_big) best = ms;
    out->big_tiles = P->use_big ? 1 : 0;
  }
  // 2. samples per pixel-window group: larger groups repeat more pixels but stream shorter chunks
  const int win_c[] = {8192, 16384, 32768, 65536};
  best = 1e300;
  int best_win = P->win_samples;
  for (int v : win_c) {
    P->win_samples = v;
    MM_TRY(build_windows(P, P->stream));
    double ms = 0.0;
    bool pass = false;
    MM_TRY(time_apply32(P, 1, kReps, &ms));
    MM_TRY(check(&pass));
    out->win_cand[out->n_win] = v;
    out->win_ms[out->n_win++] = ms;
    if (pass && ms < best) {
      best = ms;
      best_win = v;
    }
  }
  P->win_samples = best_win;
  // 2b. the FP32 P^T: per-sample sums over the windows, or segment reduction over pixel-sorted
  // sub-windows of a few sizes (each size rebuilds the windows)
  int best_seg = 0;
  if (P->precision == MM_FP32) {
    best = 1e300;
    const int seg_c[] = {0, 4096, 8192, 16384};
    for (int v : seg_c) {
      P->use_seg = v > 0;
      if (v > 0 && v != P->seg_sub) P->seg_sub = v;
      MM_TRY(build_windows(P, P->stream));
      double ms = 0.0;
      bool pass = false;
      MM_TRY(time_apply32(P, 1, kReps, &ms));
      MM_TRY(check(&pass));
      out->seg_cand[out->n_seg] = v;
      out->seg_ms[out->n_seg++] = ms;
      if (pass && ms < best) {
        best = ms;
        best_seg = v;
      }
    }
  }
  P->use_seg = best_seg > 0;
  if (best_seg > 0) P->seg_sub = best_seg;
  MM_TRY(build_windows(P, P->stream));
  out->seg_sub = best_seg;
  out->apply_ms = best;
  // 3. block width: device time per column of a batched A X
  double best_col = 1e300;
  int best_w = 1;
  for (int w = 1; w <= std::max(1, max_width); w *= 2) {
    double ms = 0.0;
    MM_TRY(time_apply32(P, w, 2, &ms));
    out->width_cand[out->n_width] = w;
    out->width_ms_per_col[out->n_width++] = ms / w;
    if (ms / w <= best_col * 1.02) {   // ties go to the wider block (fewer block iterations)
      best_col = std::min(best_col, ms / w);
      best_w = w;
    }
  }
  P->tuned_width = best_w;
  out->tile_steps = best_steps;
  out->win_samples = best_win;
  out->block_width = best_w;
  MM_CUDA(cudaStreamSynchronize(P->stream));
  return MM_OK;
}

int mm_pcg_solve(mm_plan_t plan, const double* b, double* x, int nrhs, const mm_solve_opts* opts,
                 mm_solve_info* info, void* stream) {
  return pcg_solve_impl(reinterpret_cast<Plan*>(plan), b, nullptr, x, nrhs, opts, info, stream);
}

int mm_solve_tod(mm_plan_t plan, const void* d, int d_is_fp32, double* x, int nrhs, const mm_solve_opts* opts,
                 mm_solve_info* info, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !d || !x || !opts || !info || nrhs <= 0) return fail(MM_EINVAL, "bad argument");
  if (is_host_pointer(d)) {   // the TOD is read at every residual: a device copy on the plan
    DeviceGuard g(P->device);
    const size_t bytes = (size_t)nrhs * P->N * (d_is_fp32 ? sizeof(float) : sizeof(double));
    if (P->tod_cap < bytes) {
      if (P->tod_buf) {
        cudaFree(P->tod_buf);
        P->bytes -= P->tod_cap;
      }
      P->tod_buf = nullptr;
      P->tod_cap = 0;
      unsigned char* buf = nullptr;
      MM_TRY(dalloc(P, &buf, bytes));
      P->tod_buf = buf;
      P->tod_cap = bytes;
    }
    MM_CUDA(cudaMemcpyAsync(P->tod_buf, d, bytes, cudaMemcpyHostToDevice, as_stream(stream)));
    d = P->tod_buf;
  }
  const bool tod_form = opts->precision == MM_FP32 && P->df64 && P->groups && !P->tmpl &&
                        P->algo == MM_TPLZ_FFT && opts->precond == MM_PREC_BD;
  if (tod_form) {
    const TodSrc tod{d, d_is_fp32 ? 1 : 0};
    return pcg_solve_impl(P, nullptr, &tod, x, nrhs, opts, info, stream);
  }
  // otherwise the FP64-class right-hand side (written into x, which the solve reads first) and PCG
  MM_TRY(mm_rhs(plan, d, d_is_fp32, nrhs, x, stream));
  return pcg_solve_impl(P, x, nullptr, x, nrhs, opts, info, stream);
}

int mm_block_cg_solve(mm_plan_t plan, const double* b, double* x, int nrhs, int block_width,
                      const mm_solve_opts* opts, mm_solve_info* info, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !b || !x || !opts || !info || nrhs <= 0) return fail(MM_EINVAL, "bad argument");
  if (!(opts->tol > 0.0) || opts->max_iter < 0) return fail(MM_EINVAL, "bad tol / max_iter");
  if (opts->precond != MM_PREC_BD) return fail(MM_EINVAL, "unsupported preconditioner");
  if (opts->precision != MM_FP64 && opts->precision != MM_FP32) return fail(MM_EINVAL, "bad precision");
  if (block_width < 0 || block_width > kMaxBlk) return fail(MM_EINVAL, "block_width must lie in [0, 64]");
  if (P->algo == MM_TPLZ_DIRECT) return fail(MM_EINVAL, "block CG needs an FFT plan");
  DeviceGuard g(P->device);
  const auto t0 = std::chrono::steady_clock::now();
  const int sw = block_width > 0 ? block_width : std::min(nrhs, P->tuned_width > 0 ? P->tuned_width : kMaxBlk);
  const bool fp32 = opts->precision == MM_FP32;
  const double tol2 = opts->tol * opts->tol;
  const int64_t n = P->n_obs;
  cudaStream_t us = as_stream(stream);
  cudaStream_t s = P->stream;
  BlkState* B = nullptr;
  MM_TRY(ensure_blk(P, sw, &B));
  if (fp32) MM_TRY(ensure_t32(P, sw));   // the captured iterations must find the FP32 buffers allocated
  cudaEvent_t ev;
  MM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MM_CUDA(cudaEventRecord(ev, us));
  MM_CUDA(cudaStreamWaitEvent(s, ev, 0));
  int worst = MM_OK;
  int64_t n_kernels = 0;
  int n_apply = 0, n_apply64 = 0;
  auto read_norms = [&](int v) -> int {
    MM_CUDA(cudaMemcpyAsync(B->host, B->norms, v * sizeof(double), cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    return MM_OK;
  };
  for (int g0 = 0; g0 < nrhs; g0 += sw) {
    const int sg = std::min(sw, nrhs - g0);
    const size_t n4 = (size_t)sg * n * 4;
    MM_CUDA(launch_pack3to4(b + (size_t)g0 * n * 3, n, sg, B->B, s));
    MM_CUDA(cudaMemsetAsync(B->X, 0, n4 * sizeof(double), s));
    MM_CUDA(cudaMemsetAsync(B->AX, 0, n4 * sizeof(double), s));
    MM_CUDA(launch_bresid(B->B, B->AX, sg, n, B->R, B->norm_part, blk_ctas(), B->norms, s));   // R = B
    n_kernels += 3;
    MM_TRY(read_norms(sg));
    std::vector<double> bn2(B->host, B->host + sg), rn2(bn2), tn2(bn2);
    std::vector<int> conv(sg, 0), iters(sg, 0), status(sg, MM_OK);
    std::vector<int> active;
    for (int j = 0; j < sg; j++) {
      if (bn2[j] == 0.0) conv[j] = 1; else active.push_back(j);
    }
    int it = 0, restarts = 0, r = 0;
    bool fresh = true;   // Z = M R without the A-orthogonalisation (first step, or a restart)
    bool cont = false;
    // FP64-class true residual R = B - A X; columns above tol stay active and restart from it
    // (cont) unless the iteration or restart budget is spent
    auto true_residual = [&]() -> int {
      MM_CUDA(cudaMemsetAsync(B->AX, 0, n4 * sizeof(double), s));
      MM_TRY(apply64_internal(P, B->X, B->AX, sg, s));
      MM_CUDA(launch_bresid(B->B, B->AX, sg, n, B->R, B->norm_part, blk_ctas(), B->norms, s));
      n_kernels += 3;
      n_apply64 += 1;
      MM_TRY(read_norms(sg));
      active.clear();
      for (int j = 0; j < sg; j++) {
        tn2[j] = B->host[j];
        rn2[j] = tn2[j];
        if (bn2[j] > 0.0 && !(tn2[j] < tol2 * bn2[j])) {
          conv[j] = 0;
          active.push_back(j);
        }
      }
      cont = !(active.empty() || it >= opts->max_iter || restarts >= 8);
      if (cont) {
        restarts += 1;
        fresh = true;
      }
      return MM_OK;
    };
    while (!active.empty()) {
      const int t = (int)active.size();
      const bool after_restart = fresh;
      if (it >= opts->max_iter) break;
      MM_CUDA(cudaMemcpyAsync(B->idx, active.data(), t * sizeof(int), cudaMemcpyHostToDevice, s));
      // Z = M R[active], A-orthogonalised against the previous block; AZ = A Z; G = Z^T A Z and
      // its pivoted Cholesky factor (rank r to the host).  FP32 operators: one captured graph per
      // (t, previous r) shape, replayed every iteration of that shape.
      const bool ortho = !fresh && r > 0;
      const int r_prev = r;
      auto part_a = [&]() -> int {
        MM_CUDA(launch_bprecond(P->minv, B->R, B->idx, t, n, B->Z, s));
        if (ortho) {   // Z = (I - P P^T A) M R: Z -= P (AP^T Z)
          MM_CUDA(launch_bgram(B->AP, r_prev, nullptr, B->Z, 0, t, nullptr, n, B->part, blk_ctas(), B->C2, s));
          MM_CUDA(launch_bcombine(B->Z, 0, nullptr, t, B->P, r_prev, B->C2, t, -1.0, 1, n, nullptr, blk_ctas(),
                                  nullptr, s));
        }
        MM_TRY(blk_apply(P, B, t, fp32, s));
        MM_CUDA(launch_bgram(B->Z, t, nullptr, B->AZ, 0, t, nullptr, n, B->part, blk_ctas(), B->G, s));
        MM_CUDA(launch_bchol(B->G, t, 1e-10, B->Linv, B->piv, B->rank, s));
        MM_CUDA(cudaMemcpyAsync(B->host_i, B->rank, sizeof(int), cudaMemcpyDeviceToHost, s));
        return MM_OK;
      };
      if (fp32) {
        const uint64_t key = (1ull << 60) | ((uint64_t)t << 16) | ((uint64_t)ortho << 15) | (uint64_t)r_prev;
        MM_TRY(blk_graph(P, B, key, s, part_a));
      } else {
        MM_TRY(part_a());
      }
      fresh = false;
      MM_CUDA(cudaStreamSynchronize(s));
      r = B->host_i[0];
      n_kernels += 1 + (ortho ? 3 : 0) + (fp32 ? 1 : 3) + 3;
      n_apply += 1;
      if (r == 0) {
        // every direction dropped: on the FP32 path away from a restart this is operator noise
        // along a (near-)null direction of a semi-definite A (e.g. the map offset degenerate with
        // templates), so restart from the true residual; right after a restart it is a breakdown
        if (fp32 && !after_restart) {
          MM_TRY(true_residual());
          if (cont) continue;
          break;
        }
        for (int j : active) status[j] = MM_EBREAKDOWN;
        break;
      }
      // P = Z[piv] L^-T, AP likewise; alpha = P^T R over all sg columns; X += P alpha; R -= AP alpha
      // and the residual norms to the host (FP32 operators: one captured graph per (t, r, sg))
      auto part_b = [&]() -> int {
        MM_CUDA(launch_linv_coef(B->Linv, B->piv, B->rank, t, B->Cmb, s));
        MM_CUDA(launch_bcombine(B->P, 0, nullptr, r, B->Z, t, B->Cmb, t, 1.0, 0, n, nullptr, blk_ctas(), nullptr, s));
        MM_CUDA(launch_bcombine(B->AP, 0, nullptr, r, B->AZ, t, B->Cmb, t, 1.0, 0, n, nullptr, blk_ctas(), nullptr,
                                s));
        MM_CUDA(launch_bgram(B->P, r, nullptr, B->R, 1, sg, nullptr, n, B->part, blk_ctas(), B->alpha, s));
        MM_CUDA(launch_bcombine(B->X, 1, nullptr, sg, B->P, r, B->alpha, sg, 1.0, 1, n, nullptr, blk_ctas(),
                                nullptr, s));
        MM_CUDA(launch_bcombine(B->R, 1, nullptr, sg, B->AP, r, B->alpha, sg, -1.0, 1, n, B->norm_part,
                                blk_ctas(), B->norms, s));
        MM_CUDA(cudaMemcpyAsync(B->host, B->norms, sg * sizeof(double), cudaMemcpyDeviceToHost, s));
        return MM_OK;
      };
      if (fp32) {
        const uint64_t key = (2ull << 60) | ((uint64_t)t << 24) | ((uint64_t)r << 16) | (uint64_t)sg;
        MM_TRY(blk_graph(P, B, key, s, part_b));
      } else {
        MM_TRY(part_b());
      }
      MM_CUDA(cudaStreamSynchronize(s));
      n_kernels += 9;
      it += 1;
      active.clear();
      for (int j = 0; j < sg; j++) {
        rn2[j] = B->host[j];
        if (!conv[j] && rn2[j] < tol2 * bn2[j]) {
          conv[j] = 1;
          iters[j] = it;
        }
        if (!conv[j]) active.push_back(j);
        if (!std::isfinite(rn2[j])) status[j] = MM_EBREAKDOWN;
      }
      bool bad = false;
      for (int j = 0; j < sg; j++) bad = bad || status[j] == MM_EBREAKDOWN;
      if (bad) break;
      if (active.empty() || it >= opts->max_iter) {
        MM_TRY(true_residual());
        if (!cont) break;
      }
    }
    for (int j = 0; j < sg; j++) {
      if (status[j] == MM_OK && !conv[j]) status[j] = MM_ENOTCONV;
      if (status[j] == MM_OK && iters[j] == 0 && bn2[j] > 0.0) iters[j] = it;
    }
    MM_CUDA(launch_unpack4to3(B->X, n, sg, x + (size_t)g0 * n * 3, s));
    n_kernels += 1;
    MM_CUDA(cudaStreamSynchronize(s));
    const double t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int j = 0; j < sg; j++) {
      mm_solve_info& in = info[g0 + j];
      std::memset(&in, 0, sizeof(in));
      in.status = status[j];
      in.iters = iters[j];
      in.rel_res = bn2[j] > 0 ? std::sqrt(rn2[j] / bn2[j]) : 0.0;
      in.true_rel_res = bn2[j] > 0 ? std::sqrt(tn2[j] / bn2[j]) : 0.0;
      in.t_ms = t_ms;
      in.n_true_res = restarts + 1;
      in.n_apply32 = fp32 ? n_apply : 0;
      in.n_apply64 = (fp32 ? 0 : n_apply) + n_apply64;
      in.n_kernels = n_kernels;
      if (status[j] != MM_OK && (worst == MM_OK || status[j] < worst)) worst = status[j];
    }
  }
  MM_CUDA(cudaEventRecord(ev, s));
  MM_CUDA(cudaStreamWaitEvent(us, ev, 0));
  cudaEventDestroy(ev);
  if (worst != MM_OK) set_error("block CG did not converge for every right-hand side");
  return worst;
}

int mm_ecg_solve(mm_plan_t plan, const double* b, double* x, int t, int variant, const mm_solve_opts* opts,
                 mm_solve_info* info, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !b || !x || !opts || !info) return fail(MM_EINVAL, "bad argument");
  if (t < 1 || t > kMaxBlk) return fail(MM_EINVAL, "the enlarging factor t must lie in [1, 64]");
  if (variant != MM_ECG_ORTHOMIN && variant != MM_ECG_ORTHODIR) return fail(MM_EINVAL, "bad ECG variant");
  if (!(opts->tol > 0.0) || opts->max_iter < 0) return fail(MM_EINVAL, "bad tol / max_iter");
  if (opts->precond != MM_PREC_BD) return fail(MM_EINVAL, "ECG runs with the block-Jacobi preconditioner");
  if (opts->precision != MM_FP64 && opts->precision != MM_FP32) return fail(MM_EINVAL, "bad precision");
  if (P->algo == MM_TPLZ_DIRECT) return fail(MM_EINVAL, "ECG needs an FFT plan");
  DeviceGuard g(P->device);
  const auto t0 = std::chrono::steady_clock::now();
  const bool fp32 = opts->precision == MM_FP32;
  const double tol2 = opts->tol * opts->tol;
  const int64_t n = P->n_obs;
  cudaStream_t us = as_stream(stream);
  cudaStream_t s = P->stream;
  BlkState* B = nullptr;
  MM_TRY(ensure_blk(P, t, &B));
  MM_TRY(ensure_ecg(P, B));
  if (fp32) MM_TRY(ensure_t32(P, t));   // the captured iterations must find the FP32 buffers allocated
  cudaEvent_t ev;
  MM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MM_CUDA(cudaEventRecord(ev, us));
  MM_CUDA(cudaStreamWaitEvent(s, ev, 0));
  int64_t n_kernels = 0;
  int n_apply = 0, n_apply64 = 0;
  auto read_host = [&](const double* dev, int v) -> int {
    MM_CUDA(cudaMemcpyAsync(B->host, dev, v * sizeof(double), cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    return MM_OK;
  };
  // b (column 0 of B->B), ||b||^2, x = 0, r = b
  MM_CUDA(launch_pack3to4(b, n, 1, B->B, s));
  MM_CUDA(launch_bsum(B->B, 1, n, B->re, 0, B->norm_part, blk_ctas(), B->norms, s));
  MM_CUDA(cudaMemsetAsync(B->xe, 0, (size_t)n * 4 * sizeof(double), s));
  n_kernels += 3;
  MM_TRY(read_host(B->norms, 1));
  const double bn2 = B->host[0];
  double rel2 = bn2 > 0.0 ? 1.0 : 0.0, tn2 = bn2;
  int it = 0, restarts = 0, status = MM_OK;
  bool converged = !(bn2 > 0.0);
  while (!converged) {
    // R_0 = split of r, X = 0, Z_1 = M R_0
    MM_CUDA(launch_bsplit(B->re, t, n, B->R, s));
    MM_CUDA(cudaMemsetAsync(B->X, 0, (size_t)t * n * 4 * sizeof(double), s));
    MM_CUDA(launch_bprecond(P->minv, B->R, nullptr, t, n, B->Z, s));
    n_kernels += 2;
    int tz = t, rprev = 0;
    bool inner_conv = false, stalled = false;
    // The search blocks are FP32: a recurrence whose directions do not come from the residual
    // (Orthodir) loses A-orthogonality and its recursive residual levels off near 1e-7 ||b||.
    // Once below 1e-6 ||b|| (near that floor; slow progress above it is ordinary CG behaviour on
    // ill-conditioned systems), ||sum R|| that has not halved in kStall block iterations
    // restarts the recurrence from the true residual.
    constexpr int kStall = 10;
    constexpr double kStallZone2 = 1e-12;
    double best = INFINITY;
    int since_best = 0, inner = 0;
    while (it < opts->max_iter) {
      // AZ = A Z, G = Z^T A Z and its pivoted Cholesky factor (rank to the host); FP32 operators:
      // one captured graph per shape
      auto part_a = [&]() -> int {
        MM_TRY(blk_apply(P, B, tz, fp32, s));
        MM_CUDA(launch_bgram(B->Z, tz, nullptr, B->AZ, 0, tz, nullptr, n, B->part, blk_ctas(), B->G, s));
        MM_CUDA(launch_bchol(B->G, tz, 1e-10, B->Linv, B->piv, B->rank, s));
        MM_CUDA(cudaMemcpyAsync(B->host_i, B->rank, sizeof(int), cudaMemcpyDeviceToHost, s));
        return MM_OK;
      };
      if (fp32) {
        MM_TRY(blk_graph(P, B, (3ull << 60) | ((uint64_t)tz << 16), s, part_a));
      } else {
        MM_TRY(part_a());
      }
      MM_CUDA(cudaStreamSynchronize(s));
      const int r = B->host_i[0];
      n_kernels += (fp32 ? 2 : 3) + 3;
      n_apply += 1;
      if (r == 0) {
        // every direction dropped: on the FP32 path after the first step of a recurrence this is
        // operator noise along a (near-)null direction of a semi-definite A (the map offset of
        // template plans), so the recurrence restarts from the true residual as after a stall
        if (fp32 && inner > 0) {
          stalled = true;
          break;
        }
        status = MM_EBREAKDOWN;
        break;
      }
      inner += 1;
      // P_k = Z (Z^T A Z)^{-1/2} and A P_k; alpha = P_k^T R; X += P alpha; R -= A P alpha; the norm
      // of sum_i R_i to the host; and already the next search block (unused when this step ends
      // the recurrence):
      //   Orthomin  Z_{k+1} = (I - P_k P_k^T A) M R_k
      //   Orthodir  Z_{k+1} = (I - P_k P_k^T A - P_{k-1} P_{k-1}^T A) M A P_k
      const int tz_next = (variant == MM_ECG_ORTHOMIN) ? t : r;
      auto part_b = [&]() -> int {
        MM_CUDA(launch_linv_coef(B->Linv, B->piv, B->rank, tz, B->Cmb, s));
        MM_CUDA(launch_bcombine(B->P, 0, nullptr, r, B->Z, tz, B->Cmb, tz, 1.0, 0, n, nullptr, blk_ctas(), nullptr, s));
        MM_CUDA(launch_bcombine(B->AP, 0, nullptr, r, B->AZ, tz, B->Cmb, tz, 1.0, 0, n, nullptr, blk_ctas(), nullptr,
                                s));
        MM_CUDA(launch_bgram(B->P, r, nullptr, B->R, 1, t, nullptr, n, B->part, blk_ctas(), B->alpha, s));
        MM_CUDA(launch_bcombine(B->X, 1, nullptr, t, B->P, r, B->alpha, t, 1.0, 1, n, nullptr, blk_ctas(), nullptr,
                                s));
        MM_CUDA(launch_bcombine(B->R, 1, nullptr, t, B->AP, r, B->alpha, t, -1.0, 1, n, nullptr, blk_ctas(), nullptr,
                                s));
        MM_CUDA(launch_bsum(B->R, t, n, nullptr, 0, B->norm_part, blk_ctas(), B->norms, s));   // ||sum_i R_i||^2
        MM_CUDA(cudaMemcpyAsync(B->host, B->norms, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (variant == MM_ECG_ORTHOMIN) {
          MM_CUDA(launch_bprecond(P->minv, B->R, nullptr, t, n, B->Z, s));
        } else {
          MM_CUDA(launch_bprecond32(P->minv, B->AP, r, n, B->Z, s));
        }
        MM_CUDA(launch_bgram(B->AP, r, nullptr, B->Z, 0, tz_next, nullptr, n, B->part, blk_ctas(), B->C2, s));
        MM_CUDA(launch_bcombine(B->Z, 0, nullptr, tz_next, B->P, r, B->C2, tz_next, -1.0, 1, n, nullptr, blk_ctas(),
                                nullptr, s));
        if (variant == MM_ECG_ORTHODIR && rprev > 0) {
          MM_CUDA(launch_bgram(B->APp, rprev, nullptr, B->Z, 0, tz_next, nullptr, n, B->part, blk_ctas(), B->G, s));
          MM_CUDA(launch_bcombine(B->Z, 0, nullptr, tz_next, B->Pp, rprev, B->G, tz_next, -1.0, 1, n, nullptr,
                                  blk_ctas(), nullptr, s));
        }
        return MM_OK;
      };
      if (fp32) {
        // Orthodir swaps the P / Pp buffers every step: which one is current is part of the shape
        const uint64_t key = (4ull << 60) | ((uint64_t)variant << 45) | ((uint64_t)(B->P < B->Pp) << 44) |
                             ((uint64_t)rprev << 32) | ((uint64_t)tz << 24) | ((uint64_t)r << 16) | ((uint64_t)t << 8);
        MM_TRY(blk_graph(P, B, key, s, part_b));
      } else {
        MM_TRY(part_b());
      }
      MM_CUDA(cudaStreamSynchronize(s));
      n_kernels += 14 + ((variant == MM_ECG_ORTHODIR && rprev > 0) ? 3 : 0);
      it += 1;
      rel2 = B->host[0] / bn2;
      if (!std::isfinite(rel2)) {
        status = MM_EBREAKDOWN;
        break;
      }
      if (rel2 < tol2) {
        inner_conv = true;
        break;
      }
      if (rel2 < 0.25 * best) {
        best = rel2;
        since_best = 0;
      } else if (best < kStallZone2 && ++since_best >= kStall) {
        stalled = true;
        break;
      }
      tz = tz_next;
      if (variant == MM_ECG_ORTHODIR) {
        std::swap(B->P, B->Pp);
        std::swap(B->AP, B->APp);
        rprev = r;
      }
    }
    // x += X 1, then the FP64-class true residual r = b - A x
    MM_CUDA(launch_bsum(B->X, t, n, B->xe, 1, B->norm_part, blk_ctas(), B->norms, s));
    MM_CUDA(cudaMemsetAsync(B->ax, 0, (size_t)n * 4 * sizeof(double), s));
    MM_TRY(apply64_internal(P, B->xe, B->ax, 1, s));
    MM_CUDA(launch_bresid(B->B, B->ax, 1, n, B->re, B->norm_part, blk_ctas(), B->norms, s));
    n_kernels += 5;
    n_apply64 += 1;
    MM_TRY(read_host(B->norms, 1));
    tn2 = B->host[0];
    if (tn2 < tol2 * bn2) {
      converged = true;
      break;
    }
    if (status != MM_OK || !(inner_conv || stalled) || it >= opts->max_iter || restarts >= 8) break;
    restarts += 1;   // restart from the true residual
  }
  if (status == MM_OK && !converged) status = MM_ENOTCONV;
  MM_CUDA(launch_unpack4to3(B->xe, n, 1, x, s));
  n_kernels += 1;
  MM_CUDA(cudaEventRecord(ev, s));
  MM_CUDA(cudaStreamWaitEvent(us, ev, 0));
  MM_CUDA(cudaStreamSynchronize(s));
  cudaEventDestroy(ev);
  std::memset(info, 0, sizeof(*info));
  info->status = status;
  info->iters = it;
  info->rel_res = bn2 > 0 ? std::sqrt(rel2) : 0.0;
  info->true_rel_res = bn2 > 0 ? std::sqrt(tn2 / bn2) : 0.0;
  info->t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  info->n_true_res = restarts + 1;
  info->batch = t;
  info->n_apply32 = fp32 ? n_apply : 0;
  info->n_apply64 = (fp32 ? 0 : n_apply) + n_apply64;
  info->n_kernels = n_kernels;
  if (status != MM_OK) set_error("ECG did not converge");
  return status;
}

int mm_deflation_build(mm_plan_t plan, const double* b, int m, int precision, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !b) return fail(MM_EINVAL, "bad argument");
  if (m < 1 || m > kMaxDefl) return fail(MM_EINVAL, "m must lie in [1, 64]");
  if (precision != MM_FP64 && precision != MM_FP32) return fail(MM_EINVAL, "bad precision");
  if (P->algo == MM_TPLZ_DIRECT && precision == MM_FP32) precision = MM_FP64;
  DeviceGuard g(P->device);
  cudaStream_t us = as_stream(stream);
  cudaStream_t s = P->stream;
  cudaEvent_t ev;
  MM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MM_CUDA(cudaEventRecord(ev, us));
  MM_CUDA(cudaStreamWaitEvent(s, ev, 0));
  cudaEventDestroy(ev);
  const int64_t n = P->n_obs, n4 = 4 * n;
  Scratch scr;
  double *v_prev = nullptr, *v = nullptr, *wv = nullptr, *av = nullptr, *part = nullptr, *dot = nullptr;
  double *alpha_d = nullptr, *beta_d = nullptr, *work = nullptr, *U = nullptr, *X = nullptr, *wvals = nullptr,
         *E = nullptr, *gpart = nullptr;
  float *V32 = nullptr, *AV32 = nullptr, *x32 = nullptr, *y32 = nullptr;
  const int nblk = 4 * sm_count();
  MM_TRY(scr.alloc(&v_prev, n4)); MM_TRY(scr.alloc(&v, n4)); MM_TRY(scr.alloc(&wv, n4)); MM_TRY(scr.alloc(&av, n4));
  MM_TRY(scr.alloc(&part, nblk)); MM_TRY(scr.alloc(&dot, 2));
  MM_TRY(scr.alloc(&alpha_d, kMaxDefl)); MM_TRY(scr.alloc(&beta_d, kMaxDefl));
  MM_TRY(scr.alloc(&work, kMaxDefl * kMaxDefl)); MM_TRY(scr.alloc(&U, kMaxDefl * kMaxDefl));
  MM_TRY(scr.alloc(&X, kMaxDefl * kMaxDefl)); MM_TRY(scr.alloc(&wvals, kMaxDefl));
  MM_TRY(scr.alloc(&E, kMaxDefl * kMaxDefl));
  MM_TRY(scr.alloc(&gpart, (size_t)blk_ctas() * kMaxBlk * kMaxBlk));
  MM_TRY(scr.alloc(&V32, (size_t)m * n4)); MM_TRY(scr.alloc(&AV32, (size_t)m * n4));
  if (precision == MM_FP32) { MM_TRY(scr.alloc(&x32, n4)); MM_TRY(scr.alloc(&y32, n4)); }
  auto host_dot = [&](const double* a_, const double* b_, double* out) -> int {
    MM_CUDA(launch_ldot(a_, b_, n4, part, nblk, dot, s));
    MM_CUDA(cudaMemcpyAsync(out, dot, sizeof(double), cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    return MM_OK;
  };
  // v_1 = b / ||b||, v_0 = 0
  MM_CUDA(launch_pack3to4(b, n, 1, v, s));
  MM_CUDA(cudaMemsetAsync(v_prev, 0, n4 * sizeof(double), s));
  double bb = 0.0;
  MM_TRY(host_dot(v, v, &bb));
  if (!(bb > 0.0) || !std::isfinite(bb)) return fail(MM_EBREAKDOWN, "mm_deflation_build: b = 0");
  MM_CUDA(launch_laxpby(0.0, v, 1.0 / std::sqrt(bb), v, n4, s));
  std::vector<double> alphas, betas;
  double beta_k = 0.0;
  const double eps = 2.220446049250313e-16;
  for (int kk = 0; kk < m; kk++) {
    // A v_k (stored), then w = A v_k - beta_k v_{k-1}; alpha = <w, v_k>; w -= alpha v_k
    MM_CUDA(cudaMemsetAsync(av, 0, n4 * sizeof(double), s));
    if (precision == MM_FP32) {
      MM_CUDA(launch_to32(v, n, x32, s));
      MM_CUDA(cudaMemsetAsync(y32, 0, n4 * sizeof(float), s));
      MM_TRY(apply32_internal(P, x32, y32, 1, s));
      MM_CUDA(launch_to64(y32, n, av, s));
    } else {
      MM_TRY(apply64_internal(P, v, av, 1, s));
    }
    MM_CUDA(launch_to32(v, n, V32 + (size_t)kk * n4, s));
    MM_CUDA(launch_to32(av, n, AV32 + (size_t)kk * n4, s));
    MM_CUDA(cudaMemcpyAsync(wv, av, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    MM_CUDA(launch_laxpby(-beta_k, v_prev, 1.0, wv, n4, s));
    double al = 0.0;
    MM_TRY(host_dot(wv, v, &al));
    MM_CUDA(launch_laxpby(-al, v, 1.0, wv, n4, s));
    double ww = 0.0;
    MM_TRY(host_dot(wv, wv, &ww));
    alphas.push_back(al);
    const double beta_next = std::sqrt(std::max(ww, 0.0));
    if (!std::isfinite(al) || !std::isfinite(beta_next)) return fail(MM_EBREAKDOWN, "Lanczos breakdown");
    if (beta_next < eps) break;
    betas.push_back(beta_next);
    beta_k = beta_next;
    std::swap(v_prev, v);                                       // v_prev = v_k
    MM_CUDA(launch_laxpby(1.0 / beta_next, wv, 0.0, v, n4, s));   // v = w / beta
  }
  const int k = (int)alphas.size();
  std::vector<double> bpad(kMaxDefl, 0.0);
  for (int i = 0; i + 1 < k; i++) bpad[i] = betas[i];
  MM_CUDA(cudaMemcpyAsync(alpha_d, alphas.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemcpyAsync(beta_d, bpad.data(), kMaxDefl * sizeof(double), cudaMemcpyHostToDevice, s));
  MM_CUDA(launch_tridiag_eig(alpha_d, beta_d, k, work, wvals, X, s));
  // replace the plan's space
  DeflState* d = reinterpret_cast<DeflState*>(P->defl);
  if (!d) {
    d = new DeflState();
    P->defl = d;
  }
  dfree(d->Z); dfree(d->Zp); dfree(d->Einv);
  d->k = 0;
  P->buf_gen++;
  MM_TRY(dalloc(P, &d->Z, (size_t)k * n4));
  MM_TRY(dalloc(P, &d->Zp, (size_t)k * n4));
  MM_TRY(dalloc(P, &d->Einv, (size_t)k * k));
  // Z = V X, Z' = (A V) X, E = Z^T Z', Einv = pinv(E)
  MM_CUDA(launch_bcombine(d->Z, 0, nullptr, k, V32, k, X, k, 1.0, 0, n, nullptr, blk_ctas(), nullptr, s));
  MM_CUDA(launch_bcombine(d->Zp, 0, nullptr, k, AV32, k, X, k, 1.0, 0, n, nullptr, blk_ctas(), nullptr, s));
  MM_CUDA(launch_bgram(d->Z, k, nullptr, d->Zp, 0, k, nullptr, n, gpart, blk_ctas(), E, s));
  MM_CUDA(launch_pinv_sym(E, k, 1e-12, work, U, wvals + 0, d->Einv, s));
  std::vector<double> th(k);
  MM_CUDA(launch_tridiag_eig(alpha_d, beta_d, k, work, wvals, X, s));   // Ritz values again (wvals reused)
  MM_CUDA(cudaMemcpyAsync(th.data(), wvals, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  d->theta = th;
  d->k = k;
  d->n = n;
  return MM_OK;
}

int mm_deflation_build_apriori(mm_plan_t plan, int precision, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P) return fail(MM_EINVAL, "bad argument");
  if (precision != MM_FP64 && precision != MM_FP32) return fail(MM_EINVAL, "bad precision");
  if (P->algo == MM_TPLZ_DIRECT && precision == MM_FP32) precision = MM_FP64;
  const int k = P->n_int;
  if (k < 1 || k > kMaxDefl) return fail(MM_EINVAL, "the a-priori space needs 1 <= n_int <= 64 intervals");
  DeviceGuard g(P->device);
  cudaStream_t us = as_stream(stream);
  cudaStream_t s = P->stream;
  cudaEvent_t ev;
  MM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MM_CUDA(cudaEventRecord(ev, us));
  MM_CUDA(cudaStreamWaitEvent(s, ev, 0));
  cudaEventDestroy(ev);
  const int64_t n = P->n_obs, n4 = 4 * n;
  Scratch scr;
  int32_t* hits = nullptr;
  double *E = nullptr, *work = nullptr, *U = nullptr, *wvals = nullptr, *gpart = nullptr;
  MM_TRY(scr.alloc(&hits, (size_t)k * n));
  MM_TRY(scr.alloc(&E, kMaxDefl * kMaxDefl)); MM_TRY(scr.alloc(&work, kMaxDefl * kMaxDefl));
  MM_TRY(scr.alloc(&U, kMaxDefl * kMaxDefl)); MM_TRY(scr.alloc(&wvals, kMaxDefl));
  MM_TRY(scr.alloc(&gpart, (size_t)blk_ctas() * kMaxBlk * kMaxBlk));
  DeflState* d = reinterpret_cast<DeflState*>(P->defl);
  if (!d) {
    d = new DeflState();
    P->defl = d;
  }
  dfree(d->Z); dfree(d->Zp); dfree(d->Einv);
  d->k = 0;
  P->buf_gen++;
  MM_TRY(dalloc(P, &d->Z, (size_t)k * n4));
  MM_TRY(dalloc(P, &d->Zp, (size_t)k * n4));
  MM_TRY(dalloc(P, &d->Einv, (size_t)k * k));
  MM_CUDA(launch_apriori_z(P->lpix, P->block_off_dev, P->n_blocks, k, n, hits, d->Z, s));
  // Z' = A Z for the k columns at once
  if (precision == MM_FP32) {
    MM_CUDA(cudaMemsetAsync(d->Zp, 0, (size_t)k * n4 * sizeof(float), s));
    MM_TRY(apply32_internal(P, d->Z, d->Zp, k, s));
  } else {
    MM_TRY(ensure_maps(P, k, false));
    MM_TRY(ensure_df(P, k));
    MM_CUDA(launch_to64(d->Z, (int64_t)k * n, P->map64_in, s));
    MM_CUDA(cudaMemsetAsync(P->map64_out, 0, (size_t)k * n4 * sizeof(double), s));
    MM_TRY(apply64_internal(P, P->map64_in, P->map64_out, k, s));
    MM_CUDA(launch_to32(P->map64_out, (int64_t)k * n, d->Zp, s));
  }
  // E = Z^T Z', Einv = pinv(E)
  MM_CUDA(launch_bgram(d->Z, k, nullptr, d->Zp, 0, k, nullptr, n, gpart, blk_ctas(), E, s));
  MM_CUDA(launch_pinv_sym(E, k, 1e-12, work, U, wvals, d->Einv, s));
  MM_CUDA(cudaStreamSynchronize(s));
  d->theta.assign(k, 0.0);
  d->k = k;
  d->n = n;
  return MM_OK;
}

int mm_templates_set(mm_plan_t plan, const mm_templates_desc* t, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !t) return fail(MM_EINVAL, "bad argument");
  if (P->lambda != 0) return fail(MM_EINVAL, "template map-making uses diagonal weights: the plan's lambda must be 0");
  if (t->n_poly < 0 || t->n_poly > kMaxPoly) return fail(MM_EINVAL, "n_poly must lie in [0, 16]");
  if (t->n_az < 0 || t->n_az > kMaxTmpl) return fail(MM_EINVAL, "n_az must lie in [0, 64]");
  if (t->n_hwp < 0 || t->n_hwp > kMaxHwp) return fail(MM_EINVAL, "n_hwp must lie in [0, 8]");
  const int k = t->n_poly + t->n_az + 2 * t->n_hwp;
  for (int b = 0; b < P->n_blocks; b++)
    if (P->block_off[b + 1] - P->block_off[b] >= ((int64_t)1 << 31))
      return fail(MM_EINVAL, "template map-making needs blocks shorter than 2^31 samples");
  if (k < 1 || k > kMaxTmpl) return fail(MM_EINVAL, "n_poly + n_az + 2 n_hwp must lie in [1, 64]");
  if ((t->n_az > 0 && !t->az) || (t->n_hwp > 0 && !t->hwp)) return fail(MM_EINVAL, "az / hwp missing");
  DeviceGuard g(P->device);
  cudaStream_t us = as_stream(stream);
  cudaStream_t s = P->stream;
  cudaEvent_t ev;
  MM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MM_CUDA(cudaEventRecord(ev, us));
  MM_CUDA(cudaStreamWaitEvent(s, ev, 0));
  cudaEventDestroy(ev);
  free_tmpl(reinterpret_cast<TmplState*>(P->tmpl));
  P->tmpl = nullptr;
  P->buf_gen++;
  TmplState* ts = new TmplState();
  P->tmpl = ts;
  const int nb = P->n_blocks;
  const cudaMemcpyKind kind = t->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // the angles, int32 bins and FP64 fractions only feed the setup kernels: scratch, freed on return;
  // the operators keep uint8 bins, FP32 / df64 fractions and cos/sin of the HWP angle
  Scratch scr;
  float *az = nullptr, *hwp = nullptr;
  int32_t* az_bin = nullptr;
  double* az_frac = nullptr;
  if (t->n_az > 0) {
    MM_TRY(scr.alloc(&az, P->N));
    MM_TRY(scr.alloc(&az_bin, P->N));
    MM_TRY(dalloc(P, &ts->bin8, P->N));
    MM_CUDA(cudaMemcpyAsync(az, t->az, P->N * sizeof(float), kind, s));
    if (t->az_interp) {
      MM_TRY(scr.alloc(&az_frac, P->N));
      MM_TRY(dalloc(P, &ts->frac32, P->N));
      MM_TRY(dalloc(P, &ts->fracdf, P->N));
    }
  }
  if (t->n_hwp > 0) {
    MM_TRY(scr.alloc(&hwp, P->N));
    MM_TRY(dalloc(P, &ts->hwpdf, P->N));
    MM_TRY(dalloc(P, &ts->hwp32, P->N));
    MM_CUDA(cudaMemcpyAsync(hwp, t->hwp, P->N * sizeof(float), kind, s));
  }
  if (!P->wdf) {   // df64 pointing weights of the FP64-class template operator
    MM_TRY(dalloc(P, &P->wdf, P->N));
    MM_CUDA(launch_weights_df(P->psi, P->N, P->wdf, s));
  }
  // Legendre abscissa scale 2 / (n - 1) and the orthonormal rescaling sqrt((2k + 1) / n) per block
  std::vector<double> xs(nb), xo(nb), ps((size_t)nb * std::max(t->n_poly, 1));
  for (int b = 0; b < nb; b++) {
    const int64_t n = P->block_off[b + 1] - P->block_off[b];
    xs[b] = n > 1 ? 2.0 / (double)(n - 1) : 0.0;
    xo[b] = n > 1 ? 1.0 : 0.0;
    for (int q = 0; q < t->n_poly; q++) ps[(size_t)b * t->n_poly + q] = n > 0 ? std::sqrt((2.0 * q + 1.0) / (double)n) : 0.0;
  }
  MM_TRY(dalloc(P, &ts->xscale, nb));
  MM_TRY(dalloc(P, &ts->xoff, nb));
  MM_CUDA(cudaMemcpyAsync(ts->xoff, xo.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
  MM_TRY(dalloc(P, &ts->pscale, ps.size()));
  MM_TRY(dalloc(P, &ts->kinv, (size_t)nb * k * k));
  MM_CUDA(cudaMemcpyAsync(ts->xscale, xs.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemcpyAsync(ts->pscale, ps.data(), ps.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  TmplDev& d = ts->dev;
  d.n_poly = t->n_poly; d.n_az = t->n_az; d.n_hwp = t->n_hwp; d.interp = t->az_interp ? 1 : 0; d.k = k;
  d.n_total = P->N;
  d.off = P->block_off_dev; d.lpix = P->lpix; d.w = P->c0_blk; d.xscale = ts->xscale; d.xoff = ts->xoff;
  d.pscale = ts->pscale;
  d.az = az; d.hwp = hwp; d.az_bin = az_bin; d.az_frac = az_frac; d.kinv = ts->kinv;
  d.az_bin_w = az_bin; d.az_frac_w = az_frac; d.kinv_w = ts->kinv;
  d.bin8 = ts->bin8; d.frac32 = ts->frac32; d.bin8_w = ts->bin8; d.frac32_w = ts->frac32;
  d.fracdf = ts->fracdf; d.hwpdf = ts->hwpdf; d.fracdf_w = ts->fracdf; d.hwpdf_w = ts->hwpdf;
  d.hwp32 = ts->hwp32; d.hwp32_w = ts->hwp32;
  double* K = nullptr;
  MM_TRY(scr.alloc(&K, (size_t)nb * k * k));
  MM_CUDA(launch_tmpl_setup(d, nb, K, s));
  // M = P^T W P per pixel (the operator's diagonal-weight part), FP64 and FP32
  int32_t* hits = nullptr;
  MM_TRY(scr.alloc(&hits, P->n_obs));
  MM_TRY(dalloc(P, &ts->M64, 6 * P->n_obs));
  MM_TRY(dalloc(P, &ts->M32, 2 * P->n_obs));
  MM_CUDA(cudaMemsetAsync(ts->M64, 0, 6 * P->n_obs * sizeof(double), s));
  MM_CUDA(cudaMemsetAsync(hits, 0, P->n_obs * sizeof(int32_t), s));
  MM_CUDA(launch_bd_accum(P->lpix, P->w64, P->block_off_dev, P->c0_blk, nb, P->N, ts->M64, hits, s));
  MM_CUDA(launch_m64_to_32(ts->M64, P->n_obs, ts->M32, s));
  MM_CUDA(cudaStreamSynchronize(s));
  // the scratch inputs are gone once this returns
  d.az = nullptr; d.hwp = nullptr; d.az_bin = nullptr; d.az_frac = nullptr;
  d.az_bin_w = nullptr; d.az_frac_w = nullptr;
  return MM_OK;
}

int mm_deflation_get(mm_plan_t plan, int* k, double* Z, double* theta, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !k) return fail(MM_EINVAL, "bad argument");
  DeflState* d = reinterpret_cast<DeflState*>(P->defl);
  *k = d ? d->k : 0;
  if (!d || d->k == 0) return MM_OK;
  DeviceGuard g(P->device);
  cudaStream_t s = as_stream(stream);
  if (Z) {
    // float32 [k][n][4] -> float64 [k][n][3] through a temporary FP64 copy in the map buffers
    MM_TRY(ensure_maps(P, d->k, false));
    MM_CUDA(launch_to64(d->Z, (int64_t)d->k * P->n_obs, P->map64_in, s));
    MM_CUDA(launch_unpack4to3(P->map64_in, P->n_obs, d->k, Z, s));
  }
  if (theta) std::memcpy(theta, d->theta.data(), d->k * sizeof(double));
  return MM_OK;
}

int mm_deflation_apply(mm_plan_t plan, const double* r, double* z, int nrhs, void* stream) {
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (!P || !r || !z || nrhs <= 0) return fail(MM_EINVAL, "bad argument");
  DeflState* d = reinterpret_cast<DeflState*>(P->defl);
  if (!d || d->k == 0) return fail(MM_EINVAL, "no deflation space: call mm_deflation_build first");
  DeviceGuard g(P->device);
  cudaStream_t s = as_stream(stream);
  CgState* c = nullptr;
  MM_TRY(ensure_cg(P, nrhs, false, &c, s));
  CgWork w = make_work(P, c, nrhs, false, 1.0, 1);
  DeflWork dw{};
  MM_TRY(ensure_defl_work(P, d, nrhs, w.n_blocks, &dw, s));
  MM_CUDA(launch_pack3to4(r, P->n_obs, nrhs, c->r, s));
  MM_CUDA(cudaMemsetAsync(c->scal, 0, nrhs * sizeof(CgScalars), s));   // halt = 0
  MM_CUDA(launch_defl_step(dw, w, s));
  MM_CUDA(launch_unpack4to3(c->z, P->n_obs, nrhs, z, s));
  return MM_OK;
}

int mm_server_create(size_t hbm_budget, int max_slots, mm_server_t* out) {
  if (!out || max_slots < 1) return fail(MM_EINVAL, "bad argument");
  *out = nullptr;
  MM_TRY(tile_kernels_init());
  Server* S = new Server();
  cudaGetDevice(&S->device);
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    hbm_budget = (size_t)(0.8 * (double)fr);
  }
  S->budget = hbm_budget;
  S->max_slots = max_slots;
  const cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(e, "cudaStreamCreate");
  }
  S->th = std::thread(server_loop, S);
  constexpr int kPlanners = 4;
  for (int i = 0; i < kPlanners; i++) S->planners.emplace_back(planner_loop, S);
  *out = reinterpret_cast<mm_server_t>(S);
  return MM_OK;
}

int mm_submit(mm_server_t server, const mm_problem_desc* desc, const void* d, int d_is_fp32,
              const mm_solve_opts* opts, mm_req_t* id) {
  Server* S = reinterpret_cast<Server*>(server);
  if (!S || !desc || !d || !opts || !id) return fail(MM_EINVAL, "bad argument");
  MM_TRY(validate_desc(desc));
  if (desc->inputs_on_device) return fail(MM_EINVAL, "mm_submit takes host inputs");
  if (opts->precision != MM_FP32 && opts->precision != MM_FP64)
    return fail(MM_EINVAL, "opts->precision must be MM_FP32 or MM_FP64");
  if (desc->toeplitz_algo == MM_TPLZ_DIRECT) return fail(MM_EINVAL, "the server runs FFT plans");
  if (opts->precond != MM_PREC_BD) return fail(MM_EINVAL, "the server runs the block-Jacobi preconditioner");
  if (!(opts->tol > 0.0) || opts->max_iter < 0) return fail(MM_EINVAL, "bad tol / max_iter");
  Request* r = new Request();
  r->desc = *desc;
  const int nb = desc->n_det * desc->n_int;
  r->block_len.assign(desc->block_len, desc->block_len + nb);
  int64_t N = 0;
  for (int64_t v : r->block_len) {
    if (v < 0) { delete r; return fail(MM_EINVAL, "negative block length"); }
    N += v;
  }
  r->pix.copy_from(desc->pix, (size_t)N);
  r->psi.copy_from(desc->psi, (size_t)N);
  r->band.assign(desc->band, desc->band + (size_t)nb * (desc->lambda + 1));
  r->d_is_fp32 = d_is_fp32 ? 1 : 0;
  const unsigned char* db = reinterpret_cast<const unsigned char*>(d);
  r->d.copy_from(db, (size_t)N * (d_is_fp32 ? sizeof(float) : sizeof(double)));
  r->fp32 = opts->precision == MM_FP32;
  r->opts = *opts;
  r->footprint = estimate_footprint(*r);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(S->mu);
  r->id = S->next_id++;
  S->all[r->id] = r;
  S->queue.push_back(r);
  *id = r->id;
  S->cv_plan.notify_all();
  return MM_OK;
}

int mm_poll(mm_server_t server, mm_req_t id, mm_solve_info* info) {
  Server* S = reinterpret_cast<Server*>(server);
  if (!S) return fail(MM_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return fail(MM_EINVAL, "unknown request");
  if (it->second->state != 2) return MM_EBUSY;
  if (info) *info = it->second->info;
  return MM_OK;
}

int mm_wait(mm_server_t server, mm_req_t id, int64_t timeout_us, double* map_host, mm_solve_info* info) {
  Server* S = reinterpret_cast<Server*>(server);
  if (!S) return fail(MM_EINVAL, "bad argument");
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return fail(MM_EINVAL, "unknown request");
  Request* r = it->second;
  auto pred = [&] { return r->state == 2; };
  if (timeout_us < 0) {
    S->cv_done.wait(lock, pred);
  } else if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), pred)) {
    return fail(MM_ETIMEOUT, "request still running");
  }
  if (map_host && !r->map.empty()) std::memcpy(map_host, r->map.data(), r->map.size() * sizeof(double));
  if (info) *info = r->info;
  const int st = r->info.status;
  S->all.erase(it);
  delete r;
  if (st != MM_OK) set_error("request finished with an error status");
  return st;
}

void mm_server_destroy(mm_server_t server) {
  Server* S = reinterpret_cast<Server*>(server);
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
    S->cv_plan.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  for (std::thread& t : S->planners)
    if (t.joinable()) t.join();
  for (Request* r : S->ready) finish_request(S, r, MM_ECUDA);   // planned, never run
  S->ready.clear();
  for (auto& kv : S->all) delete kv.second;
  if (S->tiles_dev) cudaFree(S->tiles_dev);
  if (S->probs_dev) cudaFree(S->probs_dev);
  if (S->ntiles_dev) cudaFree(S->ntiles_dev);
  if (S->nprobs_dev) cudaFree(S->nprobs_dev);
  if (S->wgroups_dev) cudaFree(S->wgroups_dev);
  if (S->wprobs_dev) cudaFree(S->wprobs_dev);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // extern "C"
