// Fused A-apply tiles: un-point -> banded block-Toeplitz product -> point, one overlap-save tile
// per CTA (FP32) or per 2-CTA cluster (FP64).
//
// The block-Toeplitz product y = T(c_b) t (Eq. MADCAP, stbmm of Sect. 3.1) is a linear
// convolution of each block with the symmetric kernel h = (c_lam..c_1, c_0, c_1..c_lam).
// Following the shift-and-overlap approach of Sect. 3.1, a block is cut into overlapping tiles
// of L = 32768 samples; each tile is transformed, multiplied by the kernel's spectrum on the
// L-point circulant, transformed back, and only the outputs whose whole band lies inside the
// tile are kept (L - 2 lam per tile).  Samples outside the block read as zero, so there is no
// wrap-around and no coupling between blocks.
//
// Real-input packing: the L real samples are packed as M = L/2 complex values
// z[n] = t[2n] + i t[2n+1].  Because the kernel is real and even, its spectrum H is real and the
// whole "unpack, multiply by H, repack" step reduces to a per-frequency pair update
//     Z'[k] = a_k Z[k] + i b_k conj(Z[M-k]),
//     a_k = (S_k - D_k sin th_k) / M,  b_k = D_k cos th_k / M,
//     S_k = (H_k + H_{M-k}) / 2,  D_k = (H_k - H_{M-k}) / 2,  th_k = 2 pi k / L,
// which is precomputed per band (in the FFT's storage order) at plan time.
//
// FP64: a 16384-point complex tile needs 256 KB, more than one CTA's shared memory.  The tile is
// split by one radix-2 decimation-in-frequency step done while gathering: CTA 0 transforms
// e[n] = z[n] + z[n+M/2] (the even frequencies), CTA 1 transforms o[n] = (z[n] - z[n+M/2]) W_M^n
// (the odd ones).  The pair update stays inside each CTA (k and M-k have the same parity), and
// the final radix-2 decimation-in-time step reads the partner CTA's half once through
// distributed shared memory.
#include <cooperative_groups.h>

#include <type_traits>

#include "df64.cuh"
#include "fft_smem.cuh"
#include "mm_internal.cuh"

namespace cg = cooperative_groups;

namespace mm {

namespace {

template <typename T> struct Map4;
template <> struct Map4<float> {
  // FP32 map: float4 per pixel (I, Q, U, 0)
  static __device__ __forceinline__ void load(const void* base, int64_t off, int32_t p, float& I,
                                              float& Q, float& U) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(base) + off / 4 + p);
    I = v.x; Q = v.y; U = v.z;
  }
  static __device__ __forceinline__ void add(void* base, int64_t off, int32_t p, float a, float b,
                                             float c) {
    atomicAdd(reinterpret_cast<float4*>(base) + off / 4 + p, make_float4(a, b, c, 0.f));
  }
};
template <> struct Map4<double> {
  static __device__ __forceinline__ void load(const void* base, int64_t off, int32_t p, double& I,
                                              double& Q, double& U) {
    const double2* b = reinterpret_cast<const double2*>(reinterpret_cast<const double*>(base) + off) +
                       2 * (int64_t)p;
    const double2 v0 = __ldg(b), v1 = __ldg(b + 1);
    I = v0.x; Q = v0.y; U = v1.x;
  }
  static __device__ __forceinline__ void add(void* base, int64_t off, int32_t p, double a, double b,
                                             double c) {
    double* q = reinterpret_cast<double*>(base) + off + 4 * (int64_t)p;
    atomicAdd(q, a);
    atomicAdd(q + 1, b);
    atomicAdd(q + 2, c);
  }
};
template <> struct Map4<df> {
  // df64 outputs accumulate into the FP64 map
  static __device__ __forceinline__ void add(void* base, int64_t off, int32_t p, df a, df b, df c) {
    double* q = reinterpret_cast<double*>(base) + off + 4 * (int64_t)p;
    atomicAdd(q, df_to_double(a));
    atomicAdd(q + 1, df_to_double(b));
    atomicAdd(q + 2, df_to_double(c));
  }
};

// ---- batched quad access --------------------------------------------------------------------
// The gather and scatter walk "quads" of 4 consecutive samples starting at a multiple of 4
// (tile windows start at multiples of 4).  A thread handles NQ quads at a time and issues all
// their independent loads before using any of them: first the pixel ids and weights, then the
// map values that depend on the pixel ids.  That keeps 2 x NQ memory round trips in flight per
// thread instead of one, which is what bounds a 16-warp CTA.

// Raw per-sample weight data: the (cos 2psi, sin 2psi) pair precomputed at plan time, in the
// precision of the tile (FP32 / FP64 / df64).
template <typename T> struct WRaw;
template <> struct WRaw<float> { float2 v; };
template <> struct WRaw<double> { double2 v; };
template <> struct WRaw<df> { float4 v; };   // (cos hi, cos lo, sin hi, sin lo)

template <typename T>
__device__ __forceinline__ void load_w(const TileArgs& a, int64_t g, WRaw<T>& w) {
  if constexpr (std::is_same<T, float>::value) w.v = __ldg(a.w32 + g);
  else if constexpr (std::is_same<T, df>::value) w.v = __ldg(a.wdf + g);
  else w.v = __ldg(a.w64 + g);
}
template <typename T>
__device__ __forceinline__ void weights_of(const WRaw<T>& w, T& c, T& s) {
  if constexpr (std::is_same<T, float>::value) {
    c = w.v.x;
    s = w.v.y;
  } else if constexpr (std::is_same<T, df>::value) {
    c = df_make(w.v.x, w.v.y);
    s = df_make(w.v.z, w.v.w);
  } else {
    c = w.v.x;
    s = w.v.y;
  }
}

// Pixel ids of the quad [g, g + 4) (-1 outside [lo, hi) or masked) and, when needed, weights.
template <typename T, bool NEED_W>
__device__ __forceinline__ void quad_meta(const TileArgs& a, int64_t g, int64_t lo, int64_t hi,
                                          int32_t (&p)[4], WRaw<T> (&w)[4]) {
  if (g >= lo && g + 4 <= hi) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(a.lpix + g));
    p[0] = v.x; p[1] = v.y; p[2] = v.z; p[3] = v.w;
    if (NEED_W) {
      if constexpr (std::is_same<T, float>::value) {
        const float4 f01 = __ldg(reinterpret_cast<const float4*>(a.w32 + g));
        const float4 f23 = __ldg(reinterpret_cast<const float4*>(a.w32 + g + 2));
        w[0].v = make_float2(f01.x, f01.y); w[1].v = make_float2(f01.z, f01.w);
        w[2].v = make_float2(f23.x, f23.y); w[3].v = make_float2(f23.z, f23.w);
      } else {
#pragma unroll
        for (int e = 0; e < 4; e++) load_w<T>(a, g + e, w[e]);
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const bool in = (g + e >= lo) && (g + e < hi);
      p[e] = in ? __ldg(a.lpix + g + e) : -1;
      if (NEED_W && in) load_w<T>(a, g + e, w[e]);
    }
  }
}

// Time-domain input values of NQ quads (0 outside the block and at masked samples).
template <typename T, int MODE, int NQ>
__device__ __forceinline__ void gather_quads(const TileArgs& a, int rhs, const TileDesc& td,
                                             const int64_t (&g)[NQ], T (&v)[NQ][4]) {
  if constexpr (MODE == MODE_NINV_T && std::is_same<T, float>::value) {
    // FP32 2-CTA tiles: float t, zero outside the block (g a multiple of 4: 16-byte aligned)
    const float* t = reinterpret_cast<const float*>(a.x) + rhs * a.x_stride;
#pragma unroll
    for (int u = 0; u < NQ; u++) {
      if (g[u] >= td.blk_lo && g[u] + 4 <= td.blk_hi) {
        const float4 f = __ldcs(reinterpret_cast<const float4*>(t + g[u]));
        v[u][0] = f.x; v[u][1] = f.y; v[u][2] = f.z; v[u][3] = f.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int64_t gg = g[u] + e;
          v[u][e] = (gg >= td.blk_lo && gg < td.blk_hi) ? __ldg(t + gg) : 0.f;
        }
      }
    }
  } else if constexpr (MODE == MODE_APPLY_T || MODE == MODE_NINV_T) {
    // df64 tiles: un-pointed input t = P x (or the masked TOD) as (hi, lo) pairs
    static_assert(std::is_same<T, df>::value, "2-CTA APPLY_T / NINV_T tiles are the df64 ones");
    const float2* t = reinterpret_cast<const float2*>(a.x) + rhs * a.x_stride;
#pragma unroll
    for (int u = 0; u < NQ; u++) {
      if (g[u] >= td.blk_lo && g[u] + 4 <= td.blk_hi) {
        const float4 v01 = __ldg(reinterpret_cast<const float4*>(t + g[u]));
        const float4 v23 = __ldg(reinterpret_cast<const float4*>(t + g[u] + 2));
        v[u][0] = df_make(v01.x, v01.y);
        v[u][1] = df_make(v01.z, v01.w);
        v[u][2] = df_make(v23.x, v23.y);
        v[u][3] = df_make(v23.z, v23.w);
      } else {
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int64_t gg = g[u] + e;
          if (gg >= td.blk_lo && gg < td.blk_hi) {
            const float2 f = __ldg(t + gg);
            v[u][e] = df_make(f.x, f.y);
          } else {
            v[u][e] = T(0);
          }
        }
      }
    }
  } else if constexpr (MODE == MODE_NINV) {
    const double* t = reinterpret_cast<const double*>(a.x) + rhs * a.x_stride;
#pragma unroll
    for (int u = 0; u < NQ; u++)
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int64_t gg = g[u] + e;
        v[u][e] = (gg >= td.blk_lo && gg < td.blk_hi) ? (T)__ldg(t + gg) : T(0);
      }
  } else {
    int32_t p[NQ][4];
    WRaw<T> w[NQ][4];
#pragma unroll
    for (int u = 0; u < NQ; u++) quad_meta<T, MODE == MODE_APPLY>(a, g[u], td.blk_lo, td.blk_hi, p[u], w[u]);
    if constexpr (MODE == MODE_RHS) {
#pragma unroll
      for (int u = 0; u < NQ; u++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
          T d = T(0);
          if (p[u][e] >= 0) {
            const int64_t gg = rhs * a.x_stride + g[u] + e;
            d = a.x_is_fp32 ? (T)__ldg(reinterpret_cast<const float*>(a.x) + gg)
                            : (T)__ldg(reinterpret_cast<const double*>(a.x) + gg);
          }
          v[u][e] = d;
        }
    } else {
      T I[NQ][4], Q[NQ][4], U[NQ][4];
#pragma unroll
      for (int u = 0; u < NQ; u++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
          I[u][e] = Q[u][e] = U[u][e] = T(0);
          if (p[u][e] >= 0) Map4<T>::load(a.x, rhs * a.x_stride, p[u][e], I[u][e], Q[u][e], U[u][e]);
        }
#pragma unroll
      for (int u = 0; u < NQ; u++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
          T c = T(0), s = T(0);
          if (p[u][e] >= 0) weights_of<T>(w[u][e], c, s);
          v[u][e] = (p[u][e] >= 0) ? I[u][e] + c * Q[u][e] + s * U[u][e] : T(0);
        }
    }
  }
}

// Accumulate (APPLY / RHS) or store (NINV) the outputs y of NQ quads; samples outside
// [out_lo, out_hi) are skipped.  Consecutive samples of one pixel are merged into one update.
template <typename T, int MODE, int NQ>
__device__ __forceinline__ void scatter_quads(const TileArgs& a, int rhs, const TileDesc& td,
                                              const int64_t (&g)[NQ], const T (&y)[NQ][4]) {
  if constexpr (MODE == MODE_NINV) {
    double* out = reinterpret_cast<double*>(a.y) + rhs * a.y_stride;
#pragma unroll
    for (int u = 0; u < NQ; u++)
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int64_t gg = g[u] + e;
        if (gg >= td.out_lo && gg < td.out_hi) out[gg] = (double)y[u][e];
      }
  } else {
    int32_t p[NQ][4];
    WRaw<T> w[NQ][4];
#pragma unroll
    for (int u = 0; u < NQ; u++) quad_meta<T, true>(a, g[u], td.out_lo, td.out_hi, p[u], w[u]);
#pragma unroll
    for (int u = 0; u < NQ; u++) {
      int32_t cur = -1;
      T acc0 = T(0), acc1 = T(0), acc2 = T(0);
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int32_t pe = p[u][e];
        if (pe != cur) {
          if (cur >= 0) Map4<T>::add(a.y, rhs * a.y_stride, cur, acc0, acc1, acc2);
          cur = pe;
          acc0 = acc1 = acc2 = T(0);
        }
        if (pe >= 0) {
          T c, s;
          weights_of<T>(w[u][e], c, s);
          const T ye = y[u][e];
          acc0 += ye;
          acc1 += c * ye;
          acc2 += s * ye;
        }
      }
      if (cur >= 0) Map4<T>::add(a.y, rhs * a.y_stride, cur, acc0, acc1, acc2);
    }
  }
}


// ---- strided pair access (one CTA per tile, FP32) -------------------------------------------
// Lane l of a warp handles complex value n0 + l (samples in0 + 2n, + 1), so one warp-wide load
// instruction covers 64 consecutive samples: the pointing loads are fully coalesced and the map
// gathers of a scan that moves a few pixels per sample fall on a few cache lines.  A thread keeps
// NB complex values (2 NB map loads) in flight.

// pixel ids and angles of the pair (g, g + 1), masked to [lo, hi)
template <typename T>
__device__ __forceinline__ void pair_meta(const TileArgs& a, int64_t g, int64_t lo, int64_t hi, bool need_w,
                                          int32_t (&p)[2], WRaw<T> (&w)[2]) {
  if (g >= lo && g + 2 <= hi) {
    const int2 v = __ldg(reinterpret_cast<const int2*>(a.lpix + g));
    p[0] = v.x; p[1] = v.y;
    if (need_w) {
      if constexpr (std::is_same<T, float>::value) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(a.w32 + g));
        w[0].v = make_float2(f.x, f.y); w[1].v = make_float2(f.z, f.w);
      } else {
        w[0].v = __ldg(a.w64 + g); w[1].v = __ldg(a.w64 + g + 1);
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < 2; e++) {
      const bool in = (g + e >= lo) && (g + e < hi);
      p[e] = in ? __ldg(a.lpix + g + e) : -1;
      if (need_w && in) load_w<T>(a, g + e, w[e]);
    }
  }
}

template <typename T, int MODE, int NB>
__device__ __forceinline__ void gather_pairs(const TileArgs& a, int rhs, const TileDesc& td,
                                             const int64_t (&g)[NB], T (&v)[NB][2]) {
  if constexpr (MODE == MODE_APPLY_T || MODE == MODE_NINV_T) {   // coalesced read of t, zero outside the block
    const float* t = reinterpret_cast<const float*>(a.x) + rhs * a.x_stride;
#pragma unroll
    for (int u = 0; u < NB; u++) {
      if (g[u] >= td.blk_lo && g[u] + 2 <= td.blk_hi) {   // g even and the column 8-byte aligned
        const float2 f = __ldcs(reinterpret_cast<const float2*>(t + g[u]));
        v[u][0] = f.x;
        v[u][1] = f.y;
      } else {
#pragma unroll
        for (int e = 0; e < 2; e++) {
          const int64_t gg = g[u] + e;
          v[u][e] = (gg >= td.blk_lo && gg < td.blk_hi) ? (T)__ldg(t + gg) : T(0);
        }
      }
    }
    return;
  }
  int32_t p[NB][2];
  WRaw<T> w[NB][2];
#pragma unroll
  for (int u = 0; u < NB; u++) pair_meta<T>(a, g[u], td.blk_lo, td.blk_hi, MODE == MODE_APPLY, p[u], w[u]);
  if constexpr (MODE == MODE_RHS) {
#pragma unroll
    for (int u = 0; u < NB; u++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        T d = T(0);
        if (p[u][e] >= 0) {
          const int64_t gg = rhs * a.x_stride + g[u] + e;
          d = a.x_is_fp32 ? (T)__ldg(reinterpret_cast<const float*>(a.x) + gg)
                          : (T)__ldg(reinterpret_cast<const double*>(a.x) + gg);
        }
        v[u][e] = d;
      }
  } else {
    T I[NB][2], Q[NB][2], U[NB][2];
#pragma unroll
    for (int u = 0; u < NB; u++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        I[u][e] = Q[u][e] = U[u][e] = T(0);
        if (p[u][e] >= 0) Map4<T>::load(a.x, rhs * a.x_stride, p[u][e], I[u][e], Q[u][e], U[u][e]);
      }
#pragma unroll
    for (int u = 0; u < NB; u++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        T c = T(0), s = T(0);
        if (p[u][e] >= 0) weights_of<T>(w[u][e], c, s);
        v[u][e] = (p[u][e] >= 0) ? I[u][e] + c * Q[u][e] + s * U[u][e] : T(0);
      }
  }
}

template <typename T, int MODE, int NB>
__device__ __forceinline__ void scatter_pairs(const TileArgs& a, int rhs, const TileDesc& td,
                                              const int64_t (&g)[NB], const T (&y)[NB][2]) {
  int32_t p[NB][2];
  WRaw<T> w[NB][2];
#pragma unroll
  for (int u = 0; u < NB; u++) pair_meta<T>(a, g[u], td.out_lo, td.out_hi, true, p[u], w[u]);
#pragma unroll
  for (int u = 0; u < NB; u++) {
    T c0 = T(0), s0 = T(0), c1 = T(0), s1 = T(0);
    if (p[u][0] >= 0) weights_of<T>(w[u][0], c0, s0);
    if (p[u][1] >= 0) weights_of<T>(w[u][1], c1, s1);
    const T y0 = y[u][0], y1 = y[u][1];
    if (p[u][0] >= 0 && p[u][0] == p[u][1]) {
      Map4<T>::add(a.y, rhs * a.y_stride, p[u][0], y0 + y1, c0 * y0 + c1 * y1, s0 * y0 + s1 * y1);
    } else {
      if (p[u][0] >= 0) Map4<T>::add(a.y, rhs * a.y_stride, p[u][0], y0, c0 * y0, s0 * y0);
      if (p[u][1] >= 0) Map4<T>::add(a.y, rhs * a.y_stride, p[u][1], y1, c1 * y1, s1 * y1);
    }
  }
}

// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16; a hint, no completion to wait for).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(bytes)
               : "memory");
}

// ---- fused stride-1 passes and pair update (FP32 tiles) ----------------------------------------
// After the three radix-16 passes of the forward transform (M = 2^14), position j of the
// digit-reversed layout holds the partial transform of frequency k with j = [d0|d1|d2|r]
// (k = d0 + 16 d1 + 256 d2 + 4096 r); the last forward pass is a radix-4 butterfly over the 4
// consecutive positions 4q..4q+3 (q = [d0|d1|d2]), and the first inverse pass the same.  The
// partner M - k of every frequency of quad q lies in a single quad q' (the first nonzero digit d
// of (d0, d1, d2) becomes 16 - d, the later digits 15 - d, element e pairs with element 3 - e;
// quad 0 pairs with itself with e <-> (4 - e) & 3, quad 8 with itself with e <-> 3 - e).  One
// thread therefore loads both quads, runs the last forward radix-4 on each, applies
// Z'[k] = a_k Z[k] + i b_k conj(Z[M - k]) and the first inverse radix-4, and stores them back:
// one shared-memory round trip instead of three.
__device__ __forceinline__ int partner_quad(int q) {
  const int a = q >> 8, b = (q >> 4) & 15, c = q & 15;
  if (a != 0) return ((16 - a) << 8) | ((15 - b) << 4) | (15 - c);
  if (b != 0) return ((16 - b) << 4) | (15 - c);
  if (c != 0) return 16 - c;
  return 0;
}

template <typename C, typename T>
__device__ __forceinline__ C pair_upd(C ab, C z, C zp, T sc) {
  // s (a Z + i b conj(Zp)) = s (a x + b yp, a y + b xp)
  return C{sc * (ab.x * z.x + ab.y * zp.y), sc * (ab.x * z.y + ab.y * zp.x)};
}

// The u-th quad q <= partner_quad(q) (2049 of them): a in 1..7; a = 8 with b < 8; a = 0 with b in
// 1..7; a = 0, b = 8 with c < 8; a = b = 0 with c in 1..7; then the two quads that pair with
// themselves, 8 and 0.
__device__ __forceinline__ int leader_quad(int u) {
  if (u < 1792) return ((1 + (u >> 8)) << 8) | (u & 255);
  if (u < 1920) return (8 << 8) | (u - 1792);
  if (u < 2032) return ((1 + ((u - 1920) >> 4)) << 4) | ((u - 1920) & 15);
  if (u < 2040) return (8 << 4) | (u - 2032);
  if (u < 2047) return 1 + (u - 2040);
  return u == 2047 ? 8 : 0;
}
constexpr int kLeaderQuads = 2049;

template <typename C, typename T>
__device__ __forceinline__ void fused_rem_pair(C* sm, const C* __restrict__ tab, T sc) {
  static_assert(kLogM == 14, "the quad pairing assumes 3 radix-16 passes and a radix-4 pass");
  for (int u = threadIdx.x; u < kLeaderQuads; u += kTileThreads) {
    const int q = leader_quad(u);
    const int p = partner_quad(q);
    C za[4], zb[4], ta[4], tb[4];
    C* qa = sm + smem_pad(4 * q);   // 4 consecutive positions never cross a padding group
    C* qb = sm + smem_pad(4 * p);
    if constexpr (std::is_same<C, float2>::value) {   // a quad's 4 table entries: two 16-byte loads
      const float4* t4a = reinterpret_cast<const float4*>(tab + 4 * q);
      const float4* t4b = reinterpret_cast<const float4*>(tab + 4 * p);
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const float4 va = __ldg(t4a + h), vb = __ldg(t4b + h);
        ta[2 * h] = C{va.x, va.y};
        ta[2 * h + 1] = C{va.z, va.w};
        tb[2 * h] = C{vb.x, vb.y};
        tb[2 * h + 1] = C{vb.z, vb.w};
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; e++) {
        ta[e] = ldg_c(tab + 4 * q + e);
        tb[e] = ldg_c(tab + 4 * p + e);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
      za[e] = qa[e];
      zb[e] = qb[e];
    }
    dft_small<4, true>(za);
    dft_small<4, true>(zb);
    if (p == q) {
      C o[4];
#pragma unroll
      for (int e = 0; e < 4; e++) o[e] = pair_upd(ta[e], za[e], za[q == 0 ? ((4 - e) & 3) : 3 - e], sc);
      dft_small<4, false>(o);
#pragma unroll
      for (int e = 0; e < 4; e++) qa[e] = o[e];
    } else {
      C oa[4], ob[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        oa[e] = pair_upd(ta[e], za[e], zb[3 - e], sc);
        ob[3 - e] = pair_upd(tb[3 - e], zb[3 - e], za[e], sc);
      }
      dft_small<4, false>(oa);
      dft_small<4, false>(ob);
#pragma unroll
      for (int e = 0; e < 4; e++) {
        qa[e] = oa[e];
        qb[e] = ob[e];
      }
    }
  }
}

}  // namespace

// One overlap-save tile (CL = 1) or half a tile (CL = 2) per CTA.
// LOGM: log2 of the complex points of the whole tile (L = 2^(LOGM + 1) real samples); the FP32
// 2-CTA tiles use LOGM = kLogM + 1 (65536 samples, each CTA a 16384-point half)
template <typename T, int CL, int MODE, bool MULTI = false, int LOGM = kLogM>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile(const TileArgs a_in) {
  constexpr int NT = kTileThreads;
  using C = typename V2<T>::t;
  constexpr int MT = 1 << LOGM;   // complex points of the tile
  constexpr int LT = 2 * MT;      // real samples of the tile
  constexpr int LOGMS = LOGM - (CL == 2 ? 1 : 0);
  constexpr int MS = 1 << LOGMS;
  // df64 butterflies are long: one pass body looped over the passes keeps the code in cache
  using FFT = SmemFFT<LOGMS, MT, NT, !std::is_same<T, df>::value>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  C* tw_sm = sm + smem_pad(MS);
  C* ptab = tw_sm + twiddle_tab_entries(MT);                          // per-pass twiddles
  T* halo = reinterpret_cast<T*>(ptab + FFT::kPassTabEntries);       // CL == 1 segments

  const int64_t unit = blockIdx.x / CL;
  const int rank = (CL == 2) ? (int)(blockIdx.x % CL) : 0;
  const int rhs = (int)(unit % a_in.nrhs);
  const int64_t tile_id = unit / a_in.nrhs;
  const TileDesc seg = a_in.tiles[tile_id];
  TileArgs a = a_in;
  if constexpr (MULTI) {   // this tile's problem
    const ProbPtrs pp = a_in.probs[seg.prob];
    a.lpix = pp.lpix; a.w32 = pp.w32; a.w64 = pp.w64; a.tab = pp.tab;
    a.x = pp.x; a.y = pp.y; a.done = pp.done;
  }
  // both CTAs of a cluster read the same flag, so they leave together
  if (a.done != nullptr && a.done[(int64_t)rhs * a.done_stride] != 0) return;
  const C* __restrict__ tw_g = reinterpret_cast<const C*>(a.tw);
  const TwiddleTab<C> tw = load_twiddle_tab<C, MT, NT>(tw_sm, tw_g);
  const C* __restrict__ tab =
      reinterpret_cast<const C*>(a.tab) + ((int64_t)seg.tab * CL + rank) * MS;
  const T sc = (T)seg.scale;
  constexpr int NQ = std::is_same<T, float>::value ? 4 : 2;
  constexpr int HALF_Q = MS / 2;          // quads (4 real samples) of this CTA's complex range
  const int halo_q = (LT - seg.vstep) / 4;
  __syncthreads();
  FFT::build_pass_tables(ptab, tw);
  __syncthreads();

  float umax = 0.f;   // MODE_NINV_T df64 tiles: largest |u| this thread wrote
  const int n_steps = (CL == 1) ? seg.n_steps : 1;   // only the FP32 kernel walks segments
  for (int step = 0; step < n_steps; step++) {
    TileDesc td = seg;
    td.in0 = seg.in0 + (int64_t)step * seg.vstep;
    td.out_lo = seg.out_lo + (int64_t)step * seg.vstep;
    td.out_hi = min(td.out_lo + (int64_t)seg.vstep, seg.out_hi);

    // ---- gather: packed complex input (CL = 2: with the first radix-2 DIF step) ----
    // quad q holds complex values 2q, 2q + 1 (real samples in0 + 4q .. + 3)
    if constexpr (CL == 1) {
      int q_first = 0;
      if (step > 0) {   // the previous tile's last L - vstep samples are this tile's first ones
        for (int n = threadIdx.x; n < 2 * halo_q; n += NT)
          sm[smem_pad(n)] = C{halo[2 * n], halo[2 * n + 1]};
        q_first = halo_q;
      }
      constexpr int NB = 8;
      const int n_first = 2 * q_first;
      for (int n0 = n_first + threadIdx.x; n0 < MS; n0 += NB * NT) {
        int64_t g[NB];
        T v[NB][2];
#pragma unroll
        for (int u = 0; u < NB; u++) {
          const int n = n0 + u * NT;
          g[u] = (n < MS) ? td.in0 + 2 * (int64_t)n : td.blk_hi;   // past the end: zeros
        }
        gather_pairs<T, MODE, NB>(a, rhs, td, g, v);
#pragma unroll
        for (int u = 0; u < NB; u++) {
          const int n = n0 + u * NT;
          if (n < MS) sm[smem_pad(n)] = C{v[u][0], v[u][1]};
        }
      }
      __syncthreads();
      if constexpr (MODE == MODE_NINV_T && std::is_same<T, float>::value) {
        // the next tile's new input samples [in0 + L, in0 + L + vstep) start on their way to L2 now,
        // so its gather finds them there instead of waiting on DRAM
        if (threadIdx.x == 0 && step + 1 < n_steps) {
          int64_t lo = max(td.in0 + LT, td.blk_lo), hi = min(td.in0 + LT + (int64_t)seg.vstep, td.blk_hi);
          lo = (lo + 3) & ~(int64_t)3;   // 16-byte aligned and inside the block
          hi &= ~(int64_t)3;
          if (hi > lo)
            prefetch_l2_bulk(reinterpret_cast<const float*>(a.x) + rhs * a.x_stride + lo, (uint32_t)((hi - lo) * 4));
        }
      }
      if (step + 1 < n_steps) {   // keep input samples [vstep, L) for the next tile
        const int n0 = seg.vstep / 2;
        for (int n = threadIdx.x; n < 2 * halo_q; n += NT) {
          const C z = sm[smem_pad(n0 + n)];
          halo[2 * n] = z.x;
          halo[2 * n + 1] = z.y;
        }
        __syncthreads();
      }
    } else {
      // pairs (quad q, quad q + MS/2): z[n] and z[n + MS] for n = 2q, 2q + 1
      for (int q0 = threadIdx.x; q0 < HALF_Q; q0 += (NQ / 2) * NT) {
        int64_t g[NQ];
        T v[NQ][4];
#pragma unroll
        for (int u = 0; u < NQ / 2; u++) {
          g[2 * u] = td.in0 + 4 * (int64_t)(q0 + u * NT);
          g[2 * u + 1] = g[2 * u] + 2 * (int64_t)MS;
        }
        gather_quads<T, MODE, NQ>(a, rhs, td, g, v);
#pragma unroll
        for (int u = 0; u < NQ / 2; u++) {
          const int q = q0 + u * NT;
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const int n = 2 * q + h;
            const C z{v[2 * u][2 * h], v[2 * u][2 * h + 1]};
            const C z2{v[2 * u + 1][2 * h], v[2 * u + 1][2 * h + 1]};
            sm[smem_pad(n)] = (rank == 0) ? c_add(z, z2) : c_mul(c_sub(z, z2), tw(n));
          }
        }
      }
      __syncthreads();
    }

    if constexpr (CL == 1 && LOGM == 14) {
      FFT::forward16(sm, tw, ptab);
      fused_rem_pair(sm, tab, sc);
      __syncthreads();
      FFT::inverse16(sm, tw, ptab);
    } else {
    FFT::forward(sm, tw, ptab);

    // ---- pair update with the band's precomputed (a_k, b_k) in storage order ----
    // Frequencies k and M - k pair up.  In the digit-reversed storage order the lowest frequency
    // digit d (base 16) is the top digit of the position, and the partner of a position with top
    // digit d in 1..15 has top digit 16 - d and the remaining digits complemented: so positions
    // with d in 1..7 pair upwards, d = 8 pairs within its own half, and only the d = 0 block
    // (k a multiple of 16) needs the general rule.  On the odd-frequency CTA of a cluster the
    // partner of position j is MS - 1 - j.  Work item u enumerates each pair once.
    {
      constexpr int D = MS / 16;
      const int n_items = (CL == 2 && rank == 1) ? MS / 2 : (7 * D + D / 2 + D);
      constexpr int PB = (MODE == MODE_APPLY && sizeof(T) == 4) ? 1 : 4;
      for (int u0 = threadIdx.x; u0 < n_items; u0 += PB * NT) {
        int jj[PB], jp[PB];
        bool act[PB];
        C ab[PB], abp[PB], z[PB], zp[PB];
#pragma unroll
        for (int b = 0; b < PB; b++) {
          const int u = u0 + b * NT;
          int j = 0, p = 0;
          bool ok = u < n_items;
          if (CL == 2 && rank == 1) {
            j = u;
            p = MS - 1 - u;
          } else if (u < 7 * D) {
            j = D + u;
            p = (16 - (j / D)) * D + (D - 1 - (j % D));
          } else if (u < 7 * D + D / 2) {
            j = 8 * D + (u - 7 * D);
            p = 8 * D + (D - 1 - (j % D));
          } else {
            j = u - (7 * D + D / 2);
            p = FFT::storage_of((MS - FFT::freq_of(j)) & (MS - 1));
            ok = ok && (j <= p);
          }
          jj[b] = j;
          jp[b] = p;
          act[b] = ok;
          if (ok) {
            ab[b] = ldg_c(tab + j);
            abp[b] = ldg_c(tab + p);
            z[b] = sm[smem_pad(j)];
            zp[b] = sm[smem_pad(p)];
          }
        }
#pragma unroll
        for (int b = 0; b < PB; b++) {
          if (!act[b]) continue;
          if (jj[b] == jp[b]) {
            sm[smem_pad(jj[b])] = C{sc * (ab[b].x * z[b].x + ab[b].y * z[b].y),
                                    sc * (ab[b].x * z[b].y + ab[b].y * z[b].x)};
          } else {
            // a Z + i b conj(Zp) = (a x + b yp, a y + b xp)
            sm[smem_pad(jj[b])] = C{sc * (ab[b].x * z[b].x + ab[b].y * zp[b].y),
                                    sc * (ab[b].x * z[b].y + ab[b].y * zp[b].x)};
            sm[smem_pad(jp[b])] = C{sc * (abp[b].x * zp[b].x + abp[b].y * z[b].y),
                                    sc * (abp[b].x * zp[b].y + abp[b].y * z[b].x)};
          }
        }
      }
    }
    __syncthreads();

    FFT::inverse(sm, tw, ptab);
    }

    // ---- scatter of the tile's valid outputs ----
    // output quads covering real offsets [r_lo, r_hi); rank r of a cluster owns complex indices
    // [r MS, (r + 1) MS), i.e. quads [r MS/2, (r + 1) MS/2)
    const int r_lo = (int)(td.out_lo - td.in0), r_hi = (int)(td.out_hi - td.in0);
    const C* other = sm;
    if constexpr (CL == 2) {
      cg::cluster_group cl = cg::this_cluster();
      if (rank == 1) {
        for (int n = threadIdx.x; n < MS; n += NT) {
          sm[smem_pad(n)] = c_mulc(sm[smem_pad(n)], tw(n));   // W_M^{-n} O'[n]
        }
      }
      cl.sync();
      other = cl.map_shared_rank(sm, rank ^ 1);
    }
    if constexpr (MODE == MODE_NINV_T && CL == 1) {
      // y of the tile's output range, float pairs (g even, so 8-byte aligned inside the range)
      float* yo = reinterpret_cast<float*>(a.y) + rhs * a.y_stride;
      const int n_lo = r_lo >> 1, n_hi = (r_hi + 1) >> 1;
      for (int n = n_lo + threadIdx.x; n < n_hi; n += NT) {
        const C z = sm[smem_pad(n)];
        const int64_t g = td.in0 + 2 * (int64_t)n;
        if (g >= td.out_lo && g + 2 <= td.out_hi) {
          __stcs(reinterpret_cast<float2*>(yo + g), make_float2(z.x, z.y));
        } else {
          if (g >= td.out_lo && g < td.out_hi) yo[g] = z.x;
          if (g + 1 >= td.out_lo && g + 1 < td.out_hi) yo[g + 1] = z.y;
        }
      }
    } else if constexpr (CL == 1) {
      constexpr int NB = 8;
      const int n_lo = r_lo >> 1, n_hi = (r_hi + 1) >> 1;
      for (int n0 = n_lo + threadIdx.x; n0 < n_hi; n0 += NB * NT) {
        int64_t g[NB];
        T y[NB][2];
#pragma unroll
        for (int u = 0; u < NB; u++) {
          const int n = n0 + u * NT;
          if (n < n_hi) {
            const C z = sm[smem_pad(n)];
            g[u] = td.in0 + 2 * (int64_t)n;
            y[u][0] = z.x;
            y[u][1] = z.y;
          } else {
            g[u] = td.out_hi;                          // outside the output range
            y[u][0] = y[u][1] = T(0);
          }
        }
        scatter_pairs<T, MODE, NB>(a, rhs, td, g, y);
      }
    } else {
      const int q_lo = max(r_lo >> 2, rank * HALF_Q);
      const int q_hi = min((r_hi + 3) >> 2, (rank + 1) * HALF_Q);
      for (int q0 = q_lo + threadIdx.x; q0 < q_hi; q0 += NQ * NT) {
        int64_t g[NQ];
        T y[NQ][4];
#pragma unroll
        for (int u = 0; u < NQ; u++) {
          const int q = q0 + u * NT;
          g[u] = td.in0 + 4 * (int64_t)q;
          if (q < q_hi) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
              const int n = 2 * q + h - rank * MS;      // local complex index
              C z = sm[smem_pad(n)];
              const C o = other[smem_pad(n)];
              z = (rank == 0) ? c_add(z, o) : c_sub(o, z);
              y[u][2 * h] = z.x;
              y[u][2 * h + 1] = z.y;
            }
          } else {
            g[u] = td.out_hi;                          // whole quad outside the output range
#pragma unroll
            for (int e = 0; e < 4; e++) y[u][e] = T(0);
          }
        }
        if constexpr (MODE == MODE_NINV_T && std::is_same<T, float>::value) {
          float* yo = reinterpret_cast<float*>(a.y) + rhs * a.y_stride;
#pragma unroll
          for (int u = 0; u < NQ; u++) {
            if (g[u] >= td.out_lo && g[u] + 4 <= td.out_hi) {   // g a multiple of 4: 16-byte aligned
              __stcs(reinterpret_cast<float4*>(yo + g[u]), make_float4(y[u][0], y[u][1], y[u][2], y[u][3]));
            } else {
#pragma unroll
              for (int e = 0; e < 4; e++)
                if (g[u] + e >= td.out_lo && g[u] + e < td.out_hi) yo[g[u] + e] = y[u][e];
            }
          }
        } else if constexpr (MODE == MODE_NINV_T) {
          // df64 u as (hi, lo) pairs over the tile's output range, and the CTA's max |u|
          float2* yo = reinterpret_cast<float2*>(a.y) + rhs * a.y_stride;
#pragma unroll
          for (int u = 0; u < NQ; u++) {
            if (g[u] >= td.out_lo && g[u] + 4 <= td.out_hi) {   // g a multiple of 4: 32-byte aligned
              float4* q4 = reinterpret_cast<float4*>(yo + g[u]);
              q4[0] = make_float4(y[u][0].hi, y[u][0].lo, y[u][1].hi, y[u][1].lo);
              q4[1] = make_float4(y[u][2].hi, y[u][2].lo, y[u][3].hi, y[u][3].lo);
            } else {
#pragma unroll
              for (int e = 0; e < 4; e++)
                if (g[u] + e >= td.out_lo && g[u] + e < td.out_hi) yo[g[u] + e] = make_float2(y[u][e].hi, y[u][e].lo);
            }
#pragma unroll
            for (int e = 0; e < 4; e++)
              if (g[u] + e >= td.out_lo && g[u] + e < td.out_hi) {
                const float m = fabsf(y[u][e].hi);
                umax = (m == m) ? fmaxf(umax, m) : __int_as_float(0x7f800000);   // NaN -> +inf
              }
          }
        } else {
          scatter_quads<T, MODE, NQ>(a, rhs, td, g, y);
        }
      }
    }
    if constexpr (CL == 2) cg::this_cluster().sync();
    else __syncthreads();   // the next tile overwrites the buffer
  }
  if constexpr (MODE == MODE_NINV_T && CL == 2 && std::is_same<T, df>::value) {
    if (a.amax != nullptr) {   // non-negative floats order like their bit patterns
      for (int o = 16; o > 0; o >>= 1) umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
      if ((threadIdx.x & 31) == 0) atomicMax(a.amax + rhs, __float_as_uint(umax));
    }
  }
}

constexpr size_t kSmemBytes32 =
    (size_t)(smem_pad(kM) + twiddle_tab_entries(kM) + SmemFFT<kLogM, kM, kTileThreads>::kPassTabEntries) *
    sizeof(float2);
constexpr size_t kSmemMax = 227 * 1024;
constexpr size_t kSmemBytes32Big =
    (size_t)(smem_pad(kM) + twiddle_tab_entries(2 * kM) + SmemFFT<kLogM, 2 * kM, kTileThreads>::kPassTabEntries) *
    sizeof(float2);
constexpr size_t kSmemBytes64 =
    (size_t)(smem_pad(kM / 2) + twiddle_tab_entries(kM) + SmemFFT<kLogM - 1, kM, kTileThreads>::kPassTabEntries) *
    sizeof(double2);

int tile_kernels_init() {
  static int done = 0;
  static int status = MM_OK;
  if (done) return status;
  done = 1;
  cudaError_t e = cudaSuccess;
#define MM_SET(K, B)                                                                       \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(B));
  MM_SET((k_tile<float, 1, MODE_APPLY>), kSmemMax);
  MM_SET((k_tile<float, 1, MODE_RHS>), kSmemMax);
  MM_SET((k_tile<float, 1, MODE_APPLY, true>), kSmemMax);
  MM_SET((k_tile<float, 1, MODE_NINV_T, true>), kSmemMax);
  MM_SET((k_tile<float, 1, MODE_APPLY_T>), kSmemMax);
  MM_SET((k_tile<float, 1, MODE_NINV_T>), kSmemMax);
  MM_SET((k_tile<double, 2, MODE_APPLY>), kSmemBytes64);
  MM_SET((k_tile<double, 2, MODE_RHS>), kSmemBytes64);
  MM_SET((k_tile<double, 2, MODE_NINV>), kSmemBytes64);
  MM_SET((k_tile<df, 2, MODE_APPLY_T>), kSmemBytes64);
  MM_SET((k_tile<df, 2, MODE_NINV_T>), kSmemBytes64);
  MM_SET((k_tile<float, 2, MODE_NINV_T, false, kLogM + 1>), kSmemBytes32Big);
#undef MM_SET
  if (e == cudaSuccess) {
    // 2-CTA clusters with 136 KB of dynamic shared memory each are a non-portable size only in
    // CTA count terms; allow it explicitly.
    e = cudaFuncSetAttribute((k_tile<double, 2, MODE_APPLY>), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  if (e != cudaSuccess) status = cuda_fail(e, "tile kernel attributes");
  return status;
}

template <typename T, int CL, int MODE, bool MULTI = false, int LOGM = kLogM>
static cudaError_t launch_tiles(const TileArgs& a, size_t smem, cudaStream_t s) {
  const int64_t n_cta = a.n_tiles * a.nrhs * CL;
  if (n_cta == 0) return cudaSuccess;
  if (n_cta > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_cta);
  cfg.blockDim = dim3(kTileThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  int na = 0;
  if (CL > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    na = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, k_tile<T, CL, MODE, MULTI, LOGM>, a);
}

// FP32 u = N^-1 t on 65536-sample tiles, each a 2-CTA cluster (t, u [nrhs][stride], strides
// multiples of 4; tables of the 32768-point transform)
cudaError_t launch_ninv32_big(const TileArgs& a, cudaStream_t s) {
  if (a.x_stride % 4 != 0 || a.y_stride % 4 != 0) return cudaErrorInvalidValue;
  return launch_tiles<float, 2, MODE_NINV_T, false, kLogM + 1>(a, kSmemBytes32Big, s);
}

// FP32 segments; halo_samples = largest L - vstep of the segments that walk more than one tile
cudaError_t launch_tiles_fp32(int mode, const TileArgs& a, int halo_samples, cudaStream_t s) {
  const size_t smem = kSmemBytes32 + (size_t)halo_samples * sizeof(float);
  if (smem > kSmemMax) return cudaErrorInvalidValue;
  if (mode == MODE_APPLY) return launch_tiles<float, 1, MODE_APPLY>(a, smem, s);
  if (mode == MODE_APPLY_T) return launch_tiles<float, 1, MODE_APPLY_T>(a, smem, s);
  if (mode == MODE_NINV_T) return launch_tiles<float, 1, MODE_NINV_T>(a, smem, s);
  if (mode == MODE_RHS) return launch_tiles<float, 1, MODE_RHS>(a, smem, s);
  return cudaErrorInvalidValue;
}

// t = P x over all samples at full occupancy: lane = sample, so pointing loads coalesce and the map
// gathers of a scan stay on a few cache lines per warp; the random loads of many warps overlap.
__global__ void __launch_bounds__(256) k_unpoint32(const int32_t* __restrict__ lpix,
                                                   const float2* __restrict__ w, int64_t N,
                                                   const float4* __restrict__ x4, int64_t x_stride4,
                                                   const int32_t* __restrict__ done, int done_stride,
                                                   float* __restrict__ t, int64_t t_stride) {
  const int rhs = blockIdx.y;
  if (done != nullptr && done[(int64_t)rhs * done_stride] != 0) return;
  const float4* x = x4 + rhs * x_stride4;
  float* tr = t + rhs * t_stride;
  constexpr int U = 4;
  for (int64_t i0 = (int64_t)blockIdx.x * 256 * U + threadIdx.x; i0 < N; i0 += (int64_t)gridDim.x * 256 * U) {
    int32_t p[U];
    float2 cs[U];
    float4 m[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = i0 + u * 256;
      p[u] = (i < N) ? __ldg(lpix + i) : -1;
      cs[u] = (i < N) ? __ldg(w + i) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; u++) m[u] = (p[u] >= 0) ? __ldg(x + p[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = i0 + u * 256;
      if (i < N) tr[i] = (p[u] >= 0) ? m[u].x + cs[u].x * m[u].y + cs[u].y * m[u].z : 0.f;
    }
  }
}

cudaError_t launch_unpoint32(const int32_t* lpix, const float2* w32, int64_t N, const float* x4,
                             int64_t x_stride, int nrhs, const int32_t* done, int done_stride, float* t,
                             int64_t t_stride, cudaStream_t s) {
  if (N == 0 || nrhs <= 0) return cudaSuccess;
  int64_t g = (N + 1023) / 1024;
  if (g > 16 * sm_count()) g = 16 * sm_count();
  k_unpoint32<<<dim3((unsigned)g, nrhs), 256, 0, s>>>(lpix, w32, N, reinterpret_cast<const float4*>(x4),
                                                     x_stride / 4, done, done_stride, t, t_stride);
  return cudaGetLastError();
}

cudaError_t launch_tiles_fp32_multi(const TileArgs& a, int halo_samples, cudaStream_t s) {
  const size_t smem = kSmemBytes32 + (size_t)halo_samples * sizeof(float);
  if (smem > kSmemMax || a.nrhs != 1 || a.probs == nullptr) return cudaErrorInvalidValue;
  return launch_tiles<float, 1, MODE_APPLY, true>(a, smem, s);
}

cudaError_t launch_ninv32_multi(const TileArgs& a, int halo_samples, cudaStream_t s) {
  const size_t smem = kSmemBytes32 + (size_t)halo_samples * sizeof(float);
  if (smem > kSmemMax || a.nrhs != 1 || a.probs == nullptr) return cudaErrorInvalidValue;
  return launch_tiles<float, 1, MODE_NINV_T, true>(a, smem, s);
}

int fp32_max_halo_samples() { return (int)((kSmemMax - kSmemBytes32) / sizeof(float)); }

// df64 tiles: input t (float2 hi/lo pairs [nrhs][x_stride], x_stride a multiple of 4), output
// accumulated into the FP64 map y [nrhs][n_obs][4]
cudaError_t launch_tiles_df(const TileArgs& a, cudaStream_t s) {
  if (a.x_stride % 4 != 0) return cudaErrorInvalidValue;
  return launch_tiles<df, 2, MODE_APPLY_T>(a, kSmemBytes64, s);
}

// df64 u = N^-1 t: t and u (hi, lo) pairs [nrhs][x_stride] / [nrhs][y_stride] (multiples of 4),
// a.amax (per column, zeroed by the caller) receives the bits of max |u|
cudaError_t launch_ninv_df(const TileArgs& a, cudaStream_t s) {
  if (a.x_stride % 4 != 0 || a.y_stride % 4 != 0) return cudaErrorInvalidValue;
  return launch_tiles<df, 2, MODE_NINV_T>(a, kSmemBytes64, s);
}

cudaError_t launch_tiles_fp64(int mode, const TileArgs& a, cudaStream_t s) {
  if (mode == MODE_APPLY) return launch_tiles<double, 2, MODE_APPLY>(a, kSmemBytes64, s);
  if (mode == MODE_RHS) return launch_tiles<double, 2, MODE_RHS>(a, kSmemBytes64, s);
  if (mode == MODE_NINV) return launch_tiles<double, 2, MODE_NINV>(a, kSmemBytes64, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// plan-time tables
// ---------------------------------------------------------------------------------------------

// H_j = c_0 + 2 sum_{tau=1}^{lam} c_tau cos(2 pi tau j / L), j = 0..M: the L-point circulant
// spectrum of the band (real and even because the kernel is symmetric); L = 2M = 2^(logm + 1)
__global__ void k_spectra(const double* __restrict__ band_rows, int32_t lambda,
                          const double* __restrict__ costab, double* __restrict__ H, int logm) {
  extern __shared__ double c_s[];
  const int m = 1 << logm, l = 2 * m;
  const int tab = blockIdx.y;
  const double* c = band_rows + (int64_t)tab * (lambda + 1);
  for (int i = threadIdx.x; i <= lambda; i += blockDim.x) c_s[i] = c[i];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > m) return;
  double acc = 0.0;
  for (int tau = 1; tau <= lambda; tau++) {
    acc = fma(c_s[tau], __ldg(costab + (((int64_t)tau * j) & (l - 1))), acc);
  }
  H[(int64_t)tab * (m + 1) + j] = c_s[0] + 2.0 * acc;
}

cudaError_t launch_spectra(const double* band_rows, int32_t n_tab, int32_t lambda, double* H,
                           const double* costab, cudaStream_t s, int logm) {
  if (n_tab == 0) return cudaSuccess;
  const int nt = 256, m = 1 << logm;
  const size_t sm = (size_t)(lambda + 1) * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (sm > 48 * 1024) e = cudaFuncSetAttribute(k_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  for (int32_t t0 = 0; t0 < n_tab; t0 += 65535) {   // gridDim.y limit
    const int32_t nt_y = (n_tab - t0) < 65535 ? (n_tab - t0) : 65535;
    dim3 grid((m + 1 + nt - 1) / nt, nt_y);
    k_spectra<<<grid, nt, sm, s>>>(band_rows + (int64_t)t0 * (lambda + 1), lambda, costab,
                                   H + (int64_t)t0 * (m + 1), logm);
  }
  return cudaGetLastError();
}

// (a_k, b_k) of the pair update for every storage position of a tile of 2^LOGM complex points
// split over CL CTAs (the storage order of each CTA's transform)
template <int CL, int LOGM>
__global__ void k_pair_table(const double* __restrict__ H, const double* __restrict__ costab,
                             int32_t n_tab, void* __restrict__ out, int fp32) {
  constexpr int M = 1 << LOGM, L = 2 * M;
  constexpr int LOGMS = LOGM - (CL == 2 ? 1 : 0);
  constexpr int MS = 1 << LOGMS;
  using FFT = SmemFFT<LOGMS, M, kTileThreads>;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_tab * M) return;
  const int tab = (int)(idx / M);
  const int rem = (int)(idx % M);
  const int rank = rem / MS, j = rem % MS;
  const int k = CL * FFT::freq_of(j) + rank;       // global frequency, 0 <= k < M
  const double* h = H + (int64_t)tab * (M + 1);
  const double S = 0.5 * (h[k] + h[M - k]);
  const double D = 0.5 * (h[k] - h[M - k]);
  const double cth = costab[k];
  const double sth = costab[(k - L / 4) & (L - 1)];
  const double inv_m = 1.0 / (double)M;
  const double av = (S - D * sth) * inv_m;
  const double bv = D * cth * inv_m;
  if (fp32) reinterpret_cast<float2*>(out)[idx] = make_float2((float)av, (float)bv);
  else reinterpret_cast<double2*>(out)[idx] = make_double2(av, bv);
}

cudaError_t launch_pair_tables(const double* H, int32_t n_tab, const double* costab, double2* tab64,
                               float2* tab32, cudaStream_t s) {
  if (n_tab == 0) return cudaSuccess;
  const int64_t n = (int64_t)n_tab * kM;
  const int nt = 256;
  const unsigned nb = (unsigned)((n + nt - 1) / nt);
  k_pair_table<kCl64, kLogM><<<nb, nt, 0, s>>>(H, costab, n_tab, tab64, 0);
  k_pair_table<kCl32, kLogM><<<nb, nt, 0, s>>>(H, costab, n_tab, tab32, 1);
  return cudaGetLastError();
}

// FP32 pair tables of the 65536-sample 2-CTA tiles (H and costab of that length)
cudaError_t launch_pair_table32_big(const double* H, int32_t n_tab, const double* costab, float2* tab32,
                                    cudaStream_t s) {
  if (n_tab == 0) return cudaSuccess;
  const int64_t n = (int64_t)n_tab * 2 * kM;
  k_pair_table<2, kLogM + 1><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(H, costab, n_tab, tab32, 1);
  return cudaGetLastError();
}

// tw[k] = W_M^k = exp(-2 pi i k / M) = cos(2 pi 2k / L) - i sin(2 pi 2k / L), M = 2^logm
__global__ void k_twiddles(double2* tw64, float2* tw32, const double* __restrict__ costab, int logm) {
  const int m = 1 << logm, l = 2 * m;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const double c = costab[(2 * k) & (l - 1)];
  const double s = costab[(2 * k - l / 4) & (l - 1)];
  if (tw64) tw64[k] = make_double2(c, -s);
  tw32[k] = make_float2((float)c, (float)-s);
}

cudaError_t launch_twiddles(double2* tw64, float2* tw32, const double* costab, cudaStream_t s, int logm) {
  const int m = 1 << logm;
  k_twiddles<<<(m + 255) / 256, 256, 0, s>>>(tw64, tw32, costab, logm);
  return cudaGetLastError();
}

}  // namespace mm
