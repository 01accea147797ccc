// In-shared-memory complex FFT used by the overlap-save Toeplitz tiles.
//
// Layout: MS complex values per CTA in shared memory with one padding element per 16
// (physical index i + i/16), which makes the strided radix-16 passes and the final
// short-stride pass free of bank conflicts for 8-byte (FP32) elements.
//
// Forward transform: decimation in frequency, radix-16 passes then one radix-2^REM pass;
// natural-order input, digit-reversed output.  Inverse: the same passes in reverse order
// (decimation in time), digit-reversed input, natural-order output, unnormalised.  Forward and
// inverse are used back to back with a pointwise step in between, so no reordering pass is run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

// Complex types whose products have their own overloads (double-float) set this to false, so a
// product that silently took the generic path would not compile.
template <typename C> struct GenericProduct { static constexpr bool value = true; };

template <typename C> __device__ __forceinline__ C c_add(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C c_sub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C c_mul(C a, C b) {
  static_assert(GenericProduct<C>::value, "complex type with its own product");
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C c_mulc(C a, C b) {
  static_assert(GenericProduct<C>::value, "complex type with its own product");
  return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

__host__ __device__ __forceinline__ constexpr int smem_pad(int i) { return i + (i >> 4); }

// cos(2 pi e / 16), sin(2 pi e / 16)
__device__ __forceinline__ constexpr double cos16(int e) {
  switch (e & 15) {
    case 0: return 1.0;
    case 1: return 0.92387953251128675613;
    case 2: return 0.70710678118654752440;
    case 3: return 0.38268343236508977173;
    case 4: return 0.0;
    case 5: return -0.38268343236508977173;
    case 6: return -0.70710678118654752440;
    case 7: return -0.92387953251128675613;
    case 8: return -1.0;
    case 9: return -0.92387953251128675613;
    case 10: return -0.70710678118654752440;
    case 11: return -0.38268343236508977173;
    case 12: return 0.0;
    case 13: return 0.38268343236508977173;
    case 14: return 0.70710678118654752440;
    default: return 0.92387953251128675613;
  }
}
__device__ __forceinline__ constexpr double sin16(int e) { return cos16(e - 4); }

// a * w16^e with w16 = exp(-2 pi i / 16) (FWD) or exp(+2 pi i / 16) (inverse).  After full
// unrolling e is a constant, so the axis cases cost nothing.
template <bool FWD, typename C>
__device__ __forceinline__ C rot16(C a, int e) {
  e &= 15;
  if (e == 0) return a;
  if (e == 8) return C{-a.x, -a.y};
  if (e == 4) return FWD ? C{a.y, -a.x} : C{-a.y, a.x};
  if (e == 12) return FWD ? C{-a.y, a.x} : C{a.y, -a.x};
  using T = decltype(a.x);
  const T c = (T)cos16(e);
  const T s = FWD ? (T)(-sin16(e)) : (T)sin16(e);
  return c_mul(a, C{c, s});
}

template <bool FWD, typename C>
__device__ __forceinline__ void dft2(C& a0, C& a1) {
  C t = a0;
  a0 = c_add(t, a1);
  a1 = c_sub(t, a1);
}

template <bool FWD, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C s02 = c_add(a0, a2), d02 = c_sub(a0, a2), s13 = c_add(a1, a3), d13 = c_sub(a1, a3);
  C jd = FWD ? C{d13.y, -d13.x} : C{-d13.y, d13.x};   // (-i or +i) * d13
  a0 = c_add(s02, s13);
  a2 = c_sub(s02, s13);
  a1 = c_add(d02, jd);
  a3 = c_sub(d02, jd);
}

// R-point DFT of a[0..R) into natural order (y_k = sum_m a_m w_R^{km}).
template <int R, bool FWD, typename C>
__device__ __forceinline__ void dft_small(C (&a)[R]) {
  if constexpr (R == 2) {
    dft2<FWD>(a[0], a[1]);
  } else if constexpr (R == 4) {
    dft4<FWD>(a[0], a[1], a[2], a[3]);
  } else if constexpr (R == 8) {
    // m = 2 m1 + m0, k = k0 + 4 k1
#pragma unroll
    for (int m0 = 0; m0 < 2; m0++) dft4<FWD>(a[m0], a[2 + m0], a[4 + m0], a[6 + m0]);
    // u[m0][k0] at a[2 k0 + m0]; twiddle w8^{m0 k0} = w16^{2 m0 k0}
#pragma unroll
    for (int k0 = 0; k0 < 4; k0++) a[2 * k0 + 1] = rot16<FWD>(a[2 * k0 + 1], 2 * k0);
    C b[8];
#pragma unroll
    for (int k0 = 0; k0 < 4; k0++) {
      C u0 = a[2 * k0], u1 = a[2 * k0 + 1];
      dft2<FWD>(u0, u1);
      b[k0] = u0;
      b[k0 + 4] = u1;
    }
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = b[i];
  } else {
    static_assert(R == 16, "radix");
    // m = 4 m1 + m0, k = k0 + 4 k1
#pragma unroll
    for (int m0 = 0; m0 < 4; m0++) dft4<FWD>(a[m0], a[4 + m0], a[8 + m0], a[12 + m0]);
    // u[m0][k0] now at a[4 k0 + m0]
#pragma unroll
    for (int k0 = 1; k0 < 4; k0++)
#pragma unroll
      for (int m0 = 1; m0 < 4; m0++) a[4 * k0 + m0] = rot16<FWD>(a[4 * k0 + m0], m0 * k0);
    C b[16];
#pragma unroll
    for (int k0 = 0; k0 < 4; k0++) {
      C u0 = a[4 * k0], u1 = a[4 * k0 + 1], u2 = a[4 * k0 + 2], u3 = a[4 * k0 + 3];
      dft4<FWD>(u0, u1, u2, u3);
      b[k0] = u0;
      b[k0 + 4] = u1;
      b[k0 + 8] = u2;
      b[k0 + 12] = u3;
    }
#pragma unroll
    for (int i = 0; i < 16; i++) a[i] = b[i];
  }
}

// Twiddle factors W_M^k, k in [0, M), from a two-level table in shared memory:
// W_M^k = hi[k >> 6] * lo[k & 63] with lo[i] = W_M^i (64 entries) and hi[i] = W_M^{64 i}
// (M / 64 entries); one complex product, accurate to a few ulp.
template <typename C>
struct TwiddleTab {
  const C* lo;
  const C* hi;
  __device__ __forceinline__ C operator()(int k) const { return c_mul(hi[k >> 6], lo[k & 63]); }
};
constexpr int twiddle_tab_entries(int m) { return 64 + m / 64; }

// Read-only load of one complex value; other complex types specialise it.
template <typename C>
__device__ __forceinline__ C ldg_c(const C* p) { return __ldg(p); }

// Fill the shared table from the global table tw[k] = W_M^k (called by all threads, then sync).
template <typename C, int MFULL, int NT>
__device__ __forceinline__ TwiddleTab<C> load_twiddle_tab(C* tab_sm, const C* __restrict__ tw) {
  for (int i = threadIdx.x; i < twiddle_tab_entries(MFULL); i += NT) {
    tab_sm[i] = (i < 64) ? ldg_c(tw + i) : ldg_c(tw + 64 * (i - 64));
  }
  return TwiddleTab<C>{tab_sm, tab_sm + 64};
}

// Twiddles w_j = W_C^{n1 j} = W_M^{n1 j (M / C)}, j = 1..R-1: powers 1, 2, 4, 8 from the table,
// the rest as products of two of those.
template <int R, typename C>
__device__ __forceinline__ void twiddles(const TwiddleTab<C>& tw, int base_idx, C (&w)[R]) {
  w[1] = tw(base_idx);
  if constexpr (R > 2) {
    w[2] = tw(2 * base_idx);
    w[3] = c_mul(w[1], w[2]);
  }
  if constexpr (R > 4) {
    w[4] = tw(4 * base_idx);
    w[5] = c_mul(w[4], w[1]);
    w[6] = c_mul(w[4], w[2]);
    w[7] = c_mul(w[4], w[3]);
  }
  if constexpr (R > 8) {
    w[8] = tw(8 * base_idx);
#pragma unroll
    for (int j = 1; j < 8; j++) w[8 + j] = c_mul(w[8], w[j]);
  }
}

// Pass tables of the radix-16 passes (R = 16): the 15 twiddles W^{j n1 M/CS} of offset n1, j = 1..15.
// FP32 complex values are stored in pairs, (j, j + 1) for j = 1, 3, .., 13 as one 16-byte entry of
// row (j - 1) / 2, then j = 15 alone in row 7 (float2 positions: pair row k at 2 k S + 2 n1, the last
// at 14 S + n1), so a butterfly reads its twiddles with 7 16-byte and one 8-byte load; other
// element types keep row j - 1 at (j - 1) S + n1.
template <typename C>
__host__ __device__ __forceinline__ constexpr bool paired_ptab() { return sizeof(C) == 8; }
template <typename C>
__host__ __device__ __forceinline__ int ptab_pos(int j, int s, int n1) {
  if constexpr (paired_ptab<C>()) return j == 15 ? 14 * s + n1 : (j - 1) / 2 * 2 * s + 2 * n1 + ((j - 1) & 1);
  else return (j - 1) * s + n1;
}
// a[j] *= twiddle j (CONJ: by its conjugate), j = 1 .. R - 1, from this pass's table
template <int R, bool CONJ, typename C>
__device__ __forceinline__ void ptab_twiddle(C (&a)[R], const C* __restrict__ ptab, int S, int n1) {
  if constexpr (paired_ptab<C>() && R == 16) {
    const float4* p4 = reinterpret_cast<const float4*>(ptab);
#pragma unroll
    for (int k = 0; k < 7; k++) {
      const float4 v = p4[k * S + n1];
      const C w0{v.x, v.y}, w1{v.z, v.w};
      a[2 * k + 1] = CONJ ? c_mulc(a[2 * k + 1], w0) : c_mul(a[2 * k + 1], w0);
      a[2 * k + 2] = CONJ ? c_mulc(a[2 * k + 2], w1) : c_mul(a[2 * k + 2], w1);
    }
    const C w15 = ptab[14 * S + n1];
    a[15] = CONJ ? c_mulc(a[15], w15) : c_mul(a[15], w15);
  } else {
#pragma unroll
    for (int j = 1; j < R; j++) a[j] = CONJ ? c_mulc(a[j], ptab[(j - 1) * S + n1]) : c_mul(a[j], ptab[(j - 1) * S + n1]);
  }
}

// One decimation-in-frequency (FWD) or decimation-in-time (inverse) pass over sub-transforms of
// size CS = R S with radix R and element stride S, over the MS points held by this CTA.
// `mfull_over_cs` = M / CS.  `ptab` (optional): this pass's twiddles precomputed as
// ptab[(j - 1) S + n1] = W_M^{j n1 M/CS}.
// The padded position of element m of a butterfly is its first element's padded position plus
// m S + (m S >> 4): the butterfly's first index and m S never carry across a 16-element padding
// group.  S_CT > 0 makes S a compile-time constant, so the 2R shared-memory accesses use immediate
// offsets; S_CT = 0 takes the stride s_rt at run time (one code body for several passes, for
// element types whose butterflies are long).
template <int R, bool FWD, int NT, int S_CT, int MS, typename C>
__device__ __forceinline__ void fft_pass(C* __restrict__ sm, const TwiddleTab<C>& tw, int s_rt,
                                         int mfull_over_cs, const C* __restrict__ ptab = nullptr) {
  constexpr int NBF = MS / R;
  const int S = S_CT > 0 ? S_CT : s_rt;
#pragma unroll 1
  for (int q = threadIdx.x; q < NBF; q += NT) {
    const int chunk = q / S;
    const int n1 = q - chunk * S;
    C* __restrict__ b = sm + smem_pad(chunk * (R * S) + n1);
    C a[R];
#pragma unroll
    for (int m = 0; m < R; m++) a[m] = b[m * S + ((m * S) >> 4)];
    if (FWD) {
      dft_small<R, true>(a);
      if (S > 1 && n1 != 0) {
        if (ptab) {
          ptab_twiddle<R, false>(a, ptab, S, n1);
        } else {
          C w[R];
          twiddles<R>(tw, n1 * mfull_over_cs, w);
#pragma unroll
          for (int j = 1; j < R; j++) a[j] = c_mul(a[j], w[j]);
        }
      }
    } else {
      if (S > 1 && n1 != 0) {
        if (ptab) {
          ptab_twiddle<R, true>(a, ptab, S, n1);
        } else {
          C w[R];
          twiddles<R>(tw, n1 * mfull_over_cs, w);
#pragma unroll
          for (int j = 1; j < R; j++) a[j] = c_mulc(a[j], w[j]);
        }
      }
      dft_small<R, false>(a);
    }
#pragma unroll
    for (int m = 0; m < R; m++) b[m * S + ((m * S) >> 4)] = a[m];
  }
}

// Transform of MS = 2^LOGMS points held by one CTA.  MFULL = size of the twiddle table's
// transform (the whole tile, MFULL >= MS).
// UNROLL_PASSES: one specialised body per radix-16 pass (compile-time strides) rather than one
// body looped over the passes.
template <int LOGMS, int MFULL, int NT, bool UNROLL_PASSES = true>
struct SmemFFT {
  static constexpr int MS = 1 << LOGMS;
  static constexpr int NP16 = LOGMS / 4;
  static constexpr int REM = LOGMS % 4;

  // Radix-16 passes p >= 1 have few distinct sub-transform offsets n1 (s = MS / 16^(p+1)), so
  // their 15 s twiddles are tabulated once per CTA in shared memory; pass 0 (s = MS / 16)
  // computes them from the two-level table.
  static constexpr int pass_s(int p) { return (MS >> (4 * p)) / 16; }
  static constexpr int pass_tab_offset(int p) {
    int o = 0;
    for (int q = 1; q < p; q++) o += 15 * pass_s(q);
    return o;
  }
  static constexpr int kPassTabEntries = pass_tab_offset(NP16);

  // Fill the pass tables (all threads; the caller synchronises before the first transform).
  template <typename C>
  __device__ static void build_pass_tables(C* ptab, const TwiddleTab<C>& tw) {
    for (int i = threadIdx.x; i < kPassTabEntries; i += NT) {
      int p = 1;
      while (p + 1 < NP16 && i >= pass_tab_offset(p + 1)) p++;
      const int s = pass_s(p);
      const int r = i - pass_tab_offset(p);
      const int j = r / s + 1, n1 = r % s;
      const int cs = MS >> (4 * p);
      ptab[pass_tab_offset(p) + ptab_pos<C>(j, s, n1)] = tw(j * n1 * (MFULL / cs));
    }
  }

  // radix-16 pass p (sub-transforms of MS / 16^p points), then a barrier
  template <int P, bool FWD, typename C>
  __device__ static void pass16(C* sm, const TwiddleTab<C>& tw, const C* ptab) {
    constexpr int CS = MS >> (4 * P);
    fft_pass<16, FWD, NT, CS / 16, MS>(sm, tw, CS / 16, MFULL / CS, P > 0 ? ptab + pass_tab_offset(P) : nullptr);
    __syncthreads();
  }
  template <bool FWD, typename C>
  __device__ static void pass16_rt(C* sm, const TwiddleTab<C>& tw, const C* ptab, int p) {
    const int cs = MS >> (4 * p);
    fft_pass<16, FWD, NT, 0, MS>(sm, tw, cs / 16, MFULL / cs, p > 0 ? ptab + pass_tab_offset(p) : nullptr);
    __syncthreads();
  }
  template <bool FWD, typename C>
  __device__ static void pass_rem(C* sm, const TwiddleTab<C>& tw) {
    if constexpr (REM > 0) {
      fft_pass<(1 << REM), FWD, NT, 1, MS>(sm, tw, 1, MFULL >> REM);
      __syncthreads();
    }
  }
  static_assert(NP16 == 3, "the tiles use 2^13 or 2^14 points per CTA");

  template <typename C>
  __device__ static void forward(C* sm, const TwiddleTab<C>& tw, const C* ptab) {
    if constexpr (UNROLL_PASSES) {
      pass16<0, true>(sm, tw, ptab);
      pass16<1, true>(sm, tw, ptab);
      pass16<2, true>(sm, tw, ptab);
    } else {
#pragma unroll 1
      for (int p = 0; p < NP16; p++) pass16_rt<true>(sm, tw, ptab, p);
    }
    pass_rem<true>(sm, tw);
  }

  // The radix-16 passes alone: the caller runs the stride-1 radix-2^REM passes (the last of the
  // forward transform, the first of the inverse) itself, fused with the pointwise step.
  template <typename C>
  __device__ static void forward16(C* sm, const TwiddleTab<C>& tw, const C* ptab) {
    pass16<0, true>(sm, tw, ptab);
    pass16<1, true>(sm, tw, ptab);
    pass16<2, true>(sm, tw, ptab);
  }
  template <typename C>
  __device__ static void inverse16(C* sm, const TwiddleTab<C>& tw, const C* ptab) {
    pass16<2, false>(sm, tw, ptab);
    pass16<1, false>(sm, tw, ptab);
    pass16<0, false>(sm, tw, ptab);
  }

  template <typename C>
  __device__ static void inverse(C* sm, const TwiddleTab<C>& tw, const C* ptab) {
    pass_rem<false>(sm, tw);
    if constexpr (UNROLL_PASSES) {
      pass16<2, false>(sm, tw, ptab);
      pass16<1, false>(sm, tw, ptab);
      pass16<0, false>(sm, tw, ptab);
    } else {
#pragma unroll 1
      for (int p = NP16 - 1; p >= 0; p--) pass16_rt<false>(sm, tw, ptab, p);
    }
  }

  // Position in shared memory (before padding) of frequency k after `forward`.
  __host__ __device__ static int storage_of(int k) {
    int j = 0;
#pragma unroll
    for (int i = 0; i < NP16; i++) j |= ((k >> (4 * i)) & 15) << (REM + 4 * (NP16 - 1 - i));
    if (REM > 0) j |= (k >> (4 * NP16)) & ((1 << REM) - 1);
    return j;
  }
  // Frequency held at position j after `forward`.
  __host__ __device__ static int freq_of(int j) {
    int k = 0;
#pragma unroll
    for (int i = 0; i < NP16; i++) k |= ((j >> (REM + 4 * (NP16 - 1 - i))) & 15) << (4 * i);
    if (REM > 0) k |= (j & ((1 << REM) - 1)) << (4 * NP16);
    return k;
  }
};

}  // namespace mm
