// slab.cuh -- the register-tiled (min,+) slab arithmetic shared by the TMA-fed GEMM engine
// (tgemm.cu) and the batched persistent kernel (batched.cu).
//
// A 256-thread consumer group owns a 128 x 128 output tile; thread (tm, tn) holds rows
// tm + 16 i and columns 4 tn + q + 64 h (i, h, q) in an 8 x 8 register tile.  A k-slab is
// 32 deep: A as [128 m][32 k] with 128-byte swizzle (a_off), B as [32 k][128 n].
#pragma once

#include "common.cuh"

namespace apsp {

constexpr int kSlabM = 128, kSlabN = 128, kSlabK = 32;

// Unroll factor of the loop over the eight 4-deep k-quads of a slab.
#ifndef APSP_Q_UNROLL
#define APSP_Q_UNROLL 2
#endif
constexpr int kQUnroll = APSP_Q_UNROLL;

// Offset (in elements) of the 16-byte chunk kq (k = 4 kq .. 4 kq + 3) of row r of an A slab.
// The slab is TMA-loaded with 128-byte swizzle: chunk kq of row r sits at chunk kq ^ (r & 7),
// so the four rows a warp reads at once fall in four different bank groups.
__device__ __forceinline__ int a_off(int r, int kq) { return r * kSlabK + ((kq ^ (r & 7)) << 2); }

// ---------------------------------------------------------------------------------------
// Consumer arithmetic.  Both variants compute acc[i][j] = min(acc[i][j], A[r_i][k] + B[k][c_j])
// over a 32-deep k-slab held in shared memory; they differ only in the instruction sequence.
//
// ArithF32: fp32 arithmetic.  Two consecutive k are handled at once: one packed pair add
//   (add.rn.f32x2) forms {A[i][k] + B[k][j], A[i][k+1] + B[k+1][j]} and one 3-input min folds
//   both into the accumulator -- one issued instruction per (min,+) pair, the best rate the
//   probes measure on this chip.  It also serves int32 matrices whose every shortest distance
//   is below 2^24: an int32 bit pattern v < 2^24 read as fp32 is the number v * 2^-149, sums
//   below 2^24 * 2^-149 are exact, and rounding is monotone, so a rounded (>= 2^24) candidate
//   can never undercut an exact one -- the min is bit-exact and so is its bit pattern.
// ArithI32: the int32 fallback for larger weights: two fused add-min DPX operations
//   (__viaddmin_s32) per accumulator and k-pair.
// ---------------------------------------------------------------------------------------
struct ArithF32 {
  typedef float T;
  static constexpr bool kFloat = true;
  static __device__ __forceinline__ T from(int v) { return __int_as_float(v); }
  static __device__ __forceinline__ int to(T v) { return __float_as_int(v); }
  static __device__ __forceinline__ T mn(T a, T b) { return fminf(a, b); }
  static __device__ __forceinline__ T collapse(T v, int) { return v; }
  static __device__ __forceinline__ T collapse_truncated(T v) { return v; }
  // Column pairs: {A[i][k], A[i][k]} + {B[k][c], B[k][c+1]} in one packed add (the B pair comes
  // straight from a 128-bit load, the duplicated A value is built once per row and k), the
  // four adds of one duplicated A value issued back to back so it stays in the operand reuse
  // cache, then one 3-input min folds k and k+1 into each accumulator.
  // HALF (bit 0: rows, bit 1: columns): only rows 0..63 and / or columns 0..63 of the tile are
  // computed -- register rows i < 4 and column quads h = 0; the others keep their initial
  // value.  Used for the last block of a padded graph, whose other half is padding.
  template <int HALF = 0>
  static __device__ __forceinline__ void slab_full(const int *As, const int *Bs, int tm, int tn, T (&acc)[8][8]) {
    constexpr bool MASKED = HALF != 0, fr = !(HALF & 1), fc = !(HALF & 2);
#pragma unroll kQUnroll
    for (int q = 0; q < kSlabK / 4; ++q) {
      float4 a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (MASKED && i >= 4 && !fr) {
          a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          continue;
        }
        const int4 v = lds128(As + a_off(tm + 16 * i, q));
        a[i] = make_float4(__int_as_float(v.x), __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w));
      }
#pragma unroll
      for (int kp = 0; kp < 2; ++kp) {
        const int *r0 = Bs + (4 * q + 2 * kp) * kSlabN + 4 * tn;
        uint64_t b0[4], b1[4];
        lds128_2x64(r0, b0[0], b0[1]);
        lds128_2x64(r0 + kSlabN, b1[0], b1[1]);
        if (!MASKED || fc) {
          lds128_2x64(r0 + 64, b0[2], b0[3]);
          lds128_2x64(r0 + kSlabN + 64, b1[2], b1[3]);
        } else {
          b0[2] = b0[3] = b1[2] = b1[3] = 0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (MASKED && i >= 4 && !fr) continue;
          const float a0 = kp ? a[i].z : a[i].x, a1 = kp ? a[i].w : a[i].y;
          const uint64_t aa0 = pack2(a0, a0), aa1 = pack2(a1, a1);
          uint64_t t0[4], t1[4];
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) {
            if (MASKED && jp >= 2 && !fc) continue;
            t0[jp] = fadd2_64(aa0, b0[jp]);
          }
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) {
            if (MASKED && jp >= 2 && !fc) continue;
            t1[jp] = fadd2_64(aa1, b1[jp]);
          }
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) {
            if (MASKED && jp >= 2 && !fc) continue;
            acc[i][2 * jp] = Ops<float>::min3(acc[i][2 * jp], lo_of(t0[jp]), lo_of(t1[jp]));
            acc[i][2 * jp + 1] = Ops<float>::min3(acc[i][2 * jp + 1], hi_of(t0[jp]), hi_of(t1[jp]));
          }
        }
      }
    }
  }
  template <int HALF = 0>
  static __device__ __forceinline__ void slab_part(const int *As, const int *Bs, int tm, int tn, int kc,
                                                   T (&acc)[8][8]) {
    constexpr bool MASKED = HALF != 0, fr = !(HALF & 1), fc = !(HALF & 2);
    for (int k = 0; k < kc; ++k) {
      T a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = __int_as_float(As[a_off(tm + 16 * i, k >> 2) + (k & 3)]);
      const int *r = Bs + k * kSlabN + 4 * tn;
      const int4 u0 = lds128(r), u1 = lds128(r + 64);
      b[0] = from(u0.x); b[1] = from(u0.y); b[2] = from(u0.z); b[3] = from(u0.w);
      b[4] = from(u1.x); b[5] = from(u1.y); b[6] = from(u1.z); b[7] = from(u1.w);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (MASKED && i >= 4 && !fr) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (MASKED && j >= 4 && !fc) continue;
          acc[i][j] = fminf(acc[i][j], __fadd_rn(a[i], b[j]));
        }
      }
    }
  }
};

// Accumulator registers may be typed int or float; the int32 sequence only reinterprets their
// bits (free), which lets one accumulator array serve both instruction sequences.
__device__ __forceinline__ int acc_bits(int v) { return v; }
__device__ __forceinline__ int acc_bits(float v) { return __float_as_int(v); }
__device__ __forceinline__ void set_acc(int &d, int v) { d = v; }
__device__ __forceinline__ void set_acc(float &d, int v) { d = __int_as_float(v); }

// ArithInt<false> = ArithI32: one fused DPX add-min (__viaddmin_s32) per pair.
// ArithInt<true> = ArithI16x2: every 32-bit operand word packs two 16-bit values, and one DPX
//   operation (__viaddmin_s16x2) performs two pairs.  The operands are packed so that the two
//   halves are consecutive k: A words {A[i][2w], A[i][2w+1]}, B words {B[2w][j], B[2w+1][j]}, so
//   each accumulator word keeps the running minimum over even k in its low half and over odd k in
//   its high half, and the word-level loop is exactly the int32 loop over K / 2 "k" steps.
//   Values are capped at kCap16 = 0x3FFF (sums stay below 2^15, no wrap); collapse() folds the
//   halves and maps a capped result back to the int32 sentinel.
template <bool P16>
struct ArithInt {
  typedef int T;
  static constexpr bool kFloat = false;
  static __device__ __forceinline__ T from(int v) { return v; }
  static __device__ __forceinline__ int to(T v) { return v; }
  static __device__ __forceinline__ T mn(T a, T b) { return min(a, b); }
  static __device__ __forceinline__ int addmin(int a, int b, int c) {
    if (P16) return (int)__viaddmin_s16x2((unsigned)a, (unsigned)b, (unsigned)c);
    return __viaddmin_s32(a, b, c);
  }
  // Fold the two lanes; a result at the cap (or at a sentinel below it) means unreachable.
  static __device__ __forceinline__ T collapse(T v, int inf) {
    if (!P16) return v;
    const int m = min(v & 0xFFFF, (int)((unsigned)v >> 16));
    return m >= min(kCap16, inf) ? inf : m;
  }
  // Fold the two lanes only: the result stays in [0, kCap16] (truncated closures).
  static __device__ __forceinline__ T collapse_truncated(T v) {
    if (!P16) return v;
    return min(v & 0xFFFF, (int)((unsigned)v >> 16));
  }
  // HALF: as ArithF32's -- rows (bit 0) and / or columns (bit 1) 64..127 skipped.
  template <int HALF = 0, typename A>
  static __device__ __forceinline__ void slab_full(const int *As, const int *Bs, int tm, int tn, A (&acc)[8][8]) {
    constexpr bool MASKED = HALF != 0, fr = !(HALF & 1), fc = !(HALF & 2);
#pragma unroll 1
    for (int q = 0; q < kSlabK / 4; ++q) {
      int4 a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (MASKED && i >= 4 && !fr) {
          a[i] = make_int4(0, 0, 0, 0);
          continue;
        }
        a[i] = lds128(As + a_off(tm + 16 * i, q));
      }
#pragma unroll
      for (int kp = 0; kp < 2; ++kp) {
        const int *r0 = Bs + (4 * q + 2 * kp) * kSlabN + 4 * tn;
        const int4 u0 = lds128(r0), w0 = lds128(r0 + kSlabN);
        int4 u1 = make_int4(0, 0, 0, 0), w1 = make_int4(0, 0, 0, 0);
        if (!MASKED || fc) {
          u1 = lds128(r0 + 64);
          w1 = lds128(r0 + kSlabN + 64);
        }
        const int b0[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        const int b1[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (MASKED && i >= 4 && !fr) continue;
          const int a0 = kp ? a[i].z : a[i].x, a1 = kp ? a[i].w : a[i].y;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (MASKED && j >= 4 && !fc) continue;
            set_acc(acc[i][j], addmin(a1, b1[j], addmin(a0, b0[j], acc_bits(acc[i][j]))));
          }
        }
      }
    }
  }
  template <int HALF = 0, typename A>
  static __device__ __forceinline__ void slab_part(const int *As, const int *Bs, int tm, int tn, int kc,
                                                   A (&acc)[8][8]) {
    constexpr bool MASKED = HALF != 0, fr = !(HALF & 1), fc = !(HALF & 2);
    for (int k = 0; k < kc; ++k) {
      int a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[a_off(tm + 16 * i, k >> 2) + (k & 3)];
      const int *r = Bs + k * kSlabN + 4 * tn;
      const int4 u0 = lds128(r), u1 = lds128(r + 64);
      const int b[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (MASKED && i >= 4 && !fr) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (MASKED && j >= 4 && !fc) continue;
          set_acc(acc[i][j], addmin(a[i], b[j], acc_bits(acc[i][j])));
        }
      }
    }
  }
};
typedef ArithInt<false> ArithI32;
typedef ArithInt<true> ArithI16x2;

// True when int32 operands may take the exact fp32 path: every finite sum stays below 2^24
// (w0 * mult + w1 < 2^24, with w0, w1 the largest finite entries involved).
__device__ __forceinline__ bool small_int_bound(int64_t w0, int64_t mult, int64_t w1) {
  return w0 >= 0 && w1 >= 0 && w0 * mult + w1 < (int64_t(1) << 24);
}

}  // namespace apsp
