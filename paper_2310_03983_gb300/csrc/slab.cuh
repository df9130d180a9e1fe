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

// fp32 instruction sequence of the slab loop (all exact-equivalent; chosen by measurement):
//   0: packed pair add over k-pairs + 3-input min;  1: two scalar adds + 3-input min;
//   2: packed pair add over column pairs (duplicated A operand) + 3-input min;
//   3: as 2, the adds of one A operand issued back to back before the mins;
//   4: as 3, with the k+1 pairs half-swapped so each min reads a low and a high half;
//   5: B slab transposed in shared memory by the consumers, packed adds over k-pairs with
//      both operand pairs straight from 128-bit loads (slab_full_bt).
#ifndef APSP_F32_SEQ
#define APSP_F32_SEQ 5
#endif
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
  static constexpr bool kTransposeB = APSP_F32_SEQ == 5;
  static __device__ __forceinline__ T from(int v) { return __int_as_float(v); }
  static __device__ __forceinline__ int to(T v) { return __float_as_int(v); }
  static __device__ __forceinline__ T mn(T a, T b) { return fminf(a, b); }
  // Consumer-side transpose of the [32 k][128 n] B slab into BT [128 n][32 k] (one of two
  // 16 KB buffers), 16-byte chunk kq of row n stored at chunk kq ^ ((n >> 2) & 7): the reads
  // of the transpose, its writes and the slab loop's reads are all free of bank conflicts.
  // Ends with a barrier over the 256 consumer threads (named barrier 1).
  static __device__ __forceinline__ void transpose_b(const int *Bs, int *BT) {
    const int t = threadIdx.x & 255;
    const int nq = t & 31, kq = t >> 5;  // a 4 x 4 block: k = 4 kq .. +3, n = 4 nq .. +3
    const int4 r0 = lds128(Bs + (4 * kq + 0) * kSlabN + 4 * nq);
    const int4 r1 = lds128(Bs + (4 * kq + 1) * kSlabN + 4 * nq);
    const int4 r2 = lds128(Bs + (4 * kq + 2) * kSlabN + 4 * nq);
    const int4 r3 = lds128(Bs + (4 * kq + 3) * kSlabN + 4 * nq);
    const int sw = (kq ^ (nq & 7)) << 2;
    *reinterpret_cast<int4 *>(BT + (4 * nq + 0) * kSlabK + sw) = make_int4(r0.x, r1.x, r2.x, r3.x);
    *reinterpret_cast<int4 *>(BT + (4 * nq + 1) * kSlabK + sw) = make_int4(r0.y, r1.y, r2.y, r3.y);
    *reinterpret_cast<int4 *>(BT + (4 * nq + 2) * kSlabK + sw) = make_int4(r0.z, r1.z, r2.z, r3.z);
    *reinterpret_cast<int4 *>(BT + (4 * nq + 3) * kSlabK + sw) = make_int4(r0.w, r1.w, r2.w, r3.w);
    asm volatile("bar.sync 1, 256;" ::: "memory");
  }

  // k-pair form: for column c and k-pair (k, k+1), one packed add {A[i][k] + B[k][c],
  // A[i][k+1] + B[k+1][c]} and one 3-input min of its two halves, both operand pairs read
  // straight from 128-bit shared loads (no packing moves).
  static __device__ __forceinline__ void slab_full_bt(const int *As, const int *BT, int tm, int tn, T (&acc)[8][8]) {
#pragma unroll kQUnroll
    for (int q = 0; q < kSlabK / 4; ++q) {
      uint64_t a[8][2], b[8][2];
#pragma unroll
      for (int i = 0; i < 8; ++i) lds128_2x64(As + a_off(tm + 16 * i, q), a[i][0], a[i][1]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = 4 * tn + (j & 3) + 64 * (j >> 2);
        lds128_2x64(BT + n * kSlabK + ((q ^ ((n >> 2) & 7)) << 2), b[j][0], b[j][1]);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint64_t t0 = fadd2_64(a[i][0], b[j][0]);
          const uint64_t t1 = fadd2_64(a[i][1], b[j][1]);
          acc[i][j] = Ops<float>::min3(Ops<float>::min3(acc[i][j], lo_of(t0), hi_of(t0)), lo_of(t1), hi_of(t1));
        }
    }
  }

  static __device__ __forceinline__ void slab_full(const int *As, const int *Bs, int tm, int tn, T (&acc)[8][8]) {
#pragma unroll kQUnroll
    for (int q = 0; q < kSlabK / 4; ++q) {
#if APSP_F32_SEQ == 0
      // a[i][0] = {A[r_i][4q], A[r_i][4q+1]}, a[i][1] = {A[r_i][4q+2], A[r_i][4q+3]}
      uint64_t a[8][2];
#pragma unroll
      for (int i = 0; i < 8; ++i) lds128_2x64(As + a_off(tm + 16 * i, q), a[i][0], a[i][1]);
#pragma unroll
      for (int kp = 0; kp < 2; ++kp) {
        const int *r0 = Bs + (4 * q + 2 * kp) * kSlabN + 4 * tn;
        const int4 u0 = lds128(r0), u1 = lds128(r0 + 64), w0 = lds128(r0 + kSlabN), w1 = lds128(r0 + kSlabN + 64);
        // b[j] = {B[k][c_j], B[k+1][c_j]}: built once, reused by all eight rows
        uint64_t b[8];
        b[0] = pack2(__int_as_float(u0.x), __int_as_float(w0.x));
        b[1] = pack2(__int_as_float(u0.y), __int_as_float(w0.y));
        b[2] = pack2(__int_as_float(u0.z), __int_as_float(w0.z));
        b[3] = pack2(__int_as_float(u0.w), __int_as_float(w0.w));
        b[4] = pack2(__int_as_float(u1.x), __int_as_float(w1.x));
        b[5] = pack2(__int_as_float(u1.y), __int_as_float(w1.y));
        b[6] = pack2(__int_as_float(u1.z), __int_as_float(w1.z));
        b[7] = pack2(__int_as_float(u1.w), __int_as_float(w1.w));
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint64_t t = fadd2_64(a[i][kp], b[j]);
            acc[i][j] = Ops<float>::min3(acc[i][j], lo_of(t), hi_of(t));
          }
      }
#elif APSP_F32_SEQ == 1
      // two scalar adds feeding one 3-input min
      float4 a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int4 v = lds128(As + a_off(tm + 16 * i, q));
        a[i] = make_float4(__int_as_float(v.x), __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w));
      }
#pragma unroll
      for (int kp = 0; kp < 2; ++kp) {
        const int *r0 = Bs + (4 * q + 2 * kp) * kSlabN + 4 * tn;
        const int4 u0 = lds128(r0), u1 = lds128(r0 + 64), w0 = lds128(r0 + kSlabN), w1 = lds128(r0 + kSlabN + 64);
        const float b0[8] = {__int_as_float(u0.x), __int_as_float(u0.y), __int_as_float(u0.z), __int_as_float(u0.w),
                             __int_as_float(u1.x), __int_as_float(u1.y), __int_as_float(u1.z), __int_as_float(u1.w)};
        const float b1[8] = {__int_as_float(w0.x), __int_as_float(w0.y), __int_as_float(w0.z), __int_as_float(w0.w),
                             __int_as_float(w1.x), __int_as_float(w1.y), __int_as_float(w1.z), __int_as_float(w1.w)};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float a0 = kp ? a[i].z : a[i].x, a1 = kp ? a[i].w : a[i].y;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            acc[i][j] = Ops<float>::min3(acc[i][j], __fadd_rn(a0, b0[j]), __fadd_rn(a1, b1[j]));
        }
      }
#else
      // packed adds along j: {A[i][k], A[i][k]} + {B[k][c_j], B[k][c_j+1]}
      float4 a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int4 v = lds128(As + a_off(tm + 16 * i, q));
        a[i] = make_float4(__int_as_float(v.x), __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w));
      }
#pragma unroll
      for (int kp = 0; kp < 2; ++kp) {
        const int *r0 = Bs + (4 * q + 2 * kp) * kSlabN + 4 * tn;
        uint64_t b0[4], b1[4];
        lds128_2x64(r0, b0[0], b0[1]);
        lds128_2x64(r0 + 64, b0[2], b0[3]);
        lds128_2x64(r0 + kSlabN, b1[0], b1[1]);
        lds128_2x64(r0 + kSlabN + 64, b1[2], b1[3]);
#if APSP_F32_SEQ == 4
        // swap the halves of the k+1 pairs so each 3-input min reads one low and one high half
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) b1[jp] = pack2(hi_of(b1[jp]), lo_of(b1[jp]));
#endif
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float a0 = kp ? a[i].z : a[i].x, a1 = kp ? a[i].w : a[i].y;
          const uint64_t aa0 = pack2(a0, a0), aa1 = pack2(a1, a1);
#if APSP_F32_SEQ == 2
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) {
            const uint64_t t0 = fadd2_64(aa0, b0[jp]), t1 = fadd2_64(aa1, b1[jp]);
            acc[i][2 * jp] = Ops<float>::min3(acc[i][2 * jp], lo_of(t0), lo_of(t1));
            acc[i][2 * jp + 1] = Ops<float>::min3(acc[i][2 * jp + 1], hi_of(t0), hi_of(t1));
          }
#else
          uint64_t t0[4], t1[4];
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) t0[jp] = fadd2_64(aa0, b0[jp]);
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) t1[jp] = fadd2_64(aa1, b1[jp]);
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) {
#if APSP_F32_SEQ == 4
            acc[i][2 * jp] = Ops<float>::min3(acc[i][2 * jp], lo_of(t0[jp]), hi_of(t1[jp]));
            acc[i][2 * jp + 1] = Ops<float>::min3(acc[i][2 * jp + 1], hi_of(t0[jp]), lo_of(t1[jp]));
#else
            acc[i][2 * jp] = Ops<float>::min3(acc[i][2 * jp], lo_of(t0[jp]), lo_of(t1[jp]));
            acc[i][2 * jp + 1] = Ops<float>::min3(acc[i][2 * jp + 1], hi_of(t0[jp]), hi_of(t1[jp]));
#endif
          }
#endif
        }
      }
#endif
    }
  }
  static __device__ __forceinline__ void slab_part(const int *As, const int *Bs, int tm, int tn, int kc,
                                                   T (&acc)[8][8]) {
    for (int k = 0; k < kc; ++k) {
      T a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = __int_as_float(As[a_off(tm + 16 * i, k >> 2) + (k & 3)]);
      const int *r = Bs + k * kSlabN + 4 * tn;
      const int4 u0 = lds128(r), u1 = lds128(r + 64);
      b[0] = from(u0.x); b[1] = from(u0.y); b[2] = from(u0.z); b[3] = from(u0.w);
      b[4] = from(u1.x); b[5] = from(u1.y); b[6] = from(u1.z); b[7] = from(u1.w);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fminf(acc[i][j], __fadd_rn(a[i], b[j]));
    }
  }
};

struct ArithI32 {
  typedef int T;
  static constexpr bool kTransposeB = false;
  static __device__ __forceinline__ void transpose_b(const int *, int *) {}
  static __device__ __forceinline__ void slab_full_bt(const int *, const int *, int, int, T (&)[8][8]) {}
  static __device__ __forceinline__ T from(int v) { return v; }
  static __device__ __forceinline__ int to(T v) { return v; }
  static __device__ __forceinline__ T mn(T a, T b) { return min(a, b); }
  static __device__ __forceinline__ void slab_full(const int *As, const int *Bs, int tm, int tn, T (&acc)[8][8]) {
#pragma unroll 1
    for (int q = 0; q < kSlabK / 4; ++q) {
      int4 a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = lds128(As + a_off(tm + 16 * i, q));
#pragma unroll
      for (int kp = 0; kp < 2; ++kp) {
        const int *r0 = Bs + (4 * q + 2 * kp) * kSlabN + 4 * tn;
        const int4 u0 = lds128(r0), u1 = lds128(r0 + 64), w0 = lds128(r0 + kSlabN), w1 = lds128(r0 + kSlabN + 64);
        const int b0[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        const int b1[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int a0 = kp ? a[i].z : a[i].x, a1 = kp ? a[i].w : a[i].y;
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = __viaddmin_s32(a1, b1[j], __viaddmin_s32(a0, b0[j], acc[i][j]));
        }
      }
    }
  }
  static __device__ __forceinline__ void slab_part(const int *As, const int *Bs, int tm, int tn, int kc,
                                                   T (&acc)[8][8]) {
    for (int k = 0; k < kc; ++k) {
      int a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[a_off(tm + 16 * i, k >> 2) + (k & 3)];
      const int *r = Bs + k * kSlabN + 4 * tn;
      const int4 u0 = lds128(r), u1 = lds128(r + 64);
      const int b[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = __viaddmin_s32(a[i], b[j], acc[i][j]);
    }
  }
};

// True when int32 operands may take the exact fp32 path: every finite sum stays below 2^24
// (w0 * mult + w1 < 2^24, with w0, w1 the largest finite entries involved).
__device__ __forceinline__ bool small_int_bound(int64_t w0, int64_t mult, int64_t w1) {
  return w0 >= 0 && w1 >= 0 && w0 * mult + w1 < (int64_t(1) << 24);
}

}  // namespace apsp
