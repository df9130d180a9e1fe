// diag.cuh -- Eq. 1 (Floyd-Warshall) on one tile of at most 128 x 128, held in registers.
//
// Used for blocked-FW phase 1 (the diagonal tile) by apsp_fw and by the batched kernel, and
// for whole graphs of at most 128 vertices.  256 threads own the tile with the GEMM engine's
// mapping: thread (tm, tn) holds rows tm + 16 i and columns 4 tn + q + 64 h (i, h, q).
// Step k needs column k for a thread's rows and row k for its columns.  Their owners copy them
// from registers into a small double-buffered shared array, one barrier orders the step, and
// every thread then folds min(d, d[i][k] + d[k][j]) into its 64 registers.  Row k and column k
// do not change at step k (d[k][k] = 0 and weights are non-negative), so the copies are final.
// Register indices must be compile-time constants, so the loop is unrolled over k / 16 and
// the owner copies switch on values that are uniform across the block.
#pragma once

#include "common.cuh"

namespace apsp {

template <bool FLOAT>
__device__ __forceinline__ int relax(int d, int a, int b) {
  if (FLOAT) return __float_as_int(fminf(__int_as_float(d), __fadd_rn(__int_as_float(a), __int_as_float(b))));
  return __viaddmin_s32(a, b, d);  // min(a + b, d); int32 values <= 0x3FFFFFFF cannot overflow
}

// Owner of row k (tm == k mod 16, register row kh = k / 16) publishes its 8 row entries.
template <int KH>
__device__ __forceinline__ void put_row(const int (&d)[8][8], int *rb, int tn) {
  *reinterpret_cast<int4 *>(rb + 4 * tn) = make_int4(d[KH][0], d[KH][1], d[KH][2], d[KH][3]);
  *reinterpret_cast<int4 *>(rb + 4 * tn + 64) = make_int4(d[KH][4], d[KH][5], d[KH][6], d[KH][7]);
}

template <int J>
__device__ __forceinline__ void put_col(const int (&d)[8][8], int *cb, int tm) {
#pragma unroll
  for (int i = 0; i < 8; ++i) cb[tm + 16 * i] = d[i][J];
}

// Signed closures (negative weights, int32): a published row or column value at or above
// `thr` is an unreachable entry plus negative terms and is published as exactly `inf`, so no
// such value can drift down into the finite range.  A negative d[k][k] means a negative cycle:
// the closure stops (uniformly: every thread reads the same published value) and returns true.
struct SignedCtl {
  int inf, thr;
};

template <bool FLOAT>
__device__ __forceinline__ int canon(int v, const SignedCtl *sc) {
  if (FLOAT || !sc) return v;
  return v >= sc->thr ? sc->inf : v;
}

// The barrier among the 256 threads that hold a tile: the whole CTA (BAR = 0), or named barrier
// BAR over 256 threads, when the tile's threads are part of a larger CTA (the GEMM engine's
// consumer warps).
template <int BAR>
__device__ __forceinline__ void tile_barrier() {
  if (BAR == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, 256;" ::"n"(BAR) : "memory");
}

// Closes the bk x bk leading part of the register tile d in place.  buf: 512 ints of shared
// memory.  Entries outside bk x bk are scratch (never read back by callers).  With sc (signed
// closures) returns true when a negative cycle was found (the tile is then left partly closed).
template <bool FLOAT, int BAR = 0>
__device__ bool close_tile_regs(int (&d)[8][8], int bk, int tm, int tn, int *buf, const SignedCtl *sc = nullptr) {
  bool negative = false;
#pragma unroll
  for (int kh = 0; kh < 8; ++kh) {
    if (16 * kh >= bk || negative) break;
    for (int kl = 0; kl < 16; ++kl) {
      const int k = 16 * kh + kl;
      if (k >= bk) break;
      int *rb = buf + (k & 1) * 256;
      int *cb = rb + 128;
      if (tm == kl) {
        switch (kh) {
          case 0: put_row<0>(d, rb, tn); break;
          case 1: put_row<1>(d, rb, tn); break;
          case 2: put_row<2>(d, rb, tn); break;
          case 3: put_row<3>(d, rb, tn); break;
          case 4: put_row<4>(d, rb, tn); break;
          case 5: put_row<5>(d, rb, tn); break;
          case 6: put_row<6>(d, rb, tn); break;
          default: put_row<7>(d, rb, tn); break;
        }
      }
      if (tn == ((k >> 2) & 15)) {  // column k = 4 tn + q + 64 h with q = k & 3, h = k >> 6
        const int j = 4 * (kh >> 2) + (kl & 3);
        switch (j) {
          case 0: put_col<0>(d, cb, tm); break;
          case 1: put_col<1>(d, cb, tm); break;
          case 2: put_col<2>(d, cb, tm); break;
          case 3: put_col<3>(d, cb, tm); break;
          case 4: put_col<4>(d, cb, tm); break;
          case 5: put_col<5>(d, cb, tm); break;
          case 6: put_col<6>(d, cb, tm); break;
          default: put_col<7>(d, cb, tm); break;
        }
      }
      tile_barrier<BAR>();
      if (sc) {  // d[k][k] sits in the published row at column k
        const int dkk = rb[k];
        if (FLOAT ? __int_as_float(dkk) < 0.0f : dkk < 0) {
          negative = true;
          break;
        }
      }
      int c[8], r[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) c[i] = canon<FLOAT>(cb[tm + 16 * i], sc);
      const int4 r0 = *reinterpret_cast<const int4 *>(rb + 4 * tn);
      const int4 r1 = *reinterpret_cast<const int4 *>(rb + 4 * tn + 64);
      r[0] = canon<FLOAT>(r0.x, sc); r[1] = canon<FLOAT>(r0.y, sc);
      r[2] = canon<FLOAT>(r0.z, sc); r[3] = canon<FLOAT>(r0.w, sc);
      r[4] = canon<FLOAT>(r1.x, sc); r[5] = canon<FLOAT>(r1.y, sc);
      r[6] = canon<FLOAT>(r1.z, sc); r[7] = canon<FLOAT>(r1.w, sc);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) d[i][j] = relax<FLOAT>(d[i][j], c[i], r[j]);
    }
  }
  tile_barrier<BAR>();  // buf is reused by the caller
  return negative;
}

// Load / store the bk x bk tile at T (leading dimension ld, 16-byte aligned rows) into the
// register tile.  Entries outside bk x bk are set to 0 on load and never stored.
__device__ __forceinline__ void load_tile_regs(int (&d)[8][8], const int *T, int64_t ld, int bk, int tm, int tn) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = tm + 16 * i;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = 4 * tn + 64 * h;
      int4 v = make_int4(0, 0, 0, 0);
      // L2-only load: the tile may have been written by another CTA of a cluster
      if (r < bk && c < bk) v = __ldcg(reinterpret_cast<const int4 *>(T + (int64_t)r * ld + c));
      d[i][4 * h] = v.x; d[i][4 * h + 1] = v.y; d[i][4 * h + 2] = v.z; d[i][4 * h + 3] = v.w;
    }
  }
}

__device__ __forceinline__ void store_tile_regs(const int (&d)[8][8], int *T, int64_t ld, int bk, int tm, int tn) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = tm + 16 * i;
    if (r >= bk) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = 4 * tn + 64 * h;
      int *p = T + (int64_t)r * ld + c;
      if (c + 3 < bk) {
        *reinterpret_cast<int4 *>(p) = make_int4(d[i][4 * h], d[i][4 * h + 1], d[i][4 * h + 2], d[i][4 * h + 3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (c + q < bk) p[q] = d[i][4 * h + q];
      }
    }
  }
}

}  // namespace apsp
