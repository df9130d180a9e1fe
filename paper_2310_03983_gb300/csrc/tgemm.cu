// tgemm.cu -- register-tiled (min,+) product on CUDA cores (the paper's Eq. 2, Sec. 3).
//
//   C[i][j] = min( C[i][j] or INF,  min_k A[i][k] + B[k][j] )
//
// The paper forms the whole N x N x N tensor of sums and reduces it with a library min
// (Sec. 3.1); that costs n^3 memory and capped its graphs at 1000 vertices.  Here the same
// reduction is blocked so that nothing but the n x n operands ever lives in HBM:
//
//  * A persistent grid (one CTA per SM, 384 threads) walks a list of 128 x 128 output tiles.
//  * Warps 8-11 are the producer warpgroup: one lane of warp 8 issues TMA copies of the
//    128 x 32 A slab and the 32 x 128 B slab of each k-step into a 4-stage shared-memory
//    ring (mbarrier full/empty handshakes), and, when folding into an existing C, the
//    128 x 128 C tile.
//  * Warps 0-7 are consumers: each thread owns an 8 x 8 register tile of C (rows
//    tm + 16 i, columns 4 tn + q + 64 h), reads A as 128-bit row quads (a broadcast within
//    each quarter-warp) and B as 128-bit column quads (eight lanes cover 32 banks), and
//    performs one add and one min per (i, j, k): on int32 with the fused DPX add-min, on
//    fp32 as two adds feeding one 3-input min.
//  * Epilogue: min with the prefetched C tile, 128-bit coalesced stores.
//
// No tensor cores: (min,+) is not a multiply-accumulate.  int32 results are exact; fp32
// results are bitwise deterministic (min is exact, each candidate sum is one rounding).
#include <atomic>
#include <math.h>
#include <type_traits>
#include <utility>

#include "diag.cuh"
#include "slab.cuh"
#include "tgemm.cuh"

namespace apsp {

struct TileCoords {
  int a_row, a_col, b_row, b_col, c_row, c_col;
  int m_valid, n_valid, k_len;
  bool skip;  // grouped FW: this graph does not take part in the launch
  // 16-bit launches: packed copies of the result -- column pairs into set pa_set of the packed
  // column panels (at the tile's rows), row pairs into set pb_set of the packed row panels
  // (grouped: rows pb_row.., single matrix: the set's 64 rows; the tile's columns); -1: none.
  int pa_set, pb_set, pb_row;
  // Fused launches (TileProblem::close_next): dep -- the next block's panel tiles read this
  // tile, so it is counted once stored; wait -- a panel tile, whose operands must be counted
  // complete before they are loaded.
  bool dep, wait;
  // Grouped launches: the tile's rows (half_r) / columns (half_c) 64..127 are padding of the
  // graph's last block, so only the first half is computed (the rest keeps its initial value,
  // which is what the padding's isolated vertices hold anyway).
  bool half_r, half_c;
};

// Tile t of a grouped FW launch: find its group and graph (all tiles of one graph are
// consecutive), then place the single-matrix tile of that graph at the graph's rows.  Every
// count here fits 32 bits (the staging keeps at most 2^30 rows, at least 384 per graph), and
// 32-bit unsigned arithmetic keeps this per-tile work small next to the tile's DPX stream.
template <int MODE>
__device__ __forceinline__ TileCoords grouped_tile_coords(const TileProblem &p, int64_t t) {
  TileCoords tc;
  tc.dep = tc.wait = false;
  tc.half_r = tc.half_c = false;
  unsigned rem = (unsigned)t, per = 1, row0 = 0, gnb = 1, first = 0;
  const unsigned kb = (unsigned)p.kb;
  bool found = false;
#pragma unroll
  for (int k = 0; k < kMaxGroups; ++k) {
    if (!found && k < p.ngroups) {
      const unsigned nb = (unsigned)p.groups[k].nb;
      const unsigned pg = nb <= kb ? 0u : (MODE == kModeFwPanels ? 2u * (nb - 1) : (nb - 1) * (nb - 1));
      const unsigned tot = pg * (unsigned)p.groups[k].count;
      if (rem < tot) {
        found = true;
        per = pg;
        row0 = (unsigned)p.groups[k].row0;
        first = (unsigned)p.groups[k].first;
        gnb = nb;
      } else {
        rem -= tot;
      }
    }
  }
  const unsigned ql = rem / per, lt = rem - ql * per;
  const int q = (int)(first + ql);
  const int base = (int)(row0 + ql * gnb * kBM);
  const unsigned nb1 = gnb - 1;
  const int kb0 = (int)(kb * kBM);
  int i, j;
  if (MODE == kModeFwPanels) {
    // 16-bit operands: A = the packed column panel (A16, same rows), B = the packed row panel
    // (B16, 64 rows per graph); both hold the diagonal tile as well.
    const int a_col = p.arith16 ? 0 : kb0;
    const int b_row = p.arith16 ? q * (kBM / 2) : base + kb0;
    const int cur = (int)(kb & 1), nxt = cur ^ 1;
    tc.pb_row = q * (kBM / 2);
    if (lt < nb1) {  // row panel (kb, j): phase 3's row operand; column kb + 1: the next column panel
      j = (int)(lt + (lt >= kb));
      tc.a_row = base + kb0; tc.a_col = a_col;
      tc.b_row = b_row;      tc.b_col = j * kBN;
      tc.c_row = base + kb0; tc.c_col = j * kBN;
      tc.pb_set = cur;
      tc.pa_set = j == (int)kb + 1 ? nxt : -1;
    } else {         // column panel (i, kb): phase 3's column operand; row kb + 1: the next row panel
      i = (int)(lt - nb1);
      i += (i >= (int)kb);
      tc.a_row = base + i * kBM; tc.a_col = a_col;
      tc.b_row = b_row;          tc.b_col = kb0;
      tc.c_row = base + i * kBM; tc.c_col = kb0;
      tc.pa_set = cur;
      tc.pb_set = i == (int)kb + 1 ? nxt : -1;
    }
  } else {
    const unsigned iu = lt / nb1;
    i = (int)iu;
    j = (int)(lt - iu * nb1);
    i += (i >= (int)kb);
    j += (j >= (int)kb);
    tc.a_row = base + i * kBM;
    tc.c_row = base + i * kBM; tc.c_col = j * kBN;
    tc.b_col = j * kBN;
    tc.pa_set = tc.pb_set = -1;
    tc.pb_row = q * (kBM / 2);
    if (MODE == kModeFwRest16) {
      tc.a_col = 0;
      tc.b_row = q * (kBM / 2);
      // tiles of block row / column kb + 1 (not its diagonal tile) are the next step's panels
      const int nxt = (int)((kb + 1) & 1);
      if (i == (int)kb + 1 && j != (int)kb + 1) tc.pb_set = nxt;
      if (j == (int)kb + 1 && i != (int)kb + 1) tc.pa_set = nxt;
    } else {
      tc.a_col = kb0;
      tc.b_row = base + kb0;
    }
  }
  tc.m_valid = kBM;
  tc.n_valid = kBN;
  tc.skip = !found || (p.gflags[q] & p.gmask) != p.gwant;
  int bk = kBM;
  if (p.gsize && !tc.skip) {
    const int gs = p.gsize[q], left = gs - kb0;
    bk = left < kBM ? (left > 0 ? left : 1) : kBM;
    tc.half_r = gs - (tc.c_row - base) <= kBM / 2;
    tc.half_c = gs - tc.c_col <= kBN / 2;
  }
  tc.k_len = (MODE == kModeFwRest16 || p.arith16) ? (bk + 1) >> 1 : bk;
  return tc;
}

// G: a grouped launch (its own instantiation, so a single-matrix kernel carries none of the
// grouped decode or packed-output epilogue).  alt: kModeFwRest16's 32-bit alternative (the
// block's columns and rows of the matrix, K = the block width).
template <int MODE, bool G>
__device__ __forceinline__ TileCoords tile_coords(const TileProblem &p, int64_t t, bool alt = false) {
  if (G) return grouped_tile_coords<MODE>(p, t);
  TileCoords tc;
  tc.skip = false;
  tc.pa_set = tc.pb_set = -1;
  tc.pb_row = 0;
  tc.dep = tc.wait = false;
  tc.half_r = tc.half_c = false;
  if (MODE == kModeGemm) {
    // Grouped rasterisation: 8 tile-rows advance together so A slabs are reused from L2.
    const int64_t G = 8;
    const int64_t per_group = G * p.tiles_n;
    const int64_t g = t / per_group;
    const int64_t first_m = g * G;
    const int64_t gsz = (p.tiles_m - first_m) < G ? (p.tiles_m - first_m) : G;
    const int64_t r = t - g * per_group;
    const int m0 = (int)((first_m + r % gsz) * kBM);
    const int n0 = (int)((r / gsz) * kBN);
    tc.a_row = m0; tc.a_col = 0;
    tc.b_row = 0;  tc.b_col = n0;
    tc.c_row = m0; tc.c_col = n0;
    tc.m_valid = (int)(p.M - m0 < kBM ? p.M - m0 : kBM);
    tc.n_valid = (int)(p.N - n0 < kBN ? p.N - n0 : kBN);
    tc.k_len = (int)p.K;
  } else if (MODE == kModeFwRest16 && p.bt > 1) {  // phase 3 of a block of bt tiles, K in packed words
    const int64_t bt = p.bt;
    const int64_t nt = (p.n + kBM - 1) / kBM, e0 = p.kb * bt;
    const int64_t ec = nt - e0 < bt ? nt - e0 : bt, rest = nt - ec;
    int i = (int)(t / rest), j = (int)(t - (t / rest) * rest);
    i += (i >= e0) ? (int)ec : 0;
    j += (j >= e0) ? (int)ec : 0;
    const int k0 = alt ? (int)(e0 * kBM) : 0;
    tc.a_row = i * kBM; tc.a_col = k0;
    tc.b_row = k0;      tc.b_col = j * kBN;
    tc.c_row = i * kBM; tc.c_col = j * kBN;
    tc.m_valid = (int)(p.n - tc.c_row < kBM ? p.n - tc.c_row : kBM);
    tc.n_valid = (int)(p.n - tc.c_col < kBN ? p.n - tc.c_col : kBN);
    const int64_t w = bt * kBM, b0 = p.kb * w, len = p.n - b0 < w ? p.n - b0 : w;
    tc.k_len = alt ? (int)len : (int)((len + 1) >> 1);
  } else {
    // Blocked FW over 128-vertex blocks: tile (i, j) of phase 2 (mode 1) or 3 (modes 2, 3) runs
    // over the k range of block kblk -- kb, or kb + 1 for the panel tiles of a fused launch.
    const int64_t nb1 = p.nb - 1;
    const int kb = (int)p.kb;
    int i, j, kblk = kb;
    bool panel = MODE == kModeFwPanels;
    if (MODE == kModeFwPanels) {
      if (t < nb1) {  // row panel tile (kb, j): D[kb][j] = D[kb][kb]* (x) D[kb][j]
        i = kb;
        j = (int)(t + (t >= kb));
      } else {        // column panel tile (i, kb): D[i][kb] = D[i][kb] (x) D[kb][kb]*
        i = (int)(t - nb1);
        i += (i >= kb);
        j = kb;
      }
    } else if (p.close_next) {  // the fused order (TileProblem::close_next)
      const int kb1 = kb + 1;
      const int64_t R = nb1, R1 = nb1 - 1;
      if (t == 0) {                 // the next diagonal tile
        i = j = kb1;
        tc.dep = true;
      } else if (t < R) {           // the rest of block row kb1
        const int x = (int)(t - 1);
        i = kb1;
        j = x + (x >= kb ? 2 : 0);
        tc.dep = true;
      } else if (t < 2 * R - 1) {   // the rest of block column kb1
        const int x = (int)(t - R);
        i = x + (x >= kb ? 2 : 0);
        j = kb1;
        tc.dep = true;
      } else if (t < R * R) {       // the rest of phase 3, row by row
        const int64_t u = t - (2 * R - 1);
        const int ii = (int)(u / R1), jj = (int)(u - (u / R1) * R1);
        i = ii + (ii >= kb ? 2 : 0);
        j = jj + (jj >= kb ? 2 : 0);
      } else {                      // phase 2 of block kb1: row panel tiles, then column panel tiles
        const int v = (int)(t - R * R);
        if (v < R) {
          i = kb1;
          j = v + (v >= kb1);
        } else {
          i = (v - (int)R) + ((v - (int)R) >= kb1);
          j = kb1;
        }
        kblk = kb1;
        panel = true;
        tc.wait = true;
      }
    } else {          // D[i][j] = min(D[i][j], D[i][kb] (x) D[kb][j]), i, j != kb, row by row
      i = (int)(t / nb1);
      j = (int)(t - (t / nb1) * nb1);
      i += (i >= kb);
      j += (j >= kb);
    }
    const int k0 = kblk * kBM, bk = (int)(p.n - k0 < kBM ? p.n - k0 : kBM);
    // Operands: the packed panels of block kblk (set kblk & 1: the column panel's rows i, the row
    // panel's columns j -- for a panel tile the closed diagonal tile's packed copy on one side),
    // or the matrix's own block kblk.
    const bool p16 = MODE == kModeFwRest16 && !alt;
    const int s = kblk & 1;
    if (p16) {
      tc.a_row = (int)(s * p.pk_arows) + i * kBM; tc.a_col = 0;
      tc.b_row = s * (kBM / 2);                   tc.b_col = j * kBN;
      tc.k_len = (bk + 1) >> 1;
    } else {
      tc.a_row = i * kBM; tc.a_col = k0;
      tc.b_row = k0;      tc.b_col = j * kBN;
      tc.k_len = bk;
    }
    tc.c_row = i * kBM;
    tc.c_col = j * kBN;
    tc.m_valid = (int)(p.n - tc.c_row < kBM ? p.n - tc.c_row : kBM);
    tc.n_valid = (int)(p.n - tc.c_col < kBN ? p.n - tc.c_col : kBN);
    // Packed copies of the result (phase 3 reads them from set kblk & 1; the tiles of block row /
    // column kblk + 1 are also the next block's operands, set s ^ 1).
    if (MODE == kModeFwPanels || p16) {
      if (panel) {
        if (i == kblk) {
          tc.pb_set = s;
          if (j == kblk + 1) tc.pa_set = s ^ 1;
        } else {
          tc.pa_set = s;
          if (i == kblk + 1) tc.pb_set = s ^ 1;
        }
      } else if (tc.dep) {
        if (i == kb + 1) tc.pb_set = s ^ 1;
        if (j == kb + 1) tc.pa_set = s ^ 1;
      }
    }
  }
  return tc;
}

// Tile-index ring of dynamic scheduling (TileProblem::tile_counter): the producer fetches each
// tile index from the counter and passes it to the consumer warps through kTileRing slots.
constexpr int kTileRing = 2;

struct Smem {
  const int *sA, *sB, *sC;
  uint64_t *full, *empty, *cfull, *cempty, *tq_full, *tq_empty;
  volatile int *tq;
  int *dbuf;  // row / column buffers of the in-kernel diagonal closure
};

// Consumer warps: walk the same tile sequence as the producer, fold every k-slab into the
// 8 x 8 register tile, then (optionally) min with the prefetched C tile and store.
// fstore: float storage (the in-kernel diagonal closure then relaxes in fp32, else in int32).
// CN: the phase-3 instantiation with dynamic tile scheduling and the in-kernel closure of the
// next diagonal tile (TileProblem::tile_counter, close_next).
template <typename AR, int MODE, bool ACC, bool G, bool CN>
__device__ __forceinline__ void consume(const TileProblem &p, const Smem &sm, int warp, int lane, int init_bits,
                                        bool fstore, bool alt = false) {
  typedef typename AR::T T;
  const int tm = (warp & 3) * 4 + (lane >> 3);
  const int tn = (warp >> 2) * 8 + (lane & 7);
  int *C = reinterpret_cast<int *>(p.C);
  int stage = 0;
  uint32_t phase = 0, cphase = 0;
  const T init = AR::from(init_bits);
  const bool dyn = CN && p.tile_counter;  // uniform
  int tqs = 0;
  uint32_t tqp = 0;
  for (int64_t it = blockIdx.x;; it += gridDim.x) {
    int64_t t = it;
    if (dyn) {  // the next index from the producer (-1: no tiles left)
      if (!mbar_wait(&sm.tq_full[tqs], tqp, p.status)) return;
      t = sm.tq[tqs];
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.tq_empty[tqs]);
      if (++tqs == kTileRing) { tqs = 0; tqp ^= 1; }
      if (t < 0) break;
    } else if (t >= p.ntiles) {
      break;
    }
    const TileCoords tc = tile_coords<MODE, G>(p, t, alt);
    if (tc.skip) continue;  // the producer skips the same tiles
    const int nk = (tc.k_len + kBK - 1) / kBK;
    T acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = init;
    for (int kt = 0; kt < nk; ++kt) {
      if (!mbar_wait(&sm.full[stage], phase, p.status)) return;
      const int *As = sm.sA + stage * (kBM * kBK);
      const int *Bs = sm.sB + stage * (kBK * kBN);
      const int kc = tc.k_len - kt * kBK;
      const int half = G ? (tc.half_r ? 1 : 0) | (tc.half_c ? 2 : 0) : 0;  // uniform per tile
      if (kc >= kBK) {
        switch (half) {
          case 0: AR::slab_full(As, Bs, tm, tn, acc); break;
          case 1: AR::template slab_full<1>(As, Bs, tm, tn, acc); break;
          case 2: AR::template slab_full<2>(As, Bs, tm, tn, acc); break;
          default: AR::template slab_full<3>(As, Bs, tm, tn, acc); break;
        }
      } else {
        switch (half) {
          case 0: AR::slab_part(As, Bs, tm, tn, kc, acc); break;
          case 1: AR::template slab_part<1>(As, Bs, tm, tn, kc, acc); break;
          case 2: AR::template slab_part<2>(As, Bs, tm, tn, kc, acc); break;
          default: AR::template slab_part<3>(As, Bs, tm, tn, kc, acc); break;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.empty[stage]);
      if (++stage == kStages) { stage = 0; phase ^= 1; }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        acc[i][j] = MODE == kModeGemm ? AR::collapse(acc[i][j], p.inf_i) : AR::collapse_truncated(acc[i][j]);
    if (!AR::kFloat && p.sat) {  // uniform per launch
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = acc[i][j] >= p.sat ? AR::from(p.inf_i) : acc[i][j];
    }
    if (ACC) {
      if (!mbar_wait(sm.cfull, cphase, p.status)) return;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int4 v = lds128(sm.sC + (tm + 16 * i) * kBN + 4 * tn + 64 * h);
          acc[i][4 * h + 0] = AR::mn(acc[i][4 * h + 0], AR::from(v.x));
          acc[i][4 * h + 1] = AR::mn(acc[i][4 * h + 1], AR::from(v.y));
          acc[i][4 * h + 2] = AR::mn(acc[i][4 * h + 2], AR::from(v.z));
          acc[i][4 * h + 3] = AR::mn(acc[i][4 * h + 3], AR::from(v.w));
        }
      __syncwarp();
      if (lane == 0) mbar_arrive(sm.cempty);
      cphase ^= 1;
    }
    if (CN && p.close_next && t == 0) {
      // Phase 1 of block kb + 1 on its freshly updated diagonal tile (Eq. 1 in registers, the
      // 256 consumer threads synchronised by named barrier 1).
      int d[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) d[i][j] = AR::to(acc[i][j]);
      if (fstore)
        close_tile_regs<true, 1>(d, tc.m_valid, tm, tn, sm.dbuf);
      else
        close_tile_regs<false, 1>(d, tc.m_valid, tm, tn, sm.dbuf);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = AR::from(d[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int rl = tm + 16 * i;
      if (rl >= tc.m_valid) continue;
      int *crow = C + (int64_t)(tc.c_row + rl) * p.ldc + tc.c_col;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cl = 4 * tn + 64 * h;
        if (cl + 3 < tc.n_valid) {
          *reinterpret_cast<int4 *>(crow + cl) = make_int4(AR::to(acc[i][4 * h]), AR::to(acc[i][4 * h + 1]),
                                                           AR::to(acc[i][4 * h + 2]), AR::to(acc[i][4 * h + 3]));
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (cl + q < tc.n_valid) crow[cl + q] = AR::to(acc[i][4 * h + q]);
        }
      }
    }
    if (!G && (MODE == kModeFwPanels || (MODE == kModeFwRest16 && CN && !alt)) && !fstore && p.pk_a[0] &&
        (tc.pa_set >= 0 || tc.pb_set >= 0)) {  // packed 16-bit operands of phase 3 / the next panels
      // Columns (column pairs) and rows (row pairs) past the matrix's last vertex become CAP,
      // the padding of a partial last k-word.
      int v[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const bool pad = tm + 16 * i >= tc.m_valid || 4 * tn + (j & 3) + 64 * (j >> 2) >= tc.n_valid;
          v[i][j] = pad ? kCap16 : AR::to(acc[i][j]);
        }
      if (tc.pa_set >= 0) store_col_pairs16(v, tm, tn, p.pk_a[tc.pa_set] + (int64_t)tc.c_row * 64);
      if (tc.pb_set >= 0) store_row_pairs16(v, tm, tn, lane, p.pk_b[tc.pb_set] + tc.c_col, p.pk_ldb);
    }
    if (CN && tc.dep) {  // count the tile once all of its stores are done (fused launches)
      tile_barrier<1>();
      if (warp == 0 && lane == 0) {
        __threadfence();
        counter_add_release(p.tile_counter + 2, 1);
      }
    }
    if (G && MODE != kModeGemm && !AR::kFloat && p.arith16 && p.pk_a[0] && (tc.pa_set >= 0 || tc.pb_set >= 0)) {
      int v[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) v[i][j] = AR::to(acc[i][j]);
      if (tc.pa_set >= 0) store_col_pairs16(v, tm, tn, (tc.pa_set ? p.pk_a[1] : p.pk_a[0]) + (int64_t)tc.c_row * 64);
      if (tc.pb_set >= 0)
        store_row_pairs16(v, tm, tn, lane, (tc.pb_set ? p.pk_b[1] : p.pk_b[0]) + (int64_t)tc.pb_row * p.ldc + tc.c_col,
                          p.ldc);
    }
  }
}

// S: storage type (int or float).  Float matrices always take ArithF32; int matrices take
// ArithF32 when small_int_bound holds for this launch (or *p.f32_if), else ArithI32 (uniform
// per launch).
template <typename S, int MODE, bool ACC, bool G, bool CN>
__global__ void __launch_bounds__(kThreads, 1)
    tgemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                 const __grid_constant__ CUtensorMap mC, const __grid_constant__ TileProblem p,
                 const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB2) {
  pdl_wait();  // the previous kernel on the stream has completed (programmatic launch)
  pdl_trigger();
  if ((p.skip && *p.skip) || (p.run_if && !*p.run_if)) return;  // uniform, before any barrier exists
  const bool alt = MODE == kModeFwRest16 && !G && p.alt_if && *p.alt_if;  // uniform
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  int *sA = reinterpret_cast<int *>(smem);
  int *sB = reinterpret_cast<int *>(smem + kStages * kAStageBytes);
  int *sC = reinterpret_cast<int *>(smem + kStages * (kAStageBytes + kBStageBytes));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * (kAStageBytes + kBStageBytes) + kCBytes);
  uint64_t *full = bars, *empty = bars + kStages, *cfull = bars + 2 * kStages, *cempty = cfull + 1;
  uint64_t *tq_full = cempty + 1, *tq_empty = tq_full + kTileRing;
  volatile int *tq = reinterpret_cast<volatile int *>(tq_empty + kTileRing);
  int *dbuf = reinterpret_cast<int *>(smem + kStages * (kAStageBytes + kBStageBytes) + kCBytes + 256);
  static_assert((2 * kStages + 2 + 2 * kTileRing) * 8 + kTileRing * 4 <= 256, "barrier block");

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    mbar_init(cfull, 1);
    mbar_init(cempty, kConsumerWarps);
    for (int s = 0; s < kTileRing; ++s) {
      mbar_init(&tq_full[s], 1);
      mbar_init(&tq_empty[s], kConsumerWarps);
    }
    fence_barrier_init();
  }
  __syncthreads();
  const bool dyn = CN && p.tile_counter;  // uniform

  if (warp >= kConsumerWarps) {
    // ------------------------------- producer --------------------------------------
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegs));
    if (warp == kConsumerWarps && lane == 0) {
      const CUtensorMap *ma = alt ? &mA2 : &mA, *mb = alt ? &mB2 : &mB;
      tma_prefetch_desc(ma);
      tma_prefetch_desc(mb);
      if (ACC) tma_prefetch_desc(&mC);
      int stage = 0, tqs = 0;
      uint32_t phase = 0, cphase = 0, issued = 0, issued_par = 0, tqp = 0;
      bool c_issued = false, ok = true;
      uint32_t c_par = 0;
      // Dynamic order: the next index is fetched once the current tile is issued (the producer
      // runs about one tile ahead of the consumers, so the atomic's round trip overlaps their
      // work; fetching earlier would hold tiles back from CTAs idle at the end of the launch).
      int64_t t = blockIdx.x;
      while (ok) {
        if (dyn) {  // fetch the index and hand it to the consumers
          t = atomicAdd(p.tile_counter, 1);
          if (!mbar_wait(&tq_empty[tqs], tqp ^ 1, p.status)) { ok = false; break; }
          tq[tqs] = t < p.ntiles ? (int)t : -1;
          mbar_arrive(&tq_full[tqs]);
          if (++tqs == kTileRing) { tqs = 0; tqp ^= 1; }
        }
        if (t >= p.ntiles) break;
        const int64_t t_next = t + gridDim.x;  // the static order's next tile
        const TileCoords tc = tile_coords<MODE, G>(p, t, alt);
        if (tc.skip) {  // the consumers skip the same tiles
          t = t_next;
          continue;
        }
        if (CN && tc.wait) {  // a panel tile of a fused launch: its operands must be stored first
          if (!counter_wait(p.tile_counter + 2, (int)(2 * p.nb - 3), p.status)) { ok = false; break; }
          fence_proxy_async_global();
        }
        const int nk = (tc.k_len + kBK - 1) / kBK;
        for (int kt = 0; kt < nk; ++kt) {
          if (!mbar_wait(&empty[stage], phase ^ 1, p.status)) { ok = false; break; }
          mbar_arrive_expect_tx(&full[stage], kAStageBytes + kBStageBytes);
          tma_load_2d(sA + stage * (kBM * kBK), ma, tc.a_col + kt * kBK, tc.a_row, &full[stage]);
          tma_load_2d(sB + stage * (kBK * kBN), mb, tc.b_col, tc.b_row + kt * kBK, &full[stage]);
          issued |= 1u << stage;
          issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
          if (++stage == kStages) { stage = 0; phase ^= 1; }
        }
        if (ACC && ok) {
          if (!mbar_wait(cempty, cphase ^ 1, p.status)) { ok = false; break; }
          mbar_arrive_expect_tx(cfull, kCBytes);
          tma_load_2d(sC, &mC, tc.c_col, tc.c_row, cfull);
          c_issued = true;
          c_par = cphase;
          cphase ^= 1;
        }
        t = t_next;
      }
      // Never leave a bulk copy writing into shared memory of an exiting CTA.
      for (int s = 0; s < kStages; ++s)
        if (issued & (1u << s)) mbar_wait(&full[s], (issued_par >> s) & 1, p.status);
      if (c_issued) mbar_wait(cfull, c_par, p.status);
      // The last producer to finish has seen every other producer's final fetch: it resets the
      // counter pair for the next launch on the stream.
      if (dyn && atomicAdd(p.tile_counter + 1, 1) == (int)gridDim.x - 1) {
        p.tile_counter[0] = 0;
        p.tile_counter[1] = 0;
        p.tile_counter[2] = 0;
      }
    }
    return;
  }

  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kConsumerRegs));
  const Smem sm = {sA, sB, sC, full, empty, cfull, cempty, tq_full, tq_empty, tq, dbuf};
  if (sizeof(S) == 4 && S(0.5) != S(0)) {  // float storage
    consume<ArithF32, MODE, ACC, G, CN>(p, sm, warp, lane, 0x7f800000, true, alt);
  } else if (alt) {  // the 32-bit alternative of a packed launch (int32 storage)
    if ((p.f32_if && *p.f32_if) || (p.wmax && small_int_bound(p.wmax[0], p.wmult, p.wmax[1])))
      consume<ArithF32, MODE, ACC, G, CN>(p, sm, warp, lane, p.inf_i, false, true);
    else
      consume<ArithI32, MODE, ACC, G, CN>(p, sm, warp, lane, p.inf_i, false, true);
  } else if (p.arith16) {
    consume<ArithI16x2, MODE, ACC, G, CN>(p, sm, warp, lane, (kCap16 << 16) | kCap16, false);
  } else if ((p.f32_if && *p.f32_if) || (p.wmax && small_int_bound(p.wmax[0], p.wmult, p.wmax[1]))) {
    consume<ArithF32, MODE, ACC, G, CN>(p, sm, warp, lane, p.inf_i, false);
  } else {
    consume<ArithI32, MODE, ACC, G, CN>(p, sm, warp, lane, p.inf_i, false);
  }
}

// (min,+) pairs one launch performs by definition (Eq. 2: one add and one min per (i, j, k)).
template <int MODE> static double algorithmic_pairs(const TileProblem &p) {
  if (p.trace_pairs > 0) return p.trace_pairs;
  if (MODE == kModeGemm) return (double)p.M * (double)p.N * (double)p.K * (p.arith16 ? 2.0 : 1.0);
  const int64_t w = (MODE == kModeFwRest16 && p.bt > 1 ? p.bt : 1) * kBM;
  const double bk = (double)(p.n - p.kb * w < w ? p.n - p.kb * w : w);
  const double rest = (double)p.n - bk;
  if (MODE == kModeFwPanels) return 2.0 * bk * bk * rest;
  double pairs = rest * rest * bk;
  if (p.close_next) {  // a fused launch: phase 2 of the next block as well
    const double bk1 = (double)(p.n - (p.kb + 1) * kBM < kBM ? p.n - (p.kb + 1) * kBM : kBM);
    pairs += 2.0 * bk1 * bk1 * ((double)p.n - bk1);
  }
  return pairs;
}

template <typename T, int MODE, bool ACC, bool G = false, bool CN = false>
static int launch_one(const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mC, const TileProblem &p,
                      cudaStream_t s, const CUtensorMap &mA2, const CUtensorMap &mB2) {
  auto k = tgemm_kernel<T, MODE, ACC, G, CN>;
  static std::atomic<int> checked{0};  // 1: register split verified for this instantiation
  if (!checked.load(std::memory_order_relaxed)) {
    cudaFuncAttributes fa;
    APSP_CUDA_TRY(cudaFuncGetAttributes(&fa, k));
    // setmaxnreg.inc would wait forever if the split asked for more than the launch holds.
    if (fa.numRegs < kLaunchRegs || fa.maxThreadsPerBlock < kThreads) return APSP_ERR_UNSUPPORTED;
    checked.store(1, std::memory_order_relaxed);
  }
  APSP_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes + 1024));
  const int64_t sms = sm_count();
  const int grid = (int)(p.ntiles < sms ? p.ntiles : sms);
  void *ev = nullptr;
  const bool tr = trace_on() && !p.no_trace;
  if (tr) trace_begin(s, &ev);
  launch_pdl(k, grid, kThreads, kSmemBytes + 1024, s, mA, mB, mC, p, mA2, mB2);
  APSP_LAUNCH_CHECK();
  if (tr) trace_end(s, ev, MODE + p.trace_class, algorithmic_pairs<MODE>(p));
  return APSP_OK;
}

template <typename T>
static int launch_t(int mode, bool acc, const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mC,
                    const TileProblem &p, cudaStream_t s, const CUtensorMap &mA2, const CUtensorMap &mB2) {
  if (p.ngroups > 0) {  // grouped launches: FW modes only; packed 16-bit pairs for int32 only
    switch (mode * 2 + (acc ? 1 : 0)) {
      case 2: return launch_one<T, kModeFwPanels, false, true>(mA, mB, mC, p, s, mA2, mB2);
      case 5: return launch_one<T, kModeFwRest, true, true>(mA, mB, mC, p, s, mA2, mB2);
      case 7:
        if constexpr (std::is_same<T, int>::value) return launch_one<T, kModeFwRest16, true, true>(mA, mB, mC, p, s, mA2, mB2);
        return APSP_ERR_ARG;
      default: return APSP_ERR_ARG;
    }
  }
  switch (mode * 2 + (acc ? 1 : 0)) {
    case 0: return launch_one<T, kModeGemm, false>(mA, mB, mC, p, s, mA2, mB2);
    case 1: return launch_one<T, kModeGemm, true>(mA, mB, mC, p, s, mA2, mB2);
    case 2: return launch_one<T, kModeFwPanels, false>(mA, mB, mC, p, s, mA2, mB2);
    case 5:
      if (p.tile_counter) return launch_one<T, kModeFwRest, true, false, true>(mA, mB, mC, p, s, mA2, mB2);
      return launch_one<T, kModeFwRest, true>(mA, mB, mC, p, s, mA2, mB2);
    case 7:
      if constexpr (std::is_same<T, int>::value) {
        if (p.tile_counter) return launch_one<T, kModeFwRest16, true, false, true>(mA, mB, mC, p, s, mA2, mB2);
        return launch_one<T, kModeFwRest16, true>(mA, mB, mC, p, s, mA2, mB2);
      }
      return APSP_ERR_ARG;
    default: return APSP_ERR_ARG;
  }
}

int launch_tgemm(int mode, bool acc, int dtype, const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mC,
                 const TileProblem &p, cudaStream_t s, const CUtensorMap *mA2, const CUtensorMap *mB2) {
  if (p.ntiles <= 0) return APSP_OK;
  if (p.alt_if && (!mA2 || !mB2)) return APSP_ERR_ARG;
  const CUtensorMap &a2 = mA2 ? *mA2 : mA, &b2 = mB2 ? *mB2 : mB;
  return dtype == APSP_I32 ? launch_t<int>(mode, acc, mA, mB, mC, p, s, a2, b2)
                           : launch_t<float>(mode, acc, mA, mB, mC, p, s, a2, b2);
}

int make_operand_maps(const void *base, int64_t rows, int64_t cols, int64_t ld, int dtype, CUtensorMap *mA,
                      CUtensorMap *mB, CUtensorMap *mC) {
  int r;
  if (mA && (r = make_tmap_2d(mA, base, rows, cols, ld, kBM, kBK, dtype, true))) return r;
  if (mB && (r = make_tmap_2d(mB, base, rows, cols, ld, kBK, kBN, dtype))) return r;
  if (mC && (r = make_tmap_2d(mC, base, rows, cols, ld, kBM, kBN, dtype))) return r;
  return APSP_OK;
}

// ------------------------------ 16-bit packing -----------------------------------------
__device__ __forceinline__ bool fits16(const int *words) {
  return (int64_t)words[0] + (int64_t)words[1] < kCap16;
}
__device__ __forceinline__ int cap16(int v, int inf) { return v >= inf ? kCap16 : v; }

__global__ void __launch_bounds__(256) pack16_a_kernel(const int *A, int64_t lda, int64_t M, int64_t K, int *A16,
                                                       int64_t ld16, int inf, int *words) {
  pdl_wait();
  pdl_trigger();
  if (!fits16(words)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) words[4] = 1;
  const int64_t kw = (K + 1) >> 1;
  for (int64_t i = blockIdx.x; i < M; i += gridDim.x) {
    const int *ar = A + i * lda;
    int *o = A16 + i * ld16;
    for (int64_t w = threadIdx.x; w < kw; w += blockDim.x) {
      const int64_t k = 2 * w;
      const int lo = cap16(ar[k], inf), hi = k + 1 < K ? cap16(ar[k + 1], inf) : kCap16;
      o[w] = (hi << 16) | lo;
    }
  }
}

__global__ void __launch_bounds__(256) pack16_b_kernel(const int *B, int64_t ldb, int64_t K, int64_t N, int *B16,
                                                       int64_t ld16, int inf, int *words) {
  pdl_wait();
  pdl_trigger();
  if (!fits16(words)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) words[4] = 1;
  const int64_t kw = (K + 1) >> 1;
  for (int64_t w = blockIdx.x; w < kw; w += gridDim.x) {
    const int *r0 = B + 2 * w * ldb, *r1 = r0 + ldb;
    const bool has1 = 2 * w + 1 < K;
    int *o = B16 + w * ld16;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
      const int lo = cap16(r0[j], inf), hi = has1 ? cap16(r1[j], inf) : kCap16;
      o[j] = (hi << 16) | lo;
    }
  }
}

int launch_pack16_a(const int *A, int64_t lda, int64_t M, int64_t K, int *A16, int64_t ld16, int inf, int *words,
                    cudaStream_t s) {
  if (M == 0 || K == 0) return APSP_OK;
  const int64_t cap = (int64_t)sm_count() * 8;
  launch_pdl(pack16_a_kernel, (int)(M < cap ? M : cap), 256, 0, s, A, lda, M, K, A16, ld16, inf, words);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

int launch_pack16_b(const int *B, int64_t ldb, int64_t K, int64_t N, int *B16, int64_t ld16, int inf, int *words,
                    cudaStream_t s) {
  const int64_t kw = (K + 1) >> 1;
  if (kw == 0 || N == 0) return APSP_OK;
  const int64_t cap = (int64_t)sm_count() * 8;
  launch_pdl(pack16_b_kernel, (int)(kw < cap ? kw : cap), 256, 0, s, B, ldb, K, N, B16, ld16, inf, words);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

// ------------------------------ generic fallback --------------------------------------
// Plain-load tiled kernel for operands that break TMA's 16-byte rules.  64 x 64 tiles,
// 16-deep k-slabs, 4 x 4 register tile per thread; out-of-range k reads as INF.
template <typename T>
__global__ void __launch_bounds__(256) tgemm_generic_kernel(T *C, const T *A, const T *B, int64_t M, int64_t N,
                                                            int64_t K, int64_t lda, int64_t ldb, int64_t ldc, bool acc,
                                                            T inf) {
  __shared__ T As[64][17];
  __shared__ T Bs[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
  T c[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[i][j] = inf;
  for (int64_t k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int r = e >> 4, k = e & 15;
      const int64_t gm = m0 + r, gk = k0 + k;
      As[r][k] = (gm < M && gk < K) ? A[gm * lda + gk] : inf;
      const int kr = e >> 6, cn = e & 63;
      const int64_t gk2 = k0 + kr, gn = n0 + cn;
      Bs[kr][cn] = (gk2 < K && gn < N) ? B[gk2 * ldb + gn] : inf;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[i][j] = Ops<T>::mn(c[i][j], Ops<T>::add(As[ty + 16 * i][k], Bs[k][tx + 16 * j]));
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) {
        T v = c[i][j];
        if (acc) v = Ops<T>::mn(v, C[gm * ldc + gn]);
        C[gm * ldc + gn] = v;
      }
    }
}

int launch_tgemm_generic(void *C, const void *A, const void *B, int64_t M, int64_t N, int64_t K, int64_t lda,
                         int64_t ldb, int64_t ldc, int dtype, bool acc, int inf_i, float inf_f, cudaStream_t s) {
  if (M == 0 || N == 0) return APSP_OK;
  dim3 grid((unsigned)cdiv(N, 64), (unsigned)cdiv(M, 64));
  if (grid.y > 65535) return APSP_ERR_ARG;
  if (dtype == APSP_I32)
    tgemm_generic_kernel<int><<<grid, 256, 0, s>>>((int *)C, (const int *)A, (const int *)B, M, N, K, lda, ldb, ldc,
                                                   acc, inf_i);
  else
    tgemm_generic_kernel<float><<<grid, 256, 0, s>>>((float *)C, (const float *)A, (const float *)B, M, N, K, lda,
                                                     ldb, ldc, acc, INFINITY);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

// ------------------------------------ copy --------------------------------------------
__global__ void __launch_bounds__(256) copy2d_kernel(int *dst, int64_t ldd, const int *src, int64_t lds, int64_t rows,
                                                     int64_t cols, bool vec, const int *run_if) {
  pdl_wait();
  pdl_trigger();
  if (run_if && !*run_if) return;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int *s = src + r * lds;
    int *d = dst + r * ldd;
    int64_t c0 = 0;
    if (vec) {
      for (int64_t v = threadIdx.x; v < (cols >> 2); v += blockDim.x)
        reinterpret_cast<int4 *>(d)[v] = reinterpret_cast<const int4 *>(s)[v];
      c0 = (cols >> 2) << 2;
    }
    for (int64_t c = c0 + threadIdx.x; c < cols; c += blockDim.x) d[c] = s[c];
  }
}

int launch_copy2d(void *dst, int64_t ldd, const void *src, int64_t lds, int64_t rows, int64_t cols, cudaStream_t s,
                  const int *run_if) {
  if (rows == 0 || cols == 0) return APSP_OK;
  const bool vec = reinterpret_cast<uintptr_t>(dst) % 16 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 &&
                   ldd % 4 == 0 && lds % 4 == 0;
  const int64_t cap = (int64_t)sm_count() * 8;
  launch_pdl(copy2d_kernel, (int)(rows < cap ? rows : cap), 256, 0, s, (int *)dst, ldd, (const int *)src, lds, rows,
             cols, vec, run_if);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

}  // namespace apsp

// ------------------------------------ C ABI -------------------------------------------
namespace apsp {
// Workspace of the packed 16-bit path of tropical_gemm: A16 (M x round_up(ceil(K/2), 4) words)
// and B16 (ceil(K/2) x round_up(N, 4) words) after the bound words.
static size_t packed16_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t kw = (K + 1) >> 1;
  return (size_t)round_up(M * round_up(kw, 4) * 4, 256) + (size_t)round_up(kw * round_up(N, 4) * 4, 256);
}
}  // namespace apsp

extern "C" size_t tropical_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int dtype) {
  using namespace apsp;
  if (dtype != APSP_I32 || M <= 0 || N <= 0 || K <= 0) return kFlagBytes;
  return kFlagBytes + packed16_bytes(M, N, K);
}

extern "C" int tropical_gemm(void *C, const void *A, const void *B, int64_t M, int64_t N, int64_t K, int64_t lda,
                             int64_t ldb, int64_t ldc, int dtype, const void *inf, int accumulate, void *ws,
                             size_t ws_bytes, void *stream) {
  using namespace apsp;
  if (!dtype_ok(dtype) || M < 0 || N < 0 || K < 0) return APSP_ERR_ARG;
  if (M == 0 || N == 0) return APSP_OK;
  if (!C || (K > 0 && (!A || !B)) || ldc < N || (K > 0 && (lda < K || ldb < N))) return APSP_ERR_ARG;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return APSP_ERR_ARG;
  if (ws && (ws_bytes < kFlagBytes || reinterpret_cast<uintptr_t>(ws) % 256 != 0)) return APSP_ERR_ARG;
  // C must not overlap A or B (byte ranges of the strided extents).
  auto span = [](const void *p, int64_t rows, int64_t cols, int64_t ld) {
    return std::make_pair((uintptr_t)p, (uintptr_t)p + (uintptr_t)(((rows - 1) * ld + cols) * 4));
  };
  auto cs = span(C, M, N, ldc);
  if (K > 0) {
    auto as = span(A, M, K, lda), bs = span(B, K, N, ldb);
    if ((cs.first < as.second && as.first < cs.second) || (cs.first < bs.second && bs.first < cs.second))
      return APSP_ERR_ARG;
  }
  int inf_i = 0;
  float inf_f = 0.f;
  if (dtype == APSP_I32 ? resolve_inf_i32(inf, &inf_i) : resolve_inf_f32(inf, &inf_f)) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool aligned = (uintptr_t)C % 16 == 0 && (K == 0 || ((uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0)) &&
                       ldc % 4 == 0 && (K == 0 || (lda % 4 == 0 && ldb % 4 == 0));
  if (!aligned) return launch_tgemm_generic(C, A, B, M, N, K, lda, ldb, ldc, dtype, accumulate != 0, inf_i, inf_f, s);
  CUtensorMap mA, mB, mC;
  int r;
  if ((r = make_operand_maps(K > 0 ? A : C, K > 0 ? M : 1, K > 0 ? K : 4, K > 0 ? lda : 4, dtype, &mA, nullptr, nullptr)))
    return r;
  if ((r = make_operand_maps(K > 0 ? B : C, K > 0 ? K : 1, N, K > 0 ? ldb : ldc, dtype, nullptr, &mB, nullptr))) return r;
  if ((r = make_operand_maps(C, M, N, ldc, dtype, nullptr, nullptr, &mC))) return r;
  void *own = nullptr;
  int *words = nullptr;
  const size_t p16 = dtype == APSP_I32 ? packed16_bytes(M, N, K) : 0;
  if (dtype == APSP_I32) {  // largest finite entries of A and B decide the exact fp32 path
    if (!ws) {
      ws_bytes = tropical_gemm_workspace_bytes(M, N, K, dtype);
      if (ws_alloc(&own, ws_bytes, s) != APSP_OK) {
        return APSP_ERR_NOMEM;
      }
      ws = own;
    }
    words = reinterpret_cast<int *>(ws);
    if (cudaMemsetAsync(words, 0, 32, s) != cudaSuccess) r = APSP_ERR_CUDA;
    if (!r && K > 0) r = launch_scan_max(A, M, K, lda, inf_i, words, s);
    if (!r && K > 0) r = launch_scan_max(B, K, N, ldb, inf_i, words + 1, s);
  }
  TileProblem p = {};
  p.M = M; p.N = N; p.K = K;
  p.tiles_m = cdiv(M, kBM);
  p.tiles_n = cdiv(N, kBN);
  p.ntiles = p.tiles_m * p.tiles_n;
  p.C = C;
  p.ldc = ldc;
  p.inf_i = inf_i;
  p.inf_f = inf_f;
  p.status = status_word();
  p.wmax = words;
  p.wmult = 1;
  // int32 with room for the packed copies: when the largest finite entries of A and B sum
  // below 0x3FFF (checked by the pack kernels on the device), the product runs on 16-bit pairs,
  // two (min,+) pairs per DPX operation; the plain launch then returns at once.
  void *tev = nullptr;
  const bool group = !r && dtype == APSP_I32 && K > 0 && ws_bytes >= kFlagBytes + p16;
  if (group && trace_on()) trace_begin(s, &tev);
  if (group) {
    const int64_t kw = (K + 1) >> 1, lda16 = round_up(kw, 4), ldb16 = round_up(N, 4);
    int *A16 = reinterpret_cast<int *>(reinterpret_cast<uint8_t *>(ws) + kFlagBytes);
    int *B16 = reinterpret_cast<int *>(reinterpret_cast<uint8_t *>(A16) + round_up(M * lda16 * 4, 256));
    r = launch_pack16_a(reinterpret_cast<const int *>(A), lda, M, K, A16, lda16, inf_i, words, s);
    if (!r) r = launch_pack16_b(reinterpret_cast<const int *>(B), ldb, K, N, B16, ldb16, inf_i, words, s);
    CUtensorMap pA, pB;
    if (!r) r = make_operand_maps(A16, M, kw, lda16, APSP_I32, &pA, nullptr, nullptr);
    if (!r) r = make_operand_maps(B16, kw, N, ldb16, APSP_I32, nullptr, &pB, nullptr);
    if (!r) {
      TileProblem q = p;
      q.K = kw;
      q.arith16 = 1;
      q.run_if = words + 4;
      q.no_trace = 1;
      r = launch_tgemm(kModeGemm, accumulate != 0, dtype, pA, pB, mC, q, s);
    }
    p.skip = words + 4;
    p.no_trace = 1;
  }
  if (!r) r = launch_tgemm(kModeGemm, accumulate != 0, dtype, mA, mB, mC, p, s);
  if (tev) trace_end(s, tev, kModeGemm, (double)M * (double)N * (double)K);
  ws_free(own, s);
  return r;
}
