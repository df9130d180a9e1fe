// grouped.cu -- a7 for the larger graphs of a batch: blocked Floyd-Warshall over many graphs in
// lockstep on the TMA engine.
//
// The persistent batched kernel closes each graph on one CTA with its own cp.async pipeline.
// For graphs of a few hundred vertices and more, that per-CTA pipeline runs well below the
// engine's rate, and those graphs carry nearly all of a batch's work (n^3).  Here they are
// closed together instead: copied ("staged") one below the other into one tall matrix with a
// common leading dimension, each padded to nb whole 128-tiles with isolated vertices (0 on the
// diagonal, the sentinel elsewhere; they change no distance).  Graphs are grouped by nb, and
// the groups are listed by decreasing nb, so the graphs still open at block kb (nb > kb) are a
// prefix of the staged list.  Per block kb one launch runs a step for every open graph:
//   phase 1  one CTA per graph closes its diagonal tile (Eq. 1, in registers, on packed
//            16-bit pairs: two entries per DPX add-min);
//   phase 2  the engine's panel mode on the packed panels (two (min,+) pairs per DPX op),
//            each tile also writing its result packed, as phase 3's operand;
//   phase 3  the engine's 16-bit phase 3 over all graphs' remaining tiles.
// The packed panels a step reads are written, already packed, by the kernels that produce the
// values: the diagonal kernel for its tile, and the previous step's phase-2 and phase-3 tiles
// of block row and column kb (two alternating buffer sets); only step 0 packs them in a pass.
// All three compute the closure truncated at CAP = 0x3FFF (truncation is a homomorphism of
// (min,+), so exact and truncated steps could even be mixed), certified per graph exactly as
// apsp_fw certifies one matrix: the largest stored value below CAP plus the graph's largest
// weight must stay below CAP; then every entry at or above CAP is unreachable.
// Graphs whose certificate fails, and graphs whose weights exceed CAP / 4, are finished by a
// second lockstep pass in int32 (exact fp32 on the int32 bit patterns when every (n - 1) *
// largest weight < 2^24) over the mapped matrix, which lies between the distances and the
// weights; that pass's launches return at once when no graph needs it.  Results are identical
// to closing each graph alone.
//
// Float32 batches stage the same way (the sentinel and the padding are +infinity) and run only
// the second pass, in fp32 (the engine's packed pair add and 3-input min), with no certificate.
//
// The plan (which graphs, their order and rows) is made on the host from the host copy of the
// sizes and reaches the device as kernel arguments, so the whole sequence can be captured in a
// CUDA graph.  Graphs whose device size, leading dimension or offset disagree with the plan are
// left untouched and flagged (APSP_ERR_ARG), as the persistent kernel does.
#include <algorithm>
#include <climits>
#include <vector>

#include "diag.cuh"
#include "grouped.cuh"
#include "tgemm.cuh"

namespace apsp {

namespace {

constexpr int kGfUse16 = 1, kGfRerun = 2, kGfBad = 4;
// Words of the 256-byte block at the front of the workspace (the persistent kernel's queue
// counters are words 0 and 1): [8] largest (n - 1) * weight over the staged graphs, [9] 0,
// [10] some graph needs the int32 pass.
constexpr int kWBound = 8, kWRerun = 10;
constexpr int kPlanChunk = 4096;

struct GroupSet {
  int ngroups;
  GraphGroup groups[kMaxGroups];
};

struct PlanChunk {
  int *dst;
  int n;
  int idx[kPlanChunk];
};

struct StageArgs {
  GroupSet gs;
  int *S;
  int64_t ldS, R;
  int *pool;
  const int64_t *offsets;
  const int32_t *ns, *lds;
  const int *sidx;
  int *gflags, *maxb, *wmaxg, *gsize, *words;
  int inf;       // int32: the sentinel; float32: the bits of +infinity (what staging writes)
  float inf_f;   // float32: the caller's sentinel (entries at or above it are missing edges)
  int is_float;
  unsigned int *status;
};

// Staged graph holding staged row r: its index q, first row and nb.
__device__ __forceinline__ bool row_graph(const GroupSet &gs, int64_t r, int &q, int64_t &base, int &nb) {
  bool found = false;
#pragma unroll
  for (int k = 0; k < kMaxGroups; ++k) {
    if (!found && k < gs.ngroups) {
      const GraphGroup &g = gs.groups[k];
      const int64_t rows = (int64_t)g.nb * kBM;
      if (r >= g.row0 && r < g.row0 + rows * g.count) {
        const int64_t ql = (r - g.row0) / rows;
        q = g.first + (int)ql;
        base = g.row0 + ql * rows;
        nb = g.nb;
        found = true;
      }
    }
  }
  return found;
}

// First row and nb of staged graph q.
__device__ __forceinline__ void graph_rows(const GroupSet &gs, int q, int64_t &base, int &nb) {
#pragma unroll
  for (int k = 0; k < kMaxGroups; ++k) {
    if (k < gs.ngroups) {
      const GraphGroup &g = gs.groups[k];
      if (q >= g.first && q < g.first + g.count) {
        nb = g.nb;
        base = g.row0 + (int64_t)(q - g.first) * g.nb * kBM;
      }
    }
  }
}

__global__ void plan_kernel(const __grid_constant__ PlanChunk c) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.n; i += gridDim.x * blockDim.x) c.dst[i] = c.idx[i];
}

__device__ __forceinline__ bool graph_ok(const StageArgs &a, int g, int nb, int &n, int &ld, int64_t &off) {
  n = a.ns[g];
  ld = a.lds[g];
  off = a.offsets[g];
  return n > 0 && ld >= n && !(ld & 3) && !(off & 3) && off >= 0 && (n + kBM - 1) / kBM == nb;
}

// One entry of a1 (column c of row i): the diagonal becomes 0, an entry at or above the
// sentinel becomes a.inf (int32: the sentinel; float32: +infinity), a negative entry (float32:
// or NaN) is flagged.  m keeps the largest finite int32 weight.
__device__ __forceinline__ int stage_entry(const StageArgs &a, int x, int c, int i, bool &bad, int &m) {
  if (c == i) return 0;
  if (a.is_float) {
    const float f = __int_as_float(x);
    bad |= !(f >= 0.f);
    if (f == 0.f) return 0;  // -0 stored as +0
    return f >= a.inf_f ? a.inf : x;
  }
  bad |= x < 0;
  x = x >= a.inf ? a.inf : x;
  if (x < a.inf) m = max(m, x);
  return x;
}

// a1 into the staging matrix, one warp per staged row: zero diagonal, entries >= inf become
// inf, negative entries flag APSP_ERR_DOMAIN; padding rows and columns are isolated vertices.
// The largest finite weight of each int32 graph is maxed into wmaxg[q].
__global__ void __launch_bounds__(256) stage_in_kernel(const StageArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < a.R; r += warps) {
    int q = 0, nb = 0;
    int64_t base = 0;
    if (!row_graph(a.gs, r, q, base, nb)) continue;
    const int g = a.sidx[q];
    int n = 0, ld = 0;
    int64_t off = 0;
    const bool ok = graph_ok(a, g, nb, n, ld, off);
    const int i = (int)(r - base), w = nb * kBM;
    int *dst = a.S + r * a.ldS;
    if (!ok) {
      if (i == 0 && lane == 0) {
        atomicOr(a.gflags + q, kGfBad);
        flag_status(a.status, APSP_ERR_ARG);
      }
      for (int c = lane * 4; c < w; c += 128) {
        int4 v = make_int4(a.inf, a.inf, a.inf, a.inf);
        if (i >= c && i < c + 4) (&v.x)[i - c] = 0;
        *reinterpret_cast<int4 *>(dst + c) = v;
      }
      continue;
    }
    const int *src = a.pool + off + (int64_t)i * ld;
    bool bad = false;
    int m = 0;
    for (int c = lane * 4; c < w; c += 128) {
      int4 v = make_int4(a.inf, a.inf, a.inf, a.inf);
      if (i < n) {
        if (c + 3 < n) {
          v = *reinterpret_cast<const int4 *>(src + c);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (c + e < n) (&v.x)[e] = src[c + e];
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) (&v.x)[e] = stage_entry(a, (&v.x)[e], c + e, i, bad, m);
      *reinterpret_cast<int4 *>(dst + c) = v;
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (__any_sync(0xffffffffu, bad) && lane == 0) flag_status(a.status, APSP_ERR_DOMAIN);
    if (lane == 0 && m > 0) atomicMax(a.wmaxg + q, m);
  }
}

// Per graph: the 16-bit pass is used when the largest weight is at most CAP / 4 (else the
// int32 pass does all the work), and the bound word for exact fp32 arithmetic.  Float32
// graphs all take the second pass.
__global__ void stage_decide_kernel(const StageArgs a, int64_t G) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < G; q += (int64_t)gridDim.x * blockDim.x) {
    if (a.gflags[q] & kGfBad) continue;
    const int w = a.wmaxg[q], n = a.ns[a.sidx[q]];
    a.gsize[q] = n;
    if (a.is_float) {
      a.gflags[q] |= kGfRerun;
      a.words[kWRerun] = 1;
      continue;
    }
    const int64_t prod = (int64_t)(n - 1) * (int64_t)w;
    atomicMax(a.words + kWBound, (int)(prod < INT_MAX ? prod : INT_MAX));
    if (w <= kCap16 / 4) {
      a.gflags[q] |= kGfUse16;
    } else {
      a.gflags[q] |= kGfRerun;
      a.words[kWRerun] = 1;
    }
  }
}

// Phase 1 of the truncated pass on packed 16-bit pairs.  The thread owning rows tm + 16 i and
// columns 4 tn + 64 h + q (the layout of diag.cuh) keeps w[i][2 h + p] = {d[i][4 tn + 64 h +
// 2 p], d[i][... + 1]}, values capped at CAP.  Step k: the owner of row k publishes its four
// words (the row, packed), the owners of column k publish d[i][k] in both lanes; then one DPX
// add-min per word relaxes two entries: w = min(w, {c, c} + {r0, r1}).
template <int KH>
__device__ __forceinline__ void put_row16(const int (&w)[8][4], int *rb, int tn) {
  *reinterpret_cast<int2 *>(rb + 2 * tn) = make_int2(w[KH][0], w[KH][1]);
  *reinterpret_cast<int2 *>(rb + 2 * tn + 32) = make_int2(w[KH][2], w[KH][3]);
}

template <int WJ, int HI>
__device__ __forceinline__ void put_col16(const int (&w)[8][4], int *cb, int tm) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int v = HI ? (int)((unsigned)w[i][WJ] >> 16) : (w[i][WJ] & 0xFFFF);
    cb[tm + 16 * i] = (v << 16) | v;
  }
}

__device__ void close_tile_regs16(int (&w)[8][4], int bk, int tm, int tn, int *buf) {
#pragma unroll
  for (int kh = 0; kh < 8; ++kh) {
    if (16 * kh >= bk) break;
    for (int kl = 0; kl < 16; ++kl) {
      const int k = 16 * kh + kl;
      if (k >= bk) break;
      int *rb = buf + (k & 1) * 256;
      int *cb = rb + 128;
      if (tm == kl) {
        switch (kh) {
          case 0: put_row16<0>(w, rb, tn); break;
          case 1: put_row16<1>(w, rb, tn); break;
          case 2: put_row16<2>(w, rb, tn); break;
          case 3: put_row16<3>(w, rb, tn); break;
          case 4: put_row16<4>(w, rb, tn); break;
          case 5: put_row16<5>(w, rb, tn); break;
          case 6: put_row16<6>(w, rb, tn); break;
          default: put_row16<7>(w, rb, tn); break;
        }
      }
      if (tn == ((k >> 2) & 15)) {  // column k = 4 tn + q + 64 h: word 2 h + q / 2, lane q % 2
        switch (2 * (k >> 6) + ((k >> 1) & 1) + 4 * (k & 1)) {
          case 0: put_col16<0, 0>(w, cb, tm); break;
          case 1: put_col16<1, 0>(w, cb, tm); break;
          case 2: put_col16<2, 0>(w, cb, tm); break;
          case 3: put_col16<3, 0>(w, cb, tm); break;
          case 4: put_col16<0, 1>(w, cb, tm); break;
          case 5: put_col16<1, 1>(w, cb, tm); break;
          case 6: put_col16<2, 1>(w, cb, tm); break;
          default: put_col16<3, 1>(w, cb, tm); break;
        }
      }
      __syncthreads();
      int c[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) c[i] = cb[tm + 16 * i];
      const int2 r0 = *reinterpret_cast<const int2 *>(rb + 2 * tn);
      const int2 r1 = *reinterpret_cast<const int2 *>(rb + 2 * tn + 32);
      const int r[4] = {r0.x, r0.y, r1.x, r1.y};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          w[i][j] = (int)__viaddmin_s16x2((unsigned)c[i], (unsigned)r[j], (unsigned)w[i][j]);
    }
  }
  __syncthreads();  // buf is reused by the caller
}

// Phase 1 for every graph with nb > kb (a prefix of the staged list: one CTA each) that the
// mask admits.  run_if (may be null): every CTA returns at once unless *run_if is set.  With
// truncated (the 16-bit pass), the tile is closed on packed 16-bit pairs and its part of the
// step's packed column and row panels is written to pa / pb.
__global__ void __launch_bounds__(256, 2) group_diag_kernel(int *S, int64_t ldS, GroupSet gs, int kb, const int *gflags,
                                                         const int *gsize, int mask, int want, const int *run_if,
                                                         bool truncated, int *pa, int *pb, bool is_float) {
  if (run_if && !*run_if) return;
  const int q = blockIdx.x;
  if ((gflags[q] & mask) != want) return;
  int64_t base = 0;
  int nb = 0;
  graph_rows(gs, q, base, nb);
  if (nb <= kb) return;
  __shared__ __align__(16) int buf[512];
  int *T = S + (base + (int64_t)kb * kBM) * ldS + (int64_t)kb * kBM;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (warp & 3) * 4 + (lane >> 3), tn = (warp >> 2) * 8 + (lane & 7);
  const int left = gsize[q] - kb * kBM;  // the padding vertices past the graph need no steps
  const int bk = left < kBM ? (left > 0 ? left : 1) : kBM;
  int r[8][8];
  load_tile_regs(r, T, ldS, kBM, tm, tn);
  if (truncated) {  // the 16-bit pass: packed pairs, values capped at CAP
    int w[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) w[i][j] = (min(r[i][2 * j + 1], kCap16) << 16) | min(r[i][2 * j], kCap16);
    close_tile_regs16(w, bk, tm, tn, buf);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        r[i][2 * j] = w[i][j] & 0xFFFF;
        r[i][2 * j + 1] = (int)((unsigned)w[i][j] >> 16);
      }
  } else if (is_float) {
    close_tile_regs<true>(r, bk, tm, tn, buf);
  } else {
    close_tile_regs<false>(r, bk, tm, tn, buf);
  }
  store_tile_regs(r, T, ldS, kBM, tm, tn);
  if (pa) {  // the closed tile's part of this step's packed column and row panels
    store_col_pairs16(r, tm, tn, pa + (base + (int64_t)kb * kBM) * 64);
    store_row_pairs16(r, tm, tn, lane, pb + (int64_t)q * 64 * ldS + (int64_t)kb * kBM, ldS);
  }
}

// Packs, for graph blockIdx.x of the 16-bit pass (open at block kb), its column panel (its
// rows x 64 words, at the same rows of A16) and its row panel (64 words x its columns, at rows
// 64 q of B16) as 16-bit pairs of consecutive k, every value capped at CAP; the diagonal tile
// is part of both.  blockIdx.y splits a graph's rows among gridDim.y CTAs.
__device__ __forceinline__ int pack_pair(int lo, int hi) { return (min(hi, kCap16) << 16) | min(lo, kCap16); }

__global__ void __launch_bounds__(256) group_pack16_kernel(const int *S, int64_t ldS, GroupSet gs, int kb,
                                                           const int *gflags, int *A16, int *B16) {
  const int q = blockIdx.x;
  if ((gflags[q] & (kGfBad | kGfUse16)) != kGfUse16) return;
  int64_t base = 0;
  int nb = 0;
  graph_rows(gs, q, base, nb);
  if (nb <= kb) return;
  const int W = nb * kBM, kb0 = kb * kBM, t = threadIdx.x;
  const int *D = S + base * ldS;
  // Column panel: row r, word w = t % 64 (a coalesced 512-byte row segment per 64 threads).
  for (int r = blockIdx.y * 4 + (t >> 6); r < W; r += gridDim.y * 4) {
    const int w = t & 63;
    const int2 v = *reinterpret_cast<const int2 *>(D + (int64_t)r * ldS + kb0 + 2 * w);
    A16[(base + r) * 64 + w] = pack_pair(v.x, v.y);
  }
  // Row panel: word row w, four columns per thread.
  const int quads = W / 4;
  for (int e = blockIdx.y * 256 + t; e < 64 * quads; e += gridDim.y * 256) {
    const int w = e / quads, c = 4 * (e - w * quads);
    const int4 lo = *reinterpret_cast<const int4 *>(D + (int64_t)(kb0 + 2 * w) * ldS + c);
    const int4 hi = *reinterpret_cast<const int4 *>(D + (int64_t)(kb0 + 2 * w + 1) * ldS + c);
    *reinterpret_cast<int4 *>(B16 + ((int64_t)q * 64 + w) * ldS + c) =
        make_int4(pack_pair(lo.x, hi.x), pack_pair(lo.y, hi.y), pack_pair(lo.z, hi.z), pack_pair(lo.w, hi.w));
  }
}

// For graphs of the 16-bit pass, in one pass over each graph's n x n part: maxb[q] = the
// largest stored value below CAP; every entry at or above CAP becomes the sentinel; the
// results go to the caller's pool, and the mapped entries also back into the staging matrix
// (the int32 pass starts from them if the certificate fails).  One warp per staged row.
__global__ void __launch_bounds__(256) certify_out_kernel(const StageArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < a.R; r += warps) {
    int q = 0, nb = 0;
    int64_t base = 0;
    if (!row_graph(a.gs, r, q, base, nb)) continue;
    if ((a.gflags[q] & (kGfBad | kGfUse16)) != kGfUse16) continue;
    const int g = a.sidx[q];
    const int n = a.ns[g], ld = a.lds[g];
    const int i = (int)(r - base);
    if (i >= n) continue;
    int *row = a.S + r * a.ldS;
    int *dst = a.pool + a.offsets[g] + (int64_t)i * ld;
    int m = 0;
    for (int c = lane * 4; c < n; c += 128) {
      int4 v = *reinterpret_cast<const int4 *>(row + c);
      bool changed = false;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = (&v.x)[e];
        if (c + e >= n) continue;
        if (x < kCap16) {
          m = max(m, x);
        } else if (x != a.inf) {
          (&v.x)[e] = a.inf;
          changed = true;
        }
      }
      if (changed) *reinterpret_cast<int4 *>(row + c) = v;
      if (c + 3 < n) {
        *reinterpret_cast<int4 *>(dst + c) = v;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (c + e < n) dst[c + e] = (&v.x)[e];
      }
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0 && m > 0) atomicMax(a.maxb + q, m);
  }
}

__global__ void group_verdict_kernel(const StageArgs a, int64_t G) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < G; q += (int64_t)gridDim.x * blockDim.x) {
    if ((a.gflags[q] & (kGfBad | kGfUse16)) != kGfUse16) continue;
    if ((int64_t)a.maxb[q] + (int64_t)a.wmaxg[q] >= kCap16) {
      a.gflags[q] |= kGfRerun;
      a.words[kWRerun] = 1;
    }
  }
}

// The closed n x n part of every staged graph of the int32 pass back into the caller's pool
// (the others went back with the certificate); returns at once when no graph needed the pass.
__global__ void __launch_bounds__(256) stage_out_kernel(const StageArgs a) {
  if (!a.words[kWRerun]) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < a.R; r += warps) {
    int q = 0, nb = 0;
    int64_t base = 0;
    if (!row_graph(a.gs, r, q, base, nb)) continue;
    if ((a.gflags[q] & (kGfBad | kGfRerun)) != kGfRerun) continue;
    const int g = a.sidx[q];
    const int n = a.ns[g], ld = a.lds[g];
    const int i = (int)(r - base);
    if (i >= n) continue;
    const int *src = a.S + r * a.ldS;
    int *dst = a.pool + a.offsets[g] + (int64_t)i * ld;
    for (int c = lane * 4; c < n; c += 128) {
      const int4 v = *reinterpret_cast<const int4 *>(src + c);
      if (c + 3 < n) {
        *reinterpret_cast<int4 *>(dst + c) = v;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (c + e < n) dst[c + e] = (&v.x)[e];
      }
    }
  }
}

struct Layout {
  size_t gflags, maxb, wmaxg, gsize, lists, S, A16[2], B16[2], total;
};

Layout layout_of(const StagePlan &pl, int64_t count, int dtype) {
  Layout L;
  size_t o = kFlagBytes;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (size_t)round_up((int64_t)bytes, 256);
    return at;
  };
  L.gflags = take(pl.G * 4);
  L.maxb = take(pl.G * 4);
  L.wmaxg = take(pl.G * 4);
  L.gsize = take(pl.G * 4);
  L.lists = take((size_t)count * 4);
  L.S = take((size_t)pl.R * pl.NP * 4);
  for (int k = 0; k < 2; ++k) {  // two sets: block step kb reads set kb & 1, writes the other
    L.A16[k] = dtype == APSP_I32 ? take((size_t)pl.R * 64 * 4) : 0;
    L.B16[k] = dtype == APSP_I32 ? take((size_t)pl.G * 64 * pl.NP * 4) : 0;
  }
  L.total = o;
  return L;
}

int launch_plan_lists(int *dst, const std::vector<int> &idx, cudaStream_t s) {
  for (size_t at = 0; at < idx.size(); at += kPlanChunk) {
    PlanChunk c;
    c.dst = dst + at;
    c.n = (int)std::min<size_t>(kPlanChunk, idx.size() - at);
    std::copy(idx.begin() + at, idx.begin() + at + c.n, c.idx);
    plan_kernel<<<(c.n + 255) / 256, 256, 0, s>>>(c);
    APSP_LAUNCH_CHECK();
  }
  return APSP_OK;
}

}  // namespace

bool make_stage_plan(const int32_t *ns_host, int64_t count, StagePlan &pl) {
  pl = StagePlan();
  if (!ns_host || count <= 0 || count > (1 << 24)) return false;
  std::vector<int64_t> per_nb(kGroupMaxNb + 1, 0);
  for (int64_t g = 0; g < count; ++g) {
    const int n = ns_host[g];
    const int nb = n > 0 ? (n + kBM - 1) / kBM : 0;
    if (nb >= kGroupMinNb && nb <= kGroupMaxNb) ++per_nb[nb];
  }
  std::vector<int> chosen;  // the kMaxGroups largest block counts present, decreasing
  for (int nb = kGroupMaxNb; nb >= kGroupMinNb && (int)chosen.size() < kMaxGroups; --nb)
    if (per_nb[nb] > 0) chosen.push_back(nb);
  if (chosen.empty()) return false;
  std::vector<int> order(count);
  for (int64_t g = 0; g < count; ++g) order[g] = (int)g;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ns_host[x] > ns_host[y]; });
  std::vector<char> staged(count, 0);
  int64_t row = 0;
  for (int nb : chosen) {
    GraphGroup gg = {};
    gg.row0 = row;
    gg.first = (int)pl.staged.size();
    gg.nb = nb;
    for (int g : order) {
      const int n = ns_host[g];
      if (n > 0 && (n + kBM - 1) / kBM == nb) {
        pl.staged.push_back(g);
        pl.sizes.push_back(n);
        staged[g] = 1;
        ++gg.count;
      }
    }
    row += (int64_t)gg.count * nb * kBM;
    pl.groups[pl.ngroups++] = gg;
  }
  for (int g : order)
    if (!staged[g]) pl.rest.push_back(g);
  pl.G = (int64_t)pl.staged.size();
  pl.R = row;
  pl.NP = chosen.front() * kBM;
  if (pl.R > (int64_t)1 << 30) {  // keeps every staged row index an int
    pl = StagePlan();
    return false;
  }
  return true;
}

size_t staged_workspace_bytes(const StagePlan &pl, int64_t count, int dtype) {
  return layout_of(pl, count, dtype).total;
}

int batched_staged(const StagePlan &pl, int *pool, const int64_t *offsets, const int32_t *ns, const int32_t *lds,
                   int64_t count, int dtype, int inf_i, float inf_f, void *ws,
                   int (*launch_rest)(void *ctx, const int *order, int64_t nq), void *ctx, cudaStream_t s) {
  const bool isf = dtype == APSP_F32;
  const Layout L = layout_of(pl, count, dtype);
  uint8_t *w = reinterpret_cast<uint8_t *>(ws);
  int *words = reinterpret_cast<int *>(w);
  StageArgs a = {};
  a.gs.ngroups = pl.ngroups;
  for (int k = 0; k < pl.ngroups; ++k) a.gs.groups[k] = pl.groups[k];
  a.S = reinterpret_cast<int *>(w + L.S);
  a.ldS = pl.NP;
  a.R = pl.R;
  a.pool = pool;
  a.offsets = offsets;
  a.ns = ns;
  a.lds = lds;
  int *lists = reinterpret_cast<int *>(w + L.lists);
  a.sidx = lists;
  a.gflags = reinterpret_cast<int *>(w + L.gflags);
  a.maxb = reinterpret_cast<int *>(w + L.maxb);
  a.wmaxg = reinterpret_cast<int *>(w + L.wmaxg);
  a.gsize = reinterpret_cast<int *>(w + L.gsize);
  a.words = words;
  a.inf = isf ? 0x7f800000 : inf_i;
  a.inf_f = inf_f;
  a.is_float = isf;
  a.status = status_word();
  int *A16[2] = {reinterpret_cast<int *>(w + L.A16[0]), reinterpret_cast<int *>(w + L.A16[1])};
  int *B16[2] = {reinterpret_cast<int *>(w + L.B16[0]), reinterpret_cast<int *>(w + L.B16[1])};

  APSP_CUDA_TRY(cudaMemsetAsync(words + kWBound, 0, 4 * sizeof(int), s));
  APSP_CUDA_TRY(cudaMemsetAsync(w + L.gflags, 0, L.lists - L.gflags, s));  // gflags, maxb, wmaxg, gsize
  std::vector<int> all(pl.staged);
  all.insert(all.end(), pl.rest.begin(), pl.rest.end());
  int r;
  if ((r = launch_plan_lists(lists, all, s))) return r;

  // The graphs left out of the staging go to the persistent kernel first.
  if (!pl.rest.empty() && (r = launch_rest(ctx, lists + pl.G, (int64_t)pl.rest.size()))) return r;

  const int64_t cap = (int64_t)sm_count() * 8;
  const int row_grid = (int)std::min<int64_t>(cap, cdiv(pl.R, 8));
  const int g_grid = (int)std::min<int64_t>(cap, cdiv(pl.G, 256));
  stage_in_kernel<<<row_grid, 256, 0, s>>>(a);
  APSP_LAUNCH_CHECK();
  stage_decide_kernel<<<g_grid, 256, 0, s>>>(a, pl.G);
  APSP_LAUNCH_CHECK();

  CUtensorMap mA, mB, mC, pA[2], pB[2];
  if ((r = make_operand_maps(a.S, pl.R, pl.NP, pl.NP, dtype, &mA, &mB, &mC))) return r;
  for (int k = 0; k < 2 && !isf; ++k) {
    if ((r = make_operand_maps(A16[k], pl.R, 64, 64, APSP_I32, &pA[k], nullptr, nullptr))) return r;
    if ((r = make_operand_maps(B16[k], pl.G * 64, pl.NP, pl.NP, APSP_I32, nullptr, &pB[k], nullptr))) return r;
  }

  TileProblem p = {};
  p.C = a.S;
  p.ldc = pl.NP;
  p.inf_i = inf_i;
  p.inf_f = inf_f;
  p.status = status_word();
  p.wmax = isf ? nullptr : words + kWBound;  // (n - 1) * largest weight over every staged graph, then 0
  p.wmult = 1;
  p.bt = 1;
  p.ngroups = pl.ngroups;
  for (int k = 0; k < pl.ngroups; ++k) p.groups[k] = pl.groups[k];
  p.gflags = a.gflags;
  p.gsize = a.gsize;
  const int max_nb = pl.groups[0].nb;

  // Pass 1: graphs of the 16-bit pass.  Per block: the diagonal tile (exact), the packed
  // panels, phase 2 on them (truncated), the panels packed again, phase 3 (truncated).
  for (int kb = 0; kb < max_nb && !isf; ++kb) {
    int64_t open = 0, panels = 0, rest = 0;
    double panel_pairs = 0.0, rest_pairs = 0.0;  // (min,+) pairs by definition, k to each graph's size
    for (int k = 0; k < pl.ngroups; ++k) {
      const int64_t nb = pl.groups[k].nb, c = pl.groups[k].count;
      if (nb <= kb) continue;
      open += c;
      panels += c * 2 * (nb - 1);
      rest += c * (nb - 1) * (nb - 1);
      for (int64_t g = pl.groups[k].first; g < pl.groups[k].first + c; ++g) {
        const double bk = (double)std::min<int64_t>(kBM, pl.sizes[g] - (int64_t)kb * kBM);
        panel_pairs += 2.0 * (nb - 1) * kBM * kBM * bk;
        rest_pairs += (double)(nb - 1) * (nb - 1) * kBM * kBM * bk;
      }
    }
    // The packed panels of step kb (set kb & 1): the diagonal kernel writes its tile's part; the
    // rest came from step kb - 1 (its phase-2 and phase-3 tiles of block row / column kb),
    // except at kb = 0, where one packing pass writes them.
    const int cur = kb & 1;
    group_diag_kernel<<<(int)open, 256, 0, s>>>(a.S, pl.NP, a.gs, kb, a.gflags, a.gsize, kGfBad | kGfUse16, kGfUse16,
                                                nullptr, true, A16[cur], B16[cur], false);
    APSP_LAUNCH_CHECK();
    if (kb == 0) {
      group_pack16_kernel<<<dim3((unsigned)open, 4), 256, 0, s>>>(a.S, pl.NP, a.gs, kb, a.gflags, A16[0], B16[0]);
      APSP_LAUNCH_CHECK();
    }
    TileProblem q16 = p;
    q16.kb = kb;
    q16.gmask = kGfBad | kGfUse16;
    q16.gwant = kGfUse16;
    q16.arith16 = 1;
    q16.ntiles = panels;
    q16.trace_pairs = panel_pairs;
    q16.pk_a[0] = A16[0];  // the tiles leave their results packed: phase 3's operands and the
    q16.pk_a[1] = A16[1];  // next step's panels
    q16.pk_b[0] = B16[0];
    q16.pk_b[1] = B16[1];
    if ((r = launch_tgemm(kModeFwPanels, false, APSP_I32, pA[cur], pB[cur], mC, q16, s))) return r;
    q16.ntiles = rest;
    q16.trace_pairs = rest_pairs;
    if ((r = launch_tgemm(kModeFwRest16, true, APSP_I32, pA[cur], pB[cur], mC, q16, s))) return r;
  }
  if (!isf) {
    certify_out_kernel<<<row_grid, 256, 0, s>>>(a);
    APSP_LAUNCH_CHECK();
    group_verdict_kernel<<<g_grid, 256, 0, s>>>(a, pl.G);
    APSP_LAUNCH_CHECK();
  }

  // Pass 2: the 32-bit closure of the graphs that need it (int32: none, usually, and then
  // every launch returns at once; float32: every staged graph).
  p.no_trace = !isf;
  p.run_if = words + kWRerun;
  p.gmask = kGfBad | kGfRerun;
  p.gwant = kGfRerun;
  p.arith16 = 0;
  for (int kb = 0; kb < max_nb; ++kb) {
    int64_t open = 0, panels = 0, rest = 0;
    double rest_pairs = 0.0;
    for (int k = 0; k < pl.ngroups; ++k) {
      const int64_t nb = pl.groups[k].nb, c = pl.groups[k].count;
      if (nb <= kb) continue;
      open += c;
      panels += c * 2 * (nb - 1);
      rest += c * (nb - 1) * (nb - 1);
      for (int64_t g = pl.groups[k].first; g < pl.groups[k].first + c; ++g)
        rest_pairs += (double)(nb - 1) * (nb - 1) * kBM * kBM *
                      (double)std::min<int64_t>(kBM, pl.sizes[g] - (int64_t)kb * kBM);
    }
    group_diag_kernel<<<(int)open, 256, 0, s>>>(a.S, pl.NP, a.gs, kb, a.gflags, a.gsize, kGfBad | kGfRerun,
                                                kGfRerun, words + kWRerun, false, nullptr, nullptr, isf);
    APSP_LAUNCH_CHECK();
    p.kb = kb;
    p.ntiles = panels;
    p.trace_pairs = 0.0;
    if ((r = launch_tgemm(kModeFwPanels, false, dtype, mA, mB, mC, p, s))) return r;
    p.ntiles = rest;
    p.trace_pairs = rest_pairs;
    if ((r = launch_tgemm(kModeFwRest, true, dtype, mA, mB, mC, p, s))) return r;
  }
  stage_out_kernel<<<row_grid, 256, 0, s>>>(a);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

}  // namespace apsp
