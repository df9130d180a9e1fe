// batched.cu -- a7: close many independent graphs of uneven size in ONE persistent launch.
//
// The paper's experiment solves a thousand random graphs of 4..1000 vertices one by one
// (Sec. 3.4, Sec. 4).  Launched one at a time, small closures are dominated by launch latency
// and a medium graph's phase-3 grid covers only a fraction of the 152 SMs.  Here one CTA per
// SM pulls graphs from an atomic work queue (the caller orders it largest first, so the
// largest jobs start earliest -- longest-processing-time list scheduling) and closes each
// graph alone, with the same blocked Floyd-Warshall schedule as apsp_fw:
//   a1  normalise the graph in place and find its largest finite weight;
//   for each 128-vertex diagonal block kb:
//     phase 1  Eq. 1 on the diagonal tile, resident in shared memory;
//     phase 2  row/column panel tiles = (min,+) products with the closed tile;
//     phase 3  every other tile D[i][j] = min(D[i][j], D[i][kb] (x) D[kb][j]).
// Phases 2-3 run the register-tiled slab arithmetic of the GEMM engine (slab.cuh), fed by a
// four-stage cp.async pipeline that streams across tile boundaries (each graph has its own
// shape, so no per-graph TMA descriptors are needed).  int32 graphs whose (n - 1) * largest
// finite weight < 2^24 use the exact fp32 instruction sequence; others the int32 one.  One CTA
// per graph needs no inter-CTA synchronisation: there is no spin-wait anywhere in this kernel.
//
// apsp_batched (below) gives this kernel the whole batch, or -- for an int32 batch with the
// host sizes and the staging room in the workspace -- only the graphs of at most 256 vertices
// (and any above 2048), while the others are closed in lockstep on the GEMM engine
// (grouped.cu), where a graph's work is spread over every SM instead of one CTA.
#include <cooperative_groups.h>

#include <mutex>
#include <vector>

#include "diag.cuh"
#include "grouped.cuh"
#include "slab.cuh"
#include "tgemm.cuh"

namespace cg = cooperative_groups;

namespace apsp {

constexpr int kBThreads = 256;
constexpr int kBStages = 4;
constexpr int kBSlabInts = kSlabM * kSlabK;  // 4096 ints per A or B slab
constexpr int kBTileInts = kSlabM * kSlabN;  // 16384 ints per 128 x 128 tile
constexpr int kBSmemBytes = (2 * kBStages * kBSlabInts + kBTileInts + 512) * 4 + 256;

struct BatchArgs {
  int *pool;
  const int64_t *offsets;
  const int32_t *ns, *lds, *order;
  int64_t count;  // graphs in the arrays (valid indices are 0..count-1)
  int64_t nq;     // queue entries: order[0..nq) (or 0..nq-1 without order)
  int inf_i;
  float inf_f;
  int *queue;
  unsigned int *status;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename S> struct Store;
template <> struct Store<int> {
  static constexpr bool is_float = false;
  static __device__ __forceinline__ int fix(int v, const BatchArgs &a, bool &bad) {
    bad |= v < 0;
    return v >= a.inf_i ? a.inf_i : v;
  }
  static __device__ __forceinline__ int finite_max(int v, const BatchArgs &a, int m) { return v < a.inf_i ? max(m, v) : m; }
  static __device__ __forceinline__ int add(int x, int y) { return x + y; }
};
template <> struct Store<float> {
  static constexpr bool is_float = true;
  static __device__ __forceinline__ int fix(int bits, const BatchArgs &a, bool &bad) {
    const float v = __int_as_float(bits);
    bad |= !(v >= 0.0f);
    return v >= a.inf_f ? 0x7f800000 : bits;
  }
  static __device__ __forceinline__ int finite_max(int, const BatchArgs &, int m) { return m; }
  static __device__ __forceinline__ int add(int x, int y) {
    return __float_as_int(__fadd_rn(__int_as_float(x), __int_as_float(y)));
  }
};

// a1 for one graph, whole CTA: returns the largest finite weight (int32; 0 for float32).
// rank / csize: this CTA normalises rows rank, rank + csize, ... (in warp-sized strides).
template <typename S>
__device__ int normalise_graph(int *D, int n, int ld, const BatchArgs &a, int *red, int rank, int csize) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int W = kBThreads / 32;
  bool bad = false;
  int m = 0;
  for (int i = warp + W * rank; i < n; i += W * csize) {
    int *row = D + (int64_t)i * ld;
    for (int j = lane; j < n; j += 32) {
      const int v = (j == i) ? 0 : Store<S>::fix(row[j], a, bad);
      row[j] = v;
      m = Store<S>::finite_max(v, a, m);
    }
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if (lane == 0) red[warp] = m;
  if (__syncthreads_or(bad) && threadIdx.x == 0) flag_status(a.status, APSP_ERR_DOMAIN);
  int r = 0;
#pragma unroll
  for (int w = 0; w < kBThreads / 32; ++w) r = max(r, red[w]);
  __syncthreads();  // red[] is reused by the next graph
  return r;
}

// Phase 1: Eq. 1 on the bk x bk diagonal tile at (kb0, kb0), closed in registers (diag.cuh);
// int32 graphs relax in int32 (exact), float32 graphs in fp32.
template <typename S>
__device__ void close_diag(int *D, int n, int ld, int kb0, int *buf) {
  const int bk = min(kSlabM, n - kb0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (warp & 3) * 4 + (lane >> 3), tn = (warp >> 2) * 8 + (lane & 7);
  int *T = D + (int64_t)kb0 * ld + kb0;
  int r[8][8];
  load_tile_regs(r, T, ld, bk, tm, tn);
  close_tile_regs<Store<S>::is_float>(r, bk, tm, tn, buf);
  store_tile_regs(r, T, ld, bk, tm, tn);
  __syncthreads();
}

// Operand origins of tile t of an FW phase (phase 2: row panel tiles then column panel
// tiles; phase 3: every tile outside block row/column kb).  All tiles of a phase have K = bk.
struct PhaseTile {
  int ar, ac, br, bc, cr, cc;
};
__device__ __forceinline__ PhaseTile phase_tile(bool rest, int t, int nb, int kb) {
  const int kb0 = kb * kSlabM;
  PhaseTile p;
  if (!rest) {
    if (t < nb - 1) {  // row panel: D[kb][j] = D[kb][kb]* (x) D[kb][j]
      const int j = (t + (t >= kb)) * kSlabN;
      p = {kb0, kb0, kb0, j, kb0, j};
    } else {           // column panel: D[i][kb] = D[i][kb] (x) D[kb][kb]*
      int i = t - (nb - 1);
      i = (i + (i >= kb)) * kSlabM;
      p = {i, kb0, kb0, kb0, i, kb0};
    }
  } else {             // D[i][j] = min(D[i][j], D[i][kb] (x) D[kb][j])
    int i = t / (nb - 1), j = t - i * (nb - 1);
    i = (i + (i >= kb)) * kSlabM;
    j = (j + (j >= kb)) * kSlabN;
    p = {i, kb0, kb0, j, i, j};
  }
  return p;
}

// All tiles of one FW phase by the whole CTA, as one stream of 32-deep k-slabs: the cp.async
// pipeline runs across tile boundaries, so the next tile's first slabs are already in flight
// while a tile finishes.  Out-of-graph rows
// and columns are zero-filled and never stored; the ragged last slab is bounded by kc.
// For phase 3 a tile's old C block is copied into shared memory while its slabs are computed.
// In-place safety: a phase-2 tile is both output and operand, but it is written only after
// all its own slabs have been consumed, and no other tile of the phase reads it.
// f32: the exact fp32 instruction sequence, else the int32 one; the accumulators are fp32
// registers either way (for non-negative values, ordering their bits as int32 or as fp32 agrees,
// so the final min with the old C is the same operation for both).
// This CTA takes tiles t0, t0 + tstride, ... of the phase (a cluster splits a phase this way).
template <bool ACC>
__device__ void phase_tiles(int *D, int n, int ld, int kb, int nb, int ntiles, int t0, int tstride, int *sA, int *sB,
                            int *sC, bool f32, int init_bits) {
  typedef ArithF32 AR;
  typedef float T;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tm = (warp & 3) * 4 + (lane >> 3), tn = (warp >> 2) * 8 + (lane & 7);
  const int bk = min(kSlabM, n - kb * kSlabM);
  const int nk = (bk + kSlabK - 1) / kSlabK;
  const int mine = ntiles > t0 ? (ntiles - t0 + tstride - 1) / tstride : 0;
  const int total = mine * nk;
  auto load_slab = [&](int g) {
    const PhaseTile p = phase_tile(ACC, t0 + (g / nk) * tstride, nb, kb);
    const int kt = g % nk, st = g % kBStages;
    int *As = sA + st * kBSlabInts, *Bs = sB + st * kBSlabInts;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + kBThreads * u;
      const int r = e >> 3, kq = e & 7;
      const int row = p.ar + r, col = p.ac + kt * kSlabK + 4 * kq;
      const bool ok = row < n && col < n;
      cp_async16(As + a_off(r, kq), ok ? D + (int64_t)row * ld + col : D, ok);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + kBThreads * u;
      const int r = e >> 5, c4 = e & 31;
      const int row = p.br + kt * kSlabK + r, col = p.bc + 4 * c4;
      const bool ok = row < n && col < n;
      cp_async16(Bs + r * kSlabN + 4 * c4, ok ? D + (int64_t)row * ld + col : D, ok);
    }
  };
#pragma unroll
  for (int s = 0; s < kBStages - 1; ++s) {
    if (s < total) load_slab(s);
    cp_async_commit();
  }
  T acc[8][8];
  const T init = AR::from(init_bits);
  for (int g = 0; g < total; ++g) {
    const int lt = g / nk, kt = g - lt * nk;
    const PhaseTile p = phase_tile(ACC, t0 + lt * tstride, nb, kb);
    const int m_valid = min(kSlabM, n - p.cr), n_valid = min(kSlabN, n - p.cc);
    if (kt == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = init;
    }
    cp_async_wait<kBStages - 2>();
    __syncthreads();
    if (ACC && kt == 0) {  // this tile's old C, in flight during its slabs
#pragma unroll 4
      for (int u = 0; u < 16; ++u) {
        const int e = tid + kBThreads * u;
        const int r = e >> 5, c4 = e & 31;
        const bool ok = r < m_valid && 4 * c4 < n_valid;
        cp_async16(sC + r * kSlabN + 4 * c4, ok ? D + (int64_t)(p.cr + r) * ld + p.cc + 4 * c4 : D, ok);
      }
    }
    if (g + kBStages - 1 < total) load_slab(g + kBStages - 1);
    cp_async_commit();
    const int st = g % kBStages;
    const int kc = bk - kt * kSlabK;
    const int *As = sA + st * kBSlabInts, *Bs = sB + st * kBSlabInts;
    if (f32) {
      if (kc >= kSlabK) ArithF32::slab_full(As, Bs, tm, tn, acc);
      else ArithF32::slab_part(As, Bs, tm, tn, kc, acc);
    } else {
      if (kc >= kSlabK) ArithI32::slab_full(As, Bs, tm, tn, acc);
      else ArithI32::slab_part(As, Bs, tm, tn, kc, acc);
    }
    if (kt != nk - 1) continue;
    if (ACC) {  // the slabs issued since are a slab's compute old: waiting for them costs little
      cp_async_wait<0>();
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int rl = tm + 16 * i;
      if (rl >= m_valid) continue;
      int *crow = D + (int64_t)(p.cr + rl) * ld + p.cc;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cl = 4 * tn + 64 * h;
        if (ACC) {
          const int4 v = *reinterpret_cast<const int4 *>(sC + rl * kSlabN + cl);
          acc[i][4 * h + 0] = AR::mn(acc[i][4 * h + 0], AR::from(v.x));
          acc[i][4 * h + 1] = AR::mn(acc[i][4 * h + 1], AR::from(v.y));
          acc[i][4 * h + 2] = AR::mn(acc[i][4 * h + 2], AR::from(v.z));
          acc[i][4 * h + 3] = AR::mn(acc[i][4 * h + 3], AR::from(v.w));
        }
        if (cl + 3 < n_valid) {
          *reinterpret_cast<int4 *>(crow + cl) = make_int4(AR::to(acc[i][4 * h]), AR::to(acc[i][4 * h + 1]),
                                                           AR::to(acc[i][4 * h + 2]), AR::to(acc[i][4 * h + 3]));
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (cl + q < n_valid) crow[cl + q] = AR::to(acc[i][4 * h + q]);
        }
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();  // shared buffers are reused by the next phase
}

// Orders every global-memory write of the group before every later read by the group: a CTA
// barrier for a lone CTA, the hardware cluster barrier (release / acquire) for a cluster.
__device__ __forceinline__ void group_sync(int csize) {
  __threadfence();
  if (csize > 1) cg::this_cluster().sync();
  else __syncthreads();
}

// Blocked Floyd-Warshall of one normalised graph by a group of csize CTAs (this one has
// rank `rank`): rank 0 closes each diagonal tile, the panel and remaining tiles are shared
// round-robin, and a group barrier separates the phases.
template <typename S>
__device__ void close_blocked(int *D, int n, int ld, bool f32, int init_bits, int *sA, int *sB, int *sC, int *sT,
                              int rank, int csize) {
  const int nb = (n + kSlabM - 1) / kSlabM;
  for (int kb = 0; kb < nb; ++kb) {
    if (rank == 0) close_diag<S>(D, n, ld, kb * kSlabM, sT);
    if (nb == 1) break;
    group_sync(csize);
    phase_tiles<false>(D, n, ld, kb, nb, 2 * (nb - 1), rank, csize, sA, sB, sC, f32, init_bits);
    group_sync(csize);
    phase_tiles<true>(D, n, ld, kb, nb, (nb - 1) * (nb - 1), rank, csize, sA, sB, sC, f32, init_bits);
    group_sync(csize);
  }
}

// Checks graph g's descriptor; on failure flags APSP_ERR_ARG (rank 0) and returns null.
__device__ __forceinline__ int *graph_base(const BatchArgs &a, int g, int &n, int &ld, bool flag) {
  n = a.ns[g];
  ld = a.lds[g];
  const int64_t off = a.offsets[g];
  if (n <= 0) return nullptr;
  if (ld < n || (ld & 3) || (off & 3) || off < 0) {
    if (flag && threadIdx.x == 0) flag_status(a.status, APSP_ERR_ARG);
    return nullptr;
  }
  return a.pool + off;
}

// The persistent kernel runs as clusters of csize CTAs (csize = 1 without clusters), in two
// stages.  Stage 1: the leading run of the queue order whose graphs are each too large for
// one CTA to close within the batch's average time per CTA (the order is largest first) is
// closed one graph at a time by whole clusters: rank 0 takes the next
// entry and writes it into every CTA's shared memory through distributed shared memory, and
// hardware cluster barriers separate the steps.  Stage 2: every CTA pulls the remaining
// graphs from its own counter and closes each alone, with no cluster barrier at all.  No CTA
// ever spins.
template <typename S>
__global__ void __launch_bounds__(kBThreads, 1) batched_kernel(const BatchArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  int *sA = reinterpret_cast<int *>(smem);
  int *sB = sA + kBStages * kBSlabInts;
  int *sC = sB + kBStages * kBSlabInts;  // a phase-3 tile's old C block
  int *sT = sC + kBTileInts;             // phase-1 row/column exchange buffer
  __shared__ int s_idx;   // stage 1: written by the cluster's rank 0 through DSMEM
  __shared__ int s_nbig;
  __shared__ int s_wmax;
  __shared__ int red[kBThreads / 32];
  cg::cluster_group cl = cg::this_cluster();
  const int csize = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int init_bits = Store<S>::is_float ? 0x7f800000 : a.inf_i;

  // Length of the cooperative prefix (the same for every CTA): the leading entries whose
  // graph alone would take more than half of the average work per CTA (n^3 > W / (2 CTAs),
  // W = sum of n^3) and has enough tiles for a cluster (n > 64 csize).  A batch whose graphs
  // are all small next to the whole keeps every graph on one CTA.  The cluster barrier after
  // it keeps rank 0's first remote write out of any CTA's shared memory until that CTA is ready.
  int nbig = 0;
  if (csize > 1) {
    __shared__ double s_work[kBThreads / 32];
    double w = 0.0;
    for (int k = threadIdx.x; k < a.nq; k += kBThreads) {
      const int g = a.order ? a.order[k] : k;
      if (g >= 0 && g < a.count) {
        const double n = (double)max(a.ns[g], 0);
        w += n * n * n;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) s_work[threadIdx.x >> 5] = w;
    if (threadIdx.x == 0) s_nbig = (int)a.nq;
    __syncthreads();
    double total = 0.0;
#pragma unroll
    for (int i = 0; i < kBThreads / 32; ++i) total += s_work[i];
    const double big3 = fmax(0.5 * total / (double)gridDim.x, (double)(64 * csize) * (64 * csize) * (64 * csize));
    int first_small = (int)a.nq;
    for (int k = threadIdx.x; k < a.nq; k += kBThreads) {
      const int g = a.order ? a.order[k] : k;
      const double n = (g >= 0 && g < a.count) ? (double)a.ns[g] : 0.0;
      if (!(n * n * n > big3)) {
        first_small = k;
        break;
      }
    }
    atomicMin(&s_nbig, first_small);
    __syncthreads();
    nbig = s_nbig;
    cl.sync();
  }

  // Stage 1: large graphs, one per cluster at a time.
  while (nbig > 0) {
    if (rank == 0 && threadIdx.x == 0) {
      const int idx = atomicAdd(&a.queue[0], 1);
      s_wmax = 0;
      for (int q = 0; q < csize; ++q) *cl.map_shared_rank(&s_idx, q) = idx;
    }
    cl.sync();
    const int idx = s_idx;
    if (idx >= nbig) break;  // every CTA of the cluster read the same value
    const int g = a.order ? a.order[idx] : idx;
    int n = 0, ld = 0;
    int *D = graph_base(a, g, n, ld, rank == 0);
    if (D) {
      const int w = normalise_graph<S>(D, n, ld, a, red, rank, csize);
      if (threadIdx.x == 0) atomicMax(cl.map_shared_rank(&s_wmax, 0), w);
      group_sync(csize);
      const int wmax = *cl.map_shared_rank(&s_wmax, 0);
      const bool f32 = Store<S>::is_float || small_int_bound(wmax, n - 1, 0);
      close_blocked<S>(D, n, ld, f32, init_bits, sA, sB, sC, sT, rank, csize);
    }
    group_sync(csize);  // the whole cluster is done before rank 0 writes the next index
  }

  // Stage 2: every other graph, one per CTA.
  for (;;) {
    if (threadIdx.x == 0) s_idx = nbig + atomicAdd(&a.queue[1], 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= a.nq) break;
    const int g = a.order ? a.order[idx] : idx;
    if (g < 0 || g >= a.count) {
      if (threadIdx.x == 0) flag_status(a.status, APSP_ERR_ARG);
      continue;
    }
    int n = 0, ld = 0;
    int *D = graph_base(a, g, n, ld, true);
    if (!D) continue;
    const int wmax = normalise_graph<S>(D, n, ld, a, red, 0, 1);
    group_sync(1);
    const bool f32 = Store<S>::is_float || small_int_bound(wmax, n - 1, 0);
    close_blocked<S>(D, n, ld, f32, init_bits, sA, sB, sC, sT, 0, 1);
    group_sync(1);
  }
}

// Launch shape of the persistent kernel: the largest cluster size (8, 4, 2) whose co-resident
// clusters still cover at least 7/8 of the SMs, with that many clusters; else plain CTAs.
struct BatchShape {
  int csize = 1, clusters = 0;
};

template <typename S>
static BatchShape batch_shape() {
  static BatchShape cache[64];
  static bool have[64] = {false};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(mu);
    if (have[dev]) return cache[dev];
  }
  BatchShape best;
  best.clusters = sm_count();
  for (int c : {8, 4, 2}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c * 16);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = kBSmemBytes;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = c;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, batched_kernel<S>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (num * c * 8 >= sm_count() * 7) {
      best.csize = c;
      best.clusters = num;
      break;
    }
  }
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(mu);
    cache[dev] = best;
    have[dev] = true;
  }
  return best;
}

// Clusters pay off only when some graph would, alone on one CTA, take longer than the average
// work per SM (then largest-first list scheduling cannot hide it); otherwise every graph stays
// on one CTA and all SMs take part.
static bool needs_clusters(const int32_t *ns_host, int64_t count) {
  if (!ns_host) return true;
  double w = 0.0, mx = 0.0;
  for (int64_t g = 0; g < count; ++g) {
    const double n = (double)(ns_host[g] > 0 ? ns_host[g] : 0);
    w += n * n * n;
    mx = n > mx ? n : mx;
  }
  return mx > kSlabM && mx * mx * mx > w / (double)sm_count();
}

template <typename S>
static int launch_batched(const BatchArgs &a, bool clusters, cudaStream_t s) {
  if (cudaFuncSetAttribute(batched_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBSmemBytes) != cudaSuccess)
    return APSP_ERR_CUDA;
  BatchShape sh;
  sh.clusters = sm_count();
  if (clusters) sh = batch_shape<S>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sh.csize * sh.clusters);
  cfg.blockDim = dim3(kBThreads);
  cfg.dynamicSmemBytes = kBSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = sh.csize;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  note_launch();
  if (cudaLaunchKernelEx(&cfg, batched_kernel<S>, a) != cudaSuccess) {
    cudaGetLastError();
    return APSP_ERR_CUDA;
  }
  return APSP_OK;
}

}  // namespace apsp

namespace {

struct RestCtx {
  apsp::BatchArgs a;
  bool clusters;
  cudaStream_t s;
  bool is_float;
};

// The persistent kernel over a sub-list of the batch (the graphs the staged path leaves out).
int launch_rest_graphs(void *ctx, const int *order, int64_t nq) {
  RestCtx *c = reinterpret_cast<RestCtx *>(ctx);
  apsp::BatchArgs a = c->a;
  a.order = order;
  a.nq = nq;
  return c->is_float ? apsp::launch_batched<float>(a, c->clusters, c->s) : apsp::launch_batched<int>(a, c->clusters, c->s);
}

}  // namespace

extern "C" size_t apsp_batched_workspace_bytes(int64_t count) {
  (void)count;
  return 256;
}

extern "C" size_t apsp_batched_staged_workspace_bytes(const int32_t *ns_host, int64_t count, int dtype) {
  apsp::StagePlan pl;
  if (!apsp::dtype_ok(dtype) || !apsp::make_stage_plan(ns_host, count, pl)) return 256;
  return apsp::staged_workspace_bytes(pl, count, dtype);
}

extern "C" int apsp_batched(void *pool, const int64_t *offsets, const int32_t *ns, const int32_t *lds,
                            const int32_t *order, const int32_t *ns_host, int64_t count, int dtype, const void *inf,
                            void *ws, size_t ws_bytes, void *stream) {
  using namespace apsp;
  if (!dtype_ok(dtype) || count < 0 || count > INT32_MAX) return APSP_ERR_ARG;
  if (count == 0) return APSP_OK;
  if (!pool || !offsets || !ns || !lds || reinterpret_cast<uintptr_t>(pool) % 16 != 0) return APSP_ERR_ARG;
  if (ws && (ws_bytes < 256 || reinterpret_cast<uintptr_t>(ws) % 256 != 0)) return APSP_ERR_ARG;
  BatchArgs a = {};
  if (dtype == APSP_I32 ? resolve_inf_i32(inf, &a.inf_i) : resolve_inf_f32(inf, &a.inf_f)) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void *own = nullptr;
  if (!ws) {
    if (ws_alloc(&own, 256, s) != APSP_OK) {
      return APSP_ERR_NOMEM;
    }
    ws = own;
  }
  a.pool = reinterpret_cast<int *>(pool);
  a.offsets = offsets;
  a.ns = ns;
  a.lds = lds;
  a.order = order;
  a.count = count;
  a.nq = count;
  a.queue = reinterpret_cast<int *>(ws);
  a.status = status_word();
  int r = APSP_OK;
  if (cudaMemsetAsync(a.queue, 0, 2 * sizeof(int), s) != cudaSuccess) r = APSP_ERR_CUDA;
  // Graphs of 257..2048 vertices go through the engine in lockstep when the workspace has room
  // for the staging (int32 with a sentinel above the 16-bit cap, or float32).
  StagePlan pl;
  if (!r && !own && (dtype == APSP_F32 || a.inf_i > kCap16) && make_stage_plan(ns_host, count, pl) &&
      ws_bytes >= staged_workspace_bytes(pl, count, dtype)) {
    std::vector<int32_t> rest_ns;
    rest_ns.reserve(pl.rest.size());
    for (int g : pl.rest) rest_ns.push_back(ns_host[g]);
    RestCtx ctx = {a, needs_clusters(rest_ns.data(), (int64_t)rest_ns.size()), s, dtype == APSP_F32};
    r = batched_staged(pl, a.pool, offsets, ns, lds, count, dtype, a.inf_i, a.inf_f, ws, launch_rest_graphs, &ctx, s);
    return r;
  }
  const bool clusters = needs_clusters(ns_host, count);
  if (!r) r = dtype == APSP_I32 ? launch_batched<int>(a, clusters, s) : launch_batched<float>(a, clusters, s);
  ws_free(own, s);
  return r;
}
