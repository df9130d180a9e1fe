// pred.cu -- predecessor matrix of a closed distance matrix (pred[i, j] of Sec. 2; the argmin
// of Sec. 3.1 that yields the predecessors alongside the min).
//
// pred[i][j] is the vertex just before j on a shortest i -> j path: the smallest k != j that
// minimises d[i][k] + w[k][j], where d is the closed distance matrix and w the original cost
// matrix.  It is -1 on the diagonal and where j is unreachable from i.  With positive
// off-diagonal weights (the assumption of Sec. 3.1) d[i][pred[i][j]] < d[i][j], so following
// pred back from j reaches i within n - 1 steps: the path reconstruction of Sec. 2.
//
// The argmin is itself a (min,+) product over a totally ordered encoding.  With s bits per
// vertex index (2^s >= n):
//     De[i][k] = d[i][k] << s,   We[k][j] = (w[k][j] << s) | k,   We[j][j] = INF
//     min_k (De[i][k] + We[k][j]) = (min_k (d[i][k] + w[k][j]) << s) | smallest argmin k
// so the TMA tropical-GEMM engine computes it at its full (min,+) rate -- on its exact fp32
// path when the encoded sums stay below 2^24.  The encoding is exact for int32 matrices with
// ((max finite d + max finite w) << s) + 2^s - 1 < 0x3FFFFFFF.  The device checks that bound
// after scanning both matrices; when it fails the engine launch returns at once and a direct
// argmin kernel (add, compare, two selects per (i, j, k)) computes pred instead.  float32
// matrices always take the direct kernel: their sums round, so they cannot carry an index in
// their low bits.
#include "closure.cuh"

namespace apsp {

namespace {

constexpr int kInfE = 0x3FFFFFFF;  // sentinel of the encoded operands
// Bound words at the front of the workspace.
enum { kWMaxD = 0, kWMaxW = 1, kWBoundA = 2, kWBoundB = 3, kWSkip = 4 };

__host__ __device__ inline int index_bits(int64_t n) {
  int s = 1;
  while ((int64_t(1) << s) < n) ++s;
  return s;
}

// De and We from d and w; or, when the encoded sums could reach the sentinel, only the skip
// word (every thread evaluates the same bound, so the whole grid takes the same branch).
__global__ void __launch_bounds__(256) pred_encode_kernel(const int *d, int64_t ldd, const int *w, int64_t ldw,
                                                          int *De, int *We, int64_t lde, int64_t n, int s, int inf,
                                                          int *words, unsigned int *st) {
  const int64_t md = words[kWMaxD], mw = words[kWMaxW];
  const int64_t top = ((md + mw) << s) + ((int64_t(1) << s) - 1);
  if (top >= kInfE) {
    if (blockIdx.x == 0 && threadIdx.x == 0) words[kWSkip] = 1;
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    words[kWBoundA] = (int)(md << s);
    words[kWBoundB] = (int)((mw << s) + (n - 1));
  }
  bool bad = false;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const int *dr = d + i * ldd, *wr = w + i * ldw;
    int *der = De + i * lde, *wer = We + i * lde;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const int dv = dr[j], wv = wr[j];
      bad |= dv < 0 || wv < 0;
      der[j] = (dv < 0 || dv >= inf) ? kInfE : (dv << s);
      wer[j] = (wv < 0 || wv >= inf || j == i) ? kInfE : ((wv << s) | (int)i);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) flag_status(st, APSP_ERR_DOMAIN);
}

// Engine output (min value << s | k) -> k, or -1 on the diagonal and for unreachable pairs
// (a minimum >= inf is unreachable, as in the closure, where such sums saturate to inf).
__global__ void __launch_bounds__(256) pred_decode_kernel(int *pred, int64_t ldp, int64_t n, int s, int inf,
                                                          const int *words) {
  if (words[kWSkip]) return;
  const int mask = (1 << s) - 1;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    int *row = pred + i * ldp;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const int c = row[j];
      row[j] = (j == i || c >= kInfE || (c >> s) >= inf) ? -1 : (c & mask);
    }
  }
}

template <typename T> struct PredOps;
template <> struct PredOps<int> {
  static __device__ __forceinline__ int big() { return kInfE; }
  static __device__ __forceinline__ int fix(int v, int inf, bool &bad) {
    bad |= v < 0;
    return (v < 0 || v >= inf) ? inf : v;
  }
  static __device__ __forceinline__ bool finite(int v, int inf) { return v < inf; }
  static __device__ __forceinline__ int add(int a, int b) { return a + b; }  // both <= inf <= 2^30 - 1
};
template <> struct PredOps<float> {
  static __device__ __forceinline__ float big() { return __int_as_float(0x7f800000); }
  static __device__ __forceinline__ float fix(float v, float inf, bool &bad) {
    bad |= !(v >= 0.0f);
    return (!(v >= 0.0f) || v >= inf) ? __int_as_float(0x7f800000) : v;
  }
  static __device__ __forceinline__ bool finite(float v, float) { return v < __int_as_float(0x7f800000); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
};

// Direct argmin: 128 x 128 output tile per CTA, 256 threads with 8 x 8 entries each (rows
// ty + 16 r, columns tx + 16 c), 32-deep k-slabs of d and w staged in shared memory with
// plain coalesced loads.  k ascends within each thread and only a strictly smaller sum
// replaces the best, so the smallest argmin k wins -- the same choice as the encoded product.
// run_if: device word; the kernel returns at once unless it is non-zero (nullptr: always run).
template <typename T>
__global__ void __launch_bounds__(256) pred_direct_kernel(const T *d, int64_t ldd, const T *w, int64_t ldw, int *pred,
                                                          int64_t ldp, int64_t n, T inf, const int *run_if,
                                                          unsigned int *st) {
  if (run_if && *run_if == 0) return;
  typedef PredOps<T> O;
  __shared__ T As[128][33];
  __shared__ T Bs[32][128];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t i0 = (int64_t)blockIdx.y * 128, j0 = (int64_t)blockIdx.x * 128;
  T best[8][8];
  int arg[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      best[r][c] = O::big();
      arg[r][c] = -1;
    }
  const T big = O::big();
  bool bad = false;
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
#pragma unroll
    for (int t = 0; t < 16; ++t) {  // A slab: 128 rows x 32 k, one 32-wide row segment per warp
      const int r = (tid >> 5) + 8 * t, c = tid & 31;
      const int64_t i = i0 + r, k = k0 + c;
      As[r][c] = (i < n && k < n) ? O::fix(d[i * ldd + k], inf, bad) : big;
    }
#pragma unroll
    for (int t = 0; t < 16; ++t) {  // B slab: 32 k x 128 columns; w[j][j] is never a last hop
      const int r = (tid >> 7) + 2 * t, c = tid & 127;
      const int64_t k = k0 + r, j = j0 + c;
      Bs[r][c] = (k < n && j < n && k != j) ? O::fix(w[k * ldw + j], inf, bad) : big;
    }
    __syncthreads();
    const int kc = (int)(n - k0 < 32 ? n - k0 : 32);
    for (int kk = 0; kk < kc; ++kk) {
      T a[8], b[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] = As[ty + 16 * r][kk];
#pragma unroll
      for (int c = 0; c < 8; ++c) b[c] = Bs[kk][tx + 16 * c];
      const int k = (int)(k0 + kk);
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const T v = O::add(a[r], b[c]);
          const bool lt = v < best[r][c];
          best[r][c] = lt ? v : best[r][c];
          arg[r][c] = lt ? k : arg[r][c];
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t i = i0 + ty + 16 * r;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t j = j0 + tx + 16 * c;
      if (j < n) pred[i * ldp + j] = (i == j || !O::finite(best[r][c], inf)) ? -1 : arg[r][c];
    }
  }
  if (__syncthreads_or(bad) && tid == 0) flag_status(st, APSP_ERR_DOMAIN);
}

template <typename T>
int launch_direct(const void *d, int64_t ldd, const void *w, int64_t ldw, int *pred, int64_t ldp, int64_t n, T inf,
                  const int *run_if, cudaStream_t s) {
  const int64_t t = cdiv(n, 128);
  if (t > 65535) return APSP_ERR_ARG;
  pred_direct_kernel<T><<<dim3((unsigned)t, (unsigned)t), 256, 0, s>>>(
      reinterpret_cast<const T *>(d), ldd, reinterpret_cast<const T *>(w), ldw, pred, ldp, n, inf, run_if,
      status_word());
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

// float32 argmin with the (min,+) instruction mix of the GEMM engine.  The hot loop never
// tracks k itself: it keeps each entry's running minimum and the index of the 4-deep k-quad
// in which that minimum last fell, which costs one compare and one select per quad:
//     {s0, s1} = {d[i][k], d[i][k+1]} + {w[k][j], w[k+1][j]}   (add.rn.f32x2), {s2, s3} alike
//     m = min(min(best, s0, s1), s2, s3);  if (m < best) quad = k / 4;  best = m
// The epilogue re-forms the four sums of the recorded quad with the same round-to-nearest adds
// and takes the first k whose sum equals the minimum.  Because the quad only moves on a
// strictly smaller minimum, no earlier quad reaches that value, so this k is the smallest
// argmin -- the same index as the direct kernel's.  d is staged as [i][k] and w transposed as
// [j][k] in shared memory, so both pairs of each packed add come from 128-bit loads.
__global__ void __launch_bounds__(256) pred_direct_f32_kernel(const float *d, int64_t ldd, const float *w,
                                                              int64_t ldw, int *pred, int64_t ldp, int64_t n,
                                                              float inf, unsigned int *st) {
  typedef PredOps<float> O;
  constexpr int kP = 36;  // padded row (floats): 16-byte aligned rows, spread banks
  __shared__ __align__(16) float As[128 * kP];
  __shared__ __align__(16) float Bt[128 * kP];
  const int tid = threadIdx.x, tm = tid >> 4, tn = tid & 15;
  const int64_t i0 = (int64_t)blockIdx.y * 128, j0 = (int64_t)blockIdx.x * 128;
  float best[8][8];
  int quad[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      best[r][c] = O::big();
      quad[r][c] = 0;
    }
  const float big = O::big();
  bool bad = false;
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int r = (tid >> 5) + 8 * t, c = tid & 31;
      const int64_t i = i0 + r, k = k0 + c;
      As[r * kP + c] = (i < n && k < n) ? O::fix(d[i * ldd + k], inf, bad) : big;
    }
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int r = (tid >> 7) + 2 * t, c = tid & 127;
      const int64_t k = k0 + r, j = j0 + c;
      Bt[c * kP + r] = (k < n && j < n && k != j) ? O::fix(w[k * ldw + j], inf, bad) : big;
    }
    __syncthreads();
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      uint64_t a[8][2];
#pragma unroll
      for (int r = 0; r < 8; ++r) lds128_2x64(As + (tm + 16 * r) * kP + 4 * q, a[r][0], a[r][1]);
      const int qi = (int)(k0 >> 2) + q;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint64_t b0, b1;
        lds128_2x64(Bt + (tn + 16 * c) * kP + 4 * q, b0, b1);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const uint64_t p01 = fadd2_64(a[r][0], b0), p23 = fadd2_64(a[r][1], b1);
          const float m = Ops<float>::min3(Ops<float>::min3(best[r][c], lo_of(p01), hi_of(p01)), lo_of(p23),
                                           hi_of(p23));
          quad[r][c] = m < best[r][c] ? qi : quad[r][c];
          best[r][c] = m;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t i = i0 + tm + 16 * r;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t j = j0 + tn + 16 * c;
      if (j >= n) continue;
      int out = -1;
      if (i != j && O::finite(best[r][c], inf)) {
        for (int t = 3; t >= 0; --t) {  // descending, so the first k in order is kept last
          const int64_t k = 4 * (int64_t)quad[r][c] + t;
          if (k >= n || k == j) continue;
          const float v = __fadd_rn(O::fix(d[i * ldd + k], inf, bad), O::fix(w[k * ldw + j], inf, bad));
          if (v == best[r][c]) out = (int)k;
        }
      }
      pred[i * ldp + j] = out;
    }
  }
  if (__syncthreads_or(bad) && tid == 0) flag_status(st, APSP_ERR_DOMAIN);
}

int launch_direct_f32(const void *d, int64_t ldd, const void *w, int64_t ldw, int *pred, int64_t ldp, int64_t n,
                      float inf, cudaStream_t s) {
  const int64_t t = cdiv(n, 128);
  if (t > 65535) return APSP_ERR_ARG;
  pred_direct_f32_kernel<<<dim3((unsigned)t, (unsigned)t), 256, 0, s>>>(
      reinterpret_cast<const float *>(d), ldd, reinterpret_cast<const float *>(w), ldw, pred, ldp, n, inf,
      status_word());
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

int64_t enc_ld(int64_t n) { return round_up(n, 4); }
size_t enc_bytes(int64_t n) { return (size_t)round_up(n * enc_ld(n) * 4, 256); }

}  // namespace

}  // namespace apsp

extern "C" size_t apsp_predecessors_workspace_bytes(int64_t n, int dtype) {
  using namespace apsp;
  if (n <= 0 || dtype != APSP_I32) return kFlagBytes;
  return kFlagBytes + 2 * enc_bytes(n);
}

extern "C" int apsp_predecessors(const void *d, int64_t ldd, const void *w, int64_t ldw, int32_t *pred, int64_t ldp,
                                 int64_t n, int dtype, const void *inf, void *ws, size_t ws_bytes, void *stream) {
  using namespace apsp;
  if (!dtype_ok(dtype) || n < 0) return APSP_ERR_ARG;
  if (n == 0) return APSP_OK;
  if (!d || !w || !pred || ldd < n || ldw < n || ldp < n || n > INT32_MAX) return APSP_ERR_ARG;
  if (ws && reinterpret_cast<uintptr_t>(ws) % 256 != 0) return APSP_ERR_ARG;
  int inf_i = 0;
  float inf_f = 0.f;
  if (dtype == APSP_I32 ? resolve_inf_i32(inf, &inf_i) : resolve_inf_f32(inf, &inf_f)) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == APSP_F32) return launch_direct_f32(d, ldd, w, ldw, pred, ldp, n, inf_f, s);

  // int32: encoded product when pred can be the engine's output, else the direct kernel.
  const bool engine_ok = reinterpret_cast<uintptr_t>(pred) % 16 == 0 && ldp % 4 == 0;
  if (!engine_ok) return launch_direct<int>(d, ldd, w, ldw, pred, ldp, n, inf_i, nullptr, s);
  const size_t need = apsp_predecessors_workspace_bytes(n, dtype);
  if (ws && ws_bytes < need) return APSP_ERR_ARG;
  void *own = nullptr;
  if (!ws) {
    if (ws_alloc(&own, need, s) != APSP_OK) {
      return APSP_ERR_NOMEM;
    }
    ws = own;
  }
  uint8_t *base = reinterpret_cast<uint8_t *>(ws);
  int *words = reinterpret_cast<int *>(base);
  int *De = reinterpret_cast<int *>(base + kFlagBytes);
  int *We = reinterpret_cast<int *>(base + kFlagBytes + enc_bytes(n));
  const int64_t lde = enc_ld(n);
  const int sb = index_bits(n);
  int r = APSP_OK;
  if (cudaMemsetAsync(words, 0, 32, s) != cudaSuccess) r = APSP_ERR_CUDA;
  if (!r) r = launch_scan_max(d, n, n, ldd, inf_i, words + kWMaxD, s);
  if (!r) r = launch_scan_max(w, n, n, ldw, inf_i, words + kWMaxW, s);
  if (!r) {
    const int64_t cap = (int64_t)sm_count() * 8;
    pred_encode_kernel<<<(int)(n < cap ? n : cap), 256, 0, s>>>(reinterpret_cast<const int *>(d), ldd,
                                                                reinterpret_cast<const int *>(w), ldw, De, We, lde, n,
                                                                sb, inf_i, words, status_word());
    note_launch();
    if (cudaGetLastError() != cudaSuccess) r = APSP_ERR_CUDA;
  }
  if (!r) {
    CUtensorMap mA, mB, mC;
    if (!(r = make_operand_maps(De, n, n, lde, APSP_I32, &mA, nullptr, nullptr)) &&
        !(r = make_operand_maps(We, n, n, lde, APSP_I32, nullptr, &mB, nullptr)) &&
        !(r = make_operand_maps(pred, n, n, ldp, APSP_I32, nullptr, nullptr, &mC))) {
      TileProblem p = {};
      p.M = n; p.N = n; p.K = n;
      p.tiles_m = cdiv(n, kBM);
      p.tiles_n = cdiv(n, kBN);
      p.ntiles = p.tiles_m * p.tiles_n;
      p.C = pred;
      p.ldc = ldp;
      p.inf_i = kInfE;
      p.status = status_word();
      p.wmax = words + kWBoundA;  // exact fp32 path when boundA + boundB < 2^24
      p.wmult = 1;
      p.skip = words + kWSkip;
      r = launch_tgemm(kModeGemm, false, APSP_I32, mA, mB, mC, p, s);
    }
  }
  if (!r) {
    const int64_t cap = (int64_t)sm_count() * 8;
    pred_decode_kernel<<<(int)(n < cap ? n : cap), 256, 0, s>>>(pred, ldp, n, sb, inf_i, words);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) r = APSP_ERR_CUDA;
  }
  if (!r) r = launch_direct<int>(d, ldd, w, ldw, pred, ldp, n, inf_i, words + kWSkip, s);
  ws_free(own, s);
  return r;
}
