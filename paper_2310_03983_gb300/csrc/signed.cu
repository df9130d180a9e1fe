// signed.cu -- blocked Floyd-Warshall for matrices with negative edges (Sec. 3.1 assumes only
// that no cycle is negative), with negative-cycle detection.
//
// The closure itself is the same three-phase loop as apsp_fw; what changes is the handling of
// "unreachable".  With non-negative weights an unreachable entry (the sentinel) plus anything
// stays at or above the sentinel, and min() saturates for free.  With negative weights the
// sentinel plus a negative entry drops below it.  Here the finite range is bounded instead:
// every finite distance is the length of a simple path, so |d| <= (n - 1) * max|w| < 2^27
// (checked on the device after a1).  A value derived from the sentinel then stays at or above
// inf - 2^28 >= 2^29, while every finite value stays below 2^28; each kernel that writes the
// matrix (the diagonal closure after every step, the engine's epilogue) maps values at or above
// 2^29 back to exactly inf.  int32 arithmetic only (the exact fp32 path reads the bit patterns of
// non-negative integers); float32 needs none of this, since +inf absorbs negative terms.
//
// A negative cycle shows up on the diagonal: when the block holding the cycle's largest vertex
// v is closed, d[v][v] < 0 is published as part of row v.  The diagonal closure then stops, sets
// APSP_ERR_NEGATIVE_CYCLE and a device word that makes every later launch return at once, so no
// value can run away around the cycle.
#include <algorithm>
#include <climits>

#include "closure.cuh"
#include "diag.cuh"

namespace apsp {

namespace {

constexpr int kSignedThr = 1 << 29;          // values at or above it are unreachable
constexpr int kSignedMinInf = 0x30000000;    // smallest sentinel: inf - 2^28 >= 2^29
constexpr int64_t kSignedRange = 1LL << 27;  // (n - 1) * max|w| must stay below it
// Words of the bound block: [0] largest |finite entry|, [7] stop (negative cycle or range).
constexpr int kStop = 7;

template <typename T> struct SNorm;
template <> struct SNorm<int> {
  static __device__ __forceinline__ int fix(int v, int inf, bool &, int &m) {
    if (v >= inf) return inf;
    const int a = v < 0 ? (v == INT_MIN ? INT_MAX : -v) : v;
    m = max(m, a);
    return v;
  }
};
template <> struct SNorm<float> {
  static __device__ __forceinline__ float fix(float v, float inf, bool &bad, int &) {
    bad |= v != v;  // NaN
    return v >= inf ? __int_as_float(0x7f800000) : v;
  }
};

// a1 for signed matrices: zero diagonal, entries >= inf become inf / +inf, NaN is a data error,
// and (int32) the largest |finite entry| is maxed into words[0].
template <typename T>
__global__ void __launch_bounds__(256) normalise_signed_kernel(T *d, int64_t n, int64_t ld, T inf, int *words,
                                                               unsigned int *st) {
  bool bad = false;
  int m = 0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    T *row = d + i * ld;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) row[j] = j == i ? T(0) : SNorm<T>::fix(row[j], inf, bad, m);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(words, m);
  if (__syncthreads_or(bad) && threadIdx.x == 0) flag_status(st, APSP_ERR_DOMAIN);
}

__global__ void signed_range_kernel(int *words, int64_t n, unsigned int *st) {
  if ((int64_t)words[0] * (n - 1) >= kSignedRange) {
    words[kStop] = 1;
    flag_status(st, APSP_ERR_DOMAIN);
  }
}

template <bool FLOAT>
__global__ void __launch_bounds__(256) fw_diag_signed_kernel(int *d, int64_t ld, int64_t n, int64_t kb, int inf,
                                                             int *words, unsigned int *st) {
  if (words[kStop]) return;
  __shared__ __align__(16) int buf[512];
  const int64_t kb0 = kb * kBM;
  const int bk = (int)std::min<int64_t>(kBM, n - kb0);
  int *T = d + kb0 * ld + kb0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (warp & 3) * 4 + (lane >> 3), tn = (warp >> 2) * 8 + (lane & 7);
  const SignedCtl sc = {inf, kSignedThr};
  int r[8][8];
  load_tile_regs(r, T, ld, bk, tm, tn);
  const bool negative = close_tile_regs<FLOAT>(r, bk, tm, tn, buf, &sc);
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) r[i][j] = canon<FLOAT>(r[i][j], &sc);
  store_tile_regs(r, T, ld, bk, tm, tn);
  if (negative && threadIdx.x == 0) {
    words[kStop] = 1;
    flag_status(st, APSP_ERR_NEGATIVE_CYCLE);
  }
}

// A negative diagonal entry anywhere (a cycle the block-wise check could not see is impossible,
// but the final state is checked as well).
template <typename T>
__global__ void __launch_bounds__(256) diag_check_kernel(const T *d, int64_t ld, int64_t n, unsigned int *st) {
  bool neg = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    neg |= d[i * ld + i] < T(0);
  if (__syncthreads_or(neg) && threadIdx.x == 0) flag_status(st, APSP_ERR_NEGATIVE_CYCLE);
}

int fw_signed(void *d, int64_t n, int64_t ld, int dtype, int inf_i, int *words, cudaStream_t s) {
  CUtensorMap mA, mB, mC;
  int r;
  if ((r = make_operand_maps(d, n, n, ld, dtype, &mA, &mB, &mC))) return r;
  const int64_t nb = cdiv(n, kBM);
  TileProblem p = {};
  p.n = n;
  p.nb = nb;
  p.C = d;
  p.ldc = ld;
  p.inf_i = inf_i;
  p.status = status_word();
  p.wmax = nullptr;  // int32 storage then takes the int32 instruction sequence
  p.skip = words + kStop;
  p.sat = dtype == APSP_I32 ? kSignedThr : 0;
  for (int64_t kb = 0; kb < nb; ++kb) {
    if (dtype == APSP_I32)
      fw_diag_signed_kernel<false><<<1, 256, 0, s>>>(reinterpret_cast<int *>(d), ld, n, kb, inf_i, words,
                                                     status_word());
    else
      fw_diag_signed_kernel<true><<<1, 256, 0, s>>>(reinterpret_cast<int *>(d), ld, n, kb, inf_i, words,
                                                    status_word());
    APSP_LAUNCH_CHECK();
    if (nb == 1) break;
    p.kb = kb;
    p.ntiles = 2 * (nb - 1);
    if ((r = launch_tgemm(kModeFwPanels, false, dtype, mA, mB, mC, p, s))) return r;
    p.ntiles = (nb - 1) * (nb - 1);
    if ((r = launch_tgemm(kModeFwRest, true, dtype, mA, mB, mC, p, s))) return r;
  }
  const int grid = (int)std::min<int64_t>(cdiv(n, 256), (int64_t)sm_count() * 4);
  if (dtype == APSP_I32)
    diag_check_kernel<int><<<grid, 256, 0, s>>>(reinterpret_cast<const int *>(d), ld, n, status_word());
  else
    diag_check_kernel<float><<<grid, 256, 0, s>>>(reinterpret_cast<const float *>(d), ld, n, status_word());
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

}  // namespace

}  // namespace apsp

extern "C" size_t apsp_fw_signed_workspace_bytes(int64_t n, int64_t ld, int dtype) {
  (void)dtype;
  return apsp::closure_workspace_bytes(0, n, ld, 0, APSP_F32);  // bound words (+ aligned copy)
}

extern "C" int apsp_fw_signed(void *d, int64_t n, int64_t ld, int dtype, const void *inf, void *ws,
                              size_t ws_bytes, void *stream) {
  using namespace apsp;
  if (!dtype_ok(dtype) || n < 0) return APSP_ERR_ARG;
  if (n == 0) return APSP_OK;
  if (!d || ld < n || reinterpret_cast<uintptr_t>(d) % 16 != 0 || n > (int64_t)1 << 30) return APSP_ERR_ARG;
  int inf_i = 0;
  float inf_f = 0.f;
  if (dtype == APSP_I32 ? resolve_inf_i32(inf, &inf_i) : resolve_inf_f32(inf, &inf_f)) return APSP_ERR_ARG;
  if (dtype == APSP_I32 && inf_i < kSignedMinInf) return APSP_ERR_ARG;
  const size_t need = apsp_fw_signed_workspace_bytes(n, ld, dtype);
  if (ws && (ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0)) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void *own = nullptr;
  if (!ws) {
    if (ws_alloc(&own, need, s) != APSP_OK) {
      return APSP_ERR_NOMEM;
    }
    ws = own;
  }
  int r = APSP_OK;
  uint8_t *wsp = reinterpret_cast<uint8_t *>(ws);
  int *words = reinterpret_cast<int *>(wsp);
  wsp += kFlagBytes;
  if (cudaMemsetAsync(words, 0, 32, s) != cudaSuccess) r = APSP_ERR_CUDA;
  void *work = d;
  int64_t ldw = ld;
  if (!r && ld % 4 != 0) {
    ldw = round_up(n, 4);
    work = wsp;
    r = launch_copy2d(work, ldw, d, ld, n, n, s);
  }
  if (!r) {
    const int64_t cap = (int64_t)sm_count() * 8;
    const int grid = (int)(n < cap ? n : cap);
    if (dtype == APSP_I32) {
      normalise_signed_kernel<int><<<grid, 256, 0, s>>>(reinterpret_cast<int *>(work), n, ldw, inf_i, words,
                                                        status_word());
      signed_range_kernel<<<1, 1, 0, s>>>(words, n, status_word());
      note_launch();
    } else {
      normalise_signed_kernel<float><<<grid, 256, 0, s>>>(reinterpret_cast<float *>(work), n, ldw, inf_f, words,
                                                          status_word());
    }
    note_launch();
    if (cudaGetLastError() != cudaSuccess) r = APSP_ERR_CUDA;
  }
  if (!r) r = fw_signed(work, n, ldw, dtype, inf_i, words, s);
  if (!r && work != d) r = launch_copy2d(d, ld, work, ldw, n, n, s);
  ws_free(own, s);
  return r;
}
