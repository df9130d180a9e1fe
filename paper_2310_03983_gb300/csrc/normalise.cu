// normalise.cu -- a1: validate and normalise a cost matrix before closure.
//
// The paper's input is a cost matrix with zero-cost self-loops (Sec. 3.4) and no negative
// cycles (Sec. 3.1).  In place on the n x n matrix (leading dimension ld):
//   d[i][i] = 0; entries >= the sentinel become INF (int32) or +inf (float32);
//   negative entries and NaN set APSP_ERR_DOMAIN in the device status word.
// HBM-bound: one read and one write of n^2 elements, 128-bit accesses when rows are 16-byte
// aligned.  Rows are distributed over a grid sized in multiples of the SM count.
#include "common.cuh"

namespace apsp {

template <typename T> struct Norm;
template <> struct Norm<int> {
  static __device__ __forceinline__ int fix(int v, int inf, bool &bad) {
    bad |= v < 0;
    return v >= inf ? inf : v;
  }
};
template <> struct Norm<float> {
  static __device__ __forceinline__ float fix(float v, float inf, bool &bad) {
    bad |= !(v >= 0.0f);  // catches NaN and negatives
    return v >= inf ? __int_as_float(0x7f800000) : v;
  }
};

template <typename T> __device__ __forceinline__ int finite_max(T v, T inf, int m) { return m; }
template <> __device__ __forceinline__ int finite_max<int>(int v, int inf, int m) { return v < inf ? max(m, v) : m; }

template <typename T>
__global__ void __launch_bounds__(256) normalise_kernel(T *d, int64_t n, int64_t ld, T inf, bool vec, unsigned int *st,
                                                        int *wmax) {
  bool bad = false;
  int m = 0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    T *row = d + i * ld;
    int64_t j0 = 0;
    if (vec) {
      const int64_t nv = n >> 2;
      for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
        T *p = row + 4 * v;
        float4 raw = *reinterpret_cast<float4 *>(p);
        T *e = reinterpret_cast<T *>(&raw);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          e[q] = (4 * v + q == i) ? T(0) : Norm<T>::fix(e[q], inf, bad);
          m = finite_max<T>(e[q], inf, m);
        }
        *reinterpret_cast<float4 *>(p) = raw;
      }
      j0 = nv << 2;
    }
    for (int64_t j = j0 + threadIdx.x; j < n; j += blockDim.x) {
      row[j] = (j == i) ? T(0) : Norm<T>::fix(row[j], inf, bad);
      m = finite_max<T>(row[j], inf, m);
    }
  }
  if (wmax) {
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(wmax, m);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) flag_status(st, APSP_ERR_DOMAIN);
}

__global__ void __launch_bounds__(256) scan_max_kernel(const int *x, int64_t rows, int64_t cols, int64_t ld, int inf,
                                                       int *out) {
  int m = 0;
  for (int64_t i = blockIdx.x; i < rows; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
      const int v = x[i * ld + j];
      if (v < inf) m = max(m, v);
    }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

int launch_scan_max(const void *x, int64_t rows, int64_t cols, int64_t ld, int inf, int *out, cudaStream_t s) {
  if (rows == 0 || cols == 0) return APSP_OK;
  const int64_t cap = (int64_t)sm_count() * 8;
  scan_max_kernel<<<(int)(rows < cap ? rows : cap), 256, 0, s>>>(reinterpret_cast<const int *>(x), rows, cols, ld,
                                                                 inf, out);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

int launch_normalise(void *d, int64_t n, int64_t ld, int dtype, int inf_i, float inf_f, int *wmax, cudaStream_t s) {
  if (n == 0) return APSP_OK;
  const bool vec = (reinterpret_cast<uintptr_t>(d) % 16 == 0) && (ld % 4 == 0);
  const int64_t cap = (int64_t)sm_count() * 8;
  const int grid = (int)(n < cap ? n : cap);
  if (dtype == APSP_I32)
    normalise_kernel<int><<<grid, 256, 0, s>>>(reinterpret_cast<int *>(d), n, ld, inf_i, vec, status_word(), wmax);
  else
    normalise_kernel<float><<<grid, 256, 0, s>>>(reinterpret_cast<float *>(d), n, ld, inf_f, vec, status_word(), nullptr);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

}  // namespace apsp

extern "C" int apsp_normalise(void *d, int64_t n, int64_t ld, int dtype, const void *inf, void *stream) {
  using namespace apsp;
  if (!dtype_ok(dtype) || n < 0 || (n > 0 && (d == nullptr || ld < n))) return APSP_ERR_ARG;
  int inf_i = 0;
  float inf_f = 0.f;
  if (dtype == APSP_I32 ? resolve_inf_i32(inf, &inf_i) : resolve_inf_f32(inf, &inf_f)) return APSP_ERR_ARG;
  return launch_normalise(d, n, ld, dtype, inf_i, inf_f, nullptr, reinterpret_cast<cudaStream_t>(stream));
}
