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

template <typename T>
__global__ void __launch_bounds__(256) normalise_kernel(T *d, int64_t n, int64_t ld, T inf, bool vec, unsigned int *st) {
  bool bad = false;
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
        for (int q = 0; q < 4; ++q) e[q] = (4 * v + q == i) ? T(0) : Norm<T>::fix(e[q], inf, bad);
        *reinterpret_cast<float4 *>(p) = raw;
      }
      j0 = nv << 2;
    }
    for (int64_t j = j0 + threadIdx.x; j < n; j += blockDim.x) row[j] = (j == i) ? T(0) : Norm<T>::fix(row[j], inf, bad);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) flag_status(st, APSP_ERR_DOMAIN);
}

int launch_normalise(void *d, int64_t n, int64_t ld, int dtype, int inf_i, float inf_f, cudaStream_t s) {
  if (n == 0) return APSP_OK;
  const bool vec = (reinterpret_cast<uintptr_t>(d) % 16 == 0) && (ld % 4 == 0);
  const int64_t cap = (int64_t)sm_count() * 8;
  const int grid = (int)(n < cap ? n : cap);
  if (dtype == APSP_I32)
    normalise_kernel<int><<<grid, 256, 0, s>>>(reinterpret_cast<int *>(d), n, ld, inf_i, vec, status_word());
  else
    normalise_kernel<float><<<grid, 256, 0, s>>>(reinterpret_cast<float *>(d), n, ld, inf_f, vec, status_word());
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
  return launch_normalise(d, n, ld, dtype, inf_i, inf_f, reinterpret_cast<cudaStream_t>(stream));
}
