// probe.cu -- register-only (min,+) throughput probes.
//
// Each thread keeps 32 accumulators and, per loop iteration, performs 64 (min,+) "pairs"
// (one add and one min each) among them: c[j] = min(c[j], c[j+1] + b).  The operands are
// other accumulators, so the compiler can neither hoist nor fold the work, and 32 update
// chains per thread leave plenty of instruction-level parallelism.  The measured rate of
// the best instruction sequence is the denominator of the library's roofline: the chip's
// CUDA-core (min,+) peak.  (The paper's Eq. 2 product costs one add and one min per pair.)
#include "common.cuh"

namespace apsp {

template <int V> struct ProbeBody;

// 0: int32 fused add-min, one DPX operation per pair
template <> struct ProbeBody<0> {
  typedef int T;
  static __device__ __forceinline__ void run(int *c, int b0, int b1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = __viaddmin_s32(c[(j + 1) & 31], b0, c[j]);
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = __viaddmin_s32(c[(j + 3) & 31], b1, c[j]);
  }
};
// 1: int32 add, then 2-input min
template <> struct ProbeBody<1> {
  typedef int T;
  static __device__ __forceinline__ void run(int *c, int b0, int b1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = min(c[j], c[(j + 1) & 31] + b0);
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = min(c[j], c[(j + 3) & 31] + b1);
  }
};
// 2: int32 two adds, then one 3-input min (two pairs)
template <> struct ProbeBody<2> {
  typedef int T;
  static __device__ __forceinline__ void run(int *c, int b0, int b1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = __vimin3_s32(c[j], c[(j + 1) & 31] + b0, c[(j + 3) & 31] + b1);
  }
};
// 3: fp32 add, then 2-input min
template <> struct ProbeBody<3> {
  typedef float T;
  static __device__ __forceinline__ void run(float *c, float b0, float b1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = fminf(c[j], __fadd_rn(c[(j + 1) & 31], b0));
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = fminf(c[j], __fadd_rn(c[(j + 3) & 31], b1));
  }
};
// 4: fp32 two adds, then one 3-input min
template <> struct ProbeBody<4> {
  typedef float T;
  static __device__ __forceinline__ void run(float *c, float b0, float b1) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      c[j] = Ops<float>::min3(c[j], __fadd_rn(c[(j + 1) & 31], b0), __fadd_rn(c[(j + 3) & 31], b1));
  }
};

// 5: fp32 packed pair add (two adds in one instruction), then one 3-input min
template <> struct ProbeBody<5> {
  typedef float T;
  static __device__ __forceinline__ void run(float *c, float b0, float b1) {
    const float2 bb = make_float2(b0, b1);
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      float2 t = fadd2(make_float2(c[(j + 2) & 31], c[(j + 3) & 31]), bb);
      float2 u = fadd2(make_float2(c[(j + 4) & 31], c[(j + 5) & 31]), bb);
      c[j] = Ops<float>::min3(c[j], t.x, t.y);
      c[j + 1] = Ops<float>::min3(c[j + 1], u.x, u.y);
    }
  }
};

// 6: variant 5 on subnormal operands: int32 values below 2^24 read as fp32 bit patterns
// (v * 2^-149), the form in which the library adds small integers exactly in fp32.
template <> struct ProbeBody<6> : ProbeBody<5> {};

// 7: packed int16 pairs, one fused DPX add-min over two 16-bit lanes per operation
//    (__viaddmin_s16x2): 128 pairs per iteration instead of 64.
template <> struct ProbeBody<7> {
  typedef int T;
  static __device__ __forceinline__ void run(int *c, int b0, int b1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = (int)__viaddmin_s16x2((unsigned)c[(j + 1) & 31], (unsigned)b0, (unsigned)c[j]);
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = (int)__viaddmin_s16x2((unsigned)c[(j + 3) & 31], (unsigned)b1, (unsigned)c[j]);
  }
};
// 8: packed int16 pairs, SIMD add then SIMD min (__vadd2, __vmins2): 128 pairs per iteration.
template <> struct ProbeBody<8> {
  typedef int T;
  static __device__ __forceinline__ void run(int *c, int b0, int b1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = (int)__vmins2((unsigned)c[j], __vadd2((unsigned)c[(j + 1) & 31], (unsigned)b0));
#pragma unroll
    for (int j = 0; j < 32; ++j) c[j] = (int)__vmins2((unsigned)c[j], __vadd2((unsigned)c[(j + 3) & 31], (unsigned)b1));
  }
};

template <int V> __device__ __forceinline__ typename ProbeBody<V>::T probe_init(int v) {
  return (typename ProbeBody<V>::T)v;
}
template <> __device__ __forceinline__ float probe_init<6>(int v) { return __int_as_float(v); }

template <int V>
__global__ void __launch_bounds__(256) probe_kernel(int iters, int *sink) {
  typedef typename ProbeBody<V>::T T;
  T c[32];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int j = 0; j < 32; ++j) c[j] = probe_init<V>(((tid * 7 + j * 13) & 1023) + 100000);
  const T b0 = probe_init<V>(1 + (tid & 3)), b1 = probe_init<V>(2 + (tid & 5));
  for (int it = 0; it < iters; ++it) ProbeBody<V>::run(c, b0, b1);
  int s = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) s ^= *reinterpret_cast<int *>(&c[j]);
  sink[tid] = s;
}

}  // namespace apsp

extern "C" int apsp_probe_minplus(int variant, int blocks, int threads, int iters, void *sink, void *stream) {
  using namespace apsp;
  if (blocks <= 0 || threads <= 0 || threads > 256 || iters < 0 || sink == nullptr) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int *o = reinterpret_cast<int *>(sink);
  switch (variant) {
    case 0: probe_kernel<0><<<blocks, threads, 0, s>>>(iters, o); break;
    case 1: probe_kernel<1><<<blocks, threads, 0, s>>>(iters, o); break;
    case 2: probe_kernel<2><<<blocks, threads, 0, s>>>(iters, o); break;
    case 3: probe_kernel<3><<<blocks, threads, 0, s>>>(iters, o); break;
    case 4: probe_kernel<4><<<blocks, threads, 0, s>>>(iters, o); break;
    case 5: probe_kernel<5><<<blocks, threads, 0, s>>>(iters, o); break;
    case 6: probe_kernel<6><<<blocks, threads, 0, s>>>(iters, o); break;
    case 7: probe_kernel<7><<<blocks, threads, 0, s>>>(iters, o); break;
    case 8: probe_kernel<8><<<blocks, threads, 0, s>>>(iters, o); break;
    default: return APSP_ERR_ARG;
  }
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}
