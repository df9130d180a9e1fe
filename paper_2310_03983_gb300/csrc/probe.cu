// probe.cu -- (min,+) throughput probes: register-only instruction sequences (variants 0-8)
// and the GEMM engine's fp32 slab arithmetic in isolation (variants 9-11, further below).
//
// Each thread keeps 32 accumulators and, per loop iteration, performs 64 (min,+) "pairs"
// (one add and one min each) among them: c[j] = min(c[j], c[j+1] + b).  The operands are
// other accumulators, so the compiler can neither hoist nor fold the work, and 32 update
// chains per thread leave plenty of instruction-level parallelism.  The measured rate of
// the best instruction sequence is the denominator of the library's roofline: the chip's
// CUDA-core (min,+) peak.  (The paper's Eq. 2 product costs one add and one min per pair.)
#include "common.cuh"
#include "slab.cuh"

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


// ---------------------------------------------------------------------------------------
// Slab probes: the GEMM engine's fp32 slab arithmetic (ArithF32::slab_full) in isolation.
// One CTA of 256 threads per block, the thread layout of the engine's consumer warps, four
// 128 x 32 / 32 x 128 slab pairs resident in shared memory (no TMA, no barriers, no epilogue).
// Every iteration performs one slab: 128 x 128 x 32 pairs per CTA, 2048 per thread.
//   9:  operands read from shared memory, as the engine reads them;
//   10: the same instruction sequence on operands held in registers (each duplicated A pair
//       built once per launch): the rate of the packed adds and 3-input mins alone;
//   11: as 10, plus one integer XOR per 16 pairs: what other ALU-pipe work costs beside the
//       3-input mins, which run on that pipe.
// ---------------------------------------------------------------------------------------
constexpr int kProbeSlabInts = kSlabM * kSlabK + kSlabK * kSlabN;  // one A and one B slab
constexpr int kProbeSlabs = 4;
constexpr size_t kProbeSlabSmem = (size_t)kProbeSlabs * kProbeSlabInts * 4;

template <int V>
__device__ __forceinline__ void probe_slab_regs(const int *S, int tm, int tn, float (&acc)[8][8]) {
  // Operands of k = 0, 1 for every row and column of the thread, loaded once.
  uint64_t aa[8][2];
  int junk[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int4 v = lds128(S + a_off(tm + 16 * i, 0));
    aa[i][0] = pack2(__int_as_float(v.x), __int_as_float(v.x));
    aa[i][1] = pack2(__int_as_float(v.y), __int_as_float(v.y));
    junk[i] = v.z;
  }
  const int *Bs = S + kSlabM * kSlabK + 4 * tn;
  uint64_t b0[4], b1[4];
  lds128_2x64(Bs, b0[0], b0[1]);
  lds128_2x64(Bs + kSlabN, b1[0], b1[1]);
  lds128_2x64(Bs + 64, b0[2], b0[3]);
  lds128_2x64(Bs + kSlabN + 64, b1[2], b1[3]);
#pragma unroll 1
  for (int q = 0; q < 16; ++q) {  // 16 x 128 pairs per thread, as one slab
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (V == 11) junk[i] ^= q;
      uint64_t t0[4], t1[4];
#pragma unroll
      for (int jp = 0; jp < 4; ++jp) t0[jp] = fadd2_64(aa[i][0], b0[jp]);
#pragma unroll
      for (int jp = 0; jp < 4; ++jp) t1[jp] = fadd2_64(aa[i][1], b1[jp]);
#pragma unroll
      for (int jp = 0; jp < 4; ++jp) {
        acc[i][2 * jp] = Ops<float>::min3(acc[i][2 * jp], lo_of(t0[jp]), lo_of(t1[jp]));
        acc[i][2 * jp + 1] = Ops<float>::min3(acc[i][2 * jp + 1], hi_of(t0[jp]), hi_of(t1[jp]));
      }
    }
    b0[0] ^= 1ull;  // one operand changes per round, so no round can be folded into another
  }
  if (V == 11) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = fminf(acc[i][0], __int_as_float(junk[i] & 0x3f000000));
  }
}

template <int V>
__global__ void __launch_bounds__(256, 1) probe_slab_kernel(int iters, int *sink) {
  extern __shared__ __align__(1024) int probe_smem[];
  for (int i = threadIdx.x; i < kProbeSlabs * kProbeSlabInts; i += blockDim.x)
    probe_smem[i] = __float_as_int(1.0f + (float)(((unsigned)i * 2654435761u >> 7) & 1023) * 0.001f);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (warp & 3) * 4 + (lane >> 3), tn = (warp >> 2) * 8 + (lane & 7);  // as the engine
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 1e30f;
  __syncthreads();
  const long long c0 = clock64();
  for (int it = 0; it < iters; ++it) {
    const int *S = probe_smem + (it & (kProbeSlabs - 1)) * kProbeSlabInts;
    if (V == 9)
      ArithF32::slab_full(S, S + kSlabM * kSlabK, tm, tn, acc);
    else
      probe_slab_regs<V>(S, tm, tn, acc);
  }
  __syncthreads();
  const long long c1 = clock64();
  int s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) s ^= __float_as_int(acc[i][j]);
  // Thread 0 reports the CTA's SM clocks for the loop (in units of 1024), the others a checksum.
  sink[blockIdx.x * blockDim.x + threadIdx.x] = threadIdx.x ? s : (int)((c1 - c0) >> 10);
}

template <int V>
int launch_probe_slab(int blocks, int iters, int *sink, cudaStream_t s) {
  APSP_CUDA_TRY(cudaFuncSetAttribute(probe_slab_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kProbeSlabSmem));
  probe_slab_kernel<V><<<blocks, 256, kProbeSlabSmem, s>>>(iters, sink);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

}  // namespace apsp

extern "C" int apsp_probe_minplus(int variant, int blocks, int threads, int iters, void *sink, void *stream) {
  using namespace apsp;
  if (blocks <= 0 || threads <= 0 || threads > 256 || iters < 0 || sink == nullptr) return APSP_ERR_ARG;
  if (variant >= 9 && variant <= 11 && threads != 256) return APSP_ERR_ARG;  // the slab probes' layout
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
    case 9: return launch_probe_slab<9>(blocks, iters, o, s);
    case 10: return launch_probe_slab<10>(blocks, iters, o, s);
    case 11: return launch_probe_slab<11>(blocks, iters, o, s);
    default: return APSP_ERR_ARG;
  }
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}
