// common.cuh -- shared device/host helpers of libapsp (sm_103a only).
//
// Contents: the (min,+) element operations per dtype, mbarrier and TMA wrappers written as
// inline PTX, the per-device sticky status word, and host-side error plumbing.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/apsp.h"

#ifndef __CUDACC__
#error "compile with nvcc"
#endif

namespace apsp {

// ---------------------------------------------------------------------------------------
// Status word: one per device, sticky (bits OR-ed in by kernels) until apsp_device_status
// reads and clears it.  Bit layout: 1 << APSP_ERR_DOMAIN, 1 << APSP_ERR_TIMEOUT.
// ---------------------------------------------------------------------------------------
// Kernels receive the word's device address (status_word()) as an argument, so no
// translation unit needs relocatable device code.
__device__ __forceinline__ void flag_status(unsigned int *st, int code) {
  if (st) atomicOr(st, 1u << code);
}

// Iteration limit of every spin-wait on an mbarrier.  The longest legitimate wait in these
// kernels is one tile of work (tens of microseconds); 2^24 try_wait calls take between a
// fraction of a second and a few seconds, so a wait that cannot complete ends the kernel
// with APSP_ERR_TIMEOUT instead of hanging the GPU.
constexpr uint32_t kSpinLimit = 1u << 24;

// Cap of the packed 16-bit (min,+) arithmetic: values at or above it mean "at least the cap";
// two capped values still sum below 2^15.
constexpr int kCap16 = 0x3FFF;

// ---------------------------------------------------------------------------------------
// (min,+) element operations.  int32 values live in [0, INF] with INF <= 0x3FFFFFFF, so
// a + b never overflows and min() against an accumulator <= INF saturates for free.
// ---------------------------------------------------------------------------------------
template <typename T> struct Ops;

template <> struct Ops<int> {
  static __device__ __forceinline__ int add(int a, int b) { return a + b; }
  static __device__ __forceinline__ int mn(int a, int b) { return min(a, b); }
  // c = min(c, a + b) as one fused DPX operation
  static __device__ __forceinline__ int addmin(int a, int b, int c) { return __viaddmin_s32(a, b, c); }
  static __device__ __forceinline__ int min3(int a, int b, int c) { return __vimin3_s32(a, b, c); }
};

template <> struct Ops<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mn(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float addmin(float a, float b, float c) { return fminf(c, __fadd_rn(a, b)); }
  static __device__ __forceinline__ float min3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
  }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Packed pair add (PTX add.rn.f32x2, sm_100+): {a.x + b.x, a.y + b.y} in one instruction.
// Subnormals are kept (no .ftz), which the exact small-integer path relies on.
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// The same packed add on operands already held as 64-bit register pairs, and the helpers
// that build / split such pairs.  Building each pair once and reusing it keeps the packing
// moves out of the inner loop.
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ uint64_t fadd2_64(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float lo_of(uint64_t v) {
  float f, g;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f), "=f"(g) : "l"(v));
  return f;
}
__device__ __forceinline__ float hi_of(uint64_t v) {
  float f, g;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f), "=f"(g) : "l"(v));
  return g;
}
__device__ __forceinline__ void lds128_2x64(const void *p, uint64_t &a, uint64_t &b) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(smem_u32(p)));
}

// ---------------------------------------------------------------------------------------
// mbarrier / TMA wrappers (PTX ISA: mbarrier.*, cp.async.bulk.tensor.*)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.  Returns false (and flags
// APSP_ERR_TIMEOUT) if the limit is reached.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned int *st) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  flag_status(st, APSP_ERR_TIMEOUT);
  return false;
}

// Bounded wait until the device counter *c reaches `need` (loads with acquire semantics at GPU
// scope; the writers store, then add with release semantics: counter_add_release).  Returns
// false (and flags APSP_ERR_TIMEOUT) if the limit is reached.
__device__ __forceinline__ bool counter_wait(const int *c, int need, unsigned int *st) {
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    if (v >= need) return true;
    __nanosleep(32);
  }
  flag_status(st, APSP_ERR_TIMEOUT);
  return false;
}

__device__ __forceinline__ void counter_add_release(int *c, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(c), "r"(v) : "memory");
}

// Orders this thread's earlier generic-proxy accesses (the acquire above) before its later
// async-proxy ones (TMA loads of the data the counter guards).
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

// 2-D tiled TMA load of box {x (inner), y} at coordinates (x, y) into smem, completing
// `bytes` of transaction count on bar.  x * sizeof(elem) must be a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *m, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Programmatic dependent launch (PTX griddepcontrol).  A kernel launched with
// launch_pdl() may be scheduled while the kernel before it on the stream is still running, so
// that its CTAs are resident and set up when that kernel ends.  pdl_wait() returns once every
// prerequisite grid has completed and its memory operations are visible; kernels launched that
// way call it before touching global memory.  pdl_trigger() allows the next kernel on the
// stream to be scheduled.  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ int4 lds128(const void *p) {
  int4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(smem_u32(p)));
  return v;
}

}  // namespace apsp

// ---------------------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------------------
#define APSP_CUDA_TRY(expr)                                \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return APSP_ERR_CUDA;           \
  } while (0)

namespace apsp {
// Counts one kernel launch enqueued by the library (host side; read by apsp_launch_count).
void note_launch();
}  // namespace apsp

// Follows every kernel launch: counts it and turns a launch error into APSP_ERR_CUDA.
#define APSP_LAUNCH_CHECK()                                \
  do {                                                     \
    apsp::note_launch();                                   \
    if (cudaGetLastError() != cudaSuccess) return APSP_ERR_CUDA; \
  } while (0)

namespace apsp {

inline int elem_size(int dtype) { return 4; }
inline bool dtype_ok(int dtype) { return dtype == APSP_I32 || dtype == APSP_F32; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// Number of SMs of the current device (cached per device).
int sm_count();

// Whether launch_pdl() sets the programmatic-serialization attribute: on unless the
// environment variable APSP_PDL is "0" when the library first launches.
bool pdl_enabled();

// Launches kernel k with the programmatic-serialization attribute (see pdl_wait()); k must
// call pdl_wait() before any global memory access.  Without the attribute (APSP_PDL=0) it is
// an ordinary launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Workspace the library allocates for a call made without one: stream-ordered, from a
// per-device pool that keeps freed memory for the next call (runtime.cu).
int ws_alloc(void **p, size_t bytes, cudaStream_t s);
void ws_free(void *p, cudaStream_t s);

// Device address of the current device's status word (nullptr on failure).
unsigned int *status_word();

// Encode a 2-D row-major tensor map: `rows` x `cols` elements (4 bytes each), leading
// dimension ld elements, box `box_rows` x `box_cols`, zero OOB fill.  swizzle128: the box's
// rows are 128 bytes and land in shared memory with their 16-byte chunks XOR-permuted by
// (row mod 8) (requires a 1024-byte aligned destination).
int make_tmap_2d(CUtensorMap *out, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                 int box_cols, int dtype, bool swizzle128 = false);

// Resolve the int32 sentinel (NULL -> APSP_INF_I32) or float sentinel (NULL -> +inf).
int resolve_inf_i32(const void *inf, int *out);
int resolve_inf_f32(const void *inf, float *out);

}  // namespace apsp
