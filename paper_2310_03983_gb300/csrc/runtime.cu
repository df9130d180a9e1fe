// runtime.cu -- host runtime of libapsp: status word, device queries, TMA descriptor
// encoding, sentinel handling and the small C-ABI helpers.
#include <atomic>
#include <cstdlib>
#include <math.h>
#include <mutex>
#include <string.h>
#include <vector>

#include "common.cuh"

namespace apsp {

__device__ unsigned int g_status = 0;

// Per-device caches below are atomics: calls may come from several host threads, and every
// thread that fills an entry stores the same value.
unsigned int *status_word() {
  static std::atomic<unsigned int *> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cached[dev].load(std::memory_order_acquire)) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    cached[dev].store(reinterpret_cast<unsigned int *>(p), std::memory_order_release);
  }
  return cached[dev].load(std::memory_order_acquire);
}

int sm_count() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("APSP_PDL");
    return !(e && e[0] == '0' && e[1] == 0);
  }();
  return on;
}

// Library workspace pool: a stream-ordered memory pool per device that keeps freed blocks
// (release threshold = the whole device), so a workspace the library allocates for a call
// without one is reused by the next call instead of being unmapped and mapped again whenever
// the caller synchronises (the default pool's behaviour), which costs far more than the
// allocation itself for large workspaces.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64];
static bool g_have_pool[64];

static cudaMemPool_t lib_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_have_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
    g_have_pool[dev] = true;
  }
  return g_pools[dev];
}

int ws_alloc(void **p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = lib_pool();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return APSP_ERR_NOMEM;
  }
  return APSP_OK;
}

void ws_free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

int make_tmap_2d(CUtensorMap *out, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                 int box_cols, int dtype, bool swizzle128) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return APSP_ERR_CUDA;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || (ld * 4) % 16 != 0) return APSP_ERR_ARG;
  // TMA needs non-zero extents; a zero-sized operand is never loaded, so any shape works.
  cuuint64_t dims[2] = {(cuuint64_t)(cols > 0 ? cols : 1), (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMapDataType t = dtype == APSP_I32 ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(out, t, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? APSP_OK : APSP_ERR_CUDA;
}

int resolve_inf_i32(const void *inf, int *out) {
  int v = inf ? *reinterpret_cast<const int *>(inf) : APSP_INF_I32;
  if (v < 1 || v > APSP_INF_I32) return 1;
  *out = v;
  return 0;
}

int resolve_inf_f32(const void *inf, float *out) {
  float v = inf ? *reinterpret_cast<const float *>(inf) : INFINITY;
  if (!(v > 0.0f)) return 1;  // rejects NaN, zero and negatives
  *out = v;
  return 0;
}

// ------------------------------------ launch count -------------------------------------
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ------------------------------------ tracing ------------------------------------------
struct TraceRec {
  cudaEvent_t e0, e1;
  int mode;
  double pairs;
};
static std::mutex g_trace_mu;
static std::vector<TraceRec> g_trace;
static std::atomic<bool> g_trace_on{false};

bool trace_on() { return g_trace_on.load(std::memory_order_relaxed); }

void trace_begin(cudaStream_t s, void **ev0) {
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) == cudaSuccess) cudaEventRecord(e, s);
  *ev0 = e;
}

void trace_end(cudaStream_t s, void *ev0, int mode, double pairs) {
  cudaEvent_t e1 = nullptr;
  if (!ev0 || cudaEventCreate(&e1) != cudaSuccess) return;
  cudaEventRecord(e1, s);
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace.push_back({reinterpret_cast<cudaEvent_t>(ev0), e1, mode, pairs});
}

}  // namespace apsp

extern "C" int apsp_trace_enable(int on) {
  apsp::g_trace_on = on != 0;
  return APSP_OK;
}

extern "C" int apsp_trace_read(int mode, double *total_ms, int64_t *launches, double *pairs) {
  using namespace apsp;
  if (!total_ms || !launches || !pairs) return APSP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  double ms = 0, pr = 0;
  int64_t cnt = 0;
  int rc = APSP_OK;
  std::vector<TraceRec> keep;
  for (auto &t : g_trace) {
    if (t.mode != mode && mode >= 0) {
      keep.push_back(t);
      continue;
    }
    if (cudaEventSynchronize(t.e1) != cudaSuccess) rc = APSP_ERR_CUDA;
    float e = 0.f;
    if (cudaEventElapsedTime(&e, t.e0, t.e1) != cudaSuccess) rc = APSP_ERR_CUDA;
    ms += e;
    pr += t.pairs;
    ++cnt;
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  g_trace.swap(keep);
  *total_ms = ms;
  *launches = cnt;
  *pairs = pr;
  return rc;
}

extern "C" int apsp_workspace_pool_trim(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return APSP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(apsp::g_pool_mu);
  if (apsp::g_have_pool[dev] && cudaMemPoolTrimTo(apsp::g_pools[dev], 0) != cudaSuccess) return APSP_ERR_CUDA;
  return APSP_OK;
}

extern "C" int apsp_version(void) { return APSP_VERSION; }

extern "C" const char *apsp_status_str(int s) {
  switch (s) {
    case APSP_OK: return "ok";
    case APSP_ERR_ARG: return "invalid argument";
    case APSP_ERR_DOMAIN: return "negative weight, NaN or out-of-range entry in the input";
    case APSP_ERR_NOMEM: return "workspace allocation failed";
    case APSP_ERR_CUDA: return "CUDA error";
    case APSP_ERR_TIMEOUT: return "bounded device wait timed out";
    case APSP_ERR_UNSUPPORTED: return "unsupported device or feature";
    case APSP_ERR_NEGATIVE_CYCLE: return "negative cycle";
    default: return "unknown status";
  }
}

extern "C" int apsp_device_status(void *stream, int *out) {
  if (!out) return APSP_ERR_ARG;
  APSP_CUDA_TRY(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  unsigned int bits = 0, zero = 0;
  APSP_CUDA_TRY(cudaMemcpyFromSymbol(&bits, apsp::g_status, sizeof(bits)));
  APSP_CUDA_TRY(cudaMemcpyToSymbol(apsp::g_status, &zero, sizeof(zero)));
  *out = (bits & (1u << APSP_ERR_TIMEOUT)) ? APSP_ERR_TIMEOUT
         : (bits & (1u << APSP_ERR_ARG))    ? APSP_ERR_ARG
         : (bits & (1u << APSP_ERR_NEGATIVE_CYCLE)) ? APSP_ERR_NEGATIVE_CYCLE
         : (bits & (1u << APSP_ERR_DOMAIN)) ? APSP_ERR_DOMAIN
                                            : APSP_OK;
  return APSP_OK;
}

extern "C" int64_t apsp_launch_count(int reset) {
  return reset ? apsp::g_launches.exchange(0) : apsp::g_launches.load();
}
