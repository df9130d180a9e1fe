// noalloc.cu -- R-Kleene closure that performs no device memory allocation.
//
// Some callers cannot call cudaMalloc (or cudaMallocAsync): code that runs inside a framework
// or plugin host that owns every byte of device memory through its own pool, where a stray
// allocation either fails or fragments the pool; latency-critical request paths that forbid
// allocator calls; and processes started under a hard device-memory budget.  apsp_rkleene
// needs scratch (a copy of the block it overwrites and a few bound words), which it takes
// from the caller or allocates.  This variant takes it from a fixed array compiled into the
// library instead, so the caller passes only the matrix.
//
// The array holds 256 bytes of bound words plus one 2048 x 2048 int32 block: enough for the
// required scratch of any n <= APSP_NOALLOC_MAX_N (4096), and for smaller n (up to about 2816)
// also the packed 16-bit operands of the largest products.  Every GPU that loads libapsp.so keeps these ~16 MiB until
// the process exits.  All calls share the one array per device, so calls that overlap on the
// GPU (different streams, or different host threads) race on it and must be serialised by
// the caller.  The array keeps whatever the previous call left in it; the closure zeroes the
// bound words it needs and fully overwrites the scratch block before reading it.
#include <mutex>

#include "closure.cuh"

namespace apsp {

constexpr int64_t kNoAllocMaxN = APSP_NOALLOC_MAX_N;
constexpr size_t kNoAllocBytes = kFlagBytes + size_t(kNoAllocMaxN / 2) * size_t(kNoAllocMaxN / 2) * 4;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array on the current device.  In host code the array's name is only
// a host-side stand-in, so the address is looked up once per device (with that device
// current) and cached.
static void *noalloc_scratch(int *err) {
  static void *addr[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *err = APSP_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      *err = APSP_ERR_CUDA;
      return nullptr;
    }
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace apsp

extern "C" int apsp_rkleene_noalloc(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int cutoff,
                                    void *stream) {
  using namespace apsp;
  if (n < 0 || n > kNoAllocMaxN) return APSP_ERR_ARG;   // larger graphs need apsp_rkleene
  if (n > 0 && ld % 4 != 0) return APSP_ERR_ARG;        // would need an aligned copy of the whole matrix
  // The array always holds the required scratch.  When the optional room for packed 16-bit
  // operands also fits beside it (top-level split h <= 1408, i.e. n up to about 2816), int32
  // products of at least 1e9 pairs run on 16-bit pairs inside the array, as apsp_rkleene does
  // with a full workspace; otherwise they take the 32-bit path.  Results are the same either way.
  if (closure_required_bytes(1, n, ld, cutoff) > kNoAllocBytes) return APSP_ERR_ARG;
  int err = APSP_OK;
  void *ws = noalloc_scratch(&err);
  if (!ws) return err;
  return closure_entry(1, d, n, ld, dtype, inf, cutoff, ws, kNoAllocBytes, stream);
}
