// host.cu -- entry points on HOST buffers: the matrix (or batch) is copied to the device,
// closed there by the device entry points, and copied back; the call returns once the host
// result is written.
//
// apsp_batched_host splits the batch into chunks of consecutive graphs with about equal work
// (sum of n^3) and pipelines them over three streams: the copy of chunk c + 1 to the device and
// the copy of chunk c - 1 back to the host run while chunk c is closed on the caller's stream.
// Host-device copies use their own copy engines, so on pinned host memory the step costs about
// the closure plus one chunk's copies instead of the sum of the three.
#include <sys/mman.h>
#include <unistd.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tgemm.cuh"

namespace apsp {

namespace {

struct CopyStreams {
  cudaStream_t in = nullptr, out = nullptr;
};

// Two non-blocking copy streams per device, created once and kept for the process.
int copy_streams(CopyStreams *cs) {
  static CopyStreams cache[64];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return APSP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  CopyStreams &c = cache[dev];
  if (!c.in) {
    if (cudaStreamCreateWithFlags(&c.in, cudaStreamNonBlocking) != cudaSuccess) return APSP_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&c.out, cudaStreamNonBlocking) != cudaSuccess) {
      cudaStreamDestroy(c.in);
      c.in = nullptr;
      return APSP_ERR_CUDA;
    }
  }
  *cs = c;
  return APSP_OK;
}

// --------------------------------------------------------------- huge-page host memory
// Linux madvise advice values (uapi), named here for kernels whose headers predate them.
constexpr int kMadvPopulateWrite = 23;  // MADV_POPULATE_WRITE, Linux 5.14
constexpr int kMadvCollapse = 25;       // MADV_COLLAPSE, Linux 6.1

// The transparent-huge-page size of this host (the kernel's PMD size), 0 when unknown.
size_t thp_bytes() {
  static size_t cached = [] {
    size_t v = 0;
    if (FILE *f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
      unsigned long long x = 0;
      if (std::fscanf(f, "%llu", &x) == 1) v = (size_t)x;
      std::fclose(f);
    }
    return v;
  }();
  return cached;
}

struct HostMapping {
  void *raw;       // the mmap'ed range (with room to align), or null for cudaHostAlloc memory
  size_t raw_len;
};
std::mutex g_host_mu;
std::map<void *, HostMapping> g_host_allocs;

struct Chunk {
  int64_t g0, g1;  // graphs [g0, g1)
  int64_t lo, hi;  // pool elements [lo, hi)
};

// Consecutive graph ranges of about equal sum of n^3, with the pool range each one covers.
// Empty when the ranges would overlap (a layout whose graphs are not in pool order).
std::vector<Chunk> make_chunks(const int64_t *off, const int32_t *ns, const int32_t *lds, int64_t count,
                               int chunks) {
  double total = 0.0;
  for (int64_t g = 0; g < count; ++g) total += (double)std::max(ns[g], 0) * std::max(ns[g], 0) * std::max(ns[g], 0);
  std::vector<Chunk> out;
  int64_t g = 0;
  double done = 0.0;
  for (int c = 0; c < chunks && g < count; ++c) {
    const double target = total * (c + 1) / chunks;
    Chunk ch = {g, g, INT64_MAX, INT64_MIN};
    while (g < count && (done < target || ch.g1 == ch.g0 || c == chunks - 1)) {
      const int64_t n = std::max(ns[g], 0);
      done += (double)n * n * n;
      if (n > 0) {
        ch.lo = std::min(ch.lo, off[g]);
        ch.hi = std::max(ch.hi, off[g] + (n - 1) * (int64_t)lds[g] + n);
      }
      ch.g1 = ++g;
    }
    if (ch.lo > ch.hi) ch.lo = ch.hi = 0;  // only empty graphs
    out.push_back(ch);
  }
  std::vector<Chunk> sorted = out;
  std::sort(sorted.begin(), sorted.end(), [](const Chunk &a, const Chunk &b) { return a.lo < b.lo; });
  for (size_t i = 1; i < sorted.size(); ++i)
    if (sorted[i].lo < sorted[i - 1].hi && sorted[i].hi > sorted[i].lo) return {};
  return out;
}

}  // namespace

}  // namespace apsp

extern "C" void *apsp_host_alloc(size_t bytes) {
  using namespace apsp;
  if (bytes == 0) return nullptr;
  const size_t hp = thp_bytes();
  void *p = nullptr;
  HostMapping m = {nullptr, 0};
  if (hp && bytes >= hp / 4) {
    const size_t len = (bytes + hp - 1) / hp * hp;
    void *raw = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (raw != MAP_FAILED) {
      const uintptr_t base = (reinterpret_cast<uintptr_t>(raw) + hp - 1) / hp * hp;
      p = reinterpret_cast<void *>(base);
      madvise(p, len, MADV_HUGEPAGE);  // advice only: small pages still work
      // Fault every page in now (huge where the kernel has a free huge page), then ask it to
      // collapse whatever the faults left in base pages into huge pages; both best effort (older
      // kernels refuse them), and both before the range is pinned, which rules collapsing out.
      madvise(p, len, kMadvPopulateWrite);
      madvise(p, len, kMadvCollapse);
      if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        munmap(raw, len + hp);
        p = nullptr;
      } else {
        m = {raw, len + hp};
      }
    }
  }
  if (!p) {
    if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  std::lock_guard<std::mutex> lk(g_host_mu);
  g_host_allocs[p] = m;
  return p;
}

extern "C" int apsp_host_free(void *p) {
  using namespace apsp;
  if (!p) return APSP_OK;
  HostMapping m;
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    auto it = g_host_allocs.find(p);
    if (it == g_host_allocs.end()) return APSP_ERR_ARG;
    m = it->second;
    g_host_allocs.erase(it);
  }
  if (!m.raw) return cudaFreeHost(p) == cudaSuccess ? APSP_OK : APSP_ERR_CUDA;
  const int r = cudaHostUnregister(p) == cudaSuccess ? APSP_OK : APSP_ERR_CUDA;
  munmap(m.raw, m.raw_len);
  return r;
}

extern "C" size_t apsp_batched_host_workspace_bytes(const int32_t *ns_host, const int64_t *offsets_host,
                                                    const int32_t *lds_host, int64_t count, int dtype, int chunks) {
  using namespace apsp;
  if (!ns_host || count <= 0) return 256;
  if (chunks < 1) chunks = 1;
  std::vector<Chunk> cs = offsets_host && lds_host ? make_chunks(offsets_host, ns_host, lds_host, count, chunks)
                                                   : std::vector<Chunk>();
  if (cs.empty()) cs.push_back(Chunk{0, count, 0, 0});
  size_t need = 256;
  for (const Chunk &c : cs)
    need = std::max(need, apsp_batched_staged_workspace_bytes(ns_host + c.g0, c.g1 - c.g0, dtype));
  return need;
}

extern "C" int apsp_batched_host(const void *h_in, void *h_out, void *pool, const int64_t *offsets_host,
                                 const int32_t *ns_host, const int32_t *lds_host, const int64_t *offsets,
                                 const int32_t *ns, const int32_t *lds, int64_t count, int dtype, const void *inf,
                                 int chunks, void *ws, size_t ws_bytes, void *stream) {
  using namespace apsp;
  if (!dtype_ok(dtype) || count < 0 || chunks < 0) return APSP_ERR_ARG;
  if (count == 0) return APSP_OK;
  if (!h_in || !h_out || !pool || !offsets_host || !ns_host || !lds_host || !offsets || !ns || !lds)
    return APSP_ERR_ARG;
  for (int64_t g = 0; g < count; ++g)  // the copy ranges come from these: check them on the host
    if (ns_host[g] > 0 && (offsets_host[g] < 0 || lds_host[g] < ns_host[g])) return APSP_ERR_ARG;
  std::vector<Chunk> cs = make_chunks(offsets_host, ns_host, lds_host, count, chunks ? chunks : 4);
  if (cs.empty()) cs = make_chunks(offsets_host, ns_host, lds_host, count, 1);
  const size_t need = apsp_batched_host_workspace_bytes(ns_host, offsets_host, lds_host, count, dtype,
                                                        (int)cs.size());
  if (ws && (ws_bytes < 256 || reinterpret_cast<uintptr_t>(ws) % 256 != 0)) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CopyStreams st;
  int r = copy_streams(&st);
  if (r) return r;
  void *own = nullptr;
  if (!ws) {
    if (ws_alloc(&own, need, s) != APSP_OK) return APSP_ERR_NOMEM;
    ws = own;
    ws_bytes = need;
  }
  const size_t esz = 4;
  std::vector<cudaEvent_t> ev(2 * cs.size() + 1, nullptr);
  for (auto &e : ev)
    if (!r && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) r = APSP_ERR_CUDA;
  cudaEvent_t start = ev.back();
  // The copy streams start after whatever the caller queued on its stream (the pool may be in use).
  if (!r && cudaEventRecord(start, s) != cudaSuccess) r = APSP_ERR_CUDA;
  if (!r && cudaStreamWaitEvent(st.in, start, 0) != cudaSuccess) r = APSP_ERR_CUDA;
  for (size_t c = 0; c < cs.size() && !r; ++c) {
    const Chunk &ch = cs[c];
    const size_t bytes = (size_t)(ch.hi - ch.lo) * esz;
    uint8_t *dp = reinterpret_cast<uint8_t *>(pool) + ch.lo * esz;
    if (bytes && cudaMemcpyAsync(dp, reinterpret_cast<const uint8_t *>(h_in) + ch.lo * esz, bytes,
                                 cudaMemcpyHostToDevice, st.in) != cudaSuccess)
      r = APSP_ERR_CUDA;
    if (!r && cudaEventRecord(ev[2 * c], st.in) != cudaSuccess) r = APSP_ERR_CUDA;
    if (!r && cudaStreamWaitEvent(s, ev[2 * c], 0) != cudaSuccess) r = APSP_ERR_CUDA;
    if (!r) r = apsp_batched(pool, offsets + ch.g0, ns + ch.g0, lds + ch.g0, nullptr, ns_host + ch.g0, ch.g1 - ch.g0,
                             dtype, inf, ws, ws_bytes, stream);
    if (!r && cudaEventRecord(ev[2 * c + 1], s) != cudaSuccess) r = APSP_ERR_CUDA;
    if (!r && cudaStreamWaitEvent(st.out, ev[2 * c + 1], 0) != cudaSuccess) r = APSP_ERR_CUDA;
    if (!r && bytes &&
        cudaMemcpyAsync(reinterpret_cast<uint8_t *>(h_out) + ch.lo * esz, dp, bytes, cudaMemcpyDeviceToHost,
                        st.out) != cudaSuccess)
      r = APSP_ERR_CUDA;
  }
  ws_free(own, s);
  // Every copy back is queued on st.out after the last closure: waiting for it covers all.
  if (cudaStreamSynchronize(st.out) != cudaSuccess && !r) r = APSP_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess && !r) r = APSP_ERR_CUDA;
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  return r;
}

namespace {

// n x n matrix of 4-byte elements between host and device.  Pinned host memory (registered or
// from cudaHostAlloc, so it has a device address) is copied by a kernel on the SMs, loading or
// storing through that address: the GPU reaches host memory through its own translations of the
// host pages, and after a closure has evicted them the copy engine, which walks the pages one
// after the other, was measured at 260-1423 ms for a 4 GiB copy it does in 20 ms when they are
// cached, while the kernel's thousands of concurrent accesses overlap the misses (20.3 ms in,
// 22.2 ms out, in every case measured).  Other host memory takes the copy engine: one linear
// copy when both sides are contiguous (ld == n), else a pitched copy.
int copy_matrix(void *dst, int64_t ldd, const void *src, int64_t lds, int64_t n, cudaMemcpyKind kind, cudaStream_t s) {
  void *host = kind == cudaMemcpyHostToDevice ? const_cast<void *>(src) : dst;
  void *mapped = nullptr;
  if (cudaHostGetDevicePointer(&mapped, host, 0) == cudaSuccess && mapped) {
    return kind == cudaMemcpyHostToDevice ? apsp::launch_copy2d(dst, ldd, mapped, lds, n, n, s)
                                          : apsp::launch_copy2d(mapped, ldd, src, lds, n, n, s);
  }
  cudaGetLastError();  // not pinned: no device address
  const cudaError_t e =
      (ldd == n && lds == n)
          ? cudaMemcpyAsync(dst, src, (size_t)n * (size_t)n * 4, kind, s)
          : cudaMemcpy2DAsync(dst, (size_t)ldd * 4, src, (size_t)lds * 4, (size_t)n * 4, (size_t)n, kind, s);
  return e == cudaSuccess ? APSP_OK : APSP_ERR_CUDA;
}

}  // namespace

extern "C" int apsp_solve_host(const void *h_in, void *h_out, int64_t n, int64_t ld_host, int dtype, int algo,
                               int param, const void *inf, void *d, int64_t ldd, void *ws, size_t ws_bytes,
                               void *stream) {
  using namespace apsp;
  if (!dtype_ok(dtype) || n < 0 || algo < 0 || algo > 2) return APSP_ERR_ARG;
  if (n == 0) return APSP_OK;
  if (!h_in || !h_out || ld_host < n) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void *own = nullptr;
  if (!d) {
    ldd = round_up(n, 4);
    if (ws_alloc(&own, (size_t)(n * ldd * 4), s) != APSP_OK) return APSP_ERR_NOMEM;
    d = own;
  } else if (ldd < n) {
    return APSP_ERR_ARG;
  }
  int r = copy_matrix(d, ldd, h_in, ld_host, n, cudaMemcpyHostToDevice, s);
  if (!r) {
    if (algo == 0) r = apsp_fw(d, n, ldd, dtype, inf, param, ws, ws_bytes, stream);
    else if (algo == 1) r = apsp_rkleene(d, n, ldd, dtype, inf, param, ws, ws_bytes, stream);
    else r = apsp_squaring(d, n, ldd, dtype, inf, param, ws, ws_bytes, stream);
  }
  if (!r) r = copy_matrix(h_out, ld_host, d, ldd, n, cudaMemcpyDeviceToHost, s);
  ws_free(own, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && !r) r = APSP_ERR_CUDA;
  return r;
}
