// squaring.cu -- the paper's "Floyd-Warshall on GPU" (Sec. 3.2): apply the (min,+) product of
// Eq. 2 to the cost matrix and itself, D <- D (x) D, until nothing changes.
//
// With a zero diagonal, after t products D[i][j] is the shortest walk of at most 2^t edges, so
// ceil(log2(n - 1)) products always suffice (the paper bounds the loop by N, which is safe but
// loose); graphs of small diameter settle much sooner.  Every product runs on the TMA
// tropical-GEMM engine into a scratch matrix C; a commit kernel copies the entries that fell
// back into D and clears the iteration's "unchanged" word when any did.  The next product and
// commit read that word on the device and return at once when it is still set, so the whole
// loop is enqueued up front without a host round trip per iteration (and can be captured in
// a CUDA graph), yet stops doing work at convergence.
#include "closure.cuh"

namespace apsp {

namespace {

constexpr int kWordsUnchanged = 8;  // words[8 + t]: non-zero while product t changed nothing
constexpr int kMaxIters = 48;       // 8 + 48 words fit in the 256-byte bound-word block

__global__ void __launch_bounds__(256) commit_kernel(int *D, int64_t ldd, const int *C, int64_t ldc, int64_t n,
                                                     const int *skip, int *unchanged) {
  if (skip && *skip) return;
  bool changed = false;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    int *dr = D + i * ldd;
    const int *cr = C + i * ldc;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const int c = cr[j];
      if (c != dr[j]) {  // bit patterns: the product never exceeds D (D[j][j] = 0), so this is a fall
        dr[j] = c;
        changed = true;
      }
    }
  }
  if (__syncthreads_or(changed) && threadIdx.x == 0) *unchanged = 0;
}

int iters_for(int64_t n) {
  int t = 0;
  while (t < 62 && (int64_t(1) << t) < n - 1) ++t;
  return t;
}

}  // namespace

}  // namespace apsp

extern "C" size_t apsp_squaring_workspace_bytes(int64_t n, int64_t ld, int dtype) {
  using namespace apsp;
  (void)dtype;
  if (n <= 0) return 0;
  const size_t mat = (size_t)round_up(n * round_up(n, 4) * 4, 256);
  return kFlagBytes + mat + (ld % 4 != 0 ? mat : 0);
}

extern "C" int apsp_squaring(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int max_iters, void *ws,
                             size_t ws_bytes, void *stream) {
  using namespace apsp;
  if (!dtype_ok(dtype) || n < 0 || max_iters < 0) return APSP_ERR_ARG;
  if (n == 0) return APSP_OK;
  if (!d || ld < n || reinterpret_cast<uintptr_t>(d) % 16 != 0 || n > (int64_t)1 << 30) return APSP_ERR_ARG;
  int inf_i = 0;
  float inf_f = 0.f;
  if (dtype == APSP_I32 ? resolve_inf_i32(inf, &inf_i) : resolve_inf_f32(inf, &inf_f)) return APSP_ERR_ARG;
  const int iters = max_iters == 0 ? iters_for(n) : max_iters;
  if (iters > kMaxIters) return APSP_ERR_ARG;
  const size_t need = apsp_squaring_workspace_bytes(n, ld, dtype);
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
  int *words = reinterpret_cast<int *>(wsp);  // [0]: largest finite weight, [1]: 0, [8 + t]: unchanged flags
  wsp += kFlagBytes;
  const int64_t lde = round_up(n, 4);
  int *C = reinterpret_cast<int *>(wsp);
  wsp += round_up(n * lde * 4, 256);
  if (cudaMemsetAsync(words, 0, 16, s) != cudaSuccess) r = APSP_ERR_CUDA;
  if (!r && cudaMemsetAsync(words + kWordsUnchanged, 1, 4 * kMaxIters, s) != cudaSuccess) r = APSP_ERR_CUDA;
  void *work = d;
  int64_t ldw = ld;
  if (!r && ld % 4 != 0) {  // the engine needs 16-byte rows: work on an aligned copy
    ldw = lde;
    work = wsp;
    r = launch_copy2d(work, ldw, d, ld, n, n, s);
  }
  if (!r) r = launch_normalise(work, n, ldw, dtype, inf_i, inf_f, dtype == APSP_I32 ? words : nullptr, s);
  CUtensorMap mA, mB, mC;
  if (!r) r = make_operand_maps(work, n, n, ldw, dtype, &mA, &mB, nullptr);
  if (!r) r = make_operand_maps(C, n, n, lde, dtype, nullptr, nullptr, &mC);
  const int64_t cap = (int64_t)sm_count() * 8;
  for (int t = 0; t < iters && !r; ++t) {
    const int *skip = t > 0 ? words + kWordsUnchanged + t - 1 : nullptr;
    TileProblem p = {};
    p.M = n; p.N = n; p.K = n;
    p.tiles_m = cdiv(n, kBM);
    p.tiles_n = cdiv(n, kBN);
    p.ntiles = p.tiles_m * p.tiles_n;
    p.C = C;
    p.ldc = lde;
    p.inf_i = inf_i;
    p.inf_f = inf_f;
    p.status = status_word();
    p.wmax = dtype == APSP_I32 ? words : nullptr;  // every entry is a simple path: <= (n - 1) * wmax
    p.wmult = n - 1;
    p.skip = skip;
    r = launch_tgemm(kModeGemm, false, dtype, mA, mB, mC, p, s);
    if (!r) {
      commit_kernel<<<(int)(n < cap ? n : cap), 256, 0, s>>>(reinterpret_cast<int *>(work), ldw, C, lde, n, skip,
                                                             words + kWordsUnchanged + t);
      note_launch();
      if (cudaGetLastError() != cudaSuccess) r = APSP_ERR_CUDA;
    }
  }
  if (!r && work != d) r = launch_copy2d(d, ld, work, ldw, n, n, s);
  ws_free(own, s);
  return r;
}
