// fw.cu -- a3-a5: blocked Floyd-Warshall over 128 x 128 tiles.
//
// Eq. 1 (Sec. 2) relaxes every pair through intermediate vertex k, for k = 0..n-1.  Grouping
// the k's by 128-vertex blocks kb gives the classic three phases per block:
//   phase 1  close the diagonal tile (kb, kb) by Eq. 1 restricted to its own vertices;
//   phase 2  row panel    D[kb][j] = D[kb][kb]* (x) D[kb][j]   (j != kb)
//            column panel D[i][kb] = D[i][kb] (x) D[kb][kb]*   (i != kb)
//            one (min,+) product each is exact because the closed tile has a zero diagonal,
//            so the product already contains the old entry (k = i or k = j term);
//   phase 3  D[i][j] = min(D[i][j], D[i][kb] (x) D[kb][j])      (i, j != kb)
//            -- the rank-128 (min,+) update that carries essentially all n^3 of the work.
// Phases 2 and 3 run on the TMA-fed tropical GEMM engine (tgemm.cu); phase 1 is one CTA.
#include <algorithm>

#include "closure.cuh"
#include "diag.cuh"

namespace apsp {

// Phase 1: Eq. 1 on the bk x bk diagonal tile, closed in registers by one 256-thread CTA
// (diag.cuh).  int32 tiles are relaxed in int32 (exact for any weights), float32 in fp32.
template <bool FLOAT>
__global__ void __launch_bounds__(256) fw_diag_kernel(int *d, int64_t ld, int64_t n, int64_t kb) {
  __shared__ __align__(16) int buf[512];
  const int64_t kb0 = kb * kBM;
  const int bk = (int)std::min<int64_t>(kBM, n - kb0);
  int *T = d + kb0 * ld + kb0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (warp & 3) * 4 + (lane >> 3), tn = (warp >> 2) * 8 + (lane & 7);
  int r[8][8];
  load_tile_regs(r, T, ld, bk, tm, tn);
  close_tile_regs<FLOAT>(r, bk, tm, tn, buf);
  store_tile_regs(r, T, ld, bk, tm, tn);
}

int launch_fw_diag(void *d, int64_t ld, int64_t n, int64_t kb, int dtype, cudaStream_t s) {
  if (dtype == APSP_I32)
    fw_diag_kernel<false><<<1, 256, 0, s>>>(reinterpret_cast<int *>(d), ld, n, kb);
  else
    fw_diag_kernel<true><<<1, 256, 0, s>>>(reinterpret_cast<int *>(d), ld, n, kb);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

// Closes the n x n block at d (16-byte aligned, ld % 4 == 0, already normalised) in place.
int fw_closure(void *d, int64_t n, int64_t ld, int dtype, int inf_i, Bound b, cudaStream_t s) {
  if (n == 0) return APSP_OK;
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
  p.wmax = b.w;
  p.wmult = b.mult;
  for (int64_t kb = 0; kb < nb; ++kb) {
    if ((r = launch_fw_diag(d, ld, n, kb, dtype, s))) return r;
    if (nb == 1) break;
    p.kb = kb;
    p.ntiles = 2 * (nb - 1);
    if ((r = launch_tgemm(kModeFwPanels, false, dtype, mA, mB, mC, p, s))) return r;
    p.ntiles = (nb - 1) * (nb - 1);
    if ((r = launch_tgemm(kModeFwRest, true, dtype, mA, mB, mC, p, s))) return r;
  }
  return APSP_OK;
}

// Shared entry logic of apsp_fw and apsp_rkleene: validation, the workspace (caller's or
// stream-ordered allocation), repacking when ld breaks 16-byte row alignment, a1, closure.
int closure_entry(int algo, void *d, int64_t n, int64_t ld, int dtype, const void *inf, int param, void *ws,
                  size_t ws_bytes, void *stream) {
  if (!dtype_ok(dtype) || n < 0) return APSP_ERR_ARG;
  if (n == 0) return APSP_OK;
  if (!d || ld < n || reinterpret_cast<uintptr_t>(d) % 16 != 0) return APSP_ERR_ARG;
  if (n > (int64_t)1 << 30) return APSP_ERR_ARG;
  if (algo == 0 && param != 0 && param != kBM) return APSP_ERR_ARG;
  if (algo == 1 && param != 0 && param < kBM) return APSP_ERR_ARG;
  int inf_i = 0;
  float inf_f = 0.f;
  if (dtype == APSP_I32 ? resolve_inf_i32(inf, &inf_i) : resolve_inf_f32(inf, &inf_f)) return APSP_ERR_ARG;
  const size_t need = closure_workspace_bytes(algo, n, ld, param);
  if (ws && (ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0)) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void *own = nullptr;
  if (!ws && need > 0) {
    if (cudaMallocAsync(&own, need, s) != cudaSuccess) {
      cudaGetLastError();
      return APSP_ERR_NOMEM;
    }
    ws = own;
  }
  int r = APSP_OK;
  uint8_t *wsp = reinterpret_cast<uint8_t *>(ws);
  int *words = reinterpret_cast<int *>(wsp);  // [0]: largest finite weight, [1]: 0
  wsp += kFlagBytes;
  if (cudaMemsetAsync(words, 0, 16, s) != cudaSuccess) r = APSP_ERR_CUDA;
  const Bound bound = {dtype == APSP_I32 ? words : nullptr, n - 1};
  void *work = d;
  int64_t ldw = ld;
  if (ld % 4 != 0) {  // repack into an aligned copy at the front of the workspace
    ldw = round_up(n, 4);
    work = wsp;
    wsp += round_up(n * ldw * 4, 256);
    if (!r) r = launch_copy2d(work, ldw, d, ld, n, n, s);
  }
  if (!r) r = launch_normalise(work, n, ldw, dtype, inf_i, inf_f, dtype == APSP_I32 ? words : nullptr, s);
  if (!r) r = algo == 0 ? fw_closure(work, n, ldw, dtype, inf_i, bound, s)
                        : rkleene_closure(work, n, ldw, dtype, inf_i, param ? param : 256, bound, wsp, s);
  if (!r && work != d) r = launch_copy2d(d, ld, work, ldw, n, n, s);
  if (own) cudaFreeAsync(own, s);
  return r;
}

size_t closure_workspace_bytes(int algo, int64_t n, int64_t ld, int param) {
  if (n <= 0) return 0;
  size_t b = kFlagBytes;
  if (ld % 4 != 0) b += (size_t)round_up(n * round_up(n, 4) * 4, 256);
  if (algo == 1) b += rkleene_scratch_bytes(n, param ? param : 256);
  return b;
}

}  // namespace apsp

extern "C" size_t apsp_fw_workspace_bytes(int64_t n, int64_t ld, int dtype, int tile) {
  (void)dtype; (void)tile;
  return apsp::closure_workspace_bytes(0, n, ld, 0);
}

extern "C" int apsp_fw(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int tile, void *ws,
                       size_t ws_bytes, void *stream) {
  return apsp::closure_entry(0, d, n, ld, dtype, inf, tile, ws, ws_bytes, stream);
}
