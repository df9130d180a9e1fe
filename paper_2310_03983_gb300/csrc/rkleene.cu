// rkleene.cu -- a6: R-Kleene closure (Sec. 3.3, Eq. 4).
//
// The matrix is split as H = [[A, B], [C, D]] (A: first h vertices, D: the rest) and closed by
//     A = A*;  B = A (x) B;  C = C (x) A;  D = min(D, C (x) B);
//     D = D*;  B = B (x) D;  C = D (x) C;  A = min(A, B (x) C)
// recursing on A and D until a block has at most `cutoff` vertices, which blocked
// Floyd-Warshall closes.  The split h is ceil(m/2) rounded up to a multiple of 128, so every
// block starts on a TMA-aligned boundary.  Products whose output is also an operand
// (B = A (x) B, C = C (x) A, B = B (x) D, C = D (x) C) first copy that operand to scratch, so
// no CTA reads a tile another CTA is writing; the closed factor has a zero diagonal, so the
// plain product already includes the old entry and needs no extra min.
#include "closure.cuh"

namespace apsp {

static int64_t split_of(int64_t m) { return round_up(cdiv(m, 2), kBM); }

size_t rkleene_scratch_bytes(int64_t n, int cutoff) {
  if (n <= cutoff) return 0;
  const int64_t h = split_of(n);
  return (size_t)round_up(h * round_up(h, 4) * 4, 256);
}

// Packed copies of an M x K A and a K x N B (words, 16-byte aligned rows).
static size_t packed_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t kw = (K + 1) >> 1;
  return (size_t)round_up(M * round_up(kw, 4) * 4, 256) + (size_t)round_up(kw * round_up(N, 4) * 4, 256);
}

// Products smaller than this many pairs keep the plain path: the scan and packing launches
// would cost more than the faster arithmetic saves.
constexpr double kPacked16MinPairs = 1.0e9;

int gemm_aligned(void *C, int64_t ldc, const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int64_t N,
                 int64_t K, int dtype, bool acc, int inf_i, Bound b, cudaStream_t s, Packed16 pk,
                 const int *run_if) {
  if (M == 0 || N == 0) return APSP_OK;
  CUtensorMap mA, mB, mC;
  int r;
  if ((r = make_operand_maps(A, M, K, lda, dtype, &mA, nullptr, nullptr))) return r;
  if ((r = make_operand_maps(B, K, N, ldb, dtype, nullptr, &mB, nullptr))) return r;
  if ((r = make_operand_maps(C, M, N, ldc, dtype, nullptr, nullptr, &mC))) return r;
  TileProblem p = {};
  p.M = M; p.N = N; p.K = K;
  p.tiles_m = cdiv(M, kBM);
  p.tiles_n = cdiv(N, kBN);
  p.ntiles = p.tiles_m * p.tiles_n;
  p.C = C;
  p.ldc = ldc;
  p.inf_i = inf_i;
  p.status = status_word();
  p.wmax = b.w;
  p.wmult = b.mult;
  p.run_if = run_if;
  p.no_trace = run_if != nullptr;
  const bool packed = !run_if && dtype == APSP_I32 && pk.scratch && K > 0 && pk.bytes >= packed_bytes(M, N, K) &&
                      (double)M * (double)N * (double)K >= kPacked16MinPairs;
  if (!packed) return launch_tgemm(kModeGemm, acc, dtype, mA, mB, mC, p, s);
  // words[0], words[1]: largest finite entries of A and B; words[4]: set by the pack kernels
  // when their sum is below kCap16 (then every finite sum is exact in 16 bits).
  int *w = pk.words;
  const int64_t kw = (K + 1) >> 1, lda16 = round_up(kw, 4), ldb16 = round_up(N, 4);
  int *A16 = reinterpret_cast<int *>(pk.scratch);
  int *B16 = reinterpret_cast<int *>(reinterpret_cast<uint8_t *>(pk.scratch) + round_up(M * lda16 * 4, 256));
  if (cudaMemsetAsync(w, 0, 32, s) != cudaSuccess) return APSP_ERR_CUDA;
  if ((r = launch_scan_max(A, M, K, lda, inf_i, w, s))) return r;
  if ((r = launch_scan_max(B, K, N, ldb, inf_i, w + 1, s))) return r;
  if ((r = launch_pack16_a(reinterpret_cast<const int *>(A), lda, M, K, A16, lda16, inf_i, w, s))) return r;
  if ((r = launch_pack16_b(reinterpret_cast<const int *>(B), ldb, K, N, B16, ldb16, inf_i, w, s))) return r;
  CUtensorMap pA, pB;
  if ((r = make_operand_maps(A16, M, kw, lda16, APSP_I32, &pA, nullptr, nullptr))) return r;
  if ((r = make_operand_maps(B16, kw, N, ldb16, APSP_I32, nullptr, &pB, nullptr))) return r;
  void *tev = nullptr;
  if (trace_on()) trace_begin(s, &tev);
  TileProblem q = p;
  q.K = kw;
  q.arith16 = 1;
  q.run_if = w + 4;
  q.no_trace = 1;
  if ((r = launch_tgemm(kModeGemm, acc, dtype, pA, pB, mC, q, s))) return r;
  p.skip = w + 4;
  p.no_trace = 1;
  if ((r = launch_tgemm(kModeGemm, acc, dtype, mA, mB, mC, p, s))) return r;
  if (tev) trace_end(s, tev, kModeGemm, (double)M * (double)N * (double)K);
  return APSP_OK;
}

static int rk(uint8_t *d, int64_t m, int64_t ld, int dtype, int inf_i, int cutoff, Bound bd, uint8_t *W,
              cudaStream_t s, Packed16 pk) {
  // Leaves of at least kFw16MinN vertices close with the packed 16-bit phase 3, or, when too
  // heavy for it and for the exact fp32 bound, with phase 3 truncated at 2^24 (each certified per
  // leaf: a leaf's closure is the closure of the graph its block describes).  A leaf's block holds
  // path lengths through the vertices closed before it, so the certificates' step bound is the
  // block's own largest finite entry, scanned into words[32], not the largest edge weight.  The
  // leaves reuse the product scratch, which is idle while a leaf runs.
  if (m <= cutoff) {
    void *p16 = (m >= kFw16MinN && pk.scratch && pk.bytes >= fw16_panel_bytes(m)) ? pk.scratch : nullptr;
    Bound lb = bd;
    if (dtype == APSP_I32 && bd.w && p16) {
      int *lw = const_cast<int *>(bd.w) + 32;
      if (cudaMemsetAsync(lw, 0, sizeof(int), s) != cudaSuccess) return APSP_ERR_CUDA;
      int r;
      if ((r = launch_scan_max(d, m, m, ld, inf_i, lw, s))) return r;
      lb.cert = lw;
    }
    return fw_closure(d, m, ld, dtype, inf_i, lb, s, p16);
  }
  const int64_t h = split_of(m), r2 = m - h;
  const int64_t es = 4;
  uint8_t *A = d, *B = d + h * es, *C = d + h * ld * es, *D = d + (h * ld + h) * es;
  int r;
  // First half closed; paths through it update B, C, D.
  if ((r = rk(A, h, ld, dtype, inf_i, cutoff, bd, W, s, pk))) return r;
  int64_t ldw = round_up(r2, 4);
  if ((r = launch_copy2d(W, ldw, B, ld, h, r2, s))) return r;                                     // W = B
  if ((r = gemm_aligned(B, ld, A, ld, W, ldw, h, r2, h, dtype, false, inf_i, bd, s, pk))) return r;      // B = A (x) B
  ldw = round_up(h, 4);
  if ((r = launch_copy2d(W, ldw, C, ld, r2, h, s))) return r;                                     // W = C
  if ((r = gemm_aligned(C, ld, W, ldw, A, ld, r2, h, h, dtype, false, inf_i, bd, s, pk))) return r;      // C = C (x) A
  if ((r = gemm_aligned(D, ld, C, ld, B, ld, r2, r2, h, dtype, true, inf_i, bd, s, pk))) return r;       // D = min(D, C (x) B)
  // Second half closed; paths through it update B, C, A.
  if ((r = rk(D, r2, ld, dtype, inf_i, cutoff, bd, W, s, pk))) return r;
  ldw = round_up(r2, 4);
  if ((r = launch_copy2d(W, ldw, B, ld, h, r2, s))) return r;                                     // W = B
  if ((r = gemm_aligned(B, ld, W, ldw, D, ld, h, r2, r2, dtype, false, inf_i, bd, s, pk))) return r;     // B = B (x) D
  ldw = round_up(h, 4);
  if ((r = launch_copy2d(W, ldw, C, ld, r2, h, s))) return r;                                     // W = C
  if ((r = gemm_aligned(C, ld, D, ld, W, ldw, r2, h, r2, dtype, false, inf_i, bd, s, pk))) return r;     // C = D (x) C
  return gemm_aligned(A, ld, B, ld, C, ld, h, h, r2, dtype, true, inf_i, bd, s, pk);                     // A = min(A, B (x) C)
}

int rkleene_closure(void *d, int64_t n, int64_t ld, int dtype, int inf_i, int cutoff, Bound b, void *scratch,
                    cudaStream_t s, Packed16 pk) {
  return rk(reinterpret_cast<uint8_t *>(d), n, ld, dtype, inf_i, cutoff, b, reinterpret_cast<uint8_t *>(scratch), s,
            pk);
}

// The largest product of the recursion is the top level's, h x h by h (h = split_of(n)).
size_t rk16_scratch_bytes(int64_t n, int cutoff) {
  if (n <= cutoff) return 0;
  const int64_t h = split_of(n);
  return packed_bytes(h, h, h);
}

}  // namespace apsp

extern "C" size_t apsp_rkleene_workspace_bytes(int64_t n, int64_t ld, int dtype, int cutoff) {
  return apsp::closure_workspace_bytes(1, n, ld, cutoff, dtype);
}

extern "C" int apsp_rkleene(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int cutoff, void *ws,
                            size_t ws_bytes, void *stream) {
  return apsp::closure_entry(1, d, n, ld, dtype, inf, cutoff, ws, ws_bytes, stream);
}
