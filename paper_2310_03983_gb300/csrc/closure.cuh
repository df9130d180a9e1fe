// closure.cuh -- internal interfaces between the closure drivers (fw.cu, rkleene.cu).
#pragma once

#include "tgemm.cuh"

namespace apsp {

// Device bound words of a closure (see TileProblem::wmax): w[0] = largest finite weight,
// mult = n - 1 of the whole graph.  w == nullptr for float32.  cert (may be null: then w[0])
// is the largest finite entry of the block this closure starts from, the step bound of the
// truncated passes' certificates: an R-Kleene leaf starts from path lengths, not from edge
// weights, so its own scan gives it.
struct Bound {
  const int *w;
  int64_t mult;
  const int *cert = nullptr;
  // Three device words, zero at the start: the counters of phase 3's dynamic scheduling
  // (TileProblem::tile_counter; null: static order, and phases 1 and 2 in launches of their own).
  int *counters = nullptr;
};

// Blocked Floyd-Warshall on an aligned, normalised block (fw.cu).  panels16: scratch of
// fw16_panel_bytes(n) for the packed 16-bit phase 3 of int32 closures, or null.
int fw_closure(void *d, int64_t n, int64_t ld, int dtype, int inf_i, Bound b, cudaStream_t s,
               void *panels16 = nullptr);
size_t fw16_panel_bytes(int64_t n);
// Smallest n for which apsp_fw takes the packed 16-bit phase 3 (below it the extra launches
// of the certificate cost more than the faster arithmetic saves).
constexpr int64_t kFw16MinN = 4096;

// Scratch for (min,+) products on packed 16-bit pairs: a block of 8 words (maxima of the
// operands, the "packed" flag) and room for the packed copies of the largest product.
struct Packed16 {
  int *words;
  void *scratch;
  size_t bytes;
};

// R-Kleene on an aligned, normalised block, scratch of rkleene_scratch_bytes (rkleene.cu).
// pk.scratch (may be null): rk16_scratch_bytes(n, cutoff) for 16-bit products (int32).
int rkleene_closure(void *d, int64_t n, int64_t ld, int dtype, int inf_i, int cutoff, Bound b, void *scratch,
                    cudaStream_t s, Packed16 pk = {nullptr, nullptr, 0});
size_t rkleene_scratch_bytes(int64_t n, int cutoff);
size_t rk16_scratch_bytes(int64_t n, int cutoff);

// algo 0 = FW, 1 = R-Kleene; param = tile (FW) or cutoff (R-Kleene).
int closure_entry(int algo, void *d, int64_t n, int64_t ld, int dtype, const void *inf, int param, void *ws,
                  size_t ws_bytes, void *stream);
size_t closure_workspace_bytes(int algo, int64_t n, int64_t ld, int param, int dtype);
// The part closure_entry cannot run without (bound words, aligned copy, R-Kleene scratch); the
// rest of closure_workspace_bytes is the optional room for the packed 16-bit passes.
size_t closure_required_bytes(int algo, int64_t n, int64_t ld, int param);

// (min,+) product of aligned operands through the TMA engine (rkleene.cu).  With pk.scratch
// large enough, an int32 product whose largest finite operand entries sum below kCap16 (a
// device-side scan) runs on packed 16-bit pairs; the plain launch returns at once then.
// run_if (may be null): the launch returns at once unless *run_if is non-zero (then it is not
// traced and never takes the packed path).
int gemm_aligned(void *C, int64_t ldc, const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int64_t N,
                 int64_t K, int dtype, bool acc, int inf_i, Bound b, cudaStream_t s,
                 Packed16 pk = {nullptr, nullptr, 0}, const int *run_if = nullptr);

}  // namespace apsp
