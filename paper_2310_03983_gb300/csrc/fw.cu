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
__global__ void __launch_bounds__(256) fw_diag_kernel(int *d, int64_t ld, int64_t n, int64_t kb, const int *run_if) {
  pdl_wait();
  pdl_trigger();
  if (run_if && !*run_if) return;
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

int launch_fw_diag(void *d, int64_t ld, int64_t n, int64_t kb, int dtype, cudaStream_t s, const int *run_if) {
  if (dtype == APSP_I32)
    launch_pdl(fw_diag_kernel<false>, 1, 256, 0, s, reinterpret_cast<int *>(d), ld, n, kb, run_if);
  else
    launch_pdl(fw_diag_kernel<true>, 1, 256, 0, s, reinterpret_cast<int *>(d), ld, n, kb, run_if);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

// ------------------------------------------------------------------------------------------
// Phase 3 on packed 16-bit pairs (int32 matrices).
//
// The closure is computed in the (min,+) semiring truncated at CAP = 0x3FFF: values at or above
// CAP all mean "at least CAP".  Truncation t(v) = min(v, CAP) is a homomorphism of (min,+) on
// [0, inf] (t(min(a, b)) = min(t(a), t(b)), t(a + b) = t(t(a) + t(b))), so a computation that
// mixes exact int32 steps (phases 1 and 2) with truncated ones (phase 3 on 16-bit pairs:
// operands capped at CAP, the result min(old entry, capped minimum)) keeps the invariant
// t(stored) = t(exact Floyd-Warshall value) for every entry.  Every stored value below CAP is
// therefore an exact distance of the pass, and at the end every pair whose distance is below
// CAP holds it exactly.  A pair with CAP <= distance < infinity would need a vertex on its
// shortest path whose distance lies in [CAP - w_max, CAP); so if the largest stored value below
// CAP plus the largest weight stays below CAP, no such pair exists: every entry at or above CAP
// is unreachable and becomes the sentinel, which gives the exact closure.  Otherwise (checked
// on the device) the same mapping leaves a matrix whose entries lie between the distances and
// the weights (every edge is below CAP), and the int32 Floyd-Warshall runs again over it.
//
// The same argument holds for a second cap, 2^24, with the fp32 instruction sequence on int32 bit
// patterns (ArithF32).  A pattern v < 2^24 read as fp32 is v * 2^-149; two such values add
// exactly while their sum stays below 2^24, and otherwise round to a value whose pattern is at
// least 2^24 (rounding is monotone, and every larger pattern is a larger float), so
// t(computed sum) = t(exact sum) with t(v) = min(v, 2^24), and min is exact.  An int32 closure
// whose weights are too large for the 16-bit pass and for the exact bound ((n - 1) w_max < 2^24)
// but at most 2^24 / 4 therefore runs phase 3 with that sequence (phases 1 and 2 stay exact), is
// certified in the same way, and only when the certificate fails runs the exact int32 pass.
//
// One pass does the work in every case: per block, phases 1 and 2 (exact), then one phase-3
// launch that runs on the packed 16-bit panels, or -- decided on the device -- its 32-bit
// alternative over the matrix's own panels (fp32 sequence when exact or truncated at 2^24,
// else int32).  Then one certificate for the cap in use, and the exact int32 pass, whose
// launches return at once unless that certificate failed.
// Words of the bound block used here:
//   [0] largest finite weight (a1), [4] 16-bit phase 3 in use, [5] largest stored value below
//   the cap in use, [6] the exact int32 pass must run, [7] phase 3 runs its 32-bit alternative,
//   [16] that alternative is truncated at 2^24.
constexpr int kUse16MaxWeight = kCap16 / 4;
constexpr int kCap24 = 1 << 24;
constexpr int kUse24MaxWeight = kCap24 / 4;
// From kFw16WideN vertices the 16-bit pass works on diagonal blocks of two tiles (256 vertices):
// phase 3 then has K = 256 (128 packed words) per launch, which halves the per-tile epilogue and
// C traffic per pair, at the price of a heavier phase 1 and 2 per block (a 2 x 2-tile closure,
// two panel copies and two panel products); below it the blocks are single tiles.
constexpr int kFw16Tiles = 2;
constexpr int64_t kFw16Block = kFw16Tiles * kBM;
constexpr int kFw16Words = (int)(kFw16Block / 2);
constexpr int64_t kFw16WideN = 16384;
// The plain loop (fp32, and int32 without the 16-bit pass) hands out phase-3 tiles dynamically
// and fuses phases 1 and 2 of the next block into each phase-3 launch up to this many blocks.
// Beyond it the static order with separate launches is faster: the fp32 instruction sequence is
// issue-bound, and the dynamic order's consumer loop costs it about 8% per launch (measured at
// n = 4096 .. 16384), which outweighs the saved launches once a launch has ~80 x 80 tiles
// (fp32: n = 8192 29.9 ms fused against 31.3 static; n = 12288 99.2 against 96.9).
constexpr int64_t kFusedMaxBlocks = 80;

// w = words[0]: the largest weight of the whole graph (the exact bound); c = *cert: the largest
// finite entry of the block being closed (the certificates' step bound).
__global__ void fw_decide_kernel(int *words, const int *cert, int may24, int64_t mult) {
  pdl_wait();
  pdl_trigger();
  const int w = words[0], c = *cert;
  const int use16 = c <= kUse16MaxWeight;
  words[4] = use16;
  words[5] = 0;
  words[6] = 0;
  words[7] = !use16;
  words[16] = !use16 && may24 && (int64_t)w * mult >= kCap24 && c <= kUse24MaxWeight;
}

// Packs the column panel D[:, kb0 .. kb0+bw) into A16 (n rows x lda16 words) and the row panel
// D[kb0 .. kb0+bw, :] into B16 (kFw16Words words x ldb16) as 16-bit pairs of consecutive k,
// every value capped at CAP (the sentinel included).
__global__ void __launch_bounds__(256) fw_pack16_kernel(const int *d, int64_t ld, int64_t n, int64_t kb0, int bw,
                                                        int *A16, int64_t lda16, int *B16, int64_t ldb16,
                                                        const int *words) {
  pdl_wait();
  pdl_trigger();
  if (!words[4]) return;
  const int kw = (bw + 1) >> 1;
  const int64_t na = n * kw, total = na + (int64_t)kw * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < na) {
      const int64_t i = e / kw;
      const int w = (int)(e - i * kw), k = 2 * w;
      const int *row = d + i * ld + kb0;
      const int lo = min(row[k], kCap16), hi = k + 1 < bw ? min(row[k + 1], kCap16) : kCap16;
      A16[i * lda16 + w] = (hi << 16) | lo;
    } else {
      const int64_t f = e - na;
      const int w = (int)(f / n);
      const int64_t j = f - (int64_t)w * n;
      const int k = 2 * w;
      const int *r0 = d + (kb0 + k) * ld + j;
      const int lo = min(r0[0], kCap16), hi = k + 1 < bw ? min(r0[ld], kCap16) : kCap16;
      B16[w * ldb16 + j] = (hi << 16) | lo;
    }
  }
}

// The cap of the truncated computation in use (0: none, the closure is exact).
__device__ __forceinline__ int cap_in_use(const int *words) {
  return words[4] ? kCap16 : (words[16] ? kCap24 : 0);
}

// words[5] = largest stored value below the cap in use, and every entry at or above it becomes
// the sentinel (nothing when the closure ran exact).
__global__ void __launch_bounds__(256) trunc_certify_kernel(int *d, int64_t ld, int64_t n, int inf, int *words) {
  pdl_wait();
  pdl_trigger();
  const int cap = cap_in_use(words);
  if (!cap) return;
  int m = 0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      int *e = d + i * ld + j;
      const int v = *e;
      if (v < cap) m = max(m, v);
      else if (v != inf) *e = inf;
    }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(words + 5, m);
}

// words[6] = 1 when the largest stored value below the cap plus the step bound *cert reaches the
// cap (the truncated result cannot be certified).
__global__ void trunc_verdict_kernel(int *words, const int *cert) {
  pdl_wait();
  pdl_trigger();
  const int cap = cap_in_use(words);
  words[6] = cap && (int64_t)words[5] + (int64_t)*cert >= cap;
}

static int certify(void *d, int64_t ld, int64_t n, int inf, int *words, const int *cert, cudaStream_t s) {
  const int64_t grid = std::min<int64_t>(n, (int64_t)sm_count() * 8);
  launch_pdl(trunc_certify_kernel, (int)grid, 256, 0, s, reinterpret_cast<int *>(d), ld, n, inf, words);
  APSP_LAUNCH_CHECK();
  launch_pdl(trunc_verdict_kernel, 1, 1, 0, s, words, cert);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

// Scratch of the 16-bit pass: the packed column and row panels, and copies of the int32 row and
// column panels (the operands of the in-place panel products).  Both packed panels are whole
// tiles long (round_up(n, 128) rows of the column panel, words per row of the row panel): the
// tiles store all 128 rows and columns of their register tile.
static int64_t fw16_ldb(int64_t n) { return round_up(n, kBN); }
size_t fw16_panel_bytes(int64_t n) {
  const int64_t ldp = round_up(n, 4);
  return (size_t)round_up(round_up(n, kBM) * kFw16Words * 4, 256) +
         (size_t)round_up(kFw16Words * fw16_ldb(n) * 4, 256) + (size_t)round_up(kFw16Block * ldp * 4, 256) +
         (size_t)round_up(n * kFw16Block * 4, 256);
}

// The plain three-phase loop; every launch returns at once unless *run_if (when given) is set.
// trace_class: added to the engine mode in trace records (kTraceSide for passes that
// normally return at once, and for the small sub-closures of the wide pass).
// counters (may be null): phase 3 hands out its tiles dynamically and performs phases 1 and 2
// of the next block itself (TileProblem::close_next), so the closure is phase 1 and 2 of block
// 0 and then one launch per block.
static int fw_loop(void *d, int64_t n, int64_t ld, int dtype, const CUtensorMap &mA, const CUtensorMap &mB,
                   const CUtensorMap &mC, TileProblem p, const int *run_if, cudaStream_t s, int trace_class = 0,
                   int *counters = nullptr) {
  int r;
  const int64_t nb = p.nb;
  p.run_if = run_if;
  p.trace_class = trace_class;
  for (int64_t kb = 0; kb < nb; ++kb) {
    if ((kb == 0 || !counters) && (r = launch_fw_diag(d, ld, n, kb, dtype, s, run_if))) return r;
    if (nb == 1) break;
    p.kb = kb;
    if (kb == 0 || !counters) {
      p.ntiles = 2 * (nb - 1);
      p.tile_counter = nullptr;
      p.close_next = 0;
      if ((r = launch_tgemm(kModeFwPanels, false, dtype, mA, mB, mC, p, s))) return r;
    }
    p.tile_counter = counters;
    p.close_next = counters && kb + 1 < nb;
    p.ntiles = (nb - 1) * (nb - 1) + (p.close_next ? 2 * (nb - 1) : 0);
    if ((r = launch_tgemm(kModeFwRest, true, dtype, mA, mB, mC, p, s))) return r;
  }
  return APSP_OK;
}

static int fw_wide_pass(void *d, int64_t n, int64_t ld, int dtype, int inf_i, Bound b, cudaStream_t s,
                        void *panels16, const TileProblem &p, const CUtensorMap &mA, const CUtensorMap &mB,
                        const CUtensorMap &mC);

// Phase 2 of a bw-vertex block at kb0 on packed 16-bit pairs (A16: the packed column panel, n
// rows x lda16 words; B16: the packed row panel, leading dimension ldb16; both written by
// fw_pack16_kernel from the panels before this phase, so each holds D* as well): the row panel
// D[kb0.., :] = min(itself, D* (x) row panel) and the column panel D[:, kb0..] = min(itself,
// column panel (x) D*), in the semiring truncated at kCap16 (a capped result means "at least
// the cap" and leaves the old entry).  Both launches return at once unless words[4] is set.
static int panels16_truncated(int *D, int64_t ld, int64_t n, int64_t kb0, int64_t bw, int *A16, int64_t lda16,
                              int *B16, int64_t ldb16, const TileProblem &base, int *words, cudaStream_t s) {
  int r;
  const int64_t kw = (bw + 1) >> 1;
  for (int side = 0; side < 2; ++side) {
    // side 0: the row panel (bw x n) = D* rows of A16 (x) B16; side 1: the column panel (n x bw)
    // = A16 (x) the D* columns of B16.
    const int64_t M = side ? n : bw, N = side ? bw : n;
    int *A = side ? A16 : A16 + kb0 * lda16;
    int *B = side ? B16 + kb0 : B16;
    int *C = side ? D + kb0 : D + kb0 * ld;
    CUtensorMap mA, mB, mC;
    if ((r = make_operand_maps(A, M, kw, lda16, APSP_I32, &mA, nullptr, nullptr))) return r;
    if ((r = make_operand_maps(B, kw, N, ldb16, APSP_I32, nullptr, &mB, nullptr))) return r;
    if ((r = make_operand_maps(C, M, N, ld, APSP_I32, nullptr, nullptr, &mC))) return r;
    TileProblem q = {};
    q.M = M; q.N = N; q.K = kw;
    q.tiles_m = cdiv(M, kBM);
    q.tiles_n = cdiv(N, kBN);
    q.ntiles = q.tiles_m * q.tiles_n;
    q.C = C;
    q.ldc = ld;
    q.inf_i = base.inf_i;
    q.status = base.status;
    q.arith16 = 1;
    q.run_if = words + 4;
    q.trace_class = kTraceSide;
    if ((r = launch_tgemm(kModeGemm, true, APSP_I32, mA, mB, mC, q, s))) return r;
  }
  return APSP_OK;
}

// Closes the n x n block at d (16-byte aligned, ld % 4 == 0, already normalised) in place.
// panels16 (may be null): fw16_panel_bytes(n) of device scratch; with it an int32 closure runs
// the pass above: phase 3 on packed 16-bit pairs when its largest weight (step) is at most
// CAP / 4, else its 32-bit alternative (truncated at 2^24 when allowed), then the certificate
// and the exact pass if needed.
int fw_closure(void *d, int64_t n, int64_t ld, int dtype, int inf_i, Bound b, cudaStream_t s, void *panels16) {
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
  if (!(panels16 && dtype == APSP_I32 && b.w && nb > 1 && inf_i > kCap16))
    return fw_loop(d, n, ld, dtype, mA, mB, mC, p, nullptr, s, 0, nb <= kFusedMaxBlocks ? b.counters : nullptr);
  int *words = const_cast<int *>(b.w);
  const int *cert = b.cert ? b.cert : b.w;
  launch_pdl(fw_decide_kernel, 1, 1, 0, s, words, cert, (int)(inf_i > kCap24), b.mult);
  APSP_LAUNCH_CHECK();
  if ((r = fw_wide_pass(d, n, ld, dtype, inf_i, b, s, panels16, p, mA, mB, mC))) return r;
  if ((r = certify(d, ld, n, inf_i, words, cert, s))) return r;
  return fw_loop(d, n, ld, dtype, mA, mB, mC, p, words + 6, s, kTraceSide,
                 nb <= kFusedMaxBlocks ? b.counters : nullptr);
}

// The pass over diagonal blocks of bt = 1 or 2 tiles: phases 1 and 2 exact, the block's panels
// packed (when words[4]), phase 3 on them or on the 32-bit alternative (words[7]).
static int fw_wide_pass(void *d, int64_t n, int64_t ld, int dtype, int inf_i, Bound b, cudaStream_t s,
                        void *panels16, const TileProblem &p, const CUtensorMap &mA, const CUtensorMap &mB,
                        const CUtensorMap &mC) {
  int r;
  int *words = const_cast<int *>(b.w);
  const int64_t ldp = round_up(n, 4);
  uint8_t *sp = reinterpret_cast<uint8_t *>(panels16);
  int *A16 = reinterpret_cast<int *>(sp);
  const int64_t arows = round_up(n, kBM);  // rows of one set of the packed column panel
  sp += round_up(arows * kFw16Words * 4, 256);
  int *B16 = reinterpret_cast<int *>(sp);
  const int64_t ldb16 = fw16_ldb(n);
  sp += round_up(kFw16Words * ldb16 * 4, 256);
  int *Rc = reinterpret_cast<int *>(sp);
  sp += round_up(kFw16Block * ldp * 4, 256);
  int *Cc = reinterpret_cast<int *>(sp);
  const int64_t cap = (int64_t)sm_count() * 8;
  const int64_t bt = n >= kFw16WideN ? kFw16Tiles : 1, blk = bt * kBM;
  // A16 rows hold the block's packed words: 64 for 128-vertex blocks (written by the panel tiles
  // themselves), kFw16Words for 256-vertex blocks (written by fw_pack16_kernel).
  // 128-vertex blocks: two sets of packed panels one below the other (set s of the column panel
  // at row s * arows of A16, 64 words per row; set s of the row panel at row 64 s of B16),
  // written by the panel tiles themselves and by the tiles of the next block row and column (no
  // packing pass).  256-vertex blocks: one set, 128 words per row, written by fw_pack16_kernel.
  const int64_t lda16 = bt == 1 ? kBM / 2 : kFw16Words;
  CUtensorMap pA, pB;
  if ((r = make_operand_maps(A16, bt == 1 ? 2 * arows : n, lda16, lda16, APSP_I32, &pA, nullptr, nullptr))) return r;
  if ((r = make_operand_maps(B16, kFw16Words, n, ldb16, APSP_I32, nullptr, &pB, nullptr))) return r;
  const int64_t nbb = cdiv(n, blk), nt = cdiv(n, kBM);
  int *D = reinterpret_cast<int *>(d);
  for (int64_t kbb = 0; kbb < nbb; ++kbb) {
    const int64_t kb0 = kbb * blk, bw = std::min<int64_t>(blk, n - kb0);
    int *sub = D + kb0 * ld + kb0, *rowp = D + kb0 * ld, *colp = D + kb0;
    if (bt == 1) {  // phases 1 and 2 of a single-tile block, in place (as in the plain loop); with
                    // counters, those of every block after the first ran in the previous phase 3
      if ((kbb == 0 || !b.counters) && (r = launch_fw_diag(d, ld, n, kbb, dtype, s, nullptr))) return r;
      if (kbb == 0 || !b.counters) {
        TileProblem pp = p;
        pp.kb = kbb;
        pp.ntiles = 2 * (nt - 1);
        pp.trace_class = kTraceSide;
        pp.pk_a[0] = A16;
        pp.pk_a[1] = A16 + arows * lda16;
        pp.pk_b[0] = B16;
        pp.pk_b[1] = B16 + (kBM / 2) * ldb16;
        pp.pk_ldb = ldb16;
        if ((r = launch_tgemm(kModeFwPanels, false, dtype, mA, mB, mC, pp, s))) return r;
      }
    } else {
      // Phase 1: close the diagonal block (itself a small blocked Floyd-Warshall, exact), with
      // the next tile's phases 1 and 2 inside each phase-3 launch when the counters are there
      // (four launches for a two-tile block instead of six).
      CUtensorMap dA, dB, dC;
      if ((r = make_operand_maps(sub, bw, bw, ld, dtype, &dA, &dB, &dC))) return r;
      TileProblem ps = p;
      ps.n = bw;
      ps.nb = cdiv(bw, kBM);
      ps.C = sub;
      if ((r = fw_loop(sub, bw, ld, dtype, dA, dB, dC, ps, nullptr, s, kTraceSide, b.counters))) return r;
      // Phase 2: the row panel becomes D* (x) (row panel) and the column panel (column panel) (x)
      // D*; D* is closed, so its zero diagonal keeps the old entry and the block's own entries
      // are reproduced (D* (x) D* = D*).  With the 16-bit pass in use (words[4]) both products
      // run truncated on packed copies of the panels -- which hold D* in both forms -- in place,
      // folded as min(old entry, capped product) like phase 3.  In the 32-bit alternative
      // (words[7]) each is one exact product read from an int32 copy of its panel.
      const int64_t work = 2 * n * ((bw + 1) >> 1);
      launch_pdl(fw_pack16_kernel, (int)std::min<int64_t>(cap, cdiv(work, 256)), 256, 0, s, D, ld, n, kb0, (int)bw,
                 A16, lda16, B16, ldb16, words);
      APSP_LAUNCH_CHECK();
      if ((r = panels16_truncated(D, ld, n, kb0, bw, A16, lda16, B16, ldb16, p, words, s))) return r;
      const int *alt = words + 7;
      if ((r = launch_copy2d(Rc, ldp, rowp, ld, bw, n, s, alt))) return r;
      if ((r = gemm_aligned(rowp, ld, sub, ld, Rc, ldp, bw, n, bw, dtype, false, inf_i, b, s, {}, alt))) return r;
      if ((r = launch_copy2d(Cc, kFw16Block, colp, ld, n, bw, s, alt))) return r;
      if ((r = gemm_aligned(colp, ld, Cc, kFw16Block, sub, ld, n, bw, bw, dtype, false, inf_i, b, s, {}, alt)))
        return r;
    }
    // Phase 3, K = bw: on the packed panels, or the 32-bit alternative.
    if (bt > 1) {
      const int64_t work = 2 * n * ((bw + 1) >> 1);
      launch_pdl(fw_pack16_kernel, (int)std::min<int64_t>(cap, cdiv(work, 256)), 256, 0, s, D, ld, n, kb0, (int)bw,
                 A16, lda16, B16, ldb16, words);
      APSP_LAUNCH_CHECK();
    }
    const int64_t ec = std::min<int64_t>(bt, nt - kbb * bt), rest = nt - ec;
    if (rest == 0) continue;
    TileProblem q = p;
    q.kb = kbb;
    q.bt = (int)bt;
    q.ntiles = rest * rest;
    q.arith16 = 1;
    q.alt_if = words + 7;
    q.f32_if = words + 16;
    q.no_trace = 1;
    double pairs = (double)(n - bw) * (double)(n - bw) * (double)bw;
    if (bt == 1) {
      q.pk_a[0] = A16;
      q.pk_a[1] = A16 + arows * lda16;
      q.pk_b[0] = B16;
      q.pk_b[1] = B16 + (kBM / 2) * ldb16;
      q.pk_ldb = ldb16;
      q.pk_arows = arows;
      q.tile_counter = b.counters;
      q.close_next = b.counters && kbb + 1 < nbb;
      if (q.close_next) {  // and phase 2 of the next block
        const double bw1 = (double)std::min<int64_t>(kBM, n - (kbb + 1) * kBM);
        q.ntiles += 2 * rest;
        pairs += 2.0 * bw1 * bw1 * ((double)n - bw1);
      }
    }
    void *tev = nullptr;
    if (trace_on()) trace_begin(s, &tev);
    if ((r = launch_tgemm(kModeFwRest16, true, dtype, pA, pB, mC, q, s, &mA, &mB))) return r;
    if (tev) trace_end(s, tev, kModeFwRest, pairs);
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
  // The full size includes the packed 16-bit panels of an int32 FW; a workspace of the base
  // size is still accepted and closes with the plain phase 3.
  const size_t need = closure_workspace_bytes(algo, n, ld, param, dtype);
  const size_t base = closure_required_bytes(algo, n, ld, param);
  const size_t panels = need - base;
  if (ws && (ws_bytes < base || reinterpret_cast<uintptr_t>(ws) % 256 != 0)) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void *own = nullptr;
  if (!ws && need > 0) {
    if (ws_alloc(&own, need, s) != APSP_OK) {
      return APSP_ERR_NOMEM;
    }
    ws = own;
    ws_bytes = need;
  }
  void *panels16 = (panels && ws_bytes >= need) ? reinterpret_cast<uint8_t *>(ws) + base : nullptr;
  int r = APSP_OK;
  uint8_t *wsp = reinterpret_cast<uint8_t *>(ws);
  int *words = reinterpret_cast<int *>(wsp);  // [0]: largest finite weight, [1]: 0
  wsp += kFlagBytes;
  if (cudaMemsetAsync(words, 0, kFlagBytes, s) != cudaSuccess) r = APSP_ERR_CUDA;
  Bound bound = {dtype == APSP_I32 ? words : nullptr, n - 1};
  bound.counters = words + 40;  // three words, zeroed with the rest of the block
  void *work = d;
  int64_t ldw = ld;
  if (ld % 4 != 0) {  // repack into an aligned copy at the front of the workspace
    ldw = round_up(n, 4);
    work = wsp;
    wsp += round_up(n * ldw * 4, 256);
    if (!r) r = launch_copy2d(work, ldw, d, ld, n, n, s);
  }
  if (!r) r = launch_normalise(work, n, ldw, dtype, inf_i, inf_f, dtype == APSP_I32 ? words : nullptr, s);
  const Packed16 pk = {words + 8, panels16, panels16 ? panels : 0};
  if (!r) r = algo == 0 ? fw_closure(work, n, ldw, dtype, inf_i, bound, s, panels16)
                        : rkleene_closure(work, n, ldw, dtype, inf_i, param ? param : 256, bound, wsp, s, pk);
  if (!r && work != d) r = launch_copy2d(d, ld, work, ldw, n, n, s);
  ws_free(own, s);
  return r;
}

size_t closure_required_bytes(int algo, int64_t n, int64_t ld, int param) {
  if (n <= 0) return 0;
  size_t b = kFlagBytes;
  if (ld % 4 != 0) b += (size_t)round_up(n * round_up(n, 4) * 4, 256);
  if (algo == 1) b += rkleene_scratch_bytes(n, param ? param : 256);
  return b;
}

size_t closure_workspace_bytes(int algo, int64_t n, int64_t ld, int param, int dtype) {
  if (n <= 0) return 0;
  size_t b = closure_required_bytes(algo, n, ld, param);
  // Last, and optional: room for the packed 16-bit panels (FW) or operands (R-Kleene).
  if (algo == 0 && dtype == APSP_I32 && n >= kFw16MinN) b += fw16_panel_bytes(n);
  if (algo == 1 && dtype == APSP_I32) b += rk16_scratch_bytes(n, param ? param : 256);
  return b;
}

}  // namespace apsp

extern "C" size_t apsp_fw_workspace_bytes(int64_t n, int64_t ld, int dtype, int tile) {
  (void)tile;
  return apsp::closure_workspace_bytes(0, n, ld, 0, dtype);
}

extern "C" int apsp_fw(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int tile, void *ws,
                       size_t ws_bytes, void *stream) {
  return apsp::closure_entry(0, d, n, ld, dtype, inf, tile, ws, ws_bytes, stream);
}
