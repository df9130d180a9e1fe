// tgemm.cuh -- the register-tiled (min,+) "tropical GEMM" engine shared by the standalone
// product (Eq. 2), blocked Floyd-Warshall phases 2 and 3, and R-Kleene.
#pragma once

#include "common.cuh"

namespace apsp {

// CTA tile and pipeline shape.
constexpr int kBM = 128, kBN = 128, kBK = 32, kStages = 4;
constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 4) * 32;  // 2 consumer warpgroups + 1 producer warpgroup
// Register split (setmaxnreg): the launch gives every thread kLaunchRegs; the producer
// warpgroup gives back down to kProducerRegs so the consumers can grow to kConsumerRegs.
// 128 * kProducerRegs + 256 * kConsumerRegs must not exceed 384 * kLaunchRegs.
constexpr int kLaunchRegs = 168, kProducerRegs = 40, kConsumerRegs = 232;
static_assert(128 * kProducerRegs + 256 * kConsumerRegs <= kThreads * kLaunchRegs, "register split");
constexpr int kAStageBytes = kBM * kBK * 4;         // A tile [128 m][32 k]
constexpr int kBStageBytes = kBK * kBN * 4;         // B tile [32 k][128 n]
constexpr int kCBytes = kBM * kBN * 4;              // C tile [128 m][128 n]
// Shared memory: the stage ring, the C tile, 256 bytes of mbarriers and the tile-index ring, and
// 2 KB of row / column buffers for the in-kernel diagonal closure (close_next).
constexpr int kDiagBufBytes = 512 * 4;
constexpr int kSmemBytes = kStages * (kAStageBytes + kBStageBytes) + kCBytes + 256 + kDiagBufBytes;

// Which tiles a launch visits and where their operands live.
enum TileMode : int {
  kModeGemm = 0,      // C (M x N) = [min(C,)] A (M x K) (x) B (K x N)
  kModeFwPanels = 1,  // blocked-FW phase 2: row and column panels of block kb
  kModeFwRest = 2,    // blocked-FW phase 3: every tile outside block row/column kb
  kModeFwRest16 = 3,  // phase 3 on packed 16-bit copies of the panels of a block of bt tiles:
                      // A = the column panel (n rows x 64 bt words), B = the row panel
                      // (64 bt words x n), C = the matrix; tiles of the block row/column skipped
};

// Grouped FW (the batched closure of many graphs in lockstep): graphs staged one below the
// other in one tall matrix, each padded to nb whole tiles with isolated vertices.  A group
// holds `count` graphs of the same nb, the first at staged index `first` and row `row0`; graph
// first + q starts at row row0 + q * nb * 128.  Groups are listed by decreasing nb.
constexpr int kMaxGroups = 14;
struct GraphGroup {
  int64_t row0;
  int first, count, nb, pad;
};

struct TileProblem {
  int64_t M, N, K;       // GEMM extents (kModeGemm)
  int64_t tiles_m, tiles_n;
  int64_t n;             // FW: matrix order
  int64_t kb, nb;        // FW: current diagonal block and number of blocks (block = 128)
  void *C;               // output base (GEMM: C; FW: the matrix)
  int64_t ldc;
  int64_t ntiles;
  int inf_i;
  float inf_f;
  unsigned int *status;
  // Bound words for int32 storage (device, may be null): the exact fp32 path is taken when
  // wmax[0] * wmult + wmax[1] < 2^24 (closures: max finite weight times n-1; products: the
  // largest finite entries of A and B).
  const int *wmax;
  int64_t wmult;
  // Optional device words (may be null), read before any barrier exists: every CTA returns at
  // once when *skip is non-zero, or when *run_if is zero.  They let a launch sequence that was
  // enqueued up front choose between alternative launches on the device.
  const int *skip;
  const int *run_if;
  // int32 storage only: the operands are packed 16-bit pairs (ArithI16x2) -- A words
  // {A[i][2w], A[i][2w+1]}, B words {B[2w][j], B[2w+1][j]}, K counted in words -- and C holds
  // plain int32.
  int arith16;
  // Not traced by itself: the caller brackets a group of alternative launches with one
  // trace record (only one of them does the work).
  int no_trace;
  // int32 signed closures (may be 0 = off): a result at or above sat is an unreachable entry
  // plus negative terms and is written back as exactly inf_i.
  int sat;
  // kModeFwRest16: tiles per diagonal block (0 or 1: 128-vertex blocks; 2: 256-vertex blocks).
  int bt;
  // Grouped FW (modes 1, 2 and 3 with bt = 1; ngroups = 0: one matrix).  The launch visits the
  // phase's tiles of every graph with nb > kb, group by group; a graph's tiles are skipped
  // unless (gflags[staged index] & gmask) == gwant.  In mode 3, and in mode 1 with arith16, A
  // is the packed column panels (the staged rows x 64 words) and B the packed row panels (64
  // rows per staged graph); results are folded as truncated closures (capped at kCap16).
  int ngroups;
  GraphGroup groups[kMaxGroups];
  const int *gflags;
  int gmask, gwant;
  // Grouped 16-bit launches (may be null): packed outputs.  Set s of the packed operands is
  // pk_a[s] (64 words per staged row, pairs of consecutive columns, capped at kCap16) and
  // pk_b[s] (leading dimension ldc, 64 rows per staged graph, pairs of consecutive rows); block
  // step kb reads set kb & 1.  A panel tile (mode 1) writes its result into set kb & 1 as phase
  // 3's operand (over the packed words it has itself finished reading); a tile in block row or
  // column kb + 1 (modes 1 and 3) writes it into set (kb + 1) & 1 as the next step's operand.
  int *pk_a[2], *pk_b[2];
  // Single matrix (kModeFwPanels, and kModeFwRest16 with close_next; pk_a[0] set): packed
  // copies in the same two sets -- set s of the column panel is pk_a[s] (64 words per row, pairs
  // of consecutive columns), set s of the row panel pk_b[s] (leading dimension pk_ldb, pairs of
  // consecutive rows); block step kb reads set kb & 1.  Panel tiles (mode 1) write their result
  // into set kb & 1 as phase 3's operand, and tiles of block row / column kb + 1 also into set
  // (kb + 1) & 1 (close_next above).  In kModeFwRest16 the sets sit one below the other in the
  // operand maps: set s of A starts at row s * pk_arows, set s of B at row s * 64.
  int64_t pk_ldb;
  int64_t pk_arows;
  // Grouped FW (may be null): vertices of each staged graph; the k range of a graph's last
  // block stops there (the padding vertices are isolated and add nothing).
  const int *gsize;
  // Host only, for tracing: when > 0, the launch's algorithmic pairs (grouped launches, whose
  // work the host sums over the graphs of the launch).
  double trace_pairs;
  // Added to the mode in trace records: 0, or kTraceSide for launches outside the closure's
  // main sequence (passes that normally return at once, the sub-closures and panels of a
  // wide block), so that the dominant kernel's records stay apart.
  int trace_class;
  // int32 storage (may be null): when *f32_if is non-zero the fp32 sequence runs even though
  // the exact bound does not hold -- a pass truncated at 2^24 that is certified afterwards
  // (fw.cu).
  const int *f32_if;
  // FW phase-3 launches (kModeFwRest, and kModeFwRest16 with bt <= 1; single matrix; may be
  // null): three device words, zero before the first such launch.  Tiles are then handed out by
  // an atomic counter (word 0), in the order the CTAs ask for them; word 2 counts the finished
  // tiles that the next block's panel tiles read (fuse_next); the last CTA to finish (word 1)
  // resets all three for the next launch on the stream.
  int *tile_counter;
  // With tile_counter, and kb + 1 < nb: the launch also performs phases 1 and 2 of the next
  // block kb1 = kb + 1.  Its tiles are handed out in this order:
  //   the diagonal tile (kb1, kb1) -- after its phase-3 update the CTA's consumer warps close it
  //     by Eq. 1 in registers (diag.cuh) before storing it;
  //   the other tiles of block row kb1, then of block column kb1 (phase 3 of block kb);
  //   the rest of phase 3 of block kb, row by row;
  //   phase 2 of block kb1: its row panel tiles (kb1, j), then its column panel tiles (i, kb1),
  //     each an in-place product with the closed diagonal tile; their producers wait (bounded)
  //     until every tile of the first three kinds is stored (word 2 of tile_counter).
  // A panel tile needs only tiles handed out before it, to CTAs that are already running, so
  // the wait always ends.  In kModeFwRest16 (not its 32-bit alternative) every tile of block
  // row or column kb1 also stores packed 16-bit copies (pk_a / pk_b, set (kb + 1) & 1) that the
  // panel tiles read, and the panel tiles run on them in the semiring truncated at kCap16 (their
  // result min(old entry, capped product), as phase 3's); they rewrite those copies in place as
  // the next launch's operands, and tiles of block row / column kb + 2 also into set kb & 1.
  int close_next;
  // kModeFwRest16, single matrix (may be null): when *alt_if is non-zero the launch runs its 32-bit
  // alternative instead of the packed one -- the same tiles over the block's bt * 128 columns
  // and rows of the matrix itself (maps mA2 / mB2 of launch_tgemm), K = the block width, with
  // the fp32 sequence (exact bound or *f32_if) or the int32 one.
  const int *alt_if;
};

// Packed 16-bit copies of a 128 x 128 tile held in the engine's register layout (thread (tm, tn)
// holds rows tm + 16 i and columns 4 tn + 64 h + q), values capped at kCap16.  Column pairs:
// word {v[r][2w], v[r][2w + 1]} at a + r * 64 + w.  Row pairs: word {v[2r][c], v[2r + 1][c]} at
// b + r * ldb + c; rows tm and tm ^ 1 sit in lanes lane and lane ^ 8, so every lane of the warp
// must call it.
__device__ __forceinline__ int pack_pair16(int lo, int hi) { return (min(hi, kCap16) << 16) | min(lo, kCap16); }

__device__ __forceinline__ void store_col_pairs16(const int (&v)[8][8], int tm, int tn, int *a) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h)
      *reinterpret_cast<int2 *>(a + (int64_t)(tm + 16 * i) * 64 + 2 * tn + 32 * h) =
          make_int2(pack_pair16(v[i][4 * h], v[i][4 * h + 1]), pack_pair16(v[i][4 * h + 2], v[i][4 * h + 3]));
}

__device__ __forceinline__ void store_row_pairs16(const int (&v)[8][8], int tm, int tn, int lane, int *b,
                                                  int64_t ldb) {
  const bool even = ((lane >> 3) & 1) == 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int o[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) o[q] = __shfl_xor_sync(0xffffffffu, v[i][4 * h + q], 8);
      if (even)
        *reinterpret_cast<int4 *>(b + (int64_t)((tm + 16 * i) >> 1) * ldb + 4 * tn + 64 * h) =
            make_int4(pack_pair16(v[i][4 * h], o[0]), pack_pair16(v[i][4 * h + 1], o[1]),
                      pack_pair16(v[i][4 * h + 2], o[2]), pack_pair16(v[i][4 * h + 3], o[3]));
    }
}

// 16-bit packing of int32 operands for ArithI16x2 (tgemm.cu).  Entries >= inf (and the padding
// past K) become kCap16.  They run only when words[0] + words[1] < kCap16 (the largest finite
// entries of A and B, so every finite sum is exact in 16 bits), and then set words[4] = 1.
int launch_pack16_a(const int *A, int64_t lda, int64_t M, int64_t K, int *A16, int64_t ld16, int inf, int *words,
                    cudaStream_t s);
int launch_pack16_b(const int *B, int64_t ldb, int64_t K, int64_t N, int *B16, int64_t ld16, int inf, int *words,
                    cudaStream_t s);

// Launch one tile pass.  acc: fold into the existing C (min) instead of overwriting it.
// maps: A box 128 rows x 32 cols, B box 32 rows x 128 cols, C box 128 x 128.  mA2 / mB2 (may be
// null): the matrix maps of kModeFwRest16's 32-bit alternative (TileProblem::alt_if).
int launch_tgemm(int mode, bool acc, int dtype, const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mC,
                 const TileProblem &p, cudaStream_t s, const CUtensorMap *mA2 = nullptr,
                 const CUtensorMap *mB2 = nullptr);

// Generic (any alignment, any leading dimension) tropical GEMM used when TMA's alignment
// rules do not hold.  Same semantics as tropical_gemm.
int launch_tgemm_generic(void *C, const void *A, const void *B, int64_t M, int64_t N, int64_t K, int64_t lda,
                         int64_t ldb, int64_t ldc, int dtype, bool acc, int inf_i, float inf_f, cudaStream_t s);

// Tensor maps for a row-major matrix used as A, B and C operands.
int make_operand_maps(const void *base, int64_t rows, int64_t cols, int64_t ld, int dtype, CUtensorMap *mA,
                      CUtensorMap *mB, CUtensorMap *mC);

// Strided 2-D copy (rows x cols elements of 4 bytes), used for operand copies.  run_if (may be
// null): the copy returns at once unless *run_if is non-zero.
int launch_copy2d(void *dst, int64_t ldd, const void *src, int64_t lds, int64_t rows, int64_t cols, cudaStream_t s,
                  const int *run_if = nullptr);

// a1 launcher (normalise.cu).  For int32, atomically maxes the largest finite entry into
// *wmax (device word, zeroed by the caller) when wmax is not null.
int launch_normalise(void *d, int64_t n, int64_t ld, int dtype, int inf_i, float inf_f, int *wmax, cudaStream_t s);

// Largest entry < inf of a rows x cols int32 matrix, atomically maxed into *out (normalise.cu).
int launch_scan_max(const void *x, int64_t rows, int64_t cols, int64_t ld, int inf, int *out, cudaStream_t s);

// Launch tracing (runtime.cu): when enabled, every tropical-GEMM-engine launch is bracketed
// by two CUDA events on its stream and tagged with its mode plus TileProblem::trace_class, and
// its algorithmic pair count.
constexpr int kTraceSide = 16;
bool trace_on();
void trace_begin(cudaStream_t s, void **ev0);
void trace_end(cudaStream_t s, void *ev0, int mode, double pairs);

// Bytes of the per-call bound words at the front of every workspace.
constexpr size_t kFlagBytes = 256;

}  // namespace apsp
