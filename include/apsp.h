/*
 * apsp.h -- C ABI of libapsp.so: exact all-pairs shortest paths on dense n x n distance
 * matrices over the (min,+) semiring, for NVIDIA GB300 (sm_103a).
 *
 * The problem (the paper, Sec. 2 and Sec. 3.1): given a cost matrix H whose entry [i][j] is
 * the cost of the edge i -> j, produce d[i][j], the length of a shortest directed path from
 * i to j.  Sec. 2 Eq. 1 gives the Floyd-Warshall recurrence
 *     d^{k+1}[i][j] = min{ d^k[i][j], d^k[i][k] + d^k[k][j] },
 * and Sec. 3 Eq. 2 the (min,+) product Z[i][j] = min_k (X[i][k] + Y[k][j]) on which every
 * entry point below rests.
 *
 * Conventions for every call
 * --------------------------
 *  - Matrices are row-major in DEVICE memory, with a leading dimension (elements between
 *    the starts of consecutive rows) ld >= number of columns.  The caller owns every buffer;
 *    the library never frees caller memory and keeps no pointer after a call returns.
 *  - dtype: APSP_I32 (int32) or APSP_F32 (float32).  Arithmetic happens in that type.
 *  - "No edge / unreachable":
 *      int32: a sentinel inf (pointer to an int32; NULL means APSP_INF_I32 = 0x3FFFFFFF),
 *             1 <= inf <= 0x3FFFFFFF.  Every entry >= inf is unreachable and is written back
 *             as exactly inf.  Because inf + inf < 2^31, sums never overflow and saturation
 *             is the plain min against inf.
 *      float32: a sentinel inf (pointer to a float; NULL means +infinity).  Every entry
 *             >= the sentinel becomes +infinity, and unreachable results are +infinity.
 *  - Weights must be >= 0 (Sec. 3.1 assumes no negative cycles; this library takes the
 *    stronger, checkable condition).  A negative entry, or a NaN, is a data error.
 *  - stream: a cudaStream_t passed as void* (NULL = the legacy default stream).  Every call
 *    is asynchronous on that stream and may be captured into a CUDA graph provided the
 *    caller supplies the workspace (ws != NULL).  The kernels of the closures and products
 *    are launched with programmatic dependent launch: the next kernel's blocks may be
 *    scheduled while the previous kernel on the stream drains, and each waits for it to
 *    complete before touching memory, so stream order holds for the caller's work as well.
 *    Setting the environment variable APSP_PDL=0 before the first call launches them
 *    without that attribute.
 *  - ws / ws_bytes: caller workspace in device memory (256-byte aligned, at least the size
 *    reported by the matching *_workspace_bytes function).  ws == NULL makes the library
 *    allocate it on `stream` from its own stream-ordered pool and free it after the work
 *    (apsp_workspace_pool_trim releases the pool's cached memory).
 *
 * Errors
 * ------
 *  Every entry point returns an apsp_status.  Argument errors (bad sizes, ld < columns,
 *  unsupported dtype or tile, a workspace that is too small or misaligned, an out-of-range
 *  sentinel) return APSP_ERR_ARG before anything is launched.  A failed launch or CUDA call
 *  returns APSP_ERR_CUDA.  Data errors found on the device (negative weight, NaN) cannot be
 *  returned by an asynchronous call: they set bits of a per-device status word, which stays
 *  set until apsp_device_status() reads and clears it.  After a data error the contents of
 *  the matrix are unspecified.
 */
#ifndef APSP_H_
#define APSP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define APSP_INF_I32 0x3FFFFFFF
#define APSP_VERSION 100

typedef enum apsp_dtype { APSP_I32 = 0, APSP_F32 = 1 } apsp_dtype;

typedef enum apsp_status {
  APSP_OK = 0,
  APSP_ERR_ARG = 1,         /* invalid argument; nothing was launched */
  APSP_ERR_DOMAIN = 2,      /* negative weight, NaN or out-of-range entry seen on the device */
  APSP_ERR_NOMEM = 3,       /* workspace allocation failed */
  APSP_ERR_CUDA = 4,        /* a CUDA call or launch failed */
  APSP_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  APSP_ERR_UNSUPPORTED = 6, /* no device of compute capability 10.3, or feature absent */
  APSP_ERR_NEGATIVE_CYCLE = 7 /* apsp_fw_signed found a negative cycle on the device */
} apsp_status;

/* Library version (APSP_VERSION of the build). */
int apsp_version(void);

/* Workspaces the library allocates for calls made with ws == NULL come from a stream-ordered
 * memory pool per device that keeps freed memory for later calls (so a caller that
 * synchronises between calls does not pay for mapping the memory again).  This releases the
 * current device's cached pool memory.  Returns APSP_OK or APSP_ERR_CUDA. */
int apsp_workspace_pool_trim(void);

/* Static, human-readable name of a status code. */
const char *apsp_status_str(int status);

/* Synchronises `stream`, then reads and clears the current device's sticky data-status
 * word into *out: APSP_OK, or the most severe code a kernel flagged since the last read
 * (APSP_ERR_TIMEOUT, then APSP_ERR_ARG for a skipped batch entry, then
 * APSP_ERR_NEGATIVE_CYCLE, then APSP_ERR_DOMAIN).
 * Returns APSP_OK, or APSP_ERR_CUDA if the synchronisation failed. */
int apsp_device_status(void *stream, int *out);

/* ---- a1: validate and normalise (Sec. 3.1 assumptions, Sec. 3.4 zero diagonal) --------
 * In place on the n x n matrix d (leading dimension ld): sets d[i][i] = 0; maps entries
 * >= inf to inf (int32) or +infinity (float32); flags negative entries and NaN in the
 * device status word.  n = 0 is a no-op. */
int apsp_normalise(void *d, int64_t n, int64_t ld, int dtype, const void *inf, void *stream);

/* ---- a2: tropical GEMM, the (min,+) product of Sec. 3 Eq. 2 ---------------------------
 *   accumulate = 0:  C[i][j] = min(inf, min_k A[i][k] + B[k][j])
 *   accumulate = 1:  C[i][j] = min(C[i][j], min_k A[i][k] + B[k][j])
 * A is M x K (lda), B is K x N (ldb), C is M x N (ldc), all row-major in device memory.
 * Entries of A, B (and C when accumulating) must already lie in [0, inf] (int32) or be
 * >= 0 or +infinity (float32); apsp_normalise produces that form.  C must not overlap A
 * or B (APSP_ERR_ARG).  K = 0 gives C = inf (or leaves C unchanged when accumulating);
 * M = 0 or N = 0 is a no-op.  When every base is 16-byte aligned and every leading
 * dimension a multiple of 4, the TMA-fed engine runs; otherwise a plain-load kernel.
 * int32 arithmetic is chosen on the device from the largest finite entries of A and B (a
 * scan): when they sum below 0x3FFF and the workspace has room for packed copies, the operands
 * are packed into 16-bit pairs and each DPX operation performs two (min,+) pairs; else, below
 * 2^24, exact fp32 arithmetic on the int32 bit patterns; else int32.  Results are identical.
 * The workspace (tropical_gemm_workspace_bytes) holds the two maxima (256 bytes) and, for
 * int32, the packed copies (M x round_up(ceil(K/2), 4) + ceil(K/2) x round_up(N, 4) words); a
 * workspace of only 256 bytes is accepted and skips the 16-bit path. */
size_t tropical_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K, int dtype);
int tropical_gemm(void *C, const void *A, const void *B, int64_t M, int64_t N, int64_t K,
                  int64_t lda, int64_t ldb, int64_t ldc, int dtype, const void *inf,
                  int accumulate, void *ws, size_t ws_bytes, void *stream);

/* ---- a3-a5: blocked Floyd-Warshall (Eq. 1 organised over b x b tiles) -----------------
 * Closes d (n x n, leading dimension ld) in place: after the call d[i][j] is the shortest
 * path length i -> j (inf / +infinity if none).  Runs a1 first.  For each diagonal block
 * kb: phase 1 closes tile (kb,kb) by Eq. 1; phase 2 updates the row and column panels of kb
 * by a (min,+) product with the closed tile; phase 3 updates every other tile by
 * D[i][j] = min(D[i][j], D[i][kb] (x) D[kb][j]).
 * tile: block size b; 0 selects the default (128).  Supported: 128.
 * d must be 16-byte aligned.  The workspace holds 256 bytes of bound words (int32 matrices
 * whose (n - 1) * largest finite weight < 2^24 run in exact fp32 arithmetic on their bit
 * patterns; others in int32), when ld is not a multiple of 4 an aligned copy of the matrix
 * (n x round_up(n, 4) elements), and last, for int32 with n >= 4096, room for a 16-bit pass
 * (the two panels packed into 16-bit pairs, 2 x 128 x round_up(n, 128) words, and copies of
 * the two 256-wide panels, 256 x round_up(n, 4) + n x 256 elements; apsp_fw_workspace_bytes
 * gives the total).  With that room, and a largest weight of at most 0x0FFF, phases 2 and 3
 * run on the packed pairs (two (min,+) pairs per DPX operation) in the (min,+) semiring
 * truncated at 0x3FFF; a device-side certificate (largest stored value below 0x3FFF plus the
 * largest weight stays below 0x3FFF) proves the result exact, and otherwise the int32
 * Floyd-Warshall runs again over it.  With the same room, an int32 matrix whose largest weight is above 0x0FFF and
 * at most 2^22, and too large for the exact fp32 bound, runs phase 3 in fp32 on its bit patterns
 * truncated at 2^24, certified the same way (largest stored value below 2^24 plus the largest
 * weight stays below 2^24), else followed by the exact int32 loop.  Results are bit-exact either
 * way.  A workspace without that room is accepted and closes with the plain phase 3. */
size_t apsp_fw_workspace_bytes(int64_t n, int64_t ld, int dtype, int tile);
int apsp_fw(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int tile, void *ws,
            size_t ws_bytes, void *stream);

/* ---- a6: R-Kleene (Sec. 3.3, Eq. 4) -----------------------------------------------------
 * Closes d in place by the 2 x 2 block recursion H = [[A, B], [C, D]]:
 *   A = A*;  B = A (x) B;  C = C (x) A;  D = min(D, C (x) B);  D = D*;
 *   B = B (x) D;  C = D (x) C;  A = min(A, B (x) C).
 * Blocks of size <= cutoff are closed by blocked Floyd-Warshall.  The split point is a
 * multiple of 128.  cutoff: 0 selects the default (256); it must be >= 128.
 * d must be 16-byte aligned.  The workspace holds the 256 bytes of bound words (as for
 * apsp_fw), a copy of the block being overwritten (h x round_up(h, 4) elements,
 * h = ceil(n/2) rounded up to a multiple of 128, when n > cutoff), when ld is not a multiple
 * of 4 an aligned copy of the matrix, and last, for int32, room for the operands of the
 * largest product packed into 16-bit pairs (h x round_up(ceil(h/2), 4) + ceil(h/2) x
 * round_up(h, 4) words).  With that room, a product of at least 10^9 pairs whose operands'
 * largest finite entries sum below 0x3FFF (a device-side scan) runs on the packed pairs; the
 * result is identical.  Leaves close as apsp_fw closes a matrix (those of at least 4096
 * vertices reuse that room for the 16-bit pass); their certificates step by the leaf block's own
 * largest finite entry (a device-side scan), since a leaf holds path lengths through the
 * vertices closed before it.  A workspace without the packed room is accepted. */
size_t apsp_rkleene_workspace_bytes(int64_t n, int64_t ld, int dtype, int cutoff);
int apsp_rkleene(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int cutoff,
                 void *ws, size_t ws_bytes, void *stream);

/* ---- negative weights (Sec. 3.1 assumes only that no cycle is negative) ----------------
 * Closes d in place like apsp_fw (a1, then blocked Floyd-Warshall), for matrices whose finite
 * entries may be negative.  The diagonal is set to 0; entries >= inf are missing edges.
 *   int32: the sentinel must be >= 0x30000000 (NULL: APSP_INF_I32), and (n - 1) times the
 *     largest |finite entry| must stay below 2^27, so that every distance lies in
 *     (-2^27, 2^27); this is checked on the device after a1 (else APSP_ERR_DOMAIN and the
 *     matrix is left normalised, not closed).  Sums that involve a missing edge are kept at or
 *     above 2^29 and written back as exactly inf.  Arithmetic is int32 throughout.
 *   float32: +infinity absorbs negative terms; NaN is a data error (APSP_ERR_DOMAIN).
 * A negative cycle is detected on the device: the closure of the diagonal block that holds the
 * cycle's largest vertex sees a negative d[v][v], sets APSP_ERR_NEGATIVE_CYCLE, and every later
 * launch returns at once; the matrix is then unspecified.  A final scan of the diagonal reports
 * any negative entry the same way.  d must be 16-byte aligned.  The workspace
 * (apsp_fw_signed_workspace_bytes) holds the 256 bytes of bound words and, when ld is not a
 * multiple of 4, an aligned copy of the matrix. */
size_t apsp_fw_signed_workspace_bytes(int64_t n, int64_t ld, int dtype);
int apsp_fw_signed(void *d, int64_t n, int64_t ld, int dtype, const void *inf, void *ws,
                   size_t ws_bytes, void *stream);

/* ---- the paper's "Floyd-Warshall on GPU" (Sec. 3.2): repeated (min,+) squaring ----------
 * Closes d in place by D <- D (x) D (Eq. 2) until no entry changes.  After t products D[i][j]
 * is the shortest path of at most 2^t edges, so max_iters = 0 selects ceil(log2(n - 1))
 * products, which always reach the closure; the loop stops doing work after the first product
 * that changes nothing (checked on the device, so nothing waits on the host).  A positive
 * max_iters caps the number of products (at most 48); with fewer than needed the result holds
 * the shortest paths of at most 2^max_iters edges.  Runs a1 first.  Costs n^3 (min,+) pairs per
 * product: O(n^3 log n) in the worst case against Floyd-Warshall's n^3, but only a few products
 * for graphs of small diameter.  d must be 16-byte aligned.  The workspace holds the 256 bytes
 * of bound words, the product matrix (n x round_up(n, 4) elements) and, when ld is not a
 * multiple of 4, an aligned copy of d.  int32 results equal apsp_fw's exactly; float32 results
 * differ from them only in summation order. */
size_t apsp_squaring_workspace_bytes(int64_t n, int64_t ld, int dtype);
int apsp_squaring(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int max_iters,
                  void *ws, size_t ws_bytes, void *stream);

/* ---- R-Kleene with no device allocation ------------------------------------------------
 * The paper has no counterpart to this entry point.  It is apsp_rkleene for callers that
 * cannot call cudaMalloc -- code inside a framework or plugin host that owns all device
 * memory through its own pool, request paths that forbid allocator calls, processes under a
 * hard memory budget.  Its scratch is a fixed array inside libapsp.so (about 16 MiB per GPU
 * that loads the library, held until exit), so the caller passes only the matrix:
 *   - n must be <= APSP_NOALLOC_MAX_N and ld a multiple of 4; otherwise APSP_ERR_ARG and
 *     nothing is launched (use apsp_rkleene with a workspace instead);
 *   - it calls no cudaMalloc, cudaFree or allocating library routine;
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *     make that first call before any stream capture;
 *   - every call shares the array: calls that overlap on the GPU race and must be serialised
 *     by the caller;
 *   - for n up to about 2816 the array also has room for the packed 16-bit operands of the
 *     largest int32 products, which then run on 16-bit pairs as in apsp_rkleene with a full
 *     workspace; larger n take the 32-bit products.
 * Results are identical to apsp_rkleene's. */
#define APSP_NOALLOC_MAX_N 4096
int apsp_rkleene_noalloc(void *d, int64_t n, int64_t ld, int dtype, const void *inf, int cutoff,
                         void *stream);

/* ---- a7: batched closure of many independent graphs --------------------------------------
 * Closes `count` graphs in place.  Graph g is an ns[g] x ns[g] matrix stored row-major at
 * element offset offsets[g] of `pool` with leading dimension lds[g]; it is closed exactly as
 * apsp_fw would close it (a1 normalisation, then blocked Floyd-Warshall), so results are
 * identical to closing each graph alone.  `order` (device, optional) lists the graph indices
 * in processing order -- largest first balances the persistent CTAs best; NULL = 0..count-1.
 * offsets, ns, lds and order are DEVICE arrays of `count` entries; ns_host (optional, host) is
 * a copy of ns that lets the library pick the launch shape: when some graph would take longer
 * alone than the average work per SM, the kernel runs as thread-block clusters that close
 * such graphs together; otherwise one CTA per graph on every SM (NULL: clusters).  pool must be 16-byte
 * aligned; every lds[g] and offsets[g] must be a multiple of 4 and lds[g] >= ns[g]: a graph
 * that breaks this, or an order entry outside [0, count), is skipped and sets APSP_ERR_ARG
 * in the device status word (the rest of the batch is still closed).  ns[g] <= 0 is skipped.
 * The workspace holds the work-queue counter (apsp_batched_workspace_bytes); with the room
 * reported by apsp_batched_staged_workspace_bytes (and ns_host), the larger int32 graphs are
 * closed in lockstep on the tropical-GEMM engine instead (below), the others by the persistent
 * launch in the library's own largest-first order (`order` is then not used).  Either way
 * the call is asynchronous, allocates nothing when ws is given, and can be captured in a CUDA
 * graph. */
size_t apsp_batched_workspace_bytes(int64_t count);
/* Workspace with which apsp_batched closes the larger graphs of an int32 batch in lockstep
 * on the tropical-GEMM engine instead of one per CTA (same results).  ns_host: host copy of
 * the sizes (the same values as the device ns passed to apsp_batched).  Graphs of 257..2048
 * vertices are copied into a staging matrix in the workspace, each padded to whole 128-vertex
 * tiles; per 128-vertex block, one launch per phase runs it for every such graph (phase 3 on
 * packed 16-bit pairs, certified per graph as in apsp_fw, with an int32 pass for the graphs
 * whose certificate fails).  Every other graph goes to the persistent kernel.  Returns
 * apsp_batched_workspace_bytes(count) when no graph qualifies or dtype is APSP_F32.  The
 * staged path runs only when apsp_batched gets ns_host, a caller workspace of at least this
 * size and a sentinel above 0x3FFF; a staged graph whose device size, leading dimension or
 * offset disagree with ns_host or the layout rules is left untouched and sets APSP_ERR_ARG. */
size_t apsp_batched_staged_workspace_bytes(const int32_t *ns_host, int64_t count, int dtype);
int apsp_batched(void *pool, const int64_t *offsets, const int32_t *ns, const int32_t *lds,
                 const int32_t *order, const int32_t *ns_host, int64_t count, int dtype,
                 const void *inf, void *ws, size_t ws_bytes, void *stream);

/* ---- predecessors and path reconstruction (pred[i, j] of Sec. 2; the argmin of Sec. 3.1) --
 * pred (n x n int32, leading dimension ldp) receives, for each pair, the vertex just before j
 * on a shortest i -> j path:
 *     pred[i][j] = the smallest k != j minimising d[i][k] + w[k][j]
 * where d (ldd) is the CLOSED distance matrix (the output of apsp_fw, apsp_rkleene or
 * apsp_batched) and w (ldw) the cost matrix it was closed from; w's diagonal is never used and
 * its entries >= inf count as missing edges.  pred[i][i] = -1, and pred[i][j] = -1 where j is
 * unreachable from i.  Walking back from j (p = pred[i][j], then pred[i][p], ...) reaches i and
 * spells out a shortest path whose edge costs sum to d[i][j] (int32 exactly) -- guaranteed
 * when every off-diagonal weight is positive, the assumption of Sec. 3.1.  With zero-cost
 * edges each pred entry is still a last hop of some shortest path, but a walk may cycle
 * through a zero-cost loop.  Negative entries or NaN in d or w set APSP_ERR_DOMAIN.
 * int32: sums are exact and ties go to the smallest k.  When pred is 16-byte aligned with ldp
 * a multiple of 4, the argmin runs as one (min,+) product of encoded copies of d and w
 * (index bits below the value bits) on the tropical GEMM engine, provided the encoded sums fit
 * below 0x3FFFFFFF (checked on the device); otherwise a direct argmin kernel runs.  The
 * workspace (apsp_predecessors_workspace_bytes) holds the bound words and the two encoded
 * copies (2 x n x round_up(n, 4) int32).
 * float32: the direct kernel, with each sum rounded once (round to nearest) and ties to the
 * smallest k; the workspace is only the 256 bytes of bound words. */
size_t apsp_predecessors_workspace_bytes(int64_t n, int dtype);
int apsp_predecessors(const void *d, int64_t ldd, const void *w, int64_t ldw, int32_t *pred,
                      int64_t ldp, int64_t n, int dtype, const void *inf, void *ws,
                      size_t ws_bytes, void *stream);

/* ---- a8: the planner's cost-model network ---------------------------------------------
 * A perceptron with two hidden layers of 64 ReLU units, fp32, that predicts the log run time
 * of a closure configuration from a feature vector of in_dim (1..32) floats:
 *   h1 = relu(x W1 + b1); h2 = relu(h1 W2 + b2); y = h2 . w3 + b3.
 * params is one flat device array [W1 (in_dim x 64, row-major), b1 (64), W2 (64 x 64), b2 (64),
 * w3 (64), b3 (1)] of apsp_mlp_param_count(in_dim) floats.  x is batch x in_dim row-major.
 *  - apsp_mlp_forward: out[batch]; if acts is not NULL it receives h1 and h2 per sample
 *    (batch x 2 x 64 floats), which apsp_mlp_backward needs.
 *  - apsp_mlp_loss: mean squared error *loss (device, may be NULL) and dout = dL/dout.
 *  - apsp_mlp_backward: grads (same layout as params) of the loss whose dout is given;
 *    deterministic; workspace of apsp_mlp_backward_workspace_bytes(in_dim, batch).
 *  - apsp_mlp_adam: one Adam step (bias-corrected; step counts from 1) over count floats.
 * The paper has no learned component; this serves the planner only. */
int64_t apsp_mlp_param_count(int in_dim);
size_t apsp_mlp_backward_workspace_bytes(int in_dim, int batch);
int apsp_mlp_forward(const float *params, int in_dim, const float *x, int batch, float *out,
                     float *acts, void *stream);
int apsp_mlp_loss(const float *out, const float *y, int batch, float *dout, float *loss,
                  void *stream);
int apsp_mlp_backward(const float *params, int in_dim, const float *x, const float *acts,
                      const float *dout, int batch, float *grads, void *ws, size_t ws_bytes,
                      void *stream);
int apsp_mlp_adam(float *params, const float *grads, float *m, float *v, int64_t count, float lr,
                  float beta1, float beta2, float eps, int step, void *stream);

/* ---- host memory for fast transfers ----------------------------------------------------
 * apsp_host_alloc returns `bytes` of page-locked host memory, registered with CUDA (usable by
 * cudaMemcpyAsync and the *_host calls below, and readable by kernels), or NULL on failure.
 * Large buffers (at least a quarter of the system's transparent huge page, 512 MiB on a
 * 64 KiB-page Grace host, 2 MiB with 4 KiB pages) are mapped on huge-page boundaries and
 * advised for huge pages before they are pinned.  The GPU reaches host memory through its own
 * page tables: a 4 GiB buffer of small pages needs tens of thousands of translations, and after
 * a large closure has pushed them out of the GPU's caches a copy of it ran at about a tenth of
 * the link's rate (measured on GB300: 200 ms against 20 ms for 4 GiB); the same buffer in huge
 * pages copies at full rate every time.  Smaller buffers come from cudaHostAlloc.  Free with
 * apsp_host_free (exactly the pointer returned; NULL is a no-op).  Returns APSP_OK or
 * APSP_ERR_ARG (a pointer this library did not allocate) / APSP_ERR_CUDA. */
void *apsp_host_alloc(size_t bytes);
int apsp_host_free(void *p);

/* ---- host buffers: copy in, close, copy back ------------------------------------------
 * These calls take HOST memory (pinned for full copy speed; pageable works), run the device
 * entry points above on `stream`, and return once the results are in the host buffer (they
 * synchronize; not for CUDA-graph capture).  Status and data errors as for the device calls.
 *
 * apsp_solve_host: h_in / h_out are n x n host matrices with leading dimension ld_host (they
 * may be the same buffer).  algo 0 = apsp_fw (param = tile), 1 = apsp_rkleene (param =
 * cutoff), 2 = apsp_squaring (param = max_iters).  d: optional device matrix (n x ldd, 16-byte
 * aligned rows) to work in; NULL takes it from the library's memory pool.  ws / ws_bytes as
 * for the chosen algorithm.
 *
 * apsp_batched_host: h_in / h_out are host pools laid out exactly as the device pool `pool`
 * (graph g at element offset offsets_host[g], ns_host[g] x ns_host[g], leading dimension
 * lds_host[g]); offsets / ns / lds are the same descriptors in device memory.  The batch is
 * split into `chunks` runs of consecutive graphs of about equal work (0 = 4; a layout whose
 * graph ranges are not in pool order runs as one chunk).  Chunk c is closed by apsp_batched
 * on `stream` while chunk c + 1 is copied in and chunk c - 1 copied out on two library copy
 * streams.  ws: apsp_batched_host_workspace_bytes(...) bytes (the staged path's room for the
 * largest chunk), or NULL for the library pool.  Graph sizes must satisfy ld >= n and
 * offset >= 0 on the host copies (else APSP_ERR_ARG before any copy). */
int apsp_solve_host(const void *h_in, void *h_out, int64_t n, int64_t ld_host, int dtype, int algo, int param,
                    const void *inf, void *d, int64_t ldd, void *ws, size_t ws_bytes, void *stream);
size_t apsp_batched_host_workspace_bytes(const int32_t *ns_host, const int64_t *offsets_host,
                                         const int32_t *lds_host, int64_t count, int dtype, int chunks);
int apsp_batched_host(const void *h_in, void *h_out, void *pool, const int64_t *offsets_host,
                      const int32_t *ns_host, const int32_t *lds_host, const int64_t *offsets,
                      const int32_t *ns, const int32_t *lds, int64_t count, int dtype, const void *inf,
                      int chunks, void *ws, size_t ws_bytes, void *stream);

/* ---- measurement: launch tracing ------------------------------------------------------
 * apsp_trace_enable(1) makes every launch of the tropical GEMM engine (the standalone
 * product and blocked-FW phases 2 and 3) record a CUDA event before and after itself on its
 * stream.  apsp_trace_read(mode, ...) waits for those events, returns the summed elapsed
 * time (ms), the number of launches and their algorithmic (min,+) pairs for engine mode
 * `mode` (0 = product, 1 = FW panels, 2 = FW remaining tiles; 16 + those: launches outside
 * the closure's main sequence, such as the exact int32 pass that returns at once after a
 * certified truncated one, or the small sub-closures of a 256-vertex block; -1 = all), then
 * discards the records it returned.  Host-global; not for use inside CUDA-graph capture. */
int apsp_trace_enable(int on);
int apsp_trace_read(int mode, double *total_ms, int64_t *launches, double *pairs);

/* ---- measurement: launch count ---------------------------------------------------------
 * Number of kernel launches the library has enqueued in this process (every entry point,
 * including launches that return at once on the device because an earlier step made them
 * unnecessary), counted on the host as each launch is made.  reset != 0 returns the count
 * and sets it to zero.  Host-global and thread-safe; launches captured into a CUDA graph are
 * counted once, at capture. */
int64_t apsp_launch_count(int reset);

/* ---- measurement: CUDA-core (min,+) rate probe -----------------------------------------
 * Launches `blocks` x `threads` threads, each running `iters` rounds of a register-only
 * (min,+) update of 32 independent accumulators with the instruction sequence `variant`:
 *   0: int32 fused add-min (__viaddmin_s32)      1: int32 add then 2-input min
 *   2: int32 two adds then 3-input min            3: fp32 add then 2-input min
 *   4: fp32 two adds then 3-input min             5: fp32 packed pair add then 3-input min
 *   6: as 5 on subnormal operands (int32 bit patterns below 2^24 read as fp32)
 *   7: packed 16-bit pairs, one DPX add-min (__viaddmin_s16x2) for two pairs
 *   8: packed 16-bit pairs, SIMD add then SIMD min
 * Variants 0-6 perform blocks*threads*iters*64 pairs, 7-8 blocks*threads*iters*128.
 * Variants 9-11 time the fp32 slab arithmetic of the tropical-GEMM engine in isolation, on
 * one CTA of threads = 256 per block (anything else: APSP_ERR_ARG) with four 128 x 32 and
 * 32 x 128 operand slabs resident in shared memory (128 KiB of dynamic shared memory); each
 * iteration is one 128 x 128 x 32 slab, so blocks*iters*524288 pairs:
 *   9:  the engine's instruction sequence reading its operands from shared memory;
 *   10: the same packed adds and 3-input mins on operands held in registers;
 *   11: as 10 plus one integer XOR per 16 pairs (other work on the ALU pipe, which also
 *       executes the 3-input min).
 * Writes a checksum per thread to sink (device, blocks*threads int32) so nothing is dead
 * code; for variants 9-11, thread 0 of each block writes instead the SM clocks its block
 * spent in the loop, divided by 1024.  Time it with events on `stream`. */
int apsp_probe_minplus(int variant, int blocks, int threads, int iters, void *sink,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* APSP_H_ */
