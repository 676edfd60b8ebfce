/*
 * kselect.h -- C ABI of the GB300 kernel-selection GEMM library (libkselect.so).
 *
 * Method: J. Lawson, "Performance portability through machine learning guided
 * kernel selection in SYCL libraries" (arXiv 2008.13145).  A parameterised
 * matrix-multiply kernel family (Section 3) is benchmarked over a grid of
 * shapes, pruned to a few deployed kernels by k-means clustering of
 * normalised performance vectors (Section 4), and one deployed kernel is
 * chosen per call by a decision tree on the sizes (Section 5).
 *
 * Conventions for every entry point:
 *  - Matrices are row-major.  op(A) is M x K: A itself (stored M x K,
 *    lda >= K) for transA 'N', or A^T (A stored K x M, lda >= M) for 'T'.
 *    op(B) is K x N likewise.  C is M x N with ldc >= N.
 *  - Batches are packed: batch entry b of A starts at A + b * lda * (stored
 *    rows of A); the same for B and C.
 *  - Pointers named *_dev are device pointers; all others are host pointers.
 *    The caller owns every buffer it passes and every stream; the library
 *    never frees caller memory.  A stream argument is a cudaStream_t passed as
 *    void* (NULL = the legacy default stream).  Work is enqueued
 *    asynchronously unless an entry point says it synchronises.
 *  - Errors are returned as gemm_status_t; nothing is printed and nothing
 *    aborts.  After GEMM_ERR_CUDA, gemm_last_cuda_error() gives the CUDA error
 *    code of the calling thread's last failing call.
 *  - There is no CPU fallback: every numeric step runs in the library's own
 *    CUDA kernels on the current device.
 */
#ifndef KSELECT_H
#define KSELECT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GEMM_OK = 0,
  GEMM_ERR_INVALID_ARG = -1, /* null pointer, negative size, ld too small, bad trans char */
  GEMM_ERR_UNSUPPORTED = -2, /* valid request this kernel or precision cannot run */
  GEMM_ERR_MISALIGNED = -3,  /* a tensor-core kernel needs 16-byte aligned pointers and lds */
  GEMM_ERR_CUDA = -4,        /* a CUDA call failed; see gemm_last_cuda_error() */
  GEMM_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  GEMM_ERR_NO_KERNEL = -6    /* unknown config id or empty deployment */
} gemm_status_t;

/* Kernel families (and precision classes of a handle).  F32: the FP32 SIMT family.  TF32: tcgen05 kind::tf32 on
 * FP32 storage.  BF16: tcgen05 kind::f16 on BF16 storage.  F32X3: FP32
 * storage split into BF16 hi/lo parts, three tcgen05 products accumulated in
 * FP32 (for K < 64 three parts and six products, which keep FP32-level
 * accuracy where few terms are summed).  C is FP32 in every family,
 * accumulation is FP32 in every family. */
typedef enum {
  GEMM_PREC_F32 = 0,
  GEMM_PREC_TF32 = 1,
  GEMM_PREC_BF16 = 2,
  GEMM_PREC_F32X3 = 3
} gemm_precision_t;

typedef struct kselect_library* gemm_handle_t;

const char* gemm_status_string(int32_t status);
int32_t gemm_last_cuda_error(void);

/* Debug-build hooks (no paper counterpart).  The library built with
 * KS_DEBUG_BOUNDS (libkselect_debug.so, a subset of the FP32 configs) checks
 * every global access of its FP32 kernels and of the split-K reduction
 * against the bytes each operand may span from its base -- (batch - 1)
 * strides + (rows - 1) leading dimensions + the row length -- and counts and
 * skips any access outside.  kselect_debug_bounds_errors reads the count
 * (synchronising the device; clear != 0 resets it); kselect_debug_shrink_extents
 * declares the operand extents smaller by the given bytes on later calls (a
 * test of the checker itself, which then flags accesses that are in fact
 * inside the buffers).  Release builds return GEMM_ERR_UNSUPPORTED. */
gemm_status_t kselect_debug_bounds_errors(int32_t* errors_out, int32_t clear);
gemm_status_t kselect_debug_shrink_extents(int64_t a_bytes, int64_t b_bytes, int64_t c_bytes);

/* ---------------------------------------------------------------- config space
 * Section 3: each work item computes an R x C output tile; tile sizes are
 * compile-time constants and the work-group shape is chosen per launch, giving
 * 640 configurations in the paper.  Here the FP32 family's compile-time
 * parameters are the per-thread tile TM x TN in {1,2,4,8}^2, the thread-block
 * shape (WX along N, WY along M) in {8x8, 16x16, 32x8, 8x32, 16x8, 8x16}, the
 * K-step BK in {8,16,32} and shared-memory staging on/off: 576 configs, ids
 * 0..575.  Tensor-core families (ids 1000 + 100*(family-1) + index, index =
 * (BN slot * 3 + stage slot) * 2) use a 128 x BN tile per CTA with BN in
 * {64,128,256} and a shared-memory ring of {2,3,4} stages: 9 configs per family
 * (the odd indexes are reserved and name no kernel: GEMM_ERR_NO_KERNEL).
 * gemm_config_id(family, i) = 1000 + 100*(family-1) + 2*i.  Operands are read in place by
 * TMA when K- or MN-contiguous (TF32 and BF16), 16-byte aligned and
 * batch-packed; others, and every F32X3 operand (split once into BF16 hi and
 * lo parts), are first rewritten by a pre-pass kernel.
 *
 * Split-K kind (Section 6 describes comparison libraries whose kernels for
 * tall, skinny matrices compute partial results combined by a final
 * reduction; Section 3.2 notes that such shapes behave differently): here it
 * is one more kernel kind to select.  Id 2000 + b runs FP32 config b (staged, BK
 * 16 or 32: 192 ids) with K divided among CTAs whenever its output tiles
 * alone would leave the GPU's resident-CTA slots (SMs x CTAs per SM) largely
 * idle.  Split s writes the partial product of K range [s * kchunk,
 * (s + 1) * kchunk) to a stream-ordered workspace (at most 256 MB, taken from a
 * per-device memory pool, or from the default pool while the stream is being
 * captured), and a second kernel sums the partials in split order and applies
 * alpha and beta: results are deterministic but rounded differently from the
 * base config.  gemm_config_count(GEMM_PREC_F32) = 576 + 192; indexes 576.. map
 * to the split-K ids in ascending base order.
 *
 * gemm_config_params writes 8 integers:
 *   F32: {family=0, TM, TN, WX, WY, BK, staged, splitk (0 or 1)}
 *   TC : {family, BM=128, BN, BK (elements per 128-byte row), stages, 0, 0, 0}
 */
int32_t gemm_config_count(int32_t precision);
int32_t gemm_config_id(int32_t precision, int32_t index);
gemm_status_t gemm_config_params(int32_t config_id, int32_t out_params[8]);

/* Split decision of the split-K kind, as a pure host function: the split
 * factor S >= 1 (a negative gemm_status_t on invalid arguments) for an
 * M x N x K x batch product with BM x BN tiles and K-step BK when
 * `resident_ctas_per_sm` CTAs fit on each of `sm_count` SMs; *kchunk receives
 * the K range per split (a multiple of BK; K when S == 1).  The factor
 * minimises (waves of tiles x S) x (K-steps per split + 2 for a CTA's start-up
 * and epilogue) plus the reduction's traffic, splits only when that saves at least 10 %, gives each split a
 * K range of at least 4 K-steps (the last one may be shorter), S <= 16,
 * batch x S <= 65535 and the workspace <= 256 MB. */
int32_t gemm_split_choose(int64_t M, int64_t N, int64_t K, int64_t batch, int32_t BM, int32_t BN, int32_t BK,
                          int32_t resident_ctas_per_sm, int32_t sm_count, int32_t* kchunk);

/* The split factor config `config_id` uses for these sizes on the current
 * device (1 for every config outside the split-K kind; needs a GPU for the
 * occupancy query); *kchunk as above.  Negative gemm_status_t on error. */
int32_t gemm_split_factor(int32_t config_id, int64_t M, int64_t N, int64_t K, int64_t batch, int32_t* kchunk);

/* ---------------------------------------------------------------- deployment
 * Section 5: the deployed set (<= 16 configs of one family) and a decision
 * tree mapping the sizes to one of them, evaluated as nested ifs in the
 * launcher.  Node j is a leaf when feature < 0; otherwise sizes with
 * value(feature) <= threshold go to `left`, others to `right`.  Features
 * (GEMM_TREE_FEATURES of them, kselect_selector_features): 0 = M, 1 = N,
 * 2 = K, 3 = batch, 4 = M * N * batch, the number of outputs.  The paper's
 * tree reads the matrix sizes; the output count is one more function of them
 * that a depth-limited tree cannot form from axis-aligned splits, and it is
 * what sets how many output tiles there are to spread over the SMs (whether
 * a split-K kernel pays).  A leaf's label indexes config_ids.
 * Optional MLP parameters (GEMM_MLP_PARAMS floats, layout W1 7x64, b1, W2
 * 64x64, b2, W3 64x8, b3) let select_kernels_batched rank the deployed set. */
#define GEMM_MAX_DEPLOYED 16
#define GEMM_MAX_TREE_NODES 65536
#define GEMM_MAX_TREES 256
#define GEMM_MLP_PARAMS 5192
#define GEMM_TREE_FEATURES 5

typedef struct {
  int32_t feature;
  int32_t left;
  int32_t right;
  int32_t label;
  double threshold;
} gemm_tree_node_t;

typedef struct {
  int32_t precision;            /* precision class: deployed configs are of this family, or
                                   for F32/F32X3/TF32 classes also of the F32 or F32X3
                                   family (same FP32 inputs, FP32-level accuracy) */
  int32_t n_configs;            /* 1..GEMM_MAX_DEPLOYED */
  const int32_t* config_ids;    /* host, n_configs ids */
  int32_t n_nodes;              /* 0 (always config_ids[0]) .. GEMM_MAX_TREE_NODES */
  const gemm_tree_node_t* nodes;/* host */
  const float* mlp_params;      /* host, GEMM_MLP_PARAMS floats, or NULL */
  int32_t n_known;              /* benchmarked sizes with their measured best kernel, or 0 */
  const int64_t* known_sizes;   /* host, n_known rows of (M, N, K, batch) */
  const int32_t* known_ids;     /* host, n_known config ids (any config of an allowed family) */
  int32_t n_trees;              /* 0 or 1: one tree rooted at node 0; 2..GEMM_MAX_TREES: a forest */
  const int32_t* tree_roots;    /* host, n_trees root indices into `nodes` (forest only); the
                                   trees share the node array but no node; every tree votes
                                   for one deployed config and the most-voted wins, the
                                   lowest label on ties (the random-forest classifier of
                                   Tables 1-2 as a runtime selector) */
} gemm_deployment_t;

/* Copies the deployment into a new immutable handle (host only; device
 * resources are made on first use).  Returns INVALID_ARG for a malformed tree
 * (child index out of range, cycle, leaf label outside the deployed set) and
 * NO_KERNEL for an unknown or mixed-family config id. */
gemm_status_t gemm_library_create(const gemm_deployment_t* deployment, gemm_handle_t* out);
void gemm_library_destroy(gemm_handle_t handle);

/* Deployed config id for these sizes, or a negative gemm_status_t: sizes that
 * were benchmarked (the deployment's known table) get their measured best
 * kernel -- the exhaustive selector as a fallback ahead of the classifier --
 * and all others the decision tree's choice (host walk, O(depth)). */
int32_t select_kernel(gemm_handle_t handle, int64_t M, int64_t N, int64_t K, int64_t batch);

/* ---------------------------------------------------------------- GEMM
 * C = alpha * op(A) * op(B) + beta * C for each batch entry, with the kernel
 * select_kernel() picks.  A and B are float* for F32/TF32/F32X3 handles and
 * bf16 (uint16_t*) for BF16 handles.  M, N or batch == 0 is a no-op; K == 0
 * sets C = beta * C.  When beta == 0, C is only written (it may hold NaN).
 * Sizes must be < 2^31 and batch <= 65535 (else GEMM_ERR_UNSUPPORTED). */
gemm_status_t gemm(gemm_handle_t handle, char transA, char transB, int64_t M, int64_t N, int64_t K,
                   float alpha, const void* A_dev, int64_t lda, const void* B_dev, int64_t ldb,
                   float beta, float* C_dev, int64_t ldc, int64_t batch, void* stream);

/* gemm() on host-resident data: copies A, B (and C when beta != 0) from the
 * host into the caller's device staging buffers (A_dev, B_dev, C_dev, each at
 * least the packed batch size), runs the selected kernel and copies C back,
 * all enqueued on `stream` (pinned host memory makes the copies
 * asynchronous; the caller synchronises before reading C_host). */
gemm_status_t gemm_host(gemm_handle_t handle, char transA, char transB, int64_t M, int64_t N, int64_t K,
                        float alpha, const void* A_host, int64_t lda, const void* B_host, int64_t ldb,
                        float beta, float* C_host, int64_t ldc, int64_t batch, void* A_dev, void* B_dev,
                        float* C_dev, void* stream);

/* gemm() with explicit batch strides, in elements: batch entry b uses
 * A + b * strideA, B + b * strideB, C + b * strideC.  strideA and strideB may be
 * any value >= 0 (0 uses one matrix for every entry, e.g. shared weights);
 * strideC must be >= ldc * M when batch > 1.  Tensor-core kernels read an
 * operand in place only when it is batch-packed (stride = ld x stored rows),
 * otherwise their pre-pass packs it first.  Errors as gemm(). */
gemm_status_t gemm_strided_batched(gemm_handle_t handle, char transA, char transB, int64_t M, int64_t N, int64_t K,
                                   float alpha, const void* A_dev, int64_t lda, int64_t strideA, const void* B_dev,
                                   int64_t ldb, int64_t strideB, float beta, float* C_dev, int64_t ldc,
                                   int64_t strideC, int64_t batch, void* stream);
gemm_status_t gemm_strided_batched_with_config(int32_t config_id, char transA, char transB, int64_t M, int64_t N,
                                               int64_t K, float alpha, const void* A_dev, int64_t lda,
                                               int64_t strideA, const void* B_dev, int64_t ldb, int64_t strideB,
                                               float beta, float* C_dev, int64_t ldc, int64_t strideC, int64_t batch,
                                               void* stream);

/* A sequence of gemm_host() problems as a three-stage pipeline: problem i's
 * host-to-device copies run on a library-owned upload stream, its GEMM (the
 * kernel select_kernel picks) on `stream` once they are done, and its C copy
 * back on a library-owned download stream once the GEMM is done, so uploads,
 * kernels and downloads of different problems overlap on the host link and
 * the GPU.  The uploads start after the work already queued on `stream`, and
 * `stream` ends waiting for the last download: synchronising `stream` covers
 * the whole call.  Each problem's staging buffers (A_dev, B_dev, C_dev, sized
 * as for gemm_host) must not overlap another problem's in the same call; host
 * buffers should be pinned for the copies to be asynchronous.  Problems are
 * validated before anything is enqueued (first error returned, nothing run). */
typedef struct {
  char transA, transB;
  int64_t M, N, K, batch;
  float alpha, beta;
  const void* A_host;
  int64_t lda;
  const void* B_host;
  int64_t ldb;
  float* C_host;
  int64_t ldc;
  void* A_dev;
  void* B_dev;
  float* C_dev;
} gemm_host_problem_t;

gemm_status_t gemm_host_pipeline(gemm_handle_t handle, int32_t count, const gemm_host_problem_t* problems,
                                 void* stream);

/* The same operation with an explicit config id (any family). */
gemm_status_t gemm_with_config(int32_t config_id, char transA, char transB, int64_t M, int64_t N,
                               int64_t K, float alpha, const void* A_dev, int64_t lda,
                               const void* B_dev, int64_t ldb, float beta, float* C_dev, int64_t ldc,
                               int64_t batch, void* stream);

/* ---------------------------------------------------------------- grouped GEMM
 * An uneven group of independent GEMMs in ONE persistent tensor-core launch:
 * every problem is cut into 128 x BN tiles, the tiles of all problems are
 * numbered consecutively -- problems ordered by K, longest first, so that the
 * fixed-stride walk below deals each CTA a balanced mix -- and each CTA walks
 * the global tile index with a fixed stride, mapping it to (problem, tile) by
 * binary search over the problems' first-tile offsets.  Per-problem TMA descriptors live in device
 * memory.  Problems use the row-major conventions above; K >= 1.  Operands
 * the kernel cannot read in place (any whose rows are not 16-byte aligned, and
 * every F32X3 operand) are first rewritten by one grouped pre-pass launch into
 * plan-owned scratch; TF32 and BF16 operands are read in place in either
 * storage order.
 *
 * A plan validates the problems, encodes their descriptors, uploads them and
 * allocates its scratch once (gemm_grouped_plan_create synchronises
 * `stream`); gemm_grouped_run then only launches kernels -- no allocation,
 * copy or host synchronisation -- so it can be captured in a CUDA graph and
 * replayed.  A, B and C of every problem must stay valid for the plan's life. */
typedef struct {
  int64_t M, N, K;
  char transA, transB;
  float alpha, beta;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  float* C;
  int64_t ldc;
} gemm_problem_t;

typedef struct kselect_grouped_plan* gemm_grouped_plan_t;

gemm_status_t gemm_grouped_plan_create(int32_t config_id, int32_t count, const gemm_problem_t* problems,
                                       void* stream, gemm_grouped_plan_t* out);
gemm_status_t gemm_grouped_run(gemm_grouped_plan_t plan, void* stream);
void gemm_grouped_plan_destroy(gemm_grouped_plan_t plan);

/* Tile-shape selection for a group (the benchmark / prune / classify loop run
 * on groups instead of single GEMMs): the handle's deployment is a set of
 * grouped-launch configs with a tree (or forest) over the group features
 * (median M, median N, median K, number of problems) -- the lower median of
 * each -- in place of (M, N, K, batch).  Returns the config id, or a negative
 * gemm_status_t (INVALID_ARG for a NULL handle or problems, count < 1, or a
 * negative size). */
int32_t gemm_grouped_select(gemm_handle_t handle, int32_t count, const gemm_problem_t* problems);

/* One-shot form with an explicit config: plan, run, synchronise `stream`,
 * release the plan (allocates and synchronises: not for graph capture). */
gemm_status_t gemm_grouped_with_config(int32_t config_id, int32_t count, const gemm_problem_t* problems,
                                       void* stream);

/* The library call for a group (Section 5: the selector runs inside the call,
 * before the launch).  `handle` holds a group selector -- a deployment of
 * grouped-launch configs whose tree reads the group features (see
 * gemm_grouped_select), as written for each family by the group autotuner --
 * and picks the tile configuration; `precision` is the class asked for:
 * GEMM_PREC_TF32, GEMM_PREC_BF16 (BF16 operands), or GEMM_PREC_F32X3 /
 * GEMM_PREC_F32 (FP32 operands at FP32-level accuracy, run by the split-BF16
 * family).  A selected config of another family gives GEMM_ERR_NO_KERNEL.
 *
 * Asynchronous on `stream`, with no host synchronisation and no allocation
 * once the handle's workspace on this device is large enough: the problems'
 * descriptors and pre-pass jobs are encoded on the host and written into that
 * workspace by small kernels that carry them as launch parameters, then the
 * pre-pass (if any operand needs one) and the persistent grouped launch run.
 * The call can therefore be captured in a CUDA graph; the graph holds the
 * descriptors, and each replay rewrites them before its launch.  The
 * workspace grows only outside a capture, on a call that needs more (that
 * call allocates), or through gemm_grouped_reserve; a call under capture
 * that would need to grow it, or that is the device's first tensor-core call,
 * returns GEMM_ERR_UNSUPPORTED and enqueues nothing.  A workspace that was
 * outgrown stays allocated until the handle is destroyed, so graphs captured
 * before a growth stay valid; no graph holding this call may be replayed
 * after its handle is destroyed.  Calls with one handle whose work overlaps
 * on the GPU (different streams without ordering, or concurrent graph
 * replays) share the workspace and race; calls ordered on one stream do not.
 * Problem rules as for plans (K >= 1; A, B, C valid until the launch has run). */
gemm_status_t gemm_grouped(gemm_handle_t handle, int32_t count, const gemm_problem_t* problems,
                           int32_t precision, void* stream);

/* Grows the handle's workspace on the current device to what gemm_grouped
 * needs for this group (allocates when it grows), so that later calls whose
 * groups need no more can be captured. */
gemm_status_t gemm_grouped_reserve(gemm_handle_t handle, int32_t count, const gemm_problem_t* problems,
                                   int32_t precision);

/* Section 3.1 (data collection): warm-up launches, then timed repetitions.
 * Runs `warmup` untimed launches and one timed probe launch, then times one
 * back-to-back run of R launches between two CUDA events, R = min_total_ms /
 * probe time clamped to [min_reps, max_reps], and writes the mean
 * milliseconds per launch (the paper's total time over a number of
 * iterations).  alpha = 1, beta = 0.  Synchronises `stream`.  Inputs are
 * whatever the buffers hold.  out_reps (may be NULL) receives R. */
gemm_status_t gemm_benchmark(int32_t config_id, char transA, char transB, int64_t M, int64_t N,
                             int64_t K, const void* A_dev, int64_t lda, const void* B_dev,
                             int64_t ldb, float* C_dev, int64_t ldc, int64_t batch,
                             int32_t warmup, int32_t min_reps, int32_t max_reps,
                             double min_total_ms, double* out_ms, int32_t* out_reps, void* stream);

/* Section 3.1, over a configuration list on one set of sizes.  Pass 1 times
 * one warm launch of every config (a launch longer than 2 ms is its own
 * warm-up; shorter ones are re-timed after `warmup` more launches).  Pass 2
 * re-times, as a back-to-back run sized like gemm_benchmark's, every config
 * whose pass-1 time is <= refine_ratio x the fastest; the others keep their
 * pass-1 time.  out_ms[c] is the time per launch (0 when out_status[c] != 0;
 * configs that cannot run this request report their status and are skipped).
 * Optional outputs (each may be NULL): out_probe_ms[c], the pass-1 time (0 when
 * the config did not run), and out_reps[c], the launches averaged into
 * out_ms[c]: 1 for a pass-1 time, R in [min_reps, max_reps] for a pass-2 run,
 * 0 when the config did not run.  Stops at the first GEMM_ERR_CUDA, which it
 * returns.  Synchronises `stream`. */
gemm_status_t gemm_benchmark_configs(int32_t n_configs, const int32_t* config_ids, char transA, char transB,
                                     int64_t M, int64_t N, int64_t K, const void* A_dev, int64_t lda,
                                     const void* B_dev, int64_t ldb, float* C_dev, int64_t ldc, int64_t batch,
                                     int32_t warmup, int32_t min_reps, int32_t max_reps, double min_total_ms,
                                     double refine_ratio, double* out_ms, int32_t* out_status,
                                     double* out_probe_ms, int32_t* out_reps, void* stream);

/* ---------------------------------------------------------------- pruning pipeline (Sections 3.4, 4)
 * Section 3.4: per row of an n_rows x n_cols throughput table (row-major,
 * FP32, device), x = perf / max(row) (0 for a row of zeros), then
 * mode 0 standard: x; 1 raw cutoff: 0 where x < 0.9; 2 standard cutoff:
 * 0 where x < 0.9, else (x - 0.9) / 0.1; 3 sigmoid: 1 / (1 + exp(50 (0.85 - x))).
 * out_dev may alias perf_dev. */
gemm_status_t kselect_normalise(int64_t n_rows, int32_t n_cols, const float* perf_dev, float* out_dev,
                                int32_t mode, void* stream);

/* Section 4.1: k-means over the n rows (points in R^d, FP32, device) of X.
 * n_init seeded runs, one thread block each: k-means++ seeding driven by the
 * host array draws (n_init x k uint32; centre 0 is point (draw * n) >> 32,
 * centre c picks the first point whose running sum of squared distances to
 * the nearest chosen centre exceeds draw / 2^32 times the total), then
 * Lloyd's iterations (nearest centre, lowest index on ties; each centre to
 * the mean of its points, an empty cluster keeps its centre) until the
 * total squared centre shift is <= tol x mean per-dimension variance of X,
 * or max_iter.  The run of lowest inertia (first on ties) is written:
 * centres_out_dev (k x d), labels_out_dev (n), *inertia_out, *iters_out.
 * Allocates its scratch stream-ordered; synchronises `stream`. */
gemm_status_t kselect_kmeans(int32_t n, int32_t d, int32_t k, int32_t n_init, const float* X_dev,
                             const uint32_t* draws, int32_t max_iter, float tol, float* centres_out_dev,
                             int32_t* labels_out_dev, double* inertia_out, int32_t* iters_out, void* stream);

/* Section 3.3 / 4.1 (PCA): the r leading principal components of the n rows
 * of X (n x d, device).  Covariance of the centred rows by the library's FP32
 * GEMM, `iters` rounds of subspace iteration from V0_dev (d x r starting
 * basis, e.g. seeded draws), then Rayleigh-Ritz.  Writes mean_out_dev (d),
 * V_out_dev (d x r, orthonormal columns, descending eigenvalue order),
 * Y_out_dev (n x r projections of the centred rows, or NULL), evals_out (r,
 * host) and *total_var_out (the covariance trace, host).  Allocates scratch
 * stream-ordered; synchronises `stream`. */
gemm_status_t kselect_pca(int32_t n, int32_t d, const float* X_dev, int32_t r, int32_t iters, const float* V0_dev,
                          float* mean_out_dev, float* V_out_dev, float* Y_out_dev, double* evals_out,
                          double* total_var_out, void* stream);

/* Section 4.1, spectral clustering: coordinates for k-means from the
 * similarity graph of the n rows of X_dev (n x d, device).  Adjacency
 * A_ij = exp(-gamma |x_i - x_j|^2) with a zero diagonal (distances from the
 * Gram matrix X X^T, computed by the library's FP32 GEMM); S = D^-1/2 A D^-1/2
 * with D the row sums (an isolated row gets D^-1/2 = 0); the k eigenvectors of
 * S with the largest eigenvalues -- those of the normalised Laplacian I - S
 * with the smallest -- by `iters` rounds of subspace iteration on S + I with an
 * r-column block (k <= r <= min(n, 256)) from V0_dev (n x r), then
 * Rayleigh-Ritz.  Writes U_out_dev (n x k, each row scaled to unit length) and
 * evals_out (k eigenvalues of S, host, descending).  Scratch n^2 + 2nr + r^2
 * floats, stream-ordered; synchronises `stream`. */
gemm_status_t kselect_spectral_embedding(int32_t n, int32_t d, const float* X_dev, float gamma, int32_t k, int32_t r,
                                         int32_t iters, const float* V0_dev, float* U_out_dev, double* evals_out,
                                         void* stream);

/* Section 4.2 for clusterings that give labels only: centres_out_dev (k x d)
 * = per cluster, the geometric mean over its rows of X_dev (n x d) with values
 * clamped below at `floor` (> 0); a cluster without rows gets zeros.  Labels
 * outside [0, k) are ignored.  Device arrays. */
gemm_status_t kselect_cluster_geomean(int32_t n, int32_t d, const float* X_dev, const int32_t* labels_dev, int32_t k,
                                      float floor, float* centres_out_dev, void* stream);

/* out_dev (k x d) = mean_dev + cent_dev (k x r) * V_dev^T: PCA-space centres as
 * performance vectors over the d configurations. */
gemm_status_t kselect_pca_backproject(int32_t k, int32_t d, int32_t r, const float* cent_dev, const float* V_dev,
                                      const float* mean_dev, float* out_dev, void* stream);

/* Section 4.3: over the rows of a throughput table (device), ratio =
 * perf[r, pick] / max(row) with pick = chosen_dev[r] (a classifier's column,
 * device int32) when chosen_dev is not NULL, else the best of the host list
 * deployed_cols (the deployed set's attainable maximum), else every column.
 * out[0] = geometric mean of max(ratio, floor), out[1] = arithmetic mean,
 * out[2] = number of ratios below floor.  Synchronises `stream`. */
gemm_status_t kselect_score(int32_t n_rows, int32_t n_cols, const float* perf_dev, int32_t n_deployed,
                            const int32_t* deployed_cols, const int32_t* chosen_dev, float floor_, double out[3],
                            void* stream);

/* Section 4.2 (host): the best column of each of k centres (k x d, host),
 * clusters in descending size from labels (n, host; lower index first on
 * ties).  With dedupe a cluster whose best is taken gets its best unused
 * column, without it the cluster is dropped.  Writes out_cols and *out_count. */
gemm_status_t kselect_representatives(int32_t k, int32_t d, const float* centres, int32_t n, const int32_t* labels,
                                      int32_t dedupe, int32_t* out_cols, int32_t* out_count);

/* Section 4.2 Top-N baseline (host): the n columns that are a row's best most
 * often (lowest index on ties), filled up by highest mean normalised value. */
gemm_status_t kselect_top_n(int32_t n_rows, int32_t n_cols, const float* perf, int32_t n, int32_t* out_cols);

/* Section 5.1 comparison classifier: k nearest neighbours (k <= 16).  For each
 * of n_query rows of query_dev (d features), the k training rows of train_dev
 * nearest in squared Euclidean distance (ties to the lower index) vote with
 * labels_dev; the majority label (ties to the nearest tied label) goes to
 * out_dev.  All arrays device, row-major. */
gemm_status_t kselect_knn(int32_t n_train, int32_t n_query, int32_t d, const float* train_dev,
                          const int32_t* labels_dev, const float* query_dev, int32_t k, int32_t* out_dev,
                          void* stream);

/* Section 4.1 "Decision tree" pruning (host): a multi-output regression tree
 * from the sizes (features, n x GEMM_TREE_FEATURES doubles as
 * kselect_selector_features writes them) to the normalised
 * performance vectors Y (n x d floats, host), grown best-first to at most
 * max_leaves leaves: the leaf whose best split (features in order, midpoint
 * thresholds ascending, first best kept) removes the most squared error is
 * split next, lowest leaf index on ties (gains within a relative 1e-9 count as
 * ties in both choices); growth stops early when no split
 * removes more than 1e-12 of the root's squared error.  A split leaf keeps its
 * index for the part <= threshold; the other part becomes the new last leaf.
 * Writes labels_out (n, leaf per size), centres_out (max_leaves x d, the mean
 * of Y over each leaf; rows beyond *n_leaves_out untouched) and *n_leaves_out.
 * INVALID_ARG on null pointers, sizes < 1 or non-finite inputs. */
gemm_status_t kselect_tree_regress(int32_t n, int32_t d, const double* features, const float* Y, int32_t max_leaves,
                                   int32_t* labels_out, float* centres_out, int32_t* n_leaves_out);

/* Section 5.1 classifier comparison (host): one random-forest tree -- the CART
 * of kselect_tree_train, except that node j (depth-first preorder) may split
 * only on max_features of the F = GEMM_TREE_FEATURES features: the first
 * max_features entries of the permutation (0, 1, ..., F - 1) after partial
 * Fisher-Yates steps t = 0, 1, ... that swap entry t with entry
 * t + draws[F j + t] mod (F - t); it becomes a leaf when none of them splits
 * it.  draws: F x max_nodes uint32 (host), ignored when max_features == F. */
gemm_status_t kselect_tree_train_rf(int32_t n, const double* features, const int32_t* labels, int32_t n_classes,
                                    int32_t max_depth, int32_t min_leaf, int32_t max_features, const uint32_t* draws,
                                    gemm_tree_node_t* out_nodes, int32_t max_nodes, int32_t* out_n_nodes);

/* Section 5.1 (host): the selector's feature rows of n sizes (sizes: n rows
 * of M, N, K, batch) as the tree reads them: features_out, n x
 * GEMM_TREE_FEATURES doubles (M, N, K, batch, M * N * batch).  INVALID_ARG on
 * null pointers, n < 0 or a negative size. */
gemm_status_t kselect_selector_features(int32_t n, const int64_t* sizes, double* features_out);

/* Section 5.1 (host): the training label of each size, the index j (into
 * cols, 0..n_sel-1) of its best deployed configuration, perf[row, cols[j]]
 * largest, lowest j on ties (perf: n_rows x n_cols doubles, row-major;
 * cols: n_sel column indexes).  INVALID_ARG on null pointers, sizes < 1, a
 * column outside [0, n_cols) or a NaN throughput. */
gemm_status_t kselect_best_labels(int32_t n_rows, int32_t n_cols, const double* perf, int32_t n_sel,
                                  const int32_t* cols, int32_t* labels_out);

/* Section 5.1 (host): CART classification tree on features (n x
 * GEMM_TREE_FEATURES doubles, kselect_selector_features) and labels (n, in
 * [0, n_classes)).  Gini impurity with the
 * class sum in class order; thresholds at midpoints of consecutive distinct
 * values; features in order, thresholds ascending, first best split kept; a
 * node is a leaf when pure, at max_depth (< 0: unlimited) or without a split
 * leaving >= min_leaf samples on each side; leaf label = majority, lowest
 * class on ties.  Nodes in depth-first preorder; UNSUPPORTED when more than
 * max_nodes are needed. */
gemm_status_t kselect_tree_train(int32_t n, const double* features, const int32_t* labels, int32_t n_classes,
                                 int32_t max_depth, int32_t min_leaf, gemm_tree_node_t* out_nodes,
                                 int32_t max_nodes, int32_t* out_n_nodes);

/* ---------------------------------------------------------------- learned selector (MLP)
 * A performance model beside the tree: 7 features of a GEMM -> 64 ReLU ->
 * 64 ReLU -> 8 outputs, the predicted natural-log GFLOP/s of each deployed
 * kernel (it replaces the paper's MLP classifier of Section 5.1 by a
 * regressor).  Parameters are one FP32 vector of GEMM_MLP_PARAMS values:
 * W1 (7 x 64, row = input), b1 (64), W2 (64 x 64), b2, W3 (64 x 8), b3 (8).
 * Features of (M, N, K, batch, transA, transB, dtype):
 *   [log2 M / 12, log2 N / 12, log2 K / 12, log2 batch / 4, transA, transB, dtype / 3].
 * X_dev is n x 7 FP32 features, T_dev n x 8 targets, mask_dev n x 8 (1 =
 * measured) or NULL for all measured.  All arrays are device, row-major. */

/* X_dev (n x 7) = features of the n GEMMs in shapes_dev (rows of 7 int64:
 * M, N, K, batch, transA, transB, dtype), as select_kernels_batched computes them. */
gemm_status_t mlp_features(int32_t n, const int64_t* shapes_dev, float* X_dev, void* stream);

/* Training targets from measured throughputs (perf_dev: n x d GFLOP/s, row =
 * size, column = deployed kernel, 0 = not measured): T_dev = log(perf / row
 * max), the natural log of Section 3.4's standard-normalised performance, and
 * mask_dev = 1 where perf > 0, else T = 0 and mask = 0.  The model thus
 * predicts each kernel's throughput relative to the fastest deployed kernel
 * for the size; selection (the largest output) is unaffected by the per-size
 * offset that absolute log-throughput would add.  All arrays device. */
gemm_status_t mlp_targets(int32_t n, int32_t d, const float* perf_dev, float* T_dev, float* mask_dev, void* stream);

/* Y_dev (n x 8) = network(X_dev). */
gemm_status_t mlp_forward(int32_t n, const float* params_dev, const float* X_dev, float* Y_dev, void* stream);

/* Mean squared error over the measured outputs and its gradient.  grad_dev
 * receives GEMM_MLP_PARAMS values and loss_dev one value.  Per-block partial
 * gradients are reduced in a fixed order (deterministic); their scratch is
 * allocated and freed stream-ordered. */
gemm_status_t mlp_loss_grad(int32_t n, const float* params_dev, const float* X_dev, const float* T_dev,
                            const float* mask_dev, float* grad_dev, float* loss_dev, void* stream);

/* mlp_loss_grad for callers that cannot allocate device memory: processes
 * whose device memory is owned by an external pool that reserved it all up
 * front, and latency-bound serving or training loops where a
 * cudaMalloc/cudaFree (which may synchronise the device) is not acceptable.
 * The paper has no counterpart: this is an interface choice of the library.
 * Same inputs, outputs and results as mlp_loss_grad, but its scratch is a
 * fixed array inside the library (about 5.3 MB per device, held until the
 * process exits); n is limited to 8192 samples, larger n returns
 * GEMM_ERR_UNSUPPORTED.  It calls no cudaMalloc or cudaFree.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current.  All calls on a device share the array: calls that
 * overlap on the GPU (different streams, or different host threads) race and
 * give wrong results. */
gemm_status_t mlp_loss_grad_noalloc(int32_t n, const float* params_dev, const float* X_dev, const float* T_dev,
                                    const float* mask_dev, float* grad_dev, float* loss_dev, void* stream);

/* One Adam step (Kingma & Ba, bias-corrected) at step t >= 1 on every parameter. */
gemm_status_t mlp_adam_step(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int32_t t,
                            float lr, float beta1, float beta2, float eps, void* stream);

/* `steps` full-batch Adam steps starting at step t0 + 1, captured once in a
 * CUDA graph and replayed; loss_hist_dev (steps values, or NULL) receives the
 * loss before each update.  Synchronises `stream`. */
gemm_status_t mlp_train(int32_t n, float* params_dev, const float* X_dev, const float* T_dev, const float* mask_dev,
                        float* m_dev, float* v_dev, int32_t t0, int32_t steps, float lr, float beta1, float beta2,
                        float eps, float* loss_hist_dev, void* stream);

/* Batched runtime selection for a queue of GEMMs: shapes_dev holds n rows of
 * 7 int64 (M, N, K, batch, transA, transB, dtype); the handle's MLP predicts
 * every deployed kernel's throughput and ids_dev[i] receives the config id of
 * the largest prediction among the handle's deployed kernels (lowest index on
 * ties).  pred_dev (n x 8) receives the predictions, or may be NULL.  The
 * handle must carry MLP parameters (else GEMM_ERR_UNSUPPORTED); they are
 * copied to the device on the first call per device. */
gemm_status_t select_kernels_batched(gemm_handle_t handle, int32_t n, const int64_t* shapes_dev, int32_t* ids_dev,
                                     float* pred_dev, void* stream);

/* ---------------------------------------------------------------- convolutional network layers
 * Section 6 runs VGG16 inference on the library's matrix multiply.  With NHWC
 * activations a 3x3 convolution (padding 1) is an im2col matrix times the
 * weights stored Cout x 9 Cin (op(B) = B^T), and the GEMM output rows are the
 * next NHWC activation.  All pointers device. */

/* out (N*H*W rows, leading dimension ld >= 9 C): row (n, h, w), column
 * (kh * 3 + kw) * C + c = x[n, h + kh - 1, w + kw - 1, c], 0 outside the image. */
gemm_status_t kselect_im2col3x3(const float* x_dev, int32_t N, int32_t H, int32_t W, int32_t C, float* out_dev,
                                int64_t ld, void* stream);

/* y[r, j] = y[r, j] + bias[j] (bias may be NULL), then max(., 0) if relu. */
gemm_status_t kselect_bias_act(float* y_dev, int64_t rows, int32_t cols, int64_t ld, const float* bias_dev,
                               int32_t relu, void* stream);

/* 2 x 2, stride 2 max pooling of NHWC x (H, W even) into out (N, H/2, W/2, C).
 * NCHW activations pool with N' = N * C images of one channel. */
gemm_status_t kselect_maxpool2x2(const float* x_dev, int32_t N, int32_t H, int32_t W, int32_t C, float* out_dev,
                                 void* stream);

/* The GEMM-batched layout Section 6 describes (per image, Cout x (H W) = the
 * weights Cout x 9 Cin times the image's im2col matrix transposed; batch =
 * images, weights shared through a zero batch stride in gemm_strided_batched):
 * activations are NCHW.  im2col from NCHW x: the same output rows and columns
 * as kselect_im2col3x3 (row (n, h, w), column (kh * 3 + kw) * C + c). */
gemm_status_t kselect_im2col3x3_nchw(const float* x_dev, int32_t N, int32_t C, int32_t H, int32_t W, float* out_dev,
                                     int64_t ld, void* stream);

/* y[n, c, p] = y[n, c, p] + bias[c] (bias may be NULL) for p < HW, then
 * max(., 0) if relu: per-channel bias of NCHW activations. */
gemm_status_t kselect_bias_act_nchw(float* y_dev, int32_t N, int32_t C, int64_t HW, const float* bias_dev,
                                    int32_t relu, void* stream);

/* ---------------------------------------------------------------- error check
 * The check of every GEMM result: err = max over entries of
 * |C - C_ref| / den, reduced on the GPU in FP64, where C_ref and den are the
 * FP64 exact product and its componentwise scale |alpha||op(A)||op(B)| +
 * |beta||C0| supplied by the caller.  den == 0 requires C == C_ref exactly
 * (else +inf); a NaN in C gives +inf.
 *   Full mode (pos_dev == NULL): C is rows x cols per batch entry with ldc and
 *   strideC; C_ref/den are packed (batch, rows, cols).  n is ignored.
 *   Sampled mode: n entries, pos_dev holds n (b, i, j) int64 triples, C_ref
 *   and den hold n values.
 * Writes the maximum to *out_err (host) and synchronises `stream`.  Uses a
 * device workspace of one double per block that it allocates and frees
 * stream-ordered. */
gemm_status_t gemm_error_check(int64_t rows, int64_t cols, int64_t batch, const float* C_dev,
                               int64_t ldc, int64_t strideC, int64_t n, const int64_t* pos_dev,
                               const double* Cref_dev, const double* den_dev, double* out_err,
                               void* stream);

/* The tensor-core kernels' device status word for the current device: 0, or
 * the code of the first bounded wait that gave up (1 TMA slice never landed,
 * 2 slice never released, 3 accumulator never completed, 4 accumulator never
 * drained).  The word is sticky -- once set, later tensor-core launches on
 * that device wind down early -- until read with clear != 0.  Synchronises
 * the device.  Returns GEMM_ERR_TIMEOUT when the word is nonzero. */
gemm_status_t gemm_device_status(int32_t* out_status, int32_t clear);

/* Test hook for the failure path above (no paper counterpart): one warp runs the
 * tensor-core kernels' bounded mbarrier wait, with a limit of limit_ns
 * (1 .. 2e9), on a barrier that nothing arrives at.  The wait gives up, sets the
 * status word to 1 as a stalled TMA slice would, and the kernel returns;
 * *waited_out = 0 (1 would mean the barrier completed).  The context stays
 * usable.  Synchronises `stream`. */
gemm_status_t kselect_wait_selftest(int64_t limit_ns, int32_t* waited_out, void* stream);

/* Fills a (batch, rows, ld) float array with uniform[lo, hi) values from a
 * counter-based hash of (seed, element index); padding columns get `pad`.
 * Benchmark input only (tests draw their inputs on the host). */
gemm_status_t kselect_fill_uniform(float* dst_dev, int64_t rows, int64_t cols, int64_t ld,
                                   int64_t batch, uint64_t seed, float lo, float hi, float pad,
                                   void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KSELECT_H */
