/*
 * hmgb300 — H-LU of point-cloud kernel matrices on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library libhmgb300.so.  The operations follow Börm, Christophersen and
 * Kriemann, "Semi-Automatic Task Graph Construction for H-Matrix Arithmetic"
 * (arXiv 1911.07531):
 *
 *   hm_build   H-matrix of a kernel matrix over a cluster tree (Def 2.1) and block tree
 *              (Def 2.2) with standard admissibility min(diam t, diam s) <= eta dist(t, s)
 *              (§5.1); admissible leaves stored low-rank (Def 2.3).
 *   hm_lu      H-LU factorization A = L U (Alg 2, with Alg 1 and Alg 3), executed as the
 *              task graph built by semi-automatic refinement (§3.1, Alg 9-11): the graph's
 *              longest-path levels run as waves of batched CUDA kernels.
 *   hm_solve   forward / backward substitution with the H-LU factors (the solves of Alg 3
 *              applied to vectors), optionally refined against A.
 *   hm_matvec  y = alpha op(M) x + beta y for M = A, L, U, P L U, or the exact kernel matrix.
 *
 * Conventions
 *   - Every function returns an int status: HM_OK (0) or a negative HM_E* code; the message
 *     of the last failure on the calling thread is returned by hm_last_error().
 *   - Vectors and right-hand sides are DEVICE pointers, column-major with leading dimension
 *     `ld` (>= n), in the ORIGINAL point order; the library applies its cluster permutation.
 *     Points passed to hm_build are a HOST array (n x 3, row-major, x y z).
 *   - The caller owns every buffer it passes; handles (hm_ctx, hm_matrix, hm_factor,
 *     hm_structure) are owned by the library and released with their *_free / *_destroy.
 *     A factor keeps a pointer to its matrix: free the factor before the matrix.
 *   - Device memory of the library comes from the context's allocator callbacks (e.g. the
 *     PyTorch caching allocator); with NULL callbacks cudaMalloc / cudaFree are used.
 *   - All work is enqueued on the context's stream. hm_build, hm_lu, hm_solve and
 *     hm_matvec synchronize that stream before returning (they report device status).
 *   - Arithmetic is FP64 (hm_lu can run its products in FP32 or on the tensor cores:
 *     HM_PREC_MIXED, HM_PREC_MIXED_TC).
 *     There is no CPU fallback: without a usable CUDA device every computing call fails
 *     with HM_ECUDA.
 */
#ifndef HMGB300_H
#define HMGB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HM_OK = 0,
  HM_EINVAL = -1,     /* invalid argument (NULL handle, n < 1, ld < n, ...) */
  HM_ENOMEM = -2,     /* the allocator returned NULL; no state was changed */
  HM_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
  HM_ESINGULAR = -4,  /* a numerically zero pivot in a diagonal leaf LU (see
                         hm_stats.singular_pivots; the factor is still returned)        */
  HM_ETIMEOUT = -5,   /* a bounded device wait gave up (tensor-core MMA completion) */
  HM_ENOTCONV = -6,   /* iterative refinement did not reach refine_tol */
  HM_EINTERNAL = -7   /* planner invariant violated */
};

enum { HM_OP_A = 0, HM_OP_L = 1, HM_OP_U = 2, HM_OP_LU = 3, HM_OP_EXACT = 4 };

/* Smallest truncation accuracy eps accepted by hm_build, hm_lu, hm_lu_batch, hm_truncate and
 * hm_truncate_noalloc (HM_EINVAL below it). The rounded truncation (§2.3 asks for a fixed rank
 * or a relative accuracy and leaves the method open) is computed here from the Gram
 * matrices of the stacked factors, whose rounding errors are of size u |W|^2: singular values
 * below about sqrt(K u) |W| |Z| ~ 1e-8 of the largest are not resolved, so eps below this floor
 * would return factors that silently miss 10 eps. */
#define HM_EPS_MIN 1e-8

typedef struct hm_ctx hm_ctx;
typedef struct hm_matrix hm_matrix;
typedef struct hm_factor hm_factor;
typedef struct hm_structure hm_structure;

/* Device allocator callbacks. alloc returns NULL on failure; free receives the size. */
typedef void* (*hm_alloc_fn)(size_t bytes, void* user);
typedef void (*hm_free_fn)(void* ptr, size_t bytes, void* user);

typedef struct {
  int leaf_size;     /* clusters with at most leaf_size points are leaves (default 64)   */
  double eta;        /* admissibility parameter (default 2.0)                           */
  double eps;        /* relative truncation accuracy of admissible blocks, in
                        [HM_EPS_MIN, 1) (default 1e-6)                                  */
  int rank_cap;      /* maximal rank of a low-rank block, 1..64 (default 64)            */
  double kernel_h;   /* regularisation h of 1/(4 pi (r + h)); <= 0: mean NN spacing     */
  int prepare_lu;    /* 1: while the device assembles the matrix, a host thread builds the
                        task graph (Alg 11) and the H-LU plan for hm_lu's defaults (the
                        matrix's eps, FP64, no accumulators, the current hm_set_overlap and
                        GEMM settings), so that a following hm_lu starts launching at once;
                        any later call on the matrix waits for that thread. 0 (default):
                        hm_lu builds them.                                                */
} hm_build_opts;

/* Arithmetic of hm_lu (hm_lu_opts.precision).
 *   HM_PREC_FP64      every product in FP64 (the truncation core's Jacobi sweeps in FP32).
 *   HM_PREC_MIXED     the products of Alg 1 (low-rank and dense leaf products and their
 *                     application to dense leaves) and the rebuild products of every rounded
 *                     addition in FP32 (FP64 operands rounded to FP32, FP32 FMAs and
 *                     accumulation, FP64 results: ~1e-7 relative to |A| |B|). The Gram matrices,
 *                     the truncation core, the leaf LU with its pivots and the triangular solves
 *                     stay FP64. Meant for a coarse factorization (eps ~1e-4) that hm_solve's FP64
 *                     iterative refinement turns into an accurate solve.
 *   HM_PREC_MIXED_TC  as HM_PREC_MIXED, but the products with at least 128 rows run on the
 *                     tensor cores (tcgen05 kind::tf32): FP64 operands split into two TF32 parts,
 *                     three MMAs (hi hi, hi lo, lo hi), FP32 accumulation in tensor memory
 *                     (~1e-6 relative to |A| |B|). */
enum { HM_PREC_FP64 = 0, HM_PREC_MIXED = 1, HM_PREC_MIXED_TC = 2 };

typedef struct {
  double eps;        /* relative accuracy of every rounded addition during H-LU (<=0: the
                        matrix's eps; else in [HM_EPS_MIN, 1)); the rank cap is the
                        matrix's                                                          */
  int precision;     /* HM_PREC_FP64, HM_PREC_MIXED or HM_PREC_MIXED_TC                   */
  int accumulate;    /* 0: the H-LU of Alg 2 (every update rounded into its leaf in the wave
                        that forms it). 1: the accumulator H-LU of §2.3 (Alg 4-8): the update
                        pieces of a low-rank leaf are collected (add_upd; shift_upd restricts a
                        block's pieces to its sons) and added in one rounded addition before
                        the leaf is used (apply_upd), in the wave of its last update; pieces
                        that outlive their wave are held in a device arena (stats arena_bytes).
                        Not available in hm_lu_batch.                                     */
} hm_lu_opts;

typedef struct {
  double refine_tol; /* > 0: iterate x += LU^{-1} (b - A x) until |b - A x| <= tol |b|     */
  int max_iter;      /* refinement steps (0: plain substitution)                          */
  int residual_op;   /* HM_OP_A (H-matrix) or HM_OP_EXACT (kernel evaluated on the fly)   */
} hm_solve_opts;

typedef struct {
  int iterations;          /* refinement steps taken                                     */
  double rel_residual;     /* |b - A x| / |b| after the last step (max over columns); -1
                              when no residual was computed                              */
} hm_solve_info;

typedef struct {
  int64_t n;
  int64_t nclusters, nleaf_clusters, depth;
  int64_t nleaves_dense, nleaves_lowrank;
  int64_t value_bytes;          /* device bytes of the block values                      */
  double h;                     /* kernel regularisation used                            */
  double eps;
  int64_t rank_cap;
  int64_t max_rank, sum_rank;   /* over low-rank leaves                                  */
  int64_t dag_nodes, dag_edges, dag_levels;   /* task graph (0 before the first hm_lu)  */
  double dag_seconds;           /* host time of the task graph construction (Alg 11)     */
  int64_t plan_launches, plan_phases, plan_truncations;
  int64_t scratch_bytes;        /* device scratch of the H-LU plan (both spaces with overlap) */
  double plan_seconds;          /* host time of wave planning                            */
  double seconds;               /* device time of the last hm_build / hm_lu (CUDA events) */
  double flops[5];              /* model flops of the last hm_lu: getrf, trsm, gemm,
                                   rounded truncation (QR + core + SVD + rebuild), other */
  int64_t rank_cap_hits;        /* rounded additions that hit the rank cap               */
  int64_t singular_pivots;      /* numerically zero pivots met in diagonal leaves: |p| <=
                                   b u max|a| over the b x b leaf being factored (u = 2^-53) */
  int64_t aca_unconverged;      /* ACA runs that hit their rank limit during hm_build    */
  double kind_ms[8];            /* with profiling on: device ms per kernel kind          */
  int64_t kind_launches[8];     /*   getrf trsm gemm copy stack core eval aca            */
  double kind_flops[8];         /* algorithmic flops executed per kernel kind (last hm_lu) */
  int64_t launches;             /* kernel launches of the last hm_lu                     */
  int64_t row_interchanges;     /* row interchanges of partial pivoting in the leaf LUs  */
  int64_t precision;            /* HM_PREC_* of the last hm_lu                           */
  double tc_ms;                 /* the tensor-core GEMM kind (HM_PREC_MIXED_TC): device ms */
  int64_t tc_launches;          /*   with profiling on, launches,                          */
  double tc_flops;              /*   and flops executed (2mnk per micro-op)                */
  double f32_ms;                /* the FP32 GEMM kind (mixed precision): the same three    */
  int64_t f32_launches;
  double f32_flops;
  int64_t plan_deferred;        /* rounded additions of the H-LU plan that overlap the next
                                   wave on the side stream (hm_set_overlap)               */
  int64_t accumulate;           /* 1: the last hm_lu was the accumulator H-LU             */
  int64_t arena_bytes;          /*   its accumulator arena (held update pieces)           */
  int64_t accumulated_pieces;   /*   update pieces held past the wave that formed them    */
} hm_stats;

/* Last error message of the calling thread ("" if none). */
const char* hm_last_error(void);

/* Host threads used by task-graph construction (the parallel loops of Alg 13, §4.2) and by the
 * H-LU planner, for every later call of the process (0, the default: all hardware threads).
 * The task graph and the plan do not depend on it. HM_EINVAL if threads < 0. */
int hm_set_host_threads(int threads);

/* Context: device ordinal, a cudaStream_t (NULL = the legacy default stream) and the
 * allocator callbacks (both NULL = cudaMalloc / cudaFree). */
int hm_ctx_create(int device, void* cuda_stream, hm_alloc_fn alloc, hm_free_fn free_fn, void* user,
                  hm_ctx** out);
void hm_ctx_destroy(hm_ctx* ctx);
/* With profiling on, every kernel launch of hm_lu is bracketed by CUDA events and the
 * per-kind device time is reported in hm_stats.kind_ms (adds host overhead). */
int hm_ctx_set_profiling(hm_ctx* ctx, int enable);

/* Build the H-matrix of a_ij = 1/(4 pi (|x_i - x_j| + h)) (Def 2.1-2.3, §5.1): cluster
 * tree by geometric bisection, block tree, dense leaves evaluated on the device,
 * admissible leaves by ACA with partial pivoting to eps/10 and rounded truncation to eps.
 * points: host, n x 3 row-major (copied). opts: NULL for defaults. */
int hm_build(hm_ctx* ctx, const double* points_xyz, int64_t n, const hm_build_opts* opts, hm_matrix** out);
void hm_matrix_free(hm_matrix* A);

/* H-LU factorization (Alg 2) of A executed as the Alg 11 task graph in waves. A is not
 * modified; the factor holds L (unit lower, with leaf pivots) and U in H-format. */
int hm_lu(hm_ctx* ctx, hm_matrix* A, const hm_lu_opts* opts, hm_factor** out);
void hm_factor_free(hm_factor* F);

/* H-LU of count independent matrices in one launch sequence (batching across instances): wave
 * w of every matrix's task graph is expanded into the same phases, so that one launch per
 * kernel kind and phase serves all of them. out[i] receives the factor of A[i], usable and
 * freed like one from hm_lu. The matrices are factored in consecutive groups that fit 85 % of
 * the device memory free at the call (values, ranks, pivots and the group's plan and scratch);
 * the factors of a group share one allocation, released with the last of them. A factor's
 * stats (seconds, flops, launches) are those of its group. opts->eps <= 0 needs all matrices
 * built with the same eps. Errors as hm_lu; on an error other than HM_ESINGULAR no factor is
 * returned. */
int hm_lu_batch(hm_ctx* ctx, hm_matrix* const* A, int count, const hm_lu_opts* opts, hm_factor** out);

/* x = (P L U)^{-1} b for nrhs right-hand sides (device, column-major, leading dimension
 * ld, original order). b and x may alias. With opts->max_iter > 0 and A != NULL, iterative
 * refinement against op(A) (opts->residual_op) runs until the relative residual of every
 * column is <= refine_tol (HM_ENOTCONV if max_iter is reached first). info may be NULL. */
int hm_solve(hm_ctx* ctx, hm_factor* F, hm_matrix* A, const double* b, double* x, int64_t nrhs, int64_t ld,
             const hm_solve_opts* opts, hm_solve_info* info);

/* y = alpha op(M) x + beta y. op: HM_OP_A (A, F may be NULL), HM_OP_L / HM_OP_U / HM_OP_LU
 * (the factors of F), HM_OP_EXACT (the exact kernel matrix of A's points, n^2 kernel
 * evaluations).  x, y device, column-major, original order; x and y must not alias. */
int hm_matvec(hm_ctx* ctx, hm_matrix* A, hm_factor* F, int op, double alpha, const double* x, double beta,
              double* y, int64_t nrhs, int64_t ld);

int hm_matrix_stats(const hm_matrix* A, hm_stats* out);

/* Storage layout of A's block values (Def 2.3: dense leaves and low-rank leaves U V^T), for
 * inspection, and for callers that edit the values (hm_matrix_copy_values). Host outputs, each
 * may be NULL:
 *   leaves[nleaves*10]   per block-tree leaf (pre-order): row cluster, column cluster, m, n,
 *                        low-rank (0/1), rank capacity, value offset (dense D or U, column-
 *                        major, ld m), V offset (ld n), rank index, pivot offset (-1: none)
 *   perm[n]              original point index of each position of the cluster order
 *   cluster_lo[nclusters] first position of each cluster (depth-first pre-order ids)
 *   *nleaves, *nvalues, *nclusters   the counts. */
int hm_matrix_layout(const hm_matrix* A, int64_t* leaves, int64_t* perm, int64_t* cluster_lo, int64_t* nleaves,
                     int64_t* nvalues, int64_t* nclusters);
/* Copies A's nvalues block values to (to_matrix == 0) or from (to_matrix != 0) the caller's
 * device buffer buf, on the context stream (synchronized). Writing replaces the matrix that
 * later hm_lu / hm_matvec(HM_OP_A) calls see (the ranks of the low-rank leaves stay); the
 * structure, the task graph and the plans depend only on the trees, so they remain valid.
 * HM_OP_EXACT keeps evaluating the kernel of the points. */
int hm_matrix_copy_values(hm_ctx* ctx, hm_matrix* A, double* buf, int to_matrix);
int hm_factor_stats(const hm_factor* F, hm_stats* out);

/* Rounded truncation of W Z^T (W: m x K, Z: n x K, device, column-major, ld >= m / n) to
 * relative spectral accuracy eps (keep sigma_i > eps sigma_1) and rank <= cap (<= 64):
 * U (m x k) and V (n x k, orthonormal columns) with U V^T ~ W Z^T. K <= 256. *k_out
 * (host) receives k. This is the kernel the H-LU applies to every low-rank update
 * (the "truncation operation" of §2.3); device scratch comes from the context allocator.
 * The method works on the Gram matrices W^T W and Z^T Z, so its error floor is about
 * sqrt(K u) relative to |W| |Z| (~1e-8): eps below that is not resolved, and singular values
 * within ~1e-6 (relative) of eps sigma_1 may be kept or dropped. */
int hm_truncate(hm_ctx* ctx, int64_t m, int64_t n, int K, const double* W, int64_t ldw, const double* Z,
                int64_t ldz, double eps, int cap, double* U, int64_t ldu, double* V, int64_t ldv, int* k_out);

/* Same rounded truncation as hm_truncate, for callers that must not allocate device memory
 * (a serving loop whose device buffers are all sized at start-up, or a plugin living in
 * another framework's memory pool with no allocator to hand to hm_ctx_create). The paper has
 * no counterpart; this is a property of the library, not of the method.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call. Its scratch is a
 *     file-scope device array of 16 MiB (2^21 doubles) that every GPU loading the library holds
 *     until the process exits. Sizes beyond it are rejected with HM_EINVAL; m + n <= 8192
 *     with K <= 128 always fits.
 *   - Runs on the current device and the given stream (NULL = legacy default stream); the
 *     caller passes W, Z (inputs) and U, V (outputs, at least min(cap, m, n) columns) as
 *     device buffers; *k_out (host) receives the rank. Synchronizes the stream.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.
 *   - Every call shares the one array and it keeps the last call's contents (the entry point
 *     clears what must start at zero): calls that overlap on the GPU (other streams, other
 *     host threads) race and must be serialized by the caller. */
int hm_truncate_noalloc(void* cuda_stream, int64_t m, int64_t n, int K, const double* W, int64_t ldw,
                        const double* Z, int64_t ldz, double eps, int cap, double* U, int64_t ldu, double* V,
                        int64_t ldv, int* k_out);

/* GEMM split tuning (process-wide): the number of FMAs that one CTA of the batched GEMM kernels
 * aims at when a micro-op is spread over several CTAs (default 4096). Smaller values give more,
 * shorter CTAs (more parallelism, more atomic partial sums), larger ones fewer. It changes the
 * plans (an H-LU plan built at another value is rebuilt at the next hm_lu) and the speed, not
 * the results beyond rounding. HM_EINVAL outside [256, 2^24]. */
int hm_set_gemm_work(double fmas_per_cta);
double hm_get_gemm_work(void);
/* Autotuner of that setting for one matrix: for every candidate value, plans and factors A
 * twice with opts (hm_lu) and keeps the device time of the second factorization; leaves the
 * fastest candidate set and returns it in *best (seconds[q], if not NULL, receives candidate q's
 * time). The factors are freed. Errors of hm_lu are returned (the previous setting restored). */
int hm_autotune_gemm(hm_ctx* ctx, hm_matrix* A, const hm_lu_opts* opts, const double* candidates, int ncand,
                     double* best, double* seconds);
/* Wave overlap (process-wide, default 1): a rounded addition (Alg 10) whose target leaf no task
 * of the next level of the task graph reads or updates is issued on a second stream of the
 * context and overlaps that next wave; the waves after it wait for it through CUDA events
 * before they reuse its scratch (two scratch spaces, alternating by wave, so an H-LU with
 * overlap needs twice the scratch memory). 0: every micro-op in wave order on one stream.
 * Profiled factorizations (hm_ctx_set_profiling) run without overlap. Changes the plans (an
 * H-LU plan built with the other setting is rebuilt at the next hm_lu) and the speed, not the
 * results: the same micro-ops run on the same operands. HM_EINVAL unless on is 0 or 1. */
int hm_set_overlap(int on);
int hm_get_overlap(void);

/* Diagnostic: y[i] = f(x[i]) for the FP64 reciprocal helpers that the serial sections of the
 * leaf LU and of the truncation core use instead of IEEE division and square root (no passage
 * of the paper: a property of this implementation). which: 0 Newton-Raphson 1/x from a
 * rescaled FP32 seed (any finite nonzero x), 1 Newton-Raphson 1/sqrt(x) (x > 0), 2 the
 * three-operation series 1/x (x in [1e-30, 1e30]), 3 the leaf LU's pivot reciprocal (2 inside
 * [1e-30, 1e30] in magnitude, else 0). x, y: device arrays of n doubles (may alias); runs on
 * the given stream (NULL = legacy default stream) of the current device and synchronizes it.
 * HM_EINVAL for a bad `which` or n < 0, HM_ECUDA on a launch failure. */
int hm_selftest_reciprocals(void* cuda_stream, int which, const double* x, double* y, int64_t n);

/* ---- host-only structure (no GPU needed): cluster tree, block tree, task graph -------- */
typedef struct {
  int64_t n, nclusters, nleaves, ntasks, nedges, nlevels;
  double dag_seconds;
  int64_t plan_launches, plan_phases, plan_gemm_ops, plan_truncations, plan_scratch_bytes;
} hm_structure_info;

/* Cluster tree (Def 2.1), block tree (Def 2.2) and the H-LU task graph of Alg 11 with its
 * longest-path levels. points: host n x 3. with_plan != 0 also runs the H-LU planner. */
int hm_structure_build(const double* points_xyz, int64_t n, int leaf_size, double eta, int with_plan,
                       hm_structure** out);
/* The same trees with the task graph of the accumulator-based H-LU (Alg 4-8).
 * merged == 0: semi-automatic refinement with the dependencies of Table 2 (§3.2): a refined
 *   hlu / htrsl / htrsu starts with shift_upd of its block, apply_upd of a leaf precedes the task
 *   that factorises or solves with it, add_upd (task type 1) is refined like hmul (Alg 1) and
 *   writes the block and its accumulator; the other tasks read the parent block's accumulator.
 * merged != 0: the two-part construction of §4.3: the standard graph of Alg 11 (hmul tasks as
 *   add_upd) plus one shift_upd / apply_upd task per block-tree node, linked by explicit edges
 *   (parent -> son accumulator task, add_upd -> accumulator task of its destination, apply_upd
 *   of a leaf -> the leaf task). Same tasks, fewer edges; a single-leaf matrix gets an apply_upd.
 * No plan. Errors as hm_structure_build. */
int hm_structure_build_accumulator(const double* points_xyz, int64_t n, int leaf_size, double eta, int merged,
                                   hm_structure** out);
/* The standard (accumulators == 0) or accumulator (§3.2) task graph built with the removal of
 * redundant edges of Alg 12 (§4.1) after every refinement step: an edge of a task (or of its
 * sub-tasks) goes when its target is also reached by a path of length >= 2 inside the task's
 * neighbourhood (its sub-tasks and its successors' sub-tasks). For the standard graph the
 * reachability, and so every longest-path level, is unchanged; for the accumulator graph the
 * removal can drop the ordering of an accumulator before its sons' (the hazard §4.1 points
 * out), so such a graph is for inspection only. No plan. Errors as hm_structure_build. */
int hm_structure_build_sparsified(const double* points_xyz, int64_t n, int leaf_size, double eta, int accumulators,
                                  hm_structure** out);
int hm_structure_info_get(const hm_structure* S, hm_structure_info* out);

/* Host-side plan of a structure built by hm_structure_build (the standard task graph), for
 * inspection and host-side checks; no GPU is used. which = 0: the H-LU plan at accuracy eps
 * (> 0); which = 1: the forward / backward substitution plan for up to nrhs_max (>= 1)
 * right-hand sides; which = 2..5: the product plan of hm_matvec for op = which - 2 (HM_OP_A,
 * HM_OP_L, HM_OP_U, HM_OP_LU) on a work buffer of four n x nrhs_max blocks (x, y, two
 * temporaries); which = 6: the assembly plan of hm_build at accuracy eps (dense leaves by
 * kernel evaluation, admissible leaves by ACA + rounded truncation, into the matrix-value space
 * 3 from the permuted points, space 4, n x 3 row-major); which = 7: the H-LU plan of which = 0
 * with wave overlap (hm_set_overlap): deferred rounded additions are side launches, and the
 * odd waves address the second scratch spaces (doubles 5, ints 4); which = 8: the accumulator
 * H-LU plan (hm_lu_opts.accumulate = 1; held pieces in the arena, doubles space 6), which = 9:
 * the same with wave overlap. rank_cap: 1..64, the capacity of the
 * low-rank leaves. threads: host threads of the H-LU planner (0: the hm_set_host_threads
 * setting; the plan does not depend on it). Replaces an earlier plan of S. HM_EINVAL on bad arguments or an
 * accumulator task graph, HM_EINTERNAL if the planner fails. */
int hm_structure_plan(hm_structure* S, int which, double eps, int rank_cap, int nrhs_max, int threads);

enum {
  HM_PLAN_LAUNCHES = 0,  /* {kind, begin, count, gy, gz, first, wave, side} int32 records, in
                            execution order; kind: 0 getrf, 1 trsm, 2 gemm, 3 copy, 4 stack,
                            5 core, 6 eval, 7 aca, 8 tensor-core gemm, 9 FP32 gemm (mixed
                            precision); first = 1 starts a phase (the launches of a phase are
                            independent); wave: the task-graph level of an H-LU launch (-1 in
                            the other plans); side = 1: a deferred rounded addition, which may run
                            at any time after the wave's other launches and before wave + 2 */
  HM_PLAN_GETRF = 1,     /* the micro-op descriptors of the batched kernels, laid out as the */
  HM_PLAN_TRSM = 2,      /* GetrfOp, TrsmOp, GemmOp, CopyOp, TruncOp and StackEntry structs  */
  HM_PLAN_GEMM = 3,      /* of the library's csrc/ops.h; one TRUNC record serves a stack and */
  HM_PLAN_COPY = 4,      /* a core launch; a launch covers records [begin, begin + count).   */
  HM_PLAN_TRUNC = 5,     /* Addresses are ((space + 1) << 60) | element offset, space 0 the  */
  HM_PLAN_ENTRIES = 6,   /* factor values, 1 scratch, 2 work vectors, 3 matrix values (int   */
                         /* spaces: 0 factor ranks, 1 pivots, 2 scratch ints, 3 matrix ranks) */
  HM_PLAN_LEAVES = 7,    /* per block-tree leaf, 10 int64: row cluster, col cluster, m, n,
                            low-rank (0/1), rank capacity, value offset (dense D or U, ld m),
                            V offset (ld n), rank index, pivot offset (-1: none)             */
  HM_PLAN_SIZES = 8,     /* one record of 9 int64: scratch doubles, scratch ints, value
                            doubles, ranks, pivots, rounded additions, waves, phases, arena
                            doubles (accumulator H-LU plans, else 0)                         */
  HM_PLAN_INSTANCES = 9, /* per instance, 5 int64: first leaf record, leaf records, value,
                            rank and pivot offsets (one instance unless batched)              */
  HM_PLAN_EVAL = 10,     /* EvalOp and AcaOp records of the assembly plan (kinds 6 and 7)     */
  HM_PLAN_ACA = 11
};

/* Host-side H-LU plan of count independent structures in one launch sequence (batching
 * across instances): wave w of every instance is expanded into the same phases, so that one
 * launch per kernel kind and phase serves all of them. The instances' values, ranks and
 * pivots are concatenated in the given order (value offsets rounded up to 32 doubles); the
 * leaf table lists every instance's leaves with those offsets added. The plan is kept in
 * S[0] (its tables as for hm_structure_plan). HM_EINVAL on bad arguments, a structure listed
 * twice or an accumulator task graph. */
int hm_structure_plan_lu_batch(hm_structure* const* S, int count, double eps, int rank_cap);
/* Read-only view of one table of the last plan of S: *data points into S and stays valid until
 * S is planned again or freed; *count records of *elem_bytes bytes. HM_EINVAL without a plan. */
int hm_structure_plan_table(const hm_structure* S, int table, const void** data, int64_t* count,
                            int64_t* elem_bytes);
/* Export (any pointer may be NULL):
 *   perm[n]                 original index of each permuted position
 *   clusters[nclusters*6]   lo, hi, son0, son1, level, parent (depth-first pre-order ids)
 *   leaves[nleaves*3]       row cluster, col cluster, admissible (block-tree pre-order)
 *   tasks[ntasks*4]         type (0 lu, 1 mul / add_upd, 2 trsl, 3 trsu, 4 shift_upd, 5 apply_upd),
 *                           c1, c2, c3 (-1 unused)
 *   edges[nedges*2]         src, dst task indices
 *   levels[ntasks]          longest-path level of each task */
int hm_structure_export(const hm_structure* S, int64_t* perm, int32_t* clusters, int32_t* leaves,
                        int32_t* tasks, int32_t* edges, int32_t* levels);
void hm_structure_free(hm_structure* S);

#ifdef __cplusplus
}
#endif

#endif /* HMGB300_H */
