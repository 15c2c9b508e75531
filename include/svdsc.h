/*
 * svdsc — truncated SVD on one GB300 GPU (sm_103a).
 *
 * Computes the k largest singular triplets of a sparse (CSR) or dense matrix A
 * (m x n):  A ~ U_k diag(S) V_k^T  with S descending and U_k, V_k orthonormal
 * (the problem of Eq. (1) of the svds-C paper, arXiv 2405.18966, Sec. 2).  The
 * method is the one Sec. 2.1 describes: Lanczos bidiagonalization (Alg. 1) with
 * full re-orthogonalization of every new vector (here: two classical
 * Gram-Schmidt passes, "CGS2"), the Ritz residual test of Eq. (4), and the
 * augmented restart of Eq. (5)-(7) / Alg. 2.  Options (svdsc_options): the
 * k smallest triplets instead, partial re-orthogonalization instead of the
 * full one, and a mixed-precision form; a batched form solves many matrices
 * in one launch.  Every step runs in this library's CUDA kernels on the
 * device; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *   - Dense matrices are column-major with a leading dimension (the paper's
 *     `mat` struct, Sec. 2.3).  Vectors are contiguous.
 *   - "device pointer" means memory the current CUDA device can address
 *     (cudaMalloc / torch CUDA tensors); "host pointer" means ordinary or
 *     pinned host memory.  Flags named *on_device select which.
 *   - Return value: 0 (SVDSC_OK) on success, SVDSC_NOT_CONVERGED (+1) when the
 *     outputs are written but not every residual reached tol, a negative
 *     SVDSC_ERR_* code otherwise (outputs then untouched).  svdsc_strerror
 *     gives a message.  No entry point aborts the process.
 *   - All work is issued on the stream given to svdsc_create (NULL = the
 *     legacy default stream); solve synchronizes that stream before it
 *     returns.  A context must not be used by two host threads at once.
 */
#ifndef SVDSC_H
#define SVDSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SVDSC_OK 0
#define SVDSC_NOT_CONVERGED 1
#define SVDSC_ERR_ARG (-1)        /* bad argument (NULL pointer, k < 1, tol <= 0, ...) */
#define SVDSC_ERR_SIZE (-2)       /* t = k+p does not fit: need t <= m and t+1 <= n */
#define SVDSC_ERR_CSR (-3)        /* row pointers not monotone or a column index out of range */
#define SVDSC_ERR_NOMEM (-4)      /* device or host allocation failed */
#define SVDSC_ERR_CUDA (-5)       /* a CUDA runtime call failed */
#define SVDSC_ERR_TIMEOUT (-6)    /* a bounded device-side wait ran out */
#define SVDSC_ERR_NONFINITE (-7)  /* NaN or Inf met in A or in a Lanczos vector */

enum svdsc_format { SVDSC_CSR = 0, SVDSC_DENSE = 1 };
enum svdsc_precision { SVDSC_FP64 = 0, SVDSC_MIXED = 1 };
enum svdsc_value_type { SVDSC_F64 = 0, SVDSC_F32 = 1 };
enum svdsc_which { SVDSC_LARGEST = 0, SVDSC_SMALLEST = 1 };
enum svdsc_reorth { SVDSC_REORTH_FULL = 0, SVDSC_REORTH_PARTIAL = 1 };

/*
 * Input matrix (read-only, owned by the caller; svdsc_create copies it, so
 * the caller may free it as soon as create returns).
 * CSR (format = SVDSC_CSR), following the paper's `mat_csr` (Sec. 2.3):
 *   index_base 0 or 1 (the paper's column indices start at 1);
 *   either row_ptr (m+1 entries, 3-array CSR) or row_begin/row_end (m entries
 *   each, the MKL 4-array form pointerB/pointerE the paper uses);
 *   col_idx (nnz entries, int32), values (nnz entries, double or float as
 *   value_type says).  nnz = row_ptr[m] - row_ptr[0] for 3-array input and is
 *   taken from the nnz field for 4-array input (the extent of col_idx/values).
 *   Duplicate (row, col) entries are summed by the products.
 * Dense (format = SVDSC_DENSE): `dense` column-major m x n, leading dimension
 *   ld >= m, double only.
 * on_device = 1: every pointer above is a device pointer; 0: host pointers.
 */
typedef struct svdsc_matrix {
    int32_t format;
    int32_t index_base;
    int64_t m, n, nnz;
    const int64_t *row_ptr;
    const int64_t *row_begin;
    const int64_t *row_end;
    const int32_t *col_idx;
    const void *values;
    int32_t value_type;
    int32_t on_device;
    const double *dense;
    int64_t ld;
} svdsc_matrix;

/*
 * Options.  precision: SVDSC_FP64 runs every product, projection, norm and the
 * projected SVD in FP64.  SVDSC_MIXED keeps FP32 copies of A and of the
 * Lanczos basis for the sparse products and the first CGS pass (the second
 * pass, all norms, the projected SVD and the residual test stay FP64).
 * seed selects the counter-based normal generator used for v_1 when no start
 * vector is given and for replacement vectors after a breakdown.
 * which: SVDSC_LARGEST (0) computes the k largest triplets (Alg. 2);
 * SVDSC_SMALLEST (1) the k smallest: the projected matrix's Ritz values
 * approximate both ends of the spectrum (Sec. 2), and the restart then keeps
 * the k smallest Ritz triplets instead of the k largest.  SVDSC_SMALLEST needs
 * m >= n (pass A^T for a wide matrix); svdsc_create returns SVDSC_ERR_ARG
 * otherwise.  The batched form supports SVDSC_LARGEST only.
 * reorth: SVDSC_REORTH_FULL (0, default) re-orthogonalizes every Lanczos
 * vector against all earlier ones with two classical Gram-Schmidt passes, the
 * full re-orthogonalization of Sec. 2.1.  SVDSC_REORTH_PARTIAL (1) is the
 * partial scheme of lansvd (Table 1): estimates of each new vector's inner
 * products with the earlier ones, propagated from the Lanczos relations
 * A V = U T and A^T U = V T^T + beta v e^T, send a vector (and the next of its
 * kind) to the same CGS2 only when an estimate exceeds eps^(3/4); the basis
 * is then orthogonal to ~eps^(3/4) (|u_i^T u_j| <~ 1e-11) instead of ~eps.
 * Fewer bytes, less robust; the batched form supports SVDSC_REORTH_FULL only.
 * block: 0 or 1 runs the single-vector method above; 2, 4, 8 or 16 runs its
 * block form (block Lanczos bidiagonalization of Golub, Luk & Overton 1981,
 * carried through the full re-orthogonalization of Sec. 2.1 and the
 * augmented restart of Alg. 2): each step forms b Lanczos vectors with one
 * sparse product A X (X n x b), re-orthogonalizes them together (two block
 * classical Gram-Schmidt passes) and orthonormalizes them within the block
 * (two Cholesky QR passes; a block that is numerically rank-deficient or
 * ill-conditioned is redone column by column).  The projected matrix is upper
 * triangular with bandwidth b; the residual of Eq. (4) becomes
 * ||F^T Uh(t-b:t, j)|| / sigma_j with F the b x b block that couples the last
 * block to the residual block.  The subspace is t0 = b ceil((k+p)/b) columns
 * in the first pass and t1 = k + b ceil(p/b) after each restart.  CSR input,
 * SVDSC_LARGEST and SVDSC_REORTH_FULL only; FP64 or mixed precision.
 */
typedef struct svdsc_options {
    int32_t precision;
    int32_t timing;        /* 1: time every kernel launch with CUDA events (fills svdsc_info.ms) */
    uint64_t seed;
    int32_t restart_gemm;  /* 0: tensor cores (svdsc_gemm modes 0/1, default); 1: FP64 FMA on CUDA cores */
    int32_t batch_cluster; /* batched form: CTAs (one cluster) per matrix, 1, 2, 4 or 8; 0 = automatic */
    int32_t which;         /* SVDSC_LARGEST (default) or SVDSC_SMALLEST */
    int32_t reorth;        /* SVDSC_REORTH_FULL (default) or SVDSC_REORTH_PARTIAL */
    int32_t block;         /* Lanczos block size: 0 or 1 (single vector, default), 2, 4, 8 or 16 */
    int32_t batch_handoff; /* batched form, hand-off to a second launch: 0 automatic, -1 never,
                              h > 0 once h clusters of the first launch are idle */
    int32_t batch_order;   /* batched form, queue order: 0 = estimated cost for the first solve, then
                              the SM cycles (cycles x CTAs) each matrix took in the previous solve of
                              the batch; 1 = the estimate always */
    int32_t batch_lead;    /* batched form, lead clusters of 8 CTAs beside smaller ones: 0 automatic,
                              -1 none, n > 0 (see svdsc_batch_lead) */
} svdsc_options;

/* Kernel categories of svdsc_info.ms / launches / bytes / flops. */
enum svdsc_phase {
    SVDSC_PH_SPMV = 0,     /* products with A and A^T (Alg. 1) */
    SVDSC_PH_GEMV_T = 1,   /* CGS projections h = W^T w */
    SVDSC_PH_GEMV_N = 2,   /* CGS updates w -= W h */
    SVDSC_PH_VEC = 3,      /* ordered reductions, norms, scaling (finalize) */
    SVDSC_PH_SVD = 4,      /* projected SVD (Alg. 2) */
    SVDSC_PH_GEMM = 5,     /* restart / output basis update (Alg. 2) */
    SVDSC_PH_OTHER = 6,    /* residual test, T rebuild, sign rule, copies */
    SVDSC_NUM_PHASES = 8
};

/* Per-solve report (all fields written by svdsc_solve). */
typedef struct svdsc_info {
    int32_t converged;     /* 1 if every res_j < tol */
    int32_t nconv;         /* number of j < k with res_j < tol */
    int32_t restarts;      /* augmented restarts performed */
    int32_t breakdowns;    /* Lanczos vectors replaced by random ones */
    int64_t n_matvec;      /* products with A or A^T (2t + 2R(t-k)) */
    int64_t n_steps;       /* Lanczos vectors formed */
    int64_t n_launches;    /* CUDA kernels this solve launched */
    double anorm_est;      /* largest alpha, beta or sigma seen (estimate of ||A||_2) */
    double beta_t;         /* T(t, t+1) of the last projected matrix */
    int32_t t;             /* subspace dimension used */
    int32_t reserved;
    /* Per phase (index: enum svdsc_phase).  launches, algorithmic bytes and
     * flops are always counted; ms only when the context was created with
     * timing = 1 (summed CUDA-event durations of the launches).  Algorithmic
     * bytes count each operand once: CSR SpMV 12 nnz + 20 rows + 8 cols (+8 rows
     * for the fused axpy), FP32 form 8 nnz + ...; GEMV-T 8 len ncols + 8 len;
     * GEMV-N 8 len ncols + 16 len (FP32 shadow: 4 len ncols instead of 8);
     * restart GEMM 8 rows (t + k). */
    double ms[SVDSC_NUM_PHASES];
    int64_t launches[SVDSC_NUM_PHASES];
    double bytes[SVDSC_NUM_PHASES];
    double flops[SVDSC_NUM_PHASES];
    int64_t n_reorth;      /* Lanczos vectors re-orthogonalized against their predecessors (CGS2) */
} svdsc_info;

typedef struct svdsc_ctx svdsc_ctx;

/*
 * Copies A to the device and prepares it: converts CSR to 0-based 3-array
 * form, validates it (SVDSC_ERR_CSR), builds CSR(A^T) and the row-length bins
 * of both.  `stream` is a cudaStream_t (or NULL).  On success *out owns all
 * device memory of the solver until svdsc_destroy.
 */
int svdsc_create(svdsc_ctx **out, const svdsc_matrix *A, const svdsc_options *opt,
                 void *stream);

/*
 * Alg. 2: k largest singular triplets (k smallest if the context was created
 * with which = SVDSC_SMALLEST).
 *   t = k + p (p < 0: t = max(15, 3k), Alg. 2); needs 1 <= k <= t,
 *   t <= m and t + 1 <= n, k <= 256 and t <= 512 (t <= 448 with the
 *   tensor-core restart GEMM) (SVDSC_ERR_SIZE otherwise).
 *   tol: relative residual tolerance of Eq. (4), > 0 (the paper uses 1e-10).
 *   maxit >= 1: number of projected-SVD-and-test rounds; the last round never
 *   restarts (at most maxit - 1 restarts).
 *   v0: start vector (n entries, host or device per v0_on_device) or NULL for
 *   the seeded random draw; in the block form (options.block = b > 1) a
 *   start block of n x b entries (column-major, ld n), or NULL for draws
 *   0..b-1.  Block form sizes: t0 = b ceil(t/b), t1 = k + b ceil((t-k)/b),
 *   needs k + b <= t1, max(t0, t1) <= m, max(t0, t1) + b <= n and
 *   max(t0, t1) <= 448.
 *   Outputs (written on success or SVDSC_NOT_CONVERGED): S[k] descending
 *   (ascending for SVDSC_SMALLEST: the smallest first),
 *   U (m x k, column-major, ldu >= m), V (n x k, ldv >= n), res[k] (may be
 *   NULL) with res_j = |beta_t Uh(t,j)| / sigma_j.  Each pair (u_j, v_j) is
 *   signed so that the entry of v_j with the largest magnitude (lowest index
 *   on ties) is positive.  out_on_device selects device or host outputs.
 *   info may be NULL.
 */
int svdsc_solve(svdsc_ctx *ctx, int k, int p, double tol, int maxit,
                const double *v0, int v0_on_device,
                double *S, double *U, int64_t ldu, double *V, int64_t ldv, double *res,
                int out_on_device, svdsc_info *info);

/* Frees every device and host resource of ctx (NULL is a no-op). */
int svdsc_destroy(svdsc_ctx *ctx);

/* Static message for a status code. */
const char *svdsc_strerror(int status);

/* ---------------------------------------------------------------------------
 * Component entry points (one hot-path step each, on device pointers, on the
 * context's stream).  They exist so each kernel can be checked and timed on
 * its own; svdsc_solve does not need them.
 */

/*
 * y = A x (trans = 0, Alg. 1, x: n, y: m) or y = A^T x (trans = 1,
 * Alg. 1, x: m, y: n), minus coef * z when z != NULL (the fused
 * "- beta_i u_i" / "- alpha_i v_i" term).  FP64 vectors; in MIXED contexts the
 * sparse product itself runs in FP32 as in the solver.  Device pointers.
 */
int svdsc_matvec(svdsc_ctx *ctx, int trans, const double *x, const double *z, double coef,
                 double *y);

/*
 * Full re-orthogonalization of Sec. 2.1 as CGS2: w <- (I - W W^T)(I - W W^T) w
 * for W = the first `ncols` columns of a column-major len x ncols basis with
 * leading dimension ldw, followed by the norm: *norm_out (device) = ||w||_2.
 * len must be m or n of the context (its chunking is prepared for those),
 * ncols <= t_max (the largest t the context has been solved or prepared for,
 * see svdsc_reserve).  W, w, norm_out: device pointers; w must not alias W.
 */
int svdsc_cgs2(svdsc_ctx *ctx, int64_t len, int64_t ncols, const double *W, int64_t ldw,
               double *w, double *norm_out);

/*
 * Self-test of the bounded device-side waits (the paper has no counterpart).
 * Every spin-wait in the library's kernels gives up after an iteration limit,
 * records the timeout in the context's status block and lets its kernel
 * return, so a wait that can never be satisfied ends in SVDSC_ERR_TIMEOUT
 * instead of a hung GPU.  This call makes one such wait run out on purpose:
 * kind 0, the grid barrier of the multi-CTA Jacobi SVD (a cooperative launch
 * of 4 CTAs that each wait for a fifth arrival); kind 1, the mbarrier wait of
 * the tensor-core GEMM (nothing ever arrives).  It takes a few seconds (the
 * real limits), returns SVDSC_ERR_TIMEOUT when the wait ran out as designed
 * (SVDSC_OK would mean it did not), and leaves the context usable.
 */
int svdsc_selftest_wait(svdsc_ctx *ctx, int kind);

/*
 * Projected SVD of Alg. 2 on the device: T is t x t (ldt >= t), any
 * square matrix (the solver passes the upper-triangular T(1:t,1:t)).  Outputs
 * S[t] descending, Uh (t x t, ld t) and Vh (t x t, ld t) with T = Uh diag(S)
 * Vh^T.  FP64 one-sided Jacobi.  Device pointers; t <= t_max.
 */
int svdsc_small_svd(svdsc_ctx *ctx, int t, const double *T, int64_t ldt, double *S, double *Uh,
                    double *Vh);

/* Sizes the context's workspace for subspace dimension t (solve does this
 * itself; the component entry points need it first). */
int svdsc_reserve(svdsc_ctx *ctx, int t);

/*
 * Restart / output basis update of Alg. 2 on the tensor cores:
 * C = W Q with W rows x t (leading dimension ldw), Q t x k (ldq), C rows x k
 * (ldc), all column-major FP64 device arrays; C must not overlap W.
 *   mode 0 (FP64 form): on power-of-two row (W) and column (Q) scales every
 *   entry becomes a fixed-point integer below 2^54, cut into eight balanced
 *   base-128 digits in [-64, 63] (an Ozaki-style error-free split); the 36
 *   digit products of weight s + s' <= 7 run as BF16 tcgen05 MMAs into eight
 *   TMEM accumulators, one per weight, whose FP32 sums are exact integers;
 *   the epilogue recombines them exactly in integer arithmetic before one
 *   FP64 rounding.  The dropped products (weight >= 8) and the 2^-54
 *   truncation keep the error inside the bound of an FP64 GEMM (needs
 *   t <= 448).
 *   mode 1 (mixed form): W rounded to FP32 and Q are cut into three BF16 pieces
 *   each; the six leading piece products accumulate in FP32 (about FP32
 *   accuracy).
 * Needs t <= t_max of the context (svdsc_reserve) and k <= t.  Runs on the
 * context's stream and synchronizes it.
 */
int svdsc_gemm(svdsc_ctx *ctx, int mode, int64_t rows, int t, int k, const double *W, int64_t ldw,
               const double *Q, int64_t ldq, double *C, int64_t ldc);

/*
 * The same CGS2 as svdsc_cgs2 (w <- (I - W W^T)^2 w, then *norm_out = ||w||_2),
 * for callers that cannot allocate device memory: no context, and no
 * cudaMalloc, cudaFree or allocating library call at any point.  Callers of
 * this kind include code running while a framework's caching allocator holds
 * all device memory, serving or real-time loops with a memory budget fixed up
 * front (cudaMalloc can synchronize the device and can fail mid-run), and
 * hosts that only hand a library pre-allocated buffers.  The paper has no
 * counterpart; it exists only for such callers.
 *   Scratch: one file-scope __device__ array of 4.3 MB (532,992 doubles) that
 *   every CUDA context loading this library holds until the process exits.
 *   Limits: ncols <= 512 and len <= 4,194,304 (at most 1,024 row chunks of
 *   4,096); larger sizes return SVDSC_ERR_SIZE before any GPU work.
 *   The first call in a CUDA context looks up the array's device address
 *   (cudaGetSymbolAddress, with that context current) and remembers it under
 *   the context's unique ID; a new context (for example after
 *   cudaDeviceReset) gets its own lookup on its first call.  Make that first
 *   call outside any stream capture: while `stream` is being captured, a
 *   context that has not called before gets SVDSC_ERR_ARG.  Every call shares
 *   the array and overwrites what it reads, so calls whose GPU work overlaps
 *   (two streams, two host threads) race and give wrong results; serialize
 *   them.
 *   W (len x ncols, leading dimension ldw, even, 16-byte aligned), w (len,
 *   16-byte aligned, overwritten), norm_out (one double): device pointers.
 *   stream: cudaStream_t or NULL.  The call only enqueues the work on stream
 *   and returns; results are ready once the stream reaches it.
 */
int svdsc_cgs2_noalloc(int64_t len, int64_t ncols, const double *W, int64_t ldw, double *w,
                       double *norm_out, void *stream);

/* ---------------------------------------------------------------------------
 * Batched form: many independent truncated SVDs (uneven shapes and k) solved
 * in one persistent kernel launch (plus a lead launch and a hand-off launch
 * when they are on), replayed from a
 * CUDA graph.  Thread-block clusters (1-8 CTAs) take matrices from a work
 * queue (largest cost first: estimated from the sizes for the first solve,
 * then, unless options.batch_order = 1, the SM cycles each matrix took in
 * the previous solve of the same batch) and run Alg. 2 for each.  Hand-off:
 * once the queue is empty and a set number of clusters are idle, the matrices
 * still running stop at their next restart boundary (after the restart GEMM
 * of Eq. 6) and a second launch of 8-CTA clusters resumes them from the saved
 * state (U~_k, V~_k, v_{k+1}, sigma, rho, counters), so the last matrices run
 * on more SMs than the first launch's cluster size gives them.  Precision is the mixed form (FP32
 * CSR values, FP32 SpMV and first CGS pass, FP64 second pass, norms, projected
 * SVD and residual test, FP32 restart GEMM); options.precision must be
 * SVDSC_MIXED.  Limits per matrix: CSR input, 1 <= k <= 48, t = k + p <= 80
 * (p < 0: t = max(15, 3k)), t <= m, t + 1 <= n (SVDSC_ERR_SIZE otherwise).
 * Matrix b uses seed options.seed + b for its random start vector.
 */
typedef struct svdsc_batch svdsc_batch;

/* Copies and prepares all nb matrices (as svdsc_create does), sizes one
 * workspace slot per resident CTA, and runs the autotuner: for each
 * matrix-shape class (average row length and row count of A and of A^T, basis
 * length and size) it times the SpMV lanes-per-row candidates 1..32 and the
 * CGS projection column tiles 1, 2, 4 on all SMs and keeps the fastest
 * (cached for the process).  Work runs on an internal stream; `stream` is
 * ignored (the graph needs a capturable stream). */
int svdsc_batch_create(svdsc_batch **out, int nb, const svdsc_matrix *As, const int *k, const int *p,
                       const svdsc_options *opt, void *stream);

/* Solves every matrix.  S[b] (k_b), U[b] (m_b x k_b, ld m_b), V[b] (n_b x k_b,
 * ld n_b), res[b] (k_b, or res / res[b] NULL): device pointers when
 * out_on_device, else host.  infos (nb entries, may be NULL) report per-matrix
 * convergence, restarts and products (reserved = the matrix's error code).
 * Returns the most severe per-matrix status. */
int svdsc_batch_solve(svdsc_batch *b, double tol, int maxit, double *const *S, double *const *U,
                      double *const *V, double *const *res, int out_on_device, svdsc_info *infos);

/* The autotuner's choice for matrix i and the total tuning time. */
int svdsc_batch_tuning(const svdsc_batch *b, int i, int *lanes_A, int *lanes_AT, int *gemv_cols,
                       double *tune_ms);

/* CTAs per matrix (thread-block cluster size: the rows of A, A^T and of the
 * bases are split across them) and the number of clusters of the persistent
 * launch.  Automatic choice: the smallest power of two <= 8 for which the
 * costliest matrix (estimated by the cost of one Lanczos pass), run on one
 * cluster, takes at most its share of the batch's estimated work. */
int svdsc_batch_layout(const svdsc_batch *b, int *cluster_size, int *clusters);

/* The hand-off set-up (each output may be NULL): the idle-cluster count that
 * triggers it (0: no hand-off), the second launch's cluster size (8) and
 * cluster count, and the number of matrices the last solve handed off (read
 * from the device: call after svdsc_batch_solve has returned).  Automatic
 * (options.batch_handoff = 0): on when the first launch's clusters are
 * smaller than 8 CTAs and more numerous than the second launch's, with the
 * threshold at which no more matrices are running than the second launch
 * has clusters.  A handed-off matrix reports cluster 100000 + its cluster in
 * the second launch in svdsc_batch_profile. */
int svdsc_batch_handoff(const svdsc_batch *b, int *idle_threshold, int *cluster_size, int *clusters,
                        int *handed_off);

/* The lead launch (each output may be NULL): its cluster size (8) and
 * cluster count (0: none).  When the main launch's clusters are smaller than
 * 8 CTAs, a lead launch of a few 8-CTA clusters starts first; the main launch
 * follows as soon as every lead CTA runs (programmatic dependent launch) and
 * gives up the SMs they hold.  Lead cluster i takes queue position i (the
 * costliest matrices), then shares the queue; lead clusters never hand off.
 * Automatic (options.batch_lead = 0): one, when the batch has more matrices
 * than the main launch has clusters.  A matrix solved by a lead cluster
 * reports cluster 200000 + its lead cluster in svdsc_batch_profile. */
int svdsc_batch_lead(const svdsc_batch *b, int *cluster_size, int *clusters);

/* Per-matrix profile of the last batch solve (arrays of nb entries, each may
 * be NULL): SM clock cycles of the whole solve, of the projected SVDs and of
 * the Lanczos segments on the cluster's first CTA, and the cluster that
 * solved the matrix. */
int svdsc_batch_profile(const svdsc_batch *b, int64_t *cycles_total, int64_t *cycles_svd,
                        int64_t *cycles_lbp, int32_t *cluster);

/* Per-matrix SM clock cycles of the last batch solve by phase, on the
 * cluster's first CTA (nb x 5 entries, row-major): [0] sparse products,
 * [1] the FP32 CGS pass, [2] the FP64 CGS pass with the norm, [3] the
 * normalization / breakdown test / scaling, [4] the restart and output
 * GEMMs with the sign rule.  Each phase includes its cluster barriers. */
int svdsc_batch_phase_cycles(const svdsc_batch *b, int64_t *cycles);

int svdsc_batch_destroy(svdsc_batch *b);

/* One call: create, solve, destroy. */
int svdsc_solve_batched(int nb, const svdsc_matrix *As, const int *k, const int *p, double tol, int maxit,
                        double *const *S, double *const *U, double *const *V, double *const *res,
                        int out_on_device, const svdsc_options *opt, svdsc_info *infos);

#ifdef __cplusplus
}
#endif
#endif /* SVDSC_H */
