/*
 * nmf_gb300.h - C ABI of the single-GPU (sm_103a) ANLS-NMF / BPP library.
 *
 * The library computes the per-iteration hot path of alternating nonnegative
 * least squares NMF with block principal pivoting, after Kannan, Ballard and
 * Park, "A High-Performance Parallel Algorithm for Nonnegative Matrix
 * Factorization" (arXiv 1509.09313):
 *
 *   minimise f(W, H) = ||A - W H||_F^2 over W >= 0 (m x k), H >= 0 (k x n)
 *   (Eq. 1), by the two-block scheme of Eq. 2 / Alg. 1: each iteration updates
 *   W from (H H^T, A H^T), then H from (W^T W, W^T A), every row of W and
 *   column of H being one NLS problem (Eq. 3) solved by BPP (Sec. 4.2).
 *
 * Conventions for every call:
 *   - All matrices are row-major. H is always passed and stored as H^T
 *     (n x k), so that each right-hand side of either half-step is one
 *     contiguous k-vector.
 *   - Pointers documented as "device" must point to memory the current CUDA
 *     device can read/write (cudaMalloc'd, or managed). "host" pointers are
 *     ordinary CPU memory. The library never frees memory it did not allocate.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls are asynchronous on that stream unless stated otherwise.
 *   - Arguments are validated on the host before anything is launched; an
 *     invalid argument returns NMF_ERR_INVALID_ARG and launches nothing.
 *     No call aborts the process, traps on the device or spins without bound.
 *   - 1 <= k <= NMF_MAX_K.
 */
#ifndef NMF_GB300_H
#define NMF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NMF_MAX_K 128

typedef enum nmf_status {
    NMF_OK = 0,
    NMF_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported mode */
    NMF_ERR_CUDA = 2,          /* a CUDA runtime call or launch failed */
    NMF_ERR_OOM = 3,           /* device allocation failed */
    NMF_ERR_NOT_CONVERGED = 4, /* a BPP solve hit its exchange-round cap */
    NMF_ERR_SINGULAR_GRAM = 5, /* a passive-set system was singular even in FP64 */
    NMF_ERR_NONFINITE = 6      /* NaN/Inf met in an input or a result */
} nmf_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *nmf_status_str(nmf_status s);

/* CUDA kernels this process has launched through the library so far (every
 * entry point and handle; host-side counter, no synchronisation). */
int64_t nmf_kernel_launches(void);

/* FP32 FMA throughput of the current device (a measurement utility of this
 * library, no counterpart in the paper): the FP32 SIMT kernels' arithmetic
 * is quoted against this measured rate rather than a nominal one. Runs one
 * untimed and `launches` timed launches (1..100000; each ~3e11 flops) of a
 * kernel in which every thread advances eight independent FMA chains, scalar
 * FFMA (packed = 0) or packed FP32x2 FFMA2 (packed = 1), on all SMs; times
 * them with CUDA events on `stream` and writes the rate (flop/s, one FMA =
 * 2 flops) to *flops_per_s (host). Synchronises `stream`. Changes no GPU
 * setting. */
nmf_status nmf_probe_fp32_fma(int32_t packed, int32_t launches, double *flops_per_s,
                              void *stream);

/* Arithmetic used for the two m*n*k products (A H^T and W^T A) and for the
 * objective:
 *   NMF_PREC_FP32   plain FP32 FMAs on the SIMT pipes;
 *   NMF_PREC_BF16X3 tensor cores (tcgen05): each FP32 operand is split into a
 *                   BF16 head and a BF16 tail and three products are summed in
 *                   FP32 (head*head + head*tail + tail*head). */
typedef enum nmf_precision { NMF_PREC_FP32 = 0, NMF_PREC_BF16X3 = 1 } nmf_precision;

/* ===================================================================== *
 * Stand-alone local kernels. These are the three local tasks the paper times
 * separately (Sec. 6.2, "Time Breakdown"): MM, Gram and NLS.
 * ===================================================================== */

/* Gram (Alg. 1: H H^T and W^T W).
 *   X      device, rows x k float32 row-major (X = H^T gives H H^T, X = W gives
 *          W^T W).
 *   G      device, k x k float64 output, the full symmetric matrix X^T X.
 * FP32 products summed in FP32 over short row tiles, tiles summed in FP64 in a
 * fixed order (bitwise reproducible). rows = 0 gives G = 0. */
nmf_status nmf_gram(const float *X, int64_t rows, int32_t k, double *G, void *stream);

/* Dense products of Alg. 1 (the "MM" task).
 *   A      device, m x n float32 row-major, leading dimension lda >= n.
 *   F      device, float32 row-major factor:
 *            trans = 0: F = H^T (n x k), out = A H^T       (m x k);
 *            trans = 1: F = W   (m x k), out = A^T W = (W^T A)^T (n x k).
 *   out    device float32 row-major, no aliasing with A or F.
 *   precision  an nmf_precision value. NMF_PREC_BF16X3 reads A with TMA and
 *          needs a 16-byte-aligned A with lda a multiple of 4 (else
 *          NMF_ERR_INVALID_ARG); it also needs k <= NMF_MAX_K only.
 * Zero-sized m or n is allowed (out is zero-filled when the contraction length
 * is 0). */
nmf_status nmf_mm_dense(const float *A, int64_t m, int64_t n, int64_t lda, const float *F,
                        int32_t k, int32_t trans, int32_t precision, float *out, void *stream);

/* Sparse product with a CSR matrix (the "MM" task, sparse case of Sec. 4.3):
 *   out (rows x k) = S F, S given by rowptr (rows+1, int64, rowptr[0] = 0),
 *   colidx (int32, in [0, cols)), vals (float32), all device; F (cols x k) device.
 * For A H^T pass the CSR of A and F = H^T; for (W^T A)^T pass the CSR of A^T
 * and F = W (nmf_csr_transpose builds it). Empty rows give zero rows. */
nmf_status nmf_mm_csr(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                      int64_t rows, int64_t cols, const float *F, int32_t k, float *out,
                      void *stream);

/* CSR transpose on the device: (rowptr, colidx, vals) of an m x n matrix with
 * nnz entries -> (t_rowptr (n+1), t_colidx (nnz), t_vals (nnz)) of its
 * transpose, columns of every output row in increasing order (deterministic).
 * All pointers device; output buffers caller-allocated. */
nmf_status nmf_csr_transpose(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                             int64_t m, int64_t n, int64_t nnz, int64_t *t_rowptr,
                             int32_t *t_colidx, float *t_vals, void *stream);

/* Batched NLS by block principal pivoting (Eq. 3, Eq. 4, Sec. 4.2): for every
 * row b_j of B,   x_j = argmin_{x >= 0} 0.5 x^T G x - b_j^T x,
 * i.e. Eq. 3 in normal-equations form with G = C^T C and b_j = C^T (rhs j).
 * Exchange rules: full exchange of all infeasible indices while their number
 * drops, up to three further full exchanges otherwise, then single exchange
 * of the largest infeasible index. Indices with G_ii <= 0 stay active. */
typedef struct nmf_nls_desc {
    int32_t k;                 /* problem size, 1..NMF_MAX_K */
    int64_t nrhs;              /* number of right-hand sides (>= 0) */
    const double *G;           /* device, k x k float64, symmetric PSD */
    const float *B;            /* device, nrhs x k float32 (one RHS per row) */
    float *X;                  /* device, nrhs x k float32 output; must not
                                  overlap B (NMF_ERR_INVALID_ARG) */
    const uint64_t *passive_in;/* device, nullable: nrhs x ceil(k/64) bitmasks
                                  (bit i of word i/64 set = index i passive);
                                  non-null selects a warm start */
    uint64_t *passive_out;     /* device, nullable: final passive sets, same layout */
    int32_t *rounds_out;       /* device, nullable: exchange rounds per RHS */
    int8_t *status_out;        /* device, nullable: per-RHS nmf_status */
    int32_t max_rounds;        /* exchange-round cap per RHS (>= 0) */
} nmf_nls_desc;

/* Runs asynchronously on `stream`, then waits for it and returns the worst
 * per-RHS status (NMF_OK, NMF_ERR_NOT_CONVERGED or NMF_ERR_SINGULAR_GRAM).
 * A failing right-hand side never changes the others' results. Uses a small
 * internal device workspace (stream-ordered allocation, freed on return). */
nmf_status nmf_nls_bpp(const nmf_nls_desc *d, void *stream);

/* Launch-shape autotuner for the batched solve (an interface of this library,
 * no counterpart in the paper): times the solve kernels' candidate shapes
 * (warps per CTA x right-hand sides per grab of the work counter, with the
 * group-tile pass mode of the current shape, and without the pass when that
 * mode is 1) on this batch and keeps the fastest for d->k; every later solve
 * of that k in the process (nmf_nls_bpp, handles) uses it. All candidates
 * give bit-identical results. X
 * receives the solution; passive_out, rounds_out and status_out are not
 * written. Synchronises `stream`; *warps, *chunk and *group (host, nullable)
 * get the chosen shape. */
nmf_status nmf_nls_bpp_tune(const nmf_nls_desc *d, void *stream, int32_t *warps, int32_t *chunk,
                            int32_t *group);

/* Sets the launch shape of every later solve of this k in the process, as the
 * tuner would (an interface of this library): warps per CTA 1..16 (the FP64
 * solves use at most 8), right-hand sides per grab of the work counter
 * 1..1024, and the group-tile pass of FP32 half-steps (right-hand sides whose
 * first candidate partition is all usable indices are solved together by
 * tile products with the preparation's inverse; the rest go to the per-warp
 * solves): group = 0 off, 1 on the SIMT pipes, 2 on the tensor cores (k <=
 * 112). Warps, chunk and groups 0 and 1 do not change the results; group 2
 * gives them to FP32 solve accuracy, not the same bits. Default {8, 8, 2}
 * for 65 <= k <= 112, {8, 8, 1} otherwise. Host-side only;
 * NMF_ERR_INVALID_ARG outside these ranges. */
nmf_status nmf_nls_bpp_set_shape(int32_t k, int32_t warps, int32_t chunk, int32_t group);

/* Reads the launch shape solves of this k use (host pointers, nullable). */
nmf_status nmf_nls_bpp_get_shape(int32_t k, int32_t *warps, int32_t *chunk, int32_t *group);

/* Allocation-free variant of nmf_nls_bpp (no counterpart in the paper; an
 * interface of this library). Same arguments, computation and results as
 * nmf_nls_bpp, but it never allocates device memory, for callers that cannot
 * call cudaMalloc: code under a memory manager that owns all device memory
 * (a framework's caching allocator or a fixed pool), latency-critical loops
 * where cudaMalloc / cudaFree may synchronise the device, and programs that
 * must not grow their device footprint after start-up. The caller supplies
 * every input and output buffer, as for nmf_nls_bpp.
 *   - Workspace: one fixed array of NMF_NOALLOC_SCRATCH_BYTES compiled into
 *     the library; every GPU that loads the library holds it until exit.
 *   - k > NMF_NOALLOC_MAX_K returns NMF_ERR_INVALID_ARG and launches nothing;
 *     nrhs is not limited.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *     The address is kept for the life of the process: destroying the
 *     device's primary context after that call (cudaDeviceReset) is not
 *     supported, since later calls would use the old address.
 *   - All calls share the one array and it keeps the last call's contents:
 *     calls that overlap on the GPU (for example on two streams at once)
 *     race and corrupt each other's results. Keep them ordered.
 *   - Waits for `stream` and returns the worst per-RHS status. */
#define NMF_NOALLOC_MAX_K 128
#define NMF_NOALLOC_SCRATCH_BYTES (272 * 1024)
nmf_status nmf_nls_bpp_noalloc(const nmf_nls_desc *d, void *stream);

/* One MU step (Eq. 5) of the rows of X (rows x k, float32, device, updated
 * in place), with G (k x k float64, the Gram of the fixed factor) and R (rows x k
 * float32, its right-hand sides: A H^T for W, (W^T A)^T for H^T):
 *   x_ij <- x_ij R_ij / (X G)_ij,  every (X G)_ij from the X before the step;
 * x_ij is left unchanged where (X G)_ij <= 0. Asynchronous on `stream`. */
nmf_status nmf_update_mu(int32_t k, int64_t rows, const double *G, const float *R, float *X,
                         void *stream);

/* One HALS sweep (Eq. 6) of the rows of X with the same arguments: for
 * i = 0..k-1 in order, x_i <- [R_i - sum_{l != i} G_li x_l]_+ / G_ii using the
 * newest x_l; x_i = 0 where G_ii <= 0. Asynchronous on `stream`. */
nmf_status nmf_update_hals(int32_t k, int64_t rows, const double *G, const float *R, float *X,
                           void *stream);

/* Stopping measure for Alg. 1's "while not converged" (the paper leaves the
 * test open; this is the projected-gradient norm of Lin 2007, used for ANLS by
 * Kim and Park), with half the gradient of Eq. 1:
 *   Delta(W, H) = sqrt(|P[W H H^T - A H^T]|_F^2 + |P[H^T W^T W - A^T W]|_F^2),
 * P[g]_ij = g_ij where the factor entry is > 0 and min(g_ij, 0) where it is 0.
 * This call: *out = |P[X G - R]|_F^2 for rows of X (rows x k float32) with
 * G (k x k float64) and R (rows x k float32), all device; *out is host.
 * Synchronises `stream`. */
nmf_status nmf_pgrad_sq(int32_t k, int64_t rows, const double *G, const float *R, const float *X,
                        double *out, void *stream);

/* Objective of Eq. 1 for dense A: f = sum_ij (A_ij - w_i . h_j)^2 with W
 * (m x k) and H^T (n x k), all device; the residuals are formed in FP32 and
 * their squares summed in FP64. Synchronises `stream`; writes *f_out (host). */
nmf_status nmf_objective_dense(const float *A, int64_t m, int64_t n, int64_t lda,
                               const float *W, const float *Ht, int32_t k, int32_t precision,
                               double *f_out, void *stream);

/* ===================================================================== *
 * Whole ANLS iterations (Alg. 1) on a handle.
 * ===================================================================== */

typedef struct nmf_handle nmf_handle;

typedef enum nmf_input_kind { NMF_INPUT_DENSE = 0, NMF_INPUT_CSR = 1 } nmf_input_kind;

/* How each BPP solve picks its first passive set: empty (cold, the cited
 * method's start) or the row's final passive set from the previous iteration
 * (warm). Either way the solution is the same unique minimiser. */
typedef enum nmf_start_mode { NMF_START_COLD = 0, NMF_START_WARM = 1 } nmf_start_mode;

/* Local update of each half-step: the exact NLS solve by BPP (Sec. 4.2, the
 * paper's method), or one step of the alternatives the paper names for the
 * same inputs, MU (Eq. 5) or HALS (Eq. 6). */
typedef enum nmf_solver { NMF_SOLVER_BPP = 0, NMF_SOLVER_MU = 1, NMF_SOLVER_HALS = 2 } nmf_solver;

typedef struct nmf_config {
    int64_t m, n;              /* A is m x n */
    int32_t k;                 /* rank, 1..NMF_MAX_K */
    int32_t input_kind;        /* nmf_input_kind */
    int32_t precision;         /* nmf_precision for the products and objective
                                  (NMF_PREC_BF16X3: dense A 16-byte aligned,
                                  lda a multiple of 4) */
    int32_t start_mode;        /* nmf_start_mode */
    int32_t max_bpp_rounds;    /* per-RHS exchange cap (e.g. 100) */
    int32_t objective_every;   /* 1: f after every iteration (history kept);
                                  0: only on nmf_objective() */
    int32_t solver;            /* nmf_solver (0, BPP, when zero-initialised) */
    int32_t no_split_copies;   /* dense BF16x3: 0 (default) keeps BF16 hi / lo copies of A
                                  and A^T (+8 bytes per element of A) so the products need
                                  no per-pass split; 1 splits A in every pass (same products) */
    int32_t no_fused_products; /* CSR with BPP: 0 (default) forms each right-hand side
                                  (row of A H^T or A^T W) inside the FP32 solves, in the
                                  SpMM's order, instead of a separate SpMM pass (same
                                  results); 1 runs the SpMM first. The projected-gradient
                                  record and a proposal network always use the SpMM pass */
} nmf_config;

/* The input matrix. Its device buffers are BORROWED: the caller keeps them
 * alive and unchanged until nmf_destroy. */
typedef struct nmf_matrix {
    const float *dense;        /* NMF_INPUT_DENSE: m x n float32, device */
    int64_t lda;               /* leading dimension >= n */
    const int64_t *rowptr;     /* NMF_INPUT_CSR: m+1 int64, device */
    const int32_t *colidx;     /* nnz int32, device */
    const float *vals;         /* nnz float32, device */
    int64_t nnz;
} nmf_matrix;

/* Per-handle counters, cumulative since nmf_init (or the last reset). */
typedef struct nmf_stats {
    int64_t iterations;        /* ANLS iterations run */
    int64_t bpp_rhs;           /* right-hand sides solved */
    int64_t bpp_rounds;        /* exchange rounds summed over all solves */
    int64_t bpp_max_rounds;    /* largest round count of one solve */
    int64_t bpp_fp64_solves;   /* passive-set systems redone in FP64 */
    int64_t bpp_fp64_halfsteps;/* half-steps solved in FP64 (cond_1(G) > 1e4) */
    int64_t bpp_not_converged; /* solves that hit the round cap */
    int64_t bpp_singular;      /* solves left singular in FP64 */
    double ms_gram, ms_mm, ms_nls, ms_objective; /* GPU time per task (timing on) */
    int64_t kernel_launches;   /* CUDA kernels this handle has launched */
    double ms_proposal;        /* features, proposal and training (timing on) */
    int64_t graph_launches;    /* nmf_iterate calls run as one CUDA graph */
    int64_t mm_splits_max;     /* largest number of CTAs sharing one output tile
                                  along the contraction in a tensor-core product
                                  (tall-skinny A splits the long contraction) */
} nmf_stats;

/* Create a handle. W0 (m x k) and Ht0 (n x k) are the device starting point
 * (Alg. 1 initialises H with a nonnegative matrix; W0 is only used as the
 * value W holds before its first update). They are copied; the handle owns
 * W, H^T, the Grams, right-hand-side buffers, passive-set bitmasks, the
 * transposed CSR (sparse input) and all other workspace. The handle's work
 * is issued on `stream`. Synchronises `stream` before returning. */
nmf_status nmf_init(nmf_handle **out, const nmf_config *cfg, const nmf_matrix *A,
                    const float *W0, const float *Ht0, void *stream);

/* Run `iters` ANLS iterations asynchronously on the handle's stream. Each
 * iteration: Gram H H^T, A H^T, BPP for W, Gram W^T W, W^T A, BPP for H, and
 * (objective_every = 1) f(W, H). Returns NMF_OK once launched; solve failures
 * are counted in nmf_stats and reported by nmf_sync. */
nmf_status nmf_iterate(nmf_handle *h, int32_t iters);

/* Wait for the handle's stream; return the worst BPP status since the last
 * nmf_sync (NMF_OK, NMF_ERR_NOT_CONVERGED or NMF_ERR_SINGULAR_GRAM).
 * Dense BF16x3 handles compute f of an iteration inside the next iteration's
 * A H^T pass; the last iteration's f stays pending until the handle iterates
 * again or the objective is read (nmf_objective, nmf_objective_history, which
 * then run one A H^T pass for it). Neither nmf_sync nor nmf_get_stats
 * computes it. */
nmf_status nmf_sync(nmf_handle *h);

/* f(W, H) of Eq. 1 for the current factors. Synchronises; *f_out is host. */
nmf_status nmf_objective(nmf_handle *h, double *f_out);

/* Objective history: f after each iteration run with objective_every = 1, in
 * order, up to `cap` values copied into `f_host` (host); *count gets the
 * number copied. Synchronises. */
nmf_status nmf_objective_history(nmf_handle *h, double *f_host, int64_t cap, int64_t *count);

/* Copy the current factors out to (W m x k, Ht n x k) device buffers, or in
 * from them (checkpoint / resume). Either pointer may be NULL to skip it.
 * Asynchronous on the handle's stream. Setting factors clears the warm-start
 * passive sets. */
nmf_status nmf_get_factors(nmf_handle *h, float *W, float *Ht);
nmf_status nmf_set_factors(nmf_handle *h, const float *W, const float *Ht);

/* Passive-set bitmasks of the last solves (device, m or n rows of
 * ceil(k/64) words). */
nmf_status nmf_get_passive(nmf_handle *h, uint64_t *pW, uint64_t *pH);

/* Counters; synchronises. timing != 0 turns per-task CUDA-event timing on for
 * later iterations (adds event records, no host waits inside nmf_iterate). */
nmf_status nmf_get_stats(nmf_handle *h, nmf_stats *out);
nmf_status nmf_set_timing(nmf_handle *h, int32_t timing);

/* on != 0: each nmf_iterate call captures its iterations into one CUDA graph
 * and launches that (fewer launch gaps for small problems). Calls on the
 * legacy default stream or with timing on run eagerly instead. */
nmf_status nmf_set_graph(nmf_handle *h, int32_t on);

/* Record Delta (see nmf_pgrad_sq) of every iterate from the current one on
 * (on = 1) or stop recording (0). The part in H is formed at the end of each H
 * half-step and the part in W in the next iteration's W half-step (its Gram
 * and right-hand sides are the iterate's), so Delta of iterate t is complete
 * once iteration t + 1 has run. Turning it on costs one product (A^T W of the
 * current iterate); nmf_set_factors turns it off. */
nmf_status nmf_set_pgrad(nmf_handle *h, int32_t on);

/* Delta of the recorded iterates whose value is complete, oldest first (at
 * most `cap`, host buffer); *count = values written. Synchronises. */
nmf_status nmf_pgrad_history(nmf_handle *h, double *out, int64_t cap, int64_t *count);

/* Iterate until Delta(t) <= rel_tol * Delta(t0), t0 the first recorded
 * iterate (the current one if recording was off), or max_iters iterations.
 * Delta(t) is known after iteration t + 1, so the handle ends one iteration
 * past the first iterate that meets the test. One host synchronisation per
 * iteration. *iters_done (nullable): iterations run; *ratio (nullable):
 * Delta / Delta(t0) of the last complete iterate. */
nmf_status nmf_iterate_until(nmf_handle *h, int32_t max_iters, double rel_tol,
                             int32_t *iters_done, double *ratio);

/* Release everything the handle owns. NULL is ignored. */
void nmf_destroy(nmf_handle *h);

/* ===================================================================== *
 * Learned passive-set proposal (no counterpart in the paper).
 * ===================================================================== *
 * A small network proposes each BPP solve's starting passive set. The solve
 * then runs to the KKT point of Eq. 4 as always, so every result is the same
 * unique minimiser and a poor proposal only costs exchange rounds.
 * Features of one right-hand side (G, g, the previous iterate x_p of that
 * factor row; zeros when cold), with d_i = sqrt(G_ii) (1 where G_ii <= 0)
 * and s = max_i |g_i| / d_i (1 if 0), 3k floats:
 *   [ (G x_p - g)_i / (d_i s), log(G_ii / mean_j G_jj) (0 where G_ii <= 0),
 *     x_p,i d_i / s ].
 * Network 3k -> hidden -> hidden -> k, ReLU after the first two layers,
 * BF16-rounded weights, FP32 arithmetic; proposal {i : logit_i > 0}.
 * Parameters: one flat FP32 array [W1 (hidden x 3k), b1 (hidden), W2 (hidden
 * x hidden), b2, W3 (k x hidden), b3 (k)], weight rows = outputs. Training
 * minimises the mean binary cross-entropy against the solves' final passive
 * sets with Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights.
 * All pointers are device pointers; calls are asynchronous on `stream`. */
typedef struct nmf_mlp nmf_mlp;

int64_t nmf_mlp_param_count(int32_t k, int32_t hidden);

/* k in 1..NMF_MAX_K, hidden in 1..1024; `params` (nmf_mlp_param_count
 * floats) is copied. */
nmf_status nmf_mlp_create(nmf_mlp **out, int32_t k, int32_t hidden, const float *params,
                          void *stream);
/* Current FP32 master parameters into `params`. */
nmf_status nmf_mlp_get_params(const nmf_mlp *h, float *params, void *stream);
void nmf_mlp_destroy(nmf_mlp *h);

/* F (nrhs x 3k) from G (k x k FP64), B (nrhs x k) and Xprev (nrhs x k, or
 * NULL for zeros). */
nmf_status nmf_mlp_features(const double *G, const float *B, const float *Xprev, int64_t nrhs,
                            int32_t k, float *F, void *stream);
/* Logits (nrhs x k) of features F. */
nmf_status nmf_mlp_forward(nmf_mlp *h, const float *F, int64_t nrhs, float *logits, void *stream);
/* Proposed passive sets, nrhs rows of ceil(k/64) words. */
nmf_status nmf_mlp_propose(nmf_mlp *h, const float *F, int64_t nrhs, uint64_t *passive,
                           void *stream);
/* Gradient of the mean binary cross-entropy over the batch (labels: passive
 * bitmasks) without updating; `grad` (nmf_mlp_param_count floats) and `loss`
 * (one double) may each be NULL. */
nmf_status nmf_mlp_gradient(nmf_mlp *h, const float *F, const uint64_t *passive, int64_t nrhs,
                            float *grad, double *loss, void *stream);
/* Adam steps over the nrhs samples in consecutive batches of `batch` rows;
 * the last batch's loss to `loss` (one double, nullable). */
nmf_status nmf_mlp_train(nmf_mlp *h, const float *F, const uint64_t *passive, int64_t nrhs,
                         int64_t batch, float lr, double *loss, void *stream);

/* Attach a network to an ANLS handle (NULL or NMF_PROPOSAL_OFF detaches).
 *   NMF_PROPOSAL_TRAIN: each half-step computes the features of its solves,
 *     solves as start_mode says, then trains the network on (features, final
 *     passive sets): `epochs` passes in batches of `batch` rows at rate lr.
 *   NMF_PROPOSAL_USE: each half-step's solves start from the proposal.
 * The network must have the handle's k. The handle borrows it: keep it alive
 * while attached. */
typedef enum nmf_proposal_mode {
    NMF_PROPOSAL_OFF = 0,
    NMF_PROPOSAL_TRAIN = 1,
    NMF_PROPOSAL_USE = 2
} nmf_proposal_mode;
nmf_status nmf_set_proposal(nmf_handle *h, nmf_mlp *mlp, int32_t mode, int32_t epochs,
                            int64_t batch, float lr);

#ifdef __cplusplus
}
#endif

#endif /* NMF_GB300_H */
