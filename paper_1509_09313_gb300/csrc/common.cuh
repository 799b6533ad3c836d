// Shared definitions of the sm_103a ANLS-NMF library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nmf_gb300.h"

namespace nmf {

constexpr unsigned FULL = 0xffffffffu;

// Record the first CUDA error text for nmf_last_error-style diagnostics and
// map a cudaError_t to the ABI status.
nmf_status from_cuda(cudaError_t e, const char *what);

#define NMF_CUDA(expr)                                                             \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return ::nmf::from_cuda(e_, #expr);                                    \
    } while (0)

// Every kernel launch is followed by NMF_LAUNCHED, which also counts it.
extern unsigned long long launch_count;

#define NMF_LAUNCHED(what)                                                         \
    do {                                                                           \
        ::nmf::launch_count += 1;                                                  \
        cudaError_t e_ = cudaGetLastError();                                       \
        if (e_ != cudaSuccess)                                                     \
            return ::nmf::from_cuda(e_, what);                                     \
    } while (0)

#define NMF_TRY(expr)                                                              \
    do {                                                                           \
        nmf_status s_ = (expr);                                                    \
        if (s_ != NMF_OK)                                                          \
            return s_;                                                             \
    } while (0)

inline int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0)
            n = 1;
    }
    return n;
}

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// A kernel's dynamic shared-memory opt-in is a per-device attribute: each
// launch site keeps the largest size it has set on each device and sets it
// again only when a launch needs more (or on a device it has not seen).
struct SmemOptIn {
    static constexpr int MAX_DEVICES = 64;
    int bytes[MAX_DEVICES] = {};
};

template <typename Kernel>
inline nmf_status ensure_smem(Kernel kernel, SmemOptIn &cache, size_t bytes)
{
    if (bytes <= 48 * 1024)
        return NMF_OK;
    int dev = 0;
    NMF_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < SmemOptIn::MAX_DEVICES && (int)bytes <= cache.bytes[dev])
        return NMF_OK;
    NMF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (dev >= 0 && dev < SmemOptIn::MAX_DEVICES)
        cache.bytes[dev] = (int)bytes;
    return NMF_OK;
}

// True when [a, a + bytes) and [b, b + bytes) share a byte.
inline bool ranges_overlap(const void *a, const void *b, size_t bytes)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return bytes > 0 && x < y + bytes && y < x + bytes;
}

// ---------------------------------------------------------------------------
// Internal launchers (all asynchronous on `s`).
// ---------------------------------------------------------------------------

// Gram X^T X on the tensor cores (gram_tc.cu): used by launch_gram when
// gram_tc_usable (k <= 64, enough rows, X 16-byte aligned); writes
// gram_tc_parts(rows) CTA partials in the layout of the SIMT Gram's.
bool gram_tc_usable(const float *X, int64_t rows, int k);
int gram_tc_parts(int64_t rows);
nmf_status launch_gram_tc(const float *X, int64_t rows, int k, double *partials, cudaStream_t s);

// Gram X^T X in FP64. `partials` must hold gram_partials_len(rows, k) doubles.
int64_t gram_partials_len(int64_t rows, int k);
nmf_status launch_gram(const float *X, int64_t rows, int k, double *G, double *partials,
                       cudaStream_t s);

// Dense products, plain FP32 SIMT: trans 0 -> A F (m x k), 1 -> A^T F (n x k).
nmf_status launch_mm_simt(const float *A, int64_t m, int64_t n, int64_t lda, const float *F,
                          int k, int trans, float *out, cudaStream_t s);

// Dense products in plain FP32 with packed FP32x2 FMAs (mm_f32.cu): A 16-byte
// aligned with lda a multiple of 4 (mm_f32_supported). trans = 0 with W and
// f_dev non-null (k <= 64) also writes f(W, H) = ||A - W H||^2 to *f_dev.
// `work` holds mm_f32_work_bytes(m, n, k, trans) bytes.
bool mm_f32_supported(const float *A, int64_t lda);
size_t mm_f32_work_bytes(int64_t m, int64_t n, int k, int trans);
nmf_status launch_mm_f32(const float *A, int64_t m, int64_t n, int64_t lda, const float *F, int k,
                         int trans, float *out, const float *W, double *f_dev, void *work,
                         size_t work_bytes, cudaStream_t s);
// *f_dev = sum of partials[0..parts) in a fixed order (FP64).
nmf_status launch_sum_partials(const double *partials, int parts, double *f_dev, cudaStream_t s);

// Dense products on tcgen05 tensor cores with BF16 head/tail operand splits.
nmf_status launch_mm_tc(const float *A, int64_t m, int64_t n, int64_t lda, const float *F,
                        int k, int trans, float *out, void *work, size_t work_bytes,
                        cudaStream_t s);
size_t mm_tc_work_bytes(int64_t m, int64_t n, int k, int trans);
// Contraction splits (CTAs along the contraction per output tile) the plain
// tensor-core product of this shape uses; 1 for the pass with the objective.
int mm_tc_splits(int64_t m, int64_t n, int trans);
// Same, and with W, Ht, f_dev non-null (trans = 0, k <= 64) the objective
// f(W, H) = ||A - W H||^2 fused into the pass, written to *f_dev.
nmf_status launch_mm_tc_obj(const float *A, int64_t m, int64_t n, int64_t lda, const float *F,
                            int k, int trans, float *out, const float *W, double *f_dev,
                            void *work, size_t work_bytes, cudaStream_t s);

// Products from A pre-split into BF16 hi / lo copies (tile-major, each
// mm_tc_presplit_bytes(rows, K) bytes: trans = 0 rows m, K n; trans = 1 rows
// n, K m), made once by launch_mm_tc_presplit_make. trans = 1 gives bitwise
// the result of launch_mm_tc; trans = 0 too, and with W / f_dev the objective
// from hi + lo (within 2^-18 relative of A) instead of A.
size_t mm_tc_presplit_bytes(int64_t rows, int64_t K);
nmf_status launch_mm_tc_presplit_make(const float *A, int64_t m, int64_t n, int64_t lda,
                                      int trans, void *hi, void *lo, cudaStream_t s);
nmf_status launch_mm_tc_presplit(const void *hi, const void *lo, int64_t m, int64_t n,
                                 const float *F, int k, int trans, float *out, const float *W,
                                 double *f_dev, void *work, size_t work_bytes, cudaStream_t s);

// CSR SpMM: out (rows x k) = S F.
nmf_status launch_spmm(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                       int64_t rows, const float *F, int k, float *out, cudaStream_t s);
// The same product, skipped on the device when *mode_flag == 0 (an FP32
// half-step whose solves gather their right-hand sides themselves).
nmf_status launch_spmm_unless_fp32(const int64_t *rowptr, const int32_t *colidx,
                                   const float *vals, int64_t rows, const float *F, int k,
                                   float *out, const int *mode_flag, cudaStream_t s);

// Right-hand sides formed inside the batched BPP as b_j = (S F)_j (rows of the
// CSR matrix S times F, k columns), for the sparse ANLS half-steps.
struct CsrGather {
    const int64_t *rowptr;
    const int32_t *colidx;
    const float *vals;
    const float *F;
};

// Objective pieces. Dense: per-block FP64 partial sums of squared residuals,
// reduced in a fixed order into *f_dev. `partials` holds objective_partials_len().
int64_t objective_partials_len();
nmf_status launch_objective_dense(const float *A, int64_t m, int64_t n, int64_t lda,
                                  const float *W, const float *Ht, int k, int precision,
                                  double *partials, double *f_dev, cudaStream_t s);
// Sparse: f = ||A||^2 - 2 sum_j h_j . Y_j + trace(GW GH), with Y = A^T W
// (n x k), GW = W^T W and GH = H H^T current, and *a_sq = ||A||^2.
nmf_status launch_objective_csr(const float *Ht, const float *Y, int64_t n, int k,
                                const double *a_sq, const double *GW, const double *GH,
                                double *partials, double *f_dev, cudaStream_t s);
// *out = ||v||^2 (FP64), e.g. of the stored values of A.
nmf_status launch_sq_norm(const float *v, int64_t len, double *partials, double *out,
                          cudaStream_t s);

// MU (Eq. 5) or HALS (Eq. 6) step of the rows of X in place (local_update.cu).
nmf_status launch_local_update(int solver, const double *G, int k, const float *R, float *X,
                               int64_t rows, cudaStream_t s);

// *out = squared projected-gradient norm of the rows of X (grad = X G - R;
// entries with x = 0 count only where grad < 0). `partials` holds
// pgrad_partials_len() doubles.
int pgrad_partials_len();
nmf_status launch_pgrad_sq(const double *G, int k, const float *R, const float *X, int64_t rows,
                           double *partials, double *out, cudaStream_t s);

// Batched BPP. Workspace layout is private to bpp.cu; size from bpp_work_bytes.
size_t bpp_work_bytes(int k);
struct BppStats {
    unsigned long long rhs, rounds, max_rounds, fp64_solves, not_converged, singular, nonfinite,
        fp64_halfsteps;
};
nmf_status launch_bpp(int k, int64_t nrhs, const double *G, const float *B, float *X,
                      const uint64_t *passive_in, uint64_t *passive_out, int32_t *rounds_out,
                      int8_t *status_out, int max_rounds, void *work, BppStats *stats_dev,
                      cudaStream_t s);
// The two halves of launch_bpp: the per-Gram preparation (factor, inverse,
// arithmetic mode), then the solves. A prep must complete before its solves
// and must not overlap another half-step's prep or solves on the same work.
nmf_status launch_bpp_prep(int k, const double *G, void *work, BppStats *stats_dev, cudaStream_t s);
// Measures the solve kernel's launch shapes on this batch and keeps the fastest
// for k (used by every later solve of that k); X receives the solution.
nmf_status bpp_tune(int k, int64_t nrhs, const double *G, const float *B, float *X,
                    const uint64_t *passive_in, int max_rounds, void *work, BppStats *stats_dev,
                    cudaStream_t s, int *warps_out, int *chunk_out, int *group_out);
// The launch shape every later solve of k uses (see nmf_nls_bpp_set_shape).
nmf_status bpp_set_shape(int k, int warps, int chunk, int group);
nmf_status bpp_get_shape(int k, int *warps, int *chunk, int *group);
nmf_status launch_bpp_solve(int k, int64_t nrhs, const double *G, const float *B, float *X,
                            const uint64_t *passive_in, uint64_t *passive_out, int32_t *rounds_out,
                            int8_t *status_out, int max_rounds, void *work, BppStats *stats_dev,
                            cudaStream_t s, const CsrGather *gather = nullptr);

// Learned passive-set proposal (mlp.cu).
struct MlpNet;
int64_t mlp_param_count(int k, int h);
nmf_status mlp_create(MlpNet **out, int k, int h, const float *params, cudaStream_t s);
void mlp_destroy(MlpNet *net);
int mlp_k(const MlpNet *net);
int mlp_hidden(const MlpNet *net);
int64_t mlp_nparams(const MlpNet *net);
const float *mlp_master(const MlpNet *net);
nmf_status mlp_features(const double *G, const float *B, const float *Xp, int64_t nrhs, int k,
                        float *F, cudaStream_t s);
nmf_status mlp_logits(MlpNet *net, const float *F, int64_t n, float *logits, cudaStream_t s);
nmf_status mlp_propose(MlpNet *net, const float *F, int64_t n, uint64_t *passive, cudaStream_t s);
// Inference pass on the tensor cores (mlp_tc.cu): logits (rows x k) and / or
// proposed passive sets (rows x ceil(k / 64) words), either nullable, from
// the BF16-valued working weights. Supported for k and hidden width up to 256.
// The input is the features F (rows x 3k FP32), or, with F null, formed from
// G, B and Xp as mlp_features does.
bool mlp_tc_supported(int k, int h);
// The layers' BF16 weight operands (mlp_tc_weights_bytes of device memory),
// from the BF16-valued working weights; the forward pass reads them.
size_t mlp_tc_weights_bytes(int k, int h);
nmf_status launch_mlp_tc_weights(int k, int h, const float *W1, const float *W2, const float *W3,
                                 void *dst, cudaStream_t s);
nmf_status launch_mlp_tc_forward(int k, int h, const void *wts, const float *b1, const float *b2,
                                 const float *b3, const float *F, const double *G, const float *B,
                                 const float *Xp, int64_t n, float *logits, uint64_t *bits,
                                 cudaStream_t s);
// Features of a batch straight into the first layer's BF16 hi / lo operand
// (blocks of kpf >= k columns; rows of ldd >= 3 kpf columns, a multiple of 8).
nmf_status launch_mlp_features_split(const double *G, const float *B, const float *Xp,
                                     int64_t nrhs, int k, int kpf, int ldd, __nv_bfloat16 *hi,
                                     __nv_bfloat16 *lo, cudaStream_t s);
// Features and proposal of one half-step (F: rows x 3k FP32 scratch, used
// only when the tensor-core pass does not apply).
nmf_status mlp_features_propose(MlpNet *net, const double *G, const float *B, const float *Xp,
                                int64_t n, float *F, uint64_t *passive, cudaStream_t s);
nmf_status mlp_gradient(MlpNet *net, const float *F, const uint64_t *lab, int64_t n,
                        float *grad_out, double *loss_dev, cudaStream_t s);
nmf_status mlp_train(MlpNet *net, const float *F, const uint64_t *lab, int64_t n, int64_t batch,
                     float lr, double *loss_dev, cudaStream_t s);

}  // namespace nmf
