// C ABI of the library (include/nmf_gb300.h): argument checks, workspace
// management, and the ANLS iteration of Alg. 1 / Eq. 2 on a handle.
#include <stdio.h>
#include <string.h>

#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace nmf {

nmf_status launch_csr_transpose(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                                int64_t m, int64_t n, int64_t nnz, int64_t *t_rowptr,
                                int32_t *t_colidx, float *t_vals, unsigned long long *cursor,
                                cudaStream_t s);

unsigned long long launch_count = 0;

nmf_status from_cuda(cudaError_t e, const char *what)
{
    (void)what;
    cudaGetLastError();   // clear a sticky launch error so later calls can proceed
    return e == cudaErrorMemoryAllocation ? NMF_ERR_OOM : NMF_ERR_CUDA;
}

}  // namespace nmf

using namespace nmf;

namespace {

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

bool bad_k(int32_t k) { return k < 1 || k > NMF_MAX_K; }

// Stream-ordered temporary device buffer, freed on scope exit (also
// stream-ordered), for the stand-alone entry points.
struct TempBuf {
    void *p = nullptr;
    cudaStream_t s;
    explicit TempBuf(cudaStream_t st) : s(st) {}
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes ? bytes : 16, s); }
    ~TempBuf()
    {
        if (p)
            cudaFreeAsync(p, s);
    }
};

}  // namespace

extern "C" int64_t nmf_kernel_launches(void) { return (int64_t)launch_count; }

extern "C" const char *nmf_status_str(nmf_status s)
{
    switch (s) {
    case NMF_OK: return "NMF_OK";
    case NMF_ERR_INVALID_ARG: return "NMF_ERR_INVALID_ARG";
    case NMF_ERR_CUDA: return "NMF_ERR_CUDA";
    case NMF_ERR_OOM: return "NMF_ERR_OOM";
    case NMF_ERR_NOT_CONVERGED: return "NMF_ERR_NOT_CONVERGED";
    case NMF_ERR_SINGULAR_GRAM: return "NMF_ERR_SINGULAR_GRAM";
    case NMF_ERR_NONFINITE: return "NMF_ERR_NONFINITE";
    }
    return "NMF_ERR_UNKNOWN";
}

extern "C" nmf_status nmf_gram(const float *X, int64_t rows, int32_t k, double *G, void *stream)
{
    if (bad_k(k) || rows < 0 || !G || (rows > 0 && !X))
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    TempBuf part(s);
    NMF_CUDA(part.alloc(sizeof(double) * (size_t)gram_partials_len(rows, k)));
    return launch_gram(X, rows, k, G, static_cast<double *>(part.p), s);
}

extern "C" nmf_status nmf_mm_dense(const float *A, int64_t m, int64_t n, int64_t lda,
                                   const float *F, int32_t k, int32_t trans, int32_t precision,
                                   float *out, void *stream)
{
    if (bad_k(k) || m < 0 || n < 0 || lda < n || (trans != 0 && trans != 1))
        return NMF_ERR_INVALID_ARG;
    if (precision != NMF_PREC_FP32 && precision != NMF_PREC_BF16X3)
        return NMF_ERR_INVALID_ARG;
    const int64_t P = trans ? n : m, Q = trans ? m : n;
    if (P == 0)
        return NMF_OK;
    if (!out || (Q > 0 && (!A || !F)))
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (precision == NMF_PREC_BF16X3) {
        const size_t wb = mm_tc_work_bytes(m, n, k, trans);
        TempBuf w(s);
        NMF_CUDA(w.alloc(wb));
        return launch_mm_tc(A, m, n, lda, F, k, trans, out, w.p, wb, s);
    }
    if (mm_f32_supported(A, lda)) {
        const size_t wb = mm_f32_work_bytes(m, n, k, trans);
        TempBuf w(s);
        NMF_CUDA(w.alloc(wb));
        return launch_mm_f32(A, m, n, lda, F, k, trans, out, nullptr, nullptr, w.p, wb, s);
    }
    return launch_mm_simt(A, m, n, lda, F, k, trans, out, s);
}

extern "C" nmf_status nmf_mm_csr(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                                 int64_t rows, int64_t cols, const float *F, int32_t k,
                                 float *out, void *stream)
{
    if (bad_k(k) || rows < 0 || cols < 0)
        return NMF_ERR_INVALID_ARG;
    if (rows == 0)
        return NMF_OK;
    if (!rowptr || !out || !F || !colidx || !vals)
        return NMF_ERR_INVALID_ARG;
    return launch_spmm(rowptr, colidx, vals, rows, F, k, out, as_stream(stream));
}

extern "C" nmf_status nmf_csr_transpose(const int64_t *rowptr, const int32_t *colidx,
                                        const float *vals, int64_t m, int64_t n, int64_t nnz,
                                        int64_t *t_rowptr, int32_t *t_colidx, float *t_vals,
                                        void *stream)
{
    if (m < 0 || n < 0 || nnz < 0 || !t_rowptr || !rowptr)
        return NMF_ERR_INVALID_ARG;
    if (nnz > 0 && (!colidx || !vals || !t_colidx || !t_vals))
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    TempBuf cur(s);
    NMF_CUDA(cur.alloc(sizeof(unsigned long long) * (size_t)(n > 0 ? n : 1)));
    return launch_csr_transpose(rowptr, colidx, vals, m, n, nnz, t_rowptr, t_colidx, t_vals,
                                static_cast<unsigned long long *>(cur.p), s);
}

static nmf_status worst_from_stats(const BppStats &st)
{
    if (st.nonfinite)
        return NMF_ERR_NONFINITE;
    if (st.singular)
        return NMF_ERR_SINGULAR_GRAM;
    if (st.not_converged)
        return NMF_ERR_NOT_CONVERGED;
    return NMF_OK;
}

extern "C" nmf_status nmf_nls_bpp(const nmf_nls_desc *d, void *stream)
{
    if (!d || bad_k(d->k) || d->nrhs < 0 || d->max_rounds < 0 || !d->G)
        return NMF_ERR_INVALID_ARG;
    if (d->nrhs > 0 && (!d->B || !d->X))
        return NMF_ERR_INVALID_ARG;
    if (ranges_overlap(d->B, d->X, sizeof(float) * (size_t)d->nrhs * d->k))
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    TempBuf w(s), st(s);
    NMF_CUDA(w.alloc(bpp_work_bytes(d->k)));
    NMF_CUDA(st.alloc(sizeof(BppStats)));
    NMF_CUDA(cudaMemsetAsync(st.p, 0, sizeof(BppStats), s));
    NMF_TRY(launch_bpp(d->k, d->nrhs, d->G, d->B, d->X, d->passive_in, d->passive_out,
                       d->rounds_out, d->status_out, d->max_rounds, w.p,
                       static_cast<BppStats *>(st.p), s));
    BppStats host;
    NMF_CUDA(cudaMemcpyAsync(&host, st.p, sizeof(BppStats), cudaMemcpyDeviceToHost, s));
    NMF_CUDA(cudaStreamSynchronize(s));
    return worst_from_stats(host);
}

extern "C" nmf_status nmf_nls_bpp_tune(const nmf_nls_desc *d, void *stream, int32_t *warps,
                                       int32_t *chunk, int32_t *group)
{
    if (!d || bad_k(d->k) || d->nrhs < 1 || d->max_rounds < 0 || !d->G || !d->B || !d->X)
        return NMF_ERR_INVALID_ARG;
    if (ranges_overlap(d->B, d->X, sizeof(float) * (size_t)d->nrhs * d->k))
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    TempBuf w(s), st(s);
    NMF_CUDA(w.alloc(bpp_work_bytes(d->k)));
    NMF_CUDA(st.alloc(sizeof(BppStats)));
    NMF_CUDA(cudaMemsetAsync(st.p, 0, sizeof(BppStats), s));
    int wv = 0, cv = 0, gv = 0;
    NMF_TRY(bpp_tune(d->k, d->nrhs, d->G, d->B, d->X, d->passive_in, d->max_rounds, w.p,
                     static_cast<BppStats *>(st.p), s, &wv, &cv, &gv));
    NMF_CUDA(cudaStreamSynchronize(s));
    if (warps)
        *warps = wv;
    if (chunk)
        *chunk = cv;
    if (group)
        *group = gv;
    return NMF_OK;
}

extern "C" nmf_status nmf_nls_bpp_set_shape(int32_t k, int32_t warps, int32_t chunk,
                                            int32_t group)
{
    return bpp_set_shape(k, warps, chunk, group);
}

extern "C" nmf_status nmf_nls_bpp_get_shape(int32_t k, int32_t *warps, int32_t *chunk,
                                            int32_t *group)
{
    return bpp_get_shape(k, warps, chunk, group);
}

extern "C" nmf_status nmf_objective_dense(const float *A, int64_t m, int64_t n, int64_t lda,
                                          const float *W, const float *Ht, int32_t k,
                                          int32_t precision, double *f_out, void *stream)
{
    if (bad_k(k) || m < 0 || n < 0 || lda < n || !f_out)
        return NMF_ERR_INVALID_ARG;
    if (precision != NMF_PREC_FP32 && precision != NMF_PREC_BF16X3)
        return NMF_ERR_INVALID_ARG;
    if (m > 0 && n > 0 && (!A || !W || !Ht))
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    TempBuf part(s), f(s);
    NMF_CUDA(f.alloc(sizeof(double)));
    if (precision == NMF_PREC_BF16X3 && k <= 64 && m > 0 && n > 0) {
        // Tensor cores: the objective rides on an A H^T pass whose product
        // goes to scratch.
        const size_t wb = mm_tc_work_bytes(m, n, k, 0);
        TempBuf w(s), v(s);
        NMF_CUDA(w.alloc(wb));
        NMF_CUDA(v.alloc(sizeof(float) * (size_t)m * k));
        NMF_TRY(launch_mm_tc_obj(A, m, n, lda, Ht, k, 0, static_cast<float *>(v.p), W,
                                 static_cast<double *>(f.p), w.p, wb, s));
    } else {
        NMF_CUDA(part.alloc(sizeof(double) * (size_t)objective_partials_len()));
        NMF_TRY(launch_objective_dense(A, m, n, lda, W, Ht, k, precision,
                                       static_cast<double *>(part.p), static_cast<double *>(f.p),
                                       s));
    }
    NMF_CUDA(cudaMemcpyAsync(f_out, f.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    NMF_CUDA(cudaStreamSynchronize(s));
    return NMF_OK;
}

// ===========================================================================
// Handle: whole ANLS iterations.
// ===========================================================================

struct nmf_handle {
    nmf_config cfg;
    nmf_matrix A;
    cudaStream_t stream;
    // Side stream for each half-step's Gram and BPP preparation, which depend
    // only on the other factor and so run beside the m x n x k product (in
    // the SMs its last wave leaves idle); fork / join events order them.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int nwords;
    // Owned device buffers.
    float *W = nullptr, *Ht = nullptr;          // factors (m x k, n x k)
    float *V = nullptr, *Y = nullptr;           // right-hand sides (m x k, n x k)
    double *GH = nullptr, *GW = nullptr;        // Grams (k x k)
    uint64_t *pW = nullptr, *pH = nullptr;      // passive sets
    void *bpp_work = nullptr;
    BppStats *stats_dev = nullptr;
    double *gram_part = nullptr;
    double *obj_part = nullptr;
    double *a_sq = nullptr;                     // ||A||^2 (sparse input)
    double *f_hist = nullptr;                   // ring of objective values
    double *f_now = nullptr;
    double *pgw2 = nullptr, *pgh2 = nullptr;    // rings: squared projected gradient in W, in H
    double *pg_part = nullptr;
    void *tc_work = nullptr;                    // product workspace (tensor-core or FP32 path)
    size_t tc_work_bytes = 0;
    bool f32 = false;                           // dense FP32: the packed-FMA product kernel
    void *at_hi = nullptr, *at_lo = nullptr;   // A^T pre-split, tile-major (dense BF16x3)
    void *ar_hi = nullptr, *ar_lo = nullptr;   // A pre-split, tile-major (dense BF16x3)
    int64_t *t_rowptr = nullptr;                // CSR of A^T (sparse input)
    int32_t *t_colidx = nullptr;
    float *t_vals = nullptr;
    // Host state.
    bool passive_valid = false;
    bool fused_obj = false;        // objective computed inside the next A H^T pass
    bool gh_current = false;       // GH is the Gram of the current Ht (formed by an objective)
    bool obj_pending = false;      // f of the last iteration not yet computed
    int64_t f_count = 0;
    int64_t iterations = 0;
    bool pg_on = false;                         // projected gradient recorded per iterate
    int64_t pg_base = 0;                        // first recorded iterate
    BppStats reported{};                        // stats already turned into a status
    bool timing = false;
    bool use_graph = false;                     // nmf_iterate captures a CUDA graph
    int64_t graph_launches = 0;                 // graphs launched by nmf_iterate
    int64_t mm_splits_max = 0;                  // largest contraction split of a product
    cudaGraphExec_t graph_exec = nullptr;       // last instantiated iteration graph
    int32_t graph_iters = 0;                    // its iteration count
    int64_t launches = 0;                       // kernels launched by nmf_iterate / objective
    double ms[5] = {0, 0, 0, 0, 0};             // gram, mm, nls, objective, proposal
    // Learned passive-set proposal (borrowed network; features buffer owned).
    nmf::MlpNet *mlp = nullptr;
    int32_t prop_mode = NMF_PROPOSAL_OFF;
    int32_t prop_epochs = 1;
    int64_t prop_batch = 8192;
    float prop_lr = 1e-3f;
    float *feat = nullptr;                      // max(m, n) x 3k
    struct Pending {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
};

static constexpr int64_t F_HIST_CAP = 1 << 16;

namespace {

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1));
}

cudaEvent_t take_event(nmf_handle *h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct PhaseTimer {
    nmf_handle *h;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseTimer(nmf_handle *hh, int ph, cudaStream_t st = nullptr)
        : h(hh), phase(ph), s(st ? st : hh->stream)
    {
        if (h->timing) {
            a = take_event(h);
            cudaEventRecord(a, s);
        }
    }
    ~PhaseTimer()
    {
        if (h->timing) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, s);
            h->pending.push_back({phase, a, b});
        }
    }
};

void collect_timing(nmf_handle *h)
{
    for (auto &p : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            h->ms[p.phase] += ms;
        h->pool.push_back(p.a);
        h->pool.push_back(p.b);
    }
    h->pending.clear();
}

nmf_status mm(nmf_handle *h, int trans, const float *F, float *out)
{
    const nmf_config &c = h->cfg;
    if (c.input_kind == NMF_INPUT_CSR) {
        if (trans == 0)
            return launch_spmm(h->A.rowptr, h->A.colidx, h->A.vals, c.m, F, c.k, out, h->stream);
        return launch_spmm(h->t_rowptr, h->t_colidx, h->t_vals, c.n, F, c.k, out, h->stream);
    }
    if (c.precision == NMF_PREC_BF16X3) {
        h->mm_splits_max = std::max<int64_t>(h->mm_splits_max, mm_tc_splits(c.m, c.n, trans));
        void *hi = trans ? h->at_hi : h->ar_hi, *lo = trans ? h->at_lo : h->ar_lo;
        if (hi)
            return launch_mm_tc_presplit(hi, lo, c.m, c.n, F, c.k, trans, out, nullptr, nullptr,
                                         h->tc_work, h->tc_work_bytes, h->stream);
        return launch_mm_tc(h->A.dense, c.m, c.n, h->A.lda, F, c.k, trans, out, h->tc_work,
                            h->tc_work_bytes, h->stream);
    }
    if (h->f32)
        return launch_mm_f32(h->A.dense, c.m, c.n, h->A.lda, F, c.k, trans, out, nullptr, nullptr,
                             h->tc_work, h->tc_work_bytes, h->stream);
    return launch_mm_simt(h->A.dense, c.m, c.n, h->A.lda, F, c.k, trans, out, h->stream);
}

// f(W, H) into *f_dev. Sparse input: after an H half-step (after_h) Y holds
// A^T W and GW = W^T W for the current W; otherwise both are formed here (Y
// and GW are scratch between iterations).
// A H^T into V with f(W, H) of the current factors fused (dense BF16x3, or
// dense FP32 through the packed-FMA kernel).
nmf_status mm_obj(nmf_handle *h, double *f_dev)
{
    const nmf_config &c = h->cfg;
    if (h->f32)
        return launch_mm_f32(h->A.dense, c.m, c.n, h->A.lda, h->Ht, c.k, 0, h->V, h->W, f_dev,
                             h->tc_work, h->tc_work_bytes, h->stream);
    if (h->ar_hi)
        return launch_mm_tc_presplit(h->ar_hi, h->ar_lo, c.m, c.n, h->Ht, c.k, 0, h->V, h->W,
                                     f_dev, h->tc_work, h->tc_work_bytes, h->stream);
    return launch_mm_tc_obj(h->A.dense, c.m, c.n, h->A.lda, h->Ht, c.k, 0, h->V, h->W, f_dev,
                            h->tc_work, h->tc_work_bytes, h->stream);
}

nmf_status objective_into(nmf_handle *h, double *f_dev, bool after_h = false)
{
    const nmf_config &c = h->cfg;
    if (h->fused_obj)
        return mm_obj(h, f_dev);
    if (c.input_kind == NMF_INPUT_CSR) {
        if (!after_h) {
            NMF_TRY(mm(h, 1, h->W, h->Y));
            NMF_TRY(launch_gram(h->W, c.m, c.k, h->GW, h->gram_part, h->stream));
        }
        NMF_TRY(launch_gram(h->Ht, c.n, c.k, h->GH, h->gram_part, h->stream));
        h->gh_current = true;   // the next W half-step reuses it
        return launch_objective_csr(h->Ht, h->Y, c.n, c.k, h->a_sq, h->GW, h->GH, h->obj_part,
                                    f_dev, h->stream);
    }
    return launch_objective_dense(h->A.dense, c.m, c.n, h->A.lda, h->W, h->Ht, c.k, c.precision,
                                  h->obj_part, f_dev, h->stream);
}

// The local update of one half-step: X (rows x k, the factor, updated in
// place) from Gram G and right-hand sides R. BPP: passive = that factor's
// bitmasks; with a network attached, its features are formed from the rows of
// X before the update; it proposes the starting partition (use) or learns from
// the final one (train). MU and HALS: one step of Eq. 5 or Eq. 6.
nmf_status solve_half(nmf_handle *h, int64_t rows, const double *G, const float *R, float *X,
                      uint64_t *passive, bool warm, const CsrGather *gather = nullptr)
{
    const nmf_config &c = h->cfg;
    if (c.solver != NMF_SOLVER_BPP) {
        PhaseTimer t(h, 2);
        return launch_local_update(c.solver, G, c.k, R, X, rows, h->stream);
    }
    const bool use = h->mlp && h->prop_mode == NMF_PROPOSAL_USE;
    const bool train = h->mlp && h->prop_mode == NMF_PROPOSAL_TRAIN;
    if (use) {
        PhaseTimer t(h, 4);
        NMF_TRY(mlp_features_propose(h->mlp, G, R, X, rows, h->feat, passive, h->stream));
    } else if (train) {
        PhaseTimer t(h, 4);
        NMF_TRY(mlp_features(G, R, X, rows, c.k, h->feat, h->stream));
    }
    {
        PhaseTimer t(h, 2);
        NMF_TRY(launch_bpp_solve(c.k, rows, G, R, X, (use || warm) ? passive : nullptr, passive,
                                 nullptr, nullptr, c.max_bpp_rounds, h->bpp_work, h->stats_dev,
                                 h->stream, gather));
    }
    if (train) {
        PhaseTimer t(h, 4);
        for (int e = 0; e < h->prop_epochs; ++e)
            NMF_TRY(mlp_train(h->mlp, h->feat, passive, rows, h->prop_batch, h->prop_lr, nullptr,
                              h->stream));
    }
    return NMF_OK;
}

nmf_status one_iteration(nmf_handle *h)
{
    const nmf_config &c = h->cfg;
    const bool warm = c.start_mode == NMF_START_WARM && h->passive_valid;
    // Side stream: Gram of the fixed factor, then the BPP preparation of that
    // Gram (both need only the fixed factor, current on the main stream at the
    // fork); the main stream runs the product meanwhile and joins before the
    // solves. The BPP workspace is free again at each fork: the previous
    // half-step's solves are on the main stream before it.
    auto fork_prepare = [&](const float *F, int64_t rows, double *G, bool have_gram) -> nmf_status {
        NMF_CUDA(cudaEventRecord(h->ev_fork, h->stream));
        NMF_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        PhaseTimer t(h, 0, h->side);
        if (!have_gram)
            NMF_TRY(launch_gram(F, rows, c.k, G, h->gram_part, h->side));
        if (c.solver == NMF_SOLVER_BPP)
            NMF_TRY(launch_bpp_prep(c.k, G, h->bpp_work, h->stats_dev, h->side));
        NMF_CUDA(cudaEventRecord(h->ev_join, h->side));
        return NMF_OK;
    };
    // Sparse BPP half-steps gather their right-hand sides inside the solves
    // (written to V / Y as they go) unless something reads them first: the
    // stopping measure or a proposal network.
    const bool fuse = c.input_kind == NMF_INPUT_CSR && c.solver == NMF_SOLVER_BPP &&
                      !c.no_fused_products && !h->pg_on && !h->mlp;
    const CsrGather gather_w{h->A.rowptr, h->A.colidx, h->A.vals, h->Ht};
    const CsrGather gather_h{h->t_rowptr, h->t_colidx, h->t_vals, h->W};
    // W <- argmin_{W >= 0} ||A - W H||: Gram H H^T, right-hand sides A H^T.
    NMF_TRY(fork_prepare(h->Ht, c.n, h->GH, h->gh_current));
    if (!fuse) {
        PhaseTimer t(h, 1);
        if (h->obj_pending) {
            // The previous iterate's f(W, H) rides on this A H^T pass.
            double *slot = h->f_hist + ((h->f_count - 1) % F_HIST_CAP);
            NMF_TRY(mm_obj(h, slot));
            h->obj_pending = false;
        } else {
            NMF_TRY(mm(h, 0, h->Ht, h->V));
        }
    }
    NMF_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    // Stopping measure of the current iterate (W, H), its part in W: this
    // half-step's Gram and right-hand sides are the iterate's own.
    if (h->pg_on)
        NMF_TRY(launch_pgrad_sq(h->GH, c.k, h->V, h->W, c.m, h->pg_part,
                                h->pgw2 + (h->iterations % F_HIST_CAP), h->stream));
    NMF_TRY(solve_half(h, c.m, h->GH, h->V, h->W, h->pW, warm, fuse ? &gather_w : nullptr));
    // H <- argmin_{H >= 0} ||A - W H||: Gram W^T W, right-hand sides (W^T A)^T.
    NMF_TRY(fork_prepare(h->W, c.m, h->GW, false));
    if (!fuse) {
        PhaseTimer t(h, 1);
        NMF_TRY(mm(h, 1, h->W, h->Y));
    }
    NMF_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    NMF_TRY(solve_half(h, c.n, h->GW, h->Y, h->Ht, h->pH, warm, fuse ? &gather_h : nullptr));
    h->gh_current = false;
    // ... and the new iterate's part in H (W^T W and A^T W of the new W).
    if (h->pg_on)
        NMF_TRY(launch_pgrad_sq(h->GW, c.k, h->Y, h->Ht, c.n, h->pg_part,
                                h->pgh2 + ((h->iterations + 1) % F_HIST_CAP), h->stream));
    h->passive_valid = true;
    if (c.objective_every) {
        if (h->fused_obj) {
            h->obj_pending = true;   // computed by the next A H^T pass or a flush
        } else {
            PhaseTimer t(h, 3);
            NMF_TRY(objective_into(h, h->f_hist + (h->f_count % F_HIST_CAP), true));
        }
        h->f_count += 1;
    }
    h->iterations += 1;
    return NMF_OK;
}

// Compute a pending objective (fused mode) into its history slot.
nmf_status flush_objective(nmf_handle *h)
{
    if (!h->obj_pending)
        return NMF_OK;
    const unsigned long long before = launch_count;
    PhaseTimer t(h, 3);
    const nmf_status st = objective_into(h, h->f_hist + ((h->f_count - 1) % F_HIST_CAP));
    h->launches += (int64_t)(launch_count - before);
    if (st == NMF_OK)
        h->obj_pending = false;
    return st;
}

void free_handle(nmf_handle *h)
{
    cudaFree(h->W);
    cudaFree(h->Ht);
    cudaFree(h->V);
    cudaFree(h->Y);
    cudaFree(h->GH);
    cudaFree(h->GW);
    cudaFree(h->pW);
    cudaFree(h->pH);
    cudaFree(h->bpp_work);
    cudaFree(h->stats_dev);
    cudaFree(h->gram_part);
    cudaFree(h->obj_part);
    cudaFree(h->at_hi);
    cudaFree(h->at_lo);
    cudaFree(h->ar_hi);
    cudaFree(h->ar_lo);
    cudaFree(h->pgw2);
    cudaFree(h->pgh2);
    cudaFree(h->pg_part);
    cudaFree(h->a_sq);
    cudaFree(h->f_hist);
    cudaFree(h->f_now);
    cudaFree(h->tc_work);
    cudaFree(h->t_rowptr);
    cudaFree(h->t_colidx);
    cudaFree(h->t_vals);
    cudaFree(h->feat);
    for (auto &p : h->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : h->pool)
        cudaEventDestroy(e);
    if (h->ev_fork)
        cudaEventDestroy(h->ev_fork);
    if (h->ev_join)
        cudaEventDestroy(h->ev_join);
    if (h->side)
        cudaStreamDestroy(h->side);
    if (h->graph_exec)
        cudaGraphExecDestroy(h->graph_exec);
    delete h;
}

}  // namespace

extern "C" nmf_status nmf_init(nmf_handle **out, const nmf_config *cfg, const nmf_matrix *A,
                               const float *W0, const float *Ht0, void *stream)
{
    if (!out || !cfg || !A || !W0 || !Ht0)
        return NMF_ERR_INVALID_ARG;
    *out = nullptr;
    const nmf_config c = *cfg;
    if (bad_k(c.k) || c.m < 1 || c.n < 1 || c.max_bpp_rounds < 0)
        return NMF_ERR_INVALID_ARG;
    if (c.precision != NMF_PREC_FP32 && c.precision != NMF_PREC_BF16X3)
        return NMF_ERR_INVALID_ARG;
    if (c.start_mode != NMF_START_COLD && c.start_mode != NMF_START_WARM)
        return NMF_ERR_INVALID_ARG;
    if (c.solver != NMF_SOLVER_BPP && c.solver != NMF_SOLVER_MU && c.solver != NMF_SOLVER_HALS)
        return NMF_ERR_INVALID_ARG;
    if ((c.no_split_copies != 0 && c.no_split_copies != 1) ||
        (c.no_fused_products != 0 && c.no_fused_products != 1))
        return NMF_ERR_INVALID_ARG;
    if (c.input_kind == NMF_INPUT_DENSE) {
        if (!A->dense || A->lda < c.n)
            return NMF_ERR_INVALID_ARG;
        // The tensor-core path reads A with TMA: 16-byte-aligned rows.
        if (c.precision == NMF_PREC_BF16X3 &&
            ((reinterpret_cast<uintptr_t>(A->dense) & 15) || (A->lda % 4)))
            return NMF_ERR_INVALID_ARG;
    } else if (c.input_kind == NMF_INPUT_CSR) {
        if (!A->rowptr || A->nnz < 0 || (A->nnz > 0 && (!A->colidx || !A->vals)))
            return NMF_ERR_INVALID_ARG;
    } else {
        return NMF_ERR_INVALID_ARG;
    }
    nmf_handle *h = new nmf_handle();
    h->cfg = c;
    h->A = *A;
    h->stream = as_stream(stream);
    h->nwords = (c.k + 63) / 64;
    // The side stream (Gram + BPP preparation, overlapping the product) gets
    // the highest priority, so its blocks are scheduled as soon as an SM frees
    // up instead of after every queued block of the product.
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_greatest) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        free_handle(h);
        return NMF_ERR_CUDA;
    }
    const size_t k = (size_t)c.k;
    const int64_t rmax = c.m > c.n ? c.m : c.n;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) {
        if (e == cudaSuccess)
            e = r;
    };
    chk(dalloc(&h->W, (size_t)c.m * k));
    chk(dalloc(&h->Ht, (size_t)c.n * k));
    chk(dalloc(&h->V, (size_t)c.m * k));
    chk(dalloc(&h->Y, (size_t)c.n * k));
    chk(dalloc(&h->GH, k * k));
    chk(dalloc(&h->GW, k * k));
    chk(dalloc(&h->pW, (size_t)c.m * h->nwords));
    chk(dalloc(&h->pH, (size_t)c.n * h->nwords));
    chk(cudaMalloc(&h->bpp_work, bpp_work_bytes(c.k)));
    chk(dalloc(&h->stats_dev, 1));
    chk(dalloc(&h->gram_part, (size_t)gram_partials_len(rmax, c.k)));
    chk(dalloc(&h->obj_part, (size_t)objective_partials_len()));
    chk(dalloc(&h->f_hist, (size_t)F_HIST_CAP));
    chk(dalloc(&h->f_now, 1));
    chk(dalloc(&h->pgw2, (size_t)F_HIST_CAP));
    chk(dalloc(&h->pgh2, (size_t)F_HIST_CAP));
    chk(dalloc(&h->pg_part, (size_t)pgrad_partials_len()));
    h->f32 = c.input_kind == NMF_INPUT_DENSE && c.precision == NMF_PREC_FP32 &&
             mm_f32_supported(A->dense, A->lda);
    h->fused_obj = c.input_kind == NMF_INPUT_DENSE && c.k <= 64 &&
                   (c.precision == NMF_PREC_BF16X3 || h->f32);
    if (e == cudaSuccess && h->f32) {
        h->tc_work_bytes = std::max(mm_f32_work_bytes(c.m, c.n, c.k, 0),
                                    mm_f32_work_bytes(c.m, c.n, c.k, 1));
        chk(cudaMalloc(&h->tc_work, h->tc_work_bytes));
    }
    if (e == cudaSuccess && c.input_kind == NMF_INPUT_DENSE && c.precision == NMF_PREC_BF16X3) {
        h->tc_work_bytes = mm_tc_work_bytes(c.m, c.n, c.k, 0);
        const size_t b1 = mm_tc_work_bytes(c.m, c.n, c.k, 1);
        if (b1 > h->tc_work_bytes)
            h->tc_work_bytes = b1;
        chk(cudaMalloc(&h->tc_work, h->tc_work_bytes ? h->tc_work_bytes : 16));
        // A and A^T split into BF16 hi / lo once (4 bytes per element of A
        // each): the products then need no per-call split (nor transpose).
        // Without the memory the handle splits A on the fly in every pass.
        auto alloc_pair = [&](void **hi, void **lo, size_t bytes) {
            if (cudaMalloc(hi, bytes) != cudaSuccess || cudaMalloc(lo, bytes) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(*hi);
                cudaFree(*lo);
                *hi = *lo = nullptr;
            }
        };
        if (e == cudaSuccess && !c.no_split_copies)
            alloc_pair(&h->at_hi, &h->at_lo, mm_tc_presplit_bytes(c.n, c.m));
        if (e == cudaSuccess && h->at_hi)
            alloc_pair(&h->ar_hi, &h->ar_lo, mm_tc_presplit_bytes(c.m, c.n));
    }
    if (e == cudaSuccess && c.input_kind == NMF_INPUT_CSR) {
        chk(dalloc(&h->t_rowptr, (size_t)c.n + 1));
        chk(dalloc(&h->t_colidx, (size_t)A->nnz));
        chk(dalloc(&h->t_vals, (size_t)A->nnz));
        chk(dalloc(&h->a_sq, 1));
    }
    if (e != cudaSuccess) {
        free_handle(h);
        return from_cuda(e, "nmf_init alloc");
    }
    nmf_status st = NMF_OK;
    auto run = [&]() -> nmf_status {
        NMF_CUDA(cudaMemsetAsync(h->stats_dev, 0, sizeof(BppStats), h->stream));
        NMF_CUDA(cudaMemsetAsync(h->pW, 0, sizeof(uint64_t) * (size_t)c.m * h->nwords, h->stream));
        NMF_CUDA(cudaMemsetAsync(h->pH, 0, sizeof(uint64_t) * (size_t)c.n * h->nwords, h->stream));
        NMF_CUDA(cudaMemcpyAsync(h->W, W0, sizeof(float) * (size_t)c.m * k,
                                 cudaMemcpyDeviceToDevice, h->stream));
        NMF_CUDA(cudaMemcpyAsync(h->Ht, Ht0, sizeof(float) * (size_t)c.n * k,
                                 cudaMemcpyDeviceToDevice, h->stream));
        if (h->at_hi)
            NMF_TRY(launch_mm_tc_presplit_make(A->dense, c.m, c.n, A->lda, 1, h->at_hi, h->at_lo,
                                               h->stream));
        if (h->ar_hi)
            NMF_TRY(launch_mm_tc_presplit_make(A->dense, c.m, c.n, A->lda, 0, h->ar_hi, h->ar_lo,
                                               h->stream));
        if (c.input_kind == NMF_INPUT_CSR) {
            unsigned long long *cursor = nullptr;
            NMF_CUDA(cudaMallocAsync(&cursor, sizeof(unsigned long long) * (size_t)c.n,
                                     h->stream));
            nmf_status s2 = launch_csr_transpose(A->rowptr, A->colidx, A->vals, c.m, c.n, A->nnz,
                                                 h->t_rowptr, h->t_colidx, h->t_vals, cursor,
                                                 h->stream);
            cudaFreeAsync(cursor, h->stream);
            NMF_TRY(s2);
            NMF_TRY(launch_sq_norm(A->vals, A->nnz, h->obj_part, h->a_sq, h->stream));
        }
        NMF_CUDA(cudaStreamSynchronize(h->stream));
        return NMF_OK;
    };
    st = run();
    if (st != NMF_OK) {
        free_handle(h);
        return st;
    }
    *out = h;
    return NMF_OK;
}

// Graph mode: the call's iterations are captured from the handle's stream
// (the side stream joins through the fork / join events) into one CUDA graph
// and launched once. Kernel arguments that change between calls (objective
// history slots) are captured per call. Not on the legacy default stream (it
// cannot be captured) or with per-task timing on (its events would be graph
// nodes): those calls run eagerly.
nmf_status iterate_graph(nmf_handle *h, int32_t iters)
{
    NMF_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    nmf_status st = NMF_OK;
    for (int32_t t = 0; t < iters && st == NMF_OK; ++t)
        st = one_iteration(h);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st != NMF_OK || e != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        return st != NMF_OK ? st : from_cuda(e, "cudaStreamEndCapture");
    }
    // A call with the same iteration count and state captures the same graph
    // shape with other arguments: update the instantiated graph in place
    // (much cheaper than instantiating); instantiate only when that fails.
    cudaError_t r = cudaErrorUnknown;
    if (h->graph_exec && h->graph_iters == iters) {
        cudaGraphExecUpdateResultInfo info;
        r = cudaGraphExecUpdate(h->graph_exec, g, &info);
        if (r != cudaSuccess)
            cudaGetLastError();   // clear the update failure; instantiate below
    }
    if (r != cudaSuccess) {
        if (h->graph_exec)
            cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        r = cudaGraphInstantiate(&h->graph_exec, g, 0);
        h->graph_iters = iters;
    }
    if (r == cudaSuccess)
        r = cudaGraphLaunch(h->graph_exec, h->stream);
    cudaGraphDestroy(g);
    NMF_CUDA(r);
    return NMF_OK;
}

extern "C" nmf_status nmf_iterate(nmf_handle *h, int32_t iters)
{
    if (!h || iters < 0)
        return NMF_ERR_INVALID_ARG;
    const unsigned long long before = launch_count;
    nmf_status st = NMF_OK;
    if (h->use_graph && iters > 0 && h->stream != nullptr && !h->timing) {
        st = iterate_graph(h, iters);
        h->graph_launches += 1;
    } else {
        for (int32_t t = 0; t < iters && st == NMF_OK; ++t)
            st = one_iteration(h);
    }
    h->launches += (int64_t)(launch_count - before);
    return st;
}

extern "C" nmf_status nmf_set_graph(nmf_handle *h, int32_t on)
{
    if (!h)
        return NMF_ERR_INVALID_ARG;
    h->use_graph = on != 0;
    return NMF_OK;
}

extern "C" nmf_status nmf_sync(nmf_handle *h)
{
    if (!h)
        return NMF_ERR_INVALID_ARG;
    // A pending fused objective stays pending: the next iteration's A H^T
    // pass computes it, or reading the objective flushes it.
    BppStats st;
    NMF_CUDA(cudaMemcpyAsync(&st, h->stats_dev, sizeof(BppStats), cudaMemcpyDeviceToHost,
                             h->stream));
    NMF_CUDA(cudaStreamSynchronize(h->stream));
    BppStats delta = st;
    delta.not_converged -= h->reported.not_converged;
    delta.singular -= h->reported.singular;
    delta.nonfinite -= h->reported.nonfinite;
    h->reported = st;
    return worst_from_stats(delta);
}

extern "C" nmf_status nmf_objective(nmf_handle *h, double *f_out)
{
    if (!h || !f_out)
        return NMF_ERR_INVALID_ARG;
    NMF_TRY(flush_objective(h));
    const unsigned long long before = launch_count;
    const nmf_status st = objective_into(h, h->f_now);
    h->launches += (int64_t)(launch_count - before);
    NMF_TRY(st);
    NMF_CUDA(cudaMemcpyAsync(f_out, h->f_now, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    NMF_CUDA(cudaStreamSynchronize(h->stream));
    return NMF_OK;
}

extern "C" nmf_status nmf_objective_history(nmf_handle *h, double *f_host, int64_t cap,
                                            int64_t *count)
{
    if (!h || !count || cap < 0 || (cap > 0 && !f_host))
        return NMF_ERR_INVALID_ARG;
    NMF_TRY(flush_objective(h));
    NMF_CUDA(cudaStreamSynchronize(h->stream));
    const int64_t avail = h->f_count < F_HIST_CAP ? h->f_count : F_HIST_CAP;
    const int64_t nout = avail < cap ? avail : cap;
    const int64_t first = h->f_count - nout;   // oldest value copied
    for (int64_t q = 0; q < nout; ++q) {
        const int64_t slot = (first + q) % F_HIST_CAP;
        NMF_CUDA(cudaMemcpy(f_host + q, h->f_hist + slot, sizeof(double),
                            cudaMemcpyDeviceToHost));
    }
    *count = nout;
    return NMF_OK;
}

extern "C" nmf_status nmf_get_factors(nmf_handle *h, float *W, float *Ht)
{
    if (!h)
        return NMF_ERR_INVALID_ARG;
    const size_t k = (size_t)h->cfg.k;
    if (W)
        NMF_CUDA(cudaMemcpyAsync(W, h->W, sizeof(float) * (size_t)h->cfg.m * k,
                                 cudaMemcpyDeviceToDevice, h->stream));
    if (Ht)
        NMF_CUDA(cudaMemcpyAsync(Ht, h->Ht, sizeof(float) * (size_t)h->cfg.n * k,
                                 cudaMemcpyDeviceToDevice, h->stream));
    return NMF_OK;
}

extern "C" nmf_status nmf_set_factors(nmf_handle *h, const float *W, const float *Ht)
{
    if (!h)
        return NMF_ERR_INVALID_ARG;
    NMF_TRY(flush_objective(h));
    const size_t k = (size_t)h->cfg.k;
    if (W)
        NMF_CUDA(cudaMemcpyAsync(h->W, W, sizeof(float) * (size_t)h->cfg.m * k,
                                 cudaMemcpyDeviceToDevice, h->stream));
    if (Ht)
        NMF_CUDA(cudaMemcpyAsync(h->Ht, Ht, sizeof(float) * (size_t)h->cfg.n * k,
                                 cudaMemcpyDeviceToDevice, h->stream));
    if (Ht)
        h->gh_current = false;
    h->passive_valid = false;
    h->pg_on = false;   // the recorded measures belong to the replaced iterates
    return NMF_OK;
}

extern "C" nmf_status nmf_set_pgrad(nmf_handle *h, int32_t on)
{
    if (!h)
        return NMF_ERR_INVALID_ARG;
    if (!on) {
        h->pg_on = false;
        return NMF_OK;
    }
    if (h->pg_on)
        return NMF_OK;
    const nmf_config &c = h->cfg;
    // The current iterate's part in H needs A^T W and W^T W of the current W
    // (the iteration forms them only for the next W).
    const unsigned long long before = launch_count;
    nmf_status st = mm(h, 1, h->W, h->Y);
    if (st == NMF_OK)
        st = launch_gram(h->W, c.m, c.k, h->GW, h->gram_part, h->stream);
    if (st == NMF_OK)
        st = launch_pgrad_sq(h->GW, c.k, h->Y, h->Ht, c.n, h->pg_part,
                             h->pgh2 + (h->iterations % F_HIST_CAP), h->stream);
    h->launches += (int64_t)(launch_count - before);
    NMF_TRY(st);
    h->pg_on = true;
    h->pg_base = h->iterations;
    return NMF_OK;
}

// Delta of recorded iterate t (complete once iteration t + 1 has run).
static nmf_status pgrad_of(nmf_handle *h, int64_t t, double *out)
{
    double w2 = 0.0, h2 = 0.0;
    const int64_t slot = t % F_HIST_CAP;
    NMF_CUDA(cudaMemcpyAsync(&w2, h->pgw2 + slot, sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    NMF_CUDA(cudaMemcpyAsync(&h2, h->pgh2 + slot, sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    NMF_CUDA(cudaStreamSynchronize(h->stream));
    *out = sqrt(w2 + h2);
    return NMF_OK;
}

extern "C" nmf_status nmf_pgrad_history(nmf_handle *h, double *out, int64_t cap, int64_t *count)
{
    if (!h || !count || cap < 0 || (cap > 0 && !out))
        return NMF_ERR_INVALID_ARG;
    *count = 0;
    if (!h->pg_on)
        return NMF_OK;
    int64_t avail = h->iterations - h->pg_base;   // complete iterates
    if (avail > F_HIST_CAP)
        avail = F_HIST_CAP;
    const int64_t nout = avail < cap ? avail : cap;
    const int64_t first = h->iterations - nout;
    for (int64_t q = 0; q < nout; ++q)
        NMF_TRY(pgrad_of(h, first + q, out + q));
    *count = nout;
    return NMF_OK;
}

extern "C" nmf_status nmf_iterate_until(nmf_handle *h, int32_t max_iters, double rel_tol,
                                        int32_t *iters_done, double *ratio)
{
    if (!h || max_iters < 0 || !(rel_tol >= 0.0))
        return NMF_ERR_INVALID_ARG;
    if (iters_done)
        *iters_done = 0;
    if (ratio)
        *ratio = NAN;
    NMF_TRY(nmf_set_pgrad(h, 1));
    double d0 = -1.0;
    for (int32_t done = 0; done < max_iters;) {
        NMF_TRY(nmf_iterate(h, 1));
        done += 1;
        if (iters_done)
            *iters_done = done;
        if (d0 < 0.0)
            NMF_TRY(pgrad_of(h, h->pg_base, &d0));
        double dt = 0.0;
        NMF_TRY(pgrad_of(h, h->iterations - 1, &dt));
        if (ratio)
            *ratio = d0 > 0.0 ? dt / d0 : 0.0;
        if (dt <= rel_tol * d0)
            break;
    }
    return NMF_OK;
}

extern "C" nmf_status nmf_pgrad_sq(int32_t k, int64_t rows, const double *G, const float *R,
                                   const float *X, double *out, void *stream)
{
    if (bad_k(k) || rows < 0 || !G || !out || (rows > 0 && (!R || !X)))
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    double *buf = nullptr;   // partials, then the sum
    NMF_CUDA(cudaMallocAsync(&buf, sizeof(double) * (size_t)(pgrad_partials_len() + 1), s));
    nmf_status st = launch_pgrad_sq(G, k, R, X, rows, buf, buf + pgrad_partials_len(), s);
    if (st == NMF_OK &&
        cudaMemcpyAsync(out, buf + pgrad_partials_len(), sizeof(double), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess)
        st = NMF_ERR_CUDA;
    cudaFreeAsync(buf, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == NMF_OK)
        st = NMF_ERR_CUDA;
    return st;
}

extern "C" nmf_status nmf_get_passive(nmf_handle *h, uint64_t *pW, uint64_t *pH)
{
    if (!h)
        return NMF_ERR_INVALID_ARG;
    if (pW)
        NMF_CUDA(cudaMemcpyAsync(pW, h->pW, sizeof(uint64_t) * (size_t)h->cfg.m * h->nwords,
                                 cudaMemcpyDeviceToDevice, h->stream));
    if (pH)
        NMF_CUDA(cudaMemcpyAsync(pH, h->pH, sizeof(uint64_t) * (size_t)h->cfg.n * h->nwords,
                                 cudaMemcpyDeviceToDevice, h->stream));
    return NMF_OK;
}

extern "C" nmf_status nmf_get_stats(nmf_handle *h, nmf_stats *out)
{
    if (!h || !out)
        return NMF_ERR_INVALID_ARG;
    BppStats st;
    NMF_CUDA(cudaMemcpyAsync(&st, h->stats_dev, sizeof(BppStats), cudaMemcpyDeviceToHost,
                             h->stream));
    NMF_CUDA(cudaStreamSynchronize(h->stream));
    collect_timing(h);
    memset(out, 0, sizeof(*out));
    out->iterations = h->iterations;
    out->bpp_rhs = (int64_t)st.rhs;
    out->bpp_rounds = (int64_t)st.rounds;
    out->bpp_max_rounds = (int64_t)st.max_rounds;
    out->bpp_fp64_solves = (int64_t)st.fp64_solves;
    out->bpp_fp64_halfsteps = (int64_t)st.fp64_halfsteps;
    out->bpp_not_converged = (int64_t)st.not_converged;
    out->bpp_singular = (int64_t)st.singular;
    out->ms_gram = h->ms[0];
    out->ms_mm = h->ms[1];
    out->ms_nls = h->ms[2];
    out->ms_objective = h->ms[3];
    out->kernel_launches = h->launches;
    out->ms_proposal = h->ms[4];
    out->graph_launches = h->graph_launches;
    out->mm_splits_max = h->mm_splits_max;
    return NMF_OK;
}

extern "C" nmf_status nmf_set_timing(nmf_handle *h, int32_t timing)
{
    if (!h)
        return NMF_ERR_INVALID_ARG;
    h->timing = timing != 0;
    return NMF_OK;
}

extern "C" void nmf_destroy(nmf_handle *h)
{
    if (!h)
        return;
    cudaStreamSynchronize(h->stream);
    free_handle(h);
}

// ===========================================================================
// Learned passive-set proposal.
// ===========================================================================

struct nmf_mlp {
    nmf::MlpNet *net;
};

extern "C" int64_t nmf_mlp_param_count(int32_t k, int32_t hidden)
{
    if (k < 1 || k > NMF_MAX_K || hidden < 1 || hidden > 1024)
        return 0;
    return mlp_param_count(k, hidden);
}

extern "C" nmf_status nmf_mlp_create(nmf_mlp **out, int32_t k, int32_t hidden,
                                     const float *params, void *stream)
{
    if (!out || !params || k < 1 || k > NMF_MAX_K || hidden < 1 || hidden > 1024)
        return NMF_ERR_INVALID_ARG;
    *out = nullptr;
    nmf::MlpNet *net = nullptr;
    NMF_TRY(mlp_create(&net, k, hidden, params, as_stream(stream)));
    *out = new nmf_mlp{net};
    return NMF_OK;
}

extern "C" nmf_status nmf_mlp_get_params(const nmf_mlp *h, float *params, void *stream)
{
    if (!h || !params)
        return NMF_ERR_INVALID_ARG;
    NMF_CUDA(cudaMemcpyAsync(params, mlp_master(h->net), sizeof(float) * (size_t)mlp_nparams(h->net),
                             cudaMemcpyDeviceToDevice, as_stream(stream)));
    return NMF_OK;
}

extern "C" void nmf_mlp_destroy(nmf_mlp *h)
{
    if (!h)
        return;
    mlp_destroy(h->net);
    delete h;
}

extern "C" nmf_status nmf_mlp_features(const double *G, const float *B, const float *Xprev,
                                       int64_t nrhs, int32_t k, float *F, void *stream)
{
    if (!G || k < 1 || k > NMF_MAX_K || nrhs < 0 || (nrhs > 0 && (!B || !F)))
        return NMF_ERR_INVALID_ARG;
    return mlp_features(G, B, Xprev, nrhs, k, F, as_stream(stream));
}

extern "C" nmf_status nmf_mlp_forward(nmf_mlp *h, const float *F, int64_t nrhs, float *logits,
                                      void *stream)
{
    if (!h || nrhs < 0 || nrhs > INT32_MAX || (nrhs > 0 && (!F || !logits)))
        return NMF_ERR_INVALID_ARG;
    return mlp_logits(h->net, F, nrhs, logits, as_stream(stream));
}

extern "C" nmf_status nmf_mlp_propose(nmf_mlp *h, const float *F, int64_t nrhs,
                                      uint64_t *passive, void *stream)
{
    if (!h || nrhs < 0 || nrhs > INT32_MAX || (nrhs > 0 && (!F || !passive)))
        return NMF_ERR_INVALID_ARG;
    return mlp_propose(h->net, F, nrhs, passive, as_stream(stream));
}

extern "C" nmf_status nmf_mlp_gradient(nmf_mlp *h, const float *F, const uint64_t *passive,
                                       int64_t nrhs, float *grad, double *loss, void *stream)
{
    if (!h || !F || !passive || nrhs < 1 || nrhs > INT32_MAX)
        return NMF_ERR_INVALID_ARG;
    return mlp_gradient(h->net, F, passive, nrhs, grad, loss, as_stream(stream));
}

extern "C" nmf_status nmf_mlp_train(nmf_mlp *h, const float *F, const uint64_t *passive,
                                    int64_t nrhs, int64_t batch, float lr, double *loss,
                                    void *stream)
{
    if (!h || !F || !passive || nrhs < 1 || batch < 1 || batch > INT32_MAX || !(lr > 0.0f))
        return NMF_ERR_INVALID_ARG;
    return mlp_train(h->net, F, passive, nrhs, batch, lr, loss, as_stream(stream));
}

extern "C" nmf_status nmf_set_proposal(nmf_handle *h, nmf_mlp *mlp, int32_t mode, int32_t epochs,
                                       int64_t batch, float lr)
{
    if (!h || mode < NMF_PROPOSAL_OFF || mode > NMF_PROPOSAL_USE)
        return NMF_ERR_INVALID_ARG;
    if (!mlp || mode == NMF_PROPOSAL_OFF) {
        h->mlp = nullptr;
        h->prop_mode = NMF_PROPOSAL_OFF;
        return NMF_OK;
    }
    // The network proposes BPP starting partitions: no meaning for MU or HALS.
    if (h->cfg.solver != NMF_SOLVER_BPP || mlp_k(mlp->net) != h->cfg.k || epochs < 0 ||
        batch < 1 || batch > INT32_MAX || !(lr > 0.0f))
        return NMF_ERR_INVALID_ARG;
    if (!h->feat) {
        const int64_t rows = h->cfg.m > h->cfg.n ? h->cfg.m : h->cfg.n;
        NMF_CUDA(cudaMalloc(&h->feat, sizeof(float) * (size_t)rows * 3 * h->cfg.k));
    }
    h->mlp = mlp->net;
    h->prop_mode = mode;
    h->prop_epochs = epochs;
    h->prop_batch = batch;
    h->prop_lr = lr;
    return NMF_OK;
}
