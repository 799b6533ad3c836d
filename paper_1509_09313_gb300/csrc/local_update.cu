// The paper's alternative local updates for the two steps of Alg. 1: MU
// (Eq. 5) and HALS (Eq. 6). Both take the same inputs as the BPP solves, the
// k x k Gram G of the fixed factor and the right-hand sides R (A H^T for W,
// (W^T A)^T for H^T), and update the rows of the other factor X in place.
//
//   MU    x_ij <- x_ij R_ij / (X G)_ij, all from the X before the step; where
//         (X G)_ij is not positive x_ij is left as it is (0 is a fixed point).
//   HALS  for i = 0..k-1 in order: x_i <- [R_i - sum_{l != i} G_li x_l]_+ / G_ii,
//         with the newest values of the other entries; a column with
//         G_ii <= 0 is set to 0.
//
// Rows are independent: one warp per row, lane l holding entries l, l + 32,
// ... (KW slots), G in FP32 in shared memory lane-interleaved (entry (r, c) at
// r * 32 KW + (c % 32) * KW + c / 32) so that a lane reads its KW entries of a
// row as one vector. MU forms X G with one product. HALS forms each
// coordinate's off-diagonal sum sum_{l != i} G_li x_l afresh, a warp dot
// product with G staged with a zero diagonal. Keeping x G and adding d times
// row i of G after each change would save the dot products but loses digits:
// HALS often drives whole columns to zero, and the large steps d = -x_i leave
// the updated sums as the rounding residue of a cancellation (measured on the
// sparse 20000 x 10000 test: 1e-3 relative factor error after five iterations,
// against 1e-7 for the direct form).
//
// The same row kernel also forms the projected-gradient norm of the
// stopping rule (Lin 2007): grad = X G - R, an entry counting where x_ij > 0
// and, where x_ij = 0, only if negative; squares summed in FP32 per row, FP64
// across rows, per-CTA partials added in a fixed order.
//
// Roofline: HBM (12 k bytes per row: R and X in, X out); 2 k^2 FLOPs per row.
#include "common.cuh"

namespace nmf {
namespace {

constexpr int LU_WARPS = 8;
enum LuOp { LU_MU = 0, LU_HALS = 1, LU_PGRAD = 2 };

template <int KW>
__device__ __forceinline__ void lu_row_fma(const float *__restrict__ p, float a, float (&acc)[KW])
{
    if constexpr (KW == 1) {
        acc[0] = fmaf(p[0], a, acc[0]);
    } else if constexpr (KW == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        acc[0] = fmaf(q.x, a, acc[0]);
        acc[1] = fmaf(q.y, a, acc[1]);
    } else {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        acc[0] = fmaf(q.x, a, acc[0]);
        acc[1] = fmaf(q.y, a, acc[1]);
        acc[2] = fmaf(q.z, a, acc[2]);
        acc[3] = fmaf(q.w, a, acc[3]);
    }
}

template <int KW, int OP>
__global__ void __launch_bounds__(LU_WARPS * 32)
    local_update_kernel(const double *__restrict__ G, int k, const float *__restrict__ R,
                        float *__restrict__ X, int64_t rows, double *__restrict__ partials)
{
    constexpr bool HALS = OP == LU_HALS;
    constexpr int RS = 32 * KW;
    extern __shared__ __align__(16) float lu_smem[];
    const int k4 = (k + 3) & ~3;
    float *Gs = lu_smem;                                    // k4 x RS
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *stage = Gs + k4 * RS + warp * RS;                // per-warp vector
    for (int e = threadIdx.x; e < k4 * RS; e += blockDim.x) {
        const int r = e / RS, q = e - r * RS;
        const int c = q / KW + 32 * (q % KW);
        Gs[e] = (r < k && c < k && !(HALS && r == c)) ? (float)G[r * k + c] : 0.0f;
    }
    __syncthreads();
    float gdiag[KW];   // G_ii of the lane's entries
#pragma unroll
    for (int s = 0; s < KW; ++s) {
        const int i = lane + 32 * s;
        gdiag[s] = i < k ? (float)G[i * k + i] : 0.0f;
    }
    const int64_t nwarps = (int64_t)gridDim.x * LU_WARPS;
    double pg = 0.0;   // LU_PGRAD: this lane's sum of squares
    for (int64_t row = (int64_t)blockIdx.x * LU_WARPS + warp; row < rows; row += nwarps) {
        float x[KW], r[KW], t[KW];
#pragma unroll
        for (int s = 0; s < KW; ++s) {
            const int i = lane + 32 * s;
            x[s] = i < k ? X[row * k + i] : 0.0f;
            r[s] = i < k ? R[row * k + i] : 0.0f;
            t[s] = 0.0f;
            if (!HALS)
                stage[32 * s + lane] = x[s];
        }
        __syncwarp();
        const float *base = Gs + lane * KW;
        if (!HALS) {
            // t = x G (G symmetric: t_i = sum_l x_l G_li, row l of G times x_l).
            for (int l = 0; l < k4; l += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(stage + l);
                lu_row_fma<KW>(base + (l + 0) * RS, v.x, t);
                lu_row_fma<KW>(base + (l + 1) * RS, v.y, t);
                lu_row_fma<KW>(base + (l + 2) * RS, v.z, t);
                lu_row_fma<KW>(base + (l + 3) * RS, v.w, t);
            }
            __syncwarp();   // stage is rewritten for the next row
            if constexpr (OP == LU_PGRAD) {
                float sq = 0.0f;
#pragma unroll
                for (int s = 0; s < KW; ++s) {
                    const float gr = t[s] - r[s];
                    const float pj = x[s] > 0.0f ? gr : fminf(gr, 0.0f);
                    sq = fmaf(pj, pj, sq);
                }
                pg += (double)sq;
            } else {
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    if (t[s] > 0.0f)
                        x[s] = x[s] * r[s] / t[s];
            }
        } else {
            for (int i = 0; i < k; ++i) {
                // sum_{l != i} G_il x_l: this lane's entries of row i (the
                // staged diagonal is zero), then a butterfly sum (fixed order).
                float part[KW];
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    part[s] = 0.0f;
                lu_row_fma<KW>(base + i * RS, 1.0f, part);
                float sum = 0.0f;
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    sum = fmaf(part[s], x[s], sum);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    sum += __shfl_xor_sync(FULL, sum, o);
                const int si = i >> 5, owner = i & 31;
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    if (s == si && lane == owner) {
                        const float gii = gdiag[s];
                        const float num = r[s] - sum;
                        x[s] = gii > 0.0f ? (num > 0.0f ? num : 0.0f) / gii : 0.0f;
                    }
            }
        }
        if (OP != LU_PGRAD) {
#pragma unroll
            for (int s = 0; s < KW; ++s) {
                const int i = lane + 32 * s;
                if (i < k)
                    X[row * k + i] = x[s];
            }
        }
    }
    if (OP == LU_PGRAD) {
        __shared__ double red[LU_WARPS];
        for (int o = 16; o > 0; o >>= 1)
            pg += __shfl_xor_sync(FULL, pg, o);
        if (lane == 0)
            red[warp] = pg;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int w = 0; w < LU_WARPS; ++w)
                b += red[w];
            partials[blockIdx.x] = b;
        }
    }
}

// out = sum of partials[0..n) in index order.
__global__ void lu_sum_kernel(const double *__restrict__ partials, int n, double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            s += partials[i];
        *out = s;
    }
}

// LU_PGRAD writes one partial per CTA (at most max_parts); *nparts gets the
// count.
template <int KW, int OP>
nmf_status launch_lu(const double *G, int k, const float *R, float *X, int64_t rows,
                     double *partials, int max_parts, int *nparts, cudaStream_t s)
{
    const size_t smem = sizeof(float) * (size_t)(((k + 3) & ~3) + LU_WARPS) * 32 * KW;
    static SmemOptIn opt_in;
    NMF_TRY(ensure_smem(local_update_kernel<KW, OP>, opt_in, smem));
    int per_sm = 0;
    NMF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, local_update_kernel<KW, OP>, LU_WARPS * 32, smem));
    int64_t blocks = (int64_t)(per_sm > 0 ? per_sm : 1) * sm_count();
    const int64_t need = cdiv(rows, LU_WARPS);
    if (need < blocks)
        blocks = need;
    if (OP == LU_PGRAD && blocks > max_parts)
        blocks = max_parts;
    if (blocks < 1)
        blocks = 1;
    local_update_kernel<KW, OP><<<(unsigned)blocks, LU_WARPS * 32, smem, s>>>(G, k, R, X, rows,
                                                                            partials);
    NMF_LAUNCHED(OP == LU_HALS ? "local_update_kernel<hals>"
                 : OP == LU_MU ? "local_update_kernel<mu>"
                               : "local_update_kernel<pgrad>");
    *nparts = (int)blocks;
    return NMF_OK;
}

template <int OP>
nmf_status launch_lu_k(const double *G, int k, const float *R, float *X, int64_t rows,
                       double *partials, int max_parts, int *nparts, cudaStream_t s)
{
    if (k <= 32)
        return launch_lu<1, OP>(G, k, R, X, rows, partials, max_parts, nparts, s);
    if (k <= 64)
        return launch_lu<2, OP>(G, k, R, X, rows, partials, max_parts, nparts, s);
    return launch_lu<4, OP>(G, k, R, X, rows, partials, max_parts, nparts, s);
}

}  // namespace

nmf_status launch_local_update(int solver, const double *G, int k, const float *R, float *X,
                               int64_t rows, cudaStream_t s)
{
    if (rows == 0)
        return NMF_OK;
    int np = 0;
    if (solver == NMF_SOLVER_MU)
        return launch_lu_k<LU_MU>(G, k, R, X, rows, nullptr, 0, &np, s);
    if (solver == NMF_SOLVER_HALS)
        return launch_lu_k<LU_HALS>(G, k, R, X, rows, nullptr, 0, &np, s);
    return NMF_ERR_INVALID_ARG;
}

int pgrad_partials_len() { return 2 * sm_count(); }

nmf_status launch_pgrad_sq(const double *G, int k, const float *R, const float *X, int64_t rows,
                           double *partials, double *out, cudaStream_t s)
{
    int np = 0;
    if (rows > 0)
        NMF_TRY(launch_lu_k<LU_PGRAD>(G, k, R, const_cast<float *>(X), rows, partials,
                                      pgrad_partials_len(), &np, s));
    lu_sum_kernel<<<1, 32, 0, s>>>(partials, np, out);
    NMF_LAUNCHED("lu_sum_kernel");
    return NMF_OK;
}

}  // namespace nmf

extern "C" nmf_status nmf_update_mu(int32_t k, int64_t rows, const double *G, const float *R,
                                    float *X, void *stream)
{
    if (k < 1 || k > NMF_MAX_K || rows < 0 || !G || (rows > 0 && (!R || !X)))
        return NMF_ERR_INVALID_ARG;
    return nmf::launch_local_update(NMF_SOLVER_MU, G, k, R, X, rows,
                                    static_cast<cudaStream_t>(stream));
}

extern "C" nmf_status nmf_update_hals(int32_t k, int64_t rows, const double *G, const float *R,
                                      float *X, void *stream)
{
    if (k < 1 || k > NMF_MAX_K || rows < 0 || !G || (rows > 0 && (!R || !X)))
        return NMF_ERR_INVALID_ARG;
    return nmf::launch_local_update(NMF_SOLVER_HALS, G, k, R, X, rows,
                                    static_cast<cudaStream_t>(stream));
}
