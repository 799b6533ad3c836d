// Objective of Eq. 1, f(W, H) = ||A - W H||_F^2.
//
// Dense A: every element's residual A_ij - w_i . h_j is formed directly (the
// expansion ||A||^2 - 2 tr(W^T A H^T) + tr(W^T W H H^T) cancels badly in
// floating point when the fit is good). A persistent grid walks 128 x 64
// tiles of A: the W rows and H^T rows of the tile are staged in shared memory
// (r-major), each thread forms an 8 x 4 block of W H with FP32 FMAs, subtracts
// it from A and adds the 32 squares in FP32, then into an FP64 accumulator.
// Per-CTA FP64 partials are summed in CTA order by a one-block kernel.
//
// Sparse A (CSR): the sum over all m*n positions splits exactly into
//   f = ||A||^2 - 2 sum_{stored} A_ij w_i.h_j + trace((W^T W)(H H^T)),
// and the cross term regroups by column: sum_j h_j . (A^T W)_j. The caller
// passes Y = A^T W (n x k; the right-hand sides of the H half-step, so no
// stored entry is revisited), and the cross term is one dot product of two
// n x k arrays (FP32 within a float4, FP64 across them). The trace uses the
// FP64 Grams; ||A||^2 is summed once when the matrix is loaded. A is not low
// rank, so the fit is loose and the three terms do not cancel badly.
#include "common.cuh"

namespace nmf {
namespace {

constexpr int OBJ_THREADS = 256;
constexpr int OBJ_BI = 128;
constexpr int OBJ_BJ = 64;
constexpr int OBJ_KC = 32;   // k-chunk staged in shared memory at a time

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(FULL, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            s += red[w];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(OBJ_THREADS)
    objective_dense_kernel(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                           const float *__restrict__ W, const float *__restrict__ Ht, int k,
                           double *__restrict__ partials)
{
    __shared__ __align__(16) float Ws[OBJ_KC][OBJ_BI];
    __shared__ __align__(16) float Hs[OBJ_KC][OBJ_BJ];
    __shared__ double red[OBJ_THREADS / 32];
    const int tid = threadIdx.x;
    const int ti = tid / 16, tj = tid % 16;   // 16 x 16 threads: 8 rows x 4 cols each
    const int64_t nti = cdiv(m, OBJ_BI), ntj = cdiv(n, OBJ_BJ);
    const int64_t ntiles = nti * ntj;
    double acc64 = 0.0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t i0 = (t / ntj) * OBJ_BI, j0 = (t % ntj) * OBJ_BJ;
        float wh[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                wh[a][b] = 0.0f;
        for (int r0 = 0; r0 < k; r0 += OBJ_KC) {
            const int kc = min(OBJ_KC, k - r0);
            for (int e = tid; e < OBJ_KC * OBJ_BI; e += OBJ_THREADS) {
                const int i = e / OBJ_KC, r = e % OBJ_KC;
                const int64_t gi = i0 + i;
                Ws[r][i] = (gi < m && r < kc) ? W[gi * k + r0 + r] : 0.0f;
            }
            for (int e = tid; e < OBJ_KC * OBJ_BJ; e += OBJ_THREADS) {
                const int j = e / OBJ_KC, r = e % OBJ_KC;
                const int64_t gj = j0 + j;
                Hs[r][j] = (gj < n && r < kc) ? Ht[gj * k + r0 + r] : 0.0f;
            }
            __syncthreads();
            for (int r = 0; r < kc; ++r) {
                const float4 w0 = *reinterpret_cast<const float4 *>(&Ws[r][ti * 8]);
                const float4 w1 = *reinterpret_cast<const float4 *>(&Ws[r][ti * 8 + 4]);
                const float4 h = *reinterpret_cast<const float4 *>(&Hs[r][tj * 4]);
                const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        wh[a][b] = fmaf(wv[a], hv[b], wh[a][b]);
            }
            __syncthreads();
        }
        float sq = 0.0f;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int64_t i = i0 + ti * 8 + a;
            if (i >= m)
                continue;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t j = j0 + tj * 4 + b;
                if (j < n) {
                    const float d = A[i * lda + j] - wh[a][b];
                    sq = fmaf(d, d, sq);
                }
            }
        }
        acc64 += (double)sq;
    }
    const double s = block_sum(acc64, red);
    if (tid == 0)
        partials[blockIdx.x] = s;
}

// f = base + scale * sum(partials) + trace(GW GH) (GW null: no trace), the
// three sums formed separately in a fixed order.
__global__ void sum_partials_kernel(const double *__restrict__ partials, int nparts, double scale,
                                    const double *__restrict__ base,
                                    const double *__restrict__ GW, const double *__restrict__ GH,
                                    int k, double *__restrict__ f_dev)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x)
        s += partials[p];
    const double S = block_sum(s, red);
    double t = 0.0;
    if (GW)
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int a = e / k, b = e % k;
            t += GW[a * k + b] * GH[b * k + a];
        }
    const double T = block_sum(t, red);
    if (threadIdx.x == 0)
        *f_dev = (base ? *base : 0.0) + scale * S + T;
}

// Per-block FP64 partial sums of sum_e X_e Y_e (float4 loads when both
// arrays are 16-byte aligned; products within a float4 summed in FP32).
__global__ void __launch_bounds__(OBJ_THREADS)
    dot_partials_kernel(const float *__restrict__ X, const float *__restrict__ Y, int64_t len,
                        int vec, double *__restrict__ partials)
{
    __shared__ double red[OBJ_THREADS / 32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    int64_t done = 0;
    if (vec) {
        const int64_t n4 = len >> 2;
        const float4 *X4 = reinterpret_cast<const float4 *>(X);
        const float4 *Y4 = reinterpret_cast<const float4 *>(Y);
        for (int64_t e = t0; e < n4; e += stride) {
            const float4 a = X4[e], b = Y4[e];
            float d = a.x * b.x;
            d = fmaf(a.y, b.y, d);
            d = fmaf(a.z, b.z, d);
            d = fmaf(a.w, b.w, d);
            acc += (double)d;
        }
        done = n4 << 2;
    }
    for (int64_t e = done + t0; e < len; e += stride)
        acc += (double)(X[e] * Y[e]);
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = t;
}

int obj_parts() { return 2 * sm_count(); }

}  // namespace

int64_t objective_partials_len() { return obj_parts(); }

nmf_status launch_sum_partials(const double *partials, int parts, double *f_dev, cudaStream_t s)
{
    sum_partials_kernel<<<1, 256, 0, s>>>(partials, parts, 1.0, nullptr, nullptr, nullptr, 0,
                                          f_dev);
    NMF_LAUNCHED("sum_partials_kernel");
    return NMF_OK;
}

nmf_status launch_objective_dense(const float *A, int64_t m, int64_t n, int64_t lda,
                                  const float *W, const float *Ht, int k, int precision,
                                  double *partials, double *f_dev, cudaStream_t s)
{
    (void)precision;
    const int parts = obj_parts();
    objective_dense_kernel<<<parts, OBJ_THREADS, 0, s>>>(A, m, n, lda, W, Ht, k, partials);
    NMF_LAUNCHED("objective_dense_kernel");
    sum_partials_kernel<<<1, 256, 0, s>>>(partials, parts, 1.0, nullptr, nullptr, nullptr, k,
                                          f_dev);
    NMF_LAUNCHED("sum_partials_kernel");
    return NMF_OK;
}

static nmf_status launch_dot(const float *X, const float *Y, int64_t len, double scale,
                             const double *base, const double *GW, const double *GH,
                             int k, double *partials, double *f_dev, cudaStream_t s)
{
    const int parts = obj_parts();
    const int vec = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) == 0;
    dot_partials_kernel<<<parts, OBJ_THREADS, 0, s>>>(X, Y, len, vec, partials);
    NMF_LAUNCHED("dot_partials_kernel");
    sum_partials_kernel<<<1, 256, 0, s>>>(partials, parts, scale, base, GW, GH, k, f_dev);
    NMF_LAUNCHED("sum_partials_kernel");
    return NMF_OK;
}

nmf_status launch_objective_csr(const float *Ht, const float *Y, int64_t n, int k,
                                const double *a_sq, const double *GW, const double *GH,
                                double *partials, double *f_dev, cudaStream_t s)
{
    return launch_dot(Ht, Y, n * k, -2.0, a_sq, GW, GH, k, partials, f_dev, s);
}

nmf_status launch_sq_norm(const float *v, int64_t len, double *partials, double *out,
                          cudaStream_t s)
{
    return launch_dot(v, v, len, 1.0, nullptr, nullptr, nullptr, 0, partials, out, s);
}

}  // namespace nmf
