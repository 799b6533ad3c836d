// Sparse products of Alg. 1 with CSR A (the sparse "MM" task of Sec. 4.3):
// out (rows x k) = S F, one warp per CSR row. The warp reads its row's
// (column, value) pairs 32 at a time with one coalesced load each, then
// broadcasts them by shuffle; lane l accumulates columns l, l+32, ... of the
// output, gathering the matching rows of F (k contiguous floats each). Sums
// run in the row's stored order, so results are deterministic.
//
// W^T A needs the CSR of A^T: csr_transpose builds it on the device (count
// per column, prefix sum, scatter, then each output row sorted by index so
// the layout does not depend on scheduling).
//
// Roofline: HBM. Compulsory bytes per product: rowptr + colidx + vals +
// F + out; the gathers of F rows add up to nnz * k * 4 bytes when F is not
// L2-resident.
#include "common.cuh"

namespace nmf {
namespace {

constexpr int SPMM_THREADS = 256;

template <int KW>
__global__ void __launch_bounds__(SPMM_THREADS)
    spmm_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                const float *__restrict__ vals, int64_t rows, const float *__restrict__ F, int k,
                float *__restrict__ out, const int *__restrict__ mode_flag)
{
    if (mode_flag && *mode_flag == 0)
        return;   // FP32 half-step: its solves form the product rows themselves
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * SPMM_THREADS + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * SPMM_THREADS) >> 5;
    for (int64_t i = warp0; i < rows; i += nw) {
        float acc[KW];
#pragma unroll
        for (int s = 0; s < KW; ++s)
            acc[s] = 0.0f;
        const int64_t beg = rowptr[i], end = rowptr[i + 1];
        for (int64_t p0 = beg; p0 < end; p0 += 32) {
            const int64_t p = p0 + lane;
            const int c = p < end ? colidx[p] : 0;
            const float v = p < end ? vals[p] : 0.0f;
            const int cnt = (int)min((int64_t)32, end - p0);
            for (int l = 0; l < cnt; ++l) {
                const int64_t cl = __shfl_sync(FULL, c, l);
                const float vl = __shfl_sync(FULL, v, l);
                const float *frow = F + cl * k;
#pragma unroll
                for (int s = 0; s < KW; ++s) {
                    const int r = lane + 32 * s;
                    if (r < k)
                        acc[s] = fmaf(vl, frow[r], acc[s]);
                }
            }
        }
#pragma unroll
        for (int s = 0; s < KW; ++s) {
            const int r = lane + 32 * s;
            if (r < k)
                out[i * k + r] = acc[s];
        }
    }
}

__global__ void count_cols_kernel(const int32_t *__restrict__ colidx, int64_t nnz,
                                  unsigned long long *__restrict__ counts)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&counts[colidx[p] + 1], 1ull);
}

// In-place inclusive scan of counts[0..len) by one CTA of 1024 threads,
// walking 1024-element chunks with a running carry (init-time only).
__global__ void __launch_bounds__(1024) scan_kernel(unsigned long long *__restrict__ a, int64_t len)
{
    __shared__ unsigned long long buf[1024];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < len; base += 1024) {
        const int64_t i = base + threadIdx.x;
        buf[threadIdx.x] = i < len ? a[i] : 0ull;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const unsigned long long v = threadIdx.x >= o ? buf[threadIdx.x - o] : 0ull;
            __syncthreads();
            buf[threadIdx.x] += v;
            __syncthreads();
        }
        if (i < len)
            a[i] = buf[threadIdx.x] + carry;
        __syncthreads();
        if (threadIdx.x == 1023)
            carry += buf[1023];
        __syncthreads();
    }
}

__global__ void scatter_kernel(const int64_t *__restrict__ rowptr,
                               const int32_t *__restrict__ colidx, const float *__restrict__ vals,
                               int64_t m, unsigned long long *__restrict__ cursor,
                               int32_t *__restrict__ t_colidx, float *__restrict__ t_vals)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const unsigned long long pos = atomicAdd(&cursor[colidx[p]], 1ull);
            t_colidx[pos] = (int32_t)i;
            t_vals[pos] = vals[p];
        }
}

__global__ void sort_rows_kernel(const int64_t *__restrict__ t_rowptr, int64_t n,
                                 int32_t *__restrict__ t_colidx, float *__restrict__ t_vals)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t_rowptr[j], e = t_rowptr[j + 1];
        for (int64_t p = b + 1; p < e; ++p) {
            const int32_t c = t_colidx[p];
            const float v = t_vals[p];
            int64_t q = p - 1;
            while (q >= b && t_colidx[q] > c) {
                t_colidx[q + 1] = t_colidx[q];
                t_vals[q + 1] = t_vals[q];
                --q;
            }
            t_colidx[q + 1] = c;
            t_vals[q + 1] = v;
        }
    }
}

}  // namespace

namespace {
nmf_status spmm_launch(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                       int64_t rows, const float *F, int k, float *out, const int *mode_flag,
                       cudaStream_t s)
{
    if (rows == 0)
        return NMF_OK;
    int64_t blocks = cdiv(rows * 32, SPMM_THREADS);
    const int64_t cap = 16LL * sm_count();
    if (blocks > cap)
        blocks = cap;
    const unsigned g = (unsigned)blocks;
    if (k <= 32)
        spmm_kernel<1><<<g, SPMM_THREADS, 0, s>>>(rowptr, colidx, vals, rows, F, k, out, mode_flag);
    else if (k <= 64)
        spmm_kernel<2><<<g, SPMM_THREADS, 0, s>>>(rowptr, colidx, vals, rows, F, k, out, mode_flag);
    else if (k <= 96)
        spmm_kernel<3><<<g, SPMM_THREADS, 0, s>>>(rowptr, colidx, vals, rows, F, k, out, mode_flag);
    else
        spmm_kernel<4><<<g, SPMM_THREADS, 0, s>>>(rowptr, colidx, vals, rows, F, k, out, mode_flag);
    NMF_LAUNCHED("spmm_kernel");
    return NMF_OK;
}
}  // namespace

nmf_status launch_spmm(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                       int64_t rows, const float *F, int k, float *out, cudaStream_t s)
{
    return spmm_launch(rowptr, colidx, vals, rows, F, k, out, nullptr, s);
}

nmf_status launch_spmm_unless_fp32(const int64_t *rowptr, const int32_t *colidx,
                                   const float *vals, int64_t rows, const float *F, int k,
                                   float *out, const int *mode_flag, cudaStream_t s)
{
    return spmm_launch(rowptr, colidx, vals, rows, F, k, out, mode_flag, s);
}

nmf_status launch_csr_transpose(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                                int64_t m, int64_t n, int64_t nnz, int64_t *t_rowptr,
                                int32_t *t_colidx, float *t_vals,
                                unsigned long long *cursor, cudaStream_t s)
{
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(t_rowptr);
    NMF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (size_t)(n + 1), s));
    const unsigned g = (unsigned)(4 * sm_count());
    if (nnz > 0) {
        count_cols_kernel<<<g, 256, 0, s>>>(colidx, nnz, cnt);
        NMF_LAUNCHED("count_cols_kernel");
    }
    scan_kernel<<<1, 1024, 0, s>>>(cnt, n + 1);
    NMF_LAUNCHED("scan_kernel");
    if (n > 0)
        NMF_CUDA(cudaMemcpyAsync(cursor, cnt, sizeof(int64_t) * (size_t)n,
                                 cudaMemcpyDeviceToDevice, s));
    if (m > 0 && nnz > 0) {
        scatter_kernel<<<g, 256, 0, s>>>(rowptr, colidx, vals, m, cursor, t_colidx, t_vals);
        NMF_LAUNCHED("scatter_kernel");
        sort_rows_kernel<<<g, 256, 0, s>>>(t_rowptr, n, t_colidx, t_vals);
        NMF_LAUNCHED("sort_rows_kernel");
    }
    return NMF_OK;
}

}  // namespace nmf
