// Gram matrices H H^T and W^T W of Alg. 1 (the "Gram" task of Sec. 6.2).
//
// G = X^T X for X (rows x k, float32 row-major). Each CTA walks 32-row tiles
// of X staged in shared memory; a thread owns a 4 x 4 block of G, sums the 32
// products of a tile in FP32 (fmaf) and adds the tile's sum into a
// Kahan-compensated FP32 accumulator (error ~2 ulp of the block sum whatever
// the number of tiles; GB300's FP64 pipe, two operations per clock per SM,
// made per-tile FP64 adds the kernel's bottleneck). Every CTA writes its
// block partials in FP64; a second kernel adds the partials in CTA order, so
// the result does not depend on scheduling.
//
// Roofline: HBM. Algorithmic bytes = rows * k * 4 (X read once) + k*k*8.
#include "common.cuh"

namespace nmf {
namespace {

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_TILE = 32;

// Threads per CTA: 256, or 512 for k > 64 (two 4 x 4 blocks per thread
// instead of four keeps the Kahan pairs in registers).
template <int KP> __host__ __device__ constexpr int gram_threads() { return KP > 64 ? 2 * GRAM_THREADS : GRAM_THREADS; }

template <int KP>
__global__ void __launch_bounds__(gram_threads<KP>()) gram_partial_kernel(
    const float *__restrict__ X, int64_t rows, int k, double *__restrict__ partials)
{
    constexpr int NT = gram_threads<KP>();
    constexpr int TB = KP / 4;                 // 4x4 blocks per side
    constexpr int NBLK = TB * TB;              // blocks of G
    constexpr int PER = (NBLK + NT - 1) / NT;
    __shared__ __align__(16) float xs[GRAM_TILE][KP];

    float sum[PER][4][4], cmp[PER][4][4];   // Kahan: block sum and its lost low part
#pragma unroll
    for (int q = 0; q < PER; ++q)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                sum[q][a][b] = 0.0f;
                cmp[q][a][b] = 0.0f;
            }

    // The next tile's elements are loaded into registers while the current
    // one is multiplied (NL per thread).
    constexpr int NL = (GRAM_TILE * KP + NT - 1) / NT;
    float pre[NL];
    auto load_tile = [&](int64_t t) {
        const int64_t r0 = t * GRAM_TILE;
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int e = threadIdx.x + i * NT;
            const int r = e / KP, c = e % KP;
            const int64_t row = r0 + r;
            pre[i] = (e < GRAM_TILE * KP && row < rows && c < k) ? X[row * k + c] : 0.0f;
        }
    };
    const int64_t ntiles = cdiv(rows, GRAM_TILE);
    if ((int64_t)blockIdx.x < ntiles)
        load_tile(blockIdx.x);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int e = threadIdx.x + i * NT;
            if (e < GRAM_TILE * KP)
                xs[e / KP][e % KP] = pre[i];
        }
        __syncthreads();
        if (t + gridDim.x < ntiles)
            load_tile(t + gridDim.x);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int blk = threadIdx.x + q * NT;
            if (blk < NBLK) {
                const int ta = blk / TB, tb = blk % TB;
                float acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        acc[a][b] = 0.0f;
#pragma unroll 8
                for (int r = 0; r < GRAM_TILE; ++r) {
                    const float4 va = *reinterpret_cast<const float4 *>(&xs[r][4 * ta]);
                    const float4 vb = *reinterpret_cast<const float4 *>(&xs[r][4 * tb]);
                    const float av[4] = {va.x, va.y, va.z, va.w};
                    const float bv[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float y = acc[a][b] - cmp[q][a][b];
                        const float t = sum[q][a][b] + y;
                        cmp[q][a][b] = (t - sum[q][a][b]) - y;
                        sum[q][a][b] = t;
                    }
            }
        }
        __syncthreads();
    }
    double *out = partials + (int64_t)blockIdx.x * k * k;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int blk = threadIdx.x + q * NT;
        if (blk < NBLK) {
            const int ta = blk / TB, tb = blk % TB;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int ga = 4 * ta + a, gb = 4 * tb + b;
                    if (ga < k && gb < k)
                        out[ga * k + gb] = (double)sum[q][a][b] - (double)cmp[q][a][b];
                }
        }
    }
}

__global__ void gram_reduce_kernel(const double *__restrict__ partials, int nparts, int kk,
                                   double *__restrict__ G)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kk)
        return;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p)
        s += partials[(int64_t)p * kk + e];
    G[e] = s;
}

int gram_parts(int64_t rows)
{
    const int64_t tiles = cdiv(rows, GRAM_TILE);
    int64_t p = 3 * (int64_t)sm_count();
    if (tiles < p)
        p = tiles;
    return p < 1 ? 1 : (int)p;
}

}  // namespace

int64_t gram_partials_len(int64_t rows, int k) { return (int64_t)gram_parts(rows) * k * k; }

nmf_status launch_gram(const float *X, int64_t rows, int k, double *G, double *partials,
                       cudaStream_t s)
{
    const int parts = gram_parts(rows);
    if (k <= 16)
        gram_partial_kernel<16><<<parts, GRAM_THREADS, 0, s>>>(X, rows, k, partials);
    else if (k <= 32)
        gram_partial_kernel<32><<<parts, GRAM_THREADS, 0, s>>>(X, rows, k, partials);
    else if (k <= 64)
        gram_partial_kernel<64><<<parts, GRAM_THREADS, 0, s>>>(X, rows, k, partials);
    else
        gram_partial_kernel<128><<<parts, gram_threads<128>(), 0, s>>>(X, rows, k, partials);
    NMF_LAUNCHED("gram_partial_kernel");
    const int kk = k * k;
    gram_reduce_kernel<<<(int)cdiv(kk, 256), 256, 0, s>>>(partials, parts, kk, G);
    NMF_LAUNCHED("gram_reduce_kernel");
    return NMF_OK;
}

}  // namespace nmf
