// Gram matrices H H^T and W^T W of Alg. 1 (the "Gram" task of Sec. 6.2).
//
// G = X^T X for X (rows x k, float32 row-major). Each CTA walks 32-row tiles
// of X staged in shared memory; a thread owns a 4 x 4 block of G, sums the 32
// products of a tile in FP32 (fmaf) and adds the tile's sum into FP64
// registers. Every CTA writes its FP64 block partials; a second kernel adds
// the partials in CTA order, so the result does not depend on scheduling.
//
// Roofline: HBM. Algorithmic bytes = rows * k * 4 (X read once) + k*k*8.
#include "common.cuh"

namespace nmf {
namespace {

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_TILE = 32;

template <int KP>
__global__ void __launch_bounds__(GRAM_THREADS) gram_partial_kernel(const float *__restrict__ X,
                                                                    int64_t rows, int k,
                                                                    double *__restrict__ partials)
{
    constexpr int TB = KP / 4;                 // 4x4 blocks per side
    constexpr int NBLK = TB * TB;              // blocks of G
    constexpr int PER = (NBLK + GRAM_THREADS - 1) / GRAM_THREADS;
    __shared__ __align__(16) float xs[GRAM_TILE][KP];

    double acc64[PER][4][4];
#pragma unroll
    for (int q = 0; q < PER; ++q)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                acc64[q][a][b] = 0.0;

    const int64_t ntiles = cdiv(rows, GRAM_TILE);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = t * GRAM_TILE;
        for (int e = threadIdx.x; e < GRAM_TILE * KP; e += GRAM_THREADS) {
            const int r = e / KP, c = e % KP;
            const int64_t row = r0 + r;
            xs[r][c] = (row < rows && c < k) ? X[row * k + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int blk = threadIdx.x + q * GRAM_THREADS;
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
                    for (int b = 0; b < 4; ++b)
                        acc64[q][a][b] += (double)acc[a][b];
            }
        }
        __syncthreads();
    }
    double *out = partials + (int64_t)blockIdx.x * k * k;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int blk = threadIdx.x + q * GRAM_THREADS;
        if (blk < NBLK) {
            const int ta = blk / TB, tb = blk % TB;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int ga = 4 * ta + a, gb = 4 * tb + b;
                    if (ga < k && gb < k)
                        out[ga * k + gb] = acc64[q][a][b];
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
    int64_t p = 2 * (int64_t)sm_count();
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
        gram_partial_kernel<128><<<parts, GRAM_THREADS, 0, s>>>(X, rows, k, partials);
    NMF_LAUNCHED("gram_partial_kernel");
    const int kk = k * k;
    gram_reduce_kernel<<<(int)cdiv(kk, 256), 256, 0, s>>>(partials, parts, kk, G);
    NMF_LAUNCHED("gram_reduce_kernel");
    return NMF_OK;
}

}  // namespace nmf
