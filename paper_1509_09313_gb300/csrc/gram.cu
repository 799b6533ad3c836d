// Gram matrices H H^T and W^T W of Alg. 1 (the "Gram" task of Sec. 6.2).
//
// G = X^T X for X (rows x k, float32 row-major). Each CTA walks 32-row tiles
// of X staged in shared memory; a thread owns a 4 x 4 block of the upper
// triangle of G (k padded to 4; G is symmetric, so the blocks below the
// diagonal are not formed: 1275 FMAs per row at k = 50 instead of the 4096 of
// the full padded square), or every RS-th row of a tile of one when the
// blocks are fewer than the threads; it sums the products of a tile in FP32
// (fmaf) and adds the tile's sum into a Kahan-compensated FP32 accumulator (error ~2 ulp of the block sum whatever
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

// Work items of a CTA: the upper-triangle 4 x 4 blocks (ta <= tb) of the
// k-padded-to-4 Gram, NB = TB (TB + 1) / 2 of them; when they are fewer than
// the threads, RS threads share a block, each taking every RS-th row of a
// tile (RS = floor(threads / NB)). An item is (block, row offset).
struct GramItems {
    int TB, NB, RS, items;
};

__host__ __device__ inline GramItems gram_items(int k, int threads)
{
    GramItems g;
    g.TB = (k + 3) / 4;
    g.NB = g.TB * (g.TB + 1) / 2;
    // Row sharing only with 256 threads (its partials are combined in shared
    // memory, 256 x 16 doubles).
    g.RS = g.NB >= threads || threads > 256 ? 1 : threads / g.NB;
    g.items = g.NB * g.RS;
    return g;
}

// Block index -> (ta, tb), ta <= tb, blocks numbered row by row of the upper
// triangle.
__device__ __forceinline__ void gram_block(int blk, int TB, int &ta, int &tb)
{
    int a = 0, rem = blk;
    while (rem >= TB - a) {
        rem -= TB - a;
        ++a;
    }
    ta = a;
    tb = a + rem;
}

template <int KP>
__global__ void __launch_bounds__(gram_threads<KP>()) gram_partial_kernel(
    const float *__restrict__ X, int64_t rows, int k, double *__restrict__ partials)
{
    constexpr int NT = gram_threads<KP>();
    constexpr int TBMAX = KP / 4;
    constexpr int PER = (TBMAX * (TBMAX + 1) / 2 + NT - 1) / NT;   // items per thread, at most
    __shared__ __align__(16) float xs[GRAM_TILE][KP];
    const GramItems gi = gram_items(k, NT);

    float sum[PER][4][4], cmp[PER][4][4];   // Kahan: block sum and its lost low part
    int ta[PER], tb[PER], ro[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int it = threadIdx.x + q * NT;
        const int blk = it % gi.NB;
        ro[q] = it < gi.items ? it / gi.NB : GRAM_TILE;   // GRAM_TILE: no work
        gram_block(blk, gi.TB, ta[q], tb[q]);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                sum[q][a][b] = 0.0f;
                cmp[q][a][b] = 0.0f;
            }
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
            if (ro[q] >= GRAM_TILE)
                continue;
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    acc[a][b] = 0.0f;
#pragma unroll 4
            for (int r = ro[q]; r < GRAM_TILE; r += gi.RS) {
                const float4 va = *reinterpret_cast<const float4 *>(&xs[r][4 * ta[q]]);
                const float4 vb = *reinterpret_cast<const float4 *>(&xs[r][4 * tb[q]]);
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
                    const float tt = sum[q][a][b] + y;
                    cmp[q][a][b] = (tt - sum[q][a][b]) - y;
                    sum[q][a][b] = tt;
                }
        }
        __syncthreads();
    }
    // This CTA's partial of every block, [block][16] in FP64 (the row
    // offsets' items of a block added in a fixed order).
    double *out = partials + (int64_t)blockIdx.x * gi.NB * 16;
    if constexpr (NT <= 256) {
        __shared__ double red[256 * 16];
        if (gi.RS > 1) {
            const int it = threadIdx.x;
            if (it < gi.items) {
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        red[it * 16 + 4 * a + b] = (double)sum[0][a][b] - (double)cmp[0][a][b];
            }
            __syncthreads();
            for (int slot = threadIdx.x; slot < gi.NB * 16; slot += NT) {
                double v = 0.0;
                for (int r = 0; r < gi.RS; ++r)
                    v += red[r * gi.NB * 16 + slot];
                out[slot] = v;
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int it = threadIdx.x + q * NT;
        if (it < gi.items) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    out[it * 16 + 4 * a + b] = (double)sum[q][a][b] - (double)cmp[q][a][b];
        }
    }
}

// Slot s = 16 blk + 4 a + b of the CTA partials ([part][block][16]) summed
// over the parts: 32 slots per CTA, the parts split over its 8 warps (each
// load of a warp is 32 consecutive slots), then added across the warps in a
// fixed order; the sum goes to G[i][j] and G[j][i] (i = 4 ta + a, j = 4 tb +
// b, the block's (ta, tb)).
__global__ void __launch_bounds__(256)
    gram_reduce_kernel(const double *__restrict__ partials, int nparts, int k, int threads,
                       double *__restrict__ G)
{
    __shared__ double acc[8][32];
    const GramItems gi = gram_items(k, threads);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int slot = blockIdx.x * 32 + lane;
    const bool live = slot < gi.NB * 16;
    double v = 0.0;
    if (live)
        for (int p = w; p < nparts; p += 8)
            v += partials[(int64_t)p * gi.NB * 16 + slot];
    acc[w][lane] = v;
    __syncthreads();
    if (w == 0 && live) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q)
            s += acc[q][lane];
        const int blk = slot >> 4, within = slot & 15;
        int ta = 0, rem = blk;
        while (rem >= gi.TB - ta) {
            rem -= gi.TB - ta;
            ++ta;
        }
        const int tb = ta + rem;
        const int i = 4 * ta + (within >> 2), j = 4 * tb + (within & 3);
        if (i < k && j < k) {
            G[i * k + j] = s;
            G[j * k + i] = s;
        }
    }
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

int gram_threads_for(int k)
{
    return k <= 64 ? GRAM_THREADS : 2 * GRAM_THREADS;
}

int64_t gram_partials_len(int64_t rows, int k)
{
    return (int64_t)gram_parts(rows) * gram_items(k, gram_threads_for(k)).NB * 16;
}

nmf_status launch_gram(const float *X, int64_t rows, int k, double *G, double *partials,
                       cudaStream_t s)
{
    const int slots = gram_items(k, gram_threads_for(k)).NB * 16;
    if (gram_tc_usable(X, rows, k)) {
        NMF_TRY(launch_gram_tc(X, rows, k, partials, s));
        gram_reduce_kernel<<<(int)cdiv(slots, 32), 256, 0, s>>>(partials, gram_tc_parts(rows), k,
                                                                gram_threads_for(k), G);
        NMF_LAUNCHED("gram_reduce_kernel");
        return NMF_OK;
    }
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
    gram_reduce_kernel<<<(int)cdiv(slots, 32), 256, 0, s>>>(partials, parts, k,
                                                            gram_threads_for(k), G);
    NMF_LAUNCHED("gram_reduce_kernel");
    return NMF_OK;
}

}  // namespace nmf
