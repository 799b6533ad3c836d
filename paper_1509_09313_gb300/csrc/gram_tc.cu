// Gram G = X^T X (Alg. 1: H H^T and W^T W, the "Gram" task of Sec. 6.2) on
// the tensor cores, for k <= 64 and X (rows x k, FP32 row-major, 16-byte
// aligned).
//
// Each CTA takes 128-row tiles of X in turn (tile blockIdx.x + t gridDim.x):
//  * a producer thread copies the tile's 128 k floats (contiguous in X) into
//    an FP32 ring with one bulk copy (as many stages as shared memory holds:
//    the bytes in flight per SM set the rate);
//  * sixteen worker warps, in two groups that take alternate tiles, split
//    each value into three BF16 parts,
//    x = h + m + l (h = bf16(x), m = bf16(x - h), l = bf16(x - h - m); the
//    representation error is below 2^-26 |x|), written as K-major operand
//    tiles with the 128-byte swizzle: per 64-row K-block, A = [h; m] (h for
//    features 0..63 in operand rows 0..63, m in rows 64..127; zero past k)
//    and l (rows 0..63);
//  * one thread issues, per 16-row step, D_H = A h (N = 64) and
//    D_R += A [m l] (N = 128: the l rows follow the m rows in shared memory;
//    M = 128, BF16 operands, FP32 accumulators in TMEM).
// The top half of D_H is h^T h, the leading term: it accumulates a pair of
// tiles (256 rows), then is drained into Kahan-compensated FP32 sums kept in
// TMEM (per group; 32 columns of the 64 top rows per drain warp). D_R, whose
// terms are 2^-8 of G or less, accumulates over all the CTA's tiles:
// [h^T m, h^T l] on top, [m^T m, m^T l] below. With lm, ml and ll (below
// 2^-26 of G) dropped, G = h^T h + m^T m + X + X^T, X = h^T m + h^T l,
// formed per CTA in FP64 and written as upper-triangle 4 x 4 block partials
// that the SIMT Gram's reduce kernel adds in CTA order.
//
// Roofline: HBM, rows * k * 4 bytes read once.
#include <math.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nmf {
namespace {

using namespace tc;

constexpr int GT_ROWS = 128;                       // rows of X per tile
constexpr int GT_STG_MAX = 8;                      // FP32 staging stages, at most
constexpr int GT_KB_BYTES = 24 * 1024;             // one 64-row K-block: A 16 KB + l 8 KB
constexpr int GT_SPL_BYTES = 2 * GT_KB_BYTES;      // one split tile (two K-blocks)
constexpr int GT_WORKERS = 16;                     // split / drain warps
constexpr int GT_THREADS = 32 * (GT_WORKERS + 2);  // + producer + MMA warps
// Shared memory: 2 split buffers, barriers, TMEM slot and abort flag, then
// the staging ring (as many 128 k-float stages as fit, up to GT_STG_MAX: the
// bytes in flight per SM set the rate at which tiles arrive).
constexpr int GT_OFF_SPL = 0;
constexpr int GT_OFF_BAR = 2 * GT_SPL_BYTES;
constexpr int GT_NBAR = 2 * GT_STG_MAX + 2 * 2 + 2 * 2 + 1;
constexpr int GT_OFF_TMEM = GT_OFF_BAR + 8 * GT_NBAR;
constexpr int GT_OFF_ABORT = GT_OFF_TMEM + 8;
constexpr int GT_OFF_STG = (GT_OFF_ABORT + 8 + 127) & ~127;
constexpr int GT_SMEM_MAX = 227 * 1024;
__host__ __device__ inline int gt_stage_bytes(int k) { return GT_ROWS * k * 4; }
inline int gt_stages(int k)
{
    const int n = (GT_SMEM_MAX - 1024 - GT_OFF_STG) / gt_stage_bytes(k);
    return n < GT_STG_MAX ? n : GT_STG_MAX;
}
inline int gt_smem(int k) { return GT_OFF_STG + gt_stages(k) * gt_stage_bytes(k) + 1024; }
constexpr int GT_RS = 129;                         // row stride of the final D_R copy (floats)
static_assert(128 * GT_RS * 4 <= 2 * GT_SPL_BYTES, "D_R copy fits the split buffers");

__device__ __forceinline__ void split3(float v0, float v1, uint32_t &h, uint32_t &m, uint32_t &l)
{
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v0, v1);
    const float2 hf = __bfloat1622float2(hb);
    const float2 d = __ffma2_rn(hf, make_float2(-1.0f, -1.0f), make_float2(v0, v1));   // exact
    const __nv_bfloat162 mb = __floats2bfloat162_rn(d.x, d.y);
    const float2 mf = __bfloat1622float2(mb);
    const float2 e = __ffma2_rn(mf, make_float2(-1.0f, -1.0f), d);                      // exact
    const __nv_bfloat162 lb = __floats2bfloat162_rn(e.x, e.y);
    h = *reinterpret_cast<const uint32_t *>(&hb);
    m = *reinterpret_cast<const uint32_t *>(&mb);
    l = *reinterpret_cast<const uint32_t *>(&lb);
}

__global__ void __launch_bounds__(GT_THREADS, 1)
    gram_tc_kernel(const float *__restrict__ X, int64_t rows, int k, int nstg,
                   double *__restrict__ partials)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = reinterpret_cast<volatile int *>(smem + GT_OFF_ABORT);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + GT_OFF_TMEM);

    const uint32_t bar0 = sbase + GT_OFF_BAR;
    auto stg_full = [&](int i) { return bar0 + 8u * i; };
    auto stg_empty = [&](int i) { return bar0 + 8u * (GT_STG_MAX + i); };
    auto spl_full = [&](int i) { return bar0 + 8u * (2 * GT_STG_MAX + i); };
    auto spl_empty = [&](int i) { return bar0 + 8u * (2 * GT_STG_MAX + 2 + i); };
    auto acc_full = [&](int i) { return bar0 + 8u * (2 * GT_STG_MAX + 4 + i); };
    auto acc_empty = [&](int i) { return bar0 + 8u * (2 * GT_STG_MAX + 6 + i); };
    const uint32_t r_full = bar0 + 8u * (2 * GT_STG_MAX + 8);
    const uint32_t stg_bytes = (uint32_t)gt_stage_bytes(k);

    if (threadIdx.x == 0) {
        for (int i = 0; i < nstg; ++i) {
            mbar_init(stg_full(i), 1);
            mbar_init(stg_empty(i), GT_WORKERS / 2);   // the tile's group
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(spl_full(i), GT_WORKERS / 2);
            mbar_init(spl_empty(i), 1);
            mbar_init(acc_full(i), 1);
            mbar_init(acc_empty(i), 4);   // the group's drain warps
        }
        mbar_init(r_full, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == GT_WORKERS + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t ntiles = (rows + GT_ROWS - 1) / GT_ROWS;
    const int nt = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);   // >= 1
    auto tile_row0 = [&](int t) {
        return ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * GT_ROWS;
    };
    // D_H of group g (tiles t = g mod 2) holds a pair of the group's tiles
    // (256 rows) between drains: tile t is the (t / 2)-th of its group, in
    // pair t / 4; a pair ends at its second tile or at the group's last.
    auto pair_end = [&](int t) { return ((t >> 1) & 1) == 1 || t + 2 >= nt; };
    const uint32_t tile_bytes = (uint32_t)(GT_ROWS * k * 4);

    if (warp == GT_WORKERS) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            for (int t = 0; t < nt; ++t) {
                const int s = t % nstg, u = t / nstg;
                if (!mbar_wait(stg_empty(s), (u & 1) ^ 1, abort))
                    break;
                const int64_t r0 = tile_row0(t);
                if (rows - r0 >= GT_ROWS) {
                    mbar_arrive_expect_tx(stg_full(s), tile_bytes);
                    bulk_load(sbase + GT_OFF_STG + (uint32_t)s * stg_bytes, X + r0 * k, tile_bytes,
                              stg_full(s));
                } else {
                    mbar_arrive(stg_full(s));   // the ragged last tile: read from X directly
                }
            }
        }
    } else if (warp == GT_WORKERS + 1) {
        // ---------------------------------------------------------------- MMAs
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32<64>();
            const uint32_t idesc2 = idesc_bf16_f32<128>();
            const uint64_t spl0 = sw128_desc(sbase + GT_OFF_SPL);
            constexpr uint64_t SPL16 = (uint64_t)(GT_SPL_BYTES >> 4);
            constexpr uint64_t KB16 = (uint64_t)(GT_KB_BYTES >> 4);
            constexpr uint64_t M16 = (uint64_t)(8192 >> 4);    // m rows of A, then l: [m l]
            const uint32_t dR = tmem + 128u;
            bool ok = true;
            for (int t = 0; t < nt && ok; ++t) {
                const int b = t & 1, ub = t >> 1;
                const bool pair_start = (ub & 1) == 0;
                if (!mbar_wait_fast(spl_full(b), ub & 1, abort) ||
                    (pair_start && !mbar_wait_fast(acc_empty(b), ((ub >> 1) & 1) ^ 1, abort))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dH = tmem + (uint32_t)(b * 64);
#pragma unroll
                for (int kb = 0; kb < 2; ++kb) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t a = spl0 + (uint64_t)b * SPL16 + (uint64_t)kb * KB16 +
                                           (uint64_t)(kk * 2);
                        const bool step0 = kb == 0 && kk == 0;   // D_H starts each pair
                        mma_bf16(dH, a, a, idesc, (pair_start && step0) ? 0u : 1u);
                        mma_bf16(dR, a, a + M16, idesc2, (t == 0 && step0) ? 0u : 1u);
                    }
                }
                mma_commit(spl_empty(b));
                if (pair_end(t))
                    mma_commit(acc_full(b));
            }
            if (ok)
                mma_commit(r_full);
        }
    } else {
        // ------------------------------------------------ split and drain warps
        // Two groups of eight warps take alternate tiles (group g the tiles
        // t = g mod 2, split buffer g, D_H buffer g), so that one group's
        // waits overlap the other's work. TMEM columns: D_H 0..127, D_R
        // 128..255, and for the h^T h rows (lanes 0..63) group g's Kahan
        // sums at 256 + 128 g and compensations at 320 + 128 g. A drain warp
        // (lanes 32 quarter .. + 31, quarter 0 or 1) owns 32 columns of each.
        const int g = warp >> 3, gtid = threadIdx.x & 255;
        const int fi = gtid & 63;   // the feature this thread splits
        const int quarter = warp & 3, half = (warp >> 2) & 1;
        const bool drainer = quarter < 2;
        const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
        const uint32_t tks = tmem + lanes + 256u + 128u * g + 32u * half;   // sums; +64: comps
        if (drainer) {
            const float z[16] = {};
            tmem_st16(tks, z);
            tmem_st16(tks + 16u, z);
            tmem_st16(tks + 64u, z);
            tmem_st16(tks + 80u, z);
            tmem_wait_st();
        }
        auto drain = [&](int t) -> bool {   // the pair that tile t ends
            const int b = t & 1, pr = t >> 2;
            if (!mbar_wait(acc_full(b), pr & 1, abort))
                return false;
            tc_fence_after();
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {   // 16 columns at a time
                uint32_t d[16], ks[16], kc[16];
                tmem_ld16_nowait(tmem + lanes + (uint32_t)(64 * b + 32 * half + 16 * hh), d);
                tmem_ld16_nowait(tks + 16u * hh, ks);
                tmem_ld16_nowait(tks + 64u + 16u * hh, kc);
                tmem_wait_ld();
                float so[16], co[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float sum = __uint_as_float(ks[c]), cmp = __uint_as_float(kc[c]);
                    const float y = __uint_as_float(d[c]) - cmp;
                    const float sn = sum + y;
                    co[c] = (sn - sum) - y;
                    so[c] = sn;
                }
                tmem_st16(tks + 16u * hh, so);
                tmem_st16(tks + 64u + 16u * hh, co);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(acc_empty(b));
            return true;
        };
        bool ok = true;
        int last = -1;
        for (int t = g; t < nt && ok; t += 2) {
            const int s = t % nstg, u = t / nstg;
            const int b = g, ub = t >> 1;
            if (!mbar_wait(stg_full(s), u & 1, abort) ||
                !mbar_wait(spl_empty(b), (ub & 1) ^ 1, abort)) {
                ok = false;
                break;
            }
            const int64_t r0 = tile_row0(t);
            const int nr = (int)min((int64_t)GT_ROWS, rows - r0);
            const float *stg = reinterpret_cast<const float *>(smem + GT_OFF_STG + s * stg_bytes);
            unsigned char *spl = smem + GT_OFF_SPL + b * GT_SPL_BYTES;
            // Item q of this thread: feature fi (the same for all four items),
            // 8-row chunk c = gtid / 64 + 4 q. Features past k are zero; the
            // group's split buffer holds their zeros after its first tile.
            if (fi < k || t < 2) {
                float v[4][8];
                if (fi >= k) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int w = 0; w < 8; ++w)
                            v[q][w] = 0.0f;
                } else if (nr == GT_ROWS) {
                    const float *src = stg + (8 * (gtid >> 6)) * k + fi;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int w = 0; w < 8; ++w)
                            v[q][w] = src[(32 * q + w) * k];
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            const int r = 8 * ((gtid >> 6) + 4 * q) + w;
                            v[q][w] = r < nr ? X[(r0 + r) * k + fi] : 0.0f;
                        }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = (gtid >> 6) + 4 * q;
                    uint32_t h[4], m[4], l[4];
#pragma unroll
                    for (int w = 0; w < 4; ++w)
                        split3(v[q][2 * w], v[q][2 * w + 1], h[w], m[w], l[w]);
                    unsigned char *blk = spl + (c >> 3) * GT_KB_BYTES;
                    const uint32_t sw = (uint32_t)(((c & 7) ^ (fi & 7)) << 4);
                    *reinterpret_cast<uint4 *>(blk + fi * 128 + sw) =
                        make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(blk + (64 + fi) * 128 + sw) =
                        make_uint4(m[0], m[1], m[2], m[3]);
                    *reinterpret_cast<uint4 *>(blk + 16384 + fi * 128 + sw) =
                        make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(spl_full(b));
                mbar_arrive(stg_empty(s));
            }
            if (drainer && t >= 2 && pair_end(t - 2) && !drain(t - 2)) {
                ok = false;
                break;
            }
            last = t;
        }
        if (ok && drainer && last >= 0)
            ok = drain(last);
        // D_R once all MMAs are done: a copy in shared memory (the split
        // buffers are free), rows 0..127 by 129 floats; warp w copies lanes
        // 32 (w % 4) .. + 31, columns 32 (w / 4) .. + 31.
        float *Rs = reinterpret_cast<float *>(smem + GT_OFF_SPL);
        bool rok = ok && mbar_wait(r_full, 0, abort);
        rok = __all_sync(0xffffffffu, rok);
        if (rok) {
            tc_fence_after();
            const int row = 32 * quarter + lane;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t r[16];
                tmem_ld16_nowait(tmem + lanes + 128u + (uint32_t)(32 * (warp >> 2) + 16 * hh), r);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    Rs[row * GT_RS + 32 * (warp >> 2) + 16 * hh + c] = __uint_as_float(r[c]);
            }
        }
        tc_fence_before();
        asm volatile("bar.sync 1, 512;" ::: "memory");
        tc_fence_after();
        if (drainer && g == 0) {
            // G_ij = h^T h (both groups' compensated sums) + m^T m + X_ij +
            // X_ji for row i = 32 quarter + lane and its 32 columns, written
            // where block (i / 4, j / 4) is in the upper triangle of the
            // k-padded-to-4 Gram; in a diagonal block the value for j >= i
            // fills both (i, j) and (j, i), so that the reduce's G is exactly
            // symmetric.
            const int i = 32 * quarter + lane;
            const int TB = (k + 3) / 4, NB = TB * (TB + 1) / 2;
            double *out = partials + (int64_t)blockIdx.x * NB * 16;
            const bool good = rok && !*abort;
            const int ta = i >> 2;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {   // 16 columns at a time
            uint32_t s0[16], c0[16], s1[16], c1[16];
            tmem_ld16_nowait(tks + 16u * hh, s0);
            tmem_ld16_nowait(tks + 64u + 16u * hh, c0);
            tmem_ld16_nowait(tks + 128u + 16u * hh, s1);
            tmem_ld16_nowait(tks + 192u + 16u * hh, c1);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int j = 32 * half + 16 * hh + c;
                const int tb = j >> 2;
                if (ta >= TB || tb >= TB || tb < ta || (tb == ta && j < i))
                    continue;
                double gij = ((double)__uint_as_float(s0[c]) - (double)__uint_as_float(c0[c])) +
                             ((double)__uint_as_float(s1[c]) - (double)__uint_as_float(c1[c]));
                gij += (double)Rs[(64 + i) * GT_RS + j];                            // m^T m
                gij += (double)Rs[i * GT_RS + j] + (double)Rs[i * GT_RS + 64 + j];   // X_ij
                gij += (double)Rs[j * GT_RS + i] + (double)Rs[j * GT_RS + 64 + i];   // X_ji
                const double v = good ? gij : (double)NAN;
                const int blk = ta * TB - ta * (ta - 1) / 2 + (tb - ta);
                out[blk * 16 + 4 * (i & 3) + (j & 3)] = v;
                if (tb == ta)   // both entries of a diagonal block from one value
                    out[blk * 16 + 4 * (j & 3) + (i & 3)] = v;
            }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == GT_WORKERS + 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                     : "memory");
    }
}

}  // namespace

bool gram_tc_usable(const float *X, int64_t rows, int k)
{
    return k >= 1 && k <= 64 && rows >= (int64_t)GT_ROWS * sm_count() &&
           (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
}

int gram_tc_parts(int64_t rows)
{
    const int64_t tiles = (rows + GT_ROWS - 1) / GT_ROWS;
    const int64_t sms = sm_count();
    return (int)(tiles < sms ? tiles : sms);
}

nmf_status launch_gram_tc(const float *X, int64_t rows, int k, double *partials, cudaStream_t s)
{
    static SmemOptIn opt_in;
    const int smem = gt_smem(k);
    NMF_TRY(ensure_smem(gram_tc_kernel, opt_in, (size_t)smem));
    gram_tc_kernel<<<gram_tc_parts(rows), GT_THREADS, smem, s>>>(X, rows, k, gt_stages(k),
                                                                 partials);
    NMF_LAUNCHED("gram_tc_kernel");
    return NMF_OK;
}

}  // namespace nmf
