// Dense products of Alg. 1 (the "MM" task) on the 5th-generation tensor cores,
// with BF16 head/tail operand splitting, and the objective of Eq. 1 fused into
// the A H^T pass:
//   trans = 0: out (m x k) = A H^T   (contract over n)
//   trans = 1: out (n x k) = A^T W   (contract over m)
// i.e. out[p][r] = sum_q A(p, q) F[q][r] with A(p, q) = A[p][q] or A[q][p].
//
// Every FP32 value v is split as v = hi + lo + O(2^-17 |v|), hi = bf16(v),
// lo = bf16(v - hi); a product uses hi*hi + hi*lo + lo*hi (each term exact in
// the FP32 accumulator's input), so its relative error is about 2^-17 and
// unbiased.
//
// Kernel (one CTA per 128 output rows). Shared memory is one ring of stages,
// each holding the FP32 A tile of a K-block (128 x 64, or 64 x 128 for
// trans = 1) and the pre-split BF16 F tiles of the same K-block (N x 64 hi
// and lo, 128-byte swizzle); 4 to 6 stages keep 100+ KB of A in flight per SM.
//   warp 0     TMA producer: refills a stage once every MMA reading it is done.
//   warp 1     allocates TMEM; one lane issues the product MMAs (M = 128,
//              K = 16; per 16-element step A_hi x [F_hi; F_lo] with N = 2N_k
//              and A_lo x F_hi with N = N_k, N_k = 16, 32 or 64). This
//              thread's instruction stream is the pass's critical path
//              (issuing an MMA, a commit or a try_wait costs 30-45 cycles), so
//              its descriptors are precomputed and it waits on as few barriers
//              as possible.
//   warps 2-5  split the FP32 A tile into BF16 hi/lo IN PLACE, in the
//              canonical K-major 128-byte-swizzled operand layout. trans = 0:
//              each thread owns one row (its TMEM lane); the 32 floats of a
//              128-byte row become [hi of the 32 | lo of the 32], so the MMA of
//              each 16-element step reads hi at +32 s bytes and lo at +64 + 32 s
//              of the row. trans = 1: the tile is transposed (thread = output
//              row), so the four warps first read the whole tile into
//              registers, meet at an mbarrier, then write hi and lo tiles.
//              A pre-split transpose (TRANS = 2, below) leaves them idle.
//   warps 6-13 drain the TMEM accumulators (tcgen05.ld) into registers; two
//              warps per TMEM lane quarter, each owning half of the columns.
//   warp 14    (objective only) issues the W H tile MMAs.
// Accuracy: the tensor cores' FP32 accumulation truncates, so every MMA that
// adds into an accumulator biases it by about half an ulp of its value;
// accumulating all n / 16 * 3 steps in one place would bias the result by
// ~1e-6 relative and spread it by as much, which the NLS solves amplify by
// cond(G). The accumulator of each K-block (4 accumulation steps of the
// dominant hi*hi products) is therefore drained into registers, where the
// drain warps add the hi*hi tile plus the cross-term tile (about 2^-8
// smaller) to a plain FP32 partial over TC_FOLD K-blocks (round to nearest,
// so unbiased) that is folded into a Kahan-compensated sum. Draining only
// every second K-block measured -1.4e-7 (the truncation grows with the square
// of the steps per drain), enough to push the objective of the small dense
// configuration past its 1e-5 tolerance.

// Fused objective (trans = 0, k <= 64): with W given, every K-block also
// forms the 128 x 64 tile of W H (W tile resident in shared memory, K = k
// padded to 16/32/64, three split products) in a third ping-pong TMEM pair.
// Its B operand is the stage's own F = H^T tile read MN-major (the 64 columns
// of the K-block contiguous, k along K), so H costs no extra loads; a second
// issuing thread (warp 14) runs these MMAs as soon as the stage lands. The
// split warps, each owning 32 rows of the tile (their TMEM lane quarter),
// subtract it from the FP32 A values they are about to split and add the
// squared residuals into Kahan-compensated FP32 sums, one per thread, which
// are added in FP64 across the CTA's threads at the end (one FP64 partial per
// CTA, summed in a fixed order). The A H^T pass of
// an ANLS iteration thereby yields f(W, H) of the previous iterate without
// reading A again. A relative bias b of W H shifts f by about S b with
// S = 2 mean(r) mean(WH) / mean(r^2) (|S| <= 4 on the dense workloads), far
// inside the 1e-5 tolerance.
//
// Pre-split transpose (TRANS = 2): a handle on dense A keeps A^T split into
// BF16 hi and lo copies (made once by mm_tc_presplit_kernel with the split
// warps' arithmetic, +4 bytes per element of A), stored tile by tile: each
// 128-row x 64-K operand tile is 16 contiguous KB already in the K-major
// 128-byte-swizzled shared-memory layout, the K-blocks of a row block in
// order. A^T W then reads 4 bytes per element as before, as one contiguous
// stream per CTA fetched by plain bulk copies: no transpose, no split and
// no in-place barrier per K-block, and bitwise the same products. (A
// row-major n x m copy read through a tensor map was slower on tall A: its
// 128 rows per tile lie m * 2 bytes apart.)
//
// F (H^T or W) is split once per call by mm_tc_split_kernel into a padded
// N x Qp BF16 pair (the workspace); k > 64 is processed in 64-column chunks.
// Every mbarrier wait is bounded (about 2 s); on timeout the kernel records
// an error code in the workspace, leaves its loops, frees TMEM and returns.
//
// Roofline: HBM (A read once, 4 bytes per element; 2k flops per element for
// the product, 2k more for the fused objective).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nmf {
namespace {

using namespace tc;

constexpr int TC_BM = 128;        // output rows per CTA (MMA M)
constexpr int TC_BK = 64;         // contraction elements per K-block (128-byte BF16 row)
constexpr int TC_DRAIN_WARPS = 8;
constexpr int TC_FOLD = 8;        // K-blocks per plain partial sum in the drain
constexpr int TC_SMEM_MAX = 227 * 1024;

template <int N, int OBJ>
struct TcLayout {
    // warps: 0 TMA, 1 product MMAs, 2-5 split, 6-13 drain, 14 objective MMAs.
    static constexpr int THREADS = 448 + (OBJ ? 32 : 0);
    static constexpr int F32_BYTES = TC_BM * TC_BK * 4;   // 32 KB FP32 A tile (split in place)
    static constexpr int A_BYTES = TC_BM * TC_BK * 2;     // 16 KB: one BF16 A tile
    static constexpr int B_BYTES = N * TC_BK * 2;         // one BF16 F tile (hi or lo)
    static constexpr int STAGE_BYTES = F32_BYTES + 2 * B_BYTES;
    static constexpr int W_BYTES = OBJ ? TC_BM * TC_BK * 2 : 0; // objective A (128 i x 64 r)
    static constexpr int FIT = (TC_SMEM_MAX - 2048 - 2 * W_BYTES) / STAGE_BYTES;
    static constexpr int STAGES = FIT > 6 ? 6 : FIT;
    static constexpr int OFF_WHI = STAGES * STAGE_BYTES;
    static constexpr int OFF_WLO = OFF_WHI + W_BYTES;
    static constexpr int OFF_BAR = OFF_WLO + W_BYTES;
    // barriers: full[S], empty[S], a_full[S], readb[S], acc_full[2],
    // acc_empty[2], obj_full[2], obj_empty[2], w_full
    static constexpr int NBAR = 4 * STAGES + 9;
    static constexpr int OFF_TMEM = OFF_BAR + NBAR * 8;
    static constexpr int OFF_ABORT = OFF_TMEM + 4;
    static constexpr int OFF_RED = (OFF_ABORT + 4 + 15) & ~15;    // 8 doubles
    static constexpr int BYTES = OFF_RED + 16 * 8;
    // TMEM: product accumulators x 2 ([hi*hi | cross], 2N), objective x 2 (64),
    // the drain's Kahan sums and compensations (2N).
    static constexpr int COL_KS = 4 * N + (OBJ ? 128 : 0);
    static constexpr int COLS = COL_KS + 2 * N;
    static constexpr int TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128
                                   : COLS <= 256 ? 256 : 512;
    static_assert(COLS <= 512, "tensor memory budget");
    static_assert(STAGES >= 3, "at least three stages");
    static_assert(STAGE_BYTES % 1024 == 0 && F32_BYTES % 1024 == 0 && B_BYTES % 1024 == 0 &&
                      A_BYTES % 1024 == 0 && OFF_WHI % 1024 == 0 && W_BYTES % 1024 == 0,
                  "128-byte-swizzled tiles need 1024-byte alignment");
    static_assert(BYTES + 1024 <= TC_SMEM_MAX, "shared memory budget");
};

struct TcArgs {
    int64_t P, Q;
    int k, col0, kc;
    int kb_per_split;       // K-blocks per CTA along the contraction (grid.y splits)
    float *out;             // grid.y == 1: the output; else partials [split][P][k]
    double *obj_partials;   // per-CTA sums of squared residuals (OBJ)
    int *err;
    // TRANS = 2: A^T pre-split, tile-major (see mm_tc_presplit_kernel).
    const unsigned char *at_hi, *at_lo;
    int64_t at_kbs;         // K-blocks per 128-row block of tiles
};

// -------------------------------------------------------------------- kernel
template <int N, int TRANS, int OBJ>
__global__ void __launch_bounds__(TcLayout<N, OBJ>::THREADS, 1)
    mm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                 const __grid_constant__ CUtensorMap tmBlo, const __grid_constant__ CUtensorMap tmWhi,
                 const __grid_constant__ CUtensorMap tmWlo, const TcArgs args)
{
    static_assert(!OBJ || TRANS == 0 || TRANS == 3, "the objective rides on the A H^T pass");
    // Pre-split A (TRANS = 3) with the objective: the residual warps read each
    // stage too and release it with the MMA commits.
    constexpr int EMPTY_ARRIVALS = 1 + OBJ + (TRANS == 3 && OBJ ? 4 : 0);
    using L = TcLayout<N, OBJ>;
    constexpr int S = L::STAGES;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = reinterpret_cast<volatile int *>(smem + L::OFF_ABORT);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::OFF_TMEM);
    const int64_t P = args.P, Q = args.Q;

    const uint32_t bar0 = sbase + L::OFF_BAR;
    auto full = [&](int i) { return bar0 + 8u * i; };              // TMA bytes landed
    auto empty = [&](int i) { return bar0 + 8u * (S + i); };       // MMAs of the stage done
    auto a_full = [&](int i) { return bar0 + 8u * (2 * S + i); };  // A split in place
    auto readb = [&](int i) { return bar0 + 8u * (3 * S + i); };   // trans = 1: tile read
    const uint32_t accb = bar0 + 8u * (4 * S);
    auto acc_full = [&](int i) { return accb + 8u * i; };
    auto acc_empty = [&](int i) { return accb + 8u * (2 + i); };
    auto obj_full = [&](int i) { return accb + 8u * (4 + i); };
    auto obj_empty = [&](int i) { return accb + 8u * (6 + i); };
    const uint32_t w_full = accb + 8u * 8;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(full(i), 1);
            mbar_init(empty(i), EMPTY_ARRIVALS);   // product MMAs (+ objective)
            mbar_init(a_full(i), 4);
            mbar_init(readb(i), 4);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(acc_full(i), 1);
            mbar_init(acc_empty(i), TC_DRAIN_WARPS);
            mbar_init(obj_full(i), 1);
            mbar_init(obj_empty(i), 4);
        }
        mbar_init(w_full, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"((uint32_t)L::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t p0 = (int64_t)blockIdx.x * TC_BM;
    const int nkb_all = (int)((Q + TC_BK - 1) / TC_BK);
    const int kb0 = blockIdx.y * args.kb_per_split;   // first K-block of this CTA
    const int nkb = min(args.kb_per_split, nkb_all - kb0);
    auto stage = [&](int s) { return sbase + (uint32_t)(s * L::STAGE_BYTES); };
    // Descriptors are formed once and advanced by constant adds: the start
    // address field holds addr >> 4 in its low 14 bits, and every shared
    // address here is below 256 KB, so no carry leaves the field.
    constexpr uint64_t STAGE16 = (uint64_t)(L::STAGE_BYTES >> 4);
    constexpr uint64_t F16 = (uint64_t)(L::F32_BYTES >> 4);
    constexpr uint64_t BLO16 = (uint64_t)(L::B_BYTES >> 4);

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            if (OBJ) {
                mbar_arrive_expect_tx(w_full, 2 * L::W_BYTES);
                tma_load_2d(sbase + L::OFF_WHI, &tmWhi, 0, (int)p0, w_full);
                tma_load_2d(sbase + L::OFF_WLO, &tmWlo, 0, (int)p0, w_full);
            }
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % S, u = kb / S;
                if (!mbar_wait(empty(s), (u & 1) ^ 1, abort))
                    break;
                mbar_arrive_expect_tx(full(s), L::STAGE_BYTES);
                const uint32_t dst = stage(s);
                const int q0 = (kb0 + kb) * TC_BK;
                if (TRANS == 0) {
                    // Two 128-byte-swizzled halves of 32 columns each.
                    tma_load_2d(dst, &tmA, q0, (int)p0, full(s));
                    tma_load_2d(dst + L::F32_BYTES / 2, &tmA, q0 + 32, (int)p0, full(s));
                } else if (TRANS == 1) {
                    tma_load_2d(dst, &tmA, (int)p0, q0, full(s));
                } else {
                    // Pre-split A^T (TRANS = 2) or A (3): each hi / lo tile is 16
                    // contiguous KB in global memory, already in the K-major
                    // swizzled operand layout the split warps would write.
                    const size_t toff =
                        ((size_t)blockIdx.x * (size_t)args.at_kbs + (size_t)(kb0 + kb)) *
                        (size_t)L::A_BYTES;
                    bulk_load(dst, args.at_hi + toff, L::A_BYTES, full(s));
                    bulk_load(dst + L::A_BYTES, args.at_lo + toff, L::A_BYTES, full(s));
                }
                tma_load_2d(dst + L::F32_BYTES, &tmBhi, q0, 0, full(s));
                tma_load_2d(dst + L::F32_BYTES + L::B_BYTES, &tmBlo, q0, 0, full(s));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ product MMAs
        // One thread issues the MMAs; its instruction stream is on the
        // critical path (each tcgen05.mma, commit or try_wait costs 30-45
        // cycles to issue), so per 16-element step it issues two: A_hi times
        // the stacked [F_hi; F_lo] (N' = 2N: the F lo tile follows the hi tile
        // in the stage, 8-row groups 1024 bytes apart, so the two form one
        // K-major operand) and A_lo times F_hi into the second half. The
        // accumulator of a K-block, D = [hi*hi | cross terms] (2N columns), is
        // drained after that K-block; two such buffers ping-pong at TMEM
        // columns [0, 4N), the objective's W H buffers follow at [4N, 4N + 128).
        if (lane == 0) {
            const uint32_t idesc2 = idesc_bf16_f32<2 * N>();
            const uint32_t idesc = idesc_bf16_f32<N>();
            const uint64_t a0 = sw128_desc(sbase), b0 = a0 + F16;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % S, u = kb / S;
                const int b = kb & 1, ub = kb >> 1;
                if (!mbar_wait_fast(acc_empty(b), (ub & 1) ^ 1, abort) ||
                    !mbar_wait_fast(TRANS >= 2 ? full(s) : a_full(s), u & 1, abort))
                    break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * 2 * N);
                const uint64_t as = a0 + (uint64_t)s * STAGE16;
                const uint64_t bh = b0 + (uint64_t)s * STAGE16;
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk) {
                    // A hi / lo of this 16-element step (see the split warps).
                    const uint64_t ah = TRANS == 0
                                            ? as + (uint64_t)((kk >> 1) * (L::F32_BYTES / 32) + (kk & 1) * 2)
                                            : as + (uint64_t)(kk * 2);
                    const uint64_t al = TRANS == 0 ? ah + 4 : ah + (uint64_t)(L::A_BYTES >> 4);
                    const uint64_t o = (uint64_t)(kk * 2);   // 16 BF16 = 32 bytes along K
                    mma_bf16(d, ah, bh + o, idesc2, kk ? 1u : 0u);
                    mma_bf16(d + (uint32_t)N, al, bh + o, idesc, 1u);
                }
                mma_commit(empty(s));
                mma_commit(acc_full(b));
            }
        }
    } else if (OBJ && warp == 14) {
        // ---------------------------------------------------- objective MMAs
        // W H tile of every K-block: W (K-major, K = r, resident) times the
        // stage's F = H^T tile read MN-major (N = the K-block's 64 columns),
        // issued by its own thread so it never waits behind the products.
        if (lane == 0) {
            const uint32_t idesc_obj = idesc_bf16_f32<TC_BK, 1>();
            const uint64_t wh = sw128_desc(sbase + L::OFF_WHI), wl = sw128_desc(sbase + L::OFF_WLO);
            const uint64_t f0 = sw128_mn_desc(sbase + L::F32_BYTES, 1024);
            bool ok = mbar_wait_fast(w_full, 0, abort);
            for (int j = 0; j < nkb && ok; ++j) {
                const int s = j % S, u = j / S;
                const int b = j & 1, ub = j >> 1;
                if (!mbar_wait_fast(obj_empty(b), (ub & 1) ^ 1, abort) ||
                    !mbar_wait_fast(full(s), u & 1, abort))
                    break;
                tc_fence_after();
                const uint32_t d3 = tmem + (uint32_t)(4 * N + b * 64);
                const uint64_t fh = f0 + (uint64_t)s * STAGE16, fl = fh + BLO16;
#pragma unroll
                for (int kk = 0; kk < N / 16; ++kk) {
                    const uint64_t o = (uint64_t)(kk * 2);            // 16 r along W's rows
                    const uint64_t of = (uint64_t)(kk * (2048 >> 4)); // 16 r = two 8-row groups
                    mma_bf16(d3, wh + o, fh + of, idesc_obj, kk ? 1u : 0u);
                    mma_bf16(d3, wh + o, fl + of, idesc_obj, 1u);
                    mma_bf16(d3, wl + o, fh + of, idesc_obj, 1u);
                }
                mma_commit(obj_full(b));
                mma_commit(empty(s));
            }
        }
    } else if ((TRANS <= 1 || (TRANS == 3 && OBJ)) && warp >= 2 && warp < 6) {
        // ---------------------------------------------------- split (warps 2-5)
        const int ct = threadIdx.x - 64;        // 0..127
        const int quarter = warp & 3;           // TMEM lane quarter of this warp
        const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
        // Sum of squared residuals: FP32 per half row, Kahan-compensated FP32
        // across K-blocks (FP64 adds here would queue on GB300's narrow FP64
        // pipe in the split warps' critical path), FP64 across threads.
        float fs = 0.0f, fc = 0.0f;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % S, u = kb / S;
            if (!mbar_wait(full(s), u & 1, abort))
                break;
            unsigned char *st = smem + s * L::STAGE_BYTES;
            const int b1 = kb & 1, u1 = kb >> 1;
            if (TRANS == 3) {
                // Residuals only: the stage holds A's hi and lo tiles (row r
                // = this thread's TMEM lane, K-major, 128-byte swizzled); a =
                // hi + lo, the value the products use (within 2^-18 of A).
                const int r = quarter * 32 + lane;
                if (!mbar_wait(obj_full(b1), u1 & 1, abort))
                    break;
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t whr[32];
                    tmem_ld32_nowait(tq + (uint32_t)(4 * N + b1 * 64 + h * 32), whr);
                    float a[32];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint4 qh = *reinterpret_cast<const uint4 *>(st + sw128_off(r, 4 * h + c));
                        const uint4 ql = *reinterpret_cast<const uint4 *>(st + L::A_BYTES +
                                                                          sw128_off(r, 4 * h + c));
                        const uint32_t hw[4] = {qh.x, qh.y, qh.z, qh.w};
                        const uint32_t lw[4] = {ql.x, ql.y, ql.z, ql.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float2 sum = __fadd2_rn(
                                make_float2(__uint_as_float(hw[j] << 16),
                                            __uint_as_float(hw[j] & 0xffff0000u)),
                                make_float2(__uint_as_float(lw[j] << 16),
                                            __uint_as_float(lw[j] & 0xffff0000u)));
                            a[8 * c + 2 * j] = sum.x;
                            a[8 * c + 2 * j + 1] = sum.y;
                        }
                    }
                    tmem_wait_ld();
                    float2 q01 = make_float2(0.0f, 0.0f), q23 = make_float2(0.0f, 0.0f);
                    const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
                    for (int i = 0; i < 32; i += 4) {
                        const float2 e01 = __ffma2_rn(
                            make_float2(__uint_as_float(whr[i]), __uint_as_float(whr[i + 1])), m1,
                            make_float2(a[i], a[i + 1]));
                        const float2 e23 = __ffma2_rn(
                            make_float2(__uint_as_float(whr[i + 2]), __uint_as_float(whr[i + 3])),
                            m1, make_float2(a[i + 2], a[i + 3]));
                        q01 = __ffma2_rn(e01, e01, q01);
                        q23 = __ffma2_rn(e23, e23, q23);
                    }
                    const float y = ((q01.x + q01.y) + (q23.x + q23.y)) - fc;
                    const float t = fs + y;
                    fc = (t - fs) - y;
                    fs = t;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(obj_empty(b1));
                    mbar_arrive(empty(s));   // this stage's A is read
                }
                continue;
            }
            if (TRANS == 0) {
                // Two swizzled halves of 128 rows (p) x 32 floats (q). Each
                // thread owns row r (= its TMEM lane) and rewrites the 128
                // bytes of its row in a half as [hi of the 32 | lo of the 32].
                const int r = quarter * 32 + lane;
                if (OBJ) {
                    if (!mbar_wait(obj_full(b1), u1 & 1, abort))
                        break;
                    tc_fence_after();
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    unsigned char *hs = st + h * (L::F32_BYTES / 2);
                    uint32_t whr[32];
                    if (OBJ)   // W H tile of these columns; consumed after the A loads
                        tmem_ld32_nowait(tq + (uint32_t)(4 * N + b1 * 64 + h * 32), whr);
                    float a[32];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 v = *reinterpret_cast<const float4 *>(hs + sw128_off(r, c));
                        a[4 * c] = v.x;
                        a[4 * c + 1] = v.y;
                        a[4 * c + 2] = v.z;
                        a[4 * c + 3] = v.w;
                    }
                    if (OBJ) {
                        tmem_wait_ld();
                        // Squared residuals in four chains (entries i mod 4),
                        // two per packed FP32x2 FMA: e = a + (-1) wh, q += e e.
                        float2 q01 = make_float2(0.0f, 0.0f), q23 = make_float2(0.0f, 0.0f);
                        const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
                        for (int i = 0; i < 32; i += 4) {
                            const float2 e01 = __ffma2_rn(
                                make_float2(__uint_as_float(whr[i]), __uint_as_float(whr[i + 1])),
                                m1, make_float2(a[i], a[i + 1]));
                            const float2 e23 = __ffma2_rn(
                                make_float2(__uint_as_float(whr[i + 2]),
                                            __uint_as_float(whr[i + 3])),
                                m1, make_float2(a[i + 2], a[i + 3]));
                            q01 = __ffma2_rn(e01, e01, q01);
                            q23 = __ffma2_rn(e23, e23, q23);
                        }
                        const float y = ((q01.x + q01.y) + (q23.x + q23.y)) - fc;
                        const float t = fs + y;
                        fc = (t - fs) - y;
                        fs = t;
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float w8[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            w8[j] = a[8 * c + j];
                        uint4 hi, lo;
                        split8(w8, hi, lo);
                        *reinterpret_cast<uint4 *>(hs + sw128_off(r, c)) = hi;
                        *reinterpret_cast<uint4 *>(hs + sw128_off(r, 4 + c)) = lo;
                    }
                }
                if (OBJ)
                    tc_fence_before();
            } else {
                // 64 rows (q) x 128 floats (p), 512 bytes per row; this thread
                // produces output row p = ct. Read the whole column first (the
                // hi / lo tiles overwrite other threads' columns).
                const float *sp = reinterpret_cast<const float *>(st);
                float v[TC_BK];
#pragma unroll
                for (int j = 0; j < TC_BK; ++j)
                    v[j] = sp[j * TC_BM + ct];
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(readb(s));
                if (!mbar_wait(readb(s), u & 1, abort))
                    break;
                unsigned char *ahi = st;
                unsigned char *alo = st + L::A_BYTES;
#pragma unroll
                for (int c = 0; c < TC_BK / 8; ++c) {
                    float w8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        w8[j] = v[8 * c + j];
                    uint4 hi, lo;
                    split8(w8, hi, lo);
                    *reinterpret_cast<uint4 *>(ahi + sw128_off(ct, c)) = hi;
                    *reinterpret_cast<uint4 *>(alo + sw128_off(ct, c)) = lo;
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                if (OBJ)
                    mbar_arrive(obj_empty(b1));
                mbar_arrive(a_full(s));
            }
        }
        if (OBJ) {
            double fsum = (double)fs - (double)fc;
            for (int o = 16; o > 0; o >>= 1)
                fsum += __shfl_xor_sync(FULL, fsum, o);
            if (lane == 0)
                reinterpret_cast<double *>(smem + L::OFF_RED)[warp - 2] = fsum;
        }
    } else if (warp >= 6 && warp < 14) {
        // ------------------------------------------------ drain (warps 6-13)
        // Per K-block, hi*hi tile + cross-term tile go into a plain FP32
        // partial sum (round to nearest: unbiased) which every TC_FOLD
        // K-blocks is folded into a Kahan-compensated sum. The Kahan sum and
        // compensation live in TMEM (columns [COL_KS, COL_KS + 2N)), touched
        // only at the folds, so registers hold just the partial.
        constexpr int NH = N / 2;               // product columns owned by this warp
        constexpr int CH = NH < 8 ? NH : 8;     // columns per TMEM access
        static_assert(CH % 2 == 0, "drain columns go in pairs");
        const int dw = warp - 6;
        const int quarter = warp & 3;           // TMEM lane quarter of this warp
        const int half = dw >> 2;               // which half of the columns
        const int cbase = half * NH;
        const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
        const uint32_t ks = tq + (uint32_t)(L::COL_KS + cbase);       // Kahan sums
        const uint32_t kc = tq + (uint32_t)(L::COL_KS + N + cbase);   // compensations
        float part[NH];
#pragma unroll
        for (int c = 0; c < NH; ++c)
            part[c] = 0.0f;
        auto add_tile = [&](uint32_t ta) {
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += CH) {
                float v[CH], w[CH];
                tmem_ld<CH>(ta + (uint32_t)c0, v);
                tmem_ld<CH>(ta + (uint32_t)(N + c0), w);
#pragma unroll
                for (int i = 0; i < CH; i += 2) {   // part += v + w, two columns per op
                    const float2 vw =
                        __fadd2_rn(make_float2(v[i], v[i + 1]), make_float2(w[i], w[i + 1]));
                    const float2 pt =
                        __fadd2_rn(make_float2(part[c0 + i], part[c0 + i + 1]), vw);
                    part[c0 + i] = pt.x;
                    part[c0 + i + 1] = pt.y;
                }
            }
        };
        bool folded = false;
        auto fold = [&]() {
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += CH) {
                float sm[CH], cm[CH];
                if (folded) {
                    tmem_ld<CH>(ks + (uint32_t)c0, sm);
                    tmem_ld<CH>(kc + (uint32_t)c0, cm);
                } else {
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        sm[i] = cm[i] = 0.0f;
                }
                const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
                for (int i = 0; i < CH; i += 2) {   // Kahan step, two columns per op
                    const float2 s2 = make_float2(sm[i], sm[i + 1]);
                    const float2 y = __ffma2_rn(make_float2(cm[i], cm[i + 1]), m1,
                                                make_float2(part[c0 + i], part[c0 + i + 1]));
                    const float2 t = __fadd2_rn(s2, y);
                    const float2 c = __ffma2_rn(y, m1, __ffma2_rn(s2, m1, t));   // (t - s) - y
                    cm[i] = c.x;
                    cm[i + 1] = c.y;
                    sm[i] = t.x;
                    sm[i + 1] = t.y;
                    part[c0 + i] = 0.0f;
                    part[c0 + i + 1] = 0.0f;
                }
                tmem_st<CH>(ks + (uint32_t)c0, sm);
                tmem_st<CH>(kc + (uint32_t)c0, cm);
            }
            tmem_wait_st();
            folded = true;
        };
        const int row = quarter * 32 + lane;    // row of the tile owned by this thread
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
            const int b = kb & 1, ub = kb >> 1;
            if (!mbar_wait(acc_full(b), ub & 1, abort)) {
                ok = false;
                break;
            }
            tc_fence_after();
            add_tile(tq + (uint32_t)(b * 2 * N + cbase));
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(acc_empty(b));
            if ((kb % TC_FOLD) == TC_FOLD - 1)
                fold();
        }
        if (ok) {
            fold();
            const int64_t p = p0 + row;
            float *o = args.out + (int64_t)blockIdx.y * P * args.k + p * args.k + args.col0 + cbase;
#pragma unroll
            for (int c0 = 0; c0 < NH; c0 += CH) {
                float sm[CH], cm[CH];
                tmem_ld<CH>(ks + (uint32_t)c0, sm);
                tmem_ld<CH>(kc + (uint32_t)c0, cm);
                if (p < P) {
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        if (cbase + c0 + i < args.kc)
                            o[c0 + i] = sm[i] - cm[i];
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (*abort)
            atomicExch(args.err, 1);
        if (OBJ) {
            const double *red = reinterpret_cast<const double *>(smem + L::OFF_RED);
            double s = 0.0;
            for (int w = 0; w < 4; ++w)
                s += red[w];
            args.obj_partials[blockIdx.x] = s;
        }
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)L::TMEM_COLS)
                     : "memory");
    }
}

// F (Q x k, float32 row-major) columns [col0, col0 + kc) -> BF16 hi / lo
// tiles laid out [N rows (r)][Qp cols (q)], zero-padded. 32 x 32 transposes.
__global__ void mm_tc_split_kernel(const float *__restrict__ F, int64_t Q, int k, int col0,
                                   int kc, int N, int64_t Qp, __nv_bfloat16 *__restrict__ hi,
                                   __nv_bfloat16 *__restrict__ lo)
{
    __shared__ float t[32][33];
    const int64_t q0 = (int64_t)blockIdx.x * 32;
    const int r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t q = q0 + i;
        const int r = r0 + threadIdx.x;
        t[i][threadIdx.x] = (q < Q && r < kc) ? F[q * k + col0 + r] : 0.0f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i;
        const int64_t q = q0 + threadIdx.x;
        if (r < N && q < Qp) {
            const float v = t[threadIdx.x][i];
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[(int64_t)r * Qp + q] = h;
            lo[(int64_t)r * Qp + q] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// X (rows x k, float32 row-major, k <= 64) -> BF16 hi / lo rows of 64
// (zero-padded columns and rows up to rows_p): the objective's K-major
// operands W [i][r] and H^T [j][r].
// Pre-split operand copies, hi = bf16(v), lo = bf16(v - hi) exactly as
// split2, tile-major: element (row p, K index q) of the Pp x Qp padded
// operand lies in tile (p / 128) * kbs + q / 64, at byte (p % 128) * 128 +
// ((q % 64 / 8) ^ (p % 8)) * 16 + (q % 8) * 2 of it (the SW128 K-major
// operand layout); the padding is zero. Each thread writes whole 16-byte
// chunks (8 consecutive q of one row p) of both copies.
__device__ __forceinline__ void presplit_chunk(unsigned char *__restrict__ hi_t,
                                               unsigned char *__restrict__ lo_t, int64_t p,
                                               int64_t q8, int64_t kbs, const float (&v)[8])
{
    uint4 hi, lo;
    split8(v, hi, lo);
    const int pr = (int)(p & 127), cc = (int)((q8 & 63) >> 3);
    const size_t off = ((size_t)(p >> 7) * (size_t)kbs + (size_t)(q8 >> 6)) * 16384 +
                       (size_t)(pr * 128 + ((cc ^ (pr & 7)) << 4));
    *reinterpret_cast<uint4 *>(hi_t + off) = hi;
    *reinterpret_cast<uint4 *>(lo_t + off) = lo;
}

// A (m x n FP32, row stride lda a multiple of 4, 16-byte-aligned base) as the
// operand of A H^T: p = A's row i, q = A's column j. One chunk per thread,
// grid-stride over the Pp x Qp / 8 chunks (consecutive threads: consecutive
// chunks of a row, so reads and writes are coalesced).
__global__ void __launch_bounds__(256)
    mm_tc_presplit_rows_kernel(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                               int64_t Qp, int64_t Pp, int64_t kbs,
                               unsigned char *__restrict__ hi_t, unsigned char *__restrict__ lo_t)
{
    const int64_t cpr = Qp >> 3;   // chunks per row
    const int64_t total = Pp * cpr;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / cpr, q8 = (e - p * cpr) << 3;
        float v[8];
        if (p < m && q8 + 8 <= n) {
            const float4 a0 = *reinterpret_cast<const float4 *>(A + p * lda + q8);
            const float4 a1 = *reinterpret_cast<const float4 *>(A + p * lda + q8 + 4);
            v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
            v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
        } else {
#pragma unroll
            for (int t = 0; t < 8; ++t)
                v[t] = (p < m && q8 + t < n) ? A[p * lda + q8 + t] : 0.0f;
        }
        presplit_chunk(hi_t, lo_t, p, q8, kbs, v);
    }
}

// A as the operand of A^T W: p = A's column j, q = A's row i. 64 x 64 element
// blocks of A through shared memory (read along j), each thread then writes
// the chunks of 8 consecutive i of one column j.
__global__ void __launch_bounds__(256)
    mm_tc_presplit_kernel(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                          int64_t Qp, int64_t Pp, int64_t kbs, unsigned char *__restrict__ hi_t,
                          unsigned char *__restrict__ lo_t)
{
    __shared__ float tile[64][65];
    const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
    const int tid = threadIdx.x;
    for (int e = tid; e < 64 * 64; e += 256) {
        const int r = e >> 6, c = e & 63;
        const int64_t i = i0 + r, j = j0 + c;
        tile[r][c] = (i < m && j < n) ? A[i * lda + j] : 0.0f;
    }
    __syncthreads();
    for (int e = tid; e < 64 * 8; e += 256) {   // (column c, chunk g of 8 rows)
        const int c = e >> 3, g = e & 7;
        const int64_t p = j0 + c, q8 = i0 + 8 * g;
        if (p < Pp && q8 < Qp) {
            float v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t)
                v[t] = tile[8 * g + t][c];
            presplit_chunk(hi_t, lo_t, p, q8, kbs, v);
        }
    }
}

__global__ void mm_tc_split_rows_kernel(const float *__restrict__ X, int64_t rows, int k,
                                        int64_t rows_p, __nv_bfloat16 *__restrict__ hi,
                                        __nv_bfloat16 *__restrict__ lo)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows_p * 64)
        return;
    const int64_t r = e >> 6;
    const int c = (int)(e & 63);
    const float v = (r < rows && c < k) ? X[r * k + c] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// out[p][col0 + c] = sum over splits of part[s][p][col0 + c], in split order.
__global__ void mm_tc_reduce_kernel(const float *__restrict__ part, int splits, int64_t P, int k,
                                    int col0, int kc, float *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * kc)
        return;
    const int64_t p = e / kc;
    const int c = col0 + (int)(e % kc);
    double acc = 0.0;
    for (int sp = 0; sp < splits; ++sp)
        acc += (double)part[(int64_t)sp * P * k + p * k + c];
    out[p * k + c] = (float)acc;
}

__global__ void obj_sum_kernel(const double *__restrict__ parts, int n, double *__restrict__ f)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        s += parts[i];
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_down_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            t += red[w];
        *f = t;
    }
}

// ------------------------------------------------------------ host side
constexpr size_t TC_ERR_BYTES = 256;

template <int N, int TRANS, int OBJ>
nmf_status launch_tc(const CUtensorMap (&maps)[5], const TcArgs &a, cudaStream_t s)
{
    using L = TcLayout<N, OBJ>;
    const int smem = L::BYTES + 1024;
    static SmemOptIn opt_in;
    NMF_TRY(ensure_smem(mm_tc_kernel<N, TRANS, OBJ>, opt_in, (size_t)smem));
    const int nkb = (int)cdiv(a.Q, TC_BK);
    const dim3 grid((unsigned)cdiv(a.P, TC_BM), (unsigned)cdiv(nkb, a.kb_per_split));
    mm_tc_kernel<N, TRANS, OBJ><<<grid, L::THREADS, smem, s>>>(maps[0], maps[1], maps[2], maps[3],
                                                               maps[4], a);
    NMF_LAUNCHED("mm_tc_kernel");
    return NMF_OK;
}

template <int TRANS, int OBJ>
nmf_status launch_tc_n(int N, const CUtensorMap (&maps)[5], const TcArgs &a, cudaStream_t s)
{
    if (N == 16)
        return launch_tc<16, TRANS, OBJ>(maps, a, s);
    if (N == 32)
        return launch_tc<32, TRANS, OBJ>(maps, a, s);
    return launch_tc<64, TRANS, OBJ>(maps, a, s);
}

// Workspace: [err | product F split (2 x N x Qp BF16) | objective: W split
// (2 x Pp x 64) | per-CTA partials | contraction-split partials].
struct TcWork {
    size_t f_off, w_off, part_off, split_off, total;
};

constexpr int TC_MAX_SPLITS = 16;   // tall-skinny A: few output tiles, a long contraction

// Contraction splits that fill the last wave of CTAs better (1 CTA per SM).
int choose_splits(int64_t P, int64_t Q)
{
    const int64_t tiles = cdiv(P, TC_BM), nkb = cdiv(Q, TC_BK);
    const int64_t sms = sm_count();
    auto eff = [&](int64_t ctas) { return (double)ctas / (double)(cdiv(ctas, sms) * sms); };
    int best = 1;
    double best_eff = eff(tiles);
    for (int sp = 2; sp <= TC_MAX_SPLITS; ++sp) {
        if (nkb / sp < 16)
            break;
        const double e = eff(tiles * sp);
        if (e > best_eff + 0.03) {
            best = sp;
            best_eff = e;
        }
    }
    return best;
}

TcWork tc_work(int64_t m, int64_t n, int k, int trans, bool obj)
{
    const int64_t P = trans ? n : m;
    const int64_t Q = trans ? m : n;
    const int64_t Qp = cdiv(Q > 0 ? Q : 1, TC_BK) * TC_BK;
    const int64_t Pp = cdiv(P > 0 ? P : 1, TC_BM) * TC_BM;
    const int N = k <= 16 ? 16 : k <= 32 ? 32 : 64;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    TcWork w;
    w.f_off = TC_ERR_BYTES;
    size_t off = w.f_off + al(2 * sizeof(__nv_bfloat16) * (size_t)N * (size_t)Qp);
    w.w_off = off;
    if (obj)
        off += al(2 * sizeof(__nv_bfloat16) * (size_t)Pp * 64);
    w.part_off = off;
    if (obj)
        off += al(sizeof(double) * (size_t)(Pp / TC_BM));
    w.split_off = off;
    const int splits = obj ? 1 : choose_splits(P, Q);
    if (splits > 1)
        off += al(sizeof(float) * (size_t)splits * (size_t)(P > 0 ? P : 1) * (size_t)k);
    w.total = off;
    return w;
}

}  // namespace

int mm_tc_splits(int64_t m, int64_t n, int trans)
{
    return choose_splits(trans ? n : m, trans ? m : n);
}

size_t mm_tc_work_bytes(int64_t m, int64_t n, int k, int trans)
{
    const size_t a = tc_work(m, n, k, trans, false).total;
    const size_t b = (trans == 0 && k <= 64) ? tc_work(m, n, k, trans, true).total : 0;
    return a > b ? a : b;
}

namespace {

// Products, and with W / f_dev given (trans = 0, k <= 64) the fused
// objective f(W, H) with H^T = F written to *f_dev; with at_hi / at_lo given
// (trans = 1) A^T W from the pre-split transpose instead of A.
nmf_status launch_mm_tc_impl(const float *A, int64_t m, int64_t n, int64_t lda, const float *F,
                             int k, int trans, float *out, const float *W, double *f_dev,
                             void *work, size_t work_bytes, cudaStream_t s,
                             const void *at_hi, const void *at_lo)
{
    const bool presplit = at_hi != nullptr;
    if (presplit && !at_lo)
        return NMF_ERR_INVALID_ARG;
    const int64_t P = trans ? n : m;
    const int64_t Q = trans ? m : n;
    const bool obj = f_dev != nullptr;
    if (obj && (trans != 0 || k > 64 || !W))
        return NMF_ERR_INVALID_ARG;
    if (P == 0 || Q == 0) {
        if (P > 0 && cudaMemsetAsync(out, 0, sizeof(float) * (size_t)P * k, s) != cudaSuccess)
            return NMF_ERR_CUDA;
        if (obj && cudaMemsetAsync(f_dev, 0, sizeof(double), s) != cudaSuccess)
            return NMF_ERR_CUDA;
        return NMF_OK;
    }
    // TMA needs a 16-byte-aligned base and row pitch; coordinates must fit int32.
    if (P > INT32_MAX || Q > INT32_MAX)
        return NMF_ERR_INVALID_ARG;
    if (presplit ? ((reinterpret_cast<uintptr_t>(at_hi) | reinterpret_cast<uintptr_t>(at_lo)) & 15)
                 : ((reinterpret_cast<uintptr_t>(A) & 15) || (lda % 4)))
        return NMF_ERR_INVALID_ARG;
    const TcWork wl = tc_work(m, n, k, trans, obj);
    if (!work || work_bytes < wl.total)
        return NMF_ERR_INVALID_ARG;
    const int64_t Qp = cdiv(Q, TC_BK) * TC_BK;
    const int64_t Pp = cdiv(P, TC_BM) * TC_BM;
    char *wb = static_cast<char *>(work);
    int *err = reinterpret_cast<int *>(wb);
    NMF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    __nv_bfloat16 *bhi = reinterpret_cast<__nv_bfloat16 *>(wb + wl.f_off);
    CUtensorMap maps[5];
    bool ok = true;
    if (!presplit)   // (the pre-split A^T is read by plain bulk copies, no map)
        ok = trans == 0 ? make_map_2d(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, (uint64_t)Q,
                                      (uint64_t)P, (uint64_t)lda * 4, 32, TC_BM,
                                      CU_TENSOR_MAP_SWIZZLE_128B)
                        : make_map_2d(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, (uint64_t)P,
                                      (uint64_t)Q, (uint64_t)lda * 4, TC_BM, TC_BK,
                                      CU_TENSOR_MAP_SWIZZLE_NONE);
    if (!ok)
        return NMF_ERR_CUDA;
    TcArgs a;
    a.P = P;
    a.Q = Q;
    a.k = k;
    a.out = out;
    a.err = err;
    a.obj_partials = reinterpret_cast<double *>(wb + wl.part_off);
    a.at_hi = static_cast<const unsigned char *>(at_hi);
    a.at_lo = static_cast<const unsigned char *>(at_lo);
    a.at_kbs = Qp / TC_BK;
    if (obj) {
        __nv_bfloat16 *whi = reinterpret_cast<__nv_bfloat16 *>(wb + wl.w_off);
        __nv_bfloat16 *wlo = whi + (size_t)Pp * 64;
        mm_tc_split_rows_kernel<<<(unsigned)cdiv(Pp * 64, 256), 256, 0, s>>>(W, P, k, Pp, whi, wlo);
        NMF_LAUNCHED("mm_tc_split_rows_kernel");
        if (!make_map_2d(&maps[3], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, whi, 64, (uint64_t)Pp, 128,
                         64, TC_BM, CU_TENSOR_MAP_SWIZZLE_128B) ||
            !make_map_2d(&maps[4], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, wlo, 64, (uint64_t)Pp, 128,
                         64, TC_BM, CU_TENSOR_MAP_SWIZZLE_128B))
            return NMF_ERR_CUDA;
    } else if (!presplit) {
        maps[3] = maps[4] = maps[0];   // unused
    }
    for (int col0 = 0; col0 < k; col0 += 64) {
        const int kc = k - col0 < 64 ? k - col0 : 64;
        const int N = kc <= 16 ? 16 : kc <= 32 ? 32 : 64;
        __nv_bfloat16 *blo = bhi + (size_t)N * Qp;
        dim3 sg((unsigned)cdiv(Qp, 32), (unsigned)cdiv(N, 32));
        mm_tc_split_kernel<<<sg, dim3(32, 8), 0, s>>>(F, Q, k, col0, kc, N, Qp, bhi, blo);
        NMF_LAUNCHED("mm_tc_split_kernel");
        if (!make_map_2d(&maps[1], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, bhi, (uint64_t)Qp, (uint64_t)N,
                         (uint64_t)Qp * 2, TC_BK, (uint32_t)N, CU_TENSOR_MAP_SWIZZLE_128B) ||
            !make_map_2d(&maps[2], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, blo, (uint64_t)Qp, (uint64_t)N,
                         (uint64_t)Qp * 2, TC_BK, (uint32_t)N, CU_TENSOR_MAP_SWIZZLE_128B))
            return NMF_ERR_CUDA;
        if (presplit) {                  // TRANS = 2 / 3 read A by plain bulk copies
            maps[0] = maps[1];
            if (!obj)
                maps[3] = maps[4] = maps[1];
        }
        a.col0 = col0;
        a.kc = kc;
        const bool fuse = obj && col0 == 0;
        const int splits = fuse ? 1 : choose_splits(P, Q);
        const int nkb = (int)cdiv(Q, TC_BK);
        a.kb_per_split = (int)cdiv(nkb, splits);
        const int grid_y = (int)cdiv(nkb, a.kb_per_split);
        float *partial = reinterpret_cast<float *>(wb + wl.split_off);
        a.out = grid_y > 1 ? partial : out;
        nmf_status st;
        if (trans)
            st = presplit ? launch_tc_n<2, 0>(N, maps, a, s) : launch_tc_n<1, 0>(N, maps, a, s);
        else if (fuse)
            st = presplit ? launch_tc_n<3, 1>(N, maps, a, s) : launch_tc_n<0, 1>(N, maps, a, s);
        else
            st = presplit ? launch_tc_n<3, 0>(N, maps, a, s) : launch_tc_n<0, 0>(N, maps, a, s);
        NMF_TRY(st);
        if (grid_y > 1) {
            mm_tc_reduce_kernel<<<(unsigned)cdiv(P * kc, 256), 256, 0, s>>>(partial, grid_y, P, k,
                                                                            col0, kc, out);
            NMF_LAUNCHED("mm_tc_reduce_kernel");
        }
        if (fuse) {
            obj_sum_kernel<<<1, 256, 0, s>>>(a.obj_partials, (int)(Pp / TC_BM), f_dev);
            NMF_LAUNCHED("obj_sum_kernel");
        }
    }
    return NMF_OK;
}

}  // namespace

nmf_status launch_mm_tc_obj(const float *A, int64_t m, int64_t n, int64_t lda, const float *F,
                            int k, int trans, float *out, const float *W, double *f_dev,
                            void *work, size_t work_bytes, cudaStream_t s)
{
    return launch_mm_tc_impl(A, m, n, lda, F, k, trans, out, W, f_dev, work, work_bytes, s,
                             nullptr, nullptr);
}

nmf_status launch_mm_tc(const float *A, int64_t m, int64_t n, int64_t lda, const float *F,
                        int k, int trans, float *out, void *work, size_t work_bytes,
                        cudaStream_t s)
{
    return launch_mm_tc_impl(A, m, n, lda, F, k, trans, out, nullptr, nullptr, work, work_bytes,
                             s, nullptr, nullptr);
}

size_t mm_tc_presplit_bytes(int64_t rows, int64_t K)
{
    return (size_t)(cdiv(rows, TC_BM) * TC_BM) * (size_t)(cdiv(K, TC_BK) * TC_BK) * 2;
}

nmf_status launch_mm_tc_presplit_make(const float *A, int64_t m, int64_t n, int64_t lda,
                                      int trans, void *hi, void *lo, cudaStream_t s)
{
    if (m == 0 || n == 0)
        return NMF_OK;
    const int64_t P = trans ? n : m, Q = trans ? m : n;
    const int64_t Pp = cdiv(P, TC_BM) * TC_BM, Qp = cdiv(Q, TC_BK) * TC_BK;
    unsigned char *h = static_cast<unsigned char *>(hi), *l = static_cast<unsigned char *>(lo);
    if (trans) {
        const dim3 grid((unsigned)cdiv(Pp, 64), (unsigned)cdiv(Qp, 64));
        if (grid.y > 65535u)
            return NMF_ERR_INVALID_ARG;
        mm_tc_presplit_kernel<<<grid, 256, 0, s>>>(A, m, n, lda, Qp, Pp, Qp / TC_BK, h, l);
        NMF_LAUNCHED("mm_tc_presplit_kernel");
    } else {
        if ((reinterpret_cast<uintptr_t>(A) & 15) || (lda % 4))
            return NMF_ERR_INVALID_ARG;
        const int64_t blocks = cdiv(Pp * (Qp / 8), 256);
        const int64_t cap = 16 * (int64_t)sm_count();
        mm_tc_presplit_rows_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(
            A, m, n, lda, Qp, Pp, Qp / TC_BK, h, l);
        NMF_LAUNCHED("mm_tc_presplit_rows_kernel");
    }
    return NMF_OK;
}

nmf_status launch_mm_tc_presplit(const void *hi, const void *lo, int64_t m, int64_t n,
                                 const float *F, int k, int trans, float *out, const float *W,
                                 double *f_dev, void *work, size_t work_bytes, cudaStream_t s)
{
    return launch_mm_tc_impl(nullptr, m, n, 0, F, k, trans, out, W, f_dev, work, work_bytes, s,
                             hi, lo);
}

}  // namespace nmf
