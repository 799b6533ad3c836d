// Group-tile pass of the FP32 batched BPP (Sec. 4.2) for the all-passive
// group, on the 5th-generation tensor cores (launch shape group = 2; the
// SIMT pass of bpp_group.cu is group = 1).
//
// Membership, outputs and the hand-over to the per-warp kernel are those of
// the SIMT pass: a right-hand side joins the group when its first candidate
// partition is U, all usable indices (a warm start covering U, or from the
// empty start every usable y_i = -g_i infeasible); for the group F = U and the
// factor is the inverse M = G_UU^{-1} the preparation holds, so
//     x0 = M g,   r = g - G x0 (on U),   x1 = x0 + M r,
// and x1 is kept where it passes the sign test. A member is marked
// GROUP_PENDING before its tile is solved and the mark is overwritten only by
// its solution, so anything this pass does not finish (including a wait that
// timed out) goes to the per-warp kernel.
//
// The three products run as tcgen05 MMAs (M = 128 right-hand sides, N = k
// padded to 16, K = 16) on BF16 splits, accumulated in FP32 in TMEM:
//   x0 = g M:   g = g_hi + g_lo, M = M_hi + M_lo   (3 MMAs per step)
//   G x0':      x0' = hi + lo of x0 (exact: the vector whose residual is
//               taken, and the one x1 is built on), G = G_hi + G_mid + G_lo
//               (5 MMAs per step; G is represented to 2^-24)
//   M r:        r = r_hi + r_lo, M 2-way (3 MMAs per step).
// M's 16-bit representation only slows the refinement's contraction (x1 -
// x* = (I - M'G)(x0' - x*) + O(FP32 rounding of r)), so x1 is within the FP32
// solve's cond(G) 6e-8 bound; the results are not bitwise those of the SIMT
// pass or of the per-warp kernel.
//
// Kernel: one persistent CTA per SM walking 128-right-hand-side tiles, 16
// warps. Warp 0 allocates TMEM (three accumulators of N columns); thread 0
// also issues each product's MMAs once all threads have written its A
// operand (mbarrier bar_a), and commits them to bar_d.
//   all warps  four threads per right-hand side (its TMEM lane), each with
//              a quarter of the 16-column chunks: membership, the A operands
//              (split in registers, stored in the canonical K-major
//              128-byte-swizzled layout), the masks, the sign test and the
//              outputs; per-row decisions combine the four threads' partial
//              results through shared memory (named barrier 1).
// M and G (split) stay in shared memory for the whole kernel. Every mbarrier
// wait is bounded (~2 s).
#include <math.h>

#include "bpp_internal.cuh"
#include "tc_ptx.cuh"

namespace nmf {
namespace bpp {
namespace {

using namespace tc;

constexpr int GC_BM = 128;         // right-hand sides per tile (MMA M)
constexpr int GC_PARTS = 4;        // threads per right-hand side
constexpr int GC_THREADS = GC_PARTS * GC_BM;   // 16 warps; thread 0 also issues the MMAs
constexpr int GC_MAX_K = 112;

template <int NP>   // k padded to 16: the MMA N and the columns of each accumulator
struct GcLayout {
    static constexpr int NKB = (NP + 63) / 64;       // K-blocks of 64 (K padded to 64 NKB)
    static constexpr int A_TILE = GC_BM * 128;       // 16 KB: 128 rows x 64 BF16
    static constexpr int B_TILE = NP * 128;          // NP rows x 64 BF16
    static constexpr int OFF_AHI = 0;
    static constexpr int OFF_ALO = NKB * A_TILE;
    static constexpr int OFF_B = 2 * NKB * A_TILE;   // M_hi, M_lo, G_hi, G_mid, G_lo
    static constexpr int PART = NKB * B_TILE;
    static constexpr int OFF_BAR = OFF_B + 5 * PART;
    static constexpr int OFF_TMEM = OFF_BAR + 16;
    static constexpr int OFF_ABORT = OFF_TMEM + 4;
    static constexpr int OFF_DSQ = OFF_BAR + 32;     // GC_MAX_K floats
    static constexpr int OFF_USE = OFF_DSQ + 4 * GC_MAX_K;
    static constexpr int OFF_XCH = (OFF_USE + GC_MAX_K + 15) & ~15;   // [part][row] int, float
    static constexpr int BYTES = OFF_XCH + 8 * GC_PARTS * GC_BM;
    static constexpr int TMEM_COLS = 3 * NP <= 64 ? 64 : 3 * NP <= 128 ? 128
                                   : 3 * NP <= 256 ? 256 : 512;
    static_assert(NP % 16 == 0 && NP <= GC_MAX_K, "MMA N");
    static_assert(B_TILE % 1024 == 0 && OFF_B % 1024 == 0, "128-byte-swizzled tiles");
    static_assert(BYTES + 1024 <= 227 * 1024, "shared memory budget");
};

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (no wait).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// v = hi + mid + lo to 2^-24 |v| (each step's remainder is exact in FP32).
__device__ __forceinline__ void split8_3(const float (&v)[8], uint4 &hi, uint4 &mid, uint4 &lo)
{
    uint32_t hw[4], mw[4], lw[4];
    const float2 neg1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 v2 = make_float2(v[2 * i], v[2 * i + 1]);
        const __nv_bfloat162 hb = __floats2bfloat162_rn(v2.x, v2.y);
        const float2 r1 = __ffma2_rn(__bfloat1622float2(hb), neg1, v2);   // exact
        const __nv_bfloat162 mb = __floats2bfloat162_rn(r1.x, r1.y);
        const float2 r2 = __ffma2_rn(__bfloat1622float2(mb), neg1, r1);   // exact
        const __nv_bfloat162 lb = __floats2bfloat162_rn(r2.x, r2.y);
        hw[i] = *reinterpret_cast<const uint32_t *>(&hb);
        mw[i] = *reinterpret_cast<const uint32_t *>(&mb);
        lw[i] = *reinterpret_cast<const uint32_t *>(&lb);
    }
    hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    mid = make_uint4(mw[0], mw[1], mw[2], mw[3]);
    lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// v = hi + lo within 2^-17 |v|; s = hi + lo (exact in FP32).
__device__ __forceinline__ void split8_sum(const float (&v)[8], uint4 &hi, uint4 &lo,
                                           float (&s)[8])
{
    uint32_t hw[4], lw[4];
    const float2 neg1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 v2 = make_float2(v[2 * i], v[2 * i + 1]);
        const __nv_bfloat162 hb = __floats2bfloat162_rn(v2.x, v2.y);
        const float2 hf = __bfloat1622float2(hb);
        const float2 d = __ffma2_rn(hf, neg1, v2);   // v - hi, exact
        const __nv_bfloat162 lb = __floats2bfloat162_rn(d.x, d.y);
        const float2 lf = __bfloat1622float2(lb);
        const float2 sm = __fadd2_rn(hf, lf);
        s[2 * i] = sm.x;
        s[2 * i + 1] = sm.y;
        hw[i] = *reinterpret_cast<const uint32_t *>(&hb);
        lw[i] = *reinterpret_cast<const uint32_t *>(&lb);
    }
    hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

template <int NP>
__global__ void __launch_bounds__(GC_THREADS, 1) bpp_group_tc_kernel(const SolveParams P)
{
    if (P.flags[0] != 0)
        return;   // not an FP32 half-step
    using L = GcLayout<NP>;
    constexpr int NKB = L::NKB;
    extern __shared__ unsigned char gc_smem_dyn[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(gc_smem_dyn) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int k = P.k;
    const uint32_t bar_a = sbase + L::OFF_BAR, bar_d = bar_a + 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::OFF_TMEM);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + L::OFF_ABORT);
    float *dsq = reinterpret_cast<float *>(smem + L::OFF_DSQ);
    unsigned char *use = smem + L::OFF_USE;

    int nU = 0;
    uint64_t umask[2] = {0ull, 0ull};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        nU += __popc(P.usable_words[q]);
        umask[q >> 1] |= (uint64_t)P.usable_words[q] << (32 * (q & 1));
    }
    if (tid == 0) {
        mbar_init(bar_a, GC_PARTS * GC_BM);   // the row threads
        mbar_init(bar_d, 1);     // the MMA commits
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < k; i += GC_THREADS) {
        const bool u = (P.usable_words[i >> 5] >> (i & 31)) & 1u;
        use[i] = u;
        dsq[i] = u ? sqrtf(P.G32[i * k + i]) : 1.0f;
    }
    // A operand tiles: zero (the columns past NP stay zero).
    for (int e = tid; e < 2 * NKB * L::A_TILE / 16; e += GC_THREADS)
        reinterpret_cast<uint4 *>(smem + L::OFF_AHI)[e] = make_uint4(0, 0, 0, 0);
    // B operands: row n (the output index i), 16-byte chunk c along K (the
    // contraction index j): M[n][j] 2-way, G[n][j] 3-way, zero past k.
    for (int e = tid; e < NP * NKB * 8; e += GC_THREADS) {
        const int n = e / (NKB * 8), c = e - n * (NKB * 8);
        float mv[8], gv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int j = 8 * c + t;
            const bool in = n < k && j < k;
            mv[t] = in ? P.M32[n * k + j] : 0.0f;
            gv[t] = in ? P.G32[n * k + j] : 0.0f;
        }
        uint4 mh, ml, gh, gm, gl;
        split8(mv, mh, ml);
        split8_3(gv, gh, gm, gl);
        const uint32_t off = (uint32_t)((c >> 3) * L::B_TILE) + sw128_off(n, c & 7);
        unsigned char *b = smem + L::OFF_B + off;
        *reinterpret_cast<uint4 *>(b) = mh;
        *reinterpret_cast<uint4 *>(b + L::PART) = ml;
        *reinterpret_cast<uint4 *>(b + 2 * L::PART) = gh;
        *reinterpret_cast<uint4 *>(b + 3 * L::PART) = gm;
        *reinterpret_cast<uint4 *>(b + 4 * L::PART) = gl;
    }
    fence_proxy_async();   // these writes are read by the tensor cores
    if (warp == 0) {
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
    const int64_t ntiles = cdiv(P.nrhs, (int64_t)GC_BM);

    // The MMAs of one product (thread 0, after the row threads' arrivals on
    // bar_a): x0 = g M (step 0), G x0' (1), M r (2), committed to bar_d.
    // kind::f16, BF16 A and B (both K-major), FP32 D, M = 128, N = NP.
    uint32_t ph_a = 0;
    auto issue = [&](int step) -> bool {
        if (!mbar_wait_fast(bar_a, ph_a & 1u, abort))
            return false;
        ++ph_a;
        tc_fence_after();
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(GC_BM >> 4) << 24);
        const uint64_t ahi = sw128_desc(sbase + L::OFF_AHI), alo = sw128_desc(sbase + L::OFF_ALO);
        const uint64_t b0 = sw128_desc(sbase + L::OFF_B);
        constexpr uint64_t A16 = (uint64_t)(L::A_TILE >> 4), B16 = (uint64_t)(L::B_TILE >> 4);
        constexpr uint64_t P16 = (uint64_t)(L::PART >> 4);
        const uint64_t mhi = b0, mlo = b0 + P16, ghi = b0 + 2 * P16, gmid = b0 + 3 * P16,
                       glo = b0 + 4 * P16;
        const uint32_t d = tmem + (uint32_t)(step * NP);
#pragma unroll
        for (int kb = 0; kb < NKB; ++kb)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t oa = kb * A16 + (uint64_t)(kk * 2);
                const uint64_t ob = kb * B16 + (uint64_t)(kk * 2);
                const uint32_t acc = (kb | kk) ? 1u : 0u;
                if (step != 1) {   // x0 = g M, then M r
                    mma_bf16(d, ahi + oa, mhi + ob, idesc, acc);
                    mma_bf16(d, ahi + oa, mlo + ob, idesc, 1u);
                    mma_bf16(d, alo + oa, mhi + ob, idesc, 1u);
                } else {           // G x0'
                    mma_bf16(d, ahi + oa, ghi + ob, idesc, acc);
                    mma_bf16(d, ahi + oa, gmid + ob, idesc, 1u);
                    mma_bf16(d, alo + oa, ghi + ob, idesc, 1u);
                    mma_bf16(d, ahi + oa, glo + ob, idesc, 1u);
                    mma_bf16(d, alo + oa, gmid + ob, idesc, 1u);
                }
            }
        mma_commit(bar_d);
        return true;
    };

    {
        // ------------------------------------------------ right-hand sides
        // Four threads per right-hand side (warps w and w + 4, w + 8, w + 12
        // share a TMEM lane quarter): part p takes the 16-column chunks p,
        // p + 4, ... of the row; per-row decisions combine the parts' partial
        // results through shared memory.
        const int quarter = warp & 3;            // TMEM lane quarter of this warp
        const int part = warp >> 2;              // 0..3
        const int rl = quarter * 32 + lane;      // row of the tile = TMEM lane
        const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
        constexpr int NCH = NP / 16;                       // 16-column chunks
        constexpr int MYCH = (NCH + GC_PARTS - 1) / GC_PARTS;   // chunks per part (at most)
        int *xok = reinterpret_cast<int *>(smem + L::OFF_XCH);        // [part][row]
        float *xmx = reinterpret_cast<float *>(smem + L::OFF_XCH + 4 * GC_PARTS * GC_BM);
        unsigned char *arow_hi = smem + L::OFF_AHI, *arow_lo = smem + L::OFF_ALO;
        auto put_a = [&](int c8, const uint4 &h, const uint4 &l) {
            const uint32_t off = (uint32_t)((c8 >> 3) * L::A_TILE) + sw128_off(rl, c8 & 7);
            *reinterpret_cast<uint4 *>(arow_hi + off) = h;
            *reinterpret_cast<uint4 *>(arow_lo + off) = l;
        };
        // This thread's usable columns, bit 16 m + i for column 16 (part + 4 m)
        // + i (formed once: the per-column tests below are one bit test).
        uint32_t mymask = 0;
#pragma unroll
        for (int m = 0; m < MYCH; ++m)
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = 16 * (part + GC_PARTS * m) + i;
                if (c < k && (((c < 64 ? umask[0] : umask[1]) >> (c & 63)) & 1ull))
                    mymask |= 1u << (16 * m + i);
            }
        auto use_mi = [&](int m, int i) { return (mymask >> (16 * m + i)) & 1u; };
        // The parts' partial results of one decision: AND of the flags, max of
        // the values (every part gets the same combined result).
        auto combine = [&](int okp, float vp, int &ok, float &v) {
            xok[part * GC_BM + rl] = okp;
            xmx[part * GC_BM + rl] = vp;
            asm volatile("bar.sync 1, %0;" ::"r"(GC_PARTS * GC_BM) : "memory");
            ok = 1;
            v = 0.0f;
#pragma unroll
            for (int q = 0; q < GC_PARTS; ++q) {
                ok &= xok[q * GC_BM + rl];
                v = fmaxf(v, xmx[q * GC_BM + rl]);
            }
            asm volatile("bar.sync 1, %0;" ::"r"(GC_PARTS * GC_BM) : "memory");
        };
        unsigned long long st_rhs = 0, st_rounds = 0, st_max = 0, st_nf = 0, pending = 0;
        uint32_t ph = 0;
        bool dead = false;   // a wait of this warp timed out: only mark from now on
        // Rows of B and X start on 16 bytes when k is a multiple of 4 (the
        // bases come from the allocator, 256-byte aligned, checked here).
        const bool vec4 = (k & 3) == 0 &&
                          ((reinterpret_cast<uintptr_t>(P.B) | reinterpret_cast<uintptr_t>(P.X)) & 15) == 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int64_t j = t * GC_BM + rl;
            const bool live = j < P.nrhs;
            // This part's columns of the right-hand side, in registers (16-byte
            // loads when the rows are 16-byte aligned: scalar loads flood the
            // load queue).
            float g[MYCH][16];
            {
                const float *row = P.B + (live ? j : 0) * k;
#pragma unroll
                for (int m = 0; m < MYCH; ++m)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = 16 * (part + GC_PARTS * m) + 4 * q;
                        if (vec4) {
                            const float4 v = live && c < k
                                                 ? *reinterpret_cast<const float4 *>(row + c)
                                                 : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                            g[m][4 * q] = v.x;
                            g[m][4 * q + 1] = v.y;
                            g[m][4 * q + 2] = v.z;
                            g[m][4 * q + 3] = v.w;
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                g[m][4 * q + i] = live && c + i < k ? row[c + i] : 0.0f;
                        }
                    }
            }
            // Membership: the first candidate partition is U (the test of the
            // SIMT pass and of the per-warp kernel, from the combined max).
            int member = 0;
            {
                int okp = 1;
                float gmp = 0.0f;
#pragma unroll
                for (int m = 0; m < MYCH; ++m)
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int c = 16 * (part + GC_PARTS * m) + i;
                        if (c < k) {
                            okp &= isfinite(g[m][i]) ? 1 : 0;
                            gmp = fmaxf(gmp, fabsf(g[m][i]) / dsq[c]);
                        }
                    }
                int ok;
                float gmax;
                combine(okp, gmp, ok, gmax);
                ok = ok && live && nU > 0;
                int inp = 1;
                if (ok) {
                    if (P.pin) {
                        if (part == 0)
                            for (int w = 0; w < P.nwords; ++w)
                                if ((P.pin[j * P.nwords + w] & umask[w]) != umask[w])
                                    inp = 0;
                    } else if (P.max_rounds >= 1) {
                        const float ytol = FEAS_TOL32 * gmax;
#pragma unroll
                        for (int m = 0; m < MYCH; ++m)
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int c = 16 * (part + GC_PARTS * m) + i;
                                if (use_mi(m, i) && !(-g[m][i] < -ytol * dsq[c]))
                                    inp = 0;
                            }
                    } else {
                        inp = 0;
                    }
                }
                int all_in;
                float unused;
                combine(inp, 0.0f, all_in, unused);
                member = ok && all_in;
            }
            if (member && part == 0)   // until its solution overwrites it
                reinterpret_cast<uint32_t *>(P.X)[j * k] = GROUP_PENDING;
            bool solved = false;
            if (!dead) {
                // Step 1: A = g.
#pragma unroll
                for (int m = 0; m < MYCH; ++m) {
                    const int c16 = part + GC_PARTS * m;
                    if (c16 < NCH)
#pragma unroll
                        for (int h8 = 0; h8 < 2; ++h8) {
                            float v[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                v[i] = member ? g[m][8 * h8 + i] : 0.0f;
                            uint4 h, l;
                            split8(v, h, l);
                            put_a(2 * c16 + h8, h, l);
                        }
                }
                fence_proxy_async();
                tc_fence_before();
                mbar_arrive(bar_a);
                if (tid == 0)
                    issue(0);
                // Step 2: x0 (masked to U) -> x0' = hi + lo, back into its
                // accumulator columns and into A.
                dead = !__all_sync(FULL, mbar_wait(bar_d, ph & 1u, abort));
                ++ph;
            }
            if (!dead) {
                tc_fence_after();
#pragma unroll
                for (int m = 0; m < MYCH; ++m) {
                    const int c16 = part + GC_PARTS * m;
                    if (c16 >= NCH)
                        continue;   // warp-uniform
                    uint32_t raw[16];
                    tmem_ld16_nowait(tq + (uint32_t)(16 * c16), raw);
                    tmem_wait_ld();
#pragma unroll
                    for (int h8 = 0; h8 < 2; ++h8) {
                        float v[8], sm[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int c = 16 * c16 + 8 * h8 + i;
                            v[i] = use_mi(m, 8 * h8 + i) ? __uint_as_float(raw[8 * h8 + i]) + 0.0f
                                                         : 0.0f;
                        }
                        uint4 h, l;
                        split8_sum(v, h, l, sm);
                        put_a(2 * c16 + h8, h, l);
                        tmem_st8(tq + (uint32_t)(16 * c16 + 8 * h8), sm);
                    }
                }
                tmem_wait_st();
                fence_proxy_async();
                tc_fence_before();
                mbar_arrive(bar_a);
                if (tid == 0)
                    issue(1);
                // Step 3: r = g - G x0' on U.
                dead = !__all_sync(FULL, mbar_wait(bar_d, ph & 1u, abort));
                ++ph;
            }
            if (!dead) {
                tc_fence_after();
#pragma unroll
                for (int m = 0; m < MYCH; ++m) {
                    const int c16 = part + GC_PARTS * m;
                    if (c16 >= NCH)
                        continue;
                    uint32_t raw[16];
                    tmem_ld16_nowait(tq + (uint32_t)(NP + 16 * c16), raw);
                    tmem_wait_ld();
#pragma unroll
                    for (int h8 = 0; h8 < 2; ++h8) {
                        float v[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int c = 16 * c16 + 8 * h8 + i;
                            v[i] = member && use_mi(m, 8 * h8 + i)
                                       ? g[m][8 * h8 + i] - __uint_as_float(raw[8 * h8 + i])
                                       : 0.0f;
                        }
                        uint4 h, l;
                        split8(v, h, l);
                        put_a(2 * c16 + h8, h, l);
                    }
                }
                fence_proxy_async();
                tc_fence_before();
                mbar_arrive(bar_a);
                if (tid == 0)
                    issue(2);
                // Step 4: x1 = x0' + M r, the sign test, the outputs.
                dead = !__all_sync(FULL, mbar_wait(bar_d, ph & 1u, abort));
                ++ph;
            }
            // The combines below are block-level (named barrier): every part
            // takes part in them, dead or not.
            float x1[MYCH][16];
            float xmp = 0.0f;
            if (!dead) {
                tc_fence_after();
#pragma unroll
                for (int m = 0; m < MYCH; ++m) {
                    const int c16 = part + GC_PARTS * m;
                    if (c16 >= NCH) {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            x1[m][i] = 0.0f;
                        continue;
                    }
                    uint32_t a0[16], a2[16];
                    tmem_ld16_nowait(tq + (uint32_t)(16 * c16), a0);
                    tmem_ld16_nowait(tq + (uint32_t)(2 * NP + 16 * c16), a2);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int c = 16 * c16 + i;
                        const float x = use_mi(m, i)
                                            ? __uint_as_float(a0[i]) + (__uint_as_float(a2[i]) + 0.0f)
                                            : 0.0f;
                        x1[m][i] = x;
                        if (use_mi(m, i))
                            xmp = fmaxf(xmp, fabsf(x) * dsq[c]);
                    }
                }
                tc_fence_before();   // the accumulators are read before the next tile's MMAs
            } else {
#pragma unroll
                for (int m = 0; m < MYCH; ++m)
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        x1[m][i] = 0.0f;
            }
            int okall;
            float xm;
            combine(dead ? 0 : 1, xmp, okall, xm);
            const float xtol = FEAS_TOL32 * xm;
            int feasp = 1, finp = 1;
#pragma unroll
            for (int m = 0; m < MYCH; ++m)
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = 16 * (part + GC_PARTS * m) + i;
                    if (use_mi(m, i) && x1[m][i] * dsq[c] < -xtol)
                        feasp = 0;
                    if (c < k && !isfinite(x1[m][i] > 0.0f ? x1[m][i] : 0.0f))
                        finp = 0;
                }
            int feasible;
            float fin_f;
            combine(feasp, finp ? 0.0f : 1.0f, feasible, fin_f);
            const bool keep = okall && member && feasible;
            if (keep) {
                float *xr = P.X + j * k;
#pragma unroll
                for (int m = 0; m < MYCH; ++m)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = 16 * (part + GC_PARTS * m) + 4 * q;
                        float v[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            v[i] = x1[m][4 * q + i] > 0.0f ? x1[m][4 * q + i] : 0.0f;
                        if (vec4) {
                            if (c < k)
                                *reinterpret_cast<float4 *>(xr + c) = make_float4(v[0], v[1], v[2], v[3]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (c + i < k)
                                    xr[c + i] = v[i];
                        }
                    }
                if (part == 0) {
                    const bool fin = fin_f == 0.0f;
                    const int rounds = P.pin ? 0 : 1;
                    if (P.pout)
                        for (int w = 0; w < P.nwords; ++w)
                            P.pout[j * P.nwords + w] = umask[w];
                    if (P.rounds_out)
                        P.rounds_out[j] = rounds;
                    if (P.status_out)
                        P.status_out[j] = (int8_t)(fin ? NMF_OK : NMF_ERR_NONFINITE);
                    st_rhs += 1;
                    st_rounds += rounds;
                    if ((unsigned long long)rounds > st_max)
                        st_max = (unsigned long long)rounds;
                    st_nf += fin ? 0 : 1;
                }
                solved = true;
            }
            // Members not solved keep their mark.
            if (part == 0 && live && !solved)
                pending += 1;
        }
        for (int o = 16; o > 0; o >>= 1) {
            pending += __shfl_xor_sync(FULL, pending, o);
            st_rhs += __shfl_xor_sync(FULL, st_rhs, o);
            st_rounds += __shfl_xor_sync(FULL, st_rounds, o);
            st_max = max(st_max, __shfl_xor_sync(FULL, st_max, o));
            st_nf += __shfl_xor_sync(FULL, st_nf, o);
        }
        if (lane == 0) {
            if (pending)
                atomicAdd(&P.counters[CNT_PENDING], pending);
            if (st_rhs) {
                atomicAdd(&P.stats->rhs, st_rhs);
                atomicAdd(&P.stats->rounds, st_rounds);
                atomicMax(&P.stats->max_rounds, st_max);
                if (st_nf)
                    atomicAdd(&P.stats->nonfinite, st_nf);
            }
        }
    }


    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)L::TMEM_COLS)
                     : "memory");
    }
}

template <int NP>
nmf_status launch_np(const SolveParams &P, cudaStream_t s)
{
    using L = GcLayout<NP>;
    const size_t smem = (size_t)L::BYTES + 1024;
    static SmemOptIn opt_in;
    NMF_TRY(ensure_smem(bpp_group_tc_kernel<NP>, opt_in, smem));
    const int64_t ntiles = cdiv(P.nrhs, (int64_t)GC_BM);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles < 1 ? 1 : ntiles, sm_count());
    bpp_group_tc_kernel<NP><<<grid, GC_THREADS, smem, s>>>(P);
    NMF_LAUNCHED("bpp_group_tc_kernel");
    return NMF_OK;
}

}  // namespace

bool group_tc_supported(int k) { return k >= 1 && k <= GC_MAX_K; }

nmf_status launch_group_tc(const SolveParams &P, cudaStream_t s)
{
    switch ((P.k + 15) / 16) {
    case 1: return launch_np<16>(P, s);
    case 2: return launch_np<32>(P, s);
    case 3: return launch_np<48>(P, s);
    case 4: return launch_np<64>(P, s);
    case 5: return launch_np<80>(P, s);
    case 6: return launch_np<96>(P, s);
    case 7: return launch_np<112>(P, s);
    default: return NMF_ERR_INVALID_ARG;
    }
}

}  // namespace bpp
}  // namespace nmf
