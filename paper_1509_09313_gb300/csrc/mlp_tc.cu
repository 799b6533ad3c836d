// Inference pass of the passive-set proposal network on the 5th-generation
// tensor cores: logits = relu(relu(F W1^T + b1) W2^T + b2) W3^T + b3, the same
// network as the SIMT kernels of mlp.cu (which keep the training passes).
//
// Weights are BF16 values already (the working copy is BF16-rounded), so each
// layer's B operand is exact in BF16. Each layer's input (the features, then
// the hidden activations) is FP32 and is carried as a BF16 pair hi + lo (hi =
// bf16(v), lo = bf16(v - hi), within 2^-17 |v| of v); a layer is
//   D = A_hi W^T + A_lo W^T        (two MMAs per 16-element step, FP32 in TMEM)
// so its products are those of FP32 arithmetic on 16-bit-mantissa inputs.
//
// Kernel (one layer per launch; persistent, one CTA per SM walking the 128-row
// tiles, so that a tile's epilogue overlaps the next tile's loads and MMAs):
//   warp 0     TMA producer: each K-block of 64 brings A_hi, A_lo (128 x 64
//              BF16 each) and W (N x 64 BF16) into a ring of up to 3 stages
//              (128-byte swizzle, K-major).
//   warp 1     allocates TMEM (two accumulators of N columns, used by
//              alternate tiles); one lane issues the MMAs (M = 128, N = the
//              layer's padded width, K = 16).
//   warps 2-5  epilogue, one row per thread (its TMEM lane): bias (staged in
//              shared memory), ReLU, then
//              either the next layer's hi / lo operand (zero-padded to a
//              multiple of 64 columns) or the logits and the proposed passive
//              set {i : logit_i > 0} as bitmask words.
// Every mbarrier wait is bounded (~2 s); on timeout the CTA leaves its loops,
// writes NaN logits, empty proposals and a zero next operand for its rows
// (a proposal only picks where BPP starts, so the solves stay correct), frees
// TMEM and returns.
//
// Roofline: HBM (each layer reads its hi / lo input once and writes the next;
// the weights come from L2), 4 K N flops per row per layer on the tensor cores.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace nmf {
namespace {

using namespace tc;

constexpr int ML_BM = 128;             // rows per CTA (MMA M)
constexpr int ML_BK = 64;              // K-block: 64 BF16 = one 128-byte row
constexpr int ML_MAX_N = 256;          // MMA N limit for M = 128
constexpr int ML_MAX_STAGES = 3;
constexpr int ML_THREADS = 192;
constexpr int ML_A_BYTES = ML_BM * ML_BK * 2;   // 16 KB per hi or lo tile

struct MlLayerArgs {
    int64_t rows;
    int nkb;                 // K-blocks of the input
    int n, np;               // output columns, padded to a multiple of 32 (MMA N)
    const float *bias;       // n
    int relu;
    __nv_bfloat16 *ohi, *olo;   // next operand (rows x ldo), or null
    int ldo;
    float *logits;           // rows x n, or null
    uint64_t *bits;          // rows x nwords, or null
    int nwords;
};

__host__ __device__ constexpr uint32_t ml_stage_bytes(int np) { return 2u * ML_A_BYTES + (uint32_t)np * 128u; }

__host__ __device__ inline int ml_stages(int nkb) { return nkb < ML_MAX_STAGES ? nkb : ML_MAX_STAGES; }

__global__ void __launch_bounds__(ML_THREADS, 1)
    mlp_tc_layer_kernel(const __grid_constant__ CUtensorMap tmAhi,
                        const __grid_constant__ CUtensorMap tmAlo,
                        const __grid_constant__ CUtensorMap tmW, const MlLayerArgs a)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = ml_stages(a.nkb);
    const uint32_t stage_bytes = ml_stage_bytes(a.np);
    const uint32_t bar0 = sbase + (uint32_t)S * stage_bytes;
    auto full = [&](int i) { return bar0 + 8u * i; };            // stage landed
    auto empty = [&](int i) { return bar0 + 8u * (S + i); };     // stage's MMAs done
    auto acc_full = [&](int b) { return bar0 + 8u * (2 * S + b); };      // tile's MMAs done
    auto acc_empty = [&](int b) { return bar0 + 8u * (2 * S + 2 + b); }; // accumulator read
    unsigned char *tail = smem + (size_t)S * stage_bytes + 8 * (2 * S + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tail);
    volatile int *abort = reinterpret_cast<volatile int *>(tail + 4);
    float *bias_s = reinterpret_cast<float *>(tail + 16);          // np floats
    // Two accumulators of np columns (ping-pong between tiles).
    const uint32_t tmem_cols = a.np <= 16 ? 32 : a.np <= 32 ? 64 : a.np <= 64 ? 128
                             : a.np <= 128 ? 256 : 512;
    const int64_t ntiles = (a.rows + ML_BM - 1) / ML_BM;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(full(i), 1);
            mbar_init(empty(i), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full(b), 1);
            mbar_init(acc_empty(b), 4);    // the four epilogue warps
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int c = threadIdx.x; c < a.np; c += blockDim.x)
        bias_s[c] = c < a.n ? a.bias[c] : 0.0f;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            int g = 0;   // K-blocks issued by this CTA (ring position)
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int kb = 0; kb < a.nkb; ++kb, ++g) {
                    const int s = g % S, u = g / S;
                    if (!mbar_wait(empty(s), (u & 1) ^ 1, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(full(s), stage_bytes);
                    const uint32_t dst = sbase + (uint32_t)s * stage_bytes;
                    tma_load_2d(dst, &tmAhi, kb * ML_BK, (int)(t * ML_BM), full(s));
                    tma_load_2d(dst + ML_A_BYTES, &tmAlo, kb * ML_BK, (int)(t * ML_BM), full(s));
                    tma_load_2d(dst + 2 * ML_A_BYTES, &tmW, kb * ML_BK, 0, full(s));
                }
            }
        }
    } else if (warp == 1) {
        // -------------------------------------------------------------- MMAs
        if (lane == 0) {
            // kind::f16, BF16 A and B (both K-major), FP32 D, M = 128, N = np.
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                   ((uint32_t)(a.np >> 3) << 17) | ((uint32_t)(ML_BM >> 4) << 24);
            const uint64_t d0 = sw128_desc(sbase);
            const uint64_t stage16 = (uint64_t)(stage_bytes >> 4);
            constexpr uint64_t A16 = (uint64_t)(ML_A_BYTES >> 4);
            int g = 0, j = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++j) {
                const int b = j & 1, ub = j >> 1;
                if (!mbar_wait_fast(acc_empty(b), (ub & 1) ^ 1, abort))
                    break;
                const uint32_t d = tmem + (uint32_t)(b * a.np);
                for (int kb = 0; kb < a.nkb; ++kb, ++g) {
                    const int s = g % S, u = g / S;
                    if (!mbar_wait_fast(full(s), u & 1, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ah = d0 + (uint64_t)s * stage16, al = ah + A16,
                                   w = ah + 2 * A16;
#pragma unroll
                    for (int kk = 0; kk < ML_BK / 16; ++kk) {
                        const uint64_t o = (uint64_t)(kk * 2);   // 16 BF16 = 32 bytes along K
                        mma_bf16(d, ah + o, w + o, idesc, (kb | kk) ? 1u : 0u);
                        mma_bf16(d, al + o, w + o, idesc, 1u);
                    }
                    mma_commit(empty(s));
                }
                if (ok)
                    mma_commit(acc_full(b));
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int quarter = warp & 3;            // TMEM lane quarter of this warp
        const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
        int j = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int b = j & 1, ub = j >> 1;
            const int64_t r = t * ML_BM + quarter * 32 + lane;
            // The TMEM loads below are warp-collective: the wait's outcome is
            // made the same for all 32 lanes.
            const bool ok = __all_sync(FULL, mbar_wait(acc_full(b), ub & 1, abort));
            if (!ok) {
                if (r < a.rows) {
                    if (a.ohi)
                        for (int c = 0; c < a.ldo; c += 8) {
                            *reinterpret_cast<uint4 *>(a.ohi + r * a.ldo + c) = make_uint4(0, 0, 0, 0);
                            *reinterpret_cast<uint4 *>(a.olo + r * a.ldo + c) = make_uint4(0, 0, 0, 0);
                        }
                    if (a.logits)
                        for (int c = 0; c < a.n; ++c)
                            a.logits[r * a.n + c] = __int_as_float(0x7fc00000);
                    if (a.bits)
                        for (int q = 0; q < a.nwords; ++q)
                            a.bits[r * a.nwords + q] = 0;
                }
                continue;
            }
            tc_fence_after();
            const uint32_t tb = tq + (uint32_t)(b * a.np);
            // Proposal words (k <= 256: at most four), kept in registers.
            uint64_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
            for (int c0 = 0; c0 < a.np; c0 += 32) {
                uint32_t raw[32];
                tmem_ld32_nowait(tb + (uint32_t)c0, raw);
                tmem_wait_ld();
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    float x = __uint_as_float(raw[i]) + bias_s[c0 + i];
                    if (a.relu)
                        x = fmaxf(x, 0.0f);
                    v[i] = c0 + i < a.n ? x : 0.0f;
                }
                if (r >= a.rows)
                    continue;
                if (a.ohi) {
                    __nv_bfloat16 *hrow = a.ohi + r * a.ldo + c0, *lrow = a.olo + r * a.ldo + c0;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        float v8[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            v8[i] = v[8 * g + i];
                        uint4 h, l;
                        split8(v8, h, l);
                        reinterpret_cast<uint4 *>(hrow)[g] = h;
                        reinterpret_cast<uint4 *>(lrow)[g] = l;
                    }
                }
                if (a.logits) {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (c0 + i < a.n)
                            a.logits[r * a.n + c0 + i] = v[i];
                }
                if (a.bits) {
                    uint32_t m = 0;
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        m |= (c0 + i < a.n && v[i] > 0.0f) ? (1u << i) : 0u;
                    const uint64_t mw = (uint64_t)m << (c0 & 32);
                    const int q = c0 >> 6;
                    w0 |= q == 0 ? mw : 0;
                    w1 |= q == 1 ? mw : 0;
                    w2 |= q == 2 ? mw : 0;
                    w3 |= q == 3 ? mw : 0;
                }
            }
            // The accumulator is free for the tile after next.
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(acc_empty(b));
            if (r < a.rows) {
                if (a.ohi) {
                    // Zero the padding columns [np, ldo) of the next operand.
                    const uint4 z = make_uint4(0, 0, 0, 0);
                    for (int c = a.np; c < a.ldo; c += 8) {
                        *reinterpret_cast<uint4 *>(a.ohi + r * a.ldo + c) = z;
                        *reinterpret_cast<uint4 *>(a.olo + r * a.ldo + c) = z;
                    }
                }
                if (a.bits) {
                    const uint64_t ws[4] = {w0, w1, w2, w3};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (q < a.nwords)
                            a.bits[r * a.nwords + q] = ws[q];
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tmem_cols)
                     : "memory");
    }
}

// src (rows x cols FP32, row stride cols) -> BF16 hi / lo (rows x ldd), 8
// columns per thread, in blocks: source column b bs + i (i < bs) goes to
// column b bd + i, every other column is zero (bs = bd = ldd: the plain
// zero-padded copy). lo may be null (hi only: for values that are BF16
// already).
__global__ void mlp_tc_split_kernel(const float *__restrict__ src, int64_t rows, int cols, int ldd,
                                    int bs, int bd, __nv_bfloat16 *__restrict__ hi,
                                    __nv_bfloat16 *__restrict__ lo)
{
    const int chunks = ldd / 8;
    const int64_t total = rows * chunks;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / chunks;
        const int c0 = (int)(e - r * chunks) * 8;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int d = c0 + i, b = d / bd, w = d - b * bd, sc = b * bs + w;
            v[i] = (w < bs && sc < cols) ? src[r * cols + sc] : 0.0f;
        }
        uint4 h, l;
        split8(v, h, l);
        *reinterpret_cast<uint4 *>(hi + r * ldd + c0) = h;
        if (lo)
            *reinterpret_cast<uint4 *>(lo + r * ldd + c0) = l;
    }
}

int pad(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

bool mlp_tc_supported(int k, int h)
{
    return k >= 1 && h >= 1 && pad(h, 32) <= ML_MAX_N && pad(k, 32) <= ML_MAX_N;
}

namespace {

// The layers' B operands in one buffer: W1 (nph x kp1, its columns in the
// features' three blocks), W2 (nph x kph), W3 (npk x kph), BF16, zero-padded.
struct MlWeights {
    int kpf, kp1, nph, kph, npk;
    size_t w1, w2, w3, total;   // byte offsets
};

MlWeights ml_weights(int k, int h)
{
    MlWeights w;
    w.kpf = pad(k, 16);
    w.kp1 = pad(3 * w.kpf, ML_BK);
    w.nph = pad(h, 32);
    w.kph = pad(w.nph, ML_BK);
    w.npk = pad(k, 32);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    w.w1 = 0;
    w.w2 = w.w1 + al(sizeof(__nv_bfloat16) * (size_t)w.nph * w.kp1);
    w.w3 = w.w2 + al(sizeof(__nv_bfloat16) * (size_t)w.nph * w.kph);
    w.total = w.w3 + al(sizeof(__nv_bfloat16) * (size_t)w.npk * w.kph);
    return w;
}

nmf_status split_rows(const float *src, int64_t rows, int cols, int prow, int ldd, int bs, int bd,
                      __nv_bfloat16 *hi, __nv_bfloat16 *lo, cudaStream_t s)
{
    if (prow > rows)   // zero rows past the matrix (padded output columns)
        NMF_CUDA(cudaMemsetAsync(hi + rows * ldd, 0,
                                 sizeof(__nv_bfloat16) * (size_t)(prow - rows) * ldd, s));
    const int64_t work = rows * (ldd / 8);
    const unsigned blocks = (unsigned)std::min<int64_t>(cdiv(work, 256), 8 * (int64_t)sm_count());
    mlp_tc_split_kernel<<<blocks, 256, 0, s>>>(src, rows, cols, ldd, bs, bd, hi, lo);
    NMF_LAUNCHED("mlp_tc_split_kernel");
    return NMF_OK;
}

}  // namespace

size_t mlp_tc_weights_bytes(int k, int h) { return ml_weights(k, h).total; }

nmf_status launch_mlp_tc_weights(int k, int h, const float *W1, const float *W2, const float *W3,
                                 void *dst, cudaStream_t s)
{
    if (!mlp_tc_supported(k, h))
        return NMF_ERR_INVALID_ARG;
    const MlWeights w = ml_weights(k, h);
    unsigned char *d = static_cast<unsigned char *>(dst);
    auto at = [&](size_t off) { return reinterpret_cast<__nv_bfloat16 *>(d + off); };
    NMF_TRY(split_rows(W1, h, 3 * k, w.nph, w.kp1, k, w.kpf, at(w.w1), nullptr, s));
    NMF_TRY(split_rows(W2, h, h, w.nph, w.kph, w.kph, w.kph, at(w.w2), nullptr, s));
    return split_rows(W3, k, h, w.npk, w.kph, w.kph, w.kph, at(w.w3), nullptr, s);
}

nmf_status launch_mlp_tc_forward(int k, int h, const void *wts, const float *b1, const float *b2,
                                 const float *b3, const float *F, const double *G, const float *B,
                                 const float *Xp, int64_t n, float *logits, uint64_t *bits,
                                 cudaStream_t s)
{
    if (!mlp_tc_supported(k, h) || n < 0 || n > INT32_MAX)
        return NMF_ERR_INVALID_ARG;
    if (n == 0)
        return NMF_OK;
    // Layer 1 reads the three blocks of the features (gradient, Gram
    // diagonal, previous iterate; k each) at columns [0, kpf), [kpf, 2 kpf),
    // [2 kpf, 3 kpf) of its operand, and W1's columns are placed to match.
    const int k1 = 3 * k, kpf = pad(k, 16), kp1 = pad(3 * kpf, ML_BK);
    const int nph = pad(h, 32), kph = pad(nph, ML_BK);   // hidden width, padded K of layers 2, 3
    const int npk = pad(k, 32);
    const int nwords = (k + 63) / 64;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t fbytes = al(sizeof(__nv_bfloat16) * (size_t)n * kp1);
    const size_t hbytes = al(sizeof(__nv_bfloat16) * (size_t)n * kph);
    const size_t total = 2 * fbytes + 4 * hbytes;
    struct Mem {
        void *p = nullptr;
        cudaStream_t s;
        ~Mem()
        {
            if (p)
                cudaFreeAsync(p, s);
        }
    } mem{nullptr, s};
    NMF_CUDA(cudaMallocAsync(&mem.p, total, s));
    char *p = static_cast<char *>(mem.p);
    auto take = [&](size_t b) {
        char *q = p;
        p += b;
        return reinterpret_cast<__nv_bfloat16 *>(q);
    };
    __nv_bfloat16 *fhi = take(fbytes), *flo = take(fbytes);
    __nv_bfloat16 *xhi = take(hbytes), *xlo = take(hbytes), *yhi = take(hbytes), *ylo = take(hbytes);
    const MlWeights wl = ml_weights(k, h);
    const unsigned char *wb = static_cast<const unsigned char *>(wts);
    const __nv_bfloat16 *w1 = reinterpret_cast<const __nv_bfloat16 *>(wb + wl.w1);
    const __nv_bfloat16 *w2 = reinterpret_cast<const __nv_bfloat16 *>(wb + wl.w2);
    const __nv_bfloat16 *w3 = reinterpret_cast<const __nv_bfloat16 *>(wb + wl.w3);

    // The features into hi / lo (the weights are converted already).
    if (F)
        NMF_TRY(split_rows(F, n, k1, (int)n, kp1, k, kpf, fhi, flo, s));
    else
        NMF_TRY(launch_mlp_features_split(G, B, Xp, n, k, kpf, kp1, fhi, flo, s));

    auto layer = [&](const __nv_bfloat16 *ahi, const __nv_bfloat16 *alo, int kp,
                     const __nv_bfloat16 *w, int nout, int np, const float *bias, int relu,
                     __nv_bfloat16 *ohi, __nv_bfloat16 *olo, int ldo, float *lg,
                     uint64_t *bt) -> nmf_status {
        CUtensorMap mh, ml, mw;
        if (!make_map_2d(&mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, ahi, (uint64_t)kp, (uint64_t)n,
                         (uint64_t)kp * 2, ML_BK, ML_BM, CU_TENSOR_MAP_SWIZZLE_128B) ||
            !make_map_2d(&ml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, alo, (uint64_t)kp, (uint64_t)n,
                         (uint64_t)kp * 2, ML_BK, ML_BM, CU_TENSOR_MAP_SWIZZLE_128B) ||
            !make_map_2d(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w, (uint64_t)kp, (uint64_t)np,
                         (uint64_t)kp * 2, ML_BK, (uint32_t)np, CU_TENSOR_MAP_SWIZZLE_128B))
            return NMF_ERR_CUDA;
        MlLayerArgs a;
        a.rows = n;
        a.nkb = kp / ML_BK;
        a.n = nout;
        a.np = np;
        a.bias = bias;
        a.relu = relu;
        a.ohi = ohi;
        a.olo = olo;
        a.ldo = ldo;
        a.logits = lg;
        a.bits = bt;
        a.nwords = nwords;
        // Stages, then (after up to 1023 bytes of alignment) the barriers, the
        // TMEM address, the abort flag and the bias.
        const size_t smem = (size_t)ml_stages(a.nkb) * ml_stage_bytes(np) + 1024 + 256 +
                            sizeof(float) * ML_MAX_N;
        static SmemOptIn opt_in;
        NMF_TRY(ensure_smem(mlp_tc_layer_kernel, opt_in, smem));
        // Persistent: one CTA per SM walks the 128-row tiles.
        const unsigned grid = (unsigned)std::min<int64_t>(cdiv(n, ML_BM), sm_count());
        mlp_tc_layer_kernel<<<grid, ML_THREADS, smem, s>>>(mh, ml, mw, a);
        NMF_LAUNCHED("mlp_tc_layer_kernel");
        return NMF_OK;
    };
    NMF_TRY(layer(fhi, flo, kp1, w1, h, nph, b1, 1, xhi, xlo, kph, nullptr, nullptr));
    NMF_TRY(layer(xhi, xlo, kph, w2, h, nph, b2, 1, yhi, ylo, kph, nullptr, nullptr));
    return layer(yhi, ylo, kph, w3, k, npk, b3, 0, nullptr, nullptr, 0, logits, bits);
}

}  // namespace nmf
