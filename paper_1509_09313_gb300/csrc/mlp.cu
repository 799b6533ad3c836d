// Learned passive-set proposal for block principal pivoting (no counterpart in
// the paper: it only picks the starting partition of the BPP solves of Eq. 3,
// Sec. 4.2, which then run to the KKT point of Eq. 4 as before, so every
// answer is unchanged and BPP's own tests decide on every proposal).
//
// Per right-hand side (G, g, x_p = the previous iterate of that factor row):
//   d_i = sqrt(G_ii) (1 where G_ii <= 0), s = max_i |g_i| / d_i (1 if 0),
//   features = [ (G x_p - g)_i / (d_i s), log(G_ii / mean G_jj), x_p,i d_i / s ]
// (gradient, Gram diagonal, previous iterate in the diagonally scaled
// variables); a 3k -> h -> h -> k ReLU network with BF16-rounded weights and
// FP32 arithmetic proposes passive set {i : logit_i > 0}. Training: mean
// binary cross-entropy against the solve's final passive set, Adam (0.9,
// 0.999, 1e-8) on FP32 master weights.
//
// Kernels (SIMT FP32; the inference pass runs on the tensor cores instead,
// mlp_tc.cu, when k and h are at most 256):
//   mlp_features_kernel  one warp per right-hand side, G in shared memory;
//                        G x_p by shared-memory broadcast (as in the BPP solve).
//   mlp_gemm_kernel      C = op(A) op(B) tiled 64 x 64 x 16, 4 x 4 per thread,
//                        optional ReLU on either operand as loaded, bias and
//                        ReLU-mask epilogues, deterministic split-K (partials
//                        summed in a fixed order by mlp_sum_splits_kernel).
//   mlp_bce_kernel       d loss / d logits and the loss (FP64 block partials).
//   mlp_adam_kernel      Adam on the master weights, then the BF16-rounded
//                        working copy.
//   mlp_propose_kernel   logits > 0 -> passive bitmask.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nmf {
namespace {

constexpr int MLP_BM = 64, MLP_BN = 64, MLP_BK = 16;
constexpr int MLP_THREADS = 256;
constexpr int MLP_MAX_SPLITS = 32;
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;

// -------------------------------------------------------------- features
// SPLIT: instead of Fout, the BF16 hi / lo pair the tensor-core layers read
// (hi = bf16(v), lo = bf16(v - hi)): row j of hi and lo (ldd columns) holds
// the three blocks of the features at columns [0, kpf), [kpf, 2 kpf),
// [2 kpf, 3 kpf), zero-padded.
constexpr int FEAT_R = 4;   // right-hand sides per pass of a warp

template <int KW, bool SPLIT>
__global__ void __launch_bounds__(256)
    mlp_features_kernel(const double *__restrict__ G, const float *__restrict__ B,
                        const float *__restrict__ Xp, int64_t nrhs, int k,
                        float *__restrict__ Fout, int kpf, int ldd,
                        __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo)
{
    extern __shared__ float sh[];
    float *Gs = sh;                              // k x k
    float *stage_all = Gs + ((k * k + 3) & ~3);  // 8 warps x FEAT_R x 32 KW (16-byte aligned)
    __shared__ float s_mean;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x)
        Gs[e] = (float)G[e];
    if (threadIdx.x == 0) {
        double sum = 0.0;
        int cnt = 0;
        for (int i = 0; i < k; ++i)
            if (G[i * k + i] > 0.0) {
                sum += G[i * k + i];
                ++cnt;
            }
        s_mean = cnt ? (float)(sum / cnt) : 1.0f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *stage = stage_all + warp * FEAT_R * 32 * KW;
    float d[KW], rd[KW], logd[KW];
#pragma unroll
    for (int s = 0; s < KW; ++s) {
        const int i = lane + 32 * s;
        const float gii = i < k ? Gs[i * k + i] : 0.0f;
        d[s] = gii > 0.0f ? sqrtf(gii) : 1.0f;
        rd[s] = 1.0f / d[s];
        logd[s] = gii > 0.0f ? logf(gii / s_mean) : 0.0f;
    }
    // FEAT_R right-hand sides per pass of a warp: the row of G read for index
    // c serves all of them (one shared-memory load per FEAT_R FMAs instead of
    // one per FMA); each right-hand side's sums run in the same order as one
    // at a time.
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * FEAT_R; j0 < nrhs;
         j0 += nw * FEAT_R) {
        float g[FEAT_R][KW], x[FEAT_R][KW], y[FEAT_R][KW], sc[FEAT_R];
#pragma unroll
        for (int r = 0; r < FEAT_R; ++r) {
            const int64_t j = j0 + r;
            const bool live = j < nrhs;
            float smax = 0.0f;
#pragma unroll
            for (int s = 0; s < KW; ++s) {
                const int i = lane + 32 * s;
                g[r][s] = live && i < k ? B[j * k + i] : 0.0f;
                x[r][s] = (live && i < k && Xp) ? Xp[j * k + i] : 0.0f;
                y[r][s] = -g[r][s];
                smax = fmaxf(smax, fabsf(g[r][s]) * rd[s]);
            }
            for (int o = 16; o > 0; o >>= 1)
                smax = fmaxf(smax, __shfl_xor_sync(FULL, smax, o));
            sc[r] = smax > 0.0f ? 1.0f / smax : 1.0f;
            // y = G x - g (G symmetric), x staged in shared memory and read by broadcast.
#pragma unroll
            for (int s = 0; s < KW; ++s)
                stage[(r * KW + s) * 32 + lane] = x[r][s];
        }
        __syncwarp();
        // x_c of right-hand side r sits at stage[r 32 KW + c]: four of them
        // per vector load. Rows of G past k are never read; lanes past k
        // accumulate zeros.
        int c = 0;
        for (; c + 4 <= k; c += 4) {
            float rv[4][KW];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int s = 0; s < KW; ++s) {
                    const int i = lane + 32 * s;
                    rv[q][s] = i < k ? Gs[(c + q) * k + i] : 0.0f;
                }
#pragma unroll
            for (int r = 0; r < FEAT_R; ++r) {
                const float4 xv = *reinterpret_cast<const float4 *>(stage + r * 32 * KW + c);
                const float xq[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if constexpr (KW == 1) {
                        y[r][0] = fmaf(rv[q][0], xq[q], y[r][0]);
                    } else {
#pragma unroll
                        for (int s = 0; s < KW; s += 2) {
                            const float2 t = __ffma2_rn(make_float2(rv[q][s], rv[q][s + 1]),
                                                        make_float2(xq[q], xq[q]),
                                                        make_float2(y[r][s], y[r][s + 1]));
                            y[r][s] = t.x;
                            y[r][s + 1] = t.y;
                        }
                    }
                }
            }
        }
        for (; c < k; ++c) {
            const float *row = Gs + c * k;
            float rv[KW];
#pragma unroll
            for (int s = 0; s < KW; ++s) {
                const int i = lane + 32 * s;
                rv[s] = i < k ? row[i] : 0.0f;
            }
#pragma unroll
            for (int r = 0; r < FEAT_R; ++r) {
                const float xc = stage[r * 32 * KW + c];
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    y[r][s] = fmaf(rv[s], xc, y[r][s]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < FEAT_R; ++r) {
            const int64_t j = j0 + r;
            if (j >= nrhs)
                break;
            if (!SPLIT) {
                float *f = Fout + j * (3 * k);
#pragma unroll
                for (int s = 0; s < KW; ++s) {
                    const int i = lane + 32 * s;
                    if (i < k) {
                        f[i] = y[r][s] * rd[s] * sc[r];
                        f[k + i] = logd[s];
                        f[2 * k + i] = x[r][s] * d[s] * sc[r];
                    }
                }
            } else {
                __nv_bfloat16 *hr = hi + j * ldd, *lr = lo + j * ldd;
                auto put = [&](int c, float v) {
                    const __nv_bfloat16 h = __float2bfloat16_rn(v);
                    hr[c] = h;
                    lr[c] = __float2bfloat16_rn(fmaf(__bfloat162float(h), -1.0f, v));
                };
#pragma unroll
                for (int s = 0; s < KW; ++s) {
                    const int i = lane + 32 * s;
                    if (i < k) {
                        put(i, y[r][s] * rd[s] * sc[r]);
                        put(kpf + i, logd[s]);
                        put(2 * kpf + i, x[r][s] * d[s] * sc[r]);
                    }
                }
                // Zero columns: [k, kpf) of each block, and [3 kpf, ldd).
                const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
                for (int c = k + lane; c < kpf; c += 32)
                    for (int b = 0; b < 3; ++b) {
                        hr[b * kpf + c] = z;
                        lr[b * kpf + c] = z;
                    }
                for (int c = 3 * kpf + lane; c < ldd; c += 32) {
                    hr[c] = z;
                    lr[c] = z;
                }
            }
        }
    }
}


// -------------------------------------------------------------------- GEMM
// C[z][i][j] = sum_{l in split z} opA(i, l) opB(l, j) (+ bias[j]); then, with
// mask, C = (mask[i][j] > 0) ? C : 0. opA(i, l) = TA ? A[l lda + i] : A[i lda + l],
// opB(l, j) = TB ? B[j ldb + l] : B[l ldb + j], each passed through ReLU as
// loaded when RELU_A / RELU_B.
template <bool TA, bool TB, bool RELU_A, bool RELU_B>
__global__ void __launch_bounds__(MLP_THREADS)
    mlp_gemm_kernel(int M, int N, int K, int kchunk, const float *__restrict__ A, int lda,
                    const float *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                    int64_t split_stride, const float *__restrict__ bias,
                    const float *__restrict__ mask, int ldm)
{
    __shared__ float As[MLP_BK][MLP_BM + 4];
    __shared__ float Bs[MLP_BK][MLP_BN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * MLP_BM, n0 = blockIdx.x * MLP_BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            acc[a][b] = 0.0f;
    for (int k0 = kbeg; k0 < kend; k0 += MLP_BK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + MLP_THREADS * r;     // 0..1023
            int i, l;
            if (TA) {
                i = e % MLP_BM;
                l = e / MLP_BM;
            } else {
                l = e % MLP_BK;
                i = e / MLP_BK;
            }
            const int gi = m0 + i, gl = k0 + l;
            float v = 0.0f;
            if (gi < M && gl < kend)
                v = TA ? A[(int64_t)gl * lda + gi] : A[(int64_t)gi * lda + gl];
            if (RELU_A)
                v = fmaxf(v, 0.0f);
            As[l][i] = v;
            int j, l2;
            if (TB) {
                l2 = e % MLP_BK;
                j = e / MLP_BK;
            } else {
                j = e % MLP_BN;
                l2 = e / MLP_BN;
            }
            const int gj = n0 + j, gl2 = k0 + l2;
            float w = 0.0f;
            if (gj < N && gl2 < kend)
                w = TB ? B[(int64_t)gj * ldb + gl2] : B[(int64_t)gl2 * ldb + gj];
            if (RELU_B)
                w = fmaxf(w, 0.0f);
            Bs[l2][j] = w;
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < MLP_BK; ++l) {
            float av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
                av[a] = As[l][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b)
                bv[b] = Bs[l][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    float *Cz = C + (int64_t)blockIdx.z * split_stride;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = m0 + ty * 4 + a;
        if (i >= M)
            continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = n0 + tx * 4 + b;
            if (j >= N)
                continue;
            float v = acc[a][b];
            if (bias)
                v += bias[j];
            if (mask && !(mask[(int64_t)i * ldm + j] > 0.0f))
                v = 0.0f;
            Cz[(int64_t)i * ldc + j] = v;
        }
    }
}

__global__ void mlp_sum_splits_kernel(const float *__restrict__ part, int splits, int64_t count,
                                      float *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count)
        return;
    float s = 0.0f;
    for (int z = 0; z < splits; ++z)
        s += part[(int64_t)z * count + e];
    out[e] = s;
}

// ---------------------------------------------------------- loss, gradients
// dZ = (sigmoid(z) - y) / (nrhs k); loss partial per block (FP64).
__global__ void mlp_bce_kernel(const float *__restrict__ logits, const uint64_t *__restrict__ lab,
                               int64_t nrhs, int k, int nwords, float *__restrict__ dz,
                               double *__restrict__ loss_part)
{
    __shared__ double red[8];
    const int64_t n = nrhs * k;
    const float inv = 1.0f / (float)n;
    double part = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int i = (int)(e % k);
        const float y = (float)((lab[r * nwords + (i >> 6)] >> (i & 63)) & 1ull);
        const float z = logits[e];
        const float sg = 1.0f / (1.0f + expf(-z));
        dz[e] = (sg - y) * inv;
        part += (double)(fmaxf(z, 0.0f) - z * y + log1pf(expf(-fabsf(z))));
    }
    for (int o = 16; o > 0; o >>= 1)
        part += __shfl_xor_sync(FULL, part, o);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            s += red[w];
        loss_part[blockIdx.x] = s;
    }
}

__global__ void mlp_fill_kernel(float *__restrict__ x, int64_t n, float v)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n)
        x[e] = v;
}

__global__ void mlp_loss_sum_kernel(const double *__restrict__ part, int n, int64_t count,
                                    double *__restrict__ loss)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            s += part[i];
        *loss = s / (double)count;
    }
}

__device__ __forceinline__ float bf16_round(float x)
{
    return __bfloat162float(__float2bfloat16_rn(x));
}

__global__ void mlp_adam_kernel(float *__restrict__ master, float *__restrict__ work,
                                float *__restrict__ m, float *__restrict__ v,
                                const float *__restrict__ g, int64_t n, float lr, float bc1,
                                float bc2)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n)
        return;
    const float ge = g[e];
    const float me = ADAM_B1 * m[e] + (1.0f - ADAM_B1) * ge;
    const float ve = ADAM_B2 * v[e] + (1.0f - ADAM_B2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    const float p = master[e] - lr * (me / bc1) / (sqrtf(ve / bc2) + ADAM_EPS);
    master[e] = p;
    work[e] = bf16_round(p);
}

__global__ void mlp_round_kernel(const float *__restrict__ master, float *__restrict__ work,
                                 int64_t n)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n)
        work[e] = bf16_round(master[e]);
}

__global__ void mlp_propose_kernel(const float *__restrict__ logits, int64_t nrhs, int k,
                                   int nwords, uint64_t *__restrict__ out)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nrhs * nwords)
        return;
    const int64_t r = w / nwords;
    const int q = (int)(w % nwords);
    uint64_t bitsv = 0;
    for (int b = 0; b < 64; ++b) {
        const int i = q * 64 + b;
        if (i < k && logits[r * k + i] > 0.0f)
            bitsv |= 1ull << b;
    }
    out[w] = bitsv;
}

template <bool TA, bool TB, bool RELU_A, bool RELU_B>
nmf_status gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C,
                int ldc, const float *bias, const float *mask, int ldm, float *split_buf,
                cudaStream_t s)
{
    if (M <= 0 || N <= 0)
        return NMF_OK;
    const int gx = (N + MLP_BN - 1) / MLP_BN, gy = (M + MLP_BM - 1) / MLP_BM;
    // Split the contraction when the output tiles alone leave most SMs idle.
    int splits = 1;
    if (split_buf && !bias && !mask) {
        const int tiles = gx * gy;
        while (splits < MLP_MAX_SPLITS && tiles * splits < 2 * sm_count() &&
               K / (splits * 2) >= 4 * MLP_BK)
            splits *= 2;
    }
    const int kchunk = ((K + splits - 1) / splits + MLP_BK - 1) / MLP_BK * MLP_BK;
    splits = K > 0 ? (K + kchunk - 1) / kchunk : 1;
    float *dst = splits > 1 ? split_buf : C;
    const int64_t stride = (int64_t)M * ldc;
    mlp_gemm_kernel<TA, TB, RELU_A, RELU_B><<<dim3(gx, gy, splits), MLP_THREADS, 0, s>>>(
        M, N, K, kchunk, A, lda, B, ldb, dst, ldc, stride, bias, mask, ldm);
    NMF_LAUNCHED("mlp_gemm_kernel");
    if (splits > 1) {
        const int64_t count = stride;
        mlp_sum_splits_kernel<<<(unsigned)cdiv(count, 256), 256, 0, s>>>(split_buf, splits,
                                                                          count, C);
        NMF_LAUNCHED("mlp_sum_splits_kernel");
    }
    return NMF_OK;
}

}  // namespace

// ------------------------------------------------------------ the network
struct MlpNet {
    int k, h;
    int64_t nparams;
    int64_t off[6];          // W1, b1, W2, b2, W3, b3 in the flat arrays
    float *master = nullptr, *work = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    int64_t t = 0;           // Adam steps taken
    // The tensor-core layers' BF16 weights, converted from `work` after Adam
    // step tcw_t (-1: not yet).
    void *tcw = nullptr;
    int64_t tcw_t = -1;
};

int64_t mlp_param_count(int k, int h)
{
    return (int64_t)h * 3 * k + h + (int64_t)h * h + h + (int64_t)k * h + k;
}

namespace {

nmf_status launch_features(const double *G, const float *B, const float *Xp, int64_t nrhs, int k,
                           float *F, cudaStream_t s)
{
    if (nrhs == 0)
        return NMF_OK;
    const int kw = (k + 31) / 32;
    const size_t smem = sizeof(float) * ((size_t)((k * k + 3) & ~3) + 8 * FEAT_R * 32 * kw);
    const unsigned blocks = (unsigned)std::min<int64_t>(cdiv(nrhs, 8 * FEAT_R), 4 * sm_count());
    auto go = [&](auto kern) -> nmf_status {
        if (smem > 48 * 1024)
            NMF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        kern<<<blocks, 256, smem, s>>>(G, B, Xp, nrhs, k, F, 0, 0, nullptr, nullptr);
        NMF_LAUNCHED("mlp_features_kernel");
        return NMF_OK;
    };
    if (kw == 1)
        return go(mlp_features_kernel<1, false>);
    if (kw == 2)
        return go(mlp_features_kernel<2, false>);
    if (kw == 3)
        return go(mlp_features_kernel<3, false>);
    return go(mlp_features_kernel<4, false>);
}

// Activation buffers of one batch: z1, z2 (n x h), logits (n x k), and the
// backward's dZ buffers, a column of ones (bias gradients are dZ^T 1) and a
// split-K buffer.
struct Acts {
    float *z1, *z2, *logit, *dz3, *dz2, *dz1, *ones, *split;
    double *loss_part, *loss;
    size_t bytes;
};

size_t acts_bytes(const MlpNet &net, int64_t n, bool train)
{
    const size_t nh = (size_t)n * net.h, nk = (size_t)n * net.k;
    size_t b = sizeof(float) * (2 * nh + nk);
    if (train)
        b += sizeof(float) * (nk + 2 * nh + n) +
             sizeof(float) * (size_t)MLP_MAX_SPLITS * net.h * std::max(3 * net.k, net.h) +
             sizeof(double) * 1025;
    return b + 256 * 8;
}

Acts carve(const MlpNet &net, int64_t n, bool train, void *mem)
{
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *p = static_cast<char *>(mem);
    const size_t nh = (size_t)n * net.h, nk = (size_t)n * net.k;
    Acts a{};
    a.z1 = reinterpret_cast<float *>(p); p += al(sizeof(float) * nh);
    a.z2 = reinterpret_cast<float *>(p); p += al(sizeof(float) * nh);
    a.logit = reinterpret_cast<float *>(p); p += al(sizeof(float) * nk);
    if (train) {
        a.dz3 = reinterpret_cast<float *>(p); p += al(sizeof(float) * nk);
        a.dz2 = reinterpret_cast<float *>(p); p += al(sizeof(float) * nh);
        a.dz1 = reinterpret_cast<float *>(p); p += al(sizeof(float) * nh);
        a.ones = reinterpret_cast<float *>(p); p += al(sizeof(float) * (size_t)n);
        a.split = reinterpret_cast<float *>(p);
        p += al(sizeof(float) * (size_t)MLP_MAX_SPLITS * net.h * std::max(3 * net.k, net.h));
        a.loss_part = reinterpret_cast<double *>(p); p += al(sizeof(double) * 1024);
        a.loss = reinterpret_cast<double *>(p); p += al(sizeof(double));
    }
    a.bytes = (size_t)(p - static_cast<char *>(mem));
    return a;
}

nmf_status forward(const MlpNet &net, const float *F, int64_t n, const Acts &a, cudaStream_t s)
{
    const int k = net.k, h = net.h, ki = 3 * k;
    const float *W1 = net.work + net.off[0], *b1 = net.work + net.off[1];
    const float *W2 = net.work + net.off[2], *b2 = net.work + net.off[3];
    const float *W3 = net.work + net.off[4], *b3 = net.work + net.off[5];
    // z1 = F W1^T + b1; z2 = relu(z1) W2^T + b2; logits = relu(z2) W3^T + b3.
    NMF_TRY((gemm<false, true, false, false>((int)n, h, ki, F, ki, W1, ki, a.z1, h, b1, nullptr,
                                             0, nullptr, s)));
    NMF_TRY((gemm<false, true, true, false>((int)n, h, h, a.z1, h, W2, h, a.z2, h, b2, nullptr, 0,
                                            nullptr, s)));
    return gemm<false, true, true, false>((int)n, k, h, a.z2, h, W3, h, a.logit, k, b3, nullptr,
                                          0, nullptr, s);
}

// Gradient of the mean BCE of one batch into net.grad (and the loss into *a.loss).
nmf_status backward(MlpNet &net, const float *F, const uint64_t *lab, int64_t n, const Acts &a,
                    cudaStream_t s)
{
    const int k = net.k, h = net.h, ki = 3 * k, nwords = (k + 63) / 64;
    const float *W2 = net.work + net.off[2], *W3 = net.work + net.off[4];
    float *gW1 = net.grad + net.off[0], *gb1 = net.grad + net.off[1];
    float *gW2 = net.grad + net.off[2], *gb2 = net.grad + net.off[3];
    float *gW3 = net.grad + net.off[4], *gb3 = net.grad + net.off[5];
    const unsigned lb = (unsigned)std::min<int64_t>(cdiv(n * k, 256), 1024);
    mlp_bce_kernel<<<lb, 256, 0, s>>>(a.logit, lab, n, k, nwords, a.dz3, a.loss_part);
    NMF_LAUNCHED("mlp_bce_kernel");
    mlp_loss_sum_kernel<<<1, 32, 0, s>>>(a.loss_part, (int)lb, n * k, a.loss);
    NMF_LAUNCHED("mlp_loss_sum_kernel");
    mlp_fill_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(a.ones, n, 1.0f);
    NMF_LAUNCHED("mlp_fill_kernel");
    // Layer 3: gW3 = dz3^T relu(z2); gb3 = dz3^T 1; dz2 = (dz3 W3) * (z2 > 0).
    NMF_TRY((gemm<true, false, false, true>(k, h, (int)n, a.dz3, k, a.z2, h, gW3, h, nullptr,
                                            nullptr, 0, a.split, s)));
    NMF_TRY((gemm<true, false, false, false>(k, 1, (int)n, a.dz3, k, a.ones, 1, gb3, 1, nullptr,
                                             nullptr, 0, a.split, s)));
    NMF_TRY((gemm<false, false, false, false>((int)n, h, k, a.dz3, k, W3, h, a.dz2, h, nullptr,
                                              a.z2, h, nullptr, s)));
    // Layer 2.
    NMF_TRY((gemm<true, false, false, true>(h, h, (int)n, a.dz2, h, a.z1, h, gW2, h, nullptr,
                                            nullptr, 0, a.split, s)));
    NMF_TRY((gemm<true, false, false, false>(h, 1, (int)n, a.dz2, h, a.ones, 1, gb2, 1, nullptr,
                                             nullptr, 0, a.split, s)));
    NMF_TRY((gemm<false, false, false, false>((int)n, h, h, a.dz2, h, W2, h, a.dz1, h, nullptr,
                                              a.z1, h, nullptr, s)));
    // Layer 1 (the features are not differentiated).
    NMF_TRY((gemm<true, false, false, false>(h, ki, (int)n, a.dz1, h, F, ki, gW1, ki, nullptr,
                                             nullptr, 0, a.split, s)));
    NMF_TRY((gemm<true, false, false, false>(h, 1, (int)n, a.dz1, h, a.ones, 1, gb1, 1, nullptr,
                                             nullptr, 0, a.split, s)));
    return NMF_OK;
}

nmf_status adam(MlpNet &net, float lr, cudaStream_t s)
{
    net.t += 1;
    const float bc1 = 1.0f - powf(ADAM_B1, (float)net.t);
    const float bc2 = 1.0f - powf(ADAM_B2, (float)net.t);
    mlp_adam_kernel<<<(unsigned)cdiv(net.nparams, 256), 256, 0, s>>>(
        net.master, net.work, net.m, net.v, net.grad, net.nparams, lr, bc1, bc2);
    NMF_LAUNCHED("mlp_adam_kernel");
    return NMF_OK;
}

struct Scratch {
    void *p = nullptr;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes ? bytes : 16, s); }
    ~Scratch()
    {
        if (p)
            cudaFreeAsync(p, s);
    }
};

}  // namespace

nmf_status mlp_features(const double *G, const float *B, const float *Xp, int64_t nrhs, int k,
                        float *F, cudaStream_t s)
{
    return launch_features(G, B, Xp, nrhs, k, F, s);
}

nmf_status launch_mlp_features_split(const double *G, const float *B, const float *Xp,
                                     int64_t nrhs, int k, int kpf, int ldd, __nv_bfloat16 *hi,
                                     __nv_bfloat16 *lo, cudaStream_t s)
{
    if (nrhs == 0)
        return NMF_OK;
    if (kpf < k || 3 * kpf > ldd || (ldd % 8))
        return NMF_ERR_INVALID_ARG;
    const int kw = (k + 31) / 32;
    const size_t smem = sizeof(float) * ((size_t)((k * k + 3) & ~3) + 8 * FEAT_R * 32 * kw);
    const unsigned blocks = (unsigned)std::min<int64_t>(cdiv(nrhs, 8 * FEAT_R), 4 * sm_count());
    auto go = [&](auto kern) -> nmf_status {
        if (smem > 48 * 1024)
            NMF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        kern<<<blocks, 256, smem, s>>>(G, B, Xp, nrhs, k, nullptr, kpf, ldd, hi, lo);
        NMF_LAUNCHED("mlp_features_kernel");
        return NMF_OK;
    };
    if (kw == 1)
        return go(mlp_features_kernel<1, true>);
    if (kw == 2)
        return go(mlp_features_kernel<2, true>);
    if (kw == 3)
        return go(mlp_features_kernel<3, true>);
    return go(mlp_features_kernel<4, true>);
}

namespace {

// The tensor-core layers' BF16 weights, current with the working copy.
nmf_status tc_weights(MlpNet &net, cudaStream_t s)
{
    if (!net.tcw)
        NMF_CUDA(cudaMalloc(&net.tcw, mlp_tc_weights_bytes(net.k, net.h)));
    if (net.tcw_t != net.t) {
        const float *w = net.work;
        NMF_TRY(launch_mlp_tc_weights(net.k, net.h, w + net.off[0], w + net.off[2],
                                      w + net.off[4], net.tcw, s));
        net.tcw_t = net.t;
    }
    return NMF_OK;
}

// Inference on the tensor cores (mlp_tc.cu) when the widths allow it.
nmf_status forward_tc(MlpNet &net, const float *F, int64_t n, float *logits, uint64_t *bits,
                      cudaStream_t s)
{
    NMF_TRY(tc_weights(net, s));
    const float *w = net.work;
    return launch_mlp_tc_forward(net.k, net.h, net.tcw, w + net.off[1], w + net.off[3],
                                 w + net.off[5], F, nullptr, nullptr, nullptr, n, logits, bits, s);
}

}  // namespace

nmf_status mlp_propose(MlpNet *net, const float *F, int64_t n, uint64_t *passive, cudaStream_t s)
{
    if (n == 0)
        return NMF_OK;
    if (mlp_tc_supported(net->k, net->h))
        return forward_tc(*net, F, n, nullptr, passive, s);
    Scratch mem(s);
    NMF_CUDA(mem.alloc(acts_bytes(*net, n, false)));
    const Acts a = carve(*net, n, false, mem.p);
    NMF_TRY(forward(*net, F, n, a, s));
    const int nwords = (net->k + 63) / 64;
    mlp_propose_kernel<<<(unsigned)cdiv(n * nwords, 256), 256, 0, s>>>(a.logit, n, net->k, nwords,
                                                                        passive);
    NMF_LAUNCHED("mlp_propose_kernel");
    return NMF_OK;
}

nmf_status mlp_features_propose(MlpNet *net, const double *G, const float *B, const float *Xp,
                                int64_t n, float *F, uint64_t *passive, cudaStream_t s)
{
    if (n == 0)
        return NMF_OK;
    if (mlp_tc_supported(net->k, net->h)) {
        NMF_TRY(tc_weights(*net, s));
        const float *w = net->work;
        return launch_mlp_tc_forward(net->k, net->h, net->tcw, w + net->off[1], w + net->off[3],
                                     w + net->off[5], nullptr, G, B, Xp, n, nullptr, passive, s);
    }
    NMF_TRY(launch_features(G, B, Xp, n, net->k, F, s));
    return mlp_propose(net, F, n, passive, s);
}

nmf_status mlp_logits(MlpNet *net, const float *F, int64_t n, float *logits, cudaStream_t s)
{
    if (n == 0)
        return NMF_OK;
    if (mlp_tc_supported(net->k, net->h))
        return forward_tc(*net, F, n, logits, nullptr, s);
    Scratch mem(s);
    NMF_CUDA(mem.alloc(acts_bytes(*net, n, false)));
    const Acts a = carve(*net, n, false, mem.p);
    NMF_TRY(forward(*net, F, n, a, s));
    NMF_CUDA(cudaMemcpyAsync(logits, a.logit, sizeof(float) * (size_t)n * net->k,
                             cudaMemcpyDeviceToDevice, s));
    return NMF_OK;
}

// Gradient of one batch (no update); loss to *loss_dev when given.
nmf_status mlp_gradient(MlpNet *net, const float *F, const uint64_t *lab, int64_t n,
                        float *grad_out, double *loss_dev, cudaStream_t s)
{
    if (n <= 0)
        return NMF_ERR_INVALID_ARG;
    Scratch mem(s);
    NMF_CUDA(mem.alloc(acts_bytes(*net, n, true)));
    const Acts a = carve(*net, n, true, mem.p);
    NMF_TRY(forward(*net, F, n, a, s));
    NMF_TRY(backward(*net, F, lab, n, a, s));
    if (grad_out)
        NMF_CUDA(cudaMemcpyAsync(grad_out, net->grad, sizeof(float) * (size_t)net->nparams,
                                 cudaMemcpyDeviceToDevice, s));
    if (loss_dev)
        NMF_CUDA(cudaMemcpyAsync(loss_dev, a.loss, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return NMF_OK;
}

// Adam steps over [0, n) in consecutive batches of `batch` (the last may be
// shorter); loss of the last batch to *loss_dev when given.
nmf_status mlp_train(MlpNet *net, const float *F, const uint64_t *lab, int64_t n, int64_t batch,
                     float lr, double *loss_dev, cudaStream_t s)
{
    if (n <= 0 || batch <= 0)
        return NMF_ERR_INVALID_ARG;
    const int64_t bmax = std::min(batch, n);
    Scratch mem(s);
    NMF_CUDA(mem.alloc(acts_bytes(*net, bmax, true)));
    const Acts a = carve(*net, bmax, true, mem.p);
    const int nwords = (net->k + 63) / 64;
    for (int64_t r0 = 0; r0 < n; r0 += bmax) {
        const int64_t nb = std::min(bmax, n - r0);
        const float *Fb = F + r0 * 3 * net->k;
        NMF_TRY(forward(*net, Fb, nb, a, s));
        NMF_TRY(backward(*net, Fb, lab + r0 * nwords, nb, a, s));
        NMF_TRY(adam(*net, lr, s));
    }
    if (loss_dev)
        NMF_CUDA(cudaMemcpyAsync(loss_dev, a.loss, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return NMF_OK;
}

nmf_status mlp_create(MlpNet **out, int k, int h, const float *params, cudaStream_t s)
{
    MlpNet *net = new MlpNet();
    net->k = k;
    net->h = h;
    net->nparams = mlp_param_count(k, h);
    int64_t o = 0;
    const int64_t sz[6] = {(int64_t)h * 3 * k, h, (int64_t)h * h, h, (int64_t)k * h, k};
    for (int i = 0; i < 6; ++i) {
        net->off[i] = o;
        o += sz[i];
    }
    const size_t bytes = sizeof(float) * (size_t)net->nparams;
    cudaError_t e = cudaSuccess;
    for (float **p : {&net->master, &net->work, &net->m, &net->v, &net->grad})
        if (e == cudaSuccess)
            e = cudaMalloc(p, bytes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(net->master, params, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(net->m, 0, bytes, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(net->v, 0, bytes, s);
    if (e != cudaSuccess) {
        mlp_destroy(net);
        return from_cuda(e, "mlp_create");
    }
    mlp_round_kernel<<<(unsigned)cdiv(net->nparams, 256), 256, 0, s>>>(net->master, net->work,
                                                                       net->nparams);
    const cudaError_t le = cudaGetLastError();
    launch_count += 1;
    if (le != cudaSuccess) {
        mlp_destroy(net);
        return from_cuda(le, "mlp_round_kernel");
    }
    *out = net;
    return NMF_OK;
}

void mlp_destroy(MlpNet *net)
{
    if (!net)
        return;
    cudaFree(net->master);
    cudaFree(net->work);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->grad);
    cudaFree(net->tcw);
    delete net;
}

int mlp_k(const MlpNet *net) { return net->k; }
int mlp_hidden(const MlpNet *net) { return net->h; }
int64_t mlp_nparams(const MlpNet *net) { return net->nparams; }
const float *mlp_master(const MlpNet *net) { return net->master; }

}  // namespace nmf
