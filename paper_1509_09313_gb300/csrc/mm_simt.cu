// Dense products of Alg. 1 in plain FP32 on the SIMT pipes (the "MM" task):
//   trans = 0: out (m x k) = A H^T, row i = sum_j A_ij h_j      (contract over n)
//   trans = 1: out (n x k) = A^T W, row j = sum_i A_ij w_i      (contract over m)
// Both are out[p][r] = sum_q A(p, q) F[q][r] with A(p, q) = A[p][q] or A[q][p].
//
// A CTA owns BP = 128 output rows and all k columns (padded to KP, a multiple
// of 16). It streams BQ = 16 contraction steps at a time: the A tile is staged
// q-major in shared memory (transposed on the way in when trans = 0), the F
// tile q-major with zero padding. Each of the 256 threads owns an 8 x (KP/16)
// output block: a tile's 16 products are summed in FP32, and the tile sums are
// added into the running total with Kahan compensation, so the result stays
// within a few units of FP32 rounding however long the contraction (plain
// sequential FP32 accumulation over n = 64000 terms drifts by ~1e-6, which the
// NLS solves amplify by cond(G)). Loads of the next tile are issued into
// registers before the current tile's FMAs (software pipelining).
//
// Roofline: FP32 FMA (2k flops per 4-byte A element, above the SIMT ridge for
// k >= 16); A is read from HBM once per product, F is re-read from L2 by every
// CTA.
#include "common.cuh"

namespace nmf {
namespace {

constexpr int MM_THREADS = 256;
constexpr int BP = 128;
constexpr int BQ = 16;
constexpr int AS_LD = BP + 4;

template <int KP, int TRANS, bool VEC>
__global__ void __launch_bounds__(MM_THREADS, 1)
    mm_simt_kernel(const float *__restrict__ A, int64_t P, int64_t Q, int64_t lda,
                   const float *__restrict__ F, int k, float *__restrict__ out)
{
    constexpr int TR = KP / 16;
    __shared__ __align__(16) float As[2][BQ][AS_LD];
    __shared__ __align__(16) float Fs[2][BQ][KP];

    const int tid = threadIdx.x;
    const int tr = tid % 16;   // column group: columns tr*TR .. tr*TR+TR-1
    const int tp = tid / 16;   // row group: rows tp*8 .. tp*8+7
    const int64_t p0 = (int64_t)blockIdx.x * BP;

    // Register staging for one A tile (BP*BQ = 2048 floats = 2 float4 / thread)
    // and one F tile (BQ*KP floats).
    constexpr int AV = BP * BQ / 4 / MM_THREADS;
    float4 ra[AV];
    constexpr int FPER = (BQ * KP + MM_THREADS - 1) / MM_THREADS;
    float rf[FPER];

    auto load_tile = [&](int64_t q0) {
#pragma unroll
        for (int i = 0; i < AV; ++i) {
            const int e = tid + i * MM_THREADS;   // float4 index in the tile
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (TRANS == 0) {
                // rows p (BP) x BQ/4 float4 along q
                const int pr = e / (BQ / 4), qv = e % (BQ / 4);
                const int64_t p = p0 + pr, q = q0 + 4 * qv;
                if (p < P) {
                    const float *src = A + p * lda + q;
                    if (VEC && q + 3 < Q) {
                        v = *reinterpret_cast<const float4 *>(src);
                    } else {
                        if (q + 0 < Q) v.x = src[0];
                        if (q + 1 < Q) v.y = src[1];
                        if (q + 2 < Q) v.z = src[2];
                        if (q + 3 < Q) v.w = src[3];
                    }
                }
            } else {
                // rows q (BQ) x BP/4 float4 along p
                const int qr = e / (BP / 4), pv = e % (BP / 4);
                const int64_t q = q0 + qr, p = p0 + 4 * pv;
                if (q < Q) {
                    const float *src = A + q * lda + p;
                    if (VEC && p + 3 < P) {
                        v = *reinterpret_cast<const float4 *>(src);
                    } else {
                        if (p + 0 < P) v.x = src[0];
                        if (p + 1 < P) v.y = src[1];
                        if (p + 2 < P) v.z = src[2];
                        if (p + 3 < P) v.w = src[3];
                    }
                }
            }
            ra[i] = v;
        }
#pragma unroll
        for (int i = 0; i < FPER; ++i) {
            const int e = tid + i * MM_THREADS;
            const int qr = e / KP, c = e % KP;
            const int64_t q = q0 + qr;
            rf[i] = (e < BQ * KP && q < Q && c < k) ? F[q * k + c] : 0.0f;
        }
    };
    auto store_tile = [&](int buf) {
#pragma unroll
        for (int i = 0; i < AV; ++i) {
            const int e = tid + i * MM_THREADS;
            if (TRANS == 0) {
                const int pr = e / (BQ / 4), qv = e % (BQ / 4);
                As[buf][4 * qv + 0][pr] = ra[i].x;
                As[buf][4 * qv + 1][pr] = ra[i].y;
                As[buf][4 * qv + 2][pr] = ra[i].z;
                As[buf][4 * qv + 3][pr] = ra[i].w;
            } else {
                const int qr = e / (BP / 4), pv = e % (BP / 4);
                *reinterpret_cast<float4 *>(&As[buf][qr][4 * pv]) = ra[i];
            }
        }
#pragma unroll
        for (int i = 0; i < FPER; ++i) {
            const int e = tid + i * MM_THREADS;
            if (e < BQ * KP)
                Fs[buf][e / KP][e % KP] = rf[i];
        }
    };

    float acc[8][TR], cmp[8][TR];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < TR; ++b) {
            acc[a][b] = 0.0f;
            cmp[a][b] = 0.0f;
        }

    const int64_t nq = cdiv(Q, BQ);
    if (nq > 0) {
        load_tile(0);
        store_tile(0);
    }
    __syncthreads();
    for (int64_t t = 0; t < nq; ++t) {
        const int buf = (int)(t & 1);
        if (t + 1 < nq)
            load_tile((t + 1) * BQ);
        float part[8][TR];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < TR; ++b)
                part[a][b] = 0.0f;
#pragma unroll 4
        for (int q = 0; q < BQ; ++q) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][q][tp * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][q][tp * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float fv[TR];
#pragma unroll
            for (int b = 0; b < TR; ++b)
                fv[b] = Fs[buf][q][tr * TR + b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < TR; ++b)
                    part[a][b] = fmaf(av[a], fv[b], part[a][b]);
        }
        // Kahan: acc + cmp carries the running total to ~FP32 rounding.
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < TR; ++b) {
                const float yk = part[a][b] - cmp[a][b];
                const float tk = acc[a][b] + yk;
                cmp[a][b] = (tk - acc[a][b]) - yk;
                acc[a][b] = tk;
            }
        if (t + 1 < nq)
            store_tile(buf ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int64_t p = p0 + tp * 8 + a;
        if (p < P) {
#pragma unroll
            for (int b = 0; b < TR; ++b) {
                const int c = tr * TR + b;
                if (c < k)
                    out[p * k + c] = acc[a][b];
            }
        }
    }
}

template <int KP>
nmf_status launch_kp(const float *A, int64_t P, int64_t Q, int64_t lda, const float *F, int k,
                     int trans, float *out, cudaStream_t s)
{
    const bool vec = (lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    const dim3 grid((unsigned)cdiv(P, BP));
    if (trans == 0) {
        if (vec)
            mm_simt_kernel<KP, 0, true><<<grid, MM_THREADS, 0, s>>>(A, P, Q, lda, F, k, out);
        else
            mm_simt_kernel<KP, 0, false><<<grid, MM_THREADS, 0, s>>>(A, P, Q, lda, F, k, out);
    } else {
        if (vec)
            mm_simt_kernel<KP, 1, true><<<grid, MM_THREADS, 0, s>>>(A, P, Q, lda, F, k, out);
        else
            mm_simt_kernel<KP, 1, false><<<grid, MM_THREADS, 0, s>>>(A, P, Q, lda, F, k, out);
    }
    NMF_LAUNCHED("mm_simt_kernel");
    return NMF_OK;
}

}  // namespace

nmf_status launch_mm_simt(const float *A, int64_t m, int64_t n, int64_t lda, const float *F,
                          int k, int trans, float *out, cudaStream_t s)
{
    const int64_t P = trans ? n : m;
    const int64_t Q = trans ? m : n;
    if (P == 0)
        return NMF_OK;
    const int kp = (int)cdiv(k, 16) * 16;
    switch (kp) {
    case 16: return launch_kp<16>(A, P, Q, lda, F, k, trans, out, s);
    case 32: return launch_kp<32>(A, P, Q, lda, F, k, trans, out, s);
    case 48: return launch_kp<48>(A, P, Q, lda, F, k, trans, out, s);
    case 64: return launch_kp<64>(A, P, Q, lda, F, k, trans, out, s);
    case 80: return launch_kp<80>(A, P, Q, lda, F, k, trans, out, s);
    case 96: return launch_kp<96>(A, P, Q, lda, F, k, trans, out, s);
    case 112: return launch_kp<112>(A, P, Q, lda, F, k, trans, out, s);
    default: return launch_kp<128>(A, P, Q, lda, F, k, trans, out, s);
    }
}

}  // namespace nmf
