// Dense products of Alg. 1 in plain FP32 on the SIMT pipes (the "MM" task),
// with the objective of Eq. 1 fused into the A H^T pass:
//   trans = 0: out (m x k) = A H^T, row i = sum_j A_ij h_j      (contract over n)
//   trans = 1: out (n x k) = A^T W, row j = sum_i A_ij w_i      (contract over m)
// out[p][c] = sum_q A(p, q) F[q][c] with A(p, q) = A[p][q] or A[q][p].
//
// A CTA owns 128 output rows and one chunk of up to 64 output columns (4 NCG,
// k rounded up to a multiple of 8, 16 NCG threads); each thread holds 8 rows
// x 4 columns. The contraction streams in stages (A H^T: 4 NCG steps, A^T W:
// 32) through a ring of three stages in shared memory, filled by cp.async
// (16-byte copies straight to shared memory, zero-filled past the edges; row
// strides padded so that the warps' vector reads are conflict-free).
//
// The FMAs are packed FP32x2 (FFMA2, two independent FMAs per instruction),
// which halves the issue slots the FMA pipe needs:
//  - A H^T pairs consecutive contraction steps: {A[p][q], A[p][q+1]} times
//    {F[q][c], F[q+1][c]} into an even-step and an odd-step partial sum. A is
//    staged p-major (its rows are contiguous in q) and F transposed (c-major),
//    so both pairs are halves of 16-byte shared-memory reads. The thread's
//    rows are 16 apart and its columns 16 apart, which spreads the warps'
//    reads over all banks.
//  - A^T W pairs consecutive output rows: {A[q][p], A[q][p+1]} (q-major tile)
//    times {F[q][c], F[q][c]} (the value paired with itself in registers:
//    a copy with every value twice in shared memory would double the bytes
//    each thread loads, and a warp's shared-memory bandwidth goes by those
//    bytes); the thread's 8 rows and 4 columns are contiguous.
// The partial sums of each stage (A H^T: two chains of 2 NCG steps; A^T W:
// 32 steps) are added into the running totals with Kahan compensation, and
// the output is the compensated total rounded once (with contraction splits:
// each split's total and compensation, added over the splits in FP64 and
// rounded once). So the products stay within about one FP32 rounding however
// long the contraction: plain sequential FP32 accumulation over n = 64000
// terms drifts by ~1e-6, and even product noise of a few 1e-8 moves the
// objective of a short run by ~1e-6 through the NLS solves.
//
// Objective (trans = 0, k <= 64): the CTA also forms its 128 x 64 tile of
// W H for every stage from its rows of W (held in shared memory for the whole
// pass) and the stage's tile of H (the transposed F tile already there), with
// FFMA2 over pairs of rows, and adds the squared residuals A_ij - w_i . h_j to
// a Kahan-compensated FP32 sum per thread; the threads' sums are added in
// FP64 into one partial per CTA, and the partials in a fixed order. A is read
// once for both.
//
// Roofline: FP32 FMA (2k flops per element of A, and 2k more for the fused
// objective), above the SIMT ridge for k >= 16. F is made once per call as a
// 64-column padded copy (transposed for A H^T), read from L2 by every CTA.
#include <algorithm>

#include "common.cuh"

namespace nmf {
namespace {

constexpr int F32_BQ1 = 32;                // contraction steps per stage, trans = 1

// Tile shape, from the column groups of 4 (NCG, even: whole warps) and the
// rows per thread (RPT): 16 NCG threads, 16 RPT output rows x 4 NCG columns
// per CTA. trans = 0 takes 4 NCG contraction steps per stage (so that the
// objective's 16 RPT x 4 NCG tile of W H maps 8 x 4 onto the threads),
// trans = 1 takes 64. Row strides are padded by 4 floats.
template <int TRANS, int NCG, int RPT>
struct F32Tile {
    // Three stages; A^T W at most 128 registers, so that two CTAs share an
    // SM; A H^T (with the objective's W tile): one CTA.
    static constexpr int STAGES = 3;
    static constexpr int THREADS = 16 * NCG;
    static constexpr int BP = 16 * RPT;
    static constexpr int KP = 4 * NCG;
    static constexpr int BQ = TRANS == 0 ? 4 * NCG : F32_BQ1;
    static constexpr int LDA = TRANS == 0 ? BQ + 4 : BP + 4;   // A p-major / q-major
    static constexpr int LDF = TRANS == 0 ? BQ + 4 : KP + 4;   // F^T c-major / F q-major
    static constexpr int A = TRANS == 0 ? BP * LDA : BQ * LDA;
    static constexpr int F = TRANS == 0 ? KP * LDF : BQ * LDF;
    static constexpr int STAGE = A + F;                   // floats
    static constexpr int W = KP * BP;                     // objective: W^T of the CTA's rows
    static constexpr int ACH = TRANS == 0 ? BP * BQ / 4 : BQ * BP / 4;         // 16-byte chunks
    static constexpr int FCH = KP * BQ / 4;
    static constexpr size_t bytes(bool obj)
    {
        return sizeof(float) * ((size_t)STAGES * STAGE + (obj ? W : 0)) + 64 * sizeof(double);
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte copy global -> shared; the bytes past `valid` (0..16) are zero.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ int clamp16(int64_t v) { return v <= 0 ? 0 : v >= 16 ? 16 : (int)v; }

template <int TRANS, bool OBJ, int NCG, int RPT>
__device__ __forceinline__ void mm_f32_body(const float *__restrict__ A, int64_t P, int64_t Q,
                                            int64_t lda, const float *__restrict__ Fc,
                                            int64_t ldf, int k, int64_t q_per_split,
                                            float *__restrict__ out,
                                            const float *__restrict__ W,
                                            double *__restrict__ obj_part)
{
    using T = F32Tile<TRANS, NCG, RPT>;
    constexpr int NT = T::THREADS, BP = T::BP, KP = T::KP, BQ = T::BQ, NS = T::STAGES;
    extern __shared__ __align__(16) float f32_smem[];
    float *Wt = f32_smem + NS * T::STAGE;
    const int tid = threadIdx.x;
    const int pg = tid / NCG, cg = tid % NCG;
    const int64_t p0 = (int64_t)blockIdx.x * BP;
    const int c0 = blockIdx.y * KP;            // this CTA's column chunk
    // Contraction range of this CTA (a split of it when gridDim.z > 1).
    const int64_t qb = (int64_t)blockIdx.z * q_per_split;
    const int64_t qe = min(Q, qb + q_per_split);
    const int64_t nst = qe > qb ? cdiv(qe - qb, BQ) : 0;

    auto load_stage = [&](int64_t st, int buf) {
        const int64_t q0 = qb + st * BQ;
        float *As = f32_smem + buf * T::STAGE;
        float *Fs = As + T::A;
        for (int e = tid; e < T::ACH; e += NT) {
            if (TRANS == 0) {
                const int pr = e / (BQ / 4), qc = e % (BQ / 4);
                const int64_t p = p0 + pr, q = q0 + 4 * qc;
                const int bytes = p < P ? clamp16(4 * (qe - q)) : 0;
                const float *src = A + (bytes ? p * lda + q : 0);
                cp_async16(smem_addr(As + pr * T::LDA + 4 * qc), src, bytes);
            } else {
                const int qr = e / (BP / 4), pc = e % (BP / 4);
                const int64_t q = q0 + qr, p = p0 + 4 * pc;
                const int bytes = q < qe ? clamp16(4 * (P - p)) : 0;
                const float *src = A + (bytes ? q * lda + p : 0);
                cp_async16(smem_addr(As + qr * T::LDA + 4 * pc), src, bytes);
            }
        }
        for (int e = tid; e < T::FCH; e += NT) {
            if (TRANS == 0) {
                // F^T: rows = columns c (ldf = padded Q).
                const int cr = e / (BQ / 4), qc = e % (BQ / 4);
                const int64_t q = q0 + 4 * qc;
                const int bytes = clamp16(4 * (qe - q));
                const float *src = Fc + (bytes ? (int64_t)(c0 + cr) * ldf + q : 0);
                cp_async16(smem_addr(Fs + cr * T::LDF + 4 * qc), src, bytes);
            } else {
                // F: rows = q (ldf = padded columns).
                const int qr = e / (KP / 4), cc = e % (KP / 4);
                const int64_t q = q0 + qr;
                const float *src = Fc + (q < qe ? q * ldf + c0 + 4 * cc : 0);
                cp_async16(smem_addr(Fs + qr * T::LDF + 4 * cc), src, q < qe ? 16 : 0);
            }
        }
    };

    // The objective's W rows, W^T in shared memory: Wt[r][8 pg + a] = W[p0 +
    // pg + 16 a][r] (zero past P and past k), so a thread's 8 rows are
    // contiguous.
    if (OBJ) {
        for (int e = tid; e < KP * BP; e += NT) {
            const int r = e / BP, s = e % BP;
            const int64_t p = p0 + (s >> 3) + 16 * (s & 7);
            Wt[e] = (p < P && r < k) ? W[p * k + r] : 0.0f;
        }
    }

    float acc[RPT][4], cmp[RPT][4];
#pragma unroll
    for (int a = 0; a < RPT; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            acc[a][b] = 0.0f;
            cmp[a][b] = 0.0f;
        }
    // A^T W keeps its totals as pairs of rows (a, a + 1), like its FMAs.
    float2 ac2[RPT / 2][4], nc2[RPT / 2][4];
#pragma unroll
    for (int ap = 0; ap < RPT / 2; ++ap)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            ac2[ap][b] = make_float2(0.0f, 0.0f);
            nc2[ap][b] = make_float2(0.0f, 0.0f);
        }
    float osum = 0.0f, ocmp = 0.0f;   // objective: Kahan sum of squared residuals

#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
        if (s < nst)
            load_stage(s, s);
        cp_async_commit();
    }
    for (int64_t t = 0; t < nst; ++t) {
        cp_async_wait<NS - 2>();
        __syncthreads();
        {
            const int64_t nt = t + NS - 1;
            if (nt < nst)
                load_stage(nt, (int)(nt % NS));
            cp_async_commit();
        }
        const float *As = f32_smem + (int)(t % NS) * T::STAGE;
        const float *Fs = As + T::A;
        float part[RPT][4];
        if (TRANS == 0) {
            // Rows pg + 16 a, columns cg + NCG b; pairs of contraction steps.
            float2 pp[RPT][4];
#pragma unroll
            for (int a = 0; a < RPT; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    pp[a][b] = make_float2(0.0f, 0.0f);
#pragma unroll 2
            for (int qq = 0; qq < BQ / 4; ++qq) {
                float4 av[RPT], fv[4];
#pragma unroll
                for (int a = 0; a < RPT; ++a)
                    av[a] = *reinterpret_cast<const float4 *>(As + (pg + 16 * a) * T::LDA + 4 * qq);
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    fv[b] = *reinterpret_cast<const float4 *>(Fs + (cg + NCG * b) * T::LDF + 4 * qq);
#pragma unroll
                for (int a = 0; a < RPT; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        pp[a][b] = __ffma2_rn(make_float2(av[a].x, av[a].y),
                                              make_float2(fv[b].x, fv[b].y), pp[a][b]);
#pragma unroll
                for (int a = 0; a < RPT; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        pp[a][b] = __ffma2_rn(make_float2(av[a].z, av[a].w),
                                              make_float2(fv[b].z, fv[b].w), pp[a][b]);
            }
#pragma unroll
            for (int a = 0; a < RPT; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    part[a][b] = pp[a][b].x + pp[a][b].y;
            if (OBJ) {
                // W H for rows pg + 16 a (pairs a, a + 1) and contraction
                // steps q0 + cg + NCG b of this stage, then the squared
                // residuals.
                float2 wh[RPT / 2][4];
#pragma unroll
                for (int ap = 0; ap < RPT / 2; ++ap)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        wh[ap][b] = make_float2(0.0f, 0.0f);
#pragma unroll 2
                for (int r = 0; r < k; ++r) {
                    const float4 w0 = *reinterpret_cast<const float4 *>(Wt + r * BP + 8 * pg);
                    const float4 w1 = *reinterpret_cast<const float4 *>(Wt + r * BP + 8 * pg + 4);
                    const float2 wv[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w),
                                          make_float2(w1.x, w1.y), make_float2(w1.z, w1.w)};
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float h = Fs[r * T::LDF + cg + NCG * b];
#pragma unroll
                        for (int ap = 0; ap < RPT / 2; ++ap)
                            wh[ap][b] = __ffma2_rn(wv[ap], make_float2(h, h), wh[ap][b]);
                    }
                }
#pragma unroll
                for (int a = 0; a < RPT; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float whv = (a & 1) ? wh[a >> 1][b].y : wh[a >> 1][b].x;
                        const float rsd = As[(pg + 16 * a) * T::LDA + cg + NCG * b] - whv;
                        const float yk = fmaf(rsd, rsd, -ocmp);
                        const float tk = osum + yk;
                        ocmp = (tk - osum) - yk;
                        osum = tk;
                    }
            }
        } else {
            // Rows RPT pg + a (pairs a, a + 1), columns 4 cg + b. The stage's
            // partial sums go into the running totals at its end (packed
            // Kahan: nc2 holds minus the compensation).
            float2 pp[RPT / 2][4];
#pragma unroll
            for (int ap = 0; ap < RPT / 2; ++ap)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    pp[ap][b] = make_float2(0.0f, 0.0f);
#pragma unroll 1
            for (int q = 0; q < BQ; ++q) {
                float2 av[RPT / 2];
#pragma unroll
                for (int v = 0; v < RPT / 4; ++v) {
                    const float4 a4 =
                        *reinterpret_cast<const float4 *>(As + q * T::LDA + RPT * pg + 4 * v);
                    av[2 * v] = make_float2(a4.x, a4.y);
                    av[2 * v + 1] = make_float2(a4.z, a4.w);
                }
                const float4 f4 = *reinterpret_cast<const float4 *>(Fs + q * T::LDF + 4 * cg);
                const float2 fd[4] = {make_float2(f4.x, f4.x), make_float2(f4.y, f4.y),
                                      make_float2(f4.z, f4.z), make_float2(f4.w, f4.w)};
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int ap = 0; ap < RPT / 2; ++ap)
                        pp[ap][b] = __ffma2_rn(av[ap], fd[b], pp[ap][b]);
            }
            const float2 neg1 = make_float2(-1.0f, -1.0f);
#pragma unroll
            for (int ap = 0; ap < RPT / 2; ++ap)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float2 yk = __fadd2_rn(pp[ap][b], nc2[ap][b]);
                    const float2 tk = __fadd2_rn(ac2[ap][b], yk);
                    nc2[ap][b] = __fadd2_rn(__ffma2_rn(tk, neg1, ac2[ap][b]), yk);
                    ac2[ap][b] = tk;
                }
            continue;
        }
        // Kahan: acc + cmp carries the running total to ~FP32 rounding.
#pragma unroll
        for (int a = 0; a < RPT; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float yk = part[a][b] - cmp[a][b];
                const float tk = acc[a][b] + yk;
                cmp[a][b] = (tk - acc[a][b]) - yk;
                acc[a][b] = tk;
            }
    }
    cp_async_wait<0>();
    // acc: the running total; cmp: minus its compensation.
    if (TRANS == 1) {
#pragma unroll
        for (int a = 0; a < RPT; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                acc[a][b] = (a & 1) ? ac2[a >> 1][b].y : ac2[a >> 1][b].x;
                cmp[a][b] = (a & 1) ? nc2[a >> 1][b].y : nc2[a >> 1][b].x;
            }
    } else {
#pragma unroll
        for (int a = 0; a < RPT; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                cmp[a][b] = -cmp[a][b];
    }

    // Output: the compensated total rounded once, or (contraction split)
    // this split's total and compensation, for the FP64 sum over splits.
    const bool split = gridDim.z > 1;
    float *dst = out + (int64_t)blockIdx.z * 2 * P * k;
#pragma unroll
    for (int a = 0; a < RPT; ++a) {
        const int64_t p = p0 + (TRANS == 0 ? pg + 16 * a : RPT * pg + a);
        if (p < P) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int c = c0 + (TRANS == 0 ? cg + NCG * b : 4 * cg + b);
                if (c < k) {
                    if (split) {
                        dst[p * k + c] = acc[a][b];
                        dst[P * k + p * k + c] = cmp[a][b];
                    } else {
                        dst[p * k + c] = acc[a][b] + cmp[a][b];
                    }
                }
            }
        }
    }
    if (OBJ) {
        // The threads' sums in FP64, in a fixed order.
        double v = (double)osum - (double)ocmp;
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(FULL, v, o);
        double *red = reinterpret_cast<double *>(Wt + KP * BP);
        __syncthreads();
        if ((tid & 31) == 0)
            red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w)
                s += red[w];
            obj_part[blockIdx.x] = s;
        }
    }
}

// A H^T (one CTA per SM) and A^T W (two CTAs per SM: at most 128 registers,
// since each of the SM's four quarters holds 16384 registers and up to four
// of the two CTAs' warps).
template <bool OBJ, int NCG, int RPT>
__global__ void __launch_bounds__(16 * NCG, 1)
    mm_f32_kernel(const float *__restrict__ A, int64_t P, int64_t Q, int64_t lda,
                  const float *__restrict__ Fc, int64_t ldf, int k, int64_t q_per_split,
                  float *__restrict__ out, const float *__restrict__ W,
                  double *__restrict__ obj_part)
{
    mm_f32_body<0, OBJ, NCG, RPT>(A, P, Q, lda, Fc, ldf, k, q_per_split, out, W, obj_part);
}

template <int NCG, int RPT>
__global__ void __maxnreg__(128)
    mm_f32_t_kernel(const float *__restrict__ A, int64_t P, int64_t Q, int64_t lda,
                    const float *__restrict__ Fc, int64_t ldf, int k, int64_t q_per_split,
                    float *__restrict__ out)
{
    mm_f32_body<1, false, NCG, RPT>(A, P, Q, lda, Fc, ldf, k, q_per_split, out, nullptr,
                                    nullptr);
}

// out[p][c] = the sum over splits s of total[s][p][c] + compensation[s][p][c]
// (part holds each split's two arrays in turn), in FP64 in split order,
// rounded once.
__global__ void f32_reduce_kernel(const float *__restrict__ part, int splits, int64_t len,
                                  float *__restrict__ out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp)
            s += (double)part[2 * sp * len + e] + (double)part[(2 * sp + 1) * len + e];
        out[e] = (float)s;
    }
}

// F^T (trans = 0): Ft[c][q] = F[q][c] for c < k, 0 for k <= c < kpt, rows of
// length ldq (Q rounded up to 4), through 32 x 32 shared-memory tiles.
__global__ void f32_transpose_kernel(const float *__restrict__ F, int64_t Q, int k, int kpt,
                                     int64_t ldq, float *__restrict__ Ft)
{
    __shared__ float tile[32][33];
    const int64_t q0 = (int64_t)blockIdx.x * 32;
    const int cbase = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t q = q0 + r;
        const int c = cbase + threadIdx.x;
        tile[r][threadIdx.x] = (q < Q && c < k) ? F[q * k + c] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = cbase + r;
        const int64_t q = q0 + threadIdx.x;
        if (c < kpt && q < ldq)
            Ft[(int64_t)c * ldq + q] = tile[threadIdx.x][r];   // zero past Q and k
    }
}

// F padded to kpt columns (trans = 1): Fp[q][c] = F[q][c] for c < k, 0 up to
// kpt.
__global__ void f32_pad_kernel(const float *__restrict__ F, int64_t Q, int k, int kpt,
                               float *__restrict__ Fp)
{
    const int64_t total = Q * kpt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / kpt;
        const int c = (int)(e - q * kpt);
        Fp[e] = c < k ? F[q * k + c] : 0.0f;
    }
}

// Column groups of 4 per CTA for k: whole warps (an even count), at most 16;
// k > 64 runs in chunks of 64 columns.
int f32_ncg(int k) { return k <= 16 ? 4 : k <= 32 ? 8 : k <= 48 ? 12 : k <= 56 ? 14 : 16; }
constexpr int RPT0 = 8, RPT1 = 8;   // rows per thread: A H^T, A^T W

struct F32Plan {
    int ncg, kp, nch, kpt, splits;
    int64_t P, Q, ldf, bp, q_per_split;
    size_t f_off, part_off, split_off, total;
};

F32Plan f32_plan(int64_t m, int64_t n, int k, int trans, bool obj)
{
    F32Plan w;
    w.P = trans ? n : m;
    w.Q = trans ? m : n;
    w.ncg = f32_ncg(k);
    w.kp = 4 * w.ncg;
    w.nch = (int)cdiv(k, w.kp);
    w.kpt = w.kp * w.nch;
    w.bp = 16 * (trans ? RPT1 : RPT0);
    w.ldf = trans ? w.kpt : cdiv(w.Q > 0 ? w.Q : 1, 4) * 4;
    // A^T W splits its contraction (up to 16 ways, each split keeping at
    // least 8 stages) so that its CTAs fill whole waves of two per SM: the
    // fewest splits within 2% of the best wave efficiency. A H^T never
    // splits, so that its products are the same with and without the fused
    // objective.
    const int64_t tiles = cdiv(w.P > 0 ? w.P : 1, w.bp) * w.nch;
    const int64_t bq = trans ? F32_BQ1 : 4 * w.ncg;
    w.splits = 1;
    if (trans) {
        const int64_t slots = 2 * (int64_t)sm_count();
        auto eff = [&](int64_t sp) {
            const int64_t ctas = tiles * sp;
            return (double)ctas / (double)(cdiv(ctas, slots) * slots);
        };
        auto allowed = [&](int64_t sp) { return sp == 1 || w.Q / sp >= 8 * bq; };
        double best = 0.0;
        for (int64_t sp = 1; sp <= 16; ++sp)
            if (allowed(sp))
                best = std::max(best, eff(sp));
        for (int64_t sp = 1; sp <= 16; ++sp)
            if (allowed(sp) && eff(sp) >= best - 0.02) {
                w.splits = (int)sp;
                break;
            }
    }
    (void)obj;
    w.q_per_split = cdiv(cdiv(w.Q > 0 ? w.Q : 1, w.splits), bq) * bq;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    w.f_off = 0;
    const size_t fbytes = trans ? sizeof(float) * (size_t)(w.Q > 0 ? w.Q : 1) * w.kpt
                                : sizeof(float) * (size_t)w.kpt * w.ldf;
    w.part_off = al(fbytes);
    w.split_off = w.part_off + al(sizeof(double) * (size_t)cdiv(w.P > 0 ? w.P : 1, w.bp));
    w.total = w.split_off +
              (w.splits > 1 ? al(sizeof(float) * 2 * (size_t)w.splits * (size_t)w.P * k) : 0);
    return w;
}

template <int TRANS, bool OBJ, int NCG>
nmf_status launch_tile(const float *A, const F32Plan &w, int64_t lda, const float *Fc, int k,
                       float *out, const float *W, double *part, cudaStream_t s)
{
    constexpr int RPT = TRANS ? RPT1 : RPT0;
    using T = F32Tile<TRANS, NCG, RPT>;
    const size_t smem = T::bytes(OBJ);
    static SmemOptIn opt_in;
    const dim3 grid((unsigned)cdiv(w.P, T::BP), (unsigned)w.nch, (unsigned)w.splits);
    if constexpr (TRANS == 0) {
        NMF_TRY(ensure_smem(mm_f32_kernel<OBJ, NCG, RPT>, opt_in, smem));
        mm_f32_kernel<OBJ, NCG, RPT><<<grid, T::THREADS, smem, s>>>(
            A, w.P, w.Q, lda, Fc, w.ldf, k, w.q_per_split, out, W, part);
        NMF_LAUNCHED("mm_f32_kernel");
    } else {
        NMF_TRY(ensure_smem(mm_f32_t_kernel<NCG, RPT>, opt_in, smem));
        static SmemOptIn carve;   // all of the SM's on-chip memory as shared memory
        int dev = 0;
        NMF_CUDA(cudaGetDevice(&dev));
        if (dev >= 0 && dev < SmemOptIn::MAX_DEVICES && !carve.bytes[dev]) {
            NMF_CUDA(cudaFuncSetAttribute(mm_f32_t_kernel<NCG, RPT>,
                                          cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            carve.bytes[dev] = 1;
        }
        mm_f32_t_kernel<NCG, RPT><<<grid, T::THREADS, smem, s>>>(
            A, w.P, w.Q, lda, Fc, w.ldf, k, w.q_per_split, out);
        NMF_LAUNCHED("mm_f32_t_kernel");
    }
    return NMF_OK;
}

template <int TRANS, bool OBJ>
nmf_status launch_ncg(const float *A, const F32Plan &w, int64_t lda, const float *Fc, int k,
                      float *out, const float *W, double *part, cudaStream_t s)
{
    switch (w.ncg) {
    case 4: return launch_tile<TRANS, OBJ, 4>(A, w, lda, Fc, k, out, W, part, s);
    case 8: return launch_tile<TRANS, OBJ, 8>(A, w, lda, Fc, k, out, W, part, s);
    case 12: return launch_tile<TRANS, OBJ, 12>(A, w, lda, Fc, k, out, W, part, s);
    case 14: return launch_tile<TRANS, OBJ, 14>(A, w, lda, Fc, k, out, W, part, s);
    default: return launch_tile<TRANS, OBJ, 16>(A, w, lda, Fc, k, out, W, part, s);
    }
}

}  // namespace

bool mm_f32_supported(const float *A, int64_t lda)
{
    return (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
}

size_t mm_f32_work_bytes(int64_t m, int64_t n, int k, int trans)
{
    return std::max(f32_plan(m, n, k, trans, false).total, f32_plan(m, n, k, trans, true).total);
}

nmf_status launch_mm_f32(const float *A, int64_t m, int64_t n, int64_t lda, const float *F, int k,
                         int trans, float *out, const float *W, double *f_dev, void *work,
                         size_t work_bytes, cudaStream_t s)
{
    const bool obj = W != nullptr;
    const F32Plan w = f32_plan(m, n, k, trans, obj);
    if (w.P == 0)
        return NMF_OK;
    if (!mm_f32_supported(A, lda) || work_bytes < w.total || (obj && (trans || k > 64 || !f_dev)))
        return NMF_ERR_INVALID_ARG;
    unsigned char *wb = static_cast<unsigned char *>(work);
    float *Fc = reinterpret_cast<float *>(wb + w.f_off);
    double *part = reinterpret_cast<double *>(wb + w.part_off);
    float *dst = w.splits > 1 ? reinterpret_cast<float *>(wb + w.split_off) : out;
    if (trans == 0) {
        const dim3 tg((unsigned)cdiv(w.ldf, 32), (unsigned)cdiv(w.kpt, 32));
        f32_transpose_kernel<<<tg, dim3(32, 8), 0, s>>>(F, w.Q, k, w.kpt, w.ldf, Fc);
        NMF_LAUNCHED("f32_transpose_kernel");
    } else {
        const int64_t total = w.Q * (int64_t)w.kpt;
        const unsigned blocks = (unsigned)std::min<int64_t>(cdiv(total > 0 ? total : 1, 256),
                                                            (int64_t)sm_count() * 8);
        f32_pad_kernel<<<blocks, 256, 0, s>>>(F, w.Q, k, w.kpt, Fc);
        NMF_LAUNCHED("f32_pad_kernel");
    }
    if (trans)
        NMF_TRY((launch_ncg<1, false>(A, w, lda, Fc, k, dst, nullptr, nullptr, s)));
    else if (!obj)
        NMF_TRY((launch_ncg<0, false>(A, w, lda, Fc, k, dst, nullptr, nullptr, s)));
    else
        NMF_TRY((launch_ncg<0, true>(A, w, lda, Fc, k, dst, W, part, s)));
    if (w.splits > 1) {
        const int64_t len = w.P * (int64_t)k;
        const unsigned blocks =
            (unsigned)std::min<int64_t>(cdiv(len, 256), (int64_t)sm_count() * 8);
        f32_reduce_kernel<<<blocks, 256, 0, s>>>(dst, w.splits, len, out);
        NMF_LAUNCHED("f32_reduce_kernel");
    }
    if (obj)
        return launch_sum_partials(part, (int)cdiv(w.P, w.bp), f_dev, s);
    return NMF_OK;
}

}  // namespace nmf
