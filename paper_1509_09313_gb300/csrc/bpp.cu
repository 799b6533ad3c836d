// Batched NLS by block principal pivoting (Eq. 3, Eq. 4, Sec. 4.2).
//
// Every right-hand side j solves  min_{x >= 0} 0.5 x^T G x - g_j^T x  with one
// shared k x k Gram G. BPP partitions the indices into a passive set F (free)
// and an active set (x_i = 0); for a partition the candidate is
//   x_F = G_FF^{-1} g_F, x_A = 0, y = G x - g (y_F = 0),
// and the exchange rules of the cited method (full exchange while the number
// of infeasible indices drops, three more full exchanges otherwise, then the
// backup single exchange of the largest infeasible index) move infeasible
// indices (x_i < 0 on F, y_i < 0 off F) across until Eq. 4 holds.
//
// GPU design (differs from the paper's column grouping; same result):
//  * bpp_prep_kernel (one CTA, FP64) factors the usable part of G once per
//    half-step (G = L L^T; indices with G_ii <= 0 are never passive), forms
//    M = G^{-1} and the condition number cond_1(S G S) = ||S G S||_1
//    ||S^-1 M S^-1||_1 of G with its diagonal scaled to one (S = diag(G)^-1/2),
//    and picks the arithmetic of the solves: FP32 when it is <= 1e4 (mode 0),
//    FP64 otherwise (mode 1), FP64 without M when G is numerically singular
//    (mode 2). The scaled number is the one that bounds the FP32 error: every
//    FP32 step here (rounding G and M, Cholesky, the matrix-vector products)
//    perturbs entry (i, j) relative to sqrt(G_ii G_jj), so a factor that is
//    merely badly scaled (one row of H much smaller than the rest, common in
//    early iterations) costs nothing.
//  * solve kernels: persistent, one warp per right-hand side, G and M in
//    shared memory. Lane l holds indices l, l+32, ... of g, x, y and of the
//    unconstrained solution u = M g. Each exchange round solves the smaller of
//    two equivalent systems:
//      direct      G_FF x_F = g_F                          (|F| x |F|)
//      complement  M_AA y_A = -u_A,  x_F = u_F + M_FA y_A  (|A| x |A|)
//    (the second follows from G x = g + y with y supported on A and x_A = 0),
//    by a warp-cooperative Cholesky in shared memory with shuffle-broadcast
//    substitutions. Cost per round O(min(|F|,|A|)^3 + k |F|) instead of
//    O(|F|^3). bpp_solve32_kernel (bpp32.cu) runs mode 0: it refines once
//    (residual g_F - G_FF x_F solved through the same factor: the explicit
//    inverse alone is not backward stable), recomputes y from G, and counts a
//    sign test as violated only beyond 2^-20 of the problem's scale in the
//    diagonally scaled variables (x_i sqrt(G_ii) against max over F of
//    |x_j| sqrt(G_jj); y_i / sqrt(G_ii) against max of |g_j| / sqrt(G_jj)):
//    values within FP32 noise of zero are degenerate ties that would
//    otherwise make the exchange rules cycle. The final x is clamped at 0
//    there. A system whose FP32 pivot falls below 1e-4 of its diagonal
//    defers its right-hand side to a second pass of bpp_solve_kernel in FP64.
//    bpp_solve_kernel (here) runs modes 1 and 2 in FP64 with the strict sign
//    test and no refinement.
//  * Every loop is bounded: a solve stops at max_rounds with status
//    NOT_CONVERGED; there are no spin-waits.
//
// Roofline: FP32 ALU for the pivoting; HBM traffic is nrhs * k * 8 bytes
// (right-hand sides in, solutions out) plus bitmasks.
#include <math.h>

#include <mutex>

#include "bpp_internal.cuh"

namespace nmf {
namespace {

using namespace bpp;

constexpr int BPP_WARPS = 8;               // most warps per CTA (launch bound)
constexpr int BPP_THREADS = BPP_WARPS * 32;

// Workspace layout (bytes, 256-aligned pieces).
struct WorkLayout {
    size_t g32, m32, m64, usable, flags, counters, defer, prep, total;
};

WorkLayout layout(int k)
{
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    WorkLayout w;
    size_t off = 0;
    w.g32 = off; off += al(sizeof(float) * k * k);
    w.m32 = off; off += al(sizeof(float) * k * k);
    w.m64 = off; off += al(sizeof(double) * k * k);
    w.usable = off; off += al(sizeof(uint32_t) * 4);
    w.flags = off; off += al(sizeof(int) * 4);
    w.counters = off; off += al(sizeof(unsigned long long) * CNT_WORDS);
    w.defer = off; off += al(sizeof(int64_t) * DEFER_CAP);
    w.prep = off; off += al(sizeof(double) * (NMF_MAX_K + 2));   // 1 / L_aa, two norms
    w.total = off;
    return w;
}

// Row of entry e of a lower triangle stored row by row (e = a (a + 1) / 2 + b,
// b <= a): the FP32 estimate of the root of a (a + 1) / 2 = e, corrected.
__device__ __forceinline__ int tri_row(int e)
{
    int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (a * (a + 1) / 2 > e)
        --a;
    while ((a + 1) * (a + 2) / 2 <= e)
        ++a;
    return a;
}

// ---------------------------------------------------------------------------
// Prep: FP64 Cholesky of G_UU, its inverse and the scaled cond_1.
// flags[0] = mode (0 FP32, 1 FP64 with M, 2 FP64 without M), flags[1] = |U|,
// flags[2] = 1 while the inverse and cond_1 are left to the kernels below,
// flags[3] counts their last kernel's finished CTAs.
//
// The factorisation runs on one CTA (a chain of pivots). When every index is
// usable and k >= PREP_SPLIT_K, the rest spreads over the GPU (GB300's FP64
// pipe does two operations per clock per SM, so one CTA spent most of the
// preparation on them): L^{-1} one warp per column (bpp_prep_inv_kernel), M =
// L^{-T} L^{-1} one CTA per column (bpp_prep_m_kernel), the column sums of
// cond_1 and the symmetric copy of M one CTA per column
// (bpp_prep_cond_kernel). All work inside M64: L in its lower triangle,
// L^{-1} transposed in its strict upper triangle, then M's lower triangle
// over L, then M's upper triangle over L^{-1}.
// ---------------------------------------------------------------------------
constexpr int PREP_THREADS = 256;
constexpr int PREP_SPLIT_K = 48;

// Sum over the 32 lanes (xor butterfly: every lane gets the same value).
__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__global__ void __launch_bounds__(PREP_THREADS)
    bpp_prep_kernel(const double *__restrict__ G, int k, float *__restrict__ G32,
                    float *__restrict__ M32, double *__restrict__ M64,
                    uint32_t *__restrict__ usable_words, int *__restrict__ flags,
                    unsigned long long *__restrict__ counters, BppStats *__restrict__ stats,
                    double *__restrict__ prep)
{
    extern __shared__ double sm[];
    // L: u x u, the Cholesky factor in its lower triangle (diagonal included)
    // and, once formed, L^{-1} transposed in its strict upper triangle:
    // (L^{-1})_ac for a > c at L[c * u + a]; rdiag holds (L^{-1})_aa = 1 / L_aa.
    double *L = sm;
    double *dsq = L + k * k;                          // sqrt(G_aa), a < u
    double *rdiag = dsq + k;                          // 1 / L_aa
    double *gdiag = rdiag + k;                        // G_aa
    int *uidx = reinterpret_cast<int *>(gdiag + k);   // k
    __shared__ int s_u, s_ok;
    __shared__ unsigned long long s_norm[2];
    const int tid = threadIdx.x;

    for (int e = tid; e < k * k; e += PREP_THREADS) {
        G32[e] = (float)G[e];
        M32[e] = 0.0f;
        M64[e] = 0.0;
    }
    if (tid == 0) {
        int u = 0;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        for (int i = 0; i < k; ++i)
            if (G[i * k + i] > 0.0) {
                uidx[u++] = i;
                w[i >> 5] |= 1u << (i & 31);
            }
        for (int q = 0; q < 4; ++q)
            usable_words[q] = w[q];
        s_u = u;
        s_ok = u > 0;
        s_norm[0] = s_norm[1] = 0ull;
        for (int c = 0; c < CNT_WORDS; ++c)
            counters[c] = 0ull;
    }
    __syncthreads();
    const int u = s_u;
    for (int e = tid; e < u * u; e += PREP_THREADS) {
        const int a = e / u, b = e % u;
        L[a * u + b] = G[uidx[a] * k + uidx[b]];
    }
    for (int a = tid; a < u; a += PREP_THREADS) {
        gdiag[a] = G[uidx[a] * k + uidx[a]];
        dsq[a] = sqrt(gdiag[a]);
    }
    __syncthreads();
    // Right-looking Cholesky on the lower triangle. Pivot j + 1 is final once
    // its diagonal entry has taken pivot j's update, which thread 0 makes
    // itself (row j + 1 of the trailing triangle is its first row): it forms
    // that pivot's root in the same phase, so each pivot takes two barriers.
    auto pivot = [&](int j) {
        const double d = L[j * u + j];
        if (!(d > PIVOT_TOL64 * gdiag[j])) {
            s_ok = 0;
        } else {
            // One reciprocal square root instead of a root and a division on
            // the pivots' serial path (GB300's FP64 pipe is narrow).
            const double r = rsqrt(d);
            L[j * u + j] = d * r;
            rdiag[j] = r;
        }
    };
    if (tid == 0 && u > 0)
        pivot(0);
    __syncthreads();
    for (int j = 0; j < u; ++j) {
        if (!s_ok)
            break;
        const double rj = rdiag[j];
        for (int i = j + 1 + tid; i < u; i += PREP_THREADS)
            L[i * u + j] *= rj;
        __syncthreads();
        // Trailing lower triangle (a >= b > j): rows by warp, columns by lane.
        for (int a = j + 1 + (tid >> 5); a < u; a += PREP_THREADS / 32) {
            const double laj = L[a * u + j];
            for (int b = j + 1 + (tid & 31); b <= a; b += 32)
                L[a * u + b] = fma(-laj, L[b * u + j], L[a * u + b]);
        }
        if (tid == 0 && j + 1 < u)
            pivot(j + 1);
        __syncthreads();
    }
    if (!s_ok) {
        if (tid == 0) {
            flags[0] = 2;
            flags[1] = u;
            flags[2] = 0;
            atomicAdd(&stats->fp64_halfsteps, 1ull);
        }
        return;
    }
    if (u == k && k >= PREP_SPLIT_K) {
        // L (lower triangle, diagonal included) and 1 / L_aa to the kernels
        // that finish the preparation.
        for (int e = tid; e < k * k; e += PREP_THREADS) {
            const int a = e / k, b = e - a * k;
            if (b <= a)
                M64[e] = L[a * u + b];
        }
        for (int a = tid; a < k; a += PREP_THREADS)
            prep[a] = rdiag[a];
        if (tid == 0) {
            prep[k] = 0.0;
            prep[k + 1] = 0.0;
            flags[2] = 1;
            flags[3] = 0;
        }
        return;
    }
    if (tid == 0)
        flags[2] = 0;
    // Columns of L^{-1} by forward substitution, one column per thread, into
    // the strict upper triangle of L (transposed).
    for (int c = tid; c < u; c += PREP_THREADS) {
        for (int a = c + 1; a < u; ++a) {
            double s = -L[a * u + c] * rdiag[c];
            for (int b = c + 1; b < a; ++b)
                s = fma(-L[a * u + b], L[c * u + b], s);
            L[c * u + a] = s * rdiag[a];
        }
    }
    __syncthreads();
    // M = L^{-T} L^{-1}: M_ab = sum_{c >= max(a, b)} (L^{-1})_ca (L^{-1})_cb,
    // for a <= b, written to both triangles of M64 and M32.
    for (int e = tid; e < u * (u + 1) / 2; e += PREP_THREADS) {
        const int b = tri_row(e), a = e - b * (b + 1) / 2;   // a <= b
        double s = (a == b ? rdiag[b] : L[a * u + b]) * rdiag[b];
        for (int c = b + 1; c < u; ++c)
            s = fma(L[a * u + c], L[b * u + c], s);
        const int ga = uidx[a], gb = uidx[b];
        M64[ga * k + gb] = s;
        M64[gb * k + ga] = s;
        M32[ga * k + gb] = (float)s;
        M32[gb * k + ga] = (float)s;
    }
    __syncthreads();
    // Scaled cond_1 = max column sum of |G_ac| / (d_a d_c) times max column
    // sum of |M_ac| d_a d_c, d_a = sqrt(G_aa). Non-negative doubles order like
    // their bit patterns, so an integer max reduces them.
    for (int c = tid; c < u; c += PREP_THREADS) {
        double sg = 0.0, sm2 = 0.0;
        for (int a = 0; a < u; ++a) {
            sg += fabs(G[uidx[a] * k + uidx[c]]) / dsq[a];
            sm2 += fabs(M64[uidx[a] * k + uidx[c]]) * dsq[a];
        }
        sg /= dsq[c];
        sm2 *= dsq[c];
        atomicMax(&s_norm[0], (unsigned long long)__double_as_longlong(sg));
        atomicMax(&s_norm[1], (unsigned long long)__double_as_longlong(sm2));
    }
    __syncthreads();
    if (tid == 0) {
        const double cond = __longlong_as_double((long long)s_norm[0]) *
                            __longlong_as_double((long long)s_norm[1]);
        const int mode = cond <= COND_FP32 ? 0 : 1;
        flags[0] = mode;
        flags[1] = u;
        if (mode)
            atomicAdd(&stats->fp64_halfsteps, 1ull);
    }
}


// (L^{-1})_ac, a > c, into M64[c][a]: one CTA per column c, the column's
// forward substitution in its first warp, right-looking: lane a % 32 keeps
// the pending sum of row a, s_a = -L_ac / L_cc - sum_{c < b < a} L_ab x_b,
// adding the terms in increasing b (the order of the single-thread form, so
// the values are the same); once x_b = s_b / L_bb is final its lane
// broadcasts it and every later row takes its term. L's rows from c on are
// staged in shared memory by the whole CTA first.
constexpr int INV_THREADS = 256;

__global__ void __launch_bounds__(INV_THREADS)
    bpp_prep_inv_kernel(int k, double *__restrict__ M64, const double *__restrict__ prep,
                        const int *__restrict__ flags)
{
    if (flags[2] != 1)
        return;
    extern __shared__ double inv_sm[];
    double *Ls = inv_sm;               // k x k (lower triangle, rows c and on)
    const int c = blockIdx.x;
    for (int e = c * k + (int)threadIdx.x; e < k * k; e += INV_THREADS) {
        const int a = e / k, b = e - a * k;
        Ls[e] = b <= a ? M64[e] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x >= 32)
        return;
    const int lane = threadIdx.x;
    constexpr int T = (NMF_MAX_K + 31) / 32;
    const double rc = prep[c];
    double sr[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int a = lane + 32 * t;
        sr[t] = (a > c && a < k) ? -Ls[a * k + c] * rc : 0.0;
    }
    for (int b = c + 1; b < k; ++b) {
        const int owner = b & 31, slot = b >> 5;
        double mine = 0.0;
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (t == slot)
                mine = sr[t];
        const double xb = __shfl_sync(FULL, mine * prep[b], owner);
        if (lane == owner)
            M64[c * k + b] = xb;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int a = lane + 32 * t;
            if (a > b && a < k)
                sr[t] = fma(-Ls[a * k + b], xb, sr[t]);
        }
    }
}

// M_ab = sum_{c >= a} (L^{-1})_ca (L^{-1})_cb for a >= b into M64[a][b] (and
// M32 both ways): one CTA per column b, one warp per entry.
__global__ void __launch_bounds__(128)
    bpp_prep_m_kernel(int k, double *__restrict__ M64, float *__restrict__ M32,
                      const double *__restrict__ prep, const int *__restrict__ flags)
{
    if (flags[2] != 1)
        return;
    const int b = blockIdx.x, lane = threadIdx.x & 31;
    for (int a = b + (threadIdx.x >> 5); a < k; a += 4) {
        double part = 0.0;
        for (int c = a + lane; c < k; c += 32) {
            const double xa = c == a ? prep[a] : M64[a * k + c];
            const double xb = c == b ? prep[b] : M64[b * k + c];
            part = fma(xa, xb, part);
        }
        const double m = warp_sum_d(part);
        if (lane == 0) {
            M64[a * k + b] = m;
            M32[a * k + b] = (float)m;
            M32[b * k + a] = (float)m;
        }
    }
}

// Column c of the scaled cond_1 (max column sum of |G_ac| / (d_a d_c) and of
// |M_ac| d_a d_c, d_a = sqrt(G_aa)) from M's lower triangle, and M's upper
// triangle in column c; the last CTA sets the mode.
__global__ void __launch_bounds__(32)
    bpp_prep_cond_kernel(const double *__restrict__ G, int k, double *__restrict__ M64,
                         double *__restrict__ prep, int *__restrict__ flags,
                         BppStats *__restrict__ stats)
{
    if (flags[2] != 1)
        return;
    const int c = blockIdx.x, lane = threadIdx.x;
    double sg = 0.0, sm = 0.0;
    for (int a = lane; a < k; a += 32) {
        const double da = sqrt(G[a * k + a]);
        sg += fabs(G[a * k + c]) / da;
        sm += fabs(a >= c ? M64[a * k + c] : M64[c * k + a]) * da;
    }
    const double dc = sqrt(G[c * k + c]);
    sg = warp_sum_d(sg) / dc;
    sm = warp_sum_d(sm) * dc;
    for (int a = lane; a < c; a += 32)
        M64[a * k + c] = M64[c * k + a];
    if (lane == 0) {
        unsigned long long *norm = reinterpret_cast<unsigned long long *>(prep + k);
        // Non-negative doubles order like their bit patterns.
        atomicMax(&norm[0], (unsigned long long)__double_as_longlong(sg));
        atomicMax(&norm[1], (unsigned long long)__double_as_longlong(sm));
        __threadfence();
        if (atomicAdd(&flags[3], 1) == k - 1) {
            __threadfence();
            const double cond = __longlong_as_double((long long)atomicAdd(&norm[0], 0ull)) *
                                __longlong_as_double((long long)atomicAdd(&norm[1], 0ull));
            const int mode = cond <= COND_FP32 ? 0 : 1;
            flags[0] = mode;
            flags[1] = k;
            flags[2] = 0;
            if (mode)
                atomicAdd(&stats->fp64_halfsteps, 1ull);
        }
    }
}


// FP64 Cholesky of S_ab = Src[idx[a] * ld + idx[b]], right-looking: after
// each pivot the trailing lower triangle is updated with its (a, b) entries
// spread over the 32 lanes. Output: L in the lower triangle of Lw (row stride
// LS), invd = 1 / L_jj; false, uniformly across the warp, on a pivot
// <= tol * S_jj. The FP64 solves are bound by GB300's narrow FP64 pipe (two
// lanes per clock per SM). The lane-per-row form gave step j to rows a >= j,
// j FMAs each: p^2 / 2 warp FMA instructions with most lanes idle. The
// trailing update takes about p^3 / 192 + p.
__device__ bool warp_chol_factor_rl(const double *__restrict__ Src, int ld,
                                    const int *__restrict__ idx, int p, double *__restrict__ Lw,
                                    int LS, double *__restrict__ invd, double tol, int lane)
{
    for (int e = lane; e < p * (p + 1) / 2; e += 32) {
        const int a = tri_row(e), b = e - a * (a + 1) / 2;
        Lw[a * LS + b] = Src[idx[a] * ld + idx[b]];
    }
    __syncwarp();
    for (int j = 0; j < p; ++j) {
        const double d = Lw[j * LS + j];
        const double dorig = Src[idx[j] * ld + idx[j]];
        if (!(d > tol * dorig))
            return false;
        const double l = sqrt(d);
        const double inv = 1.0 / l;
        for (int a = j + 1 + lane; a < p; a += 32)
            Lw[a * LS + j] *= inv;
        __syncwarp();
        if (lane == 0) {
            Lw[j * LS + j] = l;
            invd[j] = inv;
        }
        const int t = p - j - 1;
        for (int e = lane; e < t * (t + 1) / 2; e += 32) {
            const int a = tri_row(e), b = e - a * (a + 1) / 2;
            const int ra = j + 1 + a, rb = j + 1 + b;
            Lw[ra * LS + rb] -= Lw[ra * LS + j] * Lw[rb * LS + j];
        }
        __syncwarp();
    }
    return true;
}

// Solve L L^T z = r with the factor from warp_chol_factor_rl; row a of r / z in
// lane a % 32, slot a / 32 (shuffle-broadcast substitutions).
template <typename T, int PT>
__device__ void warp_chol_subst(int p, const T *__restrict__ Lw, int LS,
                                const T *__restrict__ invd, T (&r)[PT], int lane)
{
    for (int j = 0; j < p; ++j) {
        const int tj = j >> 5, owner = j & 31;
        T rj = r[0];
#pragma unroll
        for (int t = 1; t < PT; ++t)
            if (tj == t)
                rj = r[t];
        const T zj = __shfl_sync(FULL, rj, owner) * invd[j];
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int i = lane + 32 * t;
            if (i > j && i < p)
                r[t] -= Lw[i * LS + j] * zj;
            if (t == tj && lane == owner)
                r[t] = zj;
        }
    }
    for (int j = p - 1; j >= 0; --j) {
        const int tj = j >> 5, owner = j & 31;
        T rj = r[0];
#pragma unroll
        for (int t = 1; t < PT; ++t)
            if (tj == t)
                rj = r[t];
        const T xj = __shfl_sync(FULL, rj, owner) * invd[j];
        const T *lj = Lw + j * LS;
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int i = lane + 32 * t;
            if (i < j)
                r[t] -= lj[i] * xj;
            if (t == tj && lane == owner)
                r[t] = xj;
        }
    }
    __syncwarp();
}

template <typename T, int KW>
__device__ __forceinline__ void warp_matvec(const T *__restrict__ Mat, int k, const T (&v)[KW],
                                            T (&out)[KW], T *__restrict__ stage, int lane)
{
#pragma unroll
    for (int s = 0; s < KW; ++s)
        stage[32 * s + lane] = v[s];
    __syncwarp();
    int j = 0;
    for (; j + 4 <= k; j += 4) {
        T vj[4];
        if constexpr (sizeof(T) == 4) {
            const float4 q = *reinterpret_cast<const float4 *>(stage + j);
            vj[0] = q.x;
            vj[1] = q.y;
            vj[2] = q.z;
            vj[3] = q.w;
        } else {
            const double2 q0 = *reinterpret_cast<const double2 *>(stage + j);
            const double2 q1 = *reinterpret_cast<const double2 *>(stage + j + 2);
            vj[0] = q0.x;
            vj[1] = q0.y;
            vj[2] = q1.x;
            vj[3] = q1.y;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const T *row = Mat + (j + t) * k;
#pragma unroll
            for (int s = 0; s < KW; ++s) {
                const int i = lane + 32 * s;
                if (i < k)
                    out[s] = fma(row[i], vj[t], out[s]);
            }
        }
    }
    for (; j < k; ++j) {
        const T vj = stage[j];
        const T *row = Mat + j * k;
#pragma unroll
        for (int s = 0; s < KW; ++s) {
            const int i = lane + 32 * s;
            if (i < k)
                out[s] = fma(row[i], vj, out[s]);
        }
    }
    __syncwarp();
}

// Per warp: index list (128 ints), right-hand side and reciprocal pivots of
// the compact system (128 doubles each), the matrix-vector staging vector
// (128 doubles), the p x LS factor; rounded to 16 bytes.
__host__ __device__ inline size_t per_warp_bytes(int pmax, int LS)
{
    const size_t b = 128 * sizeof(int) + 384 * sizeof(double) + sizeof(double) * (size_t)pmax * LS;
    return (b + 15) & ~size_t(15);
}

// Shared-memory matrices of a mode: mode 1 G64 and M64, mode 2 none (no M;
// G64 read through L1/L2).
__host__ __device__ inline size_t mats_bytes(int k, int mode)
{
    const size_t b = mode == 1 ? 2 * sizeof(double) * (size_t)k * k : 0;
    return (b + 15) & ~size_t(15);
}

// FP64 solves. KW = index slots per lane (k <= 32 KW); PT = compact-system
// rows per lane (pmax <= 32 PT). The kernel of each MODE returns at once
// unless the prep kernel chose that mode, so the host never waits for the
// decision. With list_pass set (MODE 1 only) it is the second pass of mode 0:
// it re-solves, from their starting partitions, the right-hand sides that the
// FP32 kernel deferred (all of them if more than DEFER_CAP were).
template <int KW, int PT, int MODE>
__global__ void __launch_bounds__(BPP_THREADS, 2)
    bpp_solve_kernel(const SolveParams P, int pmax, int LS, int staged, int list_pass)
{
    using T = double;
    constexpr bool HAVE_M = MODE != 2;
    int64_t nwork = P.nrhs;
    bool use_list = false;
    unsigned long long *counter = &P.counters[CNT_WORK];
    if (list_pass) {
        if (P.flags[0] != 0)
            return;
        // Written by the FP32 kernel earlier in the same stream.
        const unsigned long long nd = P.counters[CNT_DEFERRED];
        if (nd == 0)
            return;
        use_list = nd <= (unsigned long long)DEFER_CAP;
        nwork = use_list ? (int64_t)nd : P.nrhs;
        counter = &P.counters[CNT_DEFER_WORK];
    } else if (P.flags[0] != MODE) {
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = P.k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *Gs;
    const T *Ms = nullptr;
    if (!staged) {
        // Matrices too large for shared memory next to the per-warp space:
        // read them through L1/L2 (mode 1 at k > ~100, mode 2 always).
        Gs = P.G64;
        if (HAVE_M)
            Ms = P.M64;
    } else {
        T *gsh = reinterpret_cast<T *>(smem_raw);
        T *msh = gsh + k * k;
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            gsh[e] = P.G64[e];
            msh[e] = P.M64[e];
        }
        Gs = gsh;
        Ms = msh;
    }
    unsigned char *wp =
        smem_raw + (staged ? mats_bytes(k, MODE) : 0) + warp * per_warp_bytes(pmax, LS);
    int *widx = reinterpret_cast<int *>(wp);
    T *zbuf = reinterpret_cast<T *>(wp + 128 * sizeof(int));
    T *invd = zbuf + 128;
    T *stage = invd + 128;
    T *Lw = stage + 128;
    __syncthreads();

    bool usable[KW];
    int nU = 0;
#pragma unroll
    for (int s = 0; s < KW; ++s) {
        const uint32_t w = P.usable_words[s];
        usable[s] = (w >> lane) & 1u;
        nU += __popc(w);
    }

    unsigned long long st_rounds = 0, st_max = 0, st_nc = 0, st_sing = 0, st_nf = 0, st_rhs = 0;

    for (;;) {
        unsigned long long j0 = 0;
        if (lane == 0)
            j0 = atomicAdd(counter, (unsigned long long)P.chunk);
        j0 = __shfl_sync(FULL, j0, 0);
        if (j0 >= (unsigned long long)nwork)
            break;
        const int64_t jend = min((int64_t)j0 + P.chunk, nwork);
        for (int64_t jj = (int64_t)j0; jj < jend; ++jj) {
            const int64_t j = use_list ? P.defer[jj] : jj;
            T g[KW], u[KW], x[KW], y[KW];
            bool inF[KW];
            bool bad = false;
#pragma unroll
            for (int s = 0; s < KW; ++s) {
                const int i = lane + 32 * s;
                g[s] = i < k ? (T)P.B[j * k + i] : (T)0;
                bad |= !isfinite(g[s]);
                u[s] = 0;
                x[s] = 0;
                y[s] = -g[s];
                inF[s] = false;
            }
            bad = __any_sync(FULL, bad);
            int status = NMF_OK;
            int rounds = 0;
            if (bad) {
                status = NMF_ERR_NONFINITE;
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    x[s] = 0;
            } else {
                // Starting partition: empty (cold) or the given bitmask (warm).
                if (P.pin) {
#pragma unroll
                    for (int s = 0; s < KW; ++s) {
                        const int i = lane + 32 * s;
                        bool f = false;
                        if (i < k) {
                            const uint64_t wv = P.pin[j * P.nwords + (i >> 6)];
                            f = (wv >> (i & 63)) & 1ull;
                        }
                        inF[s] = f && usable[s];
                    }
                }
                bool have_u = false;   // u = M g, formed when a complement solve first needs it

                // Candidate point of the current partition: fills x and y.
                auto solve = [&]() -> int {
                    int nF = 0;
#pragma unroll
                    for (int s = 0; s < KW; ++s)
                        nF += __popc(__ballot_sync(FULL, inF[s]));
                    const int nA = nU - nF;
                    const bool comp = HAVE_M && nA < nF;
                    if (comp && !have_u) {
                        warp_matvec<T, KW>(Ms, k, g, u, stage, lane);
                        have_u = true;
                    }
                    bool inS[KW];
                    int rank[KW];
                    int pos = 0;
#pragma unroll
                    for (int s = 0; s < KW; ++s) {
                        inS[s] = comp ? (usable[s] && !inF[s]) : inF[s];
                        const unsigned mk = __ballot_sync(FULL, inS[s]);
                        rank[s] = pos + __popc(mk & lanemask_lt(lane));
                        if (inS[s]) {
                            widx[rank[s]] = lane + 32 * s;
                            zbuf[rank[s]] = comp ? -u[s] : g[s];
                        }
                        pos += __popc(mk);
                    }
                    const int p = pos;
                    __syncwarp();
                    if (p > 0) {
                        if (!warp_chol_factor_rl(comp ? Ms : Gs, k, widx, p, Lw, LS, invd,
                                                 PIVOT_TOL64, lane))
                            return NMF_ERR_SINGULAR_GRAM;
                        T r[PT];
#pragma unroll
                        for (int t = 0; t < PT; ++t) {
                            const int a = lane + 32 * t;
                            r[t] = a < p ? zbuf[a] : (T)0;
                        }
                        warp_chol_subst<T, PT>(p, Lw, LS, invd, r, lane);
#pragma unroll
                        for (int t = 0; t < PT; ++t) {
                            const int a = lane + 32 * t;
                            if (a < p)
                                zbuf[a] = r[t];
                        }
                        __syncwarp();
                    }
                    // The compact solution z (zbuf, p entries) against the
                    // rows it touches: x_F = u_F + M_FA z in the complement
                    // form; y = G_{:,F} x_F - g in the direct form. Both loop
                    // over the p-entry list, not over all k rows.
                    const T *Lst = comp ? Ms : Gs;
                    T acc[KW];
#pragma unroll
                    for (int s = 0; s < KW; ++s)
                        acc[s] = comp ? u[s] : -g[s];
                    for (int a = 0; a < p; ++a) {
                        const T za = zbuf[a];
                        const T *row = Lst + widx[a] * k;
#pragma unroll
                        for (int s = 0; s < KW; ++s) {
                            const int i = lane + 32 * s;
                            if (i < k)
                                acc[s] = fma(row[i], za, acc[s]);
                        }
                    }
#pragma unroll
                    for (int s = 0; s < KW; ++s) {
                        if (comp) {
                            // y_A is the complement solution itself (accurate in FP64).
                            x[s] = inF[s] ? acc[s] : (T)0;
                            y[s] = inS[s] ? zbuf[rank[s]] : (inF[s] ? (T)0 : -g[s]);
                        } else {
                            x[s] = inF[s] ? zbuf[rank[s]] : (T)0;
                            y[s] = inF[s] ? (T)0 : acc[s];
                        }
                    }
                    __syncwarp();
                    return NMF_OK;
                };

                // One solve per exchange round, from a single call site.
                bool anyF = false;
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    anyF |= inF[s];
                bool need = __any_sync(FULL, anyF);   // else x = 0, y = -g already
                int alpha = 3, beta = k + 1;
                for (;;) {
                    if (need) {
                        status = solve();
                        if (status != NMF_OK)
                            break;
                    }
                    need = true;
                    bool inf[KW];
                    unsigned vm[KW];
                    int nV = 0;
#pragma unroll
                    for (int s = 0; s < KW; ++s) {
                        inf[s] = usable[s] && (inF[s] ? (x[s] < (T)0) : (y[s] < (T)0));
                        vm[s] = __ballot_sync(FULL, inf[s]);
                        nV += __popc(vm[s]);
                    }
                    if (nV == 0)
                        break;
                    if (rounds >= P.max_rounds) {
                        status = NMF_ERR_NOT_CONVERGED;
                        break;
                    }
                    if (nV < beta || alpha >= 1) {   // full exchange
                        if (nV < beta) {
                            beta = nV;
                            alpha = 3;
                        } else {
                            alpha -= 1;
                        }
#pragma unroll
                        for (int s = 0; s < KW; ++s)
                            inF[s] = inF[s] != inf[s];
                    } else {   // backup rule: the largest infeasible index alone
                        int top = -1;
#pragma unroll
                        for (int s = KW - 1; s >= 0; --s)
                            if (top < 0 && vm[s])
                                top = 32 * s + 31 - __clz(vm[s]);
#pragma unroll
                        for (int s = 0; s < KW; ++s)
                            if (lane + 32 * s == top)
                                inF[s] = !inF[s];
                    }
                    rounds += 1;
                }
                bool nf = false;
#pragma unroll
                for (int s = 0; s < KW; ++s) {
                    x[s] = x[s] > (T)0 ? x[s] : (T)0;
                    nf |= !isfinite(x[s]);
                }
                if (__any_sync(FULL, nf) && status == NMF_OK)
                    status = NMF_ERR_NONFINITE;
            }
#pragma unroll
            for (int s = 0; s < KW; ++s) {
                const int i = lane + 32 * s;
                if (i < k)
                    P.X[j * k + i] = (float)x[s];
            }
            if (P.pout) {
                unsigned bm[KW];
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    bm[s] = __ballot_sync(FULL, inF[s]);
                if (lane == 0) {
#pragma unroll
                    for (int w = 0; w < (KW + 1) / 2; ++w) {
                        const uint64_t lo = bm[2 * w];
                        const uint64_t hi = (2 * w + 1 < KW) ? bm[2 * w + 1] : 0u;
                        P.pout[j * P.nwords + w] = lo | (hi << 32);
                    }
                }
            }
            if (lane == 0) {
                if (P.rounds_out)
                    P.rounds_out[j] = rounds;
                if (P.status_out)
                    P.status_out[j] = (int8_t)status;
                st_rhs += 1;
                st_rounds += rounds;
                st_max = st_max > (unsigned long long)rounds ? st_max : (unsigned long long)rounds;
                st_nc += status == NMF_ERR_NOT_CONVERGED;
                st_sing += status == NMF_ERR_SINGULAR_GRAM;
                st_nf += status == NMF_ERR_NONFINITE;
            }
        }
    }
    // (After an overflow of the deferral list the second pass re-solves the
    // whole batch, and the right-hand-side and round counts include both
    // passes.)
    if (lane == 0 && st_rhs) {
        atomicAdd(&P.stats->rhs, st_rhs);
        atomicAdd(&P.stats->rounds, st_rounds);
        atomicMax(&P.stats->max_rounds, st_max);
        if (st_nc) atomicAdd(&P.stats->not_converged, st_nc);
        if (st_sing) atomicAdd(&P.stats->singular, st_sing);
        if (st_nf) atomicAdd(&P.stats->nonfinite, st_nf);
    }
}

constexpr size_t SMEM_LIMIT = 227 * 1024;

template <int KW, int PT, int MODE>
nmf_status launch_solve(const SolveParams &P, int list_pass, cudaStream_t s)
{
    const int k = P.k;
    int pmax = MODE == 2 ? k : k / 2;
    if (pmax < 1)
        pmax = 1;
    const int LS = pmax | 1;   // odd row stride: conflict-free lane-per-row reads
    int nwarps = P.warps < BPP_WARPS ? P.warps : BPP_WARPS;
    // Stage G and M in shared memory when they leave room for >= 2 warps.
    const int staged = MODE != 2 &&
                       mats_bytes(k, MODE) + 2 * per_warp_bytes(pmax, LS) <= SMEM_LIMIT;
    const size_t mats = staged ? mats_bytes(k, MODE) : 0;
    auto bytes = [&](int nw) { return mats + (size_t)nw * per_warp_bytes(pmax, LS); };
    while (nwarps > 1 && bytes(nwarps) > SMEM_LIMIT)
        --nwarps;
    const size_t smem = bytes(nwarps);
    if (smem > SMEM_LIMIT)
        return NMF_ERR_INVALID_ARG;
    static SmemOptIn opt_in;
    NMF_TRY(ensure_smem(bpp_solve_kernel<KW, PT, MODE>, opt_in, smem));
    int per_sm = 0;
    NMF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, bpp_solve_kernel<KW, PT, MODE>, nwarps * 32, smem));
    if (per_sm < 1)
        return NMF_ERR_INVALID_ARG;
    int64_t blocks = (int64_t)per_sm * sm_count();
    // The second pass's size is known only on the device: launch it at full
    // width; it returns at once when nothing was deferred.
    const int64_t need = list_pass ? blocks : cdiv(cdiv(P.nrhs, (int64_t)P.chunk), nwarps);
    if (need < blocks)
        blocks = need < 1 ? 1 : need;
    bpp_solve_kernel<KW, PT, MODE><<<(unsigned)blocks, nwarps * 32, smem, s>>>(P, pmax, LS,
                                                                              staged, list_pass);
    NMF_LAUNCHED("bpp_solve_kernel");
    return NMF_OK;
}

template <int KW>
nmf_status launch_modes(const SolveParams &P, cudaStream_t s)
{
    // Mode 0 (FP32): the group-tile pass for the all-passive group first,
    // then the per-warp solves of what it left.
    if (P.group && !P.fused) {
        if (P.group == 2)
            NMF_TRY(launch_group_tc(P, s));
        else
            NMF_TRY(launch_group32(P, s));
    }
    NMF_TRY(launch_solve32(P, s));
    if (P.fused) {
        // FP64 half-step: the right-hand sides are formed here instead.
        NMF_TRY(launch_spmm_unless_fp32(P.gat.rowptr, P.gat.colidx, P.gat.vals, P.nrhs, P.gat.F,
                                        P.k, const_cast<float *>(P.B), P.flags, s));
    }
    // Mode 1 (FP64): an FP32 pass first predicts each right-hand side's
    // partition into pout, and the FP64 solves start from it (their answer
    // does not depend on the start; they need fewer rounds).
    SolveParams P1 = P;
    if (P.pout && P.max_rounds >= 2 * PREDICT_ROUNDS) {   // (a tight cap keeps its meaning)
        SolveParams Q = P;
        Q.predict = 1;
        Q.group = 0;
        Q.fused = 0;
        NMF_TRY(launch_solve32(Q, s));
        P1.pin = P.pout;
    }
    NMF_TRY((launch_solve<KW, (KW + 1) / 2, 1>(P1, 0, s)));
    NMF_TRY((launch_solve<KW, KW, 2>(P, 0, s)));
    return launch_solve<KW, (KW + 1) / 2, 1>(P, 1, s);
}

}  // namespace

size_t bpp_work_bytes(int k) { return layout(k).total; }

namespace {

// Launch shape of the solve kernels per k (warps per CTA, right-hand sides per
// grab of the work counter, whether the group-tile pass runs first):
// {8, 8, group pass on} until bpp_tune has measured the batch or the caller
// set one; the group pass runs on the tensor cores (2) for 65 <= k <= 112,
// else on the SIMT pipes (1). Shapes with group 0 or 1 compute the same results
// (a right-hand side's arithmetic does not depend on where it runs); group 2
// solves the all-passive group with tensor-core products, to FP32 accuracy
// but not the same bits.
struct BppShape {
    int warps = BPP_WARPS, chunk = 8, group = -1;   // -1: the default for k
};
std::mutex g_shape_mu;
BppShape g_shape[NMF_MAX_K + 1];

BppShape shape_for(int k)
{
    std::lock_guard<std::mutex> lock(g_shape_mu);
    BppShape sh = g_shape[k];
    if (sh.group < 0)   // measured: the tensor-core pass wins from k = 65 (k = 100: 2.5x), the
                        // SIMT pass at k = 50 (dense ANLS, 127.1 against 126.4 iter/s)
        sh.group = k >= 65 && group_tc_supported(k) ? 2 : 1;
    return sh;
}

SolveParams solve_params(int k, int64_t nrhs, const double *G, const float *B, float *X,
                         const uint64_t *passive_in, uint64_t *passive_out, int32_t *rounds_out,
                         int8_t *status_out, int max_rounds, void *work, BppStats *stats_dev)
{
    const WorkLayout L = layout(k);
    unsigned char *w = static_cast<unsigned char *>(work);
    SolveParams P;
    P.k = k;
    P.nwords = (k + 63) / 64;
    P.max_rounds = max_rounds;
    P.nrhs = nrhs;
    P.G32 = reinterpret_cast<float *>(w + L.g32);
    P.M32 = reinterpret_cast<float *>(w + L.m32);
    P.G64 = G;
    P.M64 = reinterpret_cast<double *>(w + L.m64);
    P.usable_words = reinterpret_cast<uint32_t *>(w + L.usable);
    P.flags = reinterpret_cast<int *>(w + L.flags);
    P.B = B;
    P.X = X;
    P.pin = passive_in;
    P.pout = passive_out;
    P.rounds_out = rounds_out;
    P.status_out = status_out;
    P.counters = reinterpret_cast<unsigned long long *>(w + L.counters);
    P.predict = 0;
    P.fused = 0;
    P.gat = CsrGather{nullptr, nullptr, nullptr, nullptr};
    P.defer = reinterpret_cast<int64_t *>(w + L.defer);
    P.stats = stats_dev;
    const BppShape sh = shape_for(k);
    P.warps = sh.warps;
    P.chunk = sh.chunk;
    P.group = sh.group;
    return P;
}

nmf_status launch_solves(const SolveParams &P, cudaStream_t s)
{
    if (P.k <= 32)
        return launch_modes<1>(P, s);
    if (P.k <= 64)
        return launch_modes<2>(P, s);
    if (P.k <= 96)
        return launch_modes<3>(P, s);
    return launch_modes<4>(P, s);
}

}  // namespace

nmf_status launch_bpp_prep(int k, const double *G, void *work, BppStats *stats_dev, cudaStream_t s)
{
    const SolveParams P = solve_params(k, 0, G, nullptr, nullptr, nullptr, nullptr, nullptr,
                                       nullptr, 0, work, stats_dev);
    const size_t prep_smem = sizeof(double) * ((size_t)k * k + 3 * k) + sizeof(int) * (size_t)k;
    static SmemOptIn opt_in;
    NMF_TRY(ensure_smem(bpp_prep_kernel, opt_in, prep_smem));
    double *prep = reinterpret_cast<double *>(static_cast<unsigned char *>(work) + layout(k).prep);
    bpp_prep_kernel<<<1, PREP_THREADS, prep_smem, s>>>(
        G, k, const_cast<float *>(P.G32), const_cast<float *>(P.M32),
        const_cast<double *>(P.M64), const_cast<uint32_t *>(P.usable_words),
        const_cast<int *>(P.flags), P.counters, stats_dev, prep);
    NMF_LAUNCHED("bpp_prep_kernel");
    if (k >= PREP_SPLIT_K) {   // (each returns at once unless the prep left them the work)
        const size_t inv_smem = sizeof(double) * (size_t)k * k;
        static SmemOptIn inv_opt_in;
        NMF_TRY(ensure_smem(bpp_prep_inv_kernel, inv_opt_in, inv_smem));
        bpp_prep_inv_kernel<<<(unsigned)k, INV_THREADS, inv_smem, s>>>(
            k, const_cast<double *>(P.M64), prep, P.flags);
        NMF_LAUNCHED("bpp_prep_inv_kernel");
        bpp_prep_m_kernel<<<(unsigned)k, 128, 0, s>>>(k, const_cast<double *>(P.M64),
                                                      const_cast<float *>(P.M32), prep, P.flags);
        NMF_LAUNCHED("bpp_prep_m_kernel");
        bpp_prep_cond_kernel<<<(unsigned)k, 32, 0, s>>>(G, k, const_cast<double *>(P.M64), prep,
                                                       const_cast<int *>(P.flags), stats_dev);
        NMF_LAUNCHED("bpp_prep_cond_kernel");
    }
    return NMF_OK;
}

nmf_status launch_bpp_solve(int k, int64_t nrhs, const double *G, const float *B, float *X,
                            const uint64_t *passive_in, uint64_t *passive_out, int32_t *rounds_out,
                            int8_t *status_out, int max_rounds, void *work, BppStats *stats_dev,
                            cudaStream_t s, const CsrGather *gather)
{
    if (nrhs == 0)
        return NMF_OK;
    SolveParams P = solve_params(k, nrhs, G, B, X, passive_in, passive_out, rounds_out,
                                 status_out, max_rounds, work, stats_dev);
    if (gather) {
        P.fused = 1;
        P.gat = *gather;
    }
    return launch_solves(P, s);
}

// Times every candidate launch shape on this batch (after one warm-up each;
// the passive-set, round and status outputs are left out so every candidate
// starts from the same partitions) and keeps the fastest for k. X receives
// the solution.
nmf_status bpp_tune(int k, int64_t nrhs, const double *G, const float *B, float *X,
                    const uint64_t *passive_in, int max_rounds, void *work, BppStats *stats_dev,
                    cudaStream_t s, int *warps_out, int *chunk_out, int *group_out)
{
    // The candidates keep the group mode of the current shape (and try the
    // pass off only beside the SIMT pass, whose results it shares), so every
    // candidate gives the same bits.
    const int gm = shape_for(k).group;
    const BppShape cand[] = {{16, 4, gm}, {16, 8, gm}, {8, 1, gm},  {8, 4, gm},
                             {8, 8, gm},  {8, 32, gm}, {4, 16, gm}, {8, 8, gm == 1 ? 0 : gm}};
    NMF_TRY(launch_bpp_prep(k, G, work, stats_dev, s));
    SolveParams P = solve_params(k, nrhs, G, B, X, passive_in, nullptr, nullptr, nullptr,
                                 max_rounds, work, stats_dev);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NMF_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return NMF_ERR_CUDA;
    }
    BppShape best;
    float best_ms = -1.0f;
    nmf_status st = NMF_OK;
    for (const BppShape &c : cand) {
        P.warps = c.warps;
        P.chunk = c.chunk;
        P.group = c.group;
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && st == NMF_OK; ++rep) {
            // The prep kernel resets the work counter; re-run it per solve.
            st = launch_bpp_prep(k, G, work, stats_dev, s);
            if (st == NMF_OK && cudaEventRecord(e0, s) != cudaSuccess)
                st = NMF_ERR_CUDA;
            if (st == NMF_OK)
                st = launch_solves(P, s);
            if (st == NMF_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                 cudaEventSynchronize(e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                st = NMF_ERR_CUDA;
        }
        if (st != NMF_OK)
            break;
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    NMF_TRY(st);
    {
        std::lock_guard<std::mutex> lock(g_shape_mu);
        g_shape[k] = best;
    }
    if (warps_out)
        *warps_out = best.warps;
    if (chunk_out)
        *chunk_out = best.chunk;
    if (group_out)
        *group_out = best.group;
    return NMF_OK;
}

nmf_status bpp_set_shape(int k, int warps, int chunk, int group)
{
    if (k < 1 || k > NMF_MAX_K || warps < 1 || warps > 16 || chunk < 1 || chunk > 1024 ||
        group < 0 || group > 2 || (group == 2 && !group_tc_supported(k)))
        return NMF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_shape_mu);
    g_shape[k].warps = warps;
    g_shape[k].chunk = chunk;
    g_shape[k].group = group;
    return NMF_OK;
}

nmf_status bpp_get_shape(int k, int *warps, int *chunk, int *group)
{
    if (k < 1 || k > NMF_MAX_K)
        return NMF_ERR_INVALID_ARG;
    const BppShape sh = shape_for(k);
    if (warps)
        *warps = sh.warps;
    if (chunk)
        *chunk = sh.chunk;
    if (group)
        *group = sh.group;
    return NMF_OK;
}

nmf_status launch_bpp(int k, int64_t nrhs, const double *G, const float *B, float *X,
                      const uint64_t *passive_in, uint64_t *passive_out, int32_t *rounds_out,
                      int8_t *status_out, int max_rounds, void *work, BppStats *stats_dev,
                      cudaStream_t s)
{
    NMF_TRY(launch_bpp_prep(k, G, work, stats_dev, s));
    return launch_bpp_solve(k, nrhs, G, B, X, passive_in, passive_out, rounds_out, status_out,
                            max_rounds, work, stats_dev, s);
}

}  // namespace nmf
