// FP32 solves of batched BPP (Eq. 3, Eq. 4, Sec. 4.2) for Grams whose
// diagonally scaled cond_1 the preparation found at most 1e4 (mode 0).
//
// Same method as the FP64 kernel in bpp.cu: one warp per right-hand side,
// lane l holding indices l, l + 32, ... (KW slots); each exchange round solves
// the smaller of the direct system G_FF x_F = g_F and the complement system
// M_AA y_A = -u_A (u = M g, x_F = u_F + M_FA y_A), refines once through the
// same factor, recomputes y = G x - g, and tests the signs with the FP32
// tolerances in the diagonally scaled variables. Organised for fewer
// instructions per solve:
//  * G and M sit in shared memory lane-interleaved: entry (r, c) at
//    r * 32 KW + (c % 32) * KW + c / 32, so a lane reads its KW entries of a
//    row with one vector load and updates them with packed FP32x2 FMAs;
//  * a product with a vector supported on a short index list (F in the direct
//    form, the active set in the complement form) loops over that list only:
//    y = G_{:,F} x_F costs |F| row reads, not k;
//  * u = M g is formed only when a complement solve first needs it;
//  * k <= 64 (systems of at most k / 2 <= 32 rows): an LDL^T factor whose
//    trailing rows stay in registers, one row per lane, shifted one column per
//    step so that a rolled loop keeps constant register indices; the
//    multipliers go to shared memory for the two substitutions;
//  * k > 64: a left-looking Cholesky that keeps each row's reciprocal pivot in
//    its lane: with q = rsqrt(d), L_jj = d q and L_ij = s_i q;
//  * no FP64 arithmetic: a system that meets the pivot floor defers its
//    right-hand side to the FP64 kernel's second pass, which re-solves it from
//    its starting partition.
#include <math.h>

#include "bpp_internal.cuh"

namespace nmf {
namespace bpp {
namespace {

constexpr int S32_MAX_WARPS = 16;
constexpr int DEFERRED = -1;   // internal status: re-solve this right-hand side in FP64
constexpr size_t SMEM_LIMIT32 = 227 * 1024;

// acc[s] += p[s] * a for the KW entries of one row that a lane owns.
template <int KW>
__device__ __forceinline__ void row_fma(const float *__restrict__ p, float a, float (&acc)[KW])
{
    if constexpr (KW == 1) {
        acc[0] = fmaf(p[0], a, acc[0]);
    } else if constexpr (KW == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        const float2 r = __ffma2_rn(q, make_float2(a, a), make_float2(acc[0], acc[1]));
        acc[0] = r.x;
        acc[1] = r.y;
    } else {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        const float2 r0 =
            __ffma2_rn(make_float2(q.x, q.y), make_float2(a, a), make_float2(acc[0], acc[1]));
        const float2 r1 =
            __ffma2_rn(make_float2(q.z, q.w), make_float2(a, a), make_float2(acc[2], acc[3]));
        acc[0] = r0.x;
        acc[1] = r0.y;
        acc[2] = r1.x;
        acc[3] = r1.y;
    }
}

// out += Mat^T vec over all rows (vec staged in shared memory, k4 entries,
// zero past k). Two accumulator sets halve the FMA dependency chain.
template <int KW>
__device__ __forceinline__ void mv_full(const float *__restrict__ Mat, int k4,
                                        const float *__restrict__ vec, float (&out)[KW], int lane)
{
    constexpr int RS = 32 * KW;
    float a1[KW];
#pragma unroll
    for (int s = 0; s < KW; ++s)
        a1[s] = 0.0f;
    const float *base = Mat + lane * KW;
    for (int j = 0; j < k4; j += 4) {
        const float4 q = *reinterpret_cast<const float4 *>(vec + j);
        row_fma<KW>(base + (j + 0) * RS, q.x, out);
        row_fma<KW>(base + (j + 1) * RS, q.y, a1);
        row_fma<KW>(base + (j + 2) * RS, q.z, out);
        row_fma<KW>(base + (j + 3) * RS, q.w, a1);
    }
#pragma unroll
    for (int s = 0; s < KW; ++s)
        out[s] += a1[s];
}

// out += sum_a Mat[idx[a]] * val[a] over a list padded to n4 entries (the
// padding has idx 0 and val 0).
template <int KW>
__device__ __forceinline__ void mv_list(const float *__restrict__ Mat, const int *__restrict__ idx,
                                        const float *__restrict__ val, int n4, float (&out)[KW],
                                        int lane)
{
    constexpr int RS = 32 * KW;
    float a1[KW];
#pragma unroll
    for (int s = 0; s < KW; ++s)
        a1[s] = 0.0f;
    const float *base = Mat + lane * KW;
    for (int a = 0; a < n4; a += 4) {
        const int4 c = *reinterpret_cast<const int4 *>(idx + a);
        const float4 v = *reinterpret_cast<const float4 *>(val + a);
        row_fma<KW>(base + c.x * RS, v.x, out);
        row_fma<KW>(base + c.y * RS, v.y, a1);
        row_fma<KW>(base + c.z * RS, v.z, out);
        row_fma<KW>(base + c.w * RS, v.w, a1);
    }
#pragma unroll
    for (int s = 0; s < KW; ++s)
        out[s] += a1[s];
}

template <int KW>
__device__ __forceinline__ void stage_vec(float *__restrict__ stage, const float (&v)[KW], int lane)
{
    __syncwarp();
#pragma unroll
    for (int s = 0; s < KW; ++s)
        stage[32 * s + lane] = v[s];
    __syncwarp();
}

// Cholesky of the p x p system S_ab = Src(idx[a], idx[b]) (lane-per-row,
// left-looking, rows a = lane + 32 t). L goes to Lw (row stride LS, even, so
// that rows are read as float2); inv[t] receives 1 / L_aa for the lane's rows.
// Returns false (uniformly) when a pivot is at most PIVOT_TOL of its diagonal.
template <int KW, int PT>
__device__ __forceinline__ bool chol32(const float *__restrict__ Src, const int *__restrict__ idx,
                                       int p, float *__restrict__ Lw, int LS, float (&inv)[PT],
                                       int lane)
{
    constexpr int RS = 32 * KW;
    int roff[PT], coff[PT];
    float dg[PT];
#pragma unroll
    for (int t = 0; t < PT; ++t) {
        const int a = lane + 32 * t;
        roff[t] = 0;
        coff[t] = 0;
        dg[t] = 1.0f;
        inv[t] = 0.0f;
        if (a < p) {
            const int c = idx[a];
            roff[t] = c * RS;
            coff[t] = (c & 31) * KW + (c >> 5);
            dg[t] = Src[roff[t] + coff[t]];
        }
    }
    for (int j = 0; j < p; ++j) {
        const int tj = j >> 5, owner = j & 31;
        int cj = coff[0];
#pragma unroll
        for (int t = 1; t < PT; ++t)
            if (tj == t)
                cj = coff[t];
        cj = __shfl_sync(FULL, cj, owner);
        const float *lj = Lw + j * LS;
        float sv[PT];
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int a = lane + 32 * t;
            sv[t] = 0.0f;
            if (a >= j && a < p) {
                const float *la = Lw + a * LS;
                float2 acc = make_float2(0.0f, 0.0f);
                int c = 0;
                for (; c + 2 <= j; c += 2)
                    acc = __ffma2_rn(*reinterpret_cast<const float2 *>(la + c),
                                     *reinterpret_cast<const float2 *>(lj + c), acc);
                float s = Src[roff[t] + cj] - (acc.x + acc.y);
                if (c < j)
                    s = fmaf(-la[c], lj[c], s);
                sv[t] = s;
            }
        }
        float q = 0.0f;
#pragma unroll
        for (int t = 0; t < PT; ++t)
            if (t == tj && lane == owner)
                q = sv[t] > PIVOT_TOL * dg[t] ? rsqrtf(sv[t]) : 0.0f;
        q = __shfl_sync(FULL, q, owner);
        if (!(q > 0.0f))
            return false;
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int a = lane + 32 * t;
            if (a >= j && a < p)
                Lw[a * LS + j] = sv[t] * q;
            if (t == tj && lane == owner)
                inv[t] = q;
        }
        __syncwarp();
    }
    return true;
}

// Solve L L^T z = r in place (row a of r in lane a % 32, slot a / 32).
template <int PT>
__device__ __forceinline__ void subst32(int p, const float *__restrict__ Lw, int LS,
                                        const float (&inv)[PT], float (&r)[PT], int lane)
{
    for (int j = 0; j < p; ++j) {
        const int tj = j >> 5, owner = j & 31;
        float v = r[0] * inv[0];
#pragma unroll
        for (int t = 1; t < PT; ++t)
            if (tj == t)
                v = r[t] * inv[t];
        const float z = __shfl_sync(FULL, v, owner);
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int a = lane + 32 * t;
            if (a > j && a < p)
                r[t] = fmaf(-Lw[a * LS + j], z, r[t]);
            if (t == tj && lane == owner)
                r[t] = z;
        }
    }
    for (int j = p - 1; j >= 0; --j) {
        const int tj = j >> 5, owner = j & 31;
        float v = r[0] * inv[0];
#pragma unroll
        for (int t = 1; t < PT; ++t)
            if (tj == t)
                v = r[t] * inv[t];
        const float xj = __shfl_sync(FULL, v, owner);
        const float *lj = Lw + j * LS;
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            const int a = lane + 32 * t;
            if (a < j)
                r[t] = fmaf(-lj[a], xj, r[t]);
            if (t == tj && lane == owner)
                r[t] = xj;
        }
    }
}

// Systems of at most PM rows (k <= 64; PM >= k / 2 >= p): LDL^T of
// S_ab = Src(idx[a], idx[b]) with lane a keeping the live part of row a in
// registers. At step j, s[0 .. p - j) holds columns j .. p - 1 of row a of the
// trailing (Schur complement) matrix; the update writes column b + 1 into
// s[b], so the row shifts one place per step and every register index stays a
// constant inside a loop that is not unrolled over j (fully unrolled steps
// overflowed the instruction cache). Row j reaches the other lanes by
// shuffles, four columns at a time up to the live width. The multipliers
// L_aj = S_aj / S_jj go to Lw[a * LS + j] (LS odd: conflict-free rows and
// columns); lane a keeps rp = 1 / D_aa. col[b] is the offset of column
// idx[b] within a row of Src (the list padded to a multiple of four with
// offset 0). Returns false (uniformly) when a pivot is at most PIVOT_TOL of
// its diagonal.
template <int KW, int PM>
__device__ __forceinline__ bool ldl_regs(const float *__restrict__ Src, const int *__restrict__ idx,
                                         const int *__restrict__ col, int p,
                                         float *__restrict__ Lw, int LS, float &rp, int lane)
{
    constexpr int RS = 32 * KW;
    const int c = lane < p ? idx[lane] : 0;
    const float *row = Src + c * RS;
    const float dtol = PIVOT_TOL * row[(c & 31) * KW + (c >> 5)];
    float s[PM];
#pragma unroll
    for (int b0 = 0; b0 < PM; b0 += 4) {
        if (b0 < p) {
            const int4 o = *reinterpret_cast<const int4 *>(col + b0);
            s[b0] = row[o.x];
            s[b0 + 1] = row[o.y];
            s[b0 + 2] = row[o.z];
            s[b0 + 3] = row[o.w];
        } else {
#pragma unroll
            for (int b = b0; b < b0 + 4; ++b)
                s[b] = 0.0f;
        }
    }
    bool ok = true;
    rp = 0.0f;
    for (int j = 0; j < p; ++j) {
        const float d = __shfl_sync(FULL, s[0], j);
        const float q = rsqrtf(d);
        const float r = q * q;
        if (lane == j) {
            ok = d > dtol;
            rp = r;
        }
        const bool below = lane > j && lane < p;
        const float m = below ? s[0] * r : 0.0f;
        if (below)
            Lw[lane * LS + j] = m;
        const int w = p - j;   // live columns: s[0 .. w)
#pragma unroll
        for (int b0 = 0; b0 < PM; b0 += 4) {
            if (b0 >= w)
                break;
#pragma unroll
            for (int b = (b0 > 1 ? b0 : 1); b < b0 + 4; ++b)
                s[b - 1] = fmaf(-m, __shfl_sync(FULL, s[b], j), s[b]);
        }
    }
    return __all_sync(FULL, ok);
}

// Solve S z = r with the factor of ldl_regs (row a of r and z in lane a):
// L y = r forward, then L^T z = D^{-1} y backward. Four steps at a time with
// their multipliers loaded first, so only the shuffle and the FMA of each step
// are on the dependency chain (a lane's loads may run past its row or the
// factor: the per-warp area ends with 32 floats of slack; lanes >= p carry
// values that are never read).
__device__ __forceinline__ float ldl_solve(const float *__restrict__ Lw, int LS, float rp, int p,
                                           float r, int lane)
{
    const float *lrow = Lw + (lane < p ? lane : 0) * LS;
    int j = 0;
    for (; j + 4 < p; j += 4) {
        const float l0 = lrow[j], l1 = lrow[j + 1], l2 = lrow[j + 2], l3 = lrow[j + 3];
        float t = __shfl_sync(FULL, r, j);
        if (lane > j) r = fmaf(-l0, t, r);
        t = __shfl_sync(FULL, r, j + 1);
        if (lane > j + 1) r = fmaf(-l1, t, r);
        t = __shfl_sync(FULL, r, j + 2);
        if (lane > j + 2) r = fmaf(-l2, t, r);
        t = __shfl_sync(FULL, r, j + 3);
        if (lane > j + 3) r = fmaf(-l3, t, r);
    }
    for (; j + 1 < p; ++j) {
        const float t = __shfl_sync(FULL, r, j);
        if (lane > j)
            r = fmaf(-lrow[j], t, r);
    }
    float v = r * rp, z = 0.0f;
    j = p - 1;
    for (; j >= 3; j -= 4) {
        const float l0 = Lw[j * LS + lane], l1 = Lw[(j - 1) * LS + lane];
        const float l2 = Lw[(j - 2) * LS + lane], l3 = Lw[(j - 3) * LS + lane];
        float zj = __shfl_sync(FULL, v, j);
        if (lane < j) v = fmaf(-l0, zj, v);
        if (lane == j) z = zj;
        zj = __shfl_sync(FULL, v, j - 1);
        if (lane < j - 1) v = fmaf(-l1, zj, v);
        if (lane == j - 1) z = zj;
        zj = __shfl_sync(FULL, v, j - 2);
        if (lane < j - 2) v = fmaf(-l2, zj, v);
        if (lane == j - 2) z = zj;
        zj = __shfl_sync(FULL, v, j - 3);
        if (lane < j - 3) v = fmaf(-l3, zj, v);
        if (lane == j - 3) z = zj;
    }
    for (; j >= 0; --j) {
        const float zj = __shfl_sync(FULL, v, j);
        if (lane < j)
            v = fmaf(-Lw[j * LS + lane], zj, v);
        if (lane == j)
            z = zj;
    }
    return z;
}

// Shared memory: G and M (k rounded up to 4 rows of 32 KW floats each), then
// per warp an index list, its values, a staging vector (32 KW each), the
// list's column offsets (k <= 64) and the pmax x LS factor.
__host__ __device__ inline size_t mats_bytes32(int k, int KW)
{
    return 2 * sizeof(float) * (size_t)((k + 3) & ~3) * 32 * KW;
}
__host__ __device__ inline size_t warp_bytes32(int KW, int pmax, int LS)
{
    // k <= 64: column offsets, and 32 floats of slack after the factor (read
    // past its end by the unrolled substitutions).
    const size_t cols = KW <= 2 ? sizeof(int) * 32 * KW + sizeof(float) * 32 : 0;
    return (3 * sizeof(float) * 32 * KW + cols + sizeof(float) * (size_t)pmax * LS + 15) &
           ~size_t(15);
}

// 64 registers for KW <= 2 (two 16-warp CTAs per SM); the KW = 4 form needs
// more and runs one CTA per SM.
template <int KW, int PM>
__global__ void __launch_bounds__(S32_MAX_WARPS * 32, KW == 4 ? 1 : 2)
    bpp_solve32_kernel(const SolveParams P, int pmax, int LS)
{
    constexpr int RS = 32 * KW;
    constexpr int PT = (KW + 1) / 2;
    if (P.predict ? P.flags[0] != 1 : P.flags[0] != 0)
        return;
    const bool fused = P.fused && !P.predict;
    const bool group = P.group && !P.predict && !fused;   // no group-tile pass before fused solves
    if (group && P.counters[CNT_PENDING] == 0)
        return;   // the group-tile pass solved them all
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = P.k, k4 = (k + 3) & ~3;
    const int max_rounds = P.predict ? PREDICT_ROUNDS : P.max_rounds;
    unsigned long long *counter = &P.counters[P.predict ? CNT_PREDICT : CNT_WORK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *Gs = reinterpret_cast<float *>(smem_raw);
    float *Ms = Gs + k4 * RS;
    for (int e = threadIdx.x; e < k4 * RS; e += blockDim.x) {
        const int r = e / RS, q = e - r * RS;
        const int c = q / KW + 32 * (q % KW);
        const bool in = r < k && c < k;
        Gs[e] = in ? P.G32[r * k + c] : 0.0f;
        Ms[e] = in ? P.M32[r * k + c] : 0.0f;
    }
    unsigned char *wp = smem_raw + mats_bytes32(k, KW) + warp * warp_bytes32(KW, pmax, LS);
    int *widx = reinterpret_cast<int *>(wp);
    float *zbuf = reinterpret_cast<float *>(widx + RS);
    float *stage = zbuf + RS;
    int *wcol = reinterpret_cast<int *>(stage + RS);   // KW <= 2: column offsets of the list
    float *Lw = stage + RS + (KW <= 2 ? RS : 0);
    __syncthreads();

    bool usable[KW];
    float dsq[KW];   // sqrt(G_ii) (1 where unusable): the scale of the sign tolerances
    int nU = 0;
#pragma unroll
    for (int s = 0; s < KW; ++s) {
        const uint32_t w = P.usable_words[s];
        usable[s] = (w >> lane) & 1u;
        nU += __popc(w);
        const int i = lane + 32 * s;
        dsq[s] = usable[s] ? sqrtf(Gs[i * RS + lane * KW + s]) : 1.0f;
    }

    // Per-warp statistics in shared memory (lane 0 updates them), so that
    // they hold no registers through the solves.
    __shared__ unsigned long long wst[S32_MAX_WARPS][6];   // rhs, rounds, max, fp64, nc, nf
    if (lane < 6)
        wst[warp][lane] = 0;

    for (;;) {
        unsigned long long j0 = 0;
        if (lane == 0)
            j0 = atomicAdd(counter, (unsigned long long)P.chunk);
        j0 = __shfl_sync(FULL, j0, 0);
        if (j0 >= (unsigned long long)P.nrhs)
            break;
        const int64_t jend = min((int64_t)j0 + P.chunk, P.nrhs);
        // Fused gathers: row pointers of up to 31 consecutive rows, one per
        // lane (rowptr[rb + lane]), read once per batch.
        int64_t rb = -1, rpv = 0;
        for (int64_t j = (int64_t)j0; j < jend; ++j) {
            float g[KW], u[KW], x[KW], y[KW];
            bool inF[KW];
            bool bad = false, have_u = false;
            float gmax = 0.0f;
            if (fused) {
                // b_j = (S F)_j: the row's stored entries in order, 32 at a
                // time, broadcast by shuffle (the SpMM kernel's sum order).
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    g[s] = 0.0f;
                if (rb < 0 || j - rb >= 31) {
                    rb = j;
                    rpv = P.gat.rowptr[min(j + lane, P.nrhs)];
                }
                const int64_t beg = __shfl_sync(FULL, rpv, (int)(j - rb));
                const int64_t end = __shfl_sync(FULL, rpv, (int)(j - rb) + 1);
                for (int64_t p0 = beg; p0 < end; p0 += 32) {
                    const int64_t p = p0 + lane;
                    const int c = p < end ? P.gat.colidx[p] : 0;
                    const float v = p < end ? P.gat.vals[p] : 0.0f;
                    const int cnt = (int)min((int64_t)32, end - p0);
                    int l = 0;
                    // Four entries at a time: their F rows are loaded before
                    // the FMAs, which keep the entries' order.
                    for (; l + 4 <= cnt; l += 4) {
                        float fv[4][KW], vl[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int64_t cl = __shfl_sync(FULL, c, l + q);
                            vl[q] = __shfl_sync(FULL, v, l + q);
                            const float *frow = P.gat.F + cl * k;
#pragma unroll
                            for (int s = 0; s < KW; ++s) {
                                const int i = lane + 32 * s;
                                fv[q][s] = i < k ? frow[i] : 0.0f;
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q)
#pragma unroll
                            for (int s = 0; s < KW; ++s)
                                if (lane + 32 * s < k)
                                    g[s] = fmaf(vl[q], fv[q][s], g[s]);
                    }
                    for (; l < cnt; ++l) {
                        const int64_t cl = __shfl_sync(FULL, c, l);
                        const float vl = __shfl_sync(FULL, v, l);
                        const float *frow = P.gat.F + cl * k;
#pragma unroll
                        for (int s = 0; s < KW; ++s) {
                            const int i = lane + 32 * s;
                            if (i < k)
                                g[s] = fmaf(vl, frow[i], g[s]);
                        }
                    }
                }
                float *Bw = const_cast<float *>(P.B);   // the caller's right-hand-side buffer
#pragma unroll
                for (int s = 0; s < KW; ++s) {
                    const int i = lane + 32 * s;
                    if (i < k)
                        Bw[j * k + i] = g[s];
                }
            }
#pragma unroll
            for (int s = 0; s < KW; ++s) {
                const int i = lane + 32 * s;
                if (!fused)
                    g[s] = i < k ? P.B[j * k + i] : 0.0f;
                bad |= !isfinite(g[s]);
                gmax = fmaxf(gmax, fabsf(g[s]) / dsq[s]);
                u[s] = 0.0f;
                x[s] = 0.0f;
                y[s] = -g[s];
                inF[s] = false;
            }
            bad = __any_sync(FULL, bad);
            gmax = warp_max(gmax);
            const float ytol = FEAS_TOL32 * gmax;
            float xtol = 0.0f;
            int status = NMF_OK;
            int rounds = 0;
            if (bad) {
                status = NMF_ERR_NONFINITE;
#pragma unroll
                for (int s = 0; s < KW; ++s)
                    x[s] = 0.0f;
            } else {
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
                if (group && nU > 0) {
                    // The group-tile pass took this right-hand side when its
                    // first candidate partition is all of U (the same test),
                    // and marked it only if it could not finish it.
                    bool out = false;
#pragma unroll
                    for (int s = 0; s < KW; ++s)
                        out |= usable[s] && !(P.pin ? inF[s] : (y[s] < -ytol * dsq[s]));
                    if (!__any_sync(FULL, out) && (P.pin || max_rounds >= 1)) {
                        uint32_t mark = 0;
                        if (lane == 0)
                            mark = reinterpret_cast<const uint32_t *>(P.X)[j * k];
                        if (__shfl_sync(FULL, mark, 0) != GROUP_PENDING)
                            continue;   // solved by the group-tile pass
                    }
                }

                // Candidate point of the current partition: fills x and y.
                // The solve and its refinement are two passes of one loop
                // (substitution, the step dx, then w = G x), so each piece of
                // code appears once: the kernel is bound by instruction
                // issue and fetch, not by arithmetic.
                auto solve = [&]() -> int {
                    int nF = 0;
#pragma unroll
                    for (int s = 0; s < KW; ++s)
                        nF += __popc(__ballot_sync(FULL, inF[s]));
                    const bool comp = nU - nF < nF;
                    if (comp && !have_u) {
                        stage_vec<KW>(stage, g, lane);
                        mv_full<KW>(Ms, k4, stage, u, lane);
                        have_u = true;
                    }
                    bool inS[KW];
                    int rank[KW];
                    int pos = 0;
                    __syncwarp();
#pragma unroll
                    for (int s = 0; s < KW; ++s) {
                        inS[s] = comp ? (usable[s] && !inF[s]) : inF[s];
                        const unsigned mk = __ballot_sync(FULL, inS[s]);
                        rank[s] = pos + __popc(mk & lanemask_lt(lane));
                        if (inS[s]) {
                            widx[rank[s]] = lane + 32 * s;
                            zbuf[rank[s]] = comp ? -u[s] : g[s];
                            if constexpr (KW <= 2)
                                wcol[rank[s]] = lane * KW + s;
                        }
                        pos += __popc(mk);
                    }
                    const int p = pos, p4 = (p + 3) & ~3;
                    if (lane < p4 - p) {
                        widx[p + lane] = 0;
                        zbuf[p + lane] = 0.0f;
                        if constexpr (KW <= 2)
                            wcol[p + lane] = 0;
                    }
                    __syncwarp();
                    float inv[PT], rp = 0.0f;
                    if constexpr (KW <= 2) {
                        if (p > 0 &&
                            !ldl_regs<KW, PM>(comp ? Ms : Gs, widx, wcol, p, Lw, LS, rp, lane))
                            return DEFERRED;
                    } else {
                        if (p > 0 && !chol32<KW, PT>(comp ? Ms : Gs, widx, p, Lw, LS, inv, lane))
                            return DEFERRED;
                    }
                    // Pass 0 solves the system (zbuf = g_F, or -u_A in the
                    // complement form); pass 1 solves it again for the
                    // residual g_F - (G x)_F through the same factor (the
                    // explicit inverse alone is not backward stable in FP32).
                    float base[KW], w[KW];
#pragma unroll
                    for (int s = 0; s < KW; ++s)
                        base[s] = u[s];
                    for (int pass = 0;; ++pass) {
                        if (p > 0) {
                            float r[PT];
#pragma unroll
                            for (int t = 0; t < PT; ++t) {
                                const int a = lane + 32 * t;
                                r[t] = a < p ? zbuf[a] : 0.0f;
                            }
                            if constexpr (KW <= 2)
                                r[0] = ldl_solve(Lw, LS, rp, p, r[0], lane);
                            else
                                subst32<PT>(p, Lw, LS, inv, r, lane);
                            __syncwarp();
#pragma unroll
                            for (int t = 0; t < PT; ++t)
                                if (lane + 32 * t < p)
                                    zbuf[lane + 32 * t] = r[t];
                            __syncwarp();
                        }
                        // The step: dx_F from the direct solution, or
                        // base_F + M_FA z_A from the complement one.
                        if (comp)
                            mv_list<KW>(Ms, widx, zbuf, p4, base, lane);
#pragma unroll
                        for (int s = 0; s < KW; ++s) {
                            const float dx = inF[s] ? (comp ? base[s] : zbuf[rank[s]]) : 0.0f;
                            x[s] = pass ? x[s] + dx : dx;
                            w[s] = 0.0f;
                        }
                        // w = G x: over the F list in the direct form, all
                        // rows in the complement form.
                        if (!comp) {
                            __syncwarp();
#pragma unroll
                            for (int s = 0; s < KW; ++s)
                                if (inS[s])
                                    zbuf[rank[s]] = x[s];
                            __syncwarp();
                            mv_list<KW>(Gs, widx, zbuf, p4, w, lane);
                        } else {
                            stage_vec<KW>(stage, x, lane);
                            mv_full<KW>(Gs, k4, stage, w, lane);
                        }
                        if (pass == 1 || nF == 0)
                            break;
                        float res[KW];
#pragma unroll
                        for (int s = 0; s < KW; ++s) {
                            res[s] = inF[s] ? g[s] - w[s] : 0.0f;
                            base[s] = 0.0f;
                        }
                        if (comp) {
                            stage_vec<KW>(stage, res, lane);
                            mv_full<KW>(Ms, k4, stage, base, lane);   // up = M res
                        }
                        __syncwarp();
#pragma unroll
                        for (int s = 0; s < KW; ++s)
                            if (inS[s])
                                zbuf[rank[s]] = comp ? -base[s] : res[s];
                        __syncwarp();
                    }
                    // y = G x - g off F (0 on F), from the refined x.
                    float xm = 0.0f;
#pragma unroll
                    for (int s = 0; s < KW; ++s) {
                        y[s] = inF[s] ? 0.0f : w[s] - g[s];
                        xm = fmaxf(xm, inF[s] ? fabsf(x[s]) * dsq[s] : 0.0f);
                    }
                    xtol = FEAS_TOL32 * warp_max(xm);   // scaled: compares x_i * d_i
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
                        inf[s] = usable[s] && (inF[s] ? (x[s] * dsq[s] < -xtol)
                                                      : (y[s] < -ytol * dsq[s]));
                        vm[s] = __ballot_sync(FULL, inf[s]);
                        nV += __popc(vm[s]);
                    }
                    if (nV == 0)
                        break;
                    if (rounds >= max_rounds) {
                        status = NMF_ERR_NOT_CONVERGED;
                        break;
                    }
                    if (nV < beta || alpha >= 1) {
                        // Full exchange: the count dropped (reset the budget),
                        // or one of the three further full exchanges.
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
                if (status != DEFERRED) {
                    bool nf = false;
#pragma unroll
                    for (int s = 0; s < KW; ++s) {
                        x[s] = x[s] > 0.0f ? x[s] : 0.0f;   // within-tolerance negatives -> 0
                        nf |= !isfinite(x[s]);
                    }
                    if (__any_sync(FULL, nf) && status == NMF_OK)
                        status = NMF_ERR_NONFINITE;
                }
            }
            if (P.predict) {
                // Only the partition reached seeds the FP64 solves; where the
                // FP32 system was singular, the starting one (given or empty).
                if (P.pout) {
                    unsigned bm[KW];
#pragma unroll
                    for (int s = 0; s < KW; ++s) {
                        bool f = inF[s];
                        if (status == DEFERRED) {
                            const int i = lane + 32 * s;
                            f = P.pin && i < k && ((P.pin[j * P.nwords + (i >> 6)] >> (i & 63)) & 1ull);
                        }
                        bm[s] = __ballot_sync(FULL, f);
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int w = 0; w < (KW + 1) / 2; ++w) {
                            const uint64_t lo = bm[2 * w];
                            const uint64_t hi = (2 * w + 1 < KW) ? bm[2 * w + 1] : 0u;
                            P.pout[j * P.nwords + w] = lo | (hi << 32);
                        }
                    }
                }
                continue;
            }
            if (status == DEFERRED) {
                if (lane == 0) {
                    const unsigned long long slot = atomicAdd(&P.counters[CNT_DEFERRED], 1ull);
                    if (slot < (unsigned long long)DEFER_CAP)
                        P.defer[slot] = j;
                    wst[warp][3] += 1;
                }
                continue;
            }
#pragma unroll
            for (int s = 0; s < KW; ++s) {
                const int i = lane + 32 * s;
                if (i < k)
                    P.X[j * k + i] = x[s];
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
                wst[warp][0] += 1;
                wst[warp][1] += rounds;
                if (wst[warp][2] < (unsigned long long)rounds)
                    wst[warp][2] = rounds;
                wst[warp][4] += status == NMF_ERR_NOT_CONVERGED;
                wst[warp][5] += status == NMF_ERR_NONFINITE;
            }
        }
    }
    if (lane == 0 && (wst[warp][0] || wst[warp][3])) {
        atomicAdd(&P.stats->rhs, wst[warp][0]);
        atomicAdd(&P.stats->rounds, wst[warp][1]);
        atomicMax(&P.stats->max_rounds, wst[warp][2]);
        if (wst[warp][3]) atomicAdd(&P.stats->fp64_solves, wst[warp][3]);
        if (wst[warp][4]) atomicAdd(&P.stats->not_converged, wst[warp][4]);
        if (wst[warp][5]) atomicAdd(&P.stats->nonfinite, wst[warp][5]);
    }
}

// PM: the largest system held in registers (k <= 64), a multiple of four at
// least k / 2 (p <= k / 2).
template <int KW, int PM>
nmf_status launch32(const SolveParams &P, cudaStream_t s)
{
    const int k = P.k;
    const int pmax = k / 2 > 1 ? k / 2 : 1;   // min(|F|, |A|) <= k / 2
    int q = (pmax + 1) / 2;
    if (!(q & 1))
        ++q;
    // k > 64: 2 * odd, conflict-free float2 row reads and column accesses;
    // k <= 64: odd, conflict-free rows and columns of single floats.
    const int LS = KW <= 2 ? (pmax | 1) : 2 * q;
    int nwarps = P.warps < S32_MAX_WARPS ? P.warps : S32_MAX_WARPS;
    const size_t mats = mats_bytes32(k, KW);
    auto bytes = [&](int nw) { return mats + (size_t)nw * warp_bytes32(KW, pmax, LS); };
    while (nwarps > 1 && bytes(nwarps) > SMEM_LIMIT32)
        --nwarps;
    const size_t smem = bytes(nwarps);
    if (smem > SMEM_LIMIT32)
        return NMF_ERR_INVALID_ARG;
    static SmemOptIn opt_in;
    NMF_TRY(ensure_smem(bpp_solve32_kernel<KW, PM>, opt_in, smem));
    int per_sm = 0;
    NMF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bpp_solve32_kernel<KW, PM>,
                                                           nwarps * 32, smem));
    if (per_sm < 1)
        return NMF_ERR_INVALID_ARG;
    int64_t blocks = (int64_t)per_sm * sm_count();
    const int64_t need = cdiv(cdiv(P.nrhs, (int64_t)P.chunk), nwarps);
    if (need < blocks)
        blocks = need < 1 ? 1 : need;
    bpp_solve32_kernel<KW, PM><<<(unsigned)blocks, nwarps * 32, smem, s>>>(P, pmax, LS);
    NMF_LAUNCHED("bpp_solve32_kernel");
    return NMF_OK;
}

}  // namespace

nmf_status launch_solve32(const SolveParams &P, cudaStream_t s)
{
    if (P.k <= 32)
        return launch32<1, 16>(P, s);
    if (P.k <= 48)
        return launch32<2, 24>(P, s);
    if (P.k <= 56)
        return launch32<2, 28>(P, s);
    if (P.k <= 64)
        return launch32<2, 32>(P, s);
    return launch32<4, 4>(P, s);
}

}  // namespace bpp
}  // namespace nmf
