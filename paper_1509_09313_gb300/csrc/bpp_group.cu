// Group-tile pass of the FP32 batched BPP (Sec. 4.2) for the all-passive
// group.
//
// The cited BPP method solves right-hand sides that share a passive set F
// together: one factor of G_FF serves the whole group. On the NMF workloads
// the final passive sets are almost all distinct, and the per-warp kernel
// (bpp32.cu) handles them one at a time. One group is special: F = U, all
// usable indices. Its factor is the inverse M = G_UU^{-1} that the
// preparation kernel already holds, so the group's solves are three dense
// products over a tile of right-hand sides:
//     x0 = M g,   r = g - G x0 (on F),   x1 = x0 + M r,
// the refined solution the per-warp kernel computes for F = U. A batch whose
// solutions are all positive (the batched-BPP stress configuration) is this
// group alone.
//
// A right-hand side joins the group when its first candidate partition is U:
// the given starting passive set covers U (warm start; 0 exchange rounds), or,
// from the empty start, every usable y_i = -g_i is infeasible, so that the
// first full exchange moves all of U into F (1 round). Where x1 passes the
// sign test the pass writes the result, passive set, rounds and status. Every
// other right-hand side is left to the per-warp kernel: a member of the group
// is marked by a NaN with a fixed payload (GROUP_PENDING) in its first entry
// of X; the per-warp kernel repeats the membership test and reads the mark of
// members only.
//
// Each entry of the three products is accumulated in the same order as the
// per-warp kernel's matrix-vector products (even rows into one sum, odd rows
// into another, then added), with the same FMAs, so both paths give bitwise
// equal results.
#include <math.h>

#include "bpp_internal.cuh"

namespace nmf {
namespace bpp {
namespace {

constexpr int GT_THREADS = 512;
constexpr int PF_MAX = 64 * 128 / GT_THREADS;   // tile elements per thread (TR k4 <= 64 x 128)
constexpr size_t SMEM_LIMIT_GT = 226 * 1024;   // leaves room for the static arrays

// Dt[i][r] = sum_j Mat[j][i] St[j][r] for i < k4, r < TR, over j < k4 (rows
// of Mat and St past k are zero). 4 x 4 outputs per thread; a warp covers 4
// column groups x 8 row groups, so each of its vector loads of a Mat row or
// an St row touches at most 128 bytes (one shared-memory wavefront).
__device__ __forceinline__ void tile_product(const float *__restrict__ Mat, int k4,
                                             const float *__restrict__ St, float *__restrict__ Dt,
                                             int TR, int TRS)
{
    const int ng = k4 >> 2, nrg = TR >> 2;
    const int cbn = (ng + 3) >> 2, rbn = (nrg + 7) >> 3;
    const int nt = 32 * cbn * rbn;
    for (int t = threadIdx.x; t < nt; t += GT_THREADS) {
        const int l = t & 31, w = t >> 5;
        const int cg = (w % cbn) * 4 + (l & 3), rg = (w / cbn) * 8 + (l >> 2);
        if (cg >= ng || rg >= nrg)
            continue;
        const int i0 = cg * 4, r0 = rg * 4;
        float2 e[4][2], o[4][2];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                e[rr][h] = make_float2(0.0f, 0.0f);
                o[rr][h] = make_float2(0.0f, 0.0f);
            }
#pragma unroll 2
        for (int j = 0; j < k4; j += 2) {   // k4 / 2 is even
            const float4 a0 = *reinterpret_cast<const float4 *>(St + j * TRS + r0);
            const float4 b0 = *reinterpret_cast<const float4 *>(Mat + j * k4 + i0);
            const float4 a1 = *reinterpret_cast<const float4 *>(St + (j + 1) * TRS + r0);
            const float4 b1 = *reinterpret_cast<const float4 *>(Mat + (j + 1) * k4 + i0);
            const float av0[4] = {a0.x, a0.y, a0.z, a0.w};
            const float av1[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const float2 s0 = make_float2(av0[rr], av0[rr]);
                const float2 s1 = make_float2(av1[rr], av1[rr]);
                e[rr][0] = __ffma2_rn(make_float2(b0.x, b0.y), s0, e[rr][0]);
                e[rr][1] = __ffma2_rn(make_float2(b0.z, b0.w), s0, e[rr][1]);
                o[rr][0] = __ffma2_rn(make_float2(b1.x, b1.y), s1, o[rr][0]);
                o[rr][1] = __ffma2_rn(make_float2(b1.z, b1.w), s1, o[rr][1]);
            }
        }
        const float ev[4][4] = {{e[0][0].x, e[0][0].y, e[0][1].x, e[0][1].y},
                                {e[1][0].x, e[1][0].y, e[1][1].x, e[1][1].y},
                                {e[2][0].x, e[2][0].y, e[2][1].x, e[2][1].y},
                                {e[3][0].x, e[3][0].y, e[3][1].x, e[3][1].y}};
        const float ov[4][4] = {{o[0][0].x, o[0][0].y, o[0][1].x, o[0][1].y},
                                {o[1][0].x, o[1][0].y, o[1][1].x, o[1][1].y},
                                {o[2][0].x, o[2][0].y, o[2][1].x, o[2][1].y},
                                {o[3][0].x, o[3][0].y, o[3][1].x, o[3][1].y}};
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
            *reinterpret_cast<float4 *>(Dt + (i0 + ii) * TRS + r0) =
                make_float4(ev[0][ii] + ov[0][ii], ev[1][ii] + ov[1][ii], ev[2][ii] + ov[2][ii],
                            ev[3][ii] + ov[3][ii]);
    }
}

// Reductions over the Q consecutive lanes that share a right-hand side
// (every lane of the warp calls them).
template <typename T>
__device__ __forceinline__ T q_max(T v, int Q)
{
    for (int o = Q / 2; o > 0; o >>= 1)
        v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ int q_and(int v, int Q)
{
    for (int o = Q / 2; o > 0; o >>= 1)
        v &= __shfl_xor_sync(FULL, v, o);
    return v;
}

// Shared memory: G and M as k4 x k4 row-major (zero past k), then three k4 x
// TRS tiles (one column per right-hand side).
__host__ __device__ inline size_t group_smem(int k, int TR)
{
    const size_t k4 = (size_t)((k + 3) & ~3);
    return sizeof(float) * (2 * k4 * k4 + 3 * k4 * (size_t)(TR + 4));
}

__global__ void __launch_bounds__(GT_THREADS)
    bpp_group_kernel(const SolveParams P, int TR)
{
    if (P.flags[0] != 0)
        return;   // not an FP32 half-step
    extern __shared__ __align__(16) float gsm[];
    __shared__ float dsq[NMF_MAX_K];            // sqrt(G_ii), 1 where unusable
    __shared__ unsigned char use[NMF_MAX_K];
    __shared__ unsigned char cand[64], solved[64];
    const int k = P.k, k4 = (k + 3) & ~3, TRS = TR + 4;
    const int tid = threadIdx.x;
    float *Gs = gsm, *Ms = Gs + k4 * k4, *Bt = Ms + k4 * k4, *Xt = Bt + k4 * TRS,
          *Wt = Xt + k4 * TRS;
    for (int e = tid; e < k4 * k4; e += GT_THREADS) {
        const int r = e / k4, c = e - r * k4;
        const bool in = r < k && c < k;
        Gs[e] = in ? P.G32[r * k + c] : 0.0f;
        Ms[e] = in ? P.M32[r * k + c] : 0.0f;
    }
    int nU = 0;
    uint64_t umask[2] = {0ull, 0ull};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        nU += __popc(P.usable_words[q]);
        umask[q >> 1] |= (uint64_t)P.usable_words[q] << (32 * (q & 1));
    }
    for (int i = tid; i < k; i += GT_THREADS) {
        const bool u = (P.usable_words[i >> 5] >> (i & 31)) & 1u;
        use[i] = u;
        dsq[i] = u ? sqrtf(P.G32[i * k + i]) : 1.0f;
    }
    __syncthreads();

    unsigned long long st_rhs = 0, st_rounds = 0, st_max = 0, st_nf = 0, pending = 0;
    const int64_t ntiles = cdiv(P.nrhs, (int64_t)TR);
    // The right-hand sides of the next tile are read into registers while the
    // current one is computed (element e = tid + GT_THREADS m of the tile,
    // row e / k4, index e % k4).
    float pf[PF_MAX];
    int64_t pf_tile = -1;
    auto prefetch = [&](int64_t t) {
        pf_tile = t;
        if (t >= ntiles)
            return;
        const int64_t t0 = t * TR;
        const int tnr = (int)min((int64_t)TR, P.nrhs - t0);
#pragma unroll
        for (int m = 0; m < PF_MAX; ++m) {
            const int e = tid + GT_THREADS * m;
            const int r = e / k4, i = e - r * k4;
            pf[m] = e < TR * k4 && r < tnr && i < k ? P.B[(t0 + r) * k + i] : 0.0f;
        }
    };
    // Tiles are taken in spans of SPT consecutive tiles (GT_THREADS
    // right-hand sides). With a warm start the passive sets decide membership
    // without reading B: one thread per right-hand side of the span, one
    // round of loads for SPT tiles.
    const int SPT = GT_THREADS / TR;
    const int64_t nspans = cdiv(ntiles, (int64_t)SPT);
    const bool pretest = P.pin || P.max_rounds < 1 || nU == 0;
    __shared__ int tcount[GT_THREADS / 32];   // members per tile of the span (SPT <= 16)
    auto next_tile = [&](int64_t t) {         // the tile this CTA takes after t
        return (t + 1) % SPT != 0 ? t + 1 : t + 1 - SPT + (int64_t)gridDim.x * SPT;
    };
    for (int64_t sp = blockIdx.x; sp < nspans; sp += gridDim.x) {
        int memb = 0;
        if (pretest) {
            __syncthreads();   // the previous span's counts are no longer read
            if (tid < SPT)
                tcount[tid] = 0;
            __syncthreads();
            const int64_t j = sp * GT_THREADS + tid;
            if (j < P.nrhs && nU > 0 && P.pin) {
                memb = 1;
                for (int w = 0; w < P.nwords; ++w)
                    if ((P.pin[j * P.nwords + w] & umask[w]) != umask[w])
                        memb = 0;
            }
            if (memb)
                atomicAdd(&tcount[tid / TR], 1);
            __syncthreads();
        }
        for (int ts = 0; ts < SPT; ++ts) {
            const int64_t tile = sp * SPT + ts;
            if (tile >= ntiles)
                break;
            const int64_t j0 = tile * TR;
            const int nr = (int)min((int64_t)TR, P.nrhs - j0);
            // A tile with fewer members than half its width costs more as tile
            // products than as per-warp solves: its members are marked and left.
            const int min_members = (nr + 1) / 2;
            if (pretest && tcount[ts] < min_members) {
                if (memb && tid / TR == ts)
                    reinterpret_cast<uint32_t *>(P.X)[(sp * GT_THREADS + tid) * k] = GROUP_PENDING;
                if (tid == 0)
                    pending += nr;
                continue;
            }
            if (pf_tile != tile)
                prefetch(tile);
#pragma unroll
            for (int m = 0; m < PF_MAX; ++m) {
                const int e = tid + GT_THREADS * m;
                const int r = e / k4, i = e - r * k4;
                if (e < TR * k4)
                    Bt[i * TRS + r] = pf[m];
            }
            prefetch(next_tile(tile));
            __syncthreads();
            // Which right-hand sides start from F = U: Q threads per right-hand
            // side, each over the indices i = q (mod Q).
            const int Q = GT_THREADS / TR, rq = tid / Q, q = tid - rq * Q;
            const bool rlive = rq < nr && nU > 0;
            int ok = 1;
            float gmax = 0.0f;
            if (rlive)
                for (int i = q; i < k; i += Q) {
                    const float g = Bt[i * TRS + rq];
                    ok &= isfinite(g) ? 1 : 0;
                    gmax = fmaxf(gmax, fabsf(g) / dsq[i]);
                }
            ok = q_and(ok, Q);
            gmax = q_max(gmax, Q);
            if (rlive && ok) {
                if (P.pin) {
                    for (int w = 0; w < P.nwords; ++w)
                        if ((P.pin[(j0 + rq) * P.nwords + w] & umask[w]) != umask[w])
                            ok = 0;
                } else if (P.max_rounds >= 1) {
                    const float ytol = FEAS_TOL32 * gmax;
                    for (int i = q; i < k; i += Q)
                        if (use[i] && !(-Bt[i * TRS + rq] < -ytol * dsq[i]))
                            ok = 0;
                } else {
                    ok = 0;
                }
            }
            ok = q_and(ok, Q) && rlive;
            const int c = q == 0 ? ok : 0;
            if (q == 0) {
                cand[rq] = (unsigned char)c;
                solved[rq] = 0;
            }
            if (__syncthreads_count(c) >= min_members) {
                // x0 = M g + 0 on F (0 elsewhere), as the per-warp kernel's
                // complement form with an empty list forms it.
                tile_product(Ms, k4, Bt, Xt, TR, TRS);
                __syncthreads();
                for (int e = tid; e < k4 * TR; e += GT_THREADS) {
                    const int i = e / TR, r = e - i * TR;
                    const float v = Xt[i * TRS + r];
                    Xt[i * TRS + r] = i < k && use[i] ? v + 0.0f : 0.0f;
                }
                __syncthreads();
                tile_product(Gs, k4, Xt, Wt, TR, TRS);   // w = G x0
                __syncthreads();
                for (int e = tid; e < k4 * TR; e += GT_THREADS) {
                    const int i = e / TR, r = e - i * TR;
                    Wt[i * TRS + r] = i < k && use[i] ? Bt[i * TRS + r] - Wt[i * TRS + r] : 0.0f;
                }
                __syncthreads();
                tile_product(Ms, k4, Wt, Bt, TR, TRS);   // up = M r (g no longer needed)
                __syncthreads();
                for (int e = tid; e < k4 * TR; e += GT_THREADS) {
                    const int i = e / TR, r = e - i * TR;
                    if (i < k && use[i])
                        Xt[i * TRS + r] = Xt[i * TRS + r] + (Bt[i * TRS + r] + 0.0f);
                }
                __syncthreads();
                {
                    const bool live = rq < nr && cand[rq];
                    const int64_t j = j0 + rq;
                    float xm = 0.0f;
                    if (live)
                        for (int i = q; i < k; i += Q)
                            if (use[i])
                                xm = fmaxf(xm, fabsf(Xt[i * TRS + rq]) * dsq[i]);
                    const float xtol = FEAS_TOL32 * q_max(xm, Q);
                    int feasible = 1;
                    if (live)
                        for (int i = q; i < k; i += Q)
                            if (use[i] && Xt[i * TRS + rq] * dsq[i] < -xtol)
                                feasible = 0;
                    feasible = q_and(feasible, Q);
                    int fin = 1;
                    if (live && feasible)
                        for (int i = q; i < k; i += Q) {
                            const float v = Xt[i * TRS + rq];
                            const float x = v > 0.0f ? v : 0.0f;
                            fin &= isfinite(x) ? 1 : 0;
                            Xt[i * TRS + rq] = x;
                        }
                    const bool nf = !q_and(fin, Q);
                    if (live && feasible && q == 0) {
                        const int rounds = P.pin ? 0 : 1;
                        const int status = nf ? NMF_ERR_NONFINITE : NMF_OK;
                        solved[rq] = 1;
                        if (P.pout)
                            for (int w = 0; w < P.nwords; ++w)
                                P.pout[j * P.nwords + w] = umask[w];
                        if (P.rounds_out)
                            P.rounds_out[j] = rounds;
                        if (P.status_out)
                            P.status_out[j] = (int8_t)status;
                        st_rhs += 1;
                        st_rounds += rounds;
                        if ((unsigned long long)rounds > st_max)
                            st_max = (unsigned long long)rounds;
                        st_nf += nf;
                    }
                }
                __syncthreads();
                for (int e = tid; e < nr * k; e += GT_THREADS) {
                    const int r = e / k, i = e - r * k;
                    if (solved[r])
                        P.X[(j0 + r) * k + i] = Xt[i * TRS + r];
                }
            }
            if (tid < nr && !solved[tid]) {
                if (cand[tid])   // the per-warp kernel looks for the mark on members only
                    reinterpret_cast<uint32_t *>(P.X)[(j0 + tid) * k] = GROUP_PENDING;
                pending += 1;
            }
            __syncthreads();   // the tile buffers are reused
        }
    }
    if (pending)
        atomicAdd(&P.counters[CNT_PENDING], pending);
    if (st_rhs) {
        atomicAdd(&P.stats->rhs, st_rhs);
        atomicAdd(&P.stats->rounds, st_rounds);
        atomicMax(&P.stats->max_rounds, st_max);
        if (st_nf) atomicAdd(&P.stats->nonfinite, st_nf);
    }
}

}  // namespace

nmf_status launch_group32(const SolveParams &P, cudaStream_t s)
{
    int TR = 64;
    if (group_smem(P.k, TR) > SMEM_LIMIT_GT)
        TR = 32;
    const size_t smem = group_smem(P.k, TR);
    if (smem > SMEM_LIMIT_GT)
        return NMF_ERR_INVALID_ARG;
    static SmemOptIn opt_in;
    NMF_TRY(ensure_smem(bpp_group_kernel, opt_in, smem));
    int per_sm = 0;
    NMF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bpp_group_kernel, GT_THREADS,
                                                           smem));
    if (per_sm < 1)
        return NMF_ERR_INVALID_ARG;
    int64_t blocks = (int64_t)per_sm * sm_count();
    const int64_t spans = cdiv(P.nrhs, (int64_t)GT_THREADS);   // GT_THREADS / TR tiles each
    if (spans < blocks)
        blocks = spans < 1 ? 1 : spans;
    bpp_group_kernel<<<(unsigned)blocks, GT_THREADS, smem, s>>>(P, TR);
    NMF_LAUNCHED("bpp_group_kernel");
    return NMF_OK;
}

}  // namespace bpp
}  // namespace nmf
