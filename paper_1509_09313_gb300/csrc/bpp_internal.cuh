// Shared between the batched-BPP translation units (bpp.cu: preparation, FP64
// solves, host side; bpp32.cu: FP32 solves). Not part of the C ABI.
#pragma once

#include "common.cuh"

namespace nmf {
namespace bpp {

constexpr float PIVOT_TOL = 1e-4f;                  // FP32 pivot floor, relative to the diagonal
constexpr double PIVOT_TOL64 = 1e-13;
constexpr double COND_FP32 = 1e4;                   // scaled cond_1(G) up to which solves run in FP32
constexpr float FEAS_TOL32 = 9.5367431640625e-07f;  // 2^-20

// Right-hand sides whose FP32 system hit the pivot floor are re-solved in FP64
// by a second pass. Up to DEFER_CAP of them are listed by index; past that the
// second pass re-solves the whole batch in FP64.
constexpr int DEFER_CAP = 512;

// Work counters (one array of 64-bit words, zeroed by the prep kernel).
enum Counter {
    CNT_WORK = 0,
    CNT_DEFERRED = 1,
    CNT_DEFER_WORK = 2,
    CNT_PREDICT = 3,
    CNT_PENDING = 4,   // right-hand sides the group-tile pass left to the per-warp kernel
    CNT_WORDS = 5
};

// Bits of the NaN the group-tile pass writes to X[j][0] of a right-hand side
// it leaves to the per-warp kernel (a solved X never holds a NaN).
constexpr uint32_t GROUP_PENDING = 0x7fc0a5a5u;

// Rounds allowed to the FP32 predictor of an FP64 half-step's partitions.
constexpr int PREDICT_ROUNDS = 8;

struct SolveParams {
    int k, nwords, max_rounds;
    int warps, chunk;              // warps per CTA; right-hand sides per counter grab
    int64_t nrhs;
    const float *G32, *M32;        // plain row-major k x k (prep kernel output)
    const double *G64, *M64;
    const uint32_t *usable_words;
    const int *flags;
    const float *B;
    float *X;
    const uint64_t *pin;
    uint64_t *pout;
    int32_t *rounds_out;
    int8_t *status_out;
    unsigned long long *counters;  // CNT_WORDS words
    int64_t *defer;                // DEFER_CAP indices
    BppStats *stats;
    // predict = 1: an FP64 (mode 1) half-step's FP32 pass that only writes
    // passive sets (pout) for the FP64 solves to start from; no X, rounds,
    // status or statistics, at most PREDICT_ROUNDS rounds, its own counter.
    int predict;
    // group = 1: the group-tile pass ran first; the per-warp kernel solves
    // only the right-hand sides it marked GROUP_PENDING.
    int group;
    // fused = 1 (sparse ANLS): B is not formed beforehand. The FP32
    // per-warp kernel gathers b_j = (S F)_j from the CSR matrix S and F
    // (gat) in the same order as the SpMM kernel, writes it to B, then solves
    // it; in an FP64 half-step the flag-checked SpMM forms B before the FP64
    // solves.
    int fused;
    CsrGather gat;
};

__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
    for (int o = 16; o > 0; o >>= 1)
        v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// FP32 solve kernel (mode 0): launched for every half-step, returns at once
// unless the prep kernel chose mode 0.
nmf_status launch_solve32(const SolveParams &P, cudaStream_t s);

// Group-tile pass for the all-passive group (mode 0; returns at once
// otherwise). X must not overlap B. launch_group32: SIMT (group = 1), the
// same bits as the per-warp kernel; launch_group_tc: tensor cores (group =
// 2, k <= 112).
nmf_status launch_group32(const SolveParams &P, cudaStream_t s);
bool group_tc_supported(int k);
nmf_status launch_group_tc(const SolveParams &P, cudaStream_t s);

}  // namespace bpp
}  // namespace nmf
