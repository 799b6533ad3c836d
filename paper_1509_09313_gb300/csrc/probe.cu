// FP32 FMA throughput probe (nmf_probe_fp32_fma).
//
// The FP32 arithmetic of the library's SIMT kernels (plain FP32 products, BPP
// solves, the group-tile pass) is reported against the rate this GPU actually
// sustains for independent FMAs, measured here, instead of a nominal figure.
// Every thread runs eight independent FMA chains, x <- x * b + c, either as
// scalar FFMA or as packed FP32x2 FFMA2 (two FMAs per instruction); b and c
// are kernel arguments, so nothing folds at compile time. The grid is eight
// 256-thread CTAs per SM. The result is written only when a chain reaches an
// impossible value, which keeps the arithmetic live without memory traffic.
#include "common.cuh"

namespace nmf {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 8;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;

__device__ float g_probe_sink;

template <bool PACKED>
__global__ void __launch_bounds__(PROBE_THREADS)
    fma_probe_kernel(int iters, float b, float c)
{
    if (PACKED) {
        float2 x[PROBE_CHAINS];
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j)
            x[j] = make_float2(threadIdx.x * 1e-3f + j, blockIdx.x * 1e-3f - j);
        const float2 bb = make_float2(b, b), cc = make_float2(c, c);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PROBE_CHAINS; ++j)
                    x[j] = __ffma2_rn(x[j], bb, cc);
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j)
            s += x[j].x + x[j].y;
        if (s == -1.2345e30f)
            g_probe_sink = s;
    } else {
        float x[PROBE_CHAINS];
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j)
            x[j] = threadIdx.x * 1e-3f + j;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PROBE_CHAINS; ++j)
                    x[j] = __fmaf_rn(x[j], b, c);
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j)
            s += x[j];
        if (s == -1.2345e30f)
            g_probe_sink = s;
    }
}

}  // namespace
}  // namespace nmf

using namespace nmf;

extern "C" nmf_status nmf_probe_fp32_fma(int32_t packed, int32_t launches, double *flops_per_s,
                                         void *stream)
{
    if (!flops_per_s || launches < 1 || launches > 100000 || (packed != 0 && packed != 1))
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int iters = 2048;
    const unsigned grid = (unsigned)(sm_count() * PROBE_CTAS_PER_SM);
    // b < 1 and c small keep every chain bounded (x -> c / (1 - b)).
    const float b = 0.999f, c = 1e-3f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NMF_CUDA(cudaEventCreate(&e0));
    const cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return from_cuda(ce, "cudaEventCreate");
    }
    nmf_status st = NMF_OK;
    auto launch = [&]() -> nmf_status {
        if (packed)
            fma_probe_kernel<true><<<grid, PROBE_THREADS, 0, s>>>(iters, b, c);
        else
            fma_probe_kernel<false><<<grid, PROBE_THREADS, 0, s>>>(iters, b, c);
        NMF_LAUNCHED("fma_probe_kernel");
        return NMF_OK;
    };
    st = launch();   // warm-up launch, not timed
    for (int32_t l = 0; st == NMF_OK && l < launches; ++l) {
        if (l == 0 && cudaEventRecord(e0, s) != cudaSuccess)
            st = NMF_ERR_CUDA;
        if (st == NMF_OK)
            st = launch();
    }
    float ms = 0.f;
    if (st == NMF_OK) {
        cudaError_t e = cudaEventRecord(e1, s);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess)
            st = from_cuda(e, "probe timing");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    NMF_TRY(st);
    const double fmas = (double)grid * PROBE_THREADS * (double)iters * PROBE_UNROLL *
                        PROBE_CHAINS * (packed ? 2.0 : 1.0) * (double)launches;
    *flops_per_s = ms > 0.f ? 2.0 * fmas / (ms * 1e-3) : 0.0;
    return NMF_OK;
}
