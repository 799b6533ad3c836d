// Allocation-free entry point for the batched NLS solve (nmf_nls_bpp_noalloc).
//
// Some callers cannot call cudaMalloc: code running under a memory manager
// that owns all device memory (a framework's caching allocator, a fixed
// pool), latency-critical loops where cudaMalloc / cudaFree may synchronise
// the device, and programs that must not grow their device footprint after
// start-up. For them this entry point runs exactly the kernels of
// nmf_nls_bpp, but its workspace is a fixed array compiled into the library
// instead of a stream-ordered allocation; the caller still supplies every
// input and output buffer.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it until the process exits. Host code cannot pass the
// array's name to a kernel (on the host it is only a stand-in symbol), so the
// first call on each device asks the runtime for its device address with
// cudaGetSymbolAddress, with that device current, and caches it.
#include <mutex>

#include "common.cuh"

namespace {

static_assert(NMF_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");

// BPP workspace for k <= NMF_NOALLOC_MAX_K, followed by the call's counters.
static __device__ __align__(256) unsigned char g_bpp_scratch[NMF_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[MAX_DEVICES];

// Device address of g_bpp_scratch on the current device (looked up once).
nmf_status scratch_address(void **out)
{
    int dev = 0;
    NMF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES)
        return NMF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        NMF_CUDA(cudaGetSymbolAddress(&p, g_bpp_scratch));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return NMF_OK;
}

}  // namespace

extern "C" nmf_status nmf_nls_bpp_noalloc(const nmf_nls_desc *d, void *stream)
{
    if (!d || d->k < 1 || d->k > NMF_NOALLOC_MAX_K || d->nrhs < 0 || d->max_rounds < 0 || !d->G)
        return NMF_ERR_INVALID_ARG;
    if (d->nrhs > 0 && (!d->B || !d->X))
        return NMF_ERR_INVALID_ARG;
    if (nmf::ranges_overlap(d->B, d->X, sizeof(float) * (size_t)d->nrhs * d->k))
        return NMF_ERR_INVALID_ARG;
    const size_t work = nmf::bpp_work_bytes(d->k);
    const size_t stats_off = (work + 255) & ~size_t(255);
    if (stats_off + sizeof(nmf::BppStats) > NMF_NOALLOC_SCRATCH_BYTES)
        return NMF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *base = nullptr;
    NMF_TRY(scratch_address(&base));
    nmf::BppStats *stats =
        reinterpret_cast<nmf::BppStats *>(static_cast<unsigned char *>(base) + stats_off);
    // The array keeps the previous call's contents: the counters must start at
    // zero (the prep kernel resets the work counter and rewrites the rest).
    NMF_CUDA(cudaMemsetAsync(stats, 0, sizeof(nmf::BppStats), s));
    NMF_TRY(nmf::launch_bpp(d->k, d->nrhs, d->G, d->B, d->X, d->passive_in, d->passive_out,
                            d->rounds_out, d->status_out, d->max_rounds, base, stats, s));
    nmf::BppStats host;
    NMF_CUDA(cudaMemcpyAsync(&host, stats, sizeof(host), cudaMemcpyDeviceToHost, s));
    NMF_CUDA(cudaStreamSynchronize(s));
    if (host.nonfinite)
        return NMF_ERR_NONFINITE;
    if (host.singular)
        return NMF_ERR_SINGULAR_GRAM;
    if (host.not_converged)
        return NMF_ERR_NOT_CONVERGED;
    return NMF_OK;
}
