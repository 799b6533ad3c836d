// Dense products on tcgen05 tensor cores (BF16 head/tail split): not built yet.
#include "common.cuh"

namespace nmf {

size_t mm_tc_work_bytes(int64_t, int64_t, int, int) { return 0; }

nmf_status launch_mm_tc(const float *, int64_t, int64_t, int64_t, const float *, int, int,
                        float *, void *, size_t, cudaStream_t)
{
    return NMF_ERR_INVALID_ARG;
}

}  // namespace nmf
