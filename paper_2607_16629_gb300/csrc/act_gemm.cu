// Tensor-core search (placeholder until the tcgen05 kernel lands).
#include "act_internal.cuh"

namespace act {
struct Bf16Search {
    int unused;
};
cudaError_t bf16_search_prepare(Bf16Search **out, const __nv_bfloat16 *, int64_t, int, int) {
    *out = nullptr;
    return cudaErrorNotSupported;
}
void bf16_search_free(Bf16Search *) {}
cudaError_t launch_bf16_search(Bf16Search *, int, const __nv_bfloat16 *, const float *, int, int, const float *,
                               unsigned long long *, int *, int *, long long *, int *, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace act
