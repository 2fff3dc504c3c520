// Instantiations of the fused kernel: float, Anderson memory up to 3.
#include "nmc_fused.cuh"

namespace nmc {
int launch_fused_f32_m3(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v) {
    return launch_by_variant<float, 3>(ctx, a, stream, v);
}
cudaError_t preload_fused_f32_m3() { return preload_variants<float, 3>(); }
}  // namespace nmc
