// Instantiations of the fused kernel: float, Anderson memory up to 5.
#include "nmc_fused.cuh"

namespace nmc {
int launch_fused_f32_m5(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v) {
    return launch_by_variant<float, 5>(ctx, a, stream, v);
}
cudaError_t preload_fused_f32_m5() { return preload_variants<float, 5>(); }
}  // namespace nmc
