// Instantiations of the fused kernel: double, Anderson memory up to 5.
#include "nmc_fused.cuh"

namespace nmc {
int launch_fused_f64_m5(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v) {
    return launch_by_variant<double, 5>(ctx, a, stream, v);
}
cudaError_t preload_fused_f64_m5() { return preload_variants<double, 5>(); }
}  // namespace nmc
