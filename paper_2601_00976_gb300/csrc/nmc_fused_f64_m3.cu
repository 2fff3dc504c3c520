// Instantiations of the fused kernel: double, Anderson memory up to 3.
#include "nmc_fused.cuh"

namespace nmc {
int launch_fused_f64_m3(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v) {
    return launch_by_variant<double, 3>(ctx, a, stream, v);
}
cudaError_t preload_fused_f64_m3() { return preload_variants<double, 3>(); }
}  // namespace nmc
