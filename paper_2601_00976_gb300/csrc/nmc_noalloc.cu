// collision_solve_noalloc: the fused collision solve for callers that cannot
// allocate device memory when they solve.
//
// Some hosts own all device memory themselves: a simulation framework that
// reserves the GPU's memory for its own pool at start-up, or an integration
// that forbids allocation once its set-up phase is over.  The only scratch the
// fused kernel uses, its work-queue counter, lives here in a file-scope device
// array instead of context memory.
//
// Set-up happens in nmc_create, which already allocates: it looks up the
// array's device address for the context's device and loads every fused-kernel
// variant (under CUDA's lazy module loading a kernel's code is otherwise
// loaded, and device memory reserved for it, at its first launch).  The
// driver may still size its per-context local-memory reservation for the
// kernel at the kernel's first launch on the context, so a caller that must
// not allocate makes one call during its set-up phase (a warm-up) and any
// number afterwards.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "nmc_internal.h"

namespace nmc {
namespace {

// Maximum scratch: 64 32-bit words (256 bytes) per device.  The solve uses the
// first word as its work-queue counter; with a 32-bit counter a call may hold
// at most 2^30 nodes.
constexpr int kNoAllocWords = 64;
constexpr long long kNoAllocMaxNodes = 1LL << 30;

static __device__ __align__(256) int g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
int* g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace

// Device address of the scratch array for the current device.  The host-side
// name g_noalloc_scratch is only a stand-in, never a device address, so the
// address is looked up once per device with that device current (nmc_create
// does it for the context's device).  The context's device must be current.
int noalloc_scratch_address(nmc_ctx* ctx, int** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev != ctx->device)
        return set_error(ctx, NMC_EINVAL, "collision_solve_noalloc: the context's device is not the current device");
    if (dev < 0 || dev >= kMaxDevices) return set_error(ctx, NMC_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(ctx, NMC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<int*>(p);
    }
    *out = g_scratch_ptr[dev];
    return NMC_OK;
}

}  // namespace nmc

using namespace nmc;

extern "C" int collision_solve_noalloc(nmc_ctx* ctx, const nmc_params* params, int64_t n, const double* rho,
                                       const double* T_in, const double* Ye_in, const double* J_in,
                                       const double* H_in, const double* dt, const double* opac_scale,
                                       double* J_out, double* H_out, double* Ye_out, double* eps_out,
                                       double* T_out, int32_t* n_outer, int32_t* n_inner, uint32_t* status,
                                       void* stream) {
    if (!ctx) return NMC_EINVAL;
    if (n > kNoAllocMaxNodes)
        return set_error(ctx, NMC_EUNSUPPORTED,
                         "collision_solve_noalloc: n exceeds the 2^30 nodes its 32-bit static work counter can index");
    if (params && params->mode != NMC_MODE_FUSED)
        return set_error(ctx, NMC_EUNSUPPORTED, "collision_solve_noalloc runs the fused kernel only");
    int rc = nmc_check_params_internal(ctx, params);
    if (rc != NMC_OK) return rc;
    if (n < 0) return set_error(ctx, NMC_EINVAL, "n < 0");
    if (n == 0) return NMC_OK;
    if (!rho || !T_in || !Ye_in || !J_in || !H_in || !dt || !J_out || !H_out || !Ye_out || !eps_out ||
        !T_out || !n_outer || !n_inner || !status)
        return set_error(ctx, NMC_EINVAL, "null array argument");
    int* scratch = nullptr;
    rc = noalloc_scratch_address(ctx, &scratch);
    if (rc != NMC_OK) return rc;
    SolveArgs a{};
    a.g = ctx->g;
    a.tb = ctx->tb;
    a.p = *params;
    a.n = n;
    a.rho = rho; a.T = T_in; a.Ye = Ye_in; a.J = J_in; a.H = H_in; a.dt = dt; a.scale = opac_scale;
    a.J_out = J_out; a.H_out = H_out; a.Ye_out = Ye_out; a.eps_out = eps_out; a.T_out = T_out;
    a.n_outer = n_outer; a.n_inner = n_inner; a.status = status;
    // the work-queue counter is the first word of the static array; the
    // launcher clears it on the stream before the kernel starts
    a.queue = scratch;
    return launch_fused(ctx, a, static_cast<cudaStream_t>(stream));
}
