// Fused persistent collision solve: shared-memory footprint, variant dispatch
// and the autotuner.  The kernel itself is nmc_fused.cuh, instantiated in the
// nmc_fused_*.cu units.
#include <cuda_runtime.h>

#include <string>

#include "nmc_internal.h"
#include "nmc_fused.cuh"

namespace nmc {

static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

size_t fused_smem_bytes(const nmc_ctx* ctx, int maxm, bool mixed, SolveArgs* a) {
    const int NS = ctx->ns, NE = ctx->ne, NEP = ctx->nep, LD = NE + 1;
    const size_t rs = mixed ? sizeof(float) : sizeof(double);
    const int threads = ((NS * NEP + 31) / 32) * 32;
    size_t mats = (size_t)(NS + NS / 2) * NE * LD;
    const size_t fdq = (size_t)(mixed ? 2 : 1) * NS * ctx->n_elem * kProjQuad;
    if (fdq > mats) mats = fdq;
    const size_t b_mats = align16(mats * rs);
    const size_t b_vec = align16((size_t)8 * NS * NEP * rs);
    const size_t b_red = align16((size_t)(threads / 32) * 8 * sizeof(double));
    const size_t b_node = align16(maxm <= 3 ? sizeof(NodeShared<3>) : sizeof(NodeShared<5>));
    if (a) {
        a->off_phi = 0;
        a->off_ann = (int)((size_t)NS * NE * LD * rs);
        a->off_vec = (int)b_mats;
        a->off_red = (int)(b_mats + b_vec);
        a->off_node = (int)(b_mats + b_vec + b_red);
    }
    return b_mats + b_vec + b_red + b_node;
}


FusedVariant default_variant(const nmc_ctx* ctx) {
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    return FusedVariant{threads <= 128 ? 4 : (threads <= 256 ? 2 : 1), 100};
}

int tuning_key(const nmc_ctx* ctx, const nmc_params& p) {
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    return (p.precision == NMC_MIXED ? 1000 : 0) + (p.m_inner <= 3 ? 0 : 100) + threads / 32;
}

int launch_fused_variant(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v) {
    const bool mixed = a.p.precision == NMC_MIXED;
    if (a.p.m_inner <= 3)
        return mixed ? launch_fused_f32_m3(ctx, a, stream, v) : launch_fused_f64_m3(ctx, a, stream, v);
    return mixed ? launch_fused_f32_m5(ctx, a, stream, v) : launch_fused_f64_m5(ctx, a, stream, v);
}

int launch_fused(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream) {
    const auto it = ctx->tuned.find(tuning_key(ctx, a.p));
    const FusedVariant v = it != ctx->tuned.end() ? it->second : default_variant(ctx);
    return launch_fused_variant(ctx, a, stream, v);
}

// Times every variant of the block-size class on the caller's batch (two runs,
// each between CUDA events on the caller's stream, the faster counting: the first
// also pays the variant's cold start) and keeps the fastest for this precision,
// Anderson depth and block class.  Two launches per variant, as before, but with
// one sample of noise fewer deciding the choice.
int autotune_fused(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, int32_t* chosen, float* chosen_ms) {
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    std::vector<FusedVariant> cand;
    const int pcts[2] = {100, 50};
    if (threads <= 128) {
        for (int minb : {3, 4, 5, 6})
            for (int pct : pcts) cand.push_back(FusedVariant{minb, pct});
    } else if (threads <= 256) {
        for (int minb : {1, 2, 3})
            for (int pct : pcts) cand.push_back(FusedVariant{minb, pct});
    } else {
        for (int pct : pcts) cand.push_back(FusedVariant{1, pct});
    }

    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    float best = 1e30f;
    FusedVariant bv = default_variant(ctx);
    int rc = NMC_OK;
    for (const FusedVariant& v : cand) {
        float ms_v = 1e30f;
        bool skip = false;
        for (int r = 0; r < 2; ++r) {
            cudaEventRecord(e0, stream);
            rc = launch_fused_variant(ctx, a, stream, v);   // a variant that cannot run is skipped
            if (rc == NMC_EUNSUPPORTED) { rc = NMC_OK; skip = true; break; }
            if (rc != NMC_OK) break;
            cudaEventRecord(e1, stream);
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) { rc = set_error(ctx, NMC_ECUDA, std::string("autotune: ") + cudaGetErrorString(e)); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_v = ms < ms_v ? ms : ms_v;
        }
        if (rc != NMC_OK) break;
        if (!skip && ms_v < best) { best = ms_v; bv = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != NMC_OK) return rc;
    ctx->tuned[tuning_key(ctx, a.p)] = bv;
    if (chosen) { chosen[0] = bv.minb; chosen[1] = bv.grid_pct; }
    if (chosen_ms) *chosen_ms = best;
    return NMC_OK;
}

}  // namespace nmc
