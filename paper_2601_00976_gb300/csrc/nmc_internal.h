// Internal definitions shared by the translation units of libnmc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <map>
#include <string>
#include <vector>

#include "nmc.h"

namespace nmc {

// Gauss--Legendre points per element used for the right-hand side of the
// D^Eq projection (Eq. fermiDiracProjection); integrand of the mass matrix is a
// polynomial of degree <= 2k+2 <= 6, so it is integrated exactly as well.
constexpr int kProjQuad = 16;
constexpr int kMaxSpecies = 6;
constexpr int kMaxNq = 3;
constexpr int kMaxNe = 128;
constexpr int kMaxOuterMem = 5;

// Physical constants (MeV, cm, g, s).
constexpr double kC = 2.99792458e10;               // cm/s
constexpr double kHC = 1.23984198e-10;             // MeV cm
constexpr double kPi = 3.14159265358979323846;
constexpr double kHbarC = kHC / (2.0 * kPi);       // MeV cm
constexpr double kMB = 1.66053906660e-24;          // g (average baryon mass)
constexpr double kMeVErg = 1.602176634e-6;         // erg/MeV
constexpr double kDmNP = 1.2933;                   // MeV
constexpr double kLn10 = 2.302585092994045684;     // ln 10
constexpr double kTMin = 1.0e-3;                   // MeV, EoS range
constexpr double kTMax = 1.0e3;
constexpr double kCW = 4.0 * kPi / (kHC * kHC * kHC);   // 4 pi / (hc)^3  [cm^-3 MeV^-3]

// Bounds checks of the NMC_DEBUG build.  Each check compares an index with
// the length of the array it addresses; a failure records its site in the
// context's device error word (the first failure wins), the access is skipped,
// and the persistent kernels stop taking nodes.  Nothing traps.  In the release
// build every check is the constant true and compiles away.
enum DebugSite : unsigned {
    kDbgEmabIso = 1,      // EmAb / Iso table corner (ComputeOpacities, opacity_interp)
    kDbgNesTable = 2,     // NES table corner
    kDbgPairTable = 3,    // pair table corner
    kDbgSmemNes = 4,      // shared NES kernel matrix
    kDbgSmemPair = 5,     // shared pair kernel matrix
    kDbgSmemVec = 6,      // shared per-bin vectors
    kDbgSmemFd = 7,       // shared Fermi--Dirac values at the projection points
    kDbgHistory = 8,      // least-squares history (Gram matrix, outer history)
    kDbgOutput = 9,       // per-bin output arrays
    kDbgProj = 10,        // projection operators
};

// Stage counters of the NMC_TRACE build: thread 0 of every block of the fused
// kernel reads the SM cycle counter at each stage boundary and, when the block
// ends, adds the cycles spent in each stage to trace[stage].  Block time, not
// busy time: a stage's count includes its barrier waits and the cycles the
// SM gives to other blocks meanwhile.  Release builds compile none of it.
enum TraceStage {
    kTrSetup = 0,     // node set-up: loads, EoS at the old state, E_nu*, N_nu*
    kTrOpac = 1,      // ComputeOpacities
    kTrNorms = 2,     // reference norms and the first vectors of an outer iteration
    kTrContract = 3,  // contraction loop and map Q
    kTrGram = 4,      // least-squares partial sums and their barrier
    kTrSolve = 5,     // least-squares solve (lead warp) and its barrier
    kTrMix = 6,       // Anderson mixing and the next vectors
    kTrVote = 7,      // Algorithm 2 and the vote's barrier
    kTrMatter = 8,    // matter update: sums, outer Anderson step, EoS root
    kTrFinal = 9,     // final matter state and outputs
    kTrQueue = 10,    // taking the next node from the queue
    kTrStages = 11
};
constexpr int kTraceWords = 16;

#ifdef NMC_DEBUG
__device__ inline bool debug_in_bounds(unsigned* word, long long idx, long long n, unsigned site) {
    if (idx >= 0 && idx < n) return true;
    if (word) atomicCAS(word, 0u, site);
    return false;
}
#define NMC_IN_BOUNDS(word, idx, n, site) ::nmc::debug_in_bounds((word), (long long)(idx), (long long)(n), (site))
#else
#define NMC_IN_BOUNDS(word, idx, n, site) true
#endif

// Uniform table axis: value v maps to x = (v - lo) * inv_d with cell floor(x).
struct Axis {
    double lo, inv_d;
    int n;
};

// Everything the kernels need about one context, passed by value.
struct DevGrid {
    int ns, ne, nep, n_elem, nq, ld;   // nep: padded energies per species group; ld = ne + 1
    const double* eps;     // [ne]
    const double* w2;      // [ne]
    const double* w3;      // [ne]
    const double* lneps;   // [ne] ln eps (opacity_interp energy axis)
    const double* proj_e;  // [n_elem][Q] quadrature energies
    const double* proj_c;  // [n_elem][nq][Q] projection operator (mass^-1 * basis * weights)
    const double* proj_a;  // [n_elem][Q] eps^2-weighted cell-average weights
    const double* wt;      // [ne] W2 / (4 pi / (hc)^3) = w eps^2 Delta eps  [MeV^3]
    // FP32 copies for the mixed-precision kernel
    const float* proj_e_f;   // proj_e as double-floats: high words
    const float* proj_e_fl;  //                          low words
    const float* proj_c_f;
    const float* proj_a_f;
    const float* wt_f;
    double ends[2][kMaxNq];  // ell_p(-1/2), ell_p(+1/2)
    double sum_w2;
    double sum_wt;
    unsigned* dbg;           // NMC_DEBUG builds: the context's bounds-check error word (null otherwise)
    unsigned long long* trace;   // NMC_TRACE builds: per-stage SM-cycle counters (null otherwise)
};

struct DevTables {
    Axis rho, t, ye, kt, eta;
    const double* emab;    // [ns][nye][nt][nrho][ne] ln chi
    const double* iso;
    const double* nes;     // [ns][nkt][neta][ne][ne]
    const double* pair;    // [ns/2][nkt][neta][ne][ne]
    const double* nes1;    // linear-order (Phi_1) NES table, as nes, or null
    const double* pair1;   // linear-order (Phi_1) pair table, as pair, or null
    // FP32 copies for the mixed-precision kernel; kernels prescaled by 4 pi / (hc)^3
    const float* emab_f;
    const float* iso_f;
    const float* nes_f;
    const float* pair_f;
    long long n_op, n_nes, n_pair;   // element counts of the EmAb/Iso, NES and pair tables
    // opacity_interp_mixed: the FP32 ln tables regrouped per (rho, E) cell, one float4
    // (rho_i E_q, rho_i+1 E_q, rho_i E_q+1, rho_i+1 E_q+1) per [ns][nye][nt][nrho-1][ne-1]
    const float4* emab_q;
    const float4* iso_q;
    long long n_quad;
};

struct SolveArgs {
    DevGrid g;
    DevTables tb;
    nmc_params p;
    long long n;
    const double* rho;
    const double* T;
    const double* Ye;
    const double* J;
    const double* H;
    const double* dt;
    const double* scale;
    double* J_out;
    double* H_out;
    double* Ye_out;
    double* eps_out;
    double* T_out;
    int32_t* n_outer;
    int32_t* n_inner;
    uint32_t* status;
    int* queue;
    // shared-memory carve (byte offsets)
    int off_phi, off_ann, off_vec, off_red, off_node;
};

// A variant of the fused kernel: the register class (blocks per SM its
// registers must allow, __launch_bounds__) and the persistent grid as a
// percentage of the resident capacity.
struct FusedVariant {
    int minb;
    int grid_pct;
};

// Arguments of the adjoint kernel (collision_adjoint).
struct AdjointArgs {
    DevGrid g;
    DevTables tb;
    nmc_params p;
    long long n;
    const double* rho;
    const double* T;
    const double* Ye;
    const double* J;
    const double* H;
    const double* dt;
    const double* scale;
    const double* J_out;
    const double* T_out;
    const double* gJ;
    const double* gH;
    const double* gYe;
    const double* geps;
    const double* gT;
    double* gJ_in;
    double* gH_in;
    double* gYe_in;
    double* gT_in;
    double* gscale;
    uint32_t* status;
    double fd_rel;
    int ldm;   // leading dimension of the augmented pair matrix
    int off_phi, off_ann, off_mat, off_vec, off_red, off_node;
};

}  // namespace nmc

namespace nmc {
// Staging of collision_solve_host: device buffers for two chunks, the upload
// and download streams, and per-slot events (created on the first call).
struct HostPipe {
    void* buf = nullptr;
    long long chunk = 0;
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t uploaded[2] = {nullptr, nullptr};
    cudaEvent_t solved[2] = {nullptr, nullptr};
    cudaEvent_t downloaded[2] = {nullptr, nullptr};
};
}  // namespace nmc

struct nmc_ctx {
    int n_elem = 0, nq = 0, ns = 0, ne = 0, nep = 0;
    std::vector<double> edges, eps, w2, w3;
    nmc::DevGrid g{};
    nmc::DevTables tb{};
    // device allocations owned by the context
    std::vector<void*> allocations;
    int* queue = nullptr;
    // plain mode: chunk size (nodes) and its scratch, grown on demand and kept
    long long plain_chunk = 1LL << 17;
    void* plain_scratch = nullptr;
    size_t plain_scratch_bytes = 0;
    int* plain_counts_host = nullptr;   // pinned
    // collision_solve_host staging
    nmc::HostPipe host_pipe;
    // autotuned fused-kernel variants, keyed by precision, Anderson depth and block class
    std::map<int, nmc::FusedVariant> tuned;
    int device = 0;
    int num_sms = 0;
    int max_smem_optin = 0;
    std::string last_error;
};

namespace nmc {
// launchers (nmc_solve.cu, nmc_interp.cu)
int launch_fused(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream);
int launch_opacity_interp(nmc_ctx* ctx, int which, int species, long long p, const double* rho,
                          const double* T, const double* Ye, const double* E, double* out,
                          cudaStream_t stream);
int launch_opacity_interp_mixed(nmc_ctx* ctx, int which, int species, long long p, const double* rho,
                                const double* T, const double* Ye, const double* E, double* out,
                                cudaStream_t stream);
size_t fused_smem_bytes(const nmc_ctx* ctx, int maxm, bool mixed, SolveArgs* a);
int launch_adjoint(nmc_ctx* ctx, AdjointArgs& a, cudaStream_t stream);
int launch_plain(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream);
int launch_velocity(nmc_ctx* ctx, const SolveArgs& a, const double* v_in, double* v_out, int freeze,
                    double v_floor, cudaStream_t stream);
int launch_c2p(nmc_ctx* ctx, long long n, const double* N, const double* G, const double* v, double tol,
               int memory, int max_iter, double* D, double* I, int32_t* iters, uint32_t* status,
               cudaStream_t stream);
int launch_fused_f64_m3(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v);
int launch_fused_f64_m5(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v);
int launch_fused_f32_m3(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v);
int launch_fused_f32_m5(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v);
cudaError_t preload_fused_f64_m3();
cudaError_t preload_fused_f64_m5();
cudaError_t preload_fused_f32_m3();
cudaError_t preload_fused_f32_m5();
int noalloc_scratch_address(nmc_ctx* ctx, int** out);
int autotune_fused(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, int32_t* chosen, float* chosen_ms);
size_t adjoint_smem_bytes(const nmc_ctx* ctx, AdjointArgs* a);
int set_error(nmc_ctx* ctx, int code, const std::string& msg);
void host_pipe_release(nmc_ctx* ctx);
}  // namespace nmc

extern "C" int nmc_check_params_internal(nmc_ctx* ctx, const nmc_params* p);
