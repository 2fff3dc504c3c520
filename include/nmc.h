/*
 * nmc.h -- C ABI of libnmc, a GB300 (sm_103a) implementation of the implicit,
 * pointwise neutrino--matter collision solve of the thornado DG-IMEX
 * two-moment scheme (arXiv:2601.00976, Sec. 3.5 "Neutrino--matter coupling").
 *
 * At every spatial node the solve finds the primitive moments M = (D, I^j) of
 * each neutrino species and the matter state y = (eps, Ye) that satisfy the
 * backward-Euler collision step (Eq. imexImplicit) written as the nested
 * fixed-point problem M = Q(M, y) (Eq. implicitMomentsNodal) and
 * y = q(M, y) (Eq. implicitFluidNodal), using Algorithm 1 with Anderson
 * acceleration and the convergence checks of Algorithms 2 and 3.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Units: energies and temperatures in MeV, rho in g cm^-3, dt in s,
 *   specific internal energy eps in erg g^-1, opacities in cm^-1.
 * - The fluid velocity is zero and frozen (as in the paper's deleptonization
 *   setup), so lambda = 1/(1+|v|) = 1 and only eps and Ye are evolved.
 * - Species are ordered in particle/antiparticle pairs: (nu_e, anti-nu_e),
 *   then (nu_x, anti-nu_x) for each heavy flavour; n_species is even.
 *   Lepton numbers are +1, -1, 0, 0, ... (Sec. 2.2).
 * - Energy index q = e * n_q + q_eps (element e, LG node q_eps), ne = n_elem * n_q.
 * - "J" and "H" carry the occupation-normalised moments D and I (Eq.
 *   primitiveMoments); the energy moments are eps * (D, I) (Sec. 2.2).
 * - Array arguments of collision_solve / opacity_interp / collision_adjoint are
 *   DEVICE pointers owned by the caller, contiguous, node-major.  Host arrays
 *   passed to nmc_create / nmc_energy_nodes / nmc_geometric_edges are HOST
 *   pointers, read (or written) before the call returns.
 * - The `stream` argument is a cudaStream_t (NULL = legacy default stream);
 *   solve and interpolation calls are asynchronous on it.
 * - Every call returns an int status (NMC_OK or an error code below) and
 *   never aborts; nmc_last_error() gives a message for the last failure on a
 *   context.  Numerical trouble at a node is never an error return: it is
 *   reported in that node's status bits.
 * - One context may be used by one stream at a time: calls that overlap in
 *   time on different streams share the context's work-queue counter and race.
 */
#ifndef NMC_H
#define NMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define NMC_OK            0
#define NMC_EINVAL        1   /* invalid argument (null pointer, bad size, bad parameter) */
#define NMC_ECUDA         2   /* a CUDA runtime call failed; see nmc_last_error */
#define NMC_ENOMEM        3   /* device or host allocation failed */
#define NMC_EUNSUPPORTED  4   /* shape outside what the kernels support (see nmc_create) */

/* ---- per-node status bits (collision_solve) ---- */
#define NMC_NOT_CONVERGED_INNER 1u   /* some inner loop stopped at max_inner */
#define NMC_NOT_CONVERGED_OUTER 2u   /* outer loop stopped at max_outer */
#define NMC_NONFINITE           4u   /* a non-finite moment or matter value appeared */
#define NMC_EOS_FAIL            8u   /* eps outside the EoS range at some outer iterate; T clamped */
#define NMC_TABLE_CLAMP        16u   /* a table lookup fell outside the table and was clamped */
#define NMC_BAD_INPUT          32u   /* rho, T, Ye or dt invalid at this node; outputs = inputs */

/* ---- process mask (Eq. collisionTerm_AllProcesses) ---- */
#define NMC_PROC_EMAB 1   /* emission/absorption */
#define NMC_PROC_ISO  2   /* isoenergetic scattering */
#define NMC_PROC_NES  4   /* neutrino-electron scattering */
#define NMC_PROC_PAIR 8   /* pair processes */
#define NMC_PROC_ALL 15

/* ---- precision ---- */
#define NMC_FP64  0   /* every step in FP64 */
#define NMC_MIXED 1   /* interpolation, kernel contractions and sweeps in FP32;
                         conservation sums, matter update, EoS and the Anderson
                         least-squares solves in FP64 */

/* ---- execution mode ---- */
#define NMC_MODE_FUSED 0   /* one persistent kernel: each block takes nodes from a
                              device work queue and runs Algorithm 1 on chip */
#define NMC_MODE_PLAIN 1   /* one launch per phase and iteration over the still
                              unconverged nodes, state in global memory, the
                              batch in chunks of 2^17 nodes; FP64 only; the
                              host reads list lengths back, so the call
                              synchronises its stream and cannot be captured
                              in a CUDA graph.  The baseline of the fused mode:
                              same algorithm, same results. */

typedef struct nmc_ctx nmc_ctx;

/* Energy grid of one spatial node (Sec. 3.2, Eq. energy_integration_weights). */
typedef struct {
    int32_t n_elem;        /* energy elements, >= 1 */
    int32_t n_q;           /* LG nodes per element, N = k + 1, 1..3 */
    int32_t n_species;     /* even, 2..6 */
    const double* edges;   /* HOST, n_elem + 1 increasing interfaces, edges[0] >= 0 (MeV) */
} nmc_grid;

/*
 * Opacity and kernel tables (Sec. 2.3, paragraph on weaklib tables).
 * All arrays are HOST, C order, float64; nmc_create copies them to the device.
 *
 *   emab, iso : [n_species][n_ye][n_t][n_rho][ne]  natural log of chi_EmAb and
 *               sigma_Iso (cm^-1) on uniform axes in log10 rho, log10 T, Ye;
 *               the energy axis is the grid's node energies eps_q.
 *   nes       : [n_species][n_kt][n_eta][ne][ne]   NES Phi_Out(eps_q, eps_q') in
 *               cm^2 on uniform axes in log10 T and eta_e = mu_e / T; only
 *               entries with q >= q' are read (down-scattering), the rest
 *               follows from Eqs. inOutInvarianceNES and detailedBalanceNES.
 *   pair      : [n_species/2][n_kt][n_eta][ne][ne] pair Phi_Ann(eps_q, eps_q')
 *               of the particle of each pair, cm^2; the antiparticle's is the
 *               transpose (Eq. inOutInvariancePair), Phi_Pro follows from
 *               Eq. detailedBalancePair.
 * Axis i of n points spans [min, max] uniformly; n >= 2 on every axis.
 */
typedef struct {
    int32_t n_rho, n_t, n_ye;
    double lrho_min, lrho_max;   /* log10 rho */
    double lt_min, lt_max;       /* log10 T */
    double ye_min, ye_max;
    const double* emab;
    const double* iso;
    int32_t n_kt, n_eta;
    double klt_min, klt_max;     /* log10 T */
    double eta_min, eta_max;     /* eta_e */
    const double* nes;
    const double* pair;
    /* Optional linear-order (Legendre l = 1) kernels Phi_1 of NES and pair, laid
     * out as nes and pair (both or neither; NULL: none).  Only collision_solve_v
     * reads them: the linear corrections of Eqs. zerothMomentCollisionTerm_NES,
     * firstMomentCollisionTerm_NES, zerothMomentCollisionTerm_Pair and
     * firstMomentCollisionTerm_Pair, with <Phi_1 I> of Eqs.
     * linearCorrectionsNES and linearCorrectionsPair; Phi_1 is completed by the
     * same in-out invariance and detailed balance as Phi_0. */
    const double* nes1;
    const double* pair1;
} nmc_tables;

/* Solver parameters (Algorithm 1 parameters plus the readings the paper leaves open). */
typedef struct {
    double  tol_inner;     /* Algorithm 2 relative tolerance */
    double  tol_outer;     /* Algorithm 3 relative tolerance */
    int32_t m_inner;       /* Anderson memory M_inner, 1 (Picard) .. 5 */
    int32_t m_outer;       /* Anderson memory M_outer, 1 .. 5 */
    int32_t max_inner;     /* cap per inner loop, >= 1 */
    int32_t max_outer;     /* cap on outer iterations, >= 1 */
    int32_t precision;     /* NMC_FP64 or NMC_MIXED (mixed: n_q <= 2, else NMC_EUNSUPPORTED) */
    int32_t mode;          /* NMC_MODE_FUSED or NMC_MODE_PLAIN */
    int32_t proc_mask;     /* NMC_PROC_* bits */
    int32_t frozen_matter; /* 1: y fixed at y*, single outer iteration */
    int32_t final_q;       /* 1: return y = q(M, y) at the converged moments (exact
                              conservation); 0: the Anderson-mixed iterate of Alg. 1 */
    int32_t semi_implicit; /* 1: ComputeOpacities once, at the old state y* before
                              the outer loop of Algorithm 1, and not after matter
                              updates: the semi-implicit variant of Sec. 3.5;
                              0: fully implicit.
                              collision_solve and collision_solve_v; collision_adjoint
                              returns NMC_EUNSUPPORTED for it */
    double  d_min, d_max;  /* bounds of the D^Eq limiter (Eq. fermiDiracProjection) */
    double  norm_floor;    /* Algorithm 2 reference norm floored at norm_floor*sqrt(sum W2) */
} nmc_params;

/* Fills defaults: tol 1e-10, M = 3, caps 100, FP64, fused, all processes,
 * d_min 1e-30, d_max 1 - 1e-6, norm_floor 1e-30, final_q 1, semi_implicit 0. */
void nmc_default_params(nmc_params* p);

/*
 * Creates a context: builds the energy grid, LG rule, W2/W3 weights
 * (Eq. energy_integration_weights) and the per-element projection operators
 * of Eq. fermiDiracProjection, and uploads the tables.  Supported shapes:
 * n_q in 1..3, n_species in {2, 4, 6}, 2 <= ne = n_elem * n_q <= 128, and a
 * per-block shared-memory footprint <= 227 KB (FP64: ne <= 64 with 4 species).
 * On success *out owns all device memory it allocated; free it with
 * nmc_destroy.  On failure *out is NULL and the return code says why.
 */
int nmc_create(const nmc_grid* grid, const nmc_tables* tables, nmc_ctx** out);

/* Releases every device and host allocation of the context; NULL is a no-op. */
void nmc_destroy(nmc_ctx* ctx);

/* Message for the last failed call on ctx (static string if ctx is NULL).
 * In an NMC_DEBUG build it first reads the context's bounds-check error word
 * (a device copy, which waits for the device) and, if a check failed, names
 * its site. */
const char* nmc_last_error(const nmc_ctx* ctx);

/*
 * Bounds checks of the NMC_DEBUG build (a debugging aid; the paper has no
 * counterpart).  The library built with -DNMC_DEBUG checks every table,
 * shared-memory, least-squares-history and output index of the collision
 * solve's kernels against the length of the array it addresses; a failed
 * check records its site (1 EmAb/Iso table, 2 NES table, 3 pair table,
 * 4 shared NES matrix, 5 shared pair matrix, 6 shared vectors, 7 shared
 * Fermi--Dirac values, 8 least-squares history, 9 output, 10 projection
 * operators) in a device word of the context, skips the access, and the
 * persistent kernels stop taking nodes; nothing traps.  This call copies the
 * word to *word (0: no check failed), clearing it when `clear` is nonzero; it
 * waits for the device.  The release build returns NMC_EUNSUPPORTED.
 */
int nmc_debug_word(nmc_ctx* ctx, uint32_t* word, int32_t clear);

/*
 * Stage counters of the NMC_TRACE build (a profiling aid; the paper has no
 * counterpart).  The library built with -DNMC_TRACE has thread 0 of every block
 * of the fused collision-solve kernel read the SM cycle counter at each stage
 * boundary of Algorithm 1 and add, when the block ends, the cycles spent in
 * each stage to a counter of the context: 0 node set-up, 1 ComputeOpacities,
 * 2 reference norms and first vectors of an outer iteration, 3 contraction
 * loop and map Q, 4 least-squares partial sums, 5 least-squares solve,
 * 6 Anderson mixing and next vectors, 7 Algorithm 2 vote, 8 matter update,
 * 9 final state and outputs, 10 taking the next node (counters 11-15 are
 * zero).  The counts are block time (barrier waits and cycles the SM gives to
 * other blocks included), summed over blocks.  This call copies the 16
 * counters to the HOST array `cycles`, clearing them when `clear` is nonzero;
 * it waits for the device.  The release build returns NMC_EUNSUPPORTED with
 * the counters zeroed.
 */
int nmc_trace_read(nmc_ctx* ctx, uint64_t* cycles, int32_t clear);

/* Writes the node energies eps_q (MeV), W2_q (cm^-3) and W3_q (MeV cm^-3) of
 * the context's grid into HOST arrays of length ne (any may be NULL). */
int nmc_energy_nodes(const nmc_ctx* ctx, double* eps, double* w2, double* w3, int32_t* ne);

/* Node energies eps_q (MeV), W2_q (cm^-3) and W3_q (MeV cm^-3) of `grid`
 * (Eq. energy_integration_weights) without creating a context: callers use
 * it to build tables on the node energies.  HOST output arrays of length
 * n_elem * n_q (any may be NULL). */
int nmc_grid_nodes(const nmc_grid* grid, double* eps, double* w2, double* w3);

/* Geometric grid of Sec. 3.5.1 (Table energyGrids): n_elem elements on
 * [0, emax] with widths de1 * alpha^e, alpha solved so they sum to emax.
 * Writes n_elem + 1 interfaces to HOST `edges` and alpha to *alpha (may be NULL). */
int nmc_geometric_edges(int32_t n_elem, double de1, double emax, double* edges, double* alpha);

/*
 * SolveNeutrinoMatterCoupling (Algorithm 1) at n independent nodes.
 *
 * Inputs (DEVICE, float64):
 *   rho[n], T_in[n] (MeV), Ye_in[n]          matter state y* (eps* = eps(rho, T_in, Ye_in))
 *   J_in[n][ns][ne]                          D* (occupation-normalised zeroth moment)
 *   H_in[n][ns][ne][3]                       I* (occupation-normalised first moment)
 *   dt[n]                                    step (s); dtau = c dt (Sec. 3.5: dtau = alpha_ii dt)
 *   opac_scale[n][4] or NULL                 per-node factors on EmAb, Iso, NES, Pair
 * Outputs (DEVICE):
 *   J_out, H_out (same shapes), Ye_out[n], eps_out[n] (erg/g), T_out[n] (MeV),
 *   n_outer[n], n_inner[n] (total inner iterations), status[n] (NMC_* bits).
 * Inputs and outputs must not overlap.  n = 0 is a no-op; n <= 2^30.
 */
int collision_solve(nmc_ctx* ctx, const nmc_params* params, int64_t n,
                    const double* rho, const double* T_in, const double* Ye_in,
                    const double* J_in, const double* H_in, const double* dt,
                    const double* opac_scale,
                    double* J_out, double* H_out, double* Ye_out, double* eps_out,
                    double* T_out, int32_t* n_outer, int32_t* n_inner, uint32_t* status,
                    void* stream);

/*
 * SolveNeutrinoMatterCoupling (Algorithm 1) with the O(v/c) terms of Sec. 3.5
 * at n independent nodes, FP64: the moment map of Eq. implicitMomentsNodal
 * with v^i I_i, v^i K_ij (Minerbo closure, Eqs. eddingtonTensor and
 * eddingtonFactorMinerbo) and lambda = 1/(1+|v|); the old state's conserved
 * moments N* = D* + v*.I*, G*_j = I*_j + v*^i K_ij(M*) (Eq.
 * conservedToPrimitive); the matter map of Eq. implicitFluidNodal with the
 * momentum update and Eqs. eulerianMomentumLG, eulerianEnergyLG,
 * eulerianNumberLG.  Flat metric at the node (Cartesian components).
 *
 * Arguments as collision_solve, plus:
 *   v_in[n][3]  (DEVICE)  fluid three-velocity v* in units of c, |v*| < 1
 *   freeze_velocity       1: v stays v* (the momentum update is switched off,
 *                         as in the deleptonization setup of Sec. 6)
 *   v_floor > 0           reference speed of Algorithm 3 for the velocity
 *                         components: |delta v_j| <= tol * max(|v*|, v_floor)
 *   v_out[n][3] (DEVICE)  the new velocity
 * eps_out is the specific internal energy eps = eps_f - v^2 c^2 / 2.  With
 * final_q the returned (v, eps_f, Ye) conserve momentum, total energy and
 * lepton number to rounding (v solves the momentum update exactly).
 * Supported: NMC_FP64, NMC_MODE_FUSED, m_inner <= 3 and m_outer <= 3
 * (NMC_EUNSUPPORTED otherwise).  An invalid node (also |v*| >= 1 or a
 * non-finite v*) returns its inputs with NMC_BAD_INPUT.
 */
int collision_solve_v(nmc_ctx* ctx, const nmc_params* params, int64_t n,
                      const double* rho, const double* T_in, const double* Ye_in, const double* v_in,
                      const double* J_in, const double* H_in, const double* dt,
                      const double* opac_scale, int32_t freeze_velocity, double v_floor,
                      double* J_out, double* H_out, double* v_out, double* Ye_out, double* eps_out,
                      double* T_out, int32_t* n_outer, int32_t* n_inner, uint32_t* status,
                      void* stream);

/*
 * Conserved-to-primitive moment recovery (Sec. 3.4, Eqs. conservedToPrimitive,
 * c2p_FP, c2p_sequence), FP64, at n nodes of the context's shape.  For every
 * (node, species, energy) bin it finds M = (D, I_j) with N = D + v^i I_i and
 * G_j = I_j + v^i K_ij(M) (Minerbo closure, flat metric), iterating
 * M <- (1 - lam) M + lam (N - v.I, G - v.K(M)), lam = 1/(1 + |v|), from M = U
 * with Anderson acceleration of the given memory until
 * ||M_new - M|| <= tol ||U|| (Euclidean norms of the bin's 4-vector).
 *
 * Inputs (DEVICE, float64): N_in[n][ns][ne], G_in[n][ns][ne][3], v[n][3]
 * (units of c).  Outputs (DEVICE): D_out, I_out (same shapes), iters[n][ns][ne]
 * (iterations per bin; may be NULL), status[n]: NMC_NOT_CONVERGED_INNER if
 * some bin reached max_iter, NMC_NONFINITE if some bin went non-finite.
 * tol > 0, memory in 1..3, max_iter >= 1 (NMC_EINVAL otherwise);
 * ns * ne <= 256 (NMC_EUNSUPPORTED otherwise).  The paper's default tol is 1e-8.
 */
int conserved_to_primitive(nmc_ctx* ctx, int64_t n, const double* N_in, const double* G_in,
                           const double* v, double tol, int32_t memory, int32_t max_iter,
                           double* D_out, double* I_out, int32_t* iters, uint32_t* status,
                           void* stream);

/*
 * collision_solve without device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory when
 * they solve, for example a simulation framework that reserves the GPU's
 * memory for its own pool after set-up.  It runs the same fused kernel as
 * collision_solve (NMC_MODE_FUSED only; same arguments, same results) but
 * takes the kernel's only scratch, its work-queue counter, from a static
 * 256-byte device array instead of context memory, and calls no allocation
 * routine.  Limits and behaviour:
 * - n <= 2^30 per call (the counter is 32-bit); larger n returns
 *   NMC_EUNSUPPORTED with a message.
 * - Set-up is done by nmc_create, which may allocate: it looks up the array's
 *   device address for the context's device (with that device current) and
 *   loads the fused kernel's variants, which CUDA's lazy module loading would
 *   otherwise load, reserving memory, at their first launch.  The driver can
 *   still size its local-memory reservation for the kernel at the kernel's
 *   first launch on the context, so make one call (a warm-up) during set-up,
 *   before the phase in which nothing may allocate and before any stream
 *   capture; later calls leave the device's free memory unchanged.
 * - The context's device must be the current device (NMC_EINVAL otherwise).
 * - Every call on a device shares the array, and each call clears the counter
 *   on its stream before the kernel starts: calls that overlap on the GPU
 *   (different streams, or concurrent host threads) race and must not be
 *   issued.
 */
int collision_solve_noalloc(nmc_ctx* ctx, const nmc_params* params, int64_t n,
                            const double* rho, const double* T_in, const double* Ye_in,
                            const double* J_in, const double* H_in, const double* dt,
                            const double* opac_scale,
                            double* J_out, double* H_out, double* Ye_out, double* eps_out,
                            double* T_out, int32_t* n_outer, int32_t* n_inner, uint32_t* status,
                            void* stream);

/*
 * collision_solve on HOST buffers (the paper has no counterpart: this is the
 * call for a caller whose node data live in host memory).  Same arguments,
 * parameters and results as collision_solve, except that every array is a
 * HOST pointer (page-locked memory lets the copies overlap the solve; pageable
 * memory works but serialises them) and `chunk` sets the pipeline's chunk
 * size in nodes (0: n / 8, at least 8192).  The batch is copied to the device
 * chunk by chunk on an upload stream, each chunk is solved on `stream`, and
 * its outputs are copied back on a download stream, so that copies of
 * neighbouring chunks overlap the solve; `stream` waits for the last copies,
 * so the host outputs are complete once `stream` is (synchronise it before
 * reading them; keep the host buffers alive until then).  The context keeps
 * device staging for two chunks (allocated on the first call that needs it,
 * freed by nmc_destroy) and two streams of its own; calls on one context must
 * not overlap.  n <= 2^30; NMC_EINVAL for NULL arrays (opac_scale may be
 * NULL), NMC_ENOMEM when the staging cannot be allocated.
 */
int collision_solve_host(nmc_ctx* ctx, const nmc_params* params, int64_t n,
                         const double* rho, const double* T_in, const double* Ye_in,
                         const double* J_in, const double* H_in, const double* dt,
                         const double* opac_scale,
                         double* J_out, double* H_out, double* Ye_out, double* eps_out,
                         double* T_out, int32_t* n_outer, int32_t* n_inner, uint32_t* status,
                         int64_t chunk, void* stream);

/*
 * Autotuner of the fused mode.  Runs collision_solve on the given batch once
 * per variant of the fused kernel that fits the shape: register class
 * (__launch_bounds__ blocks per SM: 3..6 at 128 threads, 1..3 at 256) times a
 * persistent grid of 100% or 50% of the resident capacity.  Each variant runs
 * twice, each run between CUDA events on `stream` (the call synchronises it),
 * and its faster run counts.  The fastest is kept in the context for this precision,
 * Anderson depth (m_inner <= 3 or <= 5) and block class, and later
 * collision_solve calls with matching parameters use it; untuned keys use 4
 * (128 threads), 2 (256) or 1 (512) blocks per SM and the full grid.
 * Arguments as collision_solve (the outputs hold the last variant's results;
 * variants are separate compilations and agree to the solve's accuracy);
 * chosen[2] receives (blocks per SM, grid %)
 * and *ms the winner's time (either may be NULL).  n in 1..2^30.
 */
int nmc_autotune(nmc_ctx* ctx, const nmc_params* params, int64_t n,
                 const double* rho, const double* T_in, const double* Ye_in,
                 const double* J_in, const double* H_in, const double* dt,
                 const double* opac_scale,
                 double* J_out, double* H_out, double* Ye_out, double* eps_out,
                 double* T_out, int32_t* n_outer, int32_t* n_inner, uint32_t* status,
                 int32_t* chosen, float* ms, void* stream);

/*
 * Chunk size (nodes) of NMC_MODE_PLAIN, which keeps per-node state (kernel
 * matrices, Anderson history: ~80 KB per node at 4 species, ne = 32) in
 * device scratch for one chunk at a time.  Default 2^17; nodes >= 1.  The
 * scratch is allocated on the first plain call that needs it and kept until
 * nmc_destroy.
 */
int nmc_set_plain_chunk(nmc_ctx* ctx, int64_t nodes);

/*
 * Tetralinear table interpolation (Sec. 2.3): value of chi_EmAb (which = 0) or
 * sigma_Iso (which = 1) of `species` at p points (rho, T, Ye, E), linear in
 * (log10 rho, log10 T, Ye, ln E) on the table's ln values, exponentiated.
 * Points outside the table are clamped to its edge.  All arrays DEVICE
 * float64 of length p; out[p] receives cm^-1.
 */
int opacity_interp(nmc_ctx* ctx, int32_t which, int32_t species, int64_t p,
                   const double* rho, const double* T, const double* Ye, const double* E,
                   double* out, void* stream);

/*
 * The same interpolation (Sec. 2.3) in FP32: the mixed-precision solve's FP32
 * copies of the ln tables, FP32 logarithms of the coordinates, cell search,
 * weights and blend (the ln value as its first corner plus weighted
 * differences), and an FP32 exp.  Arguments, clamping and errors as
 * opacity_interp (DEVICE float64 in and out); values agree with the FP64
 * entry point to ~1e-6 relative (FP32 rounding of the ln tables and of the
 * coordinates' logarithms), for callers that run the mixed path.
 */
int opacity_interp_mixed(nmc_ctx* ctx, int32_t which, int32_t species, int64_t p,
                         const double* rho, const double* T, const double* Ye, const double* E,
                         double* out, void* stream);

/*
 * Gradient of a converged collision_solve at n nodes (FP64), by the
 * implicit-function theorem (one transposed linear solve per node).  The
 * paper states the implicit step (Eqs. implicitMomentsNodal,
 * implicitFluidNodal, with Eqs. eulerianEnergyLG and eulerianNumberLG); its
 * derivative is this library's addition.
 *
 * At v = 0 the solve's outputs are fixed by its number moments: D (J_out) is
 * the root of G(D) = D - Q_D(D, q(D)) = 0 with y = q(D) the matter update,
 * Ye_out and eps_out are q(D), T_out the EoS temperature of (eps_out, Ye_out),
 * and H_out = I* / (1 + dtau kappa(D, y)).  Given cotangents of those outputs,
 * the call returns the cotangents of the inputs D* (J_in), I* (H_in), Ye_in,
 * T_in and the four opacity scale factors.  dQ_D/dD and dkappa/dD are formed
 * analytically from the node's kernel matrices; dQ_D/dy and dkappa/dy by
 * central differences with steps 1e-6 |eps| and 1e-6 |Ye|.  Each node's
 * Jacobian is solved by Gaussian elimination with partial pivoting per
 * particle/antiparticle pair plus a rank-2 (Woodbury) update for the matter
 * coupling.  The gradient is that of the exact root, so it describes the
 * solve up to the solve's own tolerance.  params must be those of the forward
 * call: proc_mask, d_min, d_max and frozen_matter enter; tolerances,
 * precision and mode do not (the adjoint always runs in FP64).
 *
 * Inputs (DEVICE, float64):
 *   rho, T_in, Ye_in, J_in, dt, opac_scale   the forward call's inputs
 *                                            (opac_scale may be NULL = ones)
 *   H_in[n][ns][ne][3]                       I*; may be NULL when gH_out is NULL
 *   J_out[n][ns][ne]                         converged D from the forward call
 *   T_out[n] or NULL                         forward T_out, the starting guess
 *                                            of the EoS solve (NULL: T_in)
 *   gJ_out[n][ns][ne], gH_out[n][ns][ne][3], gYe_out[n], geps_out[n], gT_out[n]
 *                                            cotangents; any may be NULL = 0
 * Outputs (DEVICE, float64):
 *   gJ_in[n][ns][ne], gYe_in[n], gT_in[n]    required
 *   gH_in[n][ns][ne][3] or NULL              gH_out / (1 + dtau kappa)
 *   gscale[n][4] or NULL                     EmAb, Iso, NES, Pair
 *   status[n] or NULL                        NMC_BAD_INPUT, NMC_EOS_FAIL,
 *                                            NMC_NONFINITE (singular or
 *                                            non-finite), NMC_TABLE_CLAMP; a
 *                                            node with any of the first three
 *                                            gets zero gradients
 * Outputs must not overlap inputs.  Supported shapes: those of
 * collision_solve whose per-block shared memory (kernel matrices plus one
 * 2ne x (2ne+3) FP64 pair system) fits in 227 KB, e.g. ne <= 32 with 4 or 6
 * species; otherwise NMC_EUNSUPPORTED.
 */
int collision_adjoint(nmc_ctx* ctx, const nmc_params* params, int64_t n,
                      const double* rho, const double* T_in, const double* Ye_in,
                      const double* J_in, const double* H_in, const double* dt,
                      const double* opac_scale,
                      const double* J_out, const double* T_out,
                      const double* gJ_out, const double* gH_out, const double* gYe_out,
                      const double* geps_out, const double* gT_out,
                      double* gJ_in, double* gH_in, double* gYe_in, double* gT_in,
                      double* gscale, uint32_t* status, void* stream);

/*
 * FMA-pipe peak probe (a measurement helper; the paper has no counterpart).
 * The collision solve is per-node dense arithmetic, so its roofline is the
 * FMA pipe of its precision, not HBM: FP64 for NMC_FP64, FP32 for NMC_MIXED.
 * Launches, on `stream`, one kernel in which every thread of a full-occupancy
 * grid (blocks_per_sm <= 0: as many 512-thread blocks per SM as fit; else
 * that many) advances sixteen independent FMA chains for `iters` steps, and
 * stores in *flops the launch's flop count (2 per FMA).  The caller times the
 * launch with CUDA events on `stream`.  sink: DEVICE buffer of one element of
 * the precision's type, written only to keep the work live (its value is
 * meaningless).  NMC_EINVAL for iters < 1, a NULL sink or another precision;
 * NMC_ECUDA for a failed launch.
 */
int nmc_fma_probe(int32_t precision, int32_t blocks_per_sm, int32_t iters, void* sink, double* flops,
                  void* stream);

/*
 * Shared-memory load probe (a measurement helper; the paper has no
 * counterpart).  The mixed kernel's contraction loop reads each node's kernel
 * matrices from shared memory every inner iteration, so the shared-memory pipe
 * bounds it.  Launches, on `stream`, one kernel of 1024-thread blocks (as many
 * per SM as fit, 16 KB of static shared memory each) in which every warp issues
 * iters x 64 loads of one kind:
 *   mode 0  4-byte loads of 32 consecutive words (one 128-byte wavefront: the
 *           pipe's peak rate);
 *   mode 1  4-byte warp-uniform (broadcast) loads;
 *   mode 2  8-byte broadcast loads;
 *   mode 3  16-byte broadcast loads;
 *   mode 4  16-byte loads of consecutive words (512 bytes per warp load).
 * Stores in *warp_loads the launch's warp-load count; the caller times the
 * launch with CUDA events on `stream` (mode 0: 128 bytes per warp load).
 * sink: DEVICE buffer of one float, written only to keep the loads live.
 * NMC_EINVAL for iters < 1, a NULL sink or another mode; NMC_ECUDA for a
 * failed launch.
 */
int nmc_smem_probe(int32_t mode, int32_t iters, void* sink, double* warp_loads, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NMC_H */
