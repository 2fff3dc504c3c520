// Fused, persistent kernel for the implicit neutrino--matter collision solve
// (Sec. 3.5, Algorithm 1 with Algorithms 2 and 3), in two precisions:
//   R = double  every step in FP64;
//   R = float   mixed: table interpolation, D^Eq, kernel contractions and the
//               fixed-point sweeps (map Q, residuals, Anderson mixing, Gram
//               sums, Algorithm 2) in FP32, the number moment and the map's
//               numerator as double-floats (two FP32 words); conservation
//               sums, matter update, the Anderson least-squares solves and the
//               final EoS step in FP64.
//
// Mapping.  One thread block solves one spatial node at a time; blocks are
// persistent and take node indices from a device work queue (an atomic
// counter), so nodes with many iterations do not hold up others.  Inside a
// block, thread (s, q) owns species s at energy node q: its moments
// (D, I^1, I^2, I^3), old moments, opacities and its slice of the Anderson
// history (registers).  The node's NES kernels Phi_Out[s] (one ne x ne matrix
// per species) and pair kernels Phi_Ann[p] (one per particle/antiparticle
// pair) live in shared memory, rows padded to ne + 1 so that both row- and
// column-wise reads are free of bank conflicts.
//
// Scaling.  Rates are formed as dimensionless products: matrices hold
// K = dtau * (4 pi / (hc)^3) * Phi and vectors hold W~ D with
// W~_q = w_q eps_q^2 Delta eps_e = W2_q / (4 pi / (hc)^3), so that
// sum_q' K W~ D = dtau * (rate of Eqs. nesRatesNodal / pairRatesNodal);
// chi_EmAb and sigma_Iso are carried as dtau * chi.  Every intermediate is
// O(1e-30 .. 1e8), inside FP32 range.
//
// Per outer iteration (ComputeOpacities of Alg. 1): EoS -> chemical
// potentials; Fermi--Dirac values at the projection quadrature points (all
// threads), eps^2-weighted projection and bound limiter per (species, element)
// (Eq. fermiDiracProjection); trilinear log-table interpolation of chi_EmAb and
// sigma_Iso with coalesced rows of ne energies; bilinear (log10 T, eta)
// interpolation of the kernel tables into shared memory, each tabulated NES
// entry written together with its up-scattering mirror by detailed balance
// (Eqs. inOutInvarianceNES, detailedBalanceNES).
//
// Per inner iteration: rates as shared-memory mat-vecs (Phi_In = Phi_Out^T;
// the antiparticle's Phi_Ann is the transpose; Phi_Pro = a_s(q) a_sbar(q')
// Phi_Ann with a = D^Eq/(1 - D^Eq) by Eq. detailedBalancePair), the map Q
// (Eq. implicitMomentsNodal, v = 0), one block reduction for the Anderson
// least-squares entries, the least-squares solve by the lead warp (FP64,
// lane-parallel), the mixing update, and the Algorithm 2 vote; three barriers.
//
// Matter update (Eq. implicitFluidNodal with Eqs. eulerianEnergyLG,
// eulerianNumberLG): one FP64 block reduction for E_nu and N_nu, the outer
// Anderson step and Algorithm 3 on the lead warp, then T by EoS root finding.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <type_traits>
#include <math.h>

#include "nmc_internal.h"
#include "nmc_eos.cuh"
#include "nmc_device.cuh"

namespace nmc {

namespace {

// Finest relative change of an FP32 moment the mixed path checks (4 ulp of 1).
constexpr double kFp32Resolution = 4.0 * 1.1920928955078125e-7;

template <int MAXM>
struct NodeShared {
    double rho, dtau, T;
    double sc[4];
    double y[2], ystar[2], qv[2];
    double k_eps, k_ye, ri_ys[2];
    double EN_star[2];
    double qh[kMaxOuterMem][2], fh[kMaxOuterMem][2];
    double G[MAXM][MAXM];
    double alpha[MAXM];
    float alpha_f[MAXM];
    double thr[2][kMaxSpecies];   // Algorithm 2 thresholds on the D and I changes (FP64 path)
    float thr_f[2][kMaxSpecies];  // the same rounded to FP32 (mixed path)
    double sp_out[kMaxSpecies * 4];
    double blk_out[8];
    OpacState op;
    long long node;
    int status, n_inner, n_outer;
    int conv_out, bad, done;
};

}  // namespace

// MAXT: block-size class (threads = ns * nep rounded up to 32 must not exceed
// it); MINB blocks per SM cap registers at 128 per thread in every class.
template <typename R, int MAXM, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) fused_kernel(const SolveArgs a) {
    constexpr bool kMixed = sizeof(R) == 4;
    extern __shared__ __align__(16) unsigned char smb[];
    const DevGrid& g = a.g;
    const int NS = g.ns, NE = g.ne, NEP = g.nep, LD = g.ld;
    const int tid = threadIdx.x;
    const int s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const int sq = s * NEP + q;

    R* phi = reinterpret_cast<R*>(smb + a.off_phi);   // [NS][NE][LD]   K_Out per species
    R* ann = reinterpret_cast<R*>(smb + a.off_ann);   // [NS/2][NE][LD] K_Ann per pair (particle)
    // FP64: the contraction vectors in four arrays.  Mixed: two float2 arrays, xw[s][j] = (W~ D, w)
    // and yz[s][j] = (W~ (1 - D) of species s, a W~ (1 - D) of its partner s ^ 1), so that three
    // 8-byte broadcast loads give a bin j's every operand of the NES (own species) and pair (partner
    // species) sums.  An 8-byte broadcast costs the shared-memory pipe about as much as a 4-byte one,
    // a 16-byte broadcast more than twice as much.
    R* vWD = reinterpret_cast<R*>(smb + a.off_vec);   // [NS][NEP] W~ D
    R* vW1D = vWD + NS * NEP;                          //           W~ (1 - D)
    R* vAW1D = vW1D + NS * NEP;                        //           a W~ (1 - D)
    R* vWdev = vAW1D + NS * NEP;                       //           w = W~ (D - D^Eq) / (1 - D^Eq) (mixed)
    float2* xw = reinterpret_cast<float2*>(smb + a.off_vec);   // mixed: [NS][NEP] (W~D, w)
    float2* yz = xw + NS * NEP;                                  //        [NS][NEP] (W~(1-D), partner's aW~(1-D))
    R* vA = vWdev + NS * NEP;                          //           a = D^Eq / (1 - D^Eq)
    R* vAi = vA + NS * NEP;                            //           1 / a
    R* vDeq = vAi + NS * NEP;                          //           D^Eq
    R* vDeqc = vDeq + NS * NEP;                        //           1 - D^Eq (mixed)
    void* red = smb + a.off_red;                       // reduction scratch
    NodeShared<MAXM>* nd = reinterpret_cast<NodeShared<MAXM>*>(smb + a.off_node);
    const OpacBufs<R> ob{phi, ann, vA, vAi, vDeq, vDeqc};

    const nmc_params& P = a.p;
    const bool nes_on = (P.proc_mask & NMC_PROC_NES) != 0;
    const bool pair_on = (P.proc_mask & NMC_PROC_PAIR) != 0;
    const double gs = (s == 0) ? 1.0 : (s == 1 ? -1.0 : 0.0);
    const double W2q = act ? g.w2[q] : 0.0;
    const double W3q = act ? g.w3[q] : 0.0;
    const R Wt = act ? (kMixed ? (R)g.wt_f[q] : (R)g.wt[q]) : (R)0;

    // Mixed precision keeps the number moment D as a double-float (near a fixed
    // point where 1 + dtau chi ~ 1e4, FP32 increments of D fall below one ulp long
    // before the equation residual is small) and its Anderson history Qh[.][0] as
    // FP32 offsets Q_j - D from the current iterate, which are small near
    // convergence: the mixing then costs one double-float add.  A warp's FP64
    // instruction holds its SMSP's FP64 pipe ~64 cycles, so the inner loop issues
    // none per thread; only the lead warp's least squares stays in FP64.
    R Fh[MAXM][4], Qh[MAXM][4];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
#pragma unroll
        for (int c = 0; c < 4; ++c) Fh[j][c] = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) Qh[j][c] = 0;
    }

#ifdef NMC_TRACE
    unsigned long long tr[kTrStages] = {};
    long long tr_t = clock64();
    // thread 0 adds the cycles since the previous boundary to stage st
#define NMC_TRACE_TICK(st) do { if (tid == 0) { const long long t1_ = clock64(); tr[st] += t1_ - tr_t; tr_t = t1_; } } while (0)
#else
#define NMC_TRACE_TICK(st) do { } while (0)
#endif
    for (;;) {
        if (tid == 0) {
            long long nn = atomicAdd(a.queue, 1);
#ifdef NMC_DEBUG
            if (g.dbg && *reinterpret_cast<volatile unsigned*>(g.dbg) != 0u) nn = a.n;   // a check failed: stop
#endif
            nd->node = nn;
        }
        __syncthreads();
        const long long n = nd->node;
        NMC_TRACE_TICK(kTrQueue);
        if (n >= a.n) break;
        // The node's scalar work (EoS, least squares, matter update) runs in lane 0 of one
        // warp.  A warp's FP64 instruction holds its SMSP's FP64 pipe ~64 cycles however
        // few lanes are active, and warp w of every resident block sits on the same SMSP,
        // so the lead warp rotates with the node to spread that work over the SMSPs.
        const int lead = (int)(n % (long long)(blockDim.x >> 5)) << 5;

        // ---------------- node set-up ----------------
        double Dsd = 0.0, Isd[3] = {0.0, 0.0, 0.0};
        if (act) {
            const long long o = (n * NS + s) * NE + q;
            Dsd = a.J[o];
            Isd[0] = a.H[o * 3 + 0];
            Isd[1] = a.H[o * 3 + 1];
            Isd[2] = a.H[o * 3 + 2];
        }
        if (tid == lead) {
            const double rho = a.rho[n], T = a.T[n], Ye = a.Ye[n], dt = a.dt[n];
            nd->rho = rho;
            nd->T = T;
            nd->dtau = kC * dt;
            for (int k = 0; k < 4; ++k) nd->sc[k] = a.scale ? a.scale[n * 4 + k] : 1.0;
            const bool okin = rho > 0.0 && isfinite(rho) && T > 0.0 && isfinite(T) &&
                              Ye > 0.0 && Ye < 1.0 && dt >= 0.0 && isfinite(dt);
            nd->status = okin ? 0 : NMC_BAD_INPUT;
            double e = 0.0, de = 0.0;
            if (okin) eos_eps(rho, T, Ye, &e, &de);
            nd->ystar[0] = e;
            nd->ystar[1] = Ye;
            // per-node factors of the matter update: eps and Ye per unit change of the neutrino
            // energy and lepton number densities, and the outer residuals' scales 1 / |y*|
            nd->k_eps = kMeVErg / rho;
            nd->k_ye = kMB / rho;
            nd->ri_ys[0] = 1.0 / fabs(e);
            nd->ri_ys[1] = 1.0 / fabs(Ye);
            nd->y[0] = e;
            nd->y[1] = Ye;
            nd->n_inner = 0;
            nd->n_outer = 0;
            nd->bad = 0;
            nd->done = okin ? 0 : 1;
        }
        __syncthreads();
        if (nd->done) {   // invalid input: outputs = inputs
            if (act) {
                const long long o = (n * NS + s) * NE + q;
                a.J_out[o] = Dsd;
                for (int j = 0; j < 3; ++j) a.H_out[o * 3 + j] = Isd[j];
            }
            if (tid == lead) {
                a.Ye_out[n] = a.Ye[n];
                a.eps_out[n] = nd->ystar[0];
                a.T_out[n] = a.T[n];
                a.n_outer[n] = 0;
                a.n_inner[n] = 0;
                a.status[n] = nd->status;
            }
            __syncthreads();
            continue;
        }
        {   // E_nu*, N_nu* in FP64 (Eqs. eulerianEnergyLG, eulerianNumberLG at v = 0)
            double v[2] = {W3q * Dsd, gs * W2q * Dsd};
            block_sum<2, double>(v, red, nd->blk_out);
            if (tid == lead) { nd->EN_star[0] = nd->blk_out[0]; nd->EN_star[1] = nd->blk_out[1]; }
        }
        const R Ds = (R)Dsd;
        const R Is[3] = {(R)Isd[0], (R)Isd[1], (R)Isd[2]};
        R M[4] = {Ds, Is[0], Is[1], Is[2]};
        // mixed: the number moment as a double-float (M[0] is its high word), and per outer
        // iteration the numerator W~ (D* - D) + W~ dtau chi_EmAb (D^Eq - D) = A0 - c12 D
        F2 Dx = f2_from(Dsd), A0x = {0.f, 0.f}, c12x = {0.f, 0.f};
        R chiab = 0, sig = 0, deq = 0, deqc = 0;
        int outer_exit = 0;
        NMC_TRACE_TICK(kTrSetup);

        for (int k = 1;; ++k) {
            // ================= ComputeOpacities(y^[k]) =================
            // semi-implicit (Sec. 3.5): only at y^[1] = y*; the shared kernels, chiab, sig and
            // D^Eq of the first outer iteration stay in place (nothing else writes them)
            if (k == 1 || !P.semi_implicit)
                compute_opacities<R>(g, a.tb, P, nd->rho, nd->T, nd->y[1], nd->dtau, nd->sc, ob, &nd->op,
                                     &nd->status, chiab, sig, deq, deqc, lead);
            NMC_TRACE_TICK(kTrOpac);
            if constexpr (kMixed) {
                const double c1 = (double)Wt, c2 = c1 * (double)chiab;
                A0x = f2_from(c1 * Dsd + c2 * (double)deq);
                c12x = f2_from(c1 + c2);
            }
            // reference norm ||D^[k,1]||_W per species (Algorithm 2 input)
            {
                R v[1] = {Wt * M[0] * M[0]};
                R* out = reinterpret_cast<R*>(nd->sp_out);
                species_sum<1, R>(v, red, out, NEP, NS);
                if (tid == lead) {
                    const double fl = P.norm_floor * sqrt(g.sum_wt);
                    // mixed precision: D is a double-float iterate held to tol_inner; the first
                    // moments are FP32 values, checked against FP32 resolution at the finest
                    const double tol_i = kMixed ? fmax(P.tol_inner, kFp32Resolution) : P.tol_inner;
                    for (int sp = 0; sp < NS; ++sp) {
                        const double dn = fmax((double)r_sqrt(out[sp]), fl);
                        nd->thr[0][sp] = P.tol_inner * dn;
                        nd->thr[1][sp] = tol_i * dn;
                        nd->thr_f[0][sp] = (float)(P.tol_inner * dn);
                        nd->thr_f[1][sp] = (float)(tol_i * dn);
                    }
                }
            }
            // The vectors every bin's contractions read: W~ D, W~ (1 - D), a W~ (1 - D) and (mixed)
            // the deviation w.  Mixed: the blocking factor 1 - D and the deviation D - D^Eq are
            // formed from both words of D (1 - D in FP32 has no digits left at D ~ 1 - 1e-6);
            // 1 - D.h, and D.h - D^Eq near equilibrium, are exact.
            const R aq = act ? vA[sq] : (R)0;
            R myW1D = 0, myAW1D = 0, myWdev = 0;   // mixed: this bin's own vector entries
            auto publish = [&](R D32, F2 D2) {
                if (act) {
                    const R hole = kMixed ? (R)__fsub_rn(__fsub_rn(1.0f, D2.h), D2.l) : (R)1 - D32;
                    if constexpr (kMixed) {
                        myW1D = Wt * hole;
                        myAW1D = aq * Wt * hole;
                        myWdev = __fadd_rn(__fsub_rn(D2.h, (float)deq), D2.l) * (Wt / deqc);
                        xw[sq] = make_float2(Wt * D32, myWdev);
                        yz[sq].x = myW1D;
                        yz[(s ^ 1) * NEP + q].y = myAW1D;
                    } else {
                        vWD[sq] = Wt * D32;
                        vW1D[sq] = Wt * hole;
                        vAW1D[sq] = aq * Wt * hole;
                    }
                }
            };
            publish(M[0], Dx);
            __syncthreads();
            NMC_TRACE_TICK(kTrNorms);
            bool inner_stop = false;   // the inner loop hit its cap or a non-finite moment
            // ================= inner loop =================
            // Three barriers an iteration: the Gram row's warp partials, the least-squares
            // coefficients, and the convergence vote.  The next iterate's vectors are written once
            // the coefficients are out (no thread reads the old ones after that) and the vote's
            // barrier publishes them.
            for (int ell = 1;; ++ell) {
                R F[4] = {0, 0, 0, 0}, Qv[4] = {0, 0, 0, 0};
                R dlt = 0;         // mixed: Q_D - D, formed without cancellation
                // NMC_DEBUG: the contraction's shared-memory indices are affine in j, so their
                // extremes bound every one of them (own and partner vectors, both matrix sweeps)
                const bool idx_ok = !act ||
                    NMC_IN_BOUNDS(g.dbg, (long long)s * NE * LD + (NE - 1) * LD + q, (long long)NS * NE * LD, kDbgSmemNes) &&
                    NMC_IN_BOUNDS(g.dbg, (long long)s * NE * LD + q * LD + NE - 1, (long long)NS * NE * LD, kDbgSmemNes) &&
                    NMC_IN_BOUNDS(g.dbg, (long long)(s >> 1) * NE * LD + (NE - 1) * LD + NE - 1, (long long)(NS / 2) * NE * LD,
                                  kDbgSmemPair) &&
                    NMC_IN_BOUNDS(g.dbg, (long long)(s ^ 1) * NEP + NE - 1, (long long)NS * NEP, kDbgSmemVec);
                if (act && idx_ok) {
                    R nin = 0, nout = 0, pro = 0, an = 0;
                    R cn = 0, cp = 0;   // mixed: net NES / pair exchange terms (deviation form)
                    if (kMixed && nes_on && pair_on) {
                        // both sums in one pass over j (the terms as in the separate loops below).  The
                        // sweep is compiled for ne = 64 and 32 with the row stride a constant, so that
                        // the matrix loads take immediate offsets instead of per-load index arithmetic
                        // (5% of the headline solve); other ne take the same loop with runtime strides.
                        const int pt = s ^ 1;
                        const bool part = (s & 1) == 0;
                        const float2* Xo = xw + s * NEP;
                        const float2* Xp = xw + pt * NEP;
                        const float2* Yo = yz + s * NEP;
                        const R wq = myWdev, vq = myW1D;
                        R cw = 0;
                        auto sweep = [&](auto nec) {
                            constexpr int kNe = decltype(nec)::value;   // 0: ne known at run time only
                            const int ne = kNe ? kNe : NE, ld = kNe ? kNe + 1 : LD;
                            const R* P0 = phi + s * ne * ld;
                            const R* A0 = ann + (s >> 1) * ne * ld;
                            const int stride_j = part ? 1 : ld;
                            const int base = part ? q * ld : q;
#pragma unroll 4
                            for (int j = 0; j < ne; ++j) {
                                const float2 u = Xo[j], t = Xp[j], y = Yo[j];   // y.x: own W~(1-D), y.y: partner's aW~(1-D)
                                const R kin = P0[j * ld + q], kout = P0[q * ld + j];
                                nin = r_fma(kin, u.x, nin);
                                nout = r_fma(kout, y.x, nout);
                                const R e1 = __fmul_rn(kin, __fmul_rn(u.y, vq));
                                const R e2 = __fmul_rn(kout, __fmul_rn(wq, y.x));
                                cn = __fadd_rn(cn, __fsub_rn(e1, e2));
                                const R av = A0[base + j * stride_j];
                                pro = r_fma(av, y.y, pro);
                                an = r_fma(av, t.x, an);
                                cw = r_fma(av, t.y, cw);
                            }
                        };
                        if (NE == 64) sweep(std::integral_constant<int, 64>{});
                        else if (NE == 32) sweep(std::integral_constant<int, 32>{});
                        else sweep(std::integral_constant<int, 0>{});
                        cp = -r_fma(myWdev, cw + pro, myAW1D * cw);
                        pro *= aq;
                    } else {
                    if (nes_on) {
                        const R* P0 = phi + s * NE * LD;
                        const R* x = vWD + s * NEP;
                        const R* y = vW1D + s * NEP;
                        if constexpr (kMixed) {
                            // Net exchange with bin j: K[j][q] u_j v_q - K[q][j] u_q v_j, u = W~ D,
                            // v = W~ (1 - D).  With detailed balance K[q][j] a_q = K[j][q] a_j (the
                            // way the up-scattering half is built) it equals
                            // K[j][q] w_j v_q - K[q][j] w_q v_j, w = u - a v = W~ (D - D^Eq)/(1 - D^Eq):
                            // every term is proportional to the deviation from equilibrium, so FP32
                            // rounding is relative to the net rate, not to the gross rates that are
                            // dtau chi ~ 1e4 times larger in optically thick matter.  Each product is
                            // formed with the same operands in the two bins it couples and
                            // fl(e1 - e2) in bin q is exactly minus its counterpart in bin j, so the
                            // map conserves number to the rounding of the sums: NES then leaves no
                            // rounding source in the slowly damped number-conserving mode (factored
                            // into dot products, it raised the heavy flavours' error 20-fold).
                            const float2* Xo = xw + s * NEP;
                            const float2* Yo = yz + s * NEP;
                            const R wq = myWdev, vq = myW1D;
                            for (int j = 0; j < NE; ++j) {
                                const float2 u = Xo[j];
                                const R yj = Yo[j].x;
                                const R kin = P0[j * LD + q], kout = P0[q * LD + j];
                                nin = r_fma(kin, u.x, nin);        // K_In[q][j] = K_Out[j][q]
                                nout = r_fma(kout, yj, nout);
                                const R e1 = __fmul_rn(kin, __fmul_rn(u.y, vq));
                                const R e2 = __fmul_rn(kout, __fmul_rn(wq, yj));
                                cn = __fadd_rn(cn, __fsub_rn(e1, e2));
                            }
                        } else {
                            for (int j = 0; j < NE; ++j) {
                                nin = r_fma(P0[j * LD + q], x[j], nin);    // K_In[q][j] = K_Out[j][q]
                                nout = r_fma(P0[q * LD + j], y[j], nout);
                            }
                        }
                    }
                    if (pair_on) {
                        const int pt = s ^ 1;
                        const R* A0 = ann + (s >> 1) * NE * LD;
                        const R* x = vAW1D + pt * NEP;
                        const R* y = vWD + pt * NEP;
                        // mixed: the pair (q, j) is produced at K_Ann p_q pbar_j and annihilated at
                        // K_Ann u_q ubar_j (p = a v); with u = w + p the net gain of either bin is
                        // -K_Ann (w_P w_A + w_P p_A + p_P w_A) (P particle, A antiparticle),
                        // proportional to the deviations.  Summed over j, with s the bin's own
                        // species and t its partner, it is -(w_s (C + X) + p_s C) with
                        // C = sum_j K w_t,j and X = sum_j K p_t,j (the emissivity's dot product).
                        const bool part = (s & 1) == 0;
                        const int stride_j = part ? 1 : LD;
                        const int base = part ? q * LD : q;
                        R cw = 0;
                        if constexpr (kMixed) {
                            const float2* Xp = xw + pt * NEP;
                            const float2* Yo = yz + s * NEP;
                            for (int j = 0; j < NE; ++j) {
                                const float2 t = Xp[j];
                                const R av = A0[base + j * stride_j];
                                pro = r_fma(av, Yo[j].y, pro);
                                an = r_fma(av, t.x, an);
                                cw = r_fma(av, t.y, cw);
                            }
                            cp = -r_fma(myWdev, cw + pro, myAW1D * cw);
                        } else {
                            for (int j = 0; j < NE; ++j) {
                                const R av = A0[base + j * stride_j];
                                pro = r_fma(av, x[j], pro);
                                an = r_fma(av, y[j], an);
                            }
                        }
                        pro *= aq;
                    }
                    }
                    const R eta = chiab * deq + nin + pro;          // dtau * Eq. emissivityNodal
                    const R chi = chiab + nin + nout + pro + an;    // dtau * Eq. opacityNodal
                    const R kap = chi + sig;                        // dtau * Eq. transportOpacityNodal
                    if constexpr (kMixed) {
                        // the same map written as Q_D = D + W~ (D* - D + dtau C) / (W~ (1 + dtau chi)),
                        // with the net collision term W~ dtau C = W~ dtau chi_EmAb (D^Eq - D) + net NES
                        // + net pair exchanges.  The numerator, whose zero is the fixed point, is
                        // summed in double-float around the double-float D; the denominator only
                        // scales the step, so FP32 rounding in chi does not move the fixed point.
                        // The history holds Q_D - D (the offset of the map value from the iterate).
                        const R numW = f2_residual(A0x, c12x, Dx, cn + cp);
                        const R inv = (R)1 / ((R)1 + chi);
                        dlt = numW * (inv / Wt);
                        Qv[0] = dlt;
                    }
                    R fI;
                    if constexpr (kMixed) {
                        fI = (R)1 / ((R)1 + kap);
                    } else {
                        // Eq. implicitMomentsNodal at v = 0, both quotients from one FP64 division
                        const R d1 = (R)1 + chi, d2 = (R)1 + kap, rr = (R)1 / (d1 * d2);
                        Qv[0] = (Ds + eta) * d2 * rr;
                        fI = d1 * rr;
                    }
                    Qv[1] = Is[0] * fI;
                    Qv[2] = Is[1] * fI;
                    Qv[3] = Is[2] * fI;
#pragma unroll
                    for (int c = 0; c < 4; ++c) F[c] = Qv[c] - M[c];
                    if constexpr (kMixed) F[0] = dlt;
                }
#pragma unroll
                for (int j = 0; j < MAXM - 1; ++j) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) { Fh[j][c] = Fh[j + 1][c]; Qh[j][c] = Qh[j + 1][c]; }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) { Fh[MAXM - 1][c] = F[c]; Qh[MAXM - 1][c] = Qv[c]; }
                const int m = ell < P.m_inner ? ell : P.m_inner;
                if (!NMC_IN_BOUNDS(g.dbg, m - 1, MAXM, kDbgHistory)) nd->bad = 1;
                if constexpr (MAXM == 3) {
                    // Least squares in FP64 by the lead warp (anderson3_warp), lane k adding the warps'
                    // partials of entry k.  FP64: the new Gram row, kept in the history G.  Mixed: the
                    // block sums are the eliminated normal equations themselves, from FP32 differences
                    // dF_i = F_L - F_gi (no FP64 formation, no history, no cancellation between Gram
                    // entries).  The fit covers all four moments, as Algorithm 1 does; fitted to the
                    // number moments alone, it kept extrapolating once their residual reached the FP32
                    // noise of the exchange sums and some nodes cycled above tol_inner.
                    constexpr int K = kMixed ? 5 : 3;
                    R v[K];
                    if constexpr (kMixed) {
                        R d0[4], d1[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            d0[c] = F[c] - (m >= 3 ? Fh[0][c] : Fh[1][c]);
                            d1[c] = F[c] - Fh[1][c];
                        }
                        v[0] = d0[0] * d0[0] + d0[1] * d0[1] + d0[2] * d0[2] + d0[3] * d0[3];
                        v[1] = d0[0] * d1[0] + d0[1] * d1[1] + d0[2] * d1[2] + d0[3] * d1[3];
                        v[2] = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2] + d1[3] * d1[3];
                        v[3] = d0[0] * F[0] + d0[1] * F[1] + d0[2] * F[2] + d0[3] * F[3];
                        v[4] = d1[0] * F[0] + d1[1] * F[1] + d1[2] * F[2] + d1[3] * F[3];
                    } else {
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            v[j] = F[0] * Fh[j][0] + F[1] * Fh[j][1] + F[2] * Fh[j][2] + F[3] * Fh[j][3];
                    }
                    NMC_TRACE_TICK(kTrContract);
                    warp_partials<K, R>(v, red);
                    __syncthreads();
                    NMC_TRACE_TICK(kTrGram);
                    if ((tid >> 5) == (lead >> 5)) {
                        const int k = tid & 31;
                        const R* pr = reinterpret_cast<const R*>(red);
                        R sk = 0;
                        if (k < K)
                            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sk += pr[i * K + k];
                        double e;
                        if constexpr (kMixed) e = (double)sk;
                        else e = gram3_update_warp<3>(nd->G, sk, m);
                        double c0, c1, cL;
                        anderson3_warp(e, m - 1, c0, c1, cL);
                        if (k < 3) {
                            const double a = anderson3_coef(k, m - 1, c0, c1, cL);
                            nd->alpha[k] = a;
                            nd->alpha_f[k] = (float)a;
                        }
                    }
                    __syncthreads();
                    NMC_TRACE_TICK(kTrSolve);
                } else {   // new row of the Gram matrix; the lead adds the warps' partials and solves
                           // the least squares in FP64
                    R v[MAXM];
#pragma unroll
                    for (int j = 0; j < MAXM; ++j) {
                        v[j] = F[0] * Fh[j][0] + F[1] * Fh[j][1] + F[2] * Fh[j][2] + F[3] * Fh[j][3];
                    }
                    NMC_TRACE_TICK(kTrContract);
                    warp_partials<MAXM, R>(v, red);
                    __syncthreads();
                    NMC_TRACE_TICK(kTrGram);
                    if (tid == lead) {
                        R out[MAXM];
                        sum_partials<MAXM, R>(red, out);
                        for (int i = 0; i < MAXM - 1; ++i)
                            for (int j = 0; j < MAXM - 1; ++j) nd->G[i][j] = nd->G[i + 1][j + 1];
                        for (int j = 0; j < MAXM; ++j) {
                            nd->G[MAXM - 1][j] = (double)out[j];
                            nd->G[j][MAXM - 1] = (double)out[j];
                        }
                        anderson_solve<MAXM>(nd->G, m, nd->alpha);
                        for (int j = 0; j < MAXM; ++j) nd->alpha_f[j] = (float)nd->alpha[j];
                    }
                    __syncthreads();
                    NMC_TRACE_TICK(kTrSolve);
                }
                R Mn[4];
#pragma unroll
                for (int c = kMixed ? 1 : 0; c < 4; ++c) {   // mixed: D below, in offset form
                    R acc = 0;
#pragma unroll
                    for (int j = 0; j < MAXM; ++j)
                        if (j >= MAXM - m)   // window only
                            acc = r_fma(kMixed ? (R)nd->alpha_f[j] : (R)nd->alpha[j], Qh[j][c], acc);
                    Mn[c] = act ? acc : (R)0;
                }
                F2 Dxn = Dx;
                R sD = 0;   // mixed: D^new - D
                if constexpr (kMixed) {
                    // in difference form, o_L + sum_j alpha_j (o_j - o_L) with o = Q - D: the
                    // rounding of alpha scales only the small differences of the window
                    R acc = Qh[MAXM - 1][0];
#pragma unroll
                    for (int j = 0; j < MAXM - 1; ++j)
                        if (j >= MAXM - m) acc = r_fma((R)nd->alpha_f[j], Qh[j][0] - Qh[MAXM - 1][0], acc);
                    sD = act ? acc : (R)0;
                    Dxn = f2_add(Dx, sD);
                    Mn[0] = Dxn.h;
                }
                publish(Mn[0], Dxn);
                NMC_TRACE_TICK(kTrMix);
                int vote = 1;
                {   // Algorithm 2: per species, W-weighted squares of the change per moment
                    R v[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) { const R d = Mn[c] - M[c]; v[c] = Wt * d * d; }
                    if constexpr (kMixed) v[0] = Wt * sD * sD;
                    if (act && !(isfinite(Mn[0]) && isfinite(Mn[1]) && isfinite(Mn[2]) && isfinite(Mn[3]) &&
                                 isfinite(sD)))
                        nd->bad = 1;
                    auto species_ok = [&](const R* u, int sp) -> int {
                        R mx = u[1];
                        for (int c = 2; c < 4; ++c) mx = fmax(mx, u[c]);
                        if constexpr (kMixed)
                            return r_sqrt(u[0]) <= nd->thr_f[0][sp] && r_sqrt(mx) <= nd->thr_f[1][sp];
                        else
                            return r_sqrt(u[0]) <= nd->thr[0][sp] && r_sqrt(mx) <= nd->thr[1][sp];
                    };
                    if (NEP <= 32) {
                        // a species group lies inside one warp: its sums are formed in registers
                        // (the butterfly leaves the same sum in every lane of the group) and each
                        // lane votes for its own species
                        for (int off = NEP >> 1; off > 0; off >>= 1) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) v[c] += __shfl_xor_sync(kFull, v[c], off);
                        }
                        if (s < NS) vote = species_ok(v, s);
                    } else {
                        // a species spans NEP / 32 warps: warp sums by shuffles, then a barrier over that
                        // species' warps only (named barrier 1 + s; barrier 0 is the block's), after which
                        // every thread adds its species' partials in the same order and votes for it.  The
                        // scratch is free here: the lead warp read the Gram partials before the previous
                        // barrier, and the next ones are written after the vote's.
                        const int wps = NEP >> 5, lane = tid & 31, w = tid >> 5;
                        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) v[c] += __shfl_xor_sync(kFull, v[c], off);
                        }
                        R* pv = reinterpret_cast<R*>(red);
                        if (lane == 0) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) pv[w * 4 + c] = v[c];
                        }
                        asm volatile("bar.sync %0, %1;" ::"r"(1 + s), "r"(wps * 32) : "memory");
                        R u[4] = {0, 0, 0, 0};
                        for (int i = 0; i < wps; ++i) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) u[c] += pv[(s * wps + i) * 4 + c];
                        }
                        vote = species_ok(u, s);
                    }
                }
                const bool conv = __syncthreads_and(vote) != 0;
                const bool bad = *reinterpret_cast<volatile int*>(&nd->bad) != 0;
                const bool capped = !conv && !bad && ell >= P.max_inner;
                if (tid == lead) {
                    nd->n_inner += 1;
                    if (bad) nd->status |= NMC_NONFINITE;
                    if (capped) nd->status |= NMC_NOT_CONVERGED_INNER;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) M[c] = Mn[c];
                Dx = Dxn;
                if constexpr (kMixed) {   // offsets now relative to the new iterate
#pragma unroll
                    for (int j = 0; j < MAXM; ++j) Qh[j][0] -= sD;
                }
                NMC_TRACE_TICK(kTrVote);
                if (conv || bad || ell >= P.max_inner) {
                    inner_stop = bad || capped;
                    break;
                }
            }
            // an inner loop stopped at its cap (or a non-finite moment) ends the node
            if (P.frozen_matter || inner_stop) outer_exit = 1;
            // ================= matter update (Eq. implicitFluidNodal), FP64 =================
            if (!outer_exit) {
                const double Dcur = kMixed ? f2_to(Dx) : (double)M[0];
                double v[2] = {W3q * Dcur, gs * W2q * Dcur};
                block_sum<2, double>(v, red, nd->blk_out);
                if ((tid >> 5) == (lead >> 5)) {
                    // The lead warp, every lane carrying the node's scalars: a scalar FP64 step costs
                    // the same on 1 or 32 lanes, and the outer least squares runs lane-parallel.
                    // Lane 0 writes the shared state.
                    const int ln = tid & 31;
                    const double rho = nd->rho;
                    const double qv0 = nd->ystar[0] - (nd->blk_out[0] - nd->EN_star[0]) * nd->k_eps;
                    const double qv1 = nd->ystar[1] - (nd->blk_out[1] - nd->EN_star[1]) * nd->k_ye;
                    const double y0 = nd->y[0], y1 = nd->y[1];
                    if (ln == 0) { nd->qv[0] = qv0; nd->qv[1] = qv1; }
                    const int mo = k < P.m_outer ? k : P.m_outer;
                    double yn0, yn1;
                    outer_step_warp(nd->qh, nd->fh, qv0, qv1, y0, y1, nd->ri_ys, mo, yn0, yn1);
                    const int conv = fabs(yn0 - y0) <= P.tol_outer * fabs(nd->ystar[0]) &&
                                     fabs(yn1 - y1) <= P.tol_outer * fabs(nd->ystar[1]);   // Algorithm 3
                    int stop = conv, st = 0;
                    double Tn = nd->T;
                    if (!(isfinite(yn0) && isfinite(yn1))) { st |= NMC_NONFINITE; stop = 1; }
                    if (!stop && k >= P.max_outer) { st |= NMC_NOT_CONVERGED_OUTER; stop = 1; }
                    if (!stop) {   // an iterate outside the EoS domain stops the node
                        bool ok;
                        const double Tk = kMixed ? eos_temperature_mixed(rho, yn0, yn1, Tn, &ok)
                                                 : eos_temperature(rho, yn0, yn1, Tn, &ok);
                        if (ok) Tn = Tk;
                        else { st |= NMC_EOS_FAIL; stop = 1; }
                    }
                    if (ln == 0) {
                        nd->y[0] = yn0;
                        nd->y[1] = yn1;
                        nd->T = Tn;
                        nd->status |= st;
                        nd->conv_out = stop;
                    }
                }
                __syncthreads();
                if (nd->conv_out) outer_exit = 1;
            }
            NMC_TRACE_TICK(kTrMatter);
            if (outer_exit) {
                if (tid == lead) nd->n_outer = k;
                break;
            }
        }
        // ================= finalize =================
        {   // q(M, y) at the final moments (Eq. implicitFluidNodal), FP64
            const double Dcur = kMixed ? f2_to(Dx) : (double)M[0];
            double v[2] = {W3q * Dcur, gs * W2q * Dcur};
            block_sum<2, double>(v, red, nd->blk_out);
            if (tid == lead) {
                nd->qv[0] = nd->ystar[0] - (nd->blk_out[0] - nd->EN_star[0]) * nd->k_eps;
                nd->qv[1] = nd->ystar[1] - (nd->blk_out[1] - nd->EN_star[1]) * nd->k_ye;
            }
        }
        if (tid == lead) {
            const double rho = nd->rho;
            double yo0, yo1, To;
            if (P.frozen_matter) {
                yo0 = nd->ystar[0]; yo1 = nd->ystar[1]; To = a.T[n];
            } else if (nd->status & NMC_NONFINITE) {
                yo0 = nd->y[0]; yo1 = nd->y[1]; To = nd->T;
            } else {
                if (P.final_q) { yo0 = nd->qv[0]; yo1 = nd->qv[1]; }   // y = q(M, y) at converged M
                else { yo0 = nd->y[0]; yo1 = nd->y[1]; }                // Anderson-mixed iterate
                bool ok;
                To = kMixed ? eos_temperature_mixed(rho, yo0, yo1, nd->T, &ok)
                            : eos_temperature(rho, yo0, yo1, nd->T, &ok);
                if (!ok) { nd->status |= NMC_EOS_FAIL; To = nd->T; }   // last T inside the domain
            }
            a.Ye_out[n] = yo1;
            a.eps_out[n] = yo0;
            a.T_out[n] = To;
            a.n_outer[n] = nd->n_outer;
            a.n_inner[n] = nd->n_inner;
            a.status[n] = (uint32_t)nd->status;
        }
        if (act && NMC_IN_BOUNDS(g.dbg, (n * NS + s) * NE + q, a.n * NS * NE, kDbgOutput)) {
            const long long o = (n * NS + s) * NE + q;
            a.J_out[o] = kMixed ? f2_to(Dx) : (double)M[0];
            a.H_out[o * 3 + 0] = (double)M[1];
            a.H_out[o * 3 + 1] = (double)M[2];
            a.H_out[o * 3 + 2] = (double)M[3];
        }
        __syncthreads();
        NMC_TRACE_TICK(kTrFinal);
    }
#ifdef NMC_TRACE
    if (tid == 0 && g.trace)
        for (int st = 0; st < kTrStages; ++st) atomicAdd(g.trace + st, tr[st]);
#endif
#undef NMC_TRACE_TICK
}

template <typename R, int MAXM, int MAXT, int MINB>
static int launch_impl(nmc_ctx* ctx, SolveArgs a, cudaStream_t stream, int grid_pct) {
    auto kern = fused_kernel<R, MAXM, MAXT, MINB>;
    const size_t smem = fused_smem_bytes(ctx, MAXM, sizeof(R) == 4, &a);
    if ((int)smem > ctx->max_smem_optin)
        return set_error(ctx, NMC_EUNSUPPORTED, "shared-memory footprint of the fused kernel exceeds the per-block limit");
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess || per_sm < 1)
        return set_error(ctx, NMC_EUNSUPPORTED, "fused kernel cannot be resident with this shape");
    long long grid = (long long)per_sm * ctx->num_sms * grid_pct / 100;
    if (grid < ctx->num_sms) grid = ctx->num_sms;
    if (grid > a.n) grid = a.n;
    e = cudaMemsetAsync(a.queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    kern<<<(unsigned)grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("fused kernel launch: ") + cudaGetErrorString(e));
    return NMC_OK;
}

// Kernel variant v: register class (blocks per SM the registers must allow) and
// persistent grid size.  Block-size classes follow the shape: threads =
// ns * nep rounded up to 32 must not exceed MAXT.
template <typename R, int MAXM>
static int launch_by_variant(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream, FusedVariant v) {
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    if (threads <= 128) {
        switch (v.minb) {
            case 3: return launch_impl<R, MAXM, 128, 3>(ctx, a, stream, v.grid_pct);
            case 5: return launch_impl<R, MAXM, 128, 5>(ctx, a, stream, v.grid_pct);
            case 6: return launch_impl<R, MAXM, 128, 6>(ctx, a, stream, v.grid_pct);
            default: return launch_impl<R, MAXM, 128, 4>(ctx, a, stream, v.grid_pct);
        }
    }
    if (threads <= 256) {
        switch (v.minb) {
            case 1: return launch_impl<R, MAXM, 256, 1>(ctx, a, stream, v.grid_pct);
            case 3: return launch_impl<R, MAXM, 256, 3>(ctx, a, stream, v.grid_pct);
            default: return launch_impl<R, MAXM, 256, 2>(ctx, a, stream, v.grid_pct);
        }
    }
    return launch_impl<R, MAXM, 512, 1>(ctx, a, stream, v.grid_pct);
}

// Loads every variant launch_by_variant can pick (a function-attribute query
// loads a kernel under CUDA's lazy module loading), so that set-up, not the
// first solve, pays for it.
template <typename R, int MAXM>
static cudaError_t preload_variants() {
    cudaFuncAttributes fa;
    const void* k[] = {(const void*)fused_kernel<R, MAXM, 128, 3>, (const void*)fused_kernel<R, MAXM, 128, 4>,
                       (const void*)fused_kernel<R, MAXM, 128, 5>, (const void*)fused_kernel<R, MAXM, 128, 6>,
                       (const void*)fused_kernel<R, MAXM, 256, 1>, (const void*)fused_kernel<R, MAXM, 256, 2>,
                       (const void*)fused_kernel<R, MAXM, 256, 3>, (const void*)fused_kernel<R, MAXM, 512, 1>};
    for (const void* f : k) {
        const cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace nmc
