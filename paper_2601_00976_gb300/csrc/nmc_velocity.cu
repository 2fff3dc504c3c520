// O(v/c) collision solve (FP64): Algorithm 1 with the velocity-dependent terms
// of Sec. 3.5.
//
// Per node the fluid three-velocity v (units of c, flat metric at the node)
// enters three places:
//  - the conserved moments of the old state, N* = D* + v*^i I*_i and
//    G*_j = I*_j + v*^i K_ij(M*) (Eq. conservedToPrimitive), with K_ij = k_ij D
//    from Minerbo's closure (Eqs. eddingtonTensor, eddingtonFactorMinerbo);
//  - the moment map Q of Eq. implicitMomentsNodal,
//      D <- ((1 - lam) D + lam (N* - v.I + dtau eta)) / (1 + lam dtau chi),
//      I_j <- ((1 - lam) I_j + lam (G*_j - v^i K_ij)) / (1 + lam dtau kappa),
//    with lam = 1 / (1 + |v|) and v the velocity of the current matter iterate;
//  - with linear-order (Phi_1) kernels in the tables, their NES and pair terms
//    (Eqs. zerothMomentCollisionTerm_NES/Pair, firstMomentCollisionTerm_NES/Pair)
//    as explicit additions to dtau eta and to the flux numerator;
//  - the matter map q of Eq. implicitFluidNodal: momentum, total specific
//    energy eps_f and Ye from the Eulerian sums F_nu, E_nu, N_nu
//    (Eqs. eulerianMomentumLG, eulerianEnergyLG, eulerianNumberLG), the
//    temperature from eps = eps_f - v^2 / 2.
// The matter state y = (v_1, v_2, v_3, eps_f, Ye) is iterated by the outer
// Anderson step on residuals scaled by (max(|v*|, v_floor) x 3, |eps_f*|,
// |Ye*|), which Algorithm 3 also uses.  The returned state solves the momentum
// update for v exactly (it is affine in v: a 3 x 3 solve) and takes eps_f and
// Ye with that v, so momentum, energy and lepton number are conserved to
// rounding.
//
// Kernel layout as the fused FP64 kernel: persistent blocks on a device work
// queue, thread (s, q) owns species s at energy q, the node's kernel matrices
// in shared memory, the scalar work on a lead warp that rotates with the node
// (lane-parallel least squares), three barriers per inner iteration.  The
// Eulerian sums of a state are fifteen block sums per thread: W3 D, W3 I_j,
// W3 a and W3 c I_j I_k (K_jk = a delta_jk + c I_j I_k), W2 g D, W2 g I_j.
#include <cuda_runtime.h>
#include <math.h>

#include <string>

#include "nmc_internal.h"
#include "nmc_eos.cuh"
#include "nmc_device.cuh"

namespace nmc {

namespace {

constexpr int kNy = 5;      // (v_1, v_2, v_3, eps_f, Ye)
constexpr int kNsum = 15;   // Eulerian block sums of one state

struct VelNode {
    double rho, dtau, T;
    double sc[4];
    double y[kNy], ystar[kNy], ri[kNy];   // matter iterate, old state, 1 / Algorithm 3 reference
    double Fs[3], Es, Ns;                 // Eulerian momentum, energy and number of the old state
    double cf, k_eps, k_ye, lam;          // MeV/(rho c^2), MeV/rho, m_B/rho, 1/(1+|v|)
    double qh[kMaxOuterMem][kNy], fh[kMaxOuterMem][kNy];
    double G[3][3];
    double alpha[3];
    double thr[2][kMaxSpecies];
    double sp_out[kMaxSpecies * 4];
    double blk_out[16];
    OpacState op;
    long long node;
    int status, n_inner, n_outer, conv_out, bad, done;
};

// a = 1/2 (1 - psi) D and c = 1/2 (3 psi - 1) D / |I|^2 of K_jk = a delta_jk + c I_j I_k
// (Eq. eddingtonTensor with Minerbo's psi, Eq. eddingtonFactorMinerbo), h = |I| / D
// clipped to [0, 1].  With Minerbo's polynomial, 3 psi - 1 = (2/5)(3 - h + 3h^2) h^2,
// so for h < 1, c = (3 - h + 3h^2) / (5 D): no division by |I|^2 and no cancellation in
// 3 psi - 1 (whose FP64 rounding residue over a |I|^2 decayed into the denormals would
// overflow).  At h = 1 (|I| >= D > 0) psi = 1 and c = D / |I|^2.  D <= 0: K = (D/3) delta.
__device__ __forceinline__ void closure_ac(double D, double I0, double I1, double I2, double& a, double& c) {
    const double In2 = I0 * I0 + I1 * I1 + I2 * I2;
    if (!(D > 0.0)) {
        a = D / 3.0;
        c = 0.0;
        return;
    }
    const double h = sqrt(In2) / D;
    if (h >= 1.0) {
        a = 0.0;
        c = D / In2;
        return;
    }
    const double p = 3.0 - h + 3.0 * h * h;
    a = 0.5 * (2.0 / 3.0 - (2.0 / 15.0) * p * h * h) * D;   // 1 - psi = 2/3 - (2/15) p h^2
    c = p / (5.0 * D);
}

// The fifteen per-thread terms of the Eulerian sums at moments (D, I).
__device__ __forceinline__ void eulerian_terms(double D, const double* I, double W3, double W2g, double (&t)[kNsum]) {
    double a, c;
    closure_ac(D, I[0], I[1], I[2], a, c);
    t[0] = W3 * D;
    t[1] = W3 * I[0];
    t[2] = W3 * I[1];
    t[3] = W3 * I[2];
    t[4] = W3 * a;
    const double w = W3 * c;
    t[5] = w * I[0] * I[0];
    t[6] = w * I[1] * I[1];
    t[7] = w * I[2] * I[2];
    t[8] = w * I[0] * I[1];
    t[9] = w * I[0] * I[2];
    t[10] = w * I[1] * I[2];
    t[11] = W2g * D;
    t[12] = W2g * I[0];
    t[13] = W2g * I[1];
    t[14] = W2g * I[2];
}

// B = sum W3 (D delta + K), so that F(v) = sum W3 I + B v.
__device__ __forceinline__ void eulerian_B(const double* S, double (&B)[3][3]) {
    const double d = S[0] + S[4];
    B[0][0] = d + S[5];
    B[1][1] = d + S[6];
    B[2][2] = d + S[7];
    B[0][1] = B[1][0] = S[8];
    B[0][2] = B[2][0] = S[9];
    B[1][2] = B[2][1] = S[10];
}

// (F_nu, E_nu, N_nu) of Eqs. eulerianMomentumLG, eulerianEnergyLG, eulerianNumberLG at velocity v.
__device__ __forceinline__ void eulerian_at(const double* S, const double* v, double* F, double& E, double& N) {
    double B[3][3];
    eulerian_B(S, B);
    for (int j = 0; j < 3; ++j) F[j] = S[1 + j] + B[j][0] * v[0] + B[j][1] * v[1] + B[j][2] * v[2];
    E = S[0] + 2.0 * (v[0] * S[1] + v[1] * S[2] + v[2] * S[3]);
    N = S[11] + v[0] * S[12] + v[1] * S[13] + v[2] * S[14];
}

// Outer Anderson step on kNy-component residuals (as outer_step_warp), depth <= 3, lead warp.
__device__ inline void outer_step_warp5(double (*qh)[kNy], double (*fh)[kNy], const double* qv, const double* y,
                                        const double* ri, int mo, double* yn) {
    constexpr int MM = kMaxOuterMem;
    const int ln = threadIdx.x & 31;
    __syncwarp();
    if (ln == 0) {
        for (int j = 0; j < MM - 1; ++j)
            for (int c = 0; c < kNy; ++c) { qh[j][c] = qh[j + 1][c]; fh[j][c] = fh[j + 1][c]; }
        for (int c = 0; c < kNy; ++c) {
            qh[MM - 1][c] = qv[c];
            fh[MM - 1][c] = (qv[c] - y[c]) * ri[c];
        }
    }
    __syncwarp();
    const int L = MM - 1, g0 = MM - (mo < 2 ? 2 : mo), g1 = g0 + 1;
    const bool isr = ln >= 3;
    const int gi = (ln == 0 || ln == 1 || ln == 3) ? g0 : g1;
    const int gj = ln == 0 ? g0 : g1;
    double e = 0.0;
    for (int c = 0; c < kNy; ++c) {
        const double u = fh[L][c] - fh[gi][c];
        const double w = isr ? fh[L][c] : fh[L][c] - fh[gj][c];
        e += u * w;
    }
    double c0, c1, cL;
    anderson3_warp(e, mo - 1, c0, c1, cL);
    for (int c = 0; c < kNy; ++c) yn[c] = 0.0;
    for (int j = 3 - mo; j < 3; ++j) {
        const double b = anderson3_coef(j, mo - 1, c0, c1, cL);
        for (int c = 0; c < kNy; ++c) yn[c] += b * qh[MM - 3 + j][c];
    }
}

struct VelArgs {
    SolveArgs a;
    const double* v_in;   // [n][3]
    double* v_out;        // [n][3]
    int freeze;
    double v_floor;
    int off_red, off_node;
    int linear;                      // the tables carry linear-order (Phi_1) kernels
    int off_phi1, off_ann1, off_wI;  // their matrices and the W~ I vectors (linear only)
};

template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) velocity_kernel(const VelArgs va) {
    const SolveArgs& a = va.a;
    extern __shared__ __align__(16) unsigned char smb[];
    const DevGrid& g = a.g;
    const int NS = g.ns, NE = g.ne, NEP = g.nep, LD = g.ld;
    const int tid = threadIdx.x;
    const int s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const int sq = s * NEP + q;

    double* phi = reinterpret_cast<double*>(smb + a.off_phi);
    double* ann = reinterpret_cast<double*>(smb + a.off_ann);
    double* vWD = reinterpret_cast<double*>(smb + a.off_vec);
    double* vW1D = vWD + NS * NEP;
    double* vAW1D = vW1D + NS * NEP;
    double* vA = vAW1D + NS * NEP;
    double* vAi = vA + NS * NEP;
    double* vDeq = vAi + NS * NEP;
    double* vDeqc = vDeq + NS * NEP;
    void* red = smb + va.off_red;
    VelNode* nd = reinterpret_cast<VelNode*>(smb + va.off_node);
    const bool lin = va.linear != 0;
    double* phi1 = lin ? reinterpret_cast<double*>(smb + va.off_phi1) : nullptr;   // [NS][NE][LD] K_1,Out
    double* ann1 = lin ? reinterpret_cast<double*>(smb + va.off_ann1) : nullptr;   // [NS/2][NE][LD] K_1,Ann
    double* vWI = lin ? reinterpret_cast<double*>(smb + va.off_wI) : nullptr;      // [3][NS][NEP] W~ I^c
    const OpacBufs<double> ob{phi, ann, vA, vAi, vDeq, vDeqc, phi1, ann1};

    const nmc_params& P = a.p;
    const bool nes_on = (P.proc_mask & NMC_PROC_NES) != 0;
    const bool pair_on = (P.proc_mask & NMC_PROC_PAIR) != 0;
    const double gs = (s == 0) ? 1.0 : (s == 1 ? -1.0 : 0.0);
    const double W2q = act ? g.w2[q] : 0.0;
    const double W3q = act ? g.w3[q] : 0.0;
    const double Wt = act ? g.wt[q] : 0.0;
    double Fh[3][4], Qh[3][4];
    for (int j = 0; j < 3; ++j)
        for (int c = 0; c < 4; ++c) { Fh[j][c] = 0.0; Qh[j][c] = 0.0; }

    for (;;) {
        if (tid == 0) nd->node = atomicAdd(a.queue, 1);
        __syncthreads();
        const long long n = nd->node;
        if (n >= a.n) break;
        const int lead = (int)(n % (long long)(blockDim.x >> 5)) << 5;
        double Ds = 0.0, Is[3] = {0.0, 0.0, 0.0};
        if (act) {
            const long long o = (n * NS + s) * NE + q;
            Ds = a.J[o];
            for (int j = 0; j < 3; ++j) Is[j] = a.H[o * 3 + j];
        }
        const double vs[3] = {va.v_in[n * 3 + 0], va.v_in[n * 3 + 1], va.v_in[n * 3 + 2]};
        if (tid == lead) {
            const double rho = a.rho[n], T = a.T[n], Ye = a.Ye[n], dt = a.dt[n];
            const double v2 = vs[0] * vs[0] + vs[1] * vs[1] + vs[2] * vs[2];
            const bool okin = rho > 0.0 && isfinite(rho) && T > 0.0 && isfinite(T) && Ye > 0.0 && Ye < 1.0 &&
                              dt >= 0.0 && isfinite(dt) && v2 < 1.0;   // v2 < 1 also rejects NaN
            nd->rho = rho;
            nd->T = T;
            nd->dtau = kC * dt;
            for (int k = 0; k < 4; ++k) nd->sc[k] = a.scale ? a.scale[n * 4 + k] : 1.0;
            nd->status = okin ? 0 : NMC_BAD_INPUT;
            double e = 0.0, de = 0.0;
            if (okin) eos_eps(rho, T, Ye, &e, &de);
            const double c2 = kC * kC;
            for (int j = 0; j < 3; ++j) nd->ystar[j] = nd->y[j] = vs[j];
            nd->ystar[3] = nd->y[3] = e + 0.5 * v2 * c2;
            nd->ystar[4] = nd->y[4] = Ye;
            const double vref = fmax(sqrt(v2), va.v_floor);
            nd->ri[0] = nd->ri[1] = nd->ri[2] = 1.0 / vref;
            nd->ri[3] = 1.0 / fabs(nd->ystar[3]);
            nd->ri[4] = 1.0 / fabs(Ye);
            nd->cf = kMeVErg / (rho * c2);
            nd->k_eps = kMeVErg / rho;
            nd->k_ye = kMB / rho;
            nd->lam = 1.0 / (1.0 + sqrt(v2));
            nd->n_inner = 0;
            nd->n_outer = 0;
            nd->bad = 0;
            nd->done = okin ? 0 : 1;
        }
        __syncthreads();
        if (nd->done) {   // invalid input: outputs = inputs
            if (act) {
                const long long o = (n * NS + s) * NE + q;
                a.J_out[o] = Ds;
                for (int j = 0; j < 3; ++j) a.H_out[o * 3 + j] = Is[j];
            }
            if (tid == lead) {
                for (int j = 0; j < 3; ++j) va.v_out[n * 3 + j] = vs[j];
                a.Ye_out[n] = a.Ye[n];
                a.eps_out[n] = nd->ystar[3];
                a.T_out[n] = a.T[n];
                a.n_outer[n] = 0;
                a.n_inner[n] = 0;
                a.status[n] = nd->status;
            }
            __syncthreads();
            continue;
        }
        // conserved moments of the old state (Eq. conservedToPrimitive) and its Eulerian sums
        double Nst = 0.0, Gst[3] = {0.0, 0.0, 0.0};
        {
            double aa, cc;
            closure_ac(Ds, Is[0], Is[1], Is[2], aa, cc);
            const double vI = vs[0] * Is[0] + vs[1] * Is[1] + vs[2] * Is[2];
            Nst = Ds + vI;
            for (int j = 0; j < 3; ++j) Gst[j] = Is[j] + aa * vs[j] + cc * vI * Is[j];
            double t[kNsum];
            eulerian_terms(Ds, Is, W3q, gs * W2q, t);
            block_sum<kNsum, double>(t, red, nd->blk_out);
            if (tid == lead) {
                double F[3], E, N;
                eulerian_at(nd->blk_out, vs, F, E, N);
                for (int j = 0; j < 3; ++j) nd->Fs[j] = F[j];
                nd->Es = E;
                nd->Ns = N;
            }
        }
        double M[4] = {Ds, Is[0], Is[1], Is[2]};
        int outer_exit = 0;
        double chiab = 0, sig = 0, deq = 0, deqc = 0;

        for (int k = 1;; ++k) {
            // semi-implicit (Sec. 3.5): ComputeOpacities only at y^[1] = y*; its shared kernels
            // and this thread's chiab, sig and D^Eq stay in place for the later outer iterations
            if (k == 1 || !P.semi_implicit)
                compute_opacities<double>(g, a.tb, P, nd->rho, nd->T, nd->y[4], nd->dtau, nd->sc, ob, &nd->op,
                                          &nd->status, chiab, sig, deq, deqc, lead);
            const double vk[3] = {nd->y[0], nd->y[1], nd->y[2]};
            const double lam = nd->lam;
            {   // reference norm ||D^[k,1]||_W per species and the Algorithm 2 thresholds
                double v[1] = {Wt * M[0] * M[0]};
                species_sum<1, double>(v, red, nd->sp_out, NEP, NS);
                if (tid == lead) {
                    const double fl = P.norm_floor * sqrt(g.sum_wt);
                    for (int sp = 0; sp < NS; ++sp) {
                        const double dn = fmax(sqrt(nd->sp_out[sp]), fl);
                        nd->thr[0][sp] = P.tol_inner * dn;
                        nd->thr[1][sp] = P.tol_inner * dn;
                    }
                }
            }
            auto publish = [&](const double (&Mv)[4]) {
                if (act) {
                    vWD[sq] = Wt * Mv[0];
                    vW1D[sq] = Wt * (1.0 - Mv[0]);
                    vAW1D[sq] = vA[sq] * Wt * (1.0 - Mv[0]);
                    if (lin)
                        for (int c = 0; c < 3; ++c) vWI[c * NS * NEP + sq] = Wt * Mv[1 + c];
                }
            };
            publish(M);
            __syncthreads();
            bool inner_stop = false;
            for (int ell = 1;; ++ell) {
                double F[4] = {0, 0, 0, 0}, Qv[4] = {0, 0, 0, 0};
                if (act) {
                    double nin = 0, nout = 0, pro = 0, an = 0;
                    if (nes_on) {
                        const double* P0 = phi + s * NE * LD;
                        const double* x = vWD + s * NEP;
                        const double* y = vW1D + s * NEP;
                        for (int j = 0; j < NE; ++j) {
                            nin = fma(P0[j * LD + q], x[j], nin);    // K_In[q][j] = K_Out[j][q]
                            nout = fma(P0[q * LD + j], y[j], nout);
                        }
                    }
                    if (pair_on) {
                        const int pt = s ^ 1;
                        const double* A0 = ann + (s >> 1) * NE * LD;
                        const double* x = vAW1D + pt * NEP;
                        const double* y = vWD + pt * NEP;
                        const int stride_j = (s & 1) == 0 ? 1 : LD;
                        const int base = (s & 1) == 0 ? q * LD : q;
                        for (int j = 0; j < NE; ++j) {
                            const double av = A0[base + j * stride_j];
                            pro = fma(av, x[j], pro);
                            an = fma(av, y[j], an);
                        }
                        pro *= vA[sq];
                    }
                    const double eta = chiab * deq + nin + pro;          // dtau * Eq. emissivityNodal
                    const double chi = chiab + nin + nout + pro + an;    // dtau * Eq. opacityNodal
                    const double kap = chi + sig;                        // dtau * Eq. transportOpacityNodal
                    // Eq. implicitMomentsNodal with lambda = 1 / (1 + |v|)
                    double aa, cc;
                    closure_ac(M[0], M[1], M[2], M[3], aa, cc);
                    const double vI = vk[0] * M[1] + vk[1] * M[2] + vk[2] * M[3];
                    double cD = 0.0, cI[3] = {0.0, 0.0, 0.0};
                    if (lin) {
                        // linear-order NES and pair terms (Eqs. zerothMomentCollisionTerm_NES/Pair,
                        // firstMomentCollisionTerm_NES/Pair), explicit at the current iterate:
                        // A = <Phi_1^{In,Out} I_s>, P = <Phi_1^{Pro,Ann} I_sbar> (Eqs.
                        // linearCorrectionsNES/Pair), K_ij = aa delta_ij + cc I_i I_j
                        double Ai[3] = {0, 0, 0}, Ao[3] = {0, 0, 0}, Pp[3] = {0, 0, 0}, Pa[3] = {0, 0, 0};
                        if (nes_on) {
                            const double* P1 = phi1 + s * NE * LD;
                            for (int j = 0; j < NE; ++j) {
                                const double kin = P1[j * LD + q], kout = P1[q * LD + j];
                                for (int c = 0; c < 3; ++c) {
                                    const double wi = vWI[c * NS * NEP + s * NEP + j];
                                    Ai[c] = fma(kin, wi, Ai[c]);
                                    Ao[c] = fma(kout, wi, Ao[c]);
                                }
                            }
                        }
                        if (pair_on) {
                            const int pt = s ^ 1;
                            const double* A1 = ann1 + (s >> 1) * NE * LD;
                            const int stride_j = (s & 1) == 0 ? 1 : LD;
                            const int base = (s & 1) == 0 ? q * LD : q;
                            for (int j = 0; j < NE; ++j) {
                                const double av = A1[base + j * stride_j];
                                const double ab = vA[pt * NEP + j];
                                for (int c = 0; c < 3; ++c) {
                                    const double wi = vWI[c * NS * NEP + pt * NEP + j];
                                    Pa[c] = fma(av, wi, Pa[c]);
                                    Pp[c] = fma(av, ab * wi, Pp[c]);
                                }
                            }
                            for (int c = 0; c < 3; ++c) Pp[c] *= vA[sq];
                        }
                        auto IdotX = [&](const double* X) { return M[1] * X[0] + M[2] * X[1] + M[3] * X[2]; };
                        cD = -(IdotX(Ai) - IdotX(Ao)) + (IdotX(Pp) - IdotX(Pa));
                        const double iAi = IdotX(Ai), iAo = IdotX(Ao), iPp = IdotX(Pp), iPa = IdotX(Pa);
                        for (int c = 0; c < 3; ++c) {
                            // (K X)_c = aa X_c + cc (I.X) I_c
                            const double KAi = aa * Ai[c] + cc * iAi * M[1 + c];
                            const double KAo = aa * Ao[c] + cc * iAo * M[1 + c];
                            const double KPp = aa * Pp[c] + cc * iPp * M[1 + c];
                            const double KPa = aa * Pa[c] + cc * iPa * M[1 + c];
                            cI[c] = (Ai[c] / 3.0 - KAi) + KAo - (Pp[c] / 3.0 - KPp) - KPa;
                        }
                    }
                    Qv[0] = ((1.0 - lam) * M[0] + lam * (Nst - vI + eta + cD)) / (1.0 + lam * chi);
                    const double rI = 1.0 / (1.0 + lam * kap);
                    for (int j = 0; j < 3; ++j)
                        Qv[1 + j] = ((1.0 - lam) * M[1 + j] + lam * (Gst[j] - (aa * vk[j] + cc * vI * M[1 + j]) + cI[j])) * rI;
                    for (int c = 0; c < 4; ++c) F[c] = Qv[c] - M[c];
                }
                for (int j = 0; j < 2; ++j)
                    for (int c = 0; c < 4; ++c) { Fh[j][c] = Fh[j + 1][c]; Qh[j][c] = Qh[j + 1][c]; }
                for (int c = 0; c < 4; ++c) { Fh[2][c] = F[c]; Qh[2][c] = Qv[c]; }
                const int m = ell < P.m_inner ? ell : P.m_inner;
                {   // new Gram row; least squares by the lead warp
                    double v[3];
                    for (int j = 0; j < 3; ++j)
                        v[j] = F[0] * Fh[j][0] + F[1] * Fh[j][1] + F[2] * Fh[j][2] + F[3] * Fh[j][3];
                    warp_partials<3, double>(v, red);
                    __syncthreads();
                    if ((tid >> 5) == (lead >> 5)) {
                        const int kk = tid & 31;
                        const double* pr = reinterpret_cast<const double*>(red);
                        double sk = 0.0;
                        if (kk < 3)
                            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sk += pr[i * 3 + kk];
                        const double e = gram3_update_warp<3>(nd->G, sk, m);
                        double c0, c1, cL;
                        anderson3_warp(e, m - 1, c0, c1, cL);
                        if (kk < 3) nd->alpha[kk] = anderson3_coef(kk, m - 1, c0, c1, cL);
                    }
                    __syncthreads();
                }
                double Mn[4];
                for (int c = 0; c < 4; ++c) {
                    double acc = 0.0;
                    for (int j = 0; j < 3; ++j)
                        if (j >= 3 - m) acc = fma(nd->alpha[j], Qh[j][c], acc);
                    Mn[c] = act ? acc : 0.0;
                }
                publish(Mn);
                int vote = 1;
                {   // Algorithm 2
                    double v[4];
                    for (int c = 0; c < 4; ++c) { const double d = Mn[c] - M[c]; v[c] = Wt * d * d; }
                    if (act && !(isfinite(Mn[0]) && isfinite(Mn[1]) && isfinite(Mn[2]) && isfinite(Mn[3])))
                        nd->bad = 1;
                    auto species_ok = [&](const double* u, int sp) -> int {
                        double mx = u[1];
                        for (int c = 2; c < 4; ++c) mx = fmax(mx, u[c]);
                        return sqrt(u[0]) <= nd->thr[0][sp] && sqrt(mx) <= nd->thr[1][sp];
                    };
                    if (NEP <= 32) {
                        for (int off = NEP >> 1; off > 0; off >>= 1)
                            for (int c = 0; c < 4; ++c) v[c] += __shfl_xor_sync(kFull, v[c], off);
                        if (s < NS) vote = species_ok(v, s);
                    } else {
                        species_sum<4, double>(v, red, nd->sp_out, NEP, NS);
                        for (int sp = 0; sp < NS; ++sp) vote &= species_ok(nd->sp_out + sp * 4, sp);
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
                for (int c = 0; c < 4; ++c) M[c] = Mn[c];
                if (conv || bad || ell >= P.max_inner) {
                    inner_stop = bad || capped;
                    break;
                }
            }
            if (P.frozen_matter || inner_stop) outer_exit = 1;
            // ================= matter update (Eq. implicitFluidNodal), FP64 =================
            if (!outer_exit) {
                double t[kNsum];
                eulerian_terms(M[0], &M[1], W3q, gs * W2q, t);
                block_sum<kNsum, double>(t, red, nd->blk_out);
                if ((tid >> 5) == (lead >> 5)) {
                    const int ln = tid & 31;
                    const double rho = nd->rho;
                    double F[3], E, N;
                    eulerian_at(nd->blk_out, vk, F, E, N);
                    double qv[kNy], y[kNy], yn[kNy];
                    for (int c = 0; c < kNy; ++c) y[c] = nd->y[c];
                    for (int j = 0; j < 3; ++j) qv[j] = va.freeze ? nd->ystar[j] : nd->ystar[j] - (F[j] - nd->Fs[j]) * nd->cf;
                    qv[3] = nd->ystar[3] - (E - nd->Es) * nd->k_eps;
                    qv[4] = nd->ystar[4] - (N - nd->Ns) * nd->k_ye;
                    const int mo = k < P.m_outer ? k : P.m_outer;
                    outer_step_warp5(nd->qh, nd->fh, qv, y, nd->ri, mo, yn);
                    int conv = 1, fin = 1;
                    for (int c = 0; c < kNy; ++c) {   // Algorithm 3
                        if (!(fabs(yn[c] - y[c]) * nd->ri[c] <= P.tol_outer)) conv = 0;
                        if (!isfinite(yn[c])) fin = 0;
                    }
                    int stop = conv, st = 0;
                    double Tn = nd->T;
                    const double vn2 = yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2];
                    if (!fin || !(vn2 < 1.0)) { st |= NMC_NONFINITE; stop = 1; }
                    if (!stop && k >= P.max_outer) { st |= NMC_NOT_CONVERGED_OUTER; stop = 1; }
                    if (!stop) {   // an iterate outside the EoS domain stops the node
                        bool ok;
                        const double Tk = eos_temperature(rho, yn[3] - 0.5 * vn2 * kC * kC, yn[4], Tn, &ok);
                        if (ok) Tn = Tk;
                        else { st |= NMC_EOS_FAIL; stop = 1; }
                    }
                    if (ln == 0) {
                        for (int c = 0; c < kNy; ++c) nd->y[c] = yn[c];
                        nd->T = Tn;
                        nd->lam = 1.0 / (1.0 + sqrt(vn2));
                        nd->status |= st;
                        nd->conv_out = stop;
                    }
                }
                __syncthreads();
                if (nd->conv_out) outer_exit = 1;
            }
            if (outer_exit) {
                if (tid == lead) nd->n_outer = k;
                break;
            }
        }
        // ================= finalize: the exactly conserving matter state =================
        {
            double t[kNsum];
            eulerian_terms(M[0], &M[1], W3q, gs * W2q, t);
            block_sum<kNsum, double>(t, red, nd->blk_out);
        }
        if (tid == lead) {
            const double rho = nd->rho;
            const double* S = nd->blk_out;
            double v[3] = {nd->ystar[0], nd->ystar[1], nd->ystar[2]};
            double eps_f = nd->ystar[3], Ye = nd->ystar[4], To = a.T[n];
            if (P.frozen_matter) {
                // y = y*
            } else if (nd->status & NMC_NONFINITE) {
                for (int j = 0; j < 3; ++j) v[j] = nd->y[j];
                eps_f = nd->y[3];
                Ye = nd->y[4];
                To = nd->T;
            } else {
                if (P.final_q) {
                    if (!va.freeze) {
                        // (1 + cf B) v = v* - cf (sum W3 I - F*), by Cramer's rule
                        double B[3][3], A[3][3], r[3];
                        eulerian_B(S, B);
                        for (int i = 0; i < 3; ++i) {
                            for (int j = 0; j < 3; ++j) A[i][j] = (i == j ? 1.0 : 0.0) + nd->cf * B[i][j];
                            r[i] = nd->ystar[i] - nd->cf * (S[1 + i] - nd->Fs[i]);
                        }
                        const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
                        const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
                        const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
                        const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
                        const double rd = 1.0 / det;
                        v[0] = (r[0] * c00 + A[0][1] * (r[2] * A[1][2] - r[1] * A[2][2]) +
                                A[0][2] * (r[1] * A[2][1] - r[2] * A[1][1])) * rd;
                        v[1] = (A[0][0] * (r[1] * A[2][2] - r[2] * A[1][2]) + r[0] * c01 +
                                A[0][2] * (r[2] * A[1][0] - r[1] * A[2][0])) * rd;
                        v[2] = (A[0][0] * (r[2] * A[1][1] - r[1] * A[2][1]) +
                                A[0][1] * (r[1] * A[2][0] - r[2] * A[1][0]) + r[0] * c02) * rd;
                    }
                    double F[3], E, N;
                    eulerian_at(S, v, F, E, N);
                    eps_f = nd->ystar[3] - (E - nd->Es) * nd->k_eps;
                    Ye = nd->ystar[4] - (N - nd->Ns) * nd->k_ye;
                } else {
                    for (int j = 0; j < 3; ++j) v[j] = nd->y[j];
                    eps_f = nd->y[3];
                    Ye = nd->y[4];
                }
                bool ok;
                const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                To = eos_temperature(rho, eps_f - 0.5 * v2 * kC * kC, Ye, nd->T, &ok);
                if (!ok) { nd->status |= NMC_EOS_FAIL; To = nd->T; }
            }
            const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            for (int j = 0; j < 3; ++j) va.v_out[n * 3 + j] = v[j];
            a.Ye_out[n] = Ye;
            a.eps_out[n] = eps_f - 0.5 * v2 * kC * kC;
            a.T_out[n] = To;
            a.n_outer[n] = nd->n_outer;
            a.n_inner[n] = nd->n_inner;
            a.status[n] = (uint32_t)nd->status;
        }
        if (act) {
            const long long o = (n * NS + s) * NE + q;
            a.J_out[o] = M[0];
            for (int j = 0; j < 3; ++j) a.H_out[o * 3 + j] = M[1 + j];
        }
        __syncthreads();
    }
}

template <int MAXT, int MINB>
int launch_velocity_impl(nmc_ctx* ctx, VelArgs va, size_t smem, int threads, cudaStream_t stream) {
    auto kern = velocity_kernel<MAXT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess || per_sm < 1)
        return set_error(ctx, NMC_EUNSUPPORTED, "velocity kernel cannot be resident with this shape");
    long long grid = (long long)per_sm * ctx->num_sms;
    if (grid > va.a.n) grid = va.a.n;
    e = cudaMemsetAsync(va.a.queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    kern<<<(unsigned)grid, threads, smem, stream>>>(va);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("velocity kernel launch: ") + cudaGetErrorString(e));
    return NMC_OK;
}

}  // namespace

int launch_velocity(nmc_ctx* ctx, const SolveArgs& a, const double* v_in, double* v_out, int freeze,
                    double v_floor, cudaStream_t stream) {
    if (a.p.m_inner > 3 || a.p.m_outer > 3)
        return set_error(ctx, NMC_EUNSUPPORTED, "the O(v/c) solve supports Anderson memories <= 3");
    if (a.p.precision != NMC_FP64)
        return set_error(ctx, NMC_EUNSUPPORTED, "the O(v/c) solve runs in FP64");
    VelArgs va{};
    va.a = a;
    va.v_in = v_in;
    va.v_out = v_out;
    va.freeze = freeze;
    va.v_floor = v_floor;
    // shared memory: the fused FP64 kernel's matrices and vectors, then the reduction scratch
    // (kNsum doubles per warp) and the node state
    size_t base = fused_smem_bytes(ctx, 3, false, &va.a);
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    const size_t b_red = (((size_t)(threads / 32) * 16 * sizeof(double)) + 15) / 16 * 16;
    const size_t b_node = (sizeof(VelNode) + 15) / 16 * 16;
    va.off_red = va.a.off_red;   // replace the fused kernel's reduction and node carve
    va.off_node = (int)(va.a.off_red + b_red);
    size_t smem = (size_t)va.off_node + b_node;
    va.linear = (ctx->tb.nes1 != nullptr && ctx->tb.pair1 != nullptr) ? 1 : 0;
    if (va.linear) {
        const size_t LDb = (size_t)(ctx->ne + 1);
        const size_t b_phi1 = ((size_t)ctx->ns * ctx->ne * LDb * sizeof(double) + 15) / 16 * 16;
        const size_t b_ann1 = ((size_t)(ctx->ns / 2) * ctx->ne * LDb * sizeof(double) + 15) / 16 * 16;
        const size_t b_wI = ((size_t)3 * ctx->ns * ctx->nep * sizeof(double) + 15) / 16 * 16;
        va.off_phi1 = (int)smem;
        va.off_ann1 = (int)(smem + b_phi1);
        va.off_wI = (int)(smem + b_phi1 + b_ann1);
        smem += b_phi1 + b_ann1 + b_wI;
    }
    (void)base;
    if ((int)smem > ctx->max_smem_optin)
        return set_error(ctx, NMC_EUNSUPPORTED, "shared-memory footprint of the velocity kernel exceeds the per-block limit");
    if (threads <= 128) return launch_velocity_impl<128, 3>(ctx, va, smem, threads, stream);
    if (threads <= 256) return launch_velocity_impl<256, 2>(ctx, va, smem, threads, stream);
    return launch_velocity_impl<512, 1>(ctx, va, smem, threads, stream);
}

}  // namespace nmc
