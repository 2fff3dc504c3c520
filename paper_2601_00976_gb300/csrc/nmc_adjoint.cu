// Adjoint of the converged collision solve (FP64), one thread block per node.
//
// At v = 0 the solve's outputs are fixed by the moment equation of
// Eq. implicitMomentsNodal with the matter state eliminated through
// Eq. implicitFluidNodal (y = q(D), Eqs. eulerianEnergyLG / eulerianNumberLG):
//
//     G(D; p) = D - Q_D(D, q(D; p); p) = 0,   Q_D = (D* + dtau eta) / (1 + dtau chi),
//
// with p = (D*, I*, Ye*, T*, opacity scales); Ye and eps are q(D; p), T the EoS
// temperature of (eps, Ye), and H = I* / (1 + dtau kappa(D, y)) the first-moment
// part of Eq. implicitMomentsNodal at v = 0.  For a loss with cotangents
// (gD, gH, gYe, geps, gT) the implicit-function theorem gives
//
//     (dG/dD)^T lambda = dL_x/dD,       dL/dp = dL_x/dp - lambda . dG/dp,
//
// L_x(D; p) being the loss at given D.  Through H the loss sees kappa with
// cotangent g_kappa = -(gH . I*) / (1 + dtau kappa)^2, so
//     dL_x/dD = gD + (dkappa/dD)^T g_kappa + C^T g_y,
//     g_y = (geps, gYe) + chain rule through T(eps, Ye) + g_kappa . dkappa/dy,
// with C = dq/dD = (-MeV W3 / rho, -m_B g_s W2 / rho).  dkappa/dD is the chi
// part of A below; dkappa/dy comes from the same difference passes as B.
// The Jacobian is
//
//     dG/dD = (I - A) - B C,   A = dQ_D/dD at fixed y,   B = dQ_D/dy at fixed D.
//
// A couples a species only with itself (NES) and its antiparticle (pair), so
// I - A is block diagonal over particle/antiparticle pairs; B C has rank 2.
//  - A is formed analytically from the node's kernel matrices: with
//    inv = 1 / (1 + dtau chi),
//      d(dtau eta_q)/dD_j = s_N K_Out[j][q] W~_j,
//      d(dtau chi_q)/dD_j = s_N (K_Out[j][q] - K_Out[q][j]) W~_j      (same species),
//      d(dtau eta_q)/dDbar_j = -s_P a_q K_Ann[q][j] abar_j W~_j,
//      d(dtau chi_q)/dDbar_j = s_P K_Ann[q][j] W~_j (1 - a_q abar_j)  (partner),
//      A[q][j] = inv_q (d eta - Q_q d chi).
//  - B by central differences of Q_D in eps and Ye (each pass re-runs
//    ComputeOpacities at the perturbed state and the EoS for its T).
//  - Per pair, the transposed block (I - A)^T, augmented with the right-hand
//    sides gD + C^T g_y and the two columns of C^T, is reduced by Gaussian
//    elimination with partial pivoting in shared memory; the rank-2 term is
//    restored by the Sherman--Morrison--Woodbury identity
//      lambda = x + Z (I_2 - B^T Z)^-1 B^T x,  x = P^-1 r, Z = P^-1 C^T.
//  - Gradients:  dL/dD*_j = lambda_j inv_j - (lambda^T B + g_y) . C_j,
//                dL/dYe*  = (lambda^T B + g_y) . (deps*/dYe*, 1),
//                dL/dT*   = (lambda^T B + g_y)_eps deps*/dT*,
//                dL/ds_k  = lambda . dQ_D/ds_k + g_kappa . dkappa/ds_k
//                           (each rate is linear in its scale factor),
//                dL/dI*   = gH / (1 + dtau kappa).
#include <cuda_runtime.h>
#include <math.h>

#include "nmc_internal.h"
#include "nmc_eos.cuh"
#include "nmc_device.cuh"

namespace nmc {

namespace {

struct AdjNode {
    double rho, dtau, T, Tp;
    double Tq[4], yq[4][2];  // the four perturbed matter states of B's differences and their temperatures
    double sc[4];
    double unit[4];
    double ystar[2], y[2], yp[2], h[2];
    double deps_dT_star, deps_dYe_star;
    double g_y[2];           // cotangent of y = (eps, Ye): direct, through T_out and through kappa
    double blk_out[8];
    double dinv[128];        // reciprocals of the eliminated diagonal (2 ne <= 128)
    double cv[2][8];         // per warp: largest |entry| of the next column among its active rows,
    double cip[2][8];        //   its reciprocal,
    int ci[2][8];            //   and its row (double-buffered by column parity)
    int prow[128];           // pivot row of each eliminated column
    OpacState op;

    int status, bad;
};

// Unit-scale NES and pair rates of thread (s, q) at moments D (FP64):
// nin = K_In (W~ D), nout = K_Out (W~ (1 - D)), pro = a_q K_Ann (a W~ (1 - Dbar)),
// an = K_Ann (W~ Dbar), each a dimensionless dtau * rate.
__device__ __forceinline__ void unit_rates(const DevGrid& g, const nmc_params& P, const double* phi,
                                           const double* ann, const double* vWD, const double* vW1D,
                                           const double* vAW1D, const double* vA, int s, int q,
                                           double& nin, double& nout, double& pro, double& an) {
    const int NE = g.ne, NEP = g.nep, LD = g.ld;
    nin = nout = pro = an = 0.0;
    if (P.proc_mask & NMC_PROC_NES) {
        const double* P0 = phi + s * NE * LD;
        const double* x = vWD + s * NEP;
        const double* y = vW1D + s * NEP;
        for (int j = 0; j < NE; ++j) {
            nin = fma(P0[j * LD + q], x[j], nin);    // K_In[q][j] = K_Out[j][q]
            nout = fma(P0[q * LD + j], y[j], nout);
        }
    }
    if (P.proc_mask & NMC_PROC_PAIR) {
        const int pt = s ^ 1;
        const double* A0 = ann + (s >> 1) * NE * LD;
        const double* x = vAW1D + pt * NEP;
        const double* y = vWD + pt * NEP;
        const int stride_j = (s & 1) == 0 ? 1 : LD;   // the antiparticle reads K_Ann transposed
        const int base = (s & 1) == 0 ? q * LD : q;
        for (int j = 0; j < NE; ++j) {
            const double av = A0[base + j * stride_j];
            pro = fma(av, x[j], pro);
            an = fma(av, y[j], an);
        }
        pro *= vA[s * NEP + q];
    }
}

}  // namespace

template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) adjoint_kernel(const AdjointArgs a) {
    extern __shared__ __align__(16) unsigned char smb[];
    const DevGrid& g = a.g;
    const nmc_params& P = a.p;
    const int NS = g.ns, NE = g.ne, NEP = g.nep, LD = g.ld;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const int sq = s * NEP + q;
    const int N2 = 2 * NE, LDM = a.ldm;

    double* phi = reinterpret_cast<double*>(smb + a.off_phi);
    double* ann = reinterpret_cast<double*>(smb + a.off_ann);
    double* Mt = reinterpret_cast<double*>(smb + a.off_mat);   // [2 NE][LDM]: (I - A)^T | r | C^T
    double* vWD = reinterpret_cast<double*>(smb + a.off_vec);
    double* vW1D = vWD + NS * NEP;
    double* vAW1D = vW1D + NS * NEP;
    double* vA = vAW1D + NS * NEP;
    double* vAi = vA + NS * NEP;
    double* vDeq = vAi + NS * NEP;
    double* vDeqc = vDeq + NS * NEP;
    void* red = smb + a.off_red;
    AdjNode* nd = reinterpret_cast<AdjNode*>(smb + a.off_node);
    const OpacBufs<double> ob{phi, ann, vA, vAi, vDeq, vDeqc};

    const double gs = (s == 0) ? 1.0 : (s == 1 ? -1.0 : 0.0);
    const double W2q = act ? g.w2[q] : 0.0;
    const double W3q = act ? g.w3[q] : 0.0;
    const double Wt = act ? g.wt[q] : 0.0;
    const bool frozen = P.frozen_matter != 0;

    for (long long n = blockIdx.x; n < a.n; n += gridDim.x) {
        // ---------------- inputs, y* and the output matter state ----------------
        double Ds = 0.0, D = 0.0, gD = 0.0, gIs = 0.0;   // gIs = gH . I*
        double gH[3] = {0.0, 0.0, 0.0};
        if (act) {
            const long long o = (n * NS + s) * NE + q;
            Ds = a.J[o];
            D = a.J_out[o];
            gD = a.gJ ? a.gJ[o] : 0.0;
            if (a.gH) {
                for (int c = 0; c < 3; ++c) {
                    gH[c] = a.gH[o * 3 + c];
                    gIs += gH[c] * a.H[o * 3 + c];
                }
            }
        }
        if (tid == 0) {
            const double rho = a.rho[n], T = a.T[n], Ye = a.Ye[n], dt = a.dt[n];
            nd->rho = rho;
            nd->dtau = kC * dt;
            for (int k = 0; k < 4; ++k) {
                nd->sc[k] = a.scale ? a.scale[n * 4 + k] : 1.0;
                nd->unit[k] = 1.0;
            }
            const bool okin = rho > 0.0 && isfinite(rho) && T > 0.0 && isfinite(T) && Ye > 0.0 && Ye < 1.0 &&
                              dt >= 0.0 && isfinite(dt);
            nd->status = okin ? 0 : NMC_BAD_INPUT;
            nd->bad = okin ? 0 : 1;
            double e = 0.0, de = 0.0;
            if (okin) eos_eps(rho, T, Ye, &e, &de);
            nd->ystar[0] = e;
            nd->ystar[1] = Ye;
            nd->deps_dT_star = de;
            nd->deps_dYe_star = okin ? eos_deps_dye(rho, T, Ye) : 0.0;
        }
        {   // E_nu, N_nu at D* and D (Eqs. eulerianEnergyLG, eulerianNumberLG at v = 0)
            double v[4] = {W3q * Ds, gs * W2q * Ds, W3q * D, gs * W2q * D};
            block_sum<4, double>(v, red, nd->blk_out);
        }
        if (tid == 0 && !nd->bad && !(isfinite(nd->blk_out[2]) && isfinite(nd->blk_out[3]))) {
            nd->status |= NMC_NONFINITE;   // non-finite converged moments
            nd->bad = 1;
        }
        if (tid < 32 && !nd->bad) {
            // Warp 0: the matter state y = q(D) and the five EoS temperature solves, at y (lane 0) and at
            // the four states of B's central differences (lanes 1..4: eps + h, eps - h, Ye + h, Ye - h),
            // side by side: each solve is a chain of dependent FP64 steps, so five lanes cost one.
            const int ln = tid;
            const double rho = nd->rho;
            double y0, y1;
            if (frozen) { y0 = nd->ystar[0]; y1 = nd->ystar[1]; }
            else {
                y0 = nd->ystar[0] - (nd->blk_out[2] - nd->blk_out[0]) * kMeVErg / rho;
                y1 = nd->ystar[1] - kMB * (nd->blk_out[3] - nd->blk_out[1]) / rho;
            }
            const double h0 = a.fd_rel * fabs(y0), h1 = a.fd_rel * fabs(y1);
            double yy0 = y0, yy1 = y1;
            if (ln >= 1 && ln <= 4) {
                const double d = (ln & 1) ? 1.0 : -1.0;
                if (ln <= 2) yy0 += d * h0; else yy1 += d * h1;
            }
            const double Tg = a.T_out ? a.T_out[n] : a.T[n];
            bool ok = true;
            double Tk = Tg;
            if (ln < 5) Tk = eos_temperature(rho, yy0, yy1, Tg, &ok);
            const bool fail = __ballot_sync(kFull, ln < 5 && !ok) != 0u;
            if (ln >= 1 && ln <= 4) {
                nd->Tq[ln - 1] = Tk;
                nd->yq[ln - 1][0] = yy0;
                nd->yq[ln - 1][1] = yy1;
            }
            if (ln == 0) {
                nd->y[0] = y0;
                nd->y[1] = y1;
                if (fail) { nd->status |= NMC_EOS_FAIL; nd->bad = 1; }
                nd->T = Tk;
                // chain rule through T_out = T(eps, Ye)
                double e, de;
                eos_eps(rho, Tk, y1, &e, &de);
                const double gT = a.gT ? a.gT[n] : 0.0;
                const double ge = a.geps ? a.geps[n] : 0.0, gy = a.gYe ? a.gYe[n] : 0.0;
                nd->g_y[0] = ge + gT / de;
                nd->g_y[1] = gy - gT * eos_deps_dye(rho, Tk, y1) / de;
                nd->h[0] = h0;
                nd->h[1] = h1;
                if (!(isfinite(nd->g_y[0]) && isfinite(nd->g_y[1]))) { nd->status |= NMC_NONFINITE; nd->bad = 1; }
            }
        }
        __syncthreads();
        if (!nd->bad) {
            // W~ D and W~ (1 - D) do not change between passes
            if (act) {
                vWD[sq] = Wt * D;
                vW1D[sq] = Wt * (1.0 - D);
            }
            // ---------------- B = dQ_D/dy by central differences ----------------
            double Qp[4] = {0.0, 0.0, 0.0, 0.0}, Kp[4] = {0.0, 0.0, 0.0, 0.0};
            for (int pass = 0; pass < 5; ++pass) {
                // passes 0..3: (eps + h, eps - h, Ye + h, Ye - h); pass 4: unperturbed
                if (tid == 0) {   // the pass's state, solved above
                    nd->Tp = pass < 4 ? nd->Tq[pass] : nd->T;
                    nd->yp[0] = pass < 4 ? nd->yq[pass][0] : nd->y[0];
                    nd->yp[1] = pass < 4 ? nd->yq[pass][1] : nd->y[1];
                }
                __syncthreads();
                if (nd->bad) break;
                double chiab = 0.0, sig = 0.0, deq = 0.0, deqc = 0.0;
                compute_opacities<double>(g, a.tb, P, nd->rho, nd->Tp, nd->yp[1], nd->dtau, nd->unit, ob, &nd->op,
                                          &nd->status, chiab, sig, deq, deqc);
                if (act) vAW1D[sq] = vA[sq] * Wt * (1.0 - D);
                __syncthreads();
                double nin = 0.0, nout = 0.0, pro = 0.0, an = 0.0;
                if (act) unit_rates(g, P, phi, ann, vWD, vW1D, vAW1D, vA, s, q, nin, nout, pro, an);
                const double s0 = nd->sc[0], s1 = nd->sc[1], s2 = nd->sc[2], s3 = nd->sc[3];
                const double chi = s0 * chiab + s2 * (nin + nout) + s3 * (pro + an);
                const double kap = chi + s1 * sig;   // dtau * Eq. transportOpacityNodal
                const double inv = 1.0 / (1.0 + chi);
                const double Q = (Ds + s0 * chiab * deq + s2 * nin + s3 * pro) * inv;
                if (pass < 4) {
                    Qp[pass] = Q;
                    Kp[pass] = kap;
                    continue;
                }
                // ---------------- unperturbed pass: A, B, scale partials ----------------
                const double Be = (Qp[0] - Qp[1]) / (2.0 * nd->h[0]);
                const double By = (Qp[2] - Qp[3]) / (2.0 * nd->h[1]);
                // dQ_D/ds_k at fixed D and y: (d eta/ds - Q d chi/ds) / (1 + chi); Iso does not enter Q_D
                const double dQs0 = chiab * (deq - Q) * inv;
                const double dQs2 = (nin - Q * (nin + nout)) * inv;
                const double dQs3 = (pro - Q * (pro + an)) * inv;
                const double Ce = frozen ? 0.0 : -kMeVErg * W3q / nd->rho;
                const double Cy = frozen ? 0.0 : -kMB * gs * W2q / nd->rho;
                const double aq = act ? vA[sq] : 0.0;
                // the loss through H = I*/(1 + kappa): cotangent of kappa, and its reach into y
                const double fI = 1.0 / (1.0 + kap);
                const double gk = act ? -gIs * fI * fI : 0.0;
                {
                    double v[2] = {gk * (Kp[0] - Kp[1]) / (2.0 * nd->h[0]), gk * (Kp[2] - Kp[3]) / (2.0 * nd->h[1])};
                    block_sum<2, double>(v, red, nd->blk_out);
                    if (tid == 0) { nd->g_y[0] += nd->blk_out[0]; nd->g_y[1] += nd->blk_out[1]; }
                }
                if (act) vDeq[sq] = gk;   // D^Eq is in registers by now; the slot carries g_kappa
                __syncthreads();
                // (dkappa/dD)^T g_kappa: kappa moves with D only through the NES and pair chi
                double rhs_k = 0.0;
                if (act && a.gH && (P.proc_mask & NMC_PROC_NES)) {
                    const double* K = phi + s * NE * LD;
                    const double* gks = vDeq + s * NEP;
                    double acc = 0.0;
                    for (int i = 0; i < NE; ++i) acc += gks[i] * (K[q * LD + i] - K[i * LD + q]);
                    rhs_k = s2 * acc;
                }
                if (act && a.gH && (P.proc_mask & NMC_PROC_PAIR)) {
                    // partner sbar at energy i: d chi_{sbar,i}/dD_{s,q} = s_P Ann_sbar[i][q] W~_q (1 - a_{sbar,i} a_q)
                    const int pt = s ^ 1;
                    const double* A0 = ann + (s >> 1) * NE * LD;
                    const double* gkp = vDeq + pt * NEP;
                    const double* ap = vA + pt * NEP;
                    const int si = (pt & 1) == 0 ? LD : 1;   // Ann_sbar[i][q]: column q of K_Ann if sbar is the particle
                    const int b0 = (pt & 1) == 0 ? q : q * LD;
                    double acc = 0.0;
                    for (int i = 0; i < NE; ++i) acc += gkp[i] * A0[b0 + i * si] * (1.0 - ap[i] * aq);
                    rhs_k += s3 * acc;
                }
                const double rhs = gD + Wt * rhs_k + nd->g_y[0] * Ce + nd->g_y[1] * Cy;
                double x = 0.0, ze = 0.0, zy = 0.0;
                for (int pr = 0; pr < NS / 2; ++pr) {
                    // column c of P = (I - A)^T, written by thread (s, q) of this pair
                    const bool mine = act && (s >> 1) == pr;
                    if (mine) {
                        const int c = (s & 1) * NE + q, cp = ((s & 1) ^ 1) * NE;
                        const int pt = s ^ 1;
                        const double* K = phi + s * NE * LD;
                        const double* A0 = ann + pr * NE * LD;
                        const int sj = (s & 1) == 0 ? 1 : LD;
                        const int b0 = (s & 1) == 0 ? q * LD : q;
                        const bool nes = (P.proc_mask & NMC_PROC_NES) != 0;
                        const bool pair = (P.proc_mask & NMC_PROC_PAIR) != 0;
                        for (int j = 0; j < NE; ++j) {
                            double aself = 0.0, apart = 0.0;
                            if (nes) {
                                const double kin = K[j * LD + q], kout = K[q * LD + j];
                                aself = inv * s2 * (kin - Q * (kin - kout)) * g.wt[j];
                            }
                            if (pair) {
                                const double ab = aq * vA[pt * NEP + j];
                                apart = -inv * s3 * A0[b0 + j * sj] * g.wt[j] * (ab + Q * (1.0 - ab));
                            }
                            const int rs = (s & 1) * NE + j, rp = cp + j;
                            Mt[rs * LDM + c] = (rs == c ? 1.0 : 0.0) - aself;
                            Mt[rp * LDM + c] = -apart;
                        }
                        Mt[c * LDM + N2 + 0] = rhs;
                        Mt[c * LDM + N2 + 1] = Ce;
                        Mt[c * LDM + N2 + 2] = Cy;
                    }
                    __syncthreads();
                    // Gaussian elimination with partial pivoting on [P | r Ce Cy], rows left in place:
                    // column c's pivot row is recorded (prow[c]) and leaves the active set, and every warp
                    // tracks, among the rows it has just updated, the largest |entry| of the next column
                    // (lane 0 updates that column), so one barrier per column publishes both the updated
                    // rows and the next pivot's candidates.  Every thread then picks the same pivot.
                    unsigned long long done0 = 0ull, done1 = 0ull;   // eliminated pivot rows (2 ne <= 128)
                    auto is_done = [&](int r) {
                        return ((r < 64 ? done0 >> r : done1 >> (r - 64)) & 1ull) != 0ull;
                    };
                    if (lane == 0) {   // column 0's candidates
                        double nb = -1.0, nip = 0.0;
                        int ni = 0;
                        for (int r = warp; r < N2; r += nwarps) {
                            const double v = fabs(Mt[r * LDM]);
                            if (v > nb) { nb = v; ni = r; }
                        }
                        if (nb > 0.0) nip = 1.0 / Mt[ni * LDM];
                        nd->cv[0][warp] = nb;
                        nd->ci[0][warp] = ni;
                        nd->cip[0][warp] = nip;
                    }
                    __syncthreads();
                    for (int c = 0; c < N2; ++c) {
                        const int bsel = c & 1;
                        double best = -1.0, ip = 0.0;
                        int P = 0;
                        for (int w = 0; w < nwarps; ++w) {
                            const double v = nd->cv[bsel][w];
                            const int i = nd->ci[bsel][w];
                            if (v > best || (v == best && i < P)) { best = v; P = i; ip = nd->cip[bsel][w]; }
                        }
                        if (!(best > 1e-300) || !isfinite(best)) {   // singular: same decision in every thread
                            if (tid == 0) { nd->status |= NMC_NONFINITE; nd->bad = 1; }
                            break;
                        }
                        if (!NMC_IN_BOUNDS(g.dbg, P, N2, kDbgHistory)) break;
                        if (P < 64) done0 |= 1ull << P; else done1 |= 1ull << (P - 64);
                        if (tid == 0) nd->prow[c] = P;
                        // The warp's rows r = warp + nwarps i, 32 at a time: lane i forms row i's multiplier
                        // (one FP64 instruction for 32 rows instead of one per row), the rows are updated one
                        // after another with all lanes along j, and then lane i reads row i's new entry of
                        // column c + 1.  The warp's candidate is the largest |entry|, the smallest row among
                        // equals (as a scan in row order would pick): |entry| compared as the integer of its
                        // bits (order-preserving for non-negative doubles; NaN is no candidate), so the
                        // search issues no FP64 compare.
                        const int rows_w = (N2 - warp + nwarps - 1) / nwarps;
                        long long bkey = -1;   // best |entry| bits of this lane's rows (-1: none)
                        int brow = 0;
                        for (int i0 = 0; i0 < rows_w; i0 += 32) {
                            const int rl = warp + nwarps * (i0 + lane);
                            const bool ract = i0 + lane < rows_w && !is_done(rl);
                            const double lmul = ract ? Mt[rl * LDM + c] * ip : 0.0;
                            const int ng = rows_w - i0 < 32 ? rows_w - i0 : 32;
                            for (int k = 0; k < ng; ++k) {
                                const double l = __shfl_sync(kFull, lmul, k);
                                const int r = warp + nwarps * (i0 + k);
                                if (is_done(r)) continue;
                                for (int j = c + 1 + lane; j < N2 + 3; j += 32) Mt[r * LDM + j] -= l * Mt[P * LDM + j];
                            }
                            __syncwarp();
                            if (ract && c + 1 < N2) {
                                const double v = fabs(Mt[rl * LDM + c + 1]);
                                if (v == v) {
                                    const long long key = __double_as_longlong(v);
                                    if (key > bkey) { bkey = key; brow = rl; }
                                }
                            }
                        }
                        long long wkey = bkey;
                        for (int off = 16; off > 0; off >>= 1) {
                            const long long o = __shfl_xor_sync(kFull, wkey, off);
                            wkey = o > wkey ? o : wkey;
                        }
                        const int wrow = (int)__reduce_min_sync(kFull, (unsigned)(bkey == wkey && wkey >= 0 ? brow : 0x7fffffff));
                        if (lane == 0) {
                            const double nb = wkey >= 0 ? __longlong_as_double(wkey) : -1.0;
                            const int ni = wkey >= 0 ? wrow : 0;
                            nd->cv[bsel ^ 1][warp] = nb;
                            nd->ci[bsel ^ 1][warp] = ni;
                            nd->cip[bsel ^ 1][warp] = nb > 0.0 ? 1.0 / Mt[ni * LDM + c + 1] : 0.0;
                        }
                        __syncthreads();
                    }
                    __syncthreads();
                    if (nd->bad) break;
                    // reciprocals of the diagonal of the eliminated (row-permuted) system, then back
                    // substitution in pivot order, one warp per right-hand side
                    for (int i = tid; i < N2; i += blockDim.x)
                        if (NMC_IN_BOUNDS(g.dbg, i, 128, kDbgHistory)) nd->dinv[i] = 1.0 / Mt[nd->prow[i] * LDM + i];
                    __syncthreads();
                    for (int k = warp; k < 3; k += nwarps) {
                        const int col = N2 + k;
                        for (int i = N2 - 1; i >= 0; --i) {
                            const int pi = nd->prow[i];
                            const double xi = Mt[pi * LDM + col] * nd->dinv[i];
                            __syncwarp();
                            for (int r = lane; r < i; r += 32) {
                                const int pr = nd->prow[r];
                                Mt[pr * LDM + col] -= Mt[pr * LDM + i] * xi;
                            }
                            if (lane == 0) Mt[pi * LDM + col] = xi;
                            __syncwarp();
                        }
                    }
                    __syncthreads();
                    if (mine) {   // unknown c sits in its pivot row
                        const int c = (s & 1) * NE + q;
                        const int pc = nd->prow[c];
                        x = Mt[pc * LDM + N2 + 0];
                        ze = Mt[pc * LDM + N2 + 1];
                        zy = Mt[pc * LDM + N2 + 2];
                    }
                    __syncthreads();
                }
                if (nd->bad) break;
                // Woodbury: lambda = x + Z (I_2 - B^T Z)^-1 B^T x
                {
                    double v[6] = {Be * ze, Be * zy, By * ze, By * zy, Be * x, By * x};
                    if (!act) for (int k = 0; k < 6; ++k) v[k] = 0.0;
                    block_sum<6, double>(v, red, nd->blk_out);
                }
                double w0, w1;
                {
                    const double m00 = 1.0 - nd->blk_out[0], m01 = -nd->blk_out[1];
                    const double m10 = -nd->blk_out[2], m11 = 1.0 - nd->blk_out[3];
                    const double det = m00 * m11 - m01 * m10;
                    w0 = (m11 * nd->blk_out[4] - m01 * nd->blk_out[5]) / det;
                    w1 = (m00 * nd->blk_out[5] - m10 * nd->blk_out[4]) / det;
                }
                const double lam = act ? x + ze * w0 + zy * w1 : 0.0;
                // beta = lambda^T B and dL/ds_k = lambda . dQ_D/ds_k + g_kappa . dkappa/ds_k
                {
                    double v[6] = {lam * Be, lam * By, lam * dQs0 + gk * chiab, gk * sig,
                                   lam * dQs2 + gk * (nin + nout), lam * dQs3 + gk * (pro + an)};
                    block_sum<6, double>(v, red, nd->blk_out);
                }
                const double be = nd->blk_out[0] + nd->g_y[0];
                const double by = nd->blk_out[1] + nd->g_y[1];
                if (act) {
                    const long long o = (n * NS + s) * NE + q;
                    a.gJ_in[o] = lam * inv - be * Ce - by * Cy;
                    if (a.gH_in)
                        for (int c = 0; c < 3; ++c) a.gH_in[o * 3 + c] = gH[c] * fI;
                }
                if (tid == 0) {
                    a.gYe_in[n] = be * nd->deps_dYe_star + by;
                    a.gT_in[n] = be * nd->deps_dT_star;
                    if (a.gscale)
                        for (int k = 0; k < 4; ++k) a.gscale[n * 4 + k] = nd->blk_out[2 + k];
                    if (!(isfinite(a.gYe_in[n]) && isfinite(a.gT_in[n]))) nd->status |= NMC_NONFINITE;
                }
            }
        }
        __syncthreads();
        if (nd->bad) {   // no gradient at this node: zeros, reason in status
            if (act) {
                const long long o = (n * NS + s) * NE + q;
                a.gJ_in[o] = 0.0;
                if (a.gH_in)
                    for (int c = 0; c < 3; ++c) a.gH_in[o * 3 + c] = 0.0;
            }
            if (tid == 0) {
                a.gYe_in[n] = 0.0;
                a.gT_in[n] = 0.0;
                if (a.gscale)
                    for (int k = 0; k < 4; ++k) a.gscale[n * 4 + k] = 0.0;
            }
        }
        if (tid == 0 && a.status) a.status[n] = (uint32_t)nd->status;
        __syncthreads();
    }
}

static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

size_t adjoint_smem_bytes(const nmc_ctx* ctx, AdjointArgs* a) {
    const int NS = ctx->ns, NE = ctx->ne, NEP = ctx->nep, LD = NE + 1;
    const int threads = ((NS * NEP + 31) / 32) * 32;
    size_t mats = (size_t)(NS + NS / 2) * NE * LD;
    const size_t fdq = (size_t)NS * ctx->n_elem * kProjQuad;
    if (fdq > mats) mats = fdq;
    const int N2 = 2 * NE;
    const int ldm = (N2 + 3) | 1;   // odd row stride: column walks hit distinct banks
    const size_t b_mats = align16(mats * sizeof(double));
    const size_t b_mat = align16((size_t)N2 * ldm * sizeof(double));
    const size_t b_vec = align16((size_t)7 * NS * NEP * sizeof(double));
    const size_t b_red = align16((size_t)(threads / 32) * 8 * sizeof(double));
    const size_t b_node = align16(sizeof(AdjNode));
    if (a) {
        a->ldm = ldm;
        a->off_phi = 0;
        a->off_ann = (int)((size_t)NS * NE * LD * sizeof(double));
        a->off_mat = (int)b_mats;
        a->off_vec = (int)(b_mats + b_mat);
        a->off_red = (int)(b_mats + b_mat + b_vec);
        a->off_node = (int)(b_mats + b_mat + b_vec + b_red);
    }
    return b_mats + b_mat + b_vec + b_red + b_node;
}

template <int MAXT, int MINB>
static int launch_adj_impl(nmc_ctx* ctx, AdjointArgs& a, cudaStream_t stream) {
    auto kern = adjoint_kernel<MAXT, MINB>;
    if (2 * ctx->ne > 128)   // the reciprocal diagonal of a pair system holds 2 ne <= 128 entries
        return set_error(ctx, NMC_EUNSUPPORTED, "collision_adjoint supports at most 64 energies");
    const size_t smem = adjoint_smem_bytes(ctx, &a);
    if ((int)smem > ctx->max_smem_optin)
        return set_error(ctx, NMC_EUNSUPPORTED, "shared-memory footprint of the adjoint kernel exceeds the per-block limit");
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess || per_sm < 1)
        return set_error(ctx, NMC_EUNSUPPORTED, "adjoint kernel cannot be resident with this shape");
    long long grid = (long long)per_sm * ctx->num_sms;
    if (grid > a.n) grid = a.n;
    kern<<<(unsigned)grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("adjoint kernel launch: ") + cudaGetErrorString(e));
    return NMC_OK;
}

int launch_adjoint(nmc_ctx* ctx, AdjointArgs& a, cudaStream_t stream) {
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    if (threads <= 128) return launch_adj_impl<128, 4>(ctx, a, stream);
    if (threads <= 256) return launch_adj_impl<256, 2>(ctx, a, stream);
    return launch_adj_impl<512, 1>(ctx, a, stream);
}

}  // namespace nmc
