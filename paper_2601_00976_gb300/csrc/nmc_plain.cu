// Plain per-iteration execution of the collision solve (NMC_MODE_PLAIN, FP64).
//
// The same Algorithm 1 as the fused kernel, organised the way a conventional
// GPU port runs it: every phase is its own launch over the nodes that still
// need it, and all per-node state lives in global memory between launches.
//   setup        y*, E_nu*, N_nu*, M = M*                     (every node)
//   per outer iteration k:
//     opacities  ComputeOpacities(y^[k]) -> K_Out, K_Ann, D^Eq, chi, sigma, a
//     inner step one Anderson-accelerated inner iteration     (repeated)
//     matter     matter update, outer Anderson step, Algorithm 3, EoS
//   finalize     y_out = q(M), T_out, counts, status
// Nodes leave the work lists when they converge: each inner step appends the
// nodes that have not converged to the next list (atomic counter), so a launch
// processes only active nodes; the host reads the list length back after a
// group of inner steps and stops when it is empty.  The batch is processed in
// chunks whose per-node state (kernel matrices, Anderson history) fits a
// bounded scratch allocation.
//
// This mode exists as the baseline of the persistent fused kernel: the two
// give the same results (same algorithm and arithmetic) and differ in how the
// work is scheduled.
#include <cuda_runtime.h>
#include <math.h>

#include <string>

#include "nmc_internal.h"
#include "nmc_eos.cuh"
#include "nmc_device.cuh"

namespace nmc {

namespace {

constexpr int kPlainMaxM = 5;
constexpr int kInnerGroup = 4;   // inner steps launched between two reads of the list length

// Per-node scalar state between launches.
struct PlainNode {
    double rho, dtau, T;
    double sc[4];
    double y[2], ystar[2], EN_star[2];
    double k_eps, k_ye, ri_ys[2];   // matter-update factors and 1 / |y*|, as the fused kernel
    double dnorm[kMaxSpecies];
    double G[kPlainMaxM][kPlainMaxM];
    double qh[kMaxOuterMem][2], fh[kMaxOuterMem][2];
    int status, n_inner, n_outer, ell, k, bad, inner_cap;
};

// Device pointers of one chunk's scratch.
struct PlainState {
    PlainNode* node;     // [C]
    double* kout;        // [C][NS][NE][NE]
    double* kann;        // [C][NS/2][NE][NE]
    double* chiab;       // [C][NS][NE]  dtau s_EmAb chi_EmAb
    double* sig;         // [C][NS][NE]  dtau s_Iso sigma_Iso
    double* deq;         // [C][NS][NE]
    double* va;          // [C][NS][NE]  a = D^Eq / (1 - D^Eq)
    double* fh;          // [C][MAXM][4][NS][NE] Anderson residual history
    double* qh;          // [C][MAXM][4][NS][NE] Anderson map-value history
    int* lists;          // [4][C]: outer A, outer B, inner A, inner B
    int* counts;         // [4]
    long long base;      // first node of the chunk
    int C;
};

struct PlainShared {
    double rho, dtau, T, Ye;
    double sc[4];
    double blk_out[8];
    double sp_out[kMaxSpecies * 4];
    double alpha[kPlainMaxM];
    OpacState op;
    int status, conv, bad, slot;
    int reuse;   // semi-implicit, outer iteration > 1: the node's opacities in global memory stand
};

__device__ __forceinline__ int append(int* list, int* count, int slot) {
    const int i = atomicAdd(count, 1);
    list[i] = slot;
    return i;
}

// ---------------------------------------------------------------- setup
__global__ void __launch_bounds__(512) plain_setup_kernel(const SolveArgs a, PlainState st) {
    __shared__ double red[32 * 8];
    __shared__ double out2[8];
    const DevGrid& g = a.g;
    const int NS = g.ns, NE = g.ne, NEP = g.nep;
    const int tid = threadIdx.x, s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const double gs = (s == 0) ? 1.0 : (s == 1 ? -1.0 : 0.0);
    for (int slot = blockIdx.x; slot < st.C; slot += gridDim.x) {
        const long long n = st.base + slot;
        PlainNode* nd = st.node + slot;
        double Dsd = 0.0;
        if (act) {
            const long long o = (n * NS + s) * NE + q;
            Dsd = a.J[o];
            a.J_out[o] = Dsd;
            for (int c = 0; c < 3; ++c) a.H_out[o * 3 + c] = a.H[o * 3 + c];
        }
        double v[2] = {act ? g.w3[q] * Dsd : 0.0, act ? gs * g.w2[q] * Dsd : 0.0};
        block_sum<2, double>(v, red, out2);
        if (tid == 0) {
            const double rho = a.rho[n], T = a.T[n], Ye = a.Ye[n], dt = a.dt[n];
            const bool okin = rho > 0.0 && isfinite(rho) && T > 0.0 && isfinite(T) && Ye > 0.0 && Ye < 1.0 &&
                              dt >= 0.0 && isfinite(dt);
            nd->rho = rho;
            nd->T = T;
            nd->dtau = kC * dt;
            for (int k = 0; k < 4; ++k) nd->sc[k] = a.scale ? a.scale[n * 4 + k] : 1.0;
            double e = 0.0, de = 0.0;
            if (okin) eos_eps(rho, T, Ye, &e, &de);
            nd->ystar[0] = nd->y[0] = e;
            nd->ystar[1] = nd->y[1] = Ye;
            nd->k_eps = kMeVErg / rho;
            nd->k_ye = kMB / rho;
            nd->ri_ys[0] = 1.0 / fabs(e);
            nd->ri_ys[1] = 1.0 / fabs(Ye);
            nd->EN_star[0] = out2[0];
            nd->EN_star[1] = out2[1];
            nd->status = okin ? 0 : NMC_BAD_INPUT;
            nd->n_inner = 0;
            nd->n_outer = 0;
            nd->k = 0;
            nd->bad = 0;
            nd->inner_cap = 0;
            for (int i = 0; i < kMaxOuterMem; ++i) nd->qh[i][0] = nd->qh[i][1] = nd->fh[i][0] = nd->fh[i][1] = 0.0;
            if (okin) append(st.lists + 0 * st.C, st.counts + 0, slot);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- opacities
template <int MAXM>
__global__ void __launch_bounds__(512) plain_opacity_kernel(const SolveArgs a, PlainState st, int lin, int lout) {
    extern __shared__ __align__(16) unsigned char smb[];
    const DevGrid& g = a.g;
    const nmc_params& P = a.p;
    const int NS = g.ns, NE = g.ne, NEP = g.nep, LD = g.ld;
    const int tid = threadIdx.x, s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const int sq = s * NEP + q;
    double* phi = reinterpret_cast<double*>(smb + a.off_phi);
    double* ann = reinterpret_cast<double*>(smb + a.off_ann);
    double* vec = reinterpret_cast<double*>(smb + a.off_vec);
    double* vA = vec + 3 * NS * NEP;
    double* vAi = vA + NS * NEP;
    double* vDeq = vAi + NS * NEP;
    double* vDeqc = vDeq + NS * NEP;
    void* red = smb + a.off_red;
    PlainShared* sh = reinterpret_cast<PlainShared*>(smb + a.off_node);
    const OpacBufs<double> ob{phi, ann, vA, vAi, vDeq, vDeqc};
    const int count = st.counts[lin];
    const int* list = st.lists + lin * st.C;
    const double Wt = act ? g.wt[q] : 0.0;
    for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
        const int slot = list[idx];
        PlainNode* nd = st.node + slot;
        const long long n = st.base + slot;
        if (tid == 0) {
            sh->rho = nd->rho;
            sh->dtau = nd->dtau;
            sh->T = nd->T;
            sh->Ye = nd->y[1];
            for (int k = 0; k < 4; ++k) sh->sc[k] = nd->sc[k];
            sh->status = nd->status;
            // semi-implicit (Sec. 3.5): ComputeOpacities only at y^[1] = y*; the slot's kernel
            // matrices and per-energy opacities from the first outer iteration are kept
            sh->reuse = P.semi_implicit && nd->k > 0;
        }
        __syncthreads();
        const bool reuse = sh->reuse != 0;
        if (!reuse) {
            double chiab = 0.0, sig = 0.0, deq = 0.0, deqc = 0.0;
            compute_opacities<double>(g, a.tb, P, sh->rho, sh->T, sh->Ye, sh->dtau, sh->sc, ob, &sh->op,
                                      &sh->status, chiab, sig, deq, deqc);
            // kernel matrices and per-energy opacities to global memory
            const long long mat = (long long)NE * NE;
            for (int sp = 0; sp < NS; ++sp) {
                double* dst = st.kout + ((long long)slot * NS + sp) * mat;
                for (int i = tid; i < NE * NE; i += blockDim.x) dst[i] = phi[sp * NE * LD + (i / NE) * LD + i % NE];
            }
            for (int pr = 0; pr < NS / 2; ++pr) {
                double* dst = st.kann + ((long long)slot * (NS / 2) + pr) * mat;
                for (int i = tid; i < NE * NE; i += blockDim.x) dst[i] = ann[pr * NE * LD + (i / NE) * LD + i % NE];
            }
            if (act) {
                const long long o = ((long long)slot * NS + s) * NE + q;
                st.chiab[o] = chiab;
                st.sig[o] = sig;
                st.deq[o] = deq;
                st.va[o] = vA[sq];
            }
        }
        double M0 = 0.0;
        if (act) M0 = a.J_out[(n * NS + s) * NE + q];
        {   // reference norm ||D^[k,1]||_W per species (Algorithm 2 input)
            double v[1] = {Wt * M0 * M0};
            species_sum<1, double>(v, red, sh->sp_out, NEP, NS);
        }
        if (tid == 0) {
            const double fl = P.norm_floor * sqrt(g.sum_wt);
            for (int sp = 0; sp < NS; ++sp) nd->dnorm[sp] = fmax(sqrt(sh->sp_out[sp]), fl);
            for (int i = 0; i < MAXM; ++i)
                for (int j = 0; j < MAXM; ++j) nd->G[i][j] = 0.0;
            nd->status = sh->status;
            nd->ell = 0;
            nd->k += 1;
            append(st.lists + lout * st.C, st.counts + lout, slot);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- inner step
template <int MAXM>
__global__ void __launch_bounds__(512) plain_inner_kernel(const SolveArgs a, PlainState st, int lin, int lout) {
    extern __shared__ __align__(16) unsigned char smb[];
    const DevGrid& g = a.g;
    const nmc_params& P = a.p;
    const int NS = g.ns, NE = g.ne, NEP = g.nep, LD = g.ld;
    const int tid = threadIdx.x, s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const int sq = s * NEP + q;
    double* phi = reinterpret_cast<double*>(smb + a.off_phi);
    double* ann = reinterpret_cast<double*>(smb + a.off_ann);
    double* vWD = reinterpret_cast<double*>(smb + a.off_vec);
    double* vW1D = vWD + NS * NEP;
    double* vAW1D = vW1D + NS * NEP;
    double* vA = vAW1D + NS * NEP;
    void* red = smb + a.off_red;
    PlainShared* sh = reinterpret_cast<PlainShared*>(smb + a.off_node);
    const bool nes_on = (P.proc_mask & NMC_PROC_NES) != 0;
    const bool pair_on = (P.proc_mask & NMC_PROC_PAIR) != 0;
    const double Wt = act ? g.wt[q] : 0.0;
    const int count = st.counts[lin];
    const int* list = st.lists + lin * st.C;
    const long long nsne = (long long)NS * NE;
    for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
        const int slot = list[idx];
        PlainNode* nd = st.node + slot;
        const long long n = st.base + slot;
        // stage this node's kernel matrices (written by the opacity launch)
        const long long mat = (long long)NE * NE;
        if (nes_on)
            for (int sp = 0; sp < NS; ++sp) {
                const double* src = st.kout + ((long long)slot * NS + sp) * mat;
                for (int i = tid; i < NE * NE; i += blockDim.x) phi[sp * NE * LD + (i / NE) * LD + i % NE] = src[i];
            }
        if (pair_on)
            for (int pr = 0; pr < NS / 2; ++pr) {
                const double* src = st.kann + ((long long)slot * (NS / 2) + pr) * mat;
                for (int i = tid; i < NE * NE; i += blockDim.x) ann[pr * NE * LD + (i / NE) * LD + i % NE] = src[i];
            }
        double M[4] = {0, 0, 0, 0}, Ds = 0.0, Is[3] = {0, 0, 0}, chiab = 0.0, sig = 0.0, deq = 0.0;
        const long long so = ((long long)slot * NS + s) * NE + q;
        const long long o = (n * NS + s) * NE + q;
        if (act) {
            M[0] = a.J_out[o];
            for (int c = 0; c < 3; ++c) { M[1 + c] = a.H_out[o * 3 + c]; Is[c] = a.H[o * 3 + c]; }
            Ds = a.J[o];
            chiab = st.chiab[so];
            sig = st.sig[so];
            deq = st.deq[so];
            vA[sq] = st.va[so];
            vWD[sq] = Wt * M[0];
            vW1D[sq] = Wt * (1.0 - M[0]);
            vAW1D[sq] = st.va[so] * Wt * (1.0 - M[0]);
        }
        if (tid == 0) sh->bad = 0;
        __syncthreads();
        double F[4] = {0, 0, 0, 0}, Qv[4] = {0, 0, 0, 0};
        if (act) {
            double nin = 0, nout = 0, pro = 0, an = 0;
            if (nes_on) {
                const double* P0 = phi + s * NE * LD;
                for (int j = 0; j < NE; ++j) {
                    nin = fma(P0[j * LD + q], vWD[s * NEP + j], nin);   // K_In[q][j] = K_Out[j][q]
                    nout = fma(P0[q * LD + j], vW1D[s * NEP + j], nout);
                }
            }
            if (pair_on) {
                const int pt = s ^ 1;
                const double* A0 = ann + (s >> 1) * NE * LD;
                const int stride_j = (s & 1) == 0 ? 1 : LD;
                const int base = (s & 1) == 0 ? q * LD : q;
                for (int j = 0; j < NE; ++j) {
                    const double av = A0[base + j * stride_j];
                    pro = fma(av, vAW1D[pt * NEP + j], pro);
                    an = fma(av, vWD[pt * NEP + j], an);
                }
                pro *= vA[sq];
            }
            const double eta = chiab * deq + nin + pro;
            const double chi = chiab + nin + nout + pro + an;
            const double kap = chi + sig;
            // Eq. implicitMomentsNodal at v = 0, both quotients from one division (as the fused kernel)
            const double d1 = 1.0 + chi, d2 = 1.0 + kap, rr = 1.0 / (d1 * d2);
            Qv[0] = (Ds + eta) * d2 * rr;
            const double fI = d1 * rr;
            for (int c = 0; c < 3; ++c) Qv[1 + c] = Is[c] * fI;
            for (int c = 0; c < 4; ++c) F[c] = Qv[c] - M[c];
        }
        // Anderson history in global memory: [slot][j][c][s][q]
        double Fh[MAXM][4], Qh[MAXM][4];
        const int ell = nd->ell + 1;
        for (int j = 0; j < MAXM - 1; ++j)
            for (int c = 0; c < 4; ++c) {
                const long long h = (((long long)slot * MAXM + j + 1) * 4 + c) * nsne + s * NE + q;
                Fh[j][c] = act && ell > 1 ? st.fh[h] : 0.0;
                Qh[j][c] = act && ell > 1 ? st.qh[h] : 0.0;
            }
        for (int c = 0; c < 4; ++c) { Fh[MAXM - 1][c] = F[c]; Qh[MAXM - 1][c] = Qv[c]; }
        if (act)
            for (int j = 0; j < MAXM; ++j)
                for (int c = 0; c < 4; ++c) {
                    const long long h = (((long long)slot * MAXM + j) * 4 + c) * nsne + s * NE + q;
                    st.fh[h] = Fh[j][c];
                    st.qh[h] = Qh[j][c];
                }
        const int m = ell < P.m_inner ? ell : P.m_inner;
        {   // new row of the Gram matrix; least squares in FP64 (warp 0 at depth 3, as the fused
            // kernel; thread 0 otherwise)
            double v[MAXM];
            for (int j = 0; j < MAXM; ++j)
                v[j] = F[0] * Fh[j][0] + F[1] * Fh[j][1] + F[2] * Fh[j][2] + F[3] * Fh[j][3];
            block_sum<MAXM, double>(v, red, sh->blk_out);
            if (MAXM == 3 && tid < 32) {
                const double nr = tid < 3 ? sh->blk_out[tid] : 0.0;
                const double e = gram3_update_warp<kPlainMaxM>(nd->G, nr, m);
                double c0, c1, cL;
                anderson3_warp(e, m - 1, c0, c1, cL);
                if (tid < 3) sh->alpha[tid] = anderson3_coef(tid, m - 1, c0, c1, cL);
            } else if (MAXM != 3 && tid == 0) {
                double G[MAXM][MAXM];
                for (int i = 0; i < MAXM - 1; ++i)
                    for (int j = 0; j < MAXM - 1; ++j) G[i][j] = nd->G[i + 1][j + 1];
                for (int j = 0; j < MAXM; ++j) G[MAXM - 1][j] = G[j][MAXM - 1] = sh->blk_out[j];
                for (int i = 0; i < MAXM; ++i)
                    for (int j = 0; j < MAXM; ++j) nd->G[i][j] = G[i][j];
                anderson_solve<MAXM>(G, m, sh->alpha);
            }
            __syncthreads();
        }
        double Mn[4];
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int j = MAXM - m; j < MAXM; ++j) acc = fma(sh->alpha[j], Qh[j][c], acc);
            Mn[c] = act ? acc : 0.0;
        }
        {   // Algorithm 2
            double v[4];
            for (int c = 0; c < 4; ++c) { const double d = Mn[c] - M[c]; v[c] = Wt * d * d; }
            if (act && !(isfinite(Mn[0]) && isfinite(Mn[1]) && isfinite(Mn[2]) && isfinite(Mn[3]))) sh->bad = 1;
            species_sum<4, double>(v, red, sh->sp_out, NEP, NS);
            if (tid == 0) {
                int conv = 1;
                for (int sp = 0; sp < NS; ++sp) {
                    double mx = sh->sp_out[sp * 4];
                    for (int c = 1; c < 4; ++c) mx = fmax(mx, sh->sp_out[sp * 4 + c]);
                    if (!(sqrt(mx) <= P.tol_inner * nd->dnorm[sp])) conv = 0;
                }
                nd->ell = ell;
                nd->n_inner += 1;
                if (sh->bad) { nd->status |= NMC_NONFINITE; nd->bad = 1; }
                if (!conv && !sh->bad && ell >= P.max_inner) { nd->status |= NMC_NOT_CONVERGED_INNER; nd->inner_cap = 1; }
                const int done = conv || sh->bad || ell >= P.max_inner;
                if (!done) append(st.lists + lout * st.C, st.counts + lout, slot);
            }
        }
        if (act) {
            a.J_out[o] = Mn[0];
            for (int c = 0; c < 3; ++c) a.H_out[o * 3 + c] = Mn[1 + c];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- matter update
__global__ void __launch_bounds__(512) plain_matter_kernel(const SolveArgs a, PlainState st, int lin, int lout) {
    __shared__ double red[32 * 8];
    __shared__ double out2[8];
    const DevGrid& g = a.g;
    const nmc_params& P = a.p;
    const int NS = g.ns, NE = g.ne, NEP = g.nep;
    const int tid = threadIdx.x, s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const double gs = (s == 0) ? 1.0 : (s == 1 ? -1.0 : 0.0);
    const int count = st.counts[lin];
    const int* list = st.lists + lin * st.C;
    for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
        const int slot = list[idx];
        PlainNode* nd = st.node + slot;
        const long long n = st.base + slot;
        // an inner loop stopped at its cap (or a non-finite moment) ends the node
        const bool stop_now = P.frozen_matter || nd->bad || nd->inner_cap;
        const double D = act ? a.J_out[(n * NS + s) * NE + q] : 0.0;
        double v[2] = {act ? g.w3[q] * D : 0.0, act ? gs * g.w2[q] * D : 0.0};
        block_sum<2, double>(v, red, out2);
        if (tid < 32) {   // warp 0, every lane carrying the node's scalars (as the fused kernel)
            const int k = nd->k;
            if (stop_now) {
                if (tid == 0) nd->n_outer = k;
            } else {
                const double rho = nd->rho;
                const double qv0 = nd->ystar[0] - (out2[0] - nd->EN_star[0]) * nd->k_eps;
                const double qv1 = nd->ystar[1] - (out2[1] - nd->EN_star[1]) * nd->k_ye;
                const double y0 = nd->y[0], y1 = nd->y[1];
                const int mo = k < P.m_outer ? k : P.m_outer;
                double yn0, yn1;
                outer_step_warp(nd->qh, nd->fh, qv0, qv1, y0, y1, nd->ri_ys, mo, yn0, yn1);
                const int conv = fabs(yn0 - y0) <= P.tol_outer * fabs(nd->ystar[0]) &&
                                 fabs(yn1 - y1) <= P.tol_outer * fabs(nd->ystar[1]);   // Algorithm 3
                int stop = conv, stb = 0;
                double Tn = nd->T;
                if (!(isfinite(yn0) && isfinite(yn1))) { stb |= NMC_NONFINITE; stop = 1; }
                if (!stop && k >= P.max_outer) { stb |= NMC_NOT_CONVERGED_OUTER; stop = 1; }
                if (!stop) {
                    bool ok;
                    const double Tk = eos_temperature(rho, yn0, yn1, Tn, &ok);
                    if (ok) Tn = Tk;
                    else { stb |= NMC_EOS_FAIL; stop = 1; }
                }
                if (tid == 0) {
                    nd->y[0] = yn0;
                    nd->y[1] = yn1;
                    nd->T = Tn;
                    nd->status |= stb;
                    if (stop) nd->n_outer = k;
                    else append(st.lists + lout * st.C, st.counts + lout, slot);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- finalize
__global__ void __launch_bounds__(512) plain_finalize_kernel(const SolveArgs a, PlainState st) {
    __shared__ double red[32 * 8];
    __shared__ double out2[8];
    const DevGrid& g = a.g;
    const nmc_params& P = a.p;
    const int NS = g.ns, NE = g.ne, NEP = g.nep;
    const int tid = threadIdx.x, s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const double gs = (s == 0) ? 1.0 : (s == 1 ? -1.0 : 0.0);
    for (int slot = blockIdx.x; slot < st.C; slot += gridDim.x) {
        PlainNode* nd = st.node + slot;
        const long long n = st.base + slot;
        const double D = act ? a.J_out[(n * NS + s) * NE + q] : 0.0;
        double v[2] = {act ? g.w3[q] * D : 0.0, act ? gs * g.w2[q] * D : 0.0};
        block_sum<2, double>(v, red, out2);
        if (tid == 0) {
            const double rho = nd->rho;
            double yo0, yo1, To;
            if (nd->status & NMC_BAD_INPUT) {
                yo0 = nd->ystar[0]; yo1 = a.Ye[n]; To = a.T[n];
            } else if (P.frozen_matter) {
                yo0 = nd->ystar[0]; yo1 = nd->ystar[1]; To = a.T[n];
            } else if (nd->status & NMC_NONFINITE) {
                yo0 = nd->y[0]; yo1 = nd->y[1]; To = nd->T;
            } else {
                if (P.final_q) {   // y = q(M, y) at the converged moments
                    yo0 = nd->ystar[0] - (out2[0] - nd->EN_star[0]) * nd->k_eps;
                    yo1 = nd->ystar[1] - (out2[1] - nd->EN_star[1]) * nd->k_ye;
                } else {
                    yo0 = nd->y[0]; yo1 = nd->y[1];
                }
                bool ok;
                To = eos_temperature(rho, yo0, yo1, nd->T, &ok);
                if (!ok) { nd->status |= NMC_EOS_FAIL; To = nd->T; }
            }
            a.Ye_out[n] = yo1;
            a.eps_out[n] = yo0;
            a.T_out[n] = To;
            a.n_outer[n] = (nd->status & NMC_BAD_INPUT) ? 0 : nd->n_outer;
            a.n_inner[n] = nd->n_inner;
            a.status[n] = (uint32_t)nd->status;
        }
        __syncthreads();
    }
}

static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

size_t plain_smem_bytes(const nmc_ctx* ctx, SolveArgs* a) {
    const int NS = ctx->ns, NE = ctx->ne, NEP = ctx->nep, LD = NE + 1;
    const int threads = ((NS * NEP + 31) / 32) * 32;
    size_t mats = (size_t)(NS + NS / 2) * NE * LD;
    const size_t fdq = (size_t)NS * ctx->n_elem * kProjQuad;
    if (fdq > mats) mats = fdq;
    const size_t b_mats = align16(mats * sizeof(double));
    const size_t b_vec = align16((size_t)7 * NS * NEP * sizeof(double));
    const size_t b_red = align16((size_t)(threads / 32) * 8 * sizeof(double));
    const size_t b_node = align16(sizeof(PlainShared));
    a->off_phi = 0;
    a->off_ann = (int)((size_t)NS * NE * LD * sizeof(double));
    a->off_vec = (int)b_mats;
    a->off_red = (int)(b_mats + b_vec);
    a->off_node = (int)(b_mats + b_vec + b_red);
    return b_mats + b_vec + b_red + b_node;
}

// Per-node scratch bytes of a chunk slot.
size_t plain_slot_bytes(const nmc_ctx* ctx, int maxm) {
    const size_t NS = ctx->ns, NE = ctx->ne;
    return sizeof(PlainNode) + sizeof(double) * ((NS + NS / 2) * NE * NE + 4 * NS * NE + 2 * (size_t)maxm * 4 * NS * NE) +
           4 * sizeof(int);
}

template <typename K>
static int set_smem(nmc_ctx* ctx, K kern, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    return NMC_OK;
}

#define NMC_CU(call)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

template <int MAXM>
static int run_plain(nmc_ctx* ctx, SolveArgs a, cudaStream_t stream) {
    const size_t smem = plain_smem_bytes(ctx, &a);
    if ((int)smem > ctx->max_smem_optin)
        return set_error(ctx, NMC_EUNSUPPORTED, "shared-memory footprint of the plain kernels exceeds the per-block limit");
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    int rc = set_smem(ctx, plain_opacity_kernel<MAXM>, smem);
    if (rc != NMC_OK) return rc;
    rc = set_smem(ctx, plain_inner_kernel<MAXM>, smem);
    if (rc != NMC_OK) return rc;
    int per_sm = 0;
    NMC_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plain_inner_kernel<MAXM>, threads, smem));
    if (per_sm < 1) return set_error(ctx, NMC_EUNSUPPORTED, "plain inner kernel cannot be resident with this shape");
    const int grid = per_sm * ctx->num_sms;

    // chunk of at most plain_chunk nodes, scratch kept in the context
    const long long C = a.n < ctx->plain_chunk ? a.n : ctx->plain_chunk;
    const size_t need = (size_t)C * plain_slot_bytes(ctx, MAXM) + 4 * sizeof(int) + 4096;
    if (ctx->plain_scratch_bytes < need) {
        if (ctx->plain_scratch) cudaFree(ctx->plain_scratch);
        ctx->plain_scratch = nullptr;
        ctx->plain_scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&ctx->plain_scratch, need);
        if (e != cudaSuccess) return set_error(ctx, NMC_ENOMEM, "cannot allocate the plain mode's chunk scratch");
        ctx->plain_scratch_bytes = need;
    }
    if (!ctx->plain_counts_host) {
        cudaError_t e = cudaMallocHost(&ctx->plain_counts_host, 4 * sizeof(int));
        if (e != cudaSuccess) return set_error(ctx, NMC_ENOMEM, "cannot allocate pinned host counters");
    }
    const size_t NS = ctx->ns, NE = ctx->ne;
    char* p = static_cast<char*>(ctx->plain_scratch);
    auto take = [&](size_t bytes) { char* r = p; p += align16(bytes); return static_cast<void*>(r); };
    PlainState st{};
    st.C = (int)C;
    st.node = static_cast<PlainNode*>(take(C * sizeof(PlainNode)));
    st.kout = static_cast<double*>(take(C * NS * NE * NE * sizeof(double)));
    st.kann = static_cast<double*>(take(C * (NS / 2) * NE * NE * sizeof(double)));
    st.chiab = static_cast<double*>(take(C * NS * NE * sizeof(double)));
    st.sig = static_cast<double*>(take(C * NS * NE * sizeof(double)));
    st.deq = static_cast<double*>(take(C * NS * NE * sizeof(double)));
    st.va = static_cast<double*>(take(C * NS * NE * sizeof(double)));
    st.fh = static_cast<double*>(take(C * MAXM * 4 * NS * NE * sizeof(double)));
    st.qh = static_cast<double*>(take(C * MAXM * 4 * NS * NE * sizeof(double)));
    st.lists = static_cast<int*>(take(4 * C * sizeof(int)));
    st.counts = static_cast<int*>(take(4 * sizeof(int)));
    int* hc = ctx->plain_counts_host;

    auto read_count = [&](int which, int* out) -> int {
        NMC_CU(cudaMemcpyAsync(hc, st.counts + which, sizeof(int), cudaMemcpyDeviceToHost, stream));
        NMC_CU(cudaStreamSynchronize(stream));
        *out = hc[0];
        return NMC_OK;
    };

    for (long long base = 0; base < a.n; base += C) {
        st.base = base;
        st.C = (int)((a.n - base) < C ? (a.n - base) : C);
        NMC_CU(cudaMemsetAsync(st.counts, 0, 4 * sizeof(int), stream));
        const int gsetup = st.C < 4 * ctx->num_sms * 8 ? st.C : 4 * ctx->num_sms * 8;
        plain_setup_kernel<<<gsetup, threads, 0, stream>>>(a, st);
        NMC_CU(cudaGetLastError());
        int lo = 0;   // current outer list (0 or 1)
        for (int k = 1; k <= a.p.max_outer; ++k) {
            int nout = 0;
            rc = read_count(lo, &nout);
            if (rc != NMC_OK) return rc;
            if (nout == 0) break;
            NMC_CU(cudaMemsetAsync(st.counts + 2, 0, 2 * sizeof(int), stream));
            plain_opacity_kernel<MAXM><<<grid, threads, smem, stream>>>(a, st, lo, 2);
            NMC_CU(cudaGetLastError());
            int li = 2;
            for (;;) {
                for (int r = 0; r < kInnerGroup; ++r) {
                    const int lnext = li == 2 ? 3 : 2;
                    NMC_CU(cudaMemsetAsync(st.counts + lnext, 0, sizeof(int), stream));
                    plain_inner_kernel<MAXM><<<grid, threads, smem, stream>>>(a, st, li, lnext);
                    NMC_CU(cudaGetLastError());
                    li = lnext;
                }
                int nin = 0;
                rc = read_count(li, &nin);
                if (rc != NMC_OK) return rc;
                if (nin == 0) break;
            }
            const int lnext_o = lo ^ 1;
            NMC_CU(cudaMemsetAsync(st.counts + lnext_o, 0, sizeof(int), stream));
            plain_matter_kernel<<<grid, threads, 0, stream>>>(a, st, lo, lnext_o);
            NMC_CU(cudaGetLastError());
            lo = lnext_o;
        }
        plain_finalize_kernel<<<gsetup, threads, 0, stream>>>(a, st);
        NMC_CU(cudaGetLastError());
    }
    return NMC_OK;
}

}  // namespace

int launch_plain(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream) {
    if (a.p.precision != NMC_FP64)
        return set_error(ctx, NMC_EUNSUPPORTED, "plain mode runs in FP64 only");
    if (a.p.m_inner <= 3) return run_plain<3>(ctx, a, stream);
    return run_plain<5>(ctx, a, stream);
}

}  // namespace nmc
