// Fused, persistent FP64 kernel for the implicit neutrino--matter collision
// solve (Sec. 3.5, Algorithm 1 with Algorithms 2 and 3).
//
// Mapping.  One thread block solves one spatial node at a time; blocks are
// persistent and take node indices from a device work queue (an atomic
// counter), so nodes with many iterations do not hold up others.  Inside a
// block, thread (s, q) owns species s at energy node q: its moments
// (D, I^1, I^2, I^3), old moments, opacities, and its slice of the Anderson
// history (registers).  The node's NES kernels Phi_Out[s] (one ne x ne matrix
// per species) and pair kernels Phi_Ann[p] (one per particle/antiparticle
// pair) live in shared memory, rows padded to ne + 1 so that both row- and
// column-wise reads are free of bank conflicts.
//
// Per outer iteration (ComputeOpacities of Alg. 1): EoS -> chemical
// potentials (thread 0); Fermi--Dirac values at the projection quadrature
// points (all threads), eps^2-weighted projection and bound limiter per
// (species, element) (Eq. fermiDiracProjection); trilinear log-table
// interpolation of chi_EmAb and sigma_Iso with coalesced rows of ne energies;
// bilinear (log10 T, eta) interpolation of the kernel tables into shared
// memory, then the NES up-scattering triangle by detailed balance
// (Eqs. inOutInvarianceNES, detailedBalanceNES).
//
// Per inner iteration: rates as shared-memory mat-vecs (Eqs. nesRatesNodal,
// pairRatesNodal; Phi_In = Phi_Out^T, the antiparticle's Phi_Ann is the
// transpose, Phi_Pro = a_s(q) a_sbar(q') Phi_Ann with a = D/(1-D) by
// Eq. detailedBalancePair), the map Q (Eq. implicitMomentsNodal, v = 0), one
// block reduction for the new row of the Anderson Gram matrix, a tiny FP64
// least-squares solve in thread 0, the mixing update, and a per-species
// reduction for Algorithm 2.
//
// Matter update (Eq. implicitFluidNodal with Eqs. eulerianEnergyLG,
// eulerianNumberLG): one block reduction for E_nu and N_nu, the outer
// Anderson step and Algorithm 3 in thread 0, then T by EoS root finding.
#include <cuda_runtime.h>
#include <math.h>

#include "nmc_internal.h"
#include "nmc_eos.cuh"

namespace nmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int MAXM>
struct NodeShared {
    double rho, dtau, T, eta_e;
    double mu[kMaxSpecies];
    double sc[4];
    double y[2], ystar[2], qv[2];
    double EN_star[2];
    double qh[kMaxOuterMem][2], fh[kMaxOuterMem][2];
    double G[MAXM][MAXM];
    double alpha[MAXM];
    double dnorm[kMaxSpecies];
    double sp_out[kMaxSpecies * 4];
    double blk_out[8];
    // table cells
    double tr, tt, ty, kt, ke;
    int ir, it, iy, ikt, ike;
    long long node;
    int status, n_inner, n_outer, nho;
    int conv_in, conv_out, bad, done;
};

// Sum K values over the whole block; result in out[0..K) for every thread.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red, double* out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(kFull, v[k], off);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[w * K + k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < K) {
        const int nw = blockDim.x >> 5;
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += red[i * K + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Sum K values over each species group (threads s*nep .. s*nep+nep-1);
// result in out[s*K + k].  nep is a power of two <= 32 or a multiple of 32.
template <int K>
__device__ __forceinline__ void species_sum(double (&v)[K], double* red, double* out, int nep, int ns) {
    const int W = nep < 32 ? nep : 32;
    for (int off = W >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(kFull, v[k], off);
    }
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (nep <= 32) {
        if ((lane & (W - 1)) == 0) {
            const int sp = tid / nep;
            if (sp < ns) {
#pragma unroll
                for (int k = 0; k < K; ++k) out[sp * K + k] = v[k];
            }
        }
        __syncthreads();
    } else {
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) red[w * K + k] = v[k];
        }
        __syncthreads();
        const int wps = nep >> 5;
        if (tid < ns * K) {
            const int sp = tid / K, k = tid % K;
            double s = 0.0;
            for (int i = 0; i < wps; ++i) s += red[(sp * wps + i) * K + k];
            out[sp * K + k] = s;
        }
        __syncthreads();
    }
}

// Constrained least squares of Algorithm 1 from the Gram matrix of the
// window [base, L] (L = newest): alpha_L = 1 - sum of the others, normal
// equations of the eliminated problem solved by Gaussian elimination with
// partial pivoting.  Falls back to the newest map value (Picard step) when
// the system is numerically singular.
template <int MAXM>
__device__ void anderson_solve(const double (&G)[MAXM][MAXM], int m, double* alpha) {
    const int L = MAXM - 1, base = MAXM - m;
    for (int j = 0; j < MAXM; ++j) alpha[j] = 0.0;
    alpha[L] = 1.0;
    if (m <= 1) return;
    const int n = m - 1;
    double A[MAXM][MAXM + 1];
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) {
        const int gi = base + i;
        for (int j = 0; j < n; ++j) {
            const int gj = base + j;
            A[i][j] = G[gi][gj] - G[gi][L] - G[gj][L] + G[L][L];
        }
        A[i][n] = G[L][L] - G[gi][L];
        dmax = fmax(dmax, fabs(A[i][i]));
    }
    if (!(dmax > 0.0) || !isfinite(dmax)) return;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (!(fabs(A[piv][c]) > 1e-14 * dmax)) return;   // singular: Picard step
        if (piv != c)
            for (int j = c; j <= n; ++j) { const double t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int j = c; j <= n; ++j) A[r][j] -= f * A[c][j];
        }
    }
    double gam[MAXM];
    double sum = 0.0;
    for (int i = n - 1; i >= 0; --i) {
        double s = A[i][n];
        for (int j = i + 1; j < n; ++j) s -= A[i][j] * gam[j];
        gam[i] = s / A[i][i];
        sum += gam[i];
    }
    if (!isfinite(sum)) return;
    for (int i = 0; i < n; ++i) alpha[base + i] = gam[i];
    alpha[L] = 1.0 - sum;
}

// Outer least squares on the 2-component scaled residuals (thread 0 only).
__device__ void outer_anderson(const double (&fh)[kMaxOuterMem][2], int m, double* beta) {
    constexpr int MM = kMaxOuterMem;
    double G[MM][MM];
    for (int i = 0; i < MM; ++i)
        for (int j = 0; j < MM; ++j) G[i][j] = fh[i][0] * fh[j][0] + fh[i][1] * fh[j][1];
    anderson_solve<MM>(G, m, beta);
}

__device__ __forceinline__ void axis_cell(double v, const Axis& ax, int* i, double* t, int* clamped) {
    double x = (v - ax.lo) * ax.inv_d;
    if (!(x >= 0.0)) { if (!(x == x) || x < 0.0) *clamped = 1; x = 0.0; }
    if (x > ax.n - 1) { x = ax.n - 1; *clamped = 1; }
    int c = (int)floor(x);
    if (c > ax.n - 2) c = ax.n - 2;
    *i = c;
    *t = x - c;
}

}  // namespace

// MAXT: block-size class (threads = ns * nep rounded up to 32 must not exceed
// it); MINB blocks per SM cap registers at 128 per thread in every class.
template <int MAXM, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) fused_fp64_kernel(const SolveArgs a) {
    extern __shared__ __align__(16) double sm[];
    const DevGrid& g = a.g;
    const int NS = g.ns, NE = g.ne, NEP = g.nep, LD = g.ld;
    const int tid = threadIdx.x;
    const int s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const int sq = s * NEP + q;

    double* phi = sm + a.off_phi;        // [NS][NE][LD]   Phi_Out per species
    double* ann = sm + a.off_ann;        // [NS/2][NE][LD] Phi_Ann per pair (particle)
    double* vWD = sm + a.off_vec;        // [NS][NEP]  W2 D
    double* vW1D = vWD + NS * NEP;       //            W2 (1 - D)
    double* vAW1D = vW1D + NS * NEP;     //            a W2 (1 - D)
    double* vA = vAW1D + NS * NEP;       //            a = D^Eq / (1 - D^Eq)
    double* vAi = vA + NS * NEP;         //            1 / a
    double* vDeq = vAi + NS * NEP;       //            D^Eq
    double* red = sm + a.off_red;        // reduction scratch
    NodeShared<MAXM>* nd = reinterpret_cast<NodeShared<MAXM>*>(sm + a.off_node);
    double* fq = sm + a.off_phi;         // FD values at projection points (reuses phi)

    const nmc_params& P = a.p;
    const bool nes_on = (P.proc_mask & NMC_PROC_NES) != 0;
    const bool pair_on = (P.proc_mask & NMC_PROC_PAIR) != 0;
    const double gs = (s == 0) ? 1.0 : (s == 1 ? -1.0 : 0.0);
    const double W2q = act ? g.w2[q] : 0.0;
    const double W3q = act ? g.w3[q] : 0.0;

    double Fh[MAXM][4], Qh[MAXM][4];
#pragma unroll
    for (int j = 0; j < MAXM; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) { Fh[j][c] = 0.0; Qh[j][c] = 0.0; }

    for (;;) {
        if (tid == 0) nd->node = atomicAdd(a.queue, 1);
        __syncthreads();
        const long long n = nd->node;
        if (n >= a.n) break;

        // ---------------- node set-up ----------------
        double Ds = 0.0, Is[3] = {0.0, 0.0, 0.0};
        if (act) {
            const long long o = (n * NS + s) * NE + q;
            Ds = a.J[o];
            Is[0] = a.H[o * 3 + 0];
            Is[1] = a.H[o * 3 + 1];
            Is[2] = a.H[o * 3 + 2];
        }
        if (tid == 0) {
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
            nd->y[0] = e;
            nd->y[1] = Ye;
            nd->n_inner = 0;
            nd->n_outer = 0;
            nd->nho = 0;
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
            if (tid == 0) {
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
        {   // E_nu*, N_nu* (Eqs. eulerianEnergyLG, eulerianNumberLG at v = 0)
            double v[2] = {W3q * Ds, gs * W2q * Ds};
            block_sum<2>(v, red, nd->blk_out);
            if (tid == 0) { nd->EN_star[0] = nd->blk_out[0]; nd->EN_star[1] = nd->blk_out[1]; }
        }
        double M[4] = {Ds, Is[0], Is[1], Is[2]};
        double chiab = 0.0, sig = 0.0, deq = 0.0;
        int outer_exit = 0;

        for (int k = 1;; ++k) {
            // ================= ComputeOpacities(y^[k]) =================
            if (tid == 0) {
                const double T = nd->T, Ye = nd->y[1], rho = nd->rho;
                const double mu_e = eos_mu_e(rho, T, Ye);
                nd->eta_e = mu_e / T;
                const double mnu = mu_e - eos_mu_hat(T, Ye);
                for (int sp = 0; sp < kMaxSpecies; ++sp) nd->mu[sp] = sp == 0 ? mnu : (sp == 1 ? -mnu : 0.0);
                int cl = 0;
                axis_cell(log10(rho), a.tb.rho, &nd->ir, &nd->tr, &cl);
                axis_cell(log10(T), a.tb.t, &nd->it, &nd->tt, &cl);
                axis_cell(Ye, a.tb.ye, &nd->iy, &nd->ty, &cl);
                if (nes_on || pair_on) {
                    axis_cell(log10(T), a.tb.kt, &nd->ikt, &nd->kt, &cl);
                    axis_cell(nd->eta_e, a.tb.eta, &nd->ike, &nd->ke, &cl);
                }
                if (cl) nd->status |= NMC_TABLE_CLAMP;
            }
            __syncthreads();
            // Fermi--Dirac at the projection quadrature points of every element
            {
                const int nqp = g.n_elem * kProjQuad;
                if (s < NS) {
                    const double mu = nd->mu[s], Tinv = 1.0 / nd->T;
                    for (int i = q; i < nqp; i += NEP)
                        fq[s * nqp + i] = 1.0 / (exp((g.proj_e[i] - mu) * Tinv) + 1.0);
                }
                __syncthreads();
                // eps^2-weighted projection and bound-enforcing limiter per (species, element)
                if (s < NS && q < g.n_elem) {
                    const int e = q, nq = g.nq;
                    const double* f = fq + s * nqp + e * kProjQuad;
                    const double* pa = g.proj_a + e * kProjQuad;
                    const double* pc = g.proj_c + e * nq * kProjQuad;
                    double avg = 0.0, coef[kMaxNq] = {0.0, 0.0, 0.0};
                    for (int gq = 0; gq < kProjQuad; ++gq) {
                        const double fv = f[gq];
                        avg += pa[gq] * fv;
                        for (int pp = 0; pp < nq; ++pp) coef[pp] += pc[pp * kProjQuad + gq] * fv;
                    }
                    const double dmin = P.d_min, dmax = P.d_max;
                    if (avg < dmin || avg > dmax) {
                        const double cv = fmin(fmax(avg, dmin), dmax);
                        for (int pp = 0; pp < nq; ++pp) coef[pp] = cv;
                    } else {
                        double vmin = coef[0], vmax = coef[0];
                        for (int pp = 1; pp < nq; ++pp) { vmin = fmin(vmin, coef[pp]); vmax = fmax(vmax, coef[pp]); }
                        for (int side = 0; side < 2; ++side) {
                            double v = 0.0;
                            for (int pp = 0; pp < nq; ++pp) v += coef[pp] * g.ends[side][pp];
                            vmin = fmin(vmin, v);
                            vmax = fmax(vmax, v);
                        }
                        double theta = 1.0;
                        if (vmin < dmin) theta = fmin(theta, (avg - dmin) / (avg - vmin));
                        if (vmax > dmax) theta = fmin(theta, (dmax - avg) / (vmax - avg));
                        for (int pp = 0; pp < nq; ++pp) coef[pp] = avg + theta * (coef[pp] - avg);
                    }
                    for (int pp = 0; pp < nq; ++pp) vDeq[s * NEP + e * nq + pp] = coef[pp];
                }
                __syncthreads();
            }
            // EmAb / Iso: trilinear in (log10 rho, log10 T, Ye) on ln values
            if (act) {
                deq = vDeq[sq];
                vA[sq] = deq / (1.0 - deq);
                vAi[sq] = (1.0 - deq) / deq;
                const int nr = a.tb.rho.n, nt = a.tb.t.n, ny = a.tb.ye.n;
                const long long base = ((((long long)s * ny + nd->iy) * nt + nd->it) * nr + nd->ir) * NE + q;
                const long long dR = NE, dT = (long long)nr * NE, dY = (long long)nt * nr * NE;
                const double tr = nd->tr, tt = nd->tt, ty = nd->ty;
                double le = 0.0, li = 0.0;
#pragma unroll
                for (int c8 = 0; c8 < 8; ++c8) {
                    const int ca = c8 & 1, cb = (c8 >> 1) & 1, cc = c8 >> 2;
                    const double w = (ca ? tr : 1.0 - tr) * (cb ? tt : 1.0 - tt) * (cc ? ty : 1.0 - ty);
                    const long long o = base + ca * dR + cb * dT + cc * dY;
                    le += w * a.tb.emab[o];
                    li += w * a.tb.iso[o];
                }
                chiab = (P.proc_mask & NMC_PROC_EMAB) ? nd->sc[0] * exp(le) : 0.0;
                sig = (P.proc_mask & NMC_PROC_ISO) ? nd->sc[1] * exp(li) : 0.0;
            }
            // NES and pair kernels: bilinear in (log10 T, eta_e)
            if (nes_on || pair_on) {
                const double kt = nd->kt, ke = nd->ke;
                const double w00 = (1.0 - kt) * (1.0 - ke), w10 = kt * (1.0 - ke);
                const double w01 = (1.0 - kt) * ke, w11 = kt * ke;
                const long long mat = (long long)NE * NE;
                const long long sE = mat, sT = (long long)a.tb.eta.n * mat;
                if (nes_on && act) {
                    const double c = nd->sc[2];
                    const double* tb = a.tb.nes + (((long long)s * a.tb.kt.n + nd->ikt) * a.tb.eta.n + nd->ike) * mat;
                    double* P0 = phi + s * NE * LD;
                    for (int r = 0; r < NE; ++r) {   // lower triangle incl. diagonal; row r read coalesced
                        if (q <= r) {
                            const long long o = (long long)r * NE + q;
                            P0[r * LD + q] = c * (w00 * tb[o] + w10 * tb[o + sT] + w01 * tb[o + sE] + w11 * tb[o + sT + sE]);
                        }
                    }
                }
                if (pair_on && s < NS) {
                    const int pr = s >> 1;
                    const double c = nd->sc[3];
                    const double* tb = a.tb.pair + (((long long)pr * a.tb.kt.n + nd->ikt) * a.tb.eta.n + nd->ike) * mat;
                    double* A0 = ann + pr * NE * LD;
                    for (int idx = (s & 1) * NEP + q; idx < NE * NE; idx += 2 * NEP) {
                        const int r = idx / NE, cc = idx - r * NE;
                        const long long o = idx;
                        A0[r * LD + cc] = c * (w00 * tb[o] + w10 * tb[o + sT] + w01 * tb[o + sE] + w11 * tb[o + sT + sE]);
                    }
                }
                __syncthreads();
                if (nes_on && act) {   // up-scattering by detailed balance: Phi[r][q] = a_q / a_r Phi[q][r], r < q
                    double* P0 = phi + s * NE * LD;
                    const double aq = vA[sq];
                    for (int r = 0; r < q; ++r) P0[r * LD + q] = aq * vAi[s * NEP + r] * P0[q * LD + r];
                }
            }
            // reference norm ||D^[k,1]||_W2 per species (Algorithm 2 input)
            {
                double v[1] = {W2q * M[0] * M[0]};
                species_sum<1>(v, red, nd->sp_out, NEP, NS);
                if (tid == 0) {
                    const double fl = P.norm_floor * sqrt(g.sum_w2);
                    for (int sp = 0; sp < NS; ++sp) nd->dnorm[sp] = fmax(sqrt(nd->sp_out[sp]), fl);
                }
            }
            // ================= inner loop =================
            const double dtau = nd->dtau;
            for (int ell = 1;; ++ell) {
                if (act) {
                    vWD[sq] = W2q * M[0];
                    vW1D[sq] = W2q * (1.0 - M[0]);
                    vAW1D[sq] = vA[sq] * W2q * (1.0 - M[0]);
                }
                __syncthreads();
                double F[4] = {0.0, 0.0, 0.0, 0.0}, Qv[4] = {0.0, 0.0, 0.0, 0.0};
                if (act) {
                    double nin = 0.0, nout = 0.0, pro = 0.0, an = 0.0;
                    if (nes_on) {
                        const double* P0 = phi + s * NE * LD;
                        const double* x = vWD + s * NEP;
                        const double* y = vW1D + s * NEP;
                        for (int j = 0; j < NE; ++j) {
                            nin = fma(P0[j * LD + q], x[j], nin);    // Phi_In[q][j] = Phi_Out[j][q]
                            nout = fma(P0[q * LD + j], y[j], nout);
                        }
                    }
                    if (pair_on) {
                        const int pt = s ^ 1;
                        const double* A0 = ann + (s >> 1) * NE * LD;
                        const double* x = vAW1D + pt * NEP;
                        const double* y = vWD + pt * NEP;
                        if ((s & 1) == 0) {
                            for (int j = 0; j < NE; ++j) {
                                const double av = A0[q * LD + j];
                                pro = fma(av, x[j], pro);
                                an = fma(av, y[j], an);
                            }
                        } else {
                            for (int j = 0; j < NE; ++j) {
                                const double av = A0[j * LD + q];
                                pro = fma(av, x[j], pro);
                                an = fma(av, y[j], an);
                            }
                        }
                        pro *= vA[sq];
                    }
                    const double eta = chiab * deq + nin + pro;          // Eq. emissivityNodal
                    const double chi = chiab + nin + nout + pro + an;    // Eq. opacityNodal
                    const double kap = chi + sig;                        // Eq. transportOpacityNodal
                    Qv[0] = (Ds + dtau * eta) / (1.0 + dtau * chi);      // Eq. implicitMomentsNodal, v = 0
                    const double fI = 1.0 / (1.0 + dtau * kap);
                    Qv[1] = Is[0] * fI;
                    Qv[2] = Is[1] * fI;
                    Qv[3] = Is[2] * fI;
#pragma unroll
                    for (int c = 0; c < 4; ++c) F[c] = Qv[c] - M[c];
                }
#pragma unroll
                for (int j = 0; j < MAXM - 1; ++j)
#pragma unroll
                    for (int c = 0; c < 4; ++c) { Fh[j][c] = Fh[j + 1][c]; Qh[j][c] = Qh[j + 1][c]; }
#pragma unroll
                for (int c = 0; c < 4; ++c) { Fh[MAXM - 1][c] = F[c]; Qh[MAXM - 1][c] = Qv[c]; }
                const int m = ell < P.m_inner ? ell : P.m_inner;
                {   // new row of the Gram matrix
                    double v[MAXM];
#pragma unroll
                    for (int j = 0; j < MAXM; ++j)
                        v[j] = F[0] * Fh[j][0] + F[1] * Fh[j][1] + F[2] * Fh[j][2] + F[3] * Fh[j][3];
                    block_sum<MAXM>(v, red, nd->blk_out);
                    if (tid == 0) {
                        for (int i = 0; i < MAXM - 1; ++i)
                            for (int j = 0; j < MAXM - 1; ++j) nd->G[i][j] = nd->G[i + 1][j + 1];
                        for (int j = 0; j < MAXM; ++j) {
                            nd->G[MAXM - 1][j] = nd->blk_out[j];
                            nd->G[j][MAXM - 1] = nd->blk_out[j];
                        }
                        anderson_solve<MAXM>(nd->G, m, nd->alpha);
                    }
                    __syncthreads();
                }
                double Mn[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    double acc = 0.0;
#pragma unroll
                    for (int j = 0; j < MAXM; ++j)
                        if (j >= MAXM - m) acc = fma(nd->alpha[j], Qh[j][c], acc);   // window only
                    Mn[c] = act ? acc : 0.0;
                }
                {   // Algorithm 2: per species, W2-weighted squares of the change per moment
                    double v[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) { const double d = Mn[c] - M[c]; v[c] = W2q * d * d; }
                    if (act && !(isfinite(Mn[0]) && isfinite(Mn[1]) && isfinite(Mn[2]) && isfinite(Mn[3])))
                        nd->bad = 1;
                    species_sum<4>(v, red, nd->sp_out, NEP, NS);
                    if (tid == 0) {
                        int conv = 1;
                        for (int sp = 0; sp < NS; ++sp) {
                            double mx = nd->sp_out[sp * 4];
                            for (int c = 1; c < 4; ++c) mx = fmax(mx, nd->sp_out[sp * 4 + c]);
                            if (!(sqrt(mx) <= P.tol_inner * nd->dnorm[sp])) conv = 0;
                        }
                        nd->n_inner += 1;
                        if (nd->bad) nd->status |= NMC_NONFINITE;
                        if (!conv && !nd->bad && ell >= P.max_inner) nd->status |= NMC_NOT_CONVERGED_INNER;
                        nd->conv_in = conv || nd->bad || ell >= P.max_inner;
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) M[c] = Mn[c];
                if (nd->conv_in) break;
            }
            // an inner loop stopped at its cap (or a non-finite moment) ends the node
            if (P.frozen_matter || nd->bad || (nd->status & NMC_NOT_CONVERGED_INNER)) { outer_exit = 1; }
            // ================= matter update (Eq. implicitFluidNodal) =================
            if (!outer_exit) {
                double v[2] = {W3q * M[0], gs * W2q * M[0]};
                block_sum<2>(v, red, nd->blk_out);
                if (tid == 0) {
                    const double rho = nd->rho;
                    const double qv0 = nd->ystar[0] - (nd->blk_out[0] - nd->EN_star[0]) * kMeVErg / rho;
                    const double qv1 = nd->ystar[1] - kMB * (nd->blk_out[1] - nd->EN_star[1]) / rho;
                    nd->qv[0] = qv0;
                    nd->qv[1] = qv1;
                    // outer Anderson on residuals scaled by |y*|
                    for (int j = 0; j < kMaxOuterMem - 1; ++j) {
                        nd->qh[j][0] = nd->qh[j + 1][0]; nd->qh[j][1] = nd->qh[j + 1][1];
                        nd->fh[j][0] = nd->fh[j + 1][0]; nd->fh[j][1] = nd->fh[j + 1][1];
                    }
                    nd->qh[kMaxOuterMem - 1][0] = qv0;
                    nd->qh[kMaxOuterMem - 1][1] = qv1;
                    nd->fh[kMaxOuterMem - 1][0] = (qv0 - nd->y[0]) / fabs(nd->ystar[0]);
                    nd->fh[kMaxOuterMem - 1][1] = (qv1 - nd->y[1]) / fabs(nd->ystar[1]);
                    const int mo = k < P.m_outer ? k : P.m_outer;
                    double beta[kMaxOuterMem];
                    outer_anderson(nd->fh, mo, beta);
                    double yn0 = 0.0, yn1 = 0.0;
                    for (int j = kMaxOuterMem - mo; j < kMaxOuterMem; ++j) {
                        yn0 += beta[j] * nd->qh[j][0];
                        yn1 += beta[j] * nd->qh[j][1];
                    }
                    const int conv = fabs(yn0 - nd->y[0]) <= P.tol_outer * fabs(nd->ystar[0]) &&
                                     fabs(yn1 - nd->y[1]) <= P.tol_outer * fabs(nd->ystar[1]);   // Algorithm 3
                    nd->y[0] = yn0;
                    nd->y[1] = yn1;
                    int stop = conv;
                    if (!(isfinite(yn0) && isfinite(yn1))) { nd->status |= NMC_NONFINITE; stop = 1; }
                    if (!stop && k >= P.max_outer) { nd->status |= NMC_NOT_CONVERGED_OUTER; stop = 1; }
                    if (!stop) {   // an iterate outside the EoS domain stops the node
                        bool ok;
                        const double Tn = eos_temperature(rho, yn0, yn1, nd->T, &ok);
                        if (ok) nd->T = Tn;
                        else { nd->status |= NMC_EOS_FAIL; stop = 1; }
                    }
                    nd->conv_out = stop;
                }
                __syncthreads();
                if (nd->conv_out) outer_exit = 1;
            }
            if (outer_exit) {
                if (tid == 0) nd->n_outer = k;
                break;
            }
        }
        // ================= finalize =================
        {   // q(M, y) at the final moments (Eq. implicitFluidNodal)
            double v[2] = {W3q * M[0], gs * W2q * M[0]};
            block_sum<2>(v, red, nd->blk_out);
            if (tid == 0) {
                nd->qv[0] = nd->ystar[0] - (nd->blk_out[0] - nd->EN_star[0]) * kMeVErg / nd->rho;
                nd->qv[1] = nd->ystar[1] - kMB * (nd->blk_out[1] - nd->EN_star[1]) / nd->rho;
            }
        }
        if (tid == 0) {
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
                To = eos_temperature(rho, yo0, yo1, nd->T, &ok);
                if (!ok) { nd->status |= NMC_EOS_FAIL; To = nd->T; }   // last T inside the domain
            }
            a.Ye_out[n] = yo1;
            a.eps_out[n] = yo0;
            a.T_out[n] = To;
            a.n_outer[n] = nd->n_outer;
            a.n_inner[n] = nd->n_inner;
            a.status[n] = (uint32_t)nd->status;
        }
        if (act) {
            const long long o = (n * NS + s) * NE + q;
            a.J_out[o] = M[0];
            a.H_out[o * 3 + 0] = M[1];
            a.H_out[o * 3 + 1] = M[2];
            a.H_out[o * 3 + 2] = M[3];
        }
        __syncthreads();
    }
}

size_t fused_smem_bytes(const nmc_ctx* ctx, int maxm, SolveArgs* a) {
    const int NS = ctx->ns, NE = ctx->ne, NEP = ctx->nep, LD = NE + 1;
    const int threads = ((NS * NEP + 31) / 32) * 32;
    size_t mats = (size_t)(NS + NS / 2) * NE * LD;
    const size_t fdq = (size_t)NS * ctx->n_elem * kProjQuad;
    if (fdq > mats) mats = fdq;
    const size_t vec = (size_t)6 * NS * NEP;
    const size_t redn = (size_t)(threads / 32) * 8;
    const size_t node = (maxm <= 3 ? sizeof(NodeShared<3>) : sizeof(NodeShared<5>)) / sizeof(double) + 1;
    if (a) {
        a->off_phi = 0;
        a->off_ann = NS * NE * LD;
        a->off_vec = (int)mats;
        a->off_red = (int)(mats + vec);
        a->off_node = (int)(mats + vec + redn);
    }
    return (mats + vec + redn + node) * sizeof(double);
}

template <int MAXM, int MAXT, int MINB>
static int launch_impl(nmc_ctx* ctx, SolveArgs a, cudaStream_t stream) {
    auto kern = fused_fp64_kernel<MAXM, MAXT, MINB>;
    const size_t smem = fused_smem_bytes(ctx, MAXM, &a);
    if ((int)smem > ctx->max_smem_optin)
        return set_error(ctx, NMC_EUNSUPPORTED, "shared-memory footprint of the fused FP64 kernel exceeds the per-block limit");
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess || per_sm < 1)
        return set_error(ctx, NMC_EUNSUPPORTED, "fused FP64 kernel cannot be resident with this shape");
    long long grid = (long long)per_sm * ctx->num_sms;
    if (grid > a.n) grid = a.n;
    e = cudaMemsetAsync(a.queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    kern<<<(unsigned)grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("fused kernel launch: ") + cudaGetErrorString(e));
    return NMC_OK;
}

template <int MAXM>
static int launch_by_size(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream) {
    const int threads = ((ctx->ns * ctx->nep + 31) / 32) * 32;
    if (threads <= 128) return launch_impl<MAXM, 128, 4>(ctx, a, stream);
    if (threads <= 256) return launch_impl<MAXM, 256, 2>(ctx, a, stream);
    return launch_impl<MAXM, 512, 1>(ctx, a, stream);
}

int launch_fused_fp64(nmc_ctx* ctx, const SolveArgs& a, cudaStream_t stream) {
    if (a.p.m_inner <= 3) return launch_by_size<3>(ctx, a, stream);
    return launch_by_size<5>(ctx, a, stream);
}

}  // namespace nmc
