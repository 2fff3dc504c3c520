// Device building blocks shared by the solve and adjoint kernels: block and
// per-species reductions, table-axis lookup, and ComputeOpacities of
// Algorithm 1 (EoS chemical potentials, the projected and limited D^Eq of
// Eq. fermiDiracProjection, EmAb/Iso interpolation, and the NES and pair kernel
// matrices in shared memory).
//
// Thread mapping used throughout: thread (s, q) = s * nep + q owns species s
// at energy node q; nep is ne padded to a power of two <= 32 or a multiple of
// 32, so a species group never straddles a warp unevenly.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "nmc_internal.h"
#include "nmc_eos.cuh"

namespace nmc {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double r_exp(double x) { return exp(x); }
__device__ __forceinline__ float r_exp(float x) { return expf(x); }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double r_log10(double x) { return log10(x); }
__device__ __forceinline__ float r_log10(float x) { return log10f(x); }

// Sum K values over the whole block; result in out[0..K).
template <int K, typename T>
__device__ __forceinline__ void block_sum(T (&v)[K], void* scratch, T* out) {
    T* red = static_cast<T*>(scratch);
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
        T s = 0;
        for (int i = 0; i < nw; ++i) s += red[i * K + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Sum K values over each species group (threads s*nep .. s*nep+nep-1);
// result in out[s*K + k].  nep is a power of two <= 32 or a multiple of 32.
template <int K, typename T>
__device__ __forceinline__ void species_sum(T (&v)[K], void* scratch, T* out, int nep, int ns) {
    T* red = static_cast<T*>(scratch);
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
            T s = 0;
            for (int i = 0; i < wps; ++i) s += red[(sp * wps + i) * K + k];
            out[sp * K + k] = s;
        }
        __syncthreads();
    }
}

// Cell index and fractional offset of v on a uniform axis, clamped to the
// table; *clamped is set when v lies outside it.
template <typename R>
__device__ __forceinline__ void axis_cell(R v, const Axis& ax, int* i, double* t, int* clamped) {
    R x = (v - (R)ax.lo) * (R)ax.inv_d;
    if (!(x >= (R)0)) { *clamped = 1; x = 0; }
    if (x > (R)(ax.n - 1)) { x = (R)(ax.n - 1); *clamped = 1; }
    int c = (int)floor((double)x);
    if (c > ax.n - 2) c = ax.n - 2;
    *i = c;
    *t = (double)(x - (R)c);
}

// Constrained least squares of Algorithm 1 from the Gram matrix of the
// window [base, L] (L = newest): alpha_L = 1 - sum of the others, normal
// equations of the eliminated problem solved by Gaussian elimination with
// partial pivoting.  Falls back to the newest map value (Picard step) when
// the system is numerically singular.
template <int MAXM>
__device__ inline void anderson_solve(const double (&G)[MAXM][MAXM], int m, double* alpha) {
    const int L = MAXM - 1, base = MAXM - m;
    for (int j = 0; j < MAXM; ++j) alpha[j] = 0.0;
    alpha[L] = 1.0;
    if (m <= 1) return;
    const int n = m - 1;
    if (n <= 2) {
        // the same eliminated normal equations and pivot tests in registers (depth <= 3)
        const int g0 = base, g1 = base + 1;
        const double a00 = G[g0][g0] - 2.0 * G[g0][L] + G[L][L], r0 = G[L][L] - G[g0][L];
        if (n == 1) {
            if (!(fabs(a00) > 1e-14 * fabs(a00)) || !isfinite(a00)) return;
            const double gam = r0 / a00;
            if (!isfinite(gam)) return;
            alpha[g0] = gam;
            alpha[L] = 1.0 - gam;
            return;
        }
        const double a01 = G[g0][g1] - G[g0][L] - G[g1][L] + G[L][L];
        const double a11 = G[g1][g1] - 2.0 * G[g1][L] + G[L][L], r1 = G[L][L] - G[g1][L];
        const double dmax = fmax(fabs(a00), fabs(a11));
        if (!(dmax > 0.0) || !isfinite(dmax)) return;
        // Column 0 with partial pivoting (the system is symmetric: a10 = a01); the pivot tests of
        // the elimination, |p0| and |s11| = |det / p0| against 1e-14 dmax, need no division, and
        // Cramer's rule then needs one: a single-lane FP64 division is a long chain of FP64-pipe
        // instructions on the solve's critical path.
        double p0 = a00, p1 = a01, pr = r0, q0 = a01, q1 = a11, qr = r1;
        if (fabs(a01) > fabs(a00)) { p0 = a01; p1 = a11; pr = r1; q0 = a00; q1 = a01; qr = r0; }
        if (!(fabs(p0) > 1e-14 * dmax)) return;
        const double det = p0 * q1 - q0 * p1;
        if (!(fabs(det) > 1e-14 * dmax * fabs(p0))) return;
        const double rdet = 1.0 / det;
        const double gam1 = (p0 * qr - q0 * pr) * rdet;
        const double gam0 = (pr * q1 - p1 * qr) * rdet;
        const double sum = gam0 + gam1;
        if (!isfinite(sum)) return;
        alpha[g0] = gam0;
        alpha[g1] = gam1;
        alpha[L] = 1.0 - sum;
        return;
    }
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
__device__ inline void outer_anderson(const double (&fh)[kMaxOuterMem][2], int m, double* beta) {
    constexpr int MM = kMaxOuterMem;
    double G[MM][MM];
    for (int i = 0; i < MM; ++i)
        for (int j = 0; j < MM; ++j) G[i][j] = fh[i][0] * fh[j][0] + fh[i][1] * fh[j][1];
    anderson_solve<MM>(G, m, beta);
}


// Node-wide results of the scalar part of ComputeOpacities (shared memory,
// written by thread 0).
struct OpacState {
    double eta_e;              // mu_e / T
    double mu[kMaxSpecies];    // neutrino chemical potentials per species
    double tr, tt, ty, kt, ke; // fractional offsets in the table cells
    int ir, it, iy, ikt, ike;  // table cells
};

// Shared-memory operands ComputeOpacities fills.
template <typename R>
struct OpacBufs {
    R* phi;    // [NS][NE][LD] K_Out = dtau (4 pi/(hc)^3) s_NES Phi_Out per species;
               // also holds the FD values at the projection points while D^Eq is formed
    R* ann;    // [NS/2][NE][LD] K_Ann = dtau (4 pi/(hc)^3) s_Pair Phi_Ann per pair (particle)
    R* vA;     // [NS][NEP] a = D^Eq / (1 - D^Eq)
    R* vAi;    //           1 / a
    R* vDeq;   //           D^Eq
    R* vDeqc;  //           1 - D^Eq (mixed precision; FP64 forms it from D^Eq)
};

// ComputeOpacities of Algorithm 1 at the matter state (rho, T, Ye), called by
// every thread of the block with the same arguments (sc points to the node's
// four scale factors EmAb, Iso, NES, Pair).
//  - Chemical potentials from the EoS (thread 0; FP32 in mixed precision).
//  - Fermi--Dirac values at the projection quadrature points, the
//    eps^2-weighted L2 projection and the bound-enforcing limiter per
//    (species, element) (Eq. fermiDiracProjection).
//  - chi_EmAb and sigma_Iso by trilinear interpolation of the ln tables in
//    (log10 rho, log10 T, Ye), each times dtau and its scale: returned in the
//    calling thread's chiab and sig with its D^Eq (deq) and 1 - D^Eq (deqc).
//  - The NES kernel K_Out (bilinear in (log10 T, eta_e)) tabulated for
//    q >= q' and completed by detailed balance, K_Out[q'][q] = a_q / a_q'
//    K_Out[q][q'] for q' < q (Eqs. inOutInvarianceNES, detailedBalanceNES),
//    and the pair kernel K_Ann of each particle/antiparticle pair.
// Thread `lead` does the scalar part and ORs NMC_TABLE_CLAMP into *status when a
// lookup leaves a table.
// Ends with the block synchronised.
template <typename R>
__device__ void compute_opacities(const DevGrid& g, const DevTables& tb, const nmc_params& P, double rho,
                                  double T, double Ye, double dtau, const double* sc, const OpacBufs<R>& b,
                                  OpacState* os, int* status, R& chiab, R& sig, R& deq, R& deqc, int lead = 0) {
    constexpr bool kMixed = sizeof(R) == 4;
    const int NS = g.ns, NE = g.ne, NEP = g.nep, LD = g.ld;
    const int tid = threadIdx.x;
    const int s = tid / NEP, q = tid - s * NEP;
    const bool act = (s < NS) && (q < NE);
    const int sq = s * NEP + q;
    const bool nes_on = (P.proc_mask & NMC_PROC_NES) != 0;
    const bool pair_on = (P.proc_mask & NMC_PROC_PAIR) != 0;
    R* fq = b.phi;

    if (tid == lead) {
        double mu_e, mnu;
        if (kMixed) {
            // FP32 root of the electron cubic, then one FP64 Newton step on it (the error
            // squares): mu_e, and with it D^Eq, must move smoothly with (T, Ye), or the outer
            // iteration's map is noisy at the 1e-7 level and stalls above tol_outer
            const EosScaleF es = eos_scale(rho, Ye);
            const double m0 = eos_mu_e_f(es.ne, (float)T);
            const double pi2T2 = kPi * kPi * T * T;
            const double ned = Ye * rho / kMB * (kHbarC * kHbarC * kHbarC);   // FP64 target
            const double cub = m0 * (m0 * m0 + pi2T2) - 3.0 * kPi * kPi * ned;
            mu_e = m0 - cub / (3.0 * m0 * m0 + pi2T2);
            mnu = mu_e - eos_mu_hat(T, Ye);
        } else {
            mu_e = eos_mu_e(rho, T, Ye);
            mnu = mu_e - eos_mu_hat(T, Ye);
        }
        os->eta_e = mu_e / T;
        for (int sp = 0; sp < kMaxSpecies; ++sp) os->mu[sp] = sp == 0 ? mnu : (sp == 1 ? -mnu : 0.0);
        int cl = 0;   // table cells in FP64 in both precisions (one thread, a few operations)
        axis_cell<double>(log10(rho), tb.rho, &os->ir, &os->tr, &cl);
        axis_cell<double>(log10(T), tb.t, &os->it, &os->tt, &cl);
        axis_cell<double>(Ye, tb.ye, &os->iy, &os->ty, &cl);
        if (nes_on || pair_on) {
            axis_cell<double>(log10(T), tb.kt, &os->ikt, &os->kt, &cl);
            axis_cell<double>(os->eta_e, tb.eta, &os->ike, &os->ke, &cl);
        }
        if (cl) *status |= NMC_TABLE_CLAMP;
    }
    __syncthreads();
    // Fermi--Dirac at the projection quadrature points of every element
    {
        const int nqp = g.n_elem * kProjQuad;
        if (s < NS) {
            const R mu = (R)os->mu[s], Tinv = (R)(1.0 / T);
            const double mud = os->mu[s], Tinvd = 1.0 / T;
            for (int i = q; i < nqp; i += NEP) {
                if (kMixed) {
                    // f and 1 - f from one exp, each without cancellation.  x = (E - mu)/T reaches
                    // ~100 in the tail, where rounding x to FP32 would move exp(-|x|) by ~1e-5 in
                    // steps; x is formed in FP64 and split, e^-|x| = expf(-|x_hi|) (1 - |x|_lo)
                    const double xd = (g.proj_e[i] - mud) * Tinvd;
                    const double ax = fabs(xd);
                    const float xh = (float)ax;
                    const float xl = (float)(ax - (double)xh);
                    const R t = r_exp(-xh) * (1.0f - xl);
                    const R inv = (R)1 / ((R)1 + t);
                    fq[s * nqp + i] = xd > 0 ? t * inv : inv;
                    fq[(NS + s) * nqp + i] = xd > 0 ? inv : t * inv;
                } else {
                    fq[s * nqp + i] = (R)1 / (r_exp(((R)g.proj_e[i] - mu) * Tinv) + (R)1);
                }
            }
        }
        __syncthreads();
        // eps^2-weighted projection and bound-enforcing limiter per (species, element)
        if (s < NS && q < g.n_elem) {
            const int e = q, nq = g.nq;
            const R* f = fq + s * nqp + e * kProjQuad;
            const R* fc = fq + (NS + s) * nqp + e * kProjQuad;
            R avg = 0, avgc = 0, coef[kMaxNq] = {0, 0, 0}, coefc[kMaxNq] = {0, 0, 0};
            for (int gq = 0; gq < kProjQuad; ++gq) {
                const R pa = kMixed ? (R)g.proj_a_f[e * kProjQuad + gq] : (R)g.proj_a[e * kProjQuad + gq];
                const R fv = f[gq];
                avg += pa * fv;
                R fcv = 0;
                if (kMixed) { fcv = fc[gq]; avgc += pa * fcv; }
                for (int pp = 0; pp < nq; ++pp) {
                    const int o = (e * nq + pp) * kProjQuad + gq;
                    const R pc = kMixed ? (R)g.proj_c_f[o] : (R)g.proj_c[o];
                    coef[pp] += pc * fv;
                    if (kMixed) coefc[pp] += pc * fcv;
                }
            }
            const R dmin = (R)P.d_min, dmax = (R)P.d_max;
            if (avg < dmin || avg > dmax) {
                const bool lo = avg < dmin;
                const R cv = lo ? dmin : dmax;
                const R cvc = lo ? (R)(1.0 - P.d_min) : (R)(1.0 - P.d_max);
                for (int pp = 0; pp < nq; ++pp) { coef[pp] = cv; coefc[pp] = cvc; }
            } else {
                R vmin = coef[0], vmax = coef[0];
                for (int pp = 1; pp < nq; ++pp) { vmin = fmin(vmin, coef[pp]); vmax = fmax(vmax, coef[pp]); }
                for (int side = 0; side < 2; ++side) {
                    R v = 0;
                    for (int pp = 0; pp < nq; ++pp) v += coef[pp] * (R)g.ends[side][pp];
                    vmin = fmin(vmin, v);
                    vmax = fmax(vmax, v);
                }
                R theta = 1;
                if (vmin < dmin) theta = fmin(theta, (avg - dmin) / (avg - vmin));
                if (vmax > dmax) theta = fmin(theta, (dmax - avg) / (vmax - avg));
                for (int pp = 0; pp < nq; ++pp) {
                    coef[pp] = avg + theta * (coef[pp] - avg);
                    coefc[pp] = avgc + theta * (coefc[pp] - avgc);
                }
            }
            for (int pp = 0; pp < nq; ++pp) {
                b.vDeq[s * NEP + e * nq + pp] = coef[pp];
                b.vDeqc[s * NEP + e * nq + pp] = coefc[pp];
            }
        }
        __syncthreads();
    }
    // EmAb / Iso: trilinear in (log10 rho, log10 T, Ye) on ln values, times dtau
    if (act) {
        deq = b.vDeq[sq];
        const R dc = kMixed ? b.vDeqc[sq] : (R)1 - deq;
        deqc = dc;
        b.vA[sq] = deq / dc;
        b.vAi[sq] = dc / deq;
        const int nr = tb.rho.n, nt = tb.t.n, ny = tb.ye.n;
        const long long base = ((((long long)s * ny + os->iy) * nt + os->it) * nr + os->ir) * NE + q;
        const long long dR = NE, dT = (long long)nr * NE, dY = (long long)nt * nr * NE;
        const R tr = (R)os->tr, tt = (R)os->tt, ty = (R)os->ty;
        // ln chi as the first corner plus weighted differences: the corners are ~ -20, so an
        // FP32 sum of the corner values themselves would round ln chi by ~2e-6 in steps
        const R le0 = kMixed ? (R)tb.emab_f[base] : (R)tb.emab[base];
        const R li0 = kMixed ? (R)tb.iso_f[base] : (R)tb.iso[base];
        R le = 0, li = 0;
#pragma unroll
        for (int c8 = 1; c8 < 8; ++c8) {
            const int ca = c8 & 1, cb = (c8 >> 1) & 1, cc = c8 >> 2;
            const R w = (ca ? tr : (R)1 - tr) * (cb ? tt : (R)1 - tt) * (cc ? ty : (R)1 - ty);
            const long long o = base + ca * dR + cb * dT + cc * dY;
            if (kMixed) { le += w * ((R)tb.emab_f[o] - le0); li += w * ((R)tb.iso_f[o] - li0); }
            else { le += w * ((R)tb.emab[o] - le0); li += w * ((R)tb.iso[o] - li0); }
        }
        le += le0;
        li += li0;
        chiab = (P.proc_mask & NMC_PROC_EMAB) ? (R)(dtau * sc[0]) * r_exp(le) : (R)0;
        sig = (P.proc_mask & NMC_PROC_ISO) ? (R)(dtau * sc[1]) * r_exp(li) : (R)0;
    }
    // NES and pair kernels: bilinear in (log10 T, eta_e), times dtau 4 pi / (hc)^3
    if (nes_on || pair_on) {
        const R kt = (R)os->kt, ke = (R)os->ke;
        const R w00 = ((R)1 - kt) * ((R)1 - ke), w10 = kt * ((R)1 - ke);
        const R w01 = ((R)1 - kt) * ke, w11 = kt * ke;
        const long long mat = (long long)NE * NE;
        const long long sE = mat, sT = (long long)tb.eta.n * mat;
        const double unit = kMixed ? dtau : dtau * kCW;   // FP32 tables carry 4 pi/(hc)^3
        if (nes_on && s < NS) {
            const R c = (R)(unit * sc[2]);
            const long long off = (((long long)s * tb.kt.n + os->ikt) * tb.eta.n + os->ike) * mat;
            R* P0 = b.phi + s * NE * LD;
            // lower triangle incl. diagonal, entries enumerated row by row so that every lane of the
            // species group has one (a row loop with q <= r leaves half the lanes idle)
            const int ntri = NE * (NE + 1) / 2;
            for (int idx = q; idx < ntri; idx += NEP) {
                int r = (int)((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
                while (r * (r + 1) / 2 > idx) --r;
                while ((r + 1) * (r + 2) / 2 <= idx) ++r;
                const int cc = idx - r * (r + 1) / 2;
                const long long o = off + (long long)r * NE + cc;
                R v;
                if (kMixed) {
                    const float* t = tb.nes_f;
                    v = w00 * t[o] + w10 * t[o + sT] + w01 * t[o + sE] + w11 * t[o + sT + sE];
                } else {
                    const double* t = tb.nes;
                    v = w00 * t[o] + w10 * t[o + sT] + w01 * t[o + sE] + w11 * t[o + sT + sE];
                }
                P0[r * LD + cc] = c * v;
            }
        }
        if (pair_on && s < NS) {
            const int pr = s >> 1;
            const R c = (R)(unit * sc[3]);
            const long long off = (((long long)pr * tb.kt.n + os->ikt) * tb.eta.n + os->ike) * mat;
            R* A0 = b.ann + pr * NE * LD;
            for (int idx = (s & 1) * NEP + q; idx < NE * NE; idx += 2 * NEP) {
                const int r = idx / NE, cc = idx - r * NE;
                const long long o = off + idx;
                R v;
                if (kMixed) {
                    const float* t = tb.pair_f;
                    v = w00 * t[o] + w10 * t[o + sT] + w01 * t[o + sE] + w11 * t[o + sT + sE];
                } else {
                    const double* t = tb.pair;
                    v = w00 * t[o] + w10 * t[o + sT] + w01 * t[o + sE] + w11 * t[o + sT + sE];
                }
                A0[r * LD + cc] = c * v;
            }
        }
        __syncthreads();
        if (nes_on && s < NS) {   // up-scattering by detailed balance: K[r][c] = a_c / a_r K[c][r], r < c
            R* P0 = b.phi + s * NE * LD;
            const R* va = b.vA + s * NEP;
            const R* vai = b.vAi + s * NEP;
            const int nup = NE * (NE - 1) / 2;   // strictly upper entries, column by column
            for (int idx = q; idx < nup; idx += NEP) {
                int cc = (int)((sqrtf(8.0f * idx + 1.0f) + 1.0f) * 0.5f);
                while (cc * (cc - 1) / 2 > idx) --cc;
                while ((cc + 1) * cc / 2 <= idx) ++cc;
                const int r = idx - cc * (cc - 1) / 2;
                P0[r * LD + cc] = va[cc] * vai[r] * P0[cc * LD + r];
            }
        }
    }
    __syncthreads();
}

}  // namespace nmc
