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

#include <type_traits>

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

// ---- double-float: an unevaluated sum h + l of two FP32 words ----
// Carries about 48 significant bits in FP32 arithmetic (Dekker, Numer. Math. 18,
// 1971).  two_sum is Knuth's error-free addition (TAOCP vol. 2, 4.2.2): s + e
// equals a + b exactly for any magnitudes.  The _rn intrinsics keep the
// compiler from contracting or reassociating the error terms.
struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 f2_from(double x) {
    F2 r;
    r.h = (float)x;
    r.l = (float)(x - (double)r.h);
    return r;
}

__device__ __forceinline__ double f2_to(F2 a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ float two_sum(float a, float b, float* e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    *e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// a + b for a float b, renormalised so that |l| <= ulp(h) / 2
__device__ __forceinline__ F2 f2_add(F2 a, float b) {
    float e, e2;
    const float s = two_sum(a.h, b, &e);
    F2 r;
    r.h = two_sum(s, __fadd_rn(e, a.l), &e2);
    r.l = e2;
    return r;
}

// A - c x + t with A, c, x double-float and t a float.  Near a root the terms
// cancel: A - c x keeps ~2^-48 |A| absolute error (the high product is exact by
// two-product with an FMA, and A.h - p is exact once they are within a factor
// of two), and t is added to the high part first, which it cancels.
__device__ __forceinline__ float f2_residual(F2 A, F2 c, F2 x, float t) {
    const float p = __fmul_rn(c.h, x.h);
    float pe = fmaf(c.h, x.h, -p);   // c.h x.h = p + pe exactly
    pe = fmaf(c.h, x.l, pe);
    pe = fmaf(c.l, x.h, pe);
    float e;
    const float s = two_sum(A.h, -p, &e);
    return __fadd_rn(__fadd_rn(s, t), __fadd_rn(e, __fsub_rn(A.l, pe)));
}

// block_sum split at its first barrier: warp w's sums of the K values land in
// scratch[w * K + k]; after a barrier, sum_partials in any one thread adds the
// warps' partials in the order block_sum uses.
template <int K, typename T>
__device__ __forceinline__ void warp_partials(T (&v)[K], void* scratch) {
    T* red = static_cast<T*>(scratch);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(kFull, v[k], off);
    }
    if ((threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) red[w * K + k] = v[k];
    }
}

template <int K, typename T>
__device__ __forceinline__ void sum_partials(const void* scratch, T (&out)[K]) {
    const T* red = static_cast<const T*>(scratch);
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T s = 0;
        for (int i = 0; i < nw; ++i) s += red[i * K + k];
        out[k] = s;
    }
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

// Inner Anderson least squares at depth <= 3, run by all 32 lanes of one warp:
// the steps of anderson_solve's n <= 2 branch (same pivot tests, Cramer's rule)
// with the independent FP64 products of a step on different lanes, so that a
// step costs one warp instruction (an FP64 instruction holds its SMSP's FP64
// pipe ~64 cycles however few lanes are active).  Lane k < 5 passes entry k of
// (a00, a01, a11, r0, r1), the eliminated normal equations A gamma = r with
// A_ij = <F_L - F_gi, F_L - F_gj> and r_i = <F_L - F_gi, F_L> over the window
// g0 < g1 < L of n + 1 = m columns.  Every lane gets the coefficients (c0, c1,
// cL) of columns g0, g1 (n = 2) and L; a numerically singular system gives the
// Picard step (0, 0, 1).
__device__ __forceinline__ void anderson3_warp(double e, int n, double& c0, double& c1, double& cL) {
    const int lane = threadIdx.x & 31;
    const double a00 = __shfl_sync(kFull, e, 0), a01 = __shfl_sync(kFull, e, 1);
    const double a11 = __shfl_sync(kFull, e, 2), r0 = __shfl_sync(kFull, e, 3);
    const double r1 = __shfl_sync(kFull, e, 4);
    c0 = 0.0;
    c1 = 0.0;
    cL = 1.0;
    if (n == 1) {
        if (fabs(a00) > 1e-14 * fabs(a00) && isfinite(a00)) {
            const double gam = r0 / a00;
            if (isfinite(gam)) { c0 = gam; cL = 1.0 - gam; }
        }
    } else if (n == 2) {
        const double dmax = fmax(fabs(a00), fabs(a11));
        if (dmax > 0.0 && isfinite(dmax)) {
            // column 0 with partial pivoting (A is symmetric: a10 = a01)
            const bool sw = fabs(a01) > fabs(a00);
            const double p0 = sw ? a01 : a00, p1 = sw ? a11 : a01, pr = sw ? r1 : r0;
            const double q0 = sw ? a00 : a01, q1 = sw ? a01 : a11, qr = sw ? r0 : r1;
            if (fabs(p0) > 1e-14 * dmax) {
                // lane 0: det = p0 q1 - q0 p1; lane 1: p0 qr - q0 pr (gamma1 det);
                // lane 2: pr q1 - p1 qr (gamma0 det), as one x y - z w
                const double x = lane == 2 ? pr : p0;
                const double y = lane == 1 ? qr : q1;
                const double z = lane == 2 ? p1 : q0;
                const double w = lane == 0 ? p1 : (lane == 1 ? pr : qr);
                const double t = x * y - z * w;
                const double det = __shfl_sync(kFull, t, 0);
                if (fabs(det) > 1e-14 * dmax * fabs(p0)) {
                    const double gm = t * (1.0 / det);
                    const double gm1 = __shfl_sync(kFull, gm, 1), gm0 = __shfl_sync(kFull, gm, 2);
                    const double sum = gm0 + gm1;
                    if (isfinite(sum)) { c0 = gm0; c1 = gm1; cL = 1.0 - sum; }
                }
            }
        }
    }
}

// Coefficient of history column j (0..2, newest last) from anderson3_warp's
// (c0, c1, cL): n = 2 -> (g0, g1, L) = (0, 1, 2); n = 1 -> (g0, L) = (1, 2).
__device__ __forceinline__ double anderson3_coef(int j, int n, double c0, double c1, double cL) {
    return j == 2 ? cL : (n == 2 ? (j == 0 ? c0 : c1) : (n == 1 && j == 1 ? c0 : 0.0));
}

// The lead warp's update of the depth-3 Gram history G (the leading 3 x 3 of a
// row length LDG array in shared or global memory, newest last) with the new row (lane k < 3 holds <F_L, F_k>), returning in lane k < 5
// entry k of (a00, a01, a11, r0, r1) for the window of m columns.
template <int LDG>
__device__ __forceinline__ double gram3_update_warp(double (*G)[LDG], double nr, int m) {
    const int lane = threadIdx.x & 31;
    const int i = lane / 3, j = lane - 3 * i;
    const double ni = __shfl_sync(kFull, nr, i < 3 ? i : 0), nj = __shfl_sync(kFull, nr, j);
    double val = 0.0;
    if (lane < 9) val = (i < 2 && j < 2) ? G[i + 1][j + 1] : (i == 2 ? nj : ni);
    __syncwarp();
    if (lane < 9) G[i][j] = val;
    __syncwarp();
    const int L = 2, g0 = 3 - (m < 2 ? 2 : m), g1 = g0 + 1;
    // a_ij = G_ij - G_iL - G_jL + G_LL and r_i = G_LL - G_iL in one shape
    const bool isr = lane >= 3;
    const int gi = (lane == 0 || lane == 1 || lane == 3) ? g0 : g1;
    const int gj = lane == 0 ? g0 : g1;
    const double u = isr ? G[L][L] : G[gi][gj];
    const double w = isr ? 0.0 : G[gj][L];
    const double z = isr ? 0.0 : G[L][L];
    return ((u - G[gi][L]) - w) + z;
}

// Outer least squares on the 2-component scaled residuals, by one thread (windows deeper than 3;
// outer_step_warp handles depth <= 3 lane-parallel).
__device__ inline void outer_anderson(const double (&fh)[kMaxOuterMem][2], int m, double* beta) {
    constexpr int MM = kMaxOuterMem;
    double G[MM][MM];
    for (int i = 0; i < MM; ++i)
        for (int j = 0; j < MM; ++j) G[i][j] = fh[i][0] * fh[j][0] + fh[i][1] * fh[j][1];
    anderson_solve<MM>(G, m, beta);
}

// One outer Anderson step of Algorithm 1 (the mixing of the matter iterate,
// stopped by Algorithm 3), run by all 32 lanes of one warp with every lane
// holding the node's scalars.  Pushes q = (qv0, qv1) and its residual
// (q - y) / |y*| (ri_ys = 1 / |y*|) onto the histories qh, fh (newest last;
// shared or global memory; lane 0 writes) and returns the mixed iterate in
// every lane.  At depth mo <= 3 the least squares runs lane-parallel
// (anderson3_warp) on the eliminated normal equations formed from residual
// differences; deeper windows use outer_anderson.
__device__ inline void outer_step_warp(double (*qh)[2], double (*fh)[2], double qv0, double qv1, double y0,
                                       double y1, const double* ri_ys, int mo, double& yn0, double& yn1) {
    constexpr int MM = kMaxOuterMem;
    const int ln = threadIdx.x & 31;
    const double f0 = (qv0 - y0) * ri_ys[0], f1 = (qv1 - y1) * ri_ys[1];
    __syncwarp();
    if (ln == 0) {
        for (int j = 0; j < MM - 1; ++j) {
            qh[j][0] = qh[j + 1][0]; qh[j][1] = qh[j + 1][1];
            fh[j][0] = fh[j + 1][0]; fh[j][1] = fh[j + 1][1];
        }
        qh[MM - 1][0] = qv0;
        qh[MM - 1][1] = qv1;
        fh[MM - 1][0] = f0;
        fh[MM - 1][1] = f1;
    }
    __syncwarp();
    yn0 = 0.0;
    yn1 = 0.0;
    if (mo <= 3) {
        // lane e < 5: entry e of the eliminated normal equations over the last mo columns,
        // a_ij = <f_L - f_gi, f_L - f_gj>, r_i = <f_L - f_gi, f_L>
        const int L = MM - 1, g0 = MM - (mo < 2 ? 2 : mo), g1 = g0 + 1;
        const bool isr = ln >= 3;
        const int gi = (ln == 0 || ln == 1 || ln == 3) ? g0 : g1;
        const int gj = ln == 0 ? g0 : g1;
        const double u0 = fh[L][0] - fh[gi][0], u1 = fh[L][1] - fh[gi][1];
        const double w0 = isr ? fh[L][0] : fh[L][0] - fh[gj][0];
        const double w1 = isr ? fh[L][1] : fh[L][1] - fh[gj][1];
        double c0, c1, cL;
        anderson3_warp(u0 * w0 + u1 * w1, mo - 1, c0, c1, cL);
        for (int j = 3 - mo; j < 3; ++j) {   // history column MM - 3 + j
            const double b = anderson3_coef(j, mo - 1, c0, c1, cL);
            yn0 += b * qh[MM - 3 + j][0];
            yn1 += b * qh[MM - 3 + j][1];
        }
    } else {
        double fl[MM][2], beta[MM];
        for (int j = 0; j < MM; ++j) { fl[j][0] = fh[j][0]; fl[j][1] = fh[j][1]; }
        outer_anderson(fl, mo, beta);
        for (int j = MM - mo; j < MM; ++j) {
            yn0 += beta[j] * qh[j][0];
            yn1 += beta[j] * qh[j][1];
        }
    }
}


// Node-wide results of the scalar part of ComputeOpacities (shared memory,
// written by lane 0 of the lead warp).
struct OpacState {
    double eta_e;              // mu_e / T
    double mu[kMaxSpecies];    // neutrino chemical potentials per species
    double tinv;               // 1 / T
    double tr, tt, ty, kt, ke; // fractional offsets in the table cells
    double pre[4];             // dtau sc_EmAb, dtau sc_Iso, and the NES and pair prefactors
    // FP32 copies for the mixed-precision path: mu and 1 / T as double-floats
    float mu_h[kMaxSpecies], mu_l[kMaxSpecies], tinv_h, tinv_l;
    float wf[5];               // tr, tt, ty, kt, ke
    float pre_f[4];
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
    R* phi1 = nullptr;   // linear-order NES kernels K_1,Out (as phi), filled when the tables have them
    R* ann1 = nullptr;   // linear-order pair kernels K_1,Ann (as ann)
};

// ComputeOpacities of Algorithm 1 at the matter state (rho, T, Ye), called by
// every thread of the block with the same arguments (sc points to the node's
// four scale factors EmAb, Iso, NES, Pair).
//  - Chemical potentials from the EoS (the lead warp; an FP32 root refined in FP64 in mixed
//    precision).
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
// The warp of thread `lead` (lane 0 of its warp) does the scalar part; `lead`
// ORs NMC_TABLE_CLAMP into *status when a lookup leaves a table.
// Ends with the block synchronised.
// Thread (s, q) = s * nep + q owns species s at energy node q and gets its
// bin's chi_EmAb, sigma_Iso, D^Eq and 1 - D^Eq back.
// ComputeOpacities' load batches: Fermi--Dirac points per thread, and kernel-table entries per
// thread in the NES/pair fill (four corners each; fewer in FP64, whose values take two registers).
constexpr int kFdBatch = 8;
constexpr int kFillBatchF32 = 6;
constexpr int kFillBatchF64 = 4;

template <typename R>
__device__ void compute_opacities(const DevGrid& g, const DevTables& tb, const nmc_params& P, double rho, double T,
                                  double Ye, double dtau, const double* sc, const OpacBufs<R>& b, OpacState* os,
                                  int* status, R& chiab, R& sig, R& deq, R& deqc, int lead = 0) {
    constexpr bool kMixed = sizeof(R) == 4;
    const int NS = g.ns, NE = g.ne, NEP = g.nep, LD = g.ld;
    const int GS = NEP;   // threads per species
    const int tid = threadIdx.x;
    const int s = tid / GS, q = tid - s * GS;
    const bool nes_on = (P.proc_mask & NMC_PROC_NES) != 0;
    const bool pair_on = (P.proc_mask & NMC_PROC_PAIR) != 0;
    R* fq = b.phi;

    if ((tid >> 5) == (lead >> 5)) {
        // The lead warp, every lane carrying the node's scalars: the independent evaluations of one
        // function (the logarithms, the five table cells) run on different lanes for the cost of
        // one, since a scalar FP64 step costs the same on 1 or 32 lanes.  Lane 0 writes.
        const int ln = tid & 31;
        // log10 of rho, T, 1 - Ye and Ye on lanes 0..3; ln((1 - Ye)/Ye) = ln 10 (log10(1-Ye) - log10 Ye)
        const double lx = log10(ln == 0 ? rho : (ln == 1 ? T : (ln == 2 ? 1.0 - Ye : Ye)));
        const double lrho = __shfl_sync(kFull, lx, 0), lT = __shfl_sync(kFull, lx, 1);
        const double lratio = (__shfl_sync(kFull, lx, 2) - __shfl_sync(kFull, lx, 3)) * kLn10;
        // mixed: the FP32 root of the electron cubic, then one FP64 Newton step on it (the error
        // squares): mu_e, and with it D^Eq, must move smoothly with (T, Ye), or the outer
        // iteration's map is noisy at the 1e-7 level and stalls above tol_outer
        const double mu_e = kMixed ? eos_mu_e_refined(rho, T, Ye) : eos_mu_e(rho, T, Ye);
        const double mnu = mu_e - (T * lratio + kDmNP);   // mu_e - mu_hat
        const double tinv = 1.0 / T;
        const double eta_e = mu_e / T;
        // table cells in FP64 in both precisions, lane 0: log10 rho, 1: log10 T (EmAb/Iso axis),
        // 2: Ye, 3: log10 T (kernel axis), 4: eta_e
        const int nax = (nes_on || pair_on) ? 5 : 3;
        const Axis ax = ln == 0 ? tb.rho : (ln == 1 ? tb.t : (ln == 2 ? tb.ye : (ln == 3 ? tb.kt : tb.eta)));
        int ci = 0, cl = 0;
        double ct = 0.0;
        axis_cell<double>(ln == 0 ? lrho : ((ln == 1 || ln == 3) ? lT : (ln == 2 ? Ye : eta_e)), ax, &ci, &ct, &cl);
        const bool any_cl = __ballot_sync(kFull, cl && ln < nax) != 0u;
        if (ln == 0) { os->ir = ci; os->tr = ct; }
        if (ln == 1) { os->it = ci; os->tt = ct; }
        if (ln == 2) { os->iy = ci; os->ty = ct; }
        if (ln == 3 && nax == 5) { os->ikt = ci; os->kt = ct; }
        if (ln == 4 && nax == 5) { os->ike = ci; os->ke = ct; }
        if (kMixed && ln < nax) os->wf[ln] = (float)ct;
        if (ln == 0) {
            os->tinv = tinv;
            os->eta_e = eta_e;
            for (int sp = 0; sp < kMaxSpecies; ++sp) os->mu[sp] = sp == 0 ? mnu : (sp == 1 ? -mnu : 0.0);
            if (any_cl) *status |= NMC_TABLE_CLAMP;
            const double unit = kMixed ? dtau : dtau * kCW;   // FP32 tables carry 4 pi/(hc)^3
            os->pre[0] = dtau * sc[0];
            os->pre[1] = dtau * sc[1];
            os->pre[2] = unit * sc[2];
            os->pre[3] = unit * sc[3];
            if (kMixed) {
                const F2 m2 = f2_from(mnu), t2 = f2_from(tinv);
                for (int sp = 0; sp < kMaxSpecies; ++sp) {
                    os->mu_h[sp] = sp == 0 ? m2.h : (sp == 1 ? -m2.h : 0.f);
                    os->mu_l[sp] = sp == 0 ? m2.l : (sp == 1 ? -m2.l : 0.f);
                }
                os->tinv_h = t2.h;
                os->tinv_l = t2.l;
                for (int k = 0; k < 4; ++k) os->pre_f[k] = (float)os->pre[k];
            }
        }
    }
    __syncthreads();
    // Fermi--Dirac at the projection quadrature points of every element.  The table reads of
    // this function hit L2 at several hundred cycles each, so every stage issues its loads in
    // straight-line batches (indices clamped into range, the results' stores guarded): one
    // memory latency per batch instead of one per loop trip.
    // The heavy flavours (species 2 and up) all have mu = 0, so they share species 2's values: the
    // nfd <= 3 distinct species' points are dealt out over every thread of the block.
    {
        const int nqp = g.n_elem * kProjQuad;
        const int nfd = NS < 3 ? NS : 3, nfdp = nfd * nqp;
        if (s < NS) {
            const R Tinv = (R)os->tinv;
            const float tih = os->tinv_h, til = os->tinv_l;
            const int nthr = NS * GS;
            for (int k0 = s * GS + q; k0 < nfdp; k0 += kFdBatch * nthr) {
                R eh[kFdBatch];
                float el[kFdBatch];
#pragma unroll
                for (int u = 0; u < kFdBatch; ++u) {
                    const int k = min(k0 + u * nthr, nfdp - 1);
                    const int i = k - (k >= 2 * nqp ? 2 * nqp : (k >= nqp ? nqp : 0));
                    if constexpr (kMixed) {
                        eh[u] = __ldg(g.proj_e_f + i);
                        el[u] = __ldg(g.proj_e_fl + i);
                    } else {
                        eh[u] = __ldg(g.proj_e + i);
                        el[u] = 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < kFdBatch; ++u) {
                    const int k = k0 + u * nthr;
                    const int sf = k >= 2 * nqp ? 2 : (k >= nqp ? 1 : 0);
                    const int i = k - sf * nqp;
                    R fv, fcv = 0;
                    if constexpr (kMixed) {
                        // f and 1 - f from one exp, each without cancellation.  x = (E - mu)/T reaches
                        // ~100 in the tail, where rounding x to FP32 would move exp(-|x|) by ~1e-5 in
                        // steps; x is formed as a double-float, e^-|x| = expf(-|x_hi|) (1 - |x|_lo)
                        const float muh = os->mu_h[sf], mul = os->mu_l[sf];
                        float e1, e2;
                        const float d0 = two_sum(eh[u], -muh, &e1);
                        const float dh = two_sum(d0, __fadd_rn(e1, __fsub_rn(el[u], mul)), &e2);
                        const float x0 = __fmul_rn(dh, tih);
                        float x1 = fmaf(dh, tih, -x0);   // dh tih = x0 + x1 exactly
                        x1 = fmaf(dh, til, x1);
                        x1 = fmaf(e2, tih, x1);
                        const bool pos = x0 > 0.f;
                        const float xh = fabsf(x0), xl = pos ? x1 : -x1;
                        const R t = r_exp(-xh) * (1.0f - xl);
                        const R inv = (R)1 / ((R)1 + t);
                        fv = pos ? t * inv : inv;
                        fcv = pos ? inv : t * inv;
                    } else {
                        const R mu = (R)os->mu[sf];
                        fv = (R)1 / (r_exp((eh[u] - mu) * Tinv) + (R)1);
                    }
                    if (k < nfdp && NMC_IN_BOUNDS(g.dbg, (long long)((kMixed ? NS : 0) + sf) * nqp + i,
                                                  (long long)(kMixed ? 2 : 1) * NS * nqp, kDbgSmemFd)) {
                        fq[sf * nqp + i] = fv;
                        if constexpr (kMixed) fq[(NS + sf) * nqp + i] = fcv;
                    }
                }
            }
        }
        __syncthreads();
        // eps^2-weighted projection and bound-enforcing limiter per (species, element), the sums over
        // the quadrature points taken in order, their operator weights loaded kProjQuad / 2 points at a
        // time.  With D^Eq also a = D^Eq / (1 - D^Eq) and 1 / a, which the detailed-balance fill of the
        // NES kernel reads across the species.
        constexpr int kHalfQ = kProjQuad / 2;
        for (int e = q; s < NS && e < g.n_elem; e += GS) {
            const int nq = g.nq;
            if (!NMC_IN_BOUNDS(g.dbg, ((long long)e * nq + nq - 1) * kProjQuad + kProjQuad - 1,
                               (long long)g.n_elem * nq * kProjQuad, kDbgProj) ||
                !NMC_IN_BOUNDS(g.dbg, (long long)s * NEP + e * nq + nq - 1, (long long)NS * NEP, kDbgSmemVec))
                continue;
            const int sfd = s < 2 ? s : 2;   // the heavy flavours' Fermi--Dirac values are species 2's
            const R* f = fq + sfd * nqp + e * kProjQuad;
            const R* fc = fq + (NS + sfd) * nqp + e * kProjQuad;
            R avg = 0, avgc = 0, coef[kMaxNq] = {0, 0, 0}, coefc[kMaxNq] = {0, 0, 0};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                R pa[kHalfQ], pc[kMaxNq][kHalfQ];
#pragma unroll
                for (int gq = 0; gq < kHalfQ; ++gq) {
                    const int qa = e * kProjQuad + h * kHalfQ + gq;
                    pa[gq] = kMixed ? (R)__ldg(g.proj_a_f + qa) : (R)__ldg(g.proj_a + qa);
#pragma unroll
                    for (int pp = 0; pp < kMaxNq; ++pp) {
                        const int o = (e * nq + min(pp, nq - 1)) * kProjQuad + h * kHalfQ + gq;
                        pc[pp][gq] = kMixed ? (R)__ldg(g.proj_c_f + o) : (R)__ldg(g.proj_c + o);
                    }
                }
#pragma unroll
                for (int gq = 0; gq < kHalfQ; ++gq) {
                    const R fv = f[h * kHalfQ + gq];
                    avg += pa[gq] * fv;
                    R fcv = 0;
                    if (kMixed) { fcv = fc[h * kHalfQ + gq]; avgc += pa[gq] * fcv; }
#pragma unroll
                    for (int pp = 0; pp < kMaxNq; ++pp) {
                        if (pp >= nq) break;
                        coef[pp] += pc[pp][gq] * fv;
                        if (kMixed) coefc[pp] += pc[pp][gq] * fcv;
                    }
                }
            }
            const R dmin = (R)P.d_min, dmax = (R)P.d_max;
            // loops over the element's nq <= kMaxNq nodes, unrolled to kMaxNq so that the arrays stay in
            // registers
            if (avg < dmin || avg > dmax) {
                const bool lo = avg < dmin;
                const R cv = lo ? dmin : dmax;
                const R cvc = lo ? (R)(1.0 - P.d_min) : (R)(1.0 - P.d_max);
#pragma unroll
                for (int pp = 0; pp < kMaxNq; ++pp) { coef[pp] = cv; coefc[pp] = cvc; }
            } else {
                R vmin = coef[0], vmax = coef[0];
#pragma unroll
                for (int pp = 1; pp < kMaxNq; ++pp)
                    if (pp < nq) { vmin = fmin(vmin, coef[pp]); vmax = fmax(vmax, coef[pp]); }
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    R v = 0;
#pragma unroll
                    for (int pp = 0; pp < kMaxNq; ++pp)
                        if (pp < nq) v += coef[pp] * (R)g.ends[side][pp];
                    vmin = fmin(vmin, v);
                    vmax = fmax(vmax, v);
                }
                R theta = 1;
                if (vmin < dmin) theta = fmin(theta, (avg - dmin) / (avg - vmin));
                if (vmax > dmax) theta = fmin(theta, (dmax - avg) / (vmax - avg));
#pragma unroll
                for (int pp = 0; pp < kMaxNq; ++pp) {
                    coef[pp] = avg + theta * (coef[pp] - avg);
                    coefc[pp] = avgc + theta * (coefc[pp] - avgc);
                }
                // the limiter puts the extreme point on the bound in exact arithmetic; the rounding of
                // avg + theta (v - avg) can leave it just outside (below zero where avg is far above
                // d_min, e.g. quadratic elements on a steep tail), so the nodal values are clipped
                // (comparisons keep a NaN)
                const R cmin = (R)(1.0 - P.d_max), cmax = (R)(1.0 - P.d_min);
#pragma unroll
                for (int pp = 0; pp < kMaxNq; ++pp) {
                    coef[pp] = coef[pp] < dmin ? dmin : (coef[pp] > dmax ? dmax : coef[pp]);
                    coefc[pp] = coefc[pp] < cmin ? cmin : (coefc[pp] > cmax ? cmax : coefc[pp]);
                }
            }
#pragma unroll
            for (int pp = 0; pp < kMaxNq; ++pp) {
                if (pp >= nq) break;
                const int sq = s * NEP + e * nq + pp;
                const R dc = kMixed ? coefc[pp] : (R)1 - coef[pp];
                b.vDeq[sq] = coef[pp];
                b.vDeqc[sq] = coefc[pp];
                b.vA[sq] = coef[pp] / dc;
                b.vAi[sq] = dc / coef[pp];
            }
        }
        __syncthreads();
    }
    // EmAb / Iso: trilinear in (log10 rho, log10 T, Ye) on ln values, times dtau
    if (s < NS && q < NE) {
        const int qb = q, sq = s * NEP + q;
        deq = b.vDeq[sq];
        deqc = kMixed ? b.vDeqc[sq] : (R)1 - deq;
        const int nr = tb.rho.n, nt = tb.t.n, ny = tb.ye.n;
        const long long base = ((((long long)s * ny + os->iy) * nt + os->it) * nr + os->ir) * NE + qb;
        const long long dR = NE, dT = (long long)nr * NE, dY = (long long)nt * nr * NE;
        const bool tab_ok = NMC_IN_BOUNDS(g.dbg, base, tb.n_op, kDbgEmabIso) &&
                            NMC_IN_BOUNDS(g.dbg, base + dR + dT + dY, tb.n_op, kDbgEmabIso);
        const R tr = kMixed ? (R)os->wf[0] : (R)os->tr;
        const R tt = kMixed ? (R)os->wf[1] : (R)os->tt;
        const R ty = kMixed ? (R)os->wf[2] : (R)os->ty;
        // ln chi as the first corner plus weighted differences: the corners are ~ -20, so an
        // FP32 sum of the corner values themselves would round ln chi by ~2e-6 in steps
        const R le0 = !tab_ok ? (R)0 : (kMixed ? (R)tb.emab_f[base] : (R)tb.emab[base]);
        const R li0 = !tab_ok ? (R)0 : (kMixed ? (R)tb.iso_f[base] : (R)tb.iso[base]);
        R le = 0, li = 0;
#pragma unroll
        for (int c8 = 1; c8 < 8; ++c8) {
            if (!tab_ok) break;
            const int ca = c8 & 1, cb = (c8 >> 1) & 1, cc = c8 >> 2;
            const R w = (ca ? tr : (R)1 - tr) * (cb ? tt : (R)1 - tt) * (cc ? ty : (R)1 - ty);
            const long long o = base + ca * dR + cb * dT + cc * dY;
            if (kMixed) { le += w * ((R)tb.emab_f[o] - le0); li += w * ((R)tb.iso_f[o] - li0); }
            else { le += w * ((R)tb.emab[o] - le0); li += w * ((R)tb.iso[o] - li0); }
        }
        le += le0;
        li += li0;
        const R pe = kMixed ? (R)os->pre_f[0] : (R)os->pre[0];
        const R pi = kMixed ? (R)os->pre_f[1] : (R)os->pre[1];
        chiab = (P.proc_mask & NMC_PROC_EMAB) ? pe * r_exp(le) : (R)0;
        sig = (P.proc_mask & NMC_PROC_ISO) ? pi * r_exp(li) : (R)0;
    }
    // NES and pair kernels: bilinear in (log10 T, eta_e), times dtau 4 pi / (hc)^3
    if (nes_on || pair_on) {
        const R kt = kMixed ? (R)os->wf[3] : (R)os->kt;
        const R ke = kMixed ? (R)os->wf[4] : (R)os->ke;
        const R w00 = ((R)1 - kt) * ((R)1 - ke), w10 = kt * ((R)1 - ke);
        const R w01 = ((R)1 - kt) * ke, w11 = kt * ke;
        const long long mat = (long long)NE * NE;
        const long long sE = mat, sT = (long long)tb.eta.n * mat;
        // One kernel order (Phi_0, or Phi_1 into PH1/AN1), as a list of jobs per lane of the species
        // group, each one table entry (a row pass puts the lanes of a warp on contiguous runs of a row),
        // taken in straight-line batches whose four-corner loads are all issued before any is combined.
        //  NES: the tabulated lower triangle (q >= q'), each entry also giving its up-scattering
        //  mirror by detailed balance, K[c][r] = a_r / a_c K[r][c] for c < r (the a of the species
        //  were formed with D^Eq).  Job p < NE/2 pairs row p (p + 1 entries, lanes 0..p) with row
        //  NE-1-p (its NE-1-p off-diagonal entries, lanes p+1..NE-1); job NE/2 takes the diagonals
        //  of those rows and, for odd NE, the middle row.
        //  Pair: the whole K_Ann of each particle/antiparticle pair, the particle's group taking the
        //  even rows and the antiparticle's the odd ones (lane q: column q).
        auto fill = [&](const double* tn, const float* tnf, const double* tp, const float* tpf, R* PH, R* AN) {
            if (s >= NS || q >= NE) return;
            constexpr int kB = kMixed ? kFillBatchF32 : kFillBatchF64;
            const int half = NE >> 1, pr = s >> 1;
            const int n_nes = nes_on ? half + 1 : 0;
            const int n_pair = pair_on ? (NE - (s & 1) + 1) >> 1 : 0;
            const int njobs = n_nes + n_pair;
            const long long off_n = (((long long)s * tb.kt.n + os->ikt) * tb.eta.n + os->ike) * mat;
            const long long off_p = (((long long)pr * tb.kt.n + os->ikt) * tb.eta.n + os->ike) * mat;
            const R c_n = kMixed ? (R)os->pre_f[2] : (R)os->pre[2];
            const R c_p = kMixed ? (R)os->pre_f[3] : (R)os->pre[3];
            R* P0 = PH + s * NE * LD;
            R* A0 = AN + pr * NE * LD;
            const R* va = b.vA + s * NEP;
            const R* vai = b.vAi + s * NEP;
            for (int j0 = 0; j0 < njobs; j0 += kB) {
                int rr[kB], cl[kB];
                R t[kB][4];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int jj = min(j0 + u, njobs - 1);
                    int r, cc;
                    const bool isn = jj < n_nes;
                    if (isn) {
                        const int p = jj;
                        if (p < half) {
                            if (q <= p) { r = p; cc = q; }
                            else { r = NE - 1 - p; cc = q - p - 1; }
                        } else if (q >= NE - half) {   // diagonals of the rows paired above
                            r = q; cc = q;
                        } else if ((NE & 1) && q <= half) {   // odd NE: the middle row
                            r = half; cc = q;
                        } else {
                            r = -1; cc = 0;
                        }
                    } else {
                        r = (s & 1) + 2 * (jj - n_nes);
                        cc = q;
                    }
                    long long o = (isn ? off_n : off_p) + (long long)(r < 0 ? 0 : r) * NE + cc;
                    // NMC_DEBUG: a corner outside the table is not read (entry skipped, offset 0 read instead)
                    const bool tab_ok = isn ? NMC_IN_BOUNDS(g.dbg, o + sT + sE, tb.n_nes, kDbgNesTable)
                                            : NMC_IN_BOUNDS(g.dbg, o + sT + sE, tb.n_pair, kDbgPairTable);
                    if (!tab_ok) o = 0;
                    rr[u] = (j0 + u < njobs && tab_ok) ? r : -1;
                    cl[u] = cc;
                    if constexpr (kMixed) {
                        const float* tf = isn ? tnf : tpf;
                        t[u][0] = __ldg(tf + o); t[u][1] = __ldg(tf + o + sT);
                        t[u][2] = __ldg(tf + o + sE); t[u][3] = __ldg(tf + o + sT + sE);
                    } else {
                        const double* td = isn ? tn : tp;
                        t[u][0] = __ldg(td + o); t[u][1] = __ldg(td + o + sT);
                        t[u][2] = __ldg(td + o + sE); t[u][3] = __ldg(td + o + sT + sE);
                    }
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int r = rr[u], cc = cl[u];
                    if (r < 0) continue;
                    const bool isn = j0 + u < n_nes;
                    const R v = w00 * t[u][0] + w10 * t[u][1] + w01 * t[u][2] + w11 * t[u][3];
                    if (isn) {
                        if (!NMC_IN_BOUNDS(g.dbg, (long long)s * NE * LD + r * LD + cc, (long long)NS * NE * LD, kDbgSmemNes) ||
                            !NMC_IN_BOUNDS(g.dbg, (long long)s * NE * LD + cc * LD + r, (long long)NS * NE * LD, kDbgSmemNes))
                            continue;
                        const R k = c_n * v;
                        P0[r * LD + cc] = k;
                        if (cc < r) P0[cc * LD + r] = va[r] * vai[cc] * k;
                    } else {
                        if (!NMC_IN_BOUNDS(g.dbg, (long long)pr * NE * LD + r * LD + cc, (long long)(NS / 2) * NE * LD,
                                           kDbgSmemPair))
                            continue;
                        A0[r * LD + cc] = c_p * v;
                    }
                }
            }
        };
        // The same fill with 16-byte table loads (kV entries of a row per load), when rows split into
        // whole 16-byte chunks (NE a multiple of kV; the tables' rows then start on 16-byte boundaries).
        //  NES: row pair (p, NE-1-p) covers its lower-triangle columns in NE/kV + 1 chunks (the last chunk
        //  of a row may reach above the diagonal; those entries are not stored).  Pair: the group's rows
        //  in NE/kV chunks each.  Chunks are dealt to the lanes of the species group in turn.
        constexpr int kV = 16 / (int)sizeof(R);
        using VecR = typename std::conditional<kMixed, float4, double2>::type;
        auto fill_vec = [&](const double* tn, const float* tnf, const double* tp, const float* tpf, R* PH, R* AN) {
            if (s >= NS) return;
            const int nc = NE / kV, pr = s >> 1;
            auto corners = [&](const double* td, const float* tf, long long o, R (&v)[kV]) {
                const VecR* p00 = reinterpret_cast<const VecR*>(kMixed ? (const void*)(tf + o) : (const void*)(td + o));
                const long long vT = sT / kV, vE = sE / kV;
                const VecR a = __ldg(p00), bq = __ldg(p00 + vT), cq = __ldg(p00 + vE), dq = __ldg(p00 + vT + vE);
                const R* ra = reinterpret_cast<const R*>(&a);
                const R* rb = reinterpret_cast<const R*>(&bq);
                const R* rc = reinterpret_cast<const R*>(&cq);
                const R* rd = reinterpret_cast<const R*>(&dq);
#pragma unroll
                for (int i = 0; i < kV; ++i) v[i] = w00 * ra[i] + w10 * rb[i] + w01 * rc[i] + w11 * rd[i];
            };
            if (nes_on) {
                const R c_n = kMixed ? (R)os->pre_f[2] : (R)os->pre[2];
                const long long off_n = (((long long)s * tb.kt.n + os->ikt) * tb.eta.n + os->ike) * mat;
                R* P0 = PH + s * NE * LD;
                const R* va = b.vA + s * NEP;
                const R* vai = b.vAi + s * NEP;
                const int per = nc + 1, total = (NE >> 1) * per;
#pragma unroll 2
                for (int c = q; c < total; c += GS) {
                    const int p = c / per, k = c - p * per, kp = p / kV + 1;
                    const int r = k < kp ? p : NE - 1 - p;
                    const int c0 = (k < kp ? k : k - kp) * kV;
                    const long long o = off_n + (long long)r * NE + c0;
                    if (!NMC_IN_BOUNDS(g.dbg, o + sT + sE + kV - 1, tb.n_nes, kDbgNesTable) ||
                        !NMC_IN_BOUNDS(g.dbg, (long long)s * NE * LD + r * LD + c0 + kV - 1, (long long)NS * NE * LD, kDbgSmemNes) ||
                        !NMC_IN_BOUNDS(g.dbg, (long long)s * NE * LD + (c0 + kV - 1) * LD + r, (long long)NS * NE * LD, kDbgSmemNes))
                        continue;
                    R v[kV];
                    corners(tn, tnf, o, v);
                    const R ar = va[r];
#pragma unroll
                    for (int i = 0; i < kV; ++i) {
                        const int col = c0 + i;
                        if (col > r) break;
                        const R kk = c_n * v[i];
                        P0[r * LD + col] = kk;
                        if (col < r) P0[col * LD + r] = ar * vai[col] * kk;
                    }
                }
            }
            if (pair_on) {
                const R c_p = kMixed ? (R)os->pre_f[3] : (R)os->pre[3];
                const long long off_p = (((long long)pr * tb.kt.n + os->ikt) * tb.eta.n + os->ike) * mat;
                R* A0 = AN + pr * NE * LD;
                const int total = ((NE - (s & 1) + 1) >> 1) * nc;
#pragma unroll 2
                for (int c = q; c < total; c += GS) {
                    const int rr2 = c / nc, c0 = (c - rr2 * nc) * kV;
                    const int r = (s & 1) + 2 * rr2;
                    const long long o = off_p + (long long)r * NE + c0;
                    if (!NMC_IN_BOUNDS(g.dbg, o + sT + sE + kV - 1, tb.n_pair, kDbgPairTable) ||
                        !NMC_IN_BOUNDS(g.dbg, (long long)pr * NE * LD + r * LD + c0 + kV - 1, (long long)(NS / 2) * NE * LD,
                                       kDbgSmemPair))
                        continue;
                    R v[kV];
                    corners(tp, tpf, o, v);
#pragma unroll
                    for (int i = 0; i < kV; ++i) A0[r * LD + c0 + i] = c_p * v[i];
                }
            }
        };
        const bool vec = NE % kV == 0;
        if (vec) fill_vec(tb.nes, tb.nes_f, tb.pair, tb.pair_f, b.phi, b.ann);
        else fill(tb.nes, tb.nes_f, tb.pair, tb.pair_f, b.phi, b.ann);
        // linear-order kernels: the same interpolation, scale factors and relations (in-out invariance,
        // detailed balance) as the isotropic ones
        if (!kMixed && b.phi1 != nullptr && tb.nes1 != nullptr) {
            if (vec) fill_vec(tb.nes1, nullptr, tb.pair1, nullptr, b.phi1, b.ann1);
            else fill(tb.nes1, nullptr, tb.pair1, nullptr, b.phi1, b.ann1);
        }
    }
    __syncthreads();
}

}  // namespace nmc
