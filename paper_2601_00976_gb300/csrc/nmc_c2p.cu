// Conserved-to-primitive moment recovery (Sec. 3.4, Eqs. conservedToPrimitive,
// c2p_FP and c2p_sequence), FP64.
//
// For conserved moments U = (N, G_j) and fluid velocity v (units of c, flat
// metric) the primitive moments M = (D, I_j) solve N = D + v^i I_i and
// G_j = I_j + v^i K_ij(M), K_ij = a delta_ij + c I_i I_j from Minerbo's
// closure (Eqs. eddingtonTensor, eddingtonFactorMinerbo).  The fixed-point map
//   g(M) = (1 - lam) M + lam (N - v.I, G - v.K(M)),  lam = 1 / (1 + |v|),
// is iterated from M = U with Anderson acceleration (memory <= 3, constraint
// eliminated, the 2 x 2 normal equations by Cramer's rule with the pivot tests
// of the collision solve) until ||M_new - M|| <= tol ||U||.
//
// Every (node, species, energy) bin is an independent four-unknown problem,
// so one thread owns one bin and keeps its Anderson history in registers: no
// shared memory, no barriers.  Blocks cover whole nodes (ns * ne bins, the
// node's velocity read once per thread from L1/L2) in a grid-stride loop;
// a node's status is the OR of its bins' flags (__syncthreads_or).
#include <cuda_runtime.h>
#include <math.h>

#include <string>

#include "nmc_internal.h"

namespace nmc {

namespace {

struct C2pArgs {
    long long n;
    int bins;             // ns * ne per node
    const double* N;      // [n][ns][ne]
    const double* G;      // [n][ns][ne][3]
    const double* v;      // [n][3]
    double tol;
    int memory, max_iter;
    double* D;            // [n][ns][ne]
    double* I;            // [n][ns][ne][3]
    int32_t* iters;       // [n][ns][ne] or null
    uint32_t* status;     // [n]
};

// g(M) of Eq. c2p_FP for one bin.  K_ij = a delta_ij + c I_i I_j with Minerbo's psi: for
// h = |I| / D < 1, 3 psi - 1 = (2/5)(3 - h + 3h^2) h^2 gives c = (3 - h + 3h^2) / (5 D), with no
// division by |I|^2 (whose rounding residue would overflow once |I| decays into the denormals)
// and one reciprocal of D; FP64 division and square root are instruction sequences on the FP64
// pipe, which bounds this kernel.  At h >= 1, psi = 1 and c = D / |I|^2; D <= 0 gives K = (D/3) delta.
__device__ __forceinline__ void c2p_map(const double (&M)[4], double N, const double* G, const double* v,
                                        double lam, double (&g)[4]) {
    const double In2 = M[1] * M[1] + M[2] * M[2] + M[3] * M[3];
    double a, c;
    if (!(M[0] > 0.0)) {
        a = M[0] / 3.0;
        c = 0.0;
    } else {
        const double rD = 1.0 / M[0];
        const double h = sqrt(In2) * rD;
        if (h >= 1.0) {
            a = 0.0;
            c = M[0] / In2;
        } else {
            const double p = 3.0 - h + 3.0 * h * h;
            a = 0.5 * (2.0 / 3.0 - (2.0 / 15.0) * p * h * h) * M[0];
            c = 0.2 * p * rD;
        }
    }
    const double vI = v[0] * M[1] + v[1] * M[2] + v[2] * M[3];
    const double ml = 1.0 - lam;
    g[0] = ml * M[0] + lam * (N - vI);
    for (int j = 0; j < 3; ++j) g[1 + j] = ml * M[1 + j] + lam * (G[j] - (a * v[j] + c * vI * M[1 + j]));
}

__device__ __forceinline__ double dot4(const double (&x)[4], const double (&y)[4]) {
    return x[0] * y[0] + x[1] * y[1] + x[2] * y[2] + x[3] * y[3];
}

__global__ void __launch_bounds__(256) c2p_kernel(const C2pArgs a) {
    const int b = threadIdx.x;
    for (long long n = blockIdx.x; n < a.n; n += gridDim.x) {
        int fail = 0;
        if (b < a.bins) {
            const long long o = n * a.bins + b;
            const double v[3] = {a.v[n * 3 + 0], a.v[n * 3 + 1], a.v[n * 3 + 2]};
            const double lam = 1.0 / (1.0 + sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
            const double Nv = a.N[o];
            const double G[3] = {a.G[o * 3 + 0], a.G[o * 3 + 1], a.G[o * 3 + 2]};
            double M[4] = {Nv, G[0], G[1], G[2]};
            // the stopping test ||M_new - M|| <= tol ||U||, squared
            const double ref2 = a.tol * a.tol * (Nv * Nv + G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
            double Fh[3][4], Gh[3][4];   // residual and map-value history, newest last
            for (int j = 0; j < 3; ++j)
                for (int c = 0; c < 4; ++c) { Fh[j][c] = 0.0; Gh[j][c] = 0.0; }
            int k = 0, conv = 0;
            while (k < a.max_iter) {
                ++k;
                double g[4];
                c2p_map(M, Nv, G, v, lam, g);
                for (int j = 0; j < 2; ++j)
                    for (int c = 0; c < 4; ++c) { Fh[j][c] = Fh[j + 1][c]; Gh[j][c] = Gh[j + 1][c]; }
                for (int c = 0; c < 4; ++c) { Fh[2][c] = g[c] - M[c]; Gh[2][c] = g[c]; }
                const int m = k < a.memory ? k : a.memory;
                // coefficients of the window's columns (g0, g1, L = 2): Picard unless the eliminated
                // normal equations are well posed (same tests as the collision solve's least squares)
                double c0 = 0.0, c1 = 0.0, cL = 1.0;
                if (m >= 2) {
                    double d0[4], d1[4];   // F_L - F_g0 (g0 = 0 at m = 3, 1 at m = 2) and F_L - F_1
                    for (int c = 0; c < 4; ++c) {
                        d0[c] = Fh[2][c] - (m == 3 ? Fh[0][c] : Fh[1][c]);
                        d1[c] = Fh[2][c] - Fh[1][c];
                    }
                    const double a00 = dot4(d0, d0), r0 = dot4(d0, Fh[2]);
                    if (m == 2) {
                        if (a00 > 0.0 && isfinite(a00)) {
                            const double gm = r0 / a00;
                            if (isfinite(gm)) { c0 = gm; cL = 1.0 - gm; }
                        }
                    } else {
                        const double a01 = dot4(d0, d1), a11 = dot4(d1, d1), r1 = dot4(d1, Fh[2]);
                        const double dmax = fmax(fabs(a00), fabs(a11));
                        if (dmax > 0.0 && isfinite(dmax)) {
                            const bool sw = fabs(a01) > fabs(a00);
                            const double p0 = sw ? a01 : a00, p1 = sw ? a11 : a01, pr = sw ? r1 : r0;
                            const double q0 = sw ? a00 : a01, q1 = sw ? a01 : a11, qr = sw ? r0 : r1;
                            if (fabs(p0) > 1e-14 * dmax) {
                                const double det = p0 * q1 - q0 * p1;
                                if (fabs(det) > 1e-14 * dmax * fabs(p0)) {
                                    const double rd = 1.0 / det;
                                    const double gm1 = (p0 * qr - q0 * pr) * rd, gm0 = (pr * q1 - p1 * qr) * rd;
                                    if (isfinite(gm0 + gm1)) { c0 = gm0; c1 = gm1; cL = 1.0 - gm0 - gm1; }
                                }
                            }
                        }
                    }
                }
                double Mn[4];
                for (int c = 0; c < 4; ++c) {
                    double acc = cL * Gh[2][c];
                    if (m == 3) acc = fma(c0, Gh[0][c], fma(c1, Gh[1][c], acc));
                    else if (m == 2) acc = fma(c0, Gh[1][c], acc);
                    Mn[c] = acc;
                }
                double d2 = 0.0;
                for (int c = 0; c < 4; ++c) { const double d = Mn[c] - M[c]; d2 += d * d; M[c] = Mn[c]; }
                if (!(isfinite(M[0]) && isfinite(M[1]) && isfinite(M[2]) && isfinite(M[3]))) break;
                if (d2 <= ref2) { conv = 1; break; }
            }
            fail = conv ? 0 : (isfinite(M[0]) && isfinite(M[1]) && isfinite(M[2]) && isfinite(M[3])
                                   ? (int)NMC_NOT_CONVERGED_INNER : (int)NMC_NONFINITE);
            a.D[o] = M[0];
            for (int j = 0; j < 3; ++j) a.I[o * 3 + j] = M[1 + j];
            if (a.iters) a.iters[o] = k;
        }
        const int any_nc = __syncthreads_or(fail & NMC_NOT_CONVERGED_INNER);
        const int any_nf = __syncthreads_or(fail & NMC_NONFINITE);
        if (b == 0) a.status[n] = (any_nc ? NMC_NOT_CONVERGED_INNER : 0u) | (any_nf ? NMC_NONFINITE : 0u);
    }
}

}  // namespace

int launch_c2p(nmc_ctx* ctx, long long n, const double* N, const double* G, const double* v, double tol,
               int memory, int max_iter, double* D, double* I, int32_t* iters, uint32_t* status,
               cudaStream_t stream) {
    C2pArgs a{};
    a.n = n;
    a.bins = ctx->ns * ctx->ne;
    a.N = N; a.G = G; a.v = v;
    a.tol = tol; a.memory = memory; a.max_iter = max_iter;
    a.D = D; a.I = I; a.iters = iters; a.status = status;
    const int threads = ((a.bins + 31) / 32) * 32;
    if (threads > 256) return set_error(ctx, NMC_EUNSUPPORTED, "conserved_to_primitive supports ns * ne <= 256");
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c2p_kernel, threads, 0);
    if (e != cudaSuccess || per_sm < 1) return set_error(ctx, NMC_ECUDA, "c2p kernel cannot be resident");
    long long grid = (long long)per_sm * ctx->num_sms;
    if (grid > n) grid = n;
    c2p_kernel<<<(unsigned)grid, threads, 0, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("c2p kernel launch: ") + cudaGetErrorString(e));
    return NMC_OK;
}

}  // namespace nmc
