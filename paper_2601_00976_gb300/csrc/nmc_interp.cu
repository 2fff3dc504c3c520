// opacity_interp: tetralinear interpolation of the EmAb / Iso log tables at
// arbitrary points (Sec. 2.3, tetralinear interpolation of chi_EmAb and the
// isoenergetic kernels).  One thread per point: uniform axes in
// (log10 rho, log10 T, Ye) give the cell directly, the energy axis (the node
// energies of the grid) is searched by bisection in ln E; the 16 corner ln
// values are combined with the tensor-product weights and exponentiated.
//
// opacity_interp_mixed: the same interpolation in FP32 on FP32 copies of the
// ln tables: FP32 logarithms, cell search and weights, the ln value as the
// first corner plus weighted differences (the corners are ~ -20, whose FP32
// sum would round ln chi by ~2e-6 in steps), and an FP32 exp; inputs and
// outputs stay FP64.  The energy axis is searched in a shared-memory copy of
// ln eps.  The table copy is regrouped per (rho, E) cell, four corners to a
// float4, so a point's 16 corner values take four 16-byte loads (four L2
// sectors) rather than sixteen scattered words.
#include <cuda_runtime.h>
#include <math.h>

#include "nmc_internal.h"

namespace nmc {

namespace {

__device__ __forceinline__ void cell(double v, const Axis& ax, int* i, double* t) {
    double x = (v - ax.lo) * ax.inv_d;
    if (!(x >= 0.0)) x = 0.0;
    if (x > ax.n - 1) x = ax.n - 1;
    int c = (int)floor(x);
    if (c > ax.n - 2) c = ax.n - 2;
    *i = c;
    *t = x - c;
}

__global__ void opacity_interp_kernel(const DevGrid g, const DevTables tb, int which, int species,
                                      long long p, const double* __restrict__ rho,
                                      const double* __restrict__ T, const double* __restrict__ Ye,
                                      const double* __restrict__ E, double* __restrict__ out) {
    const double* tab = which == 0 ? tb.emab : tb.iso;
    const int NE = g.ne;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p; i += (long long)gridDim.x * blockDim.x) {
        int ir, it, iy;
        double tr, tt, ty;
        cell(log10(rho[i]), tb.rho, &ir, &tr);
        cell(log10(T[i]), tb.t, &it, &tt);
        cell(Ye[i], tb.ye, &iy, &ty);
        // energy: ln E clamped to [ln eps_0, ln eps_{ne-1}], bisection for the cell
        double le = log(E[i]);
        if (!(le >= g.lneps[0])) le = g.lneps[0];
        if (le > g.lneps[NE - 1]) le = g.lneps[NE - 1];
        int lo = 0, hi = NE - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (g.lneps[mid] <= le) lo = mid; else hi = mid;
        }
        const double te = (le - g.lneps[lo]) / (g.lneps[lo + 1] - g.lneps[lo]);
        const long long base = ((((long long)species * tb.ye.n + iy) * tb.t.n + it) * tb.rho.n + ir) * NE + lo;
        const long long dR = NE, dT = (long long)tb.rho.n * NE, dY = (long long)tb.t.n * tb.rho.n * NE;
        if (!NMC_IN_BOUNDS(g.dbg, base, tb.n_op, kDbgEmabIso) ||
            !NMC_IN_BOUNDS(g.dbg, base + dR + dT + dY + 1, tb.n_op, kDbgEmabIso))
            continue;
        double v = 0.0;
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            const int ca = c8 & 1, cb = (c8 >> 1) & 1, cc = c8 >> 2;
            const double w = (ca ? tr : 1.0 - tr) * (cb ? tt : 1.0 - tt) * (cc ? ty : 1.0 - ty);
            const long long o = base + ca * dR + cb * dT + cc * dY;
            v += w * ((1.0 - te) * tab[o] + te * tab[o + 1]);
        }
        out[i] = exp(v);
    }
}

__device__ __forceinline__ void cell_f(float v, const Axis& ax, int* i, float* t) {
    float x = (v - (float)ax.lo) * (float)ax.inv_d;
    if (!(x >= 0.0f)) x = 0.0f;
    if (x > (float)(ax.n - 1)) x = (float)(ax.n - 1);
    int c = (int)floorf(x);
    if (c > ax.n - 2) c = ax.n - 2;
    *i = c;
    *t = x - (float)c;
}

__global__ void __launch_bounds__(256) opacity_interp_mixed_kernel(const DevGrid g, const DevTables tb, int which,
                                                                   int species, long long p,
                                                                   const double* __restrict__ rho,
                                                                   const double* __restrict__ T,
                                                                   const double* __restrict__ Ye,
                                                                   const double* __restrict__ E,
                                                                   double* __restrict__ out) {
    __shared__ float lne[kMaxNe];
    const int NE = g.ne;
    for (int q = threadIdx.x; q < NE; q += blockDim.x) lne[q] = (float)g.lneps[q];
    __syncthreads();
    const float4* __restrict__ tab = which == 0 ? tb.emab_q : tb.iso_q;
    const long long nrc = tb.rho.n - 1, nec = NE - 1;
    const long long dT = nrc * nec, dY = (long long)tb.t.n * nrc * nec;
    const long long sp0 = (long long)species * tb.ye.n;
    const float lo_e = lne[0], hi_e = lne[NE - 1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p; i += (long long)gridDim.x * blockDim.x) {
        int ir, it, iy;
        float tr, tt, ty;
        cell_f(log10f((float)rho[i]), tb.rho, &ir, &tr);
        cell_f(log10f((float)T[i]), tb.t, &it, &tt);
        cell_f((float)Ye[i], tb.ye, &iy, &ty);
        float le = logf((float)E[i]);
        if (!(le >= lo_e)) le = lo_e;
        if (le > hi_e) le = hi_e;
        int lo = 0, hi = NE - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (lne[mid] <= le) lo = mid; else hi = mid;
        }
        const float te = (le - lne[lo]) / (lne[lo + 1] - lne[lo]);
        // the (rho, E) cell's four corners per load: (T, Ye) corners k = cb + 2 cc
        const long long base = (((sp0 + iy) * tb.t.n + it) * nrc + ir) * nec + lo;
        if (!NMC_IN_BOUNDS(g.dbg, base, tb.n_quad, kDbgEmabIso) ||
            !NMC_IN_BOUNDS(g.dbg, base + dT + dY, tb.n_quad, kDbgEmabIso))
            continue;
        float4 c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = __ldg(tab + base + (k & 1) * dT + (k >> 1) * dY);
        const float c0 = c[0].x;
        float v = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float wk = ((k & 1) ? tt : 1.0f - tt) * ((k >> 1) ? ty : 1.0f - ty);
            // rho_i and rho_i+1, each linear in ln E between the two energy nodes
            const float a0 = fmaf(te, c[k].z - c[k].x, c[k].x - c0);
            const float a1 = fmaf(te, c[k].w - c[k].y, c[k].y - c0);
            v = fmaf(wk, fmaf(tr, a1 - a0, a0), v);
        }
        out[i] = (double)expf(c0 + v);
    }
}

}  // namespace

int launch_opacity_interp_mixed(nmc_ctx* ctx, int which, int species, long long p, const double* rho,
                                const double* T, const double* Ye, const double* E, double* out,
                                cudaStream_t stream) {
    const int threads = 256;
    long long blocks = (p + threads - 1) / threads;
    const long long cap = (long long)ctx->num_sms * 8;
    if (blocks > cap) blocks = cap;
    opacity_interp_mixed_kernel<<<(unsigned)blocks, threads, 0, stream>>>(ctx->g, ctx->tb, which, species, p, rho, T,
                                                                          Ye, E, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(ctx, NMC_ECUDA, std::string("opacity_interp_mixed launch: ") + cudaGetErrorString(e));
    return NMC_OK;
}

int launch_opacity_interp(nmc_ctx* ctx, int which, int species, long long p, const double* rho,
                          const double* T, const double* Ye, const double* E, double* out,
                          cudaStream_t stream) {
    const int threads = 256;
    long long blocks = (p + threads - 1) / threads;
    const long long cap = (long long)ctx->num_sms * 8;
    if (blocks > cap) blocks = cap;
    opacity_interp_kernel<<<(unsigned)blocks, threads, 0, stream>>>(ctx->g, ctx->tb, which, species, p, rho, T, Ye, E, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("opacity_interp launch: ") + cudaGetErrorString(e));
    return NMC_OK;
}

}  // namespace nmc
