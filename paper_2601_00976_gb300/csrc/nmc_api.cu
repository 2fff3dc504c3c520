// C-ABI entry points of libnmc: context set-up (energy grid, quadrature,
// projection operators, table upload), argument checking and dispatch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "nmc_internal.h"

namespace nmc {

int set_error(nmc_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

namespace {

// N-point Gauss--Legendre rule on (-1/2, 1/2) with weights summing to one
// (Sec. 3.2: LG nodes on the unit reference interval).  Newton iteration on
// the Legendre recurrence from the Chebyshev-like initial guesses.
void lg_rule(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = 0.5 * z;                       // ascending order
        w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n == 1) { x[0] = 0.0; w[0] = 1.0; }
}

double lagrange(const std::vector<double>& nodes, int p, double xi) {
    double v = 1.0;
    for (size_t r = 0; r < nodes.size(); ++r)
        if ((int)r != p) v *= (xi - nodes[r]) / (nodes[p] - nodes[r]);
    return v;
}

bool invert_small(std::vector<double>& A, int n) {   // Gauss--Jordan, row-major n x n
    std::vector<double> I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        for (int j = 0; j < n; ++j) { std::swap(A[c * n + j], A[piv * n + j]); std::swap(I[c * n + j], I[piv * n + j]); }
        const double d = A[c * n + c];
        for (int j = 0; j < n; ++j) { A[c * n + j] /= d; I[c * n + j] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r * n + c];
            for (int j = 0; j < n; ++j) { A[r * n + j] -= f * A[c * n + j]; I[r * n + j] -= f * I[c * n + j]; }
        }
    }
    A = I;
    return true;
}

template <typename T>
int upload(nmc_ctx* ctx, const T* host, size_t count, const T** dev) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) return set_error(ctx, NMC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    ctx->allocations.push_back(p);
    e = cudaMemcpy(p, host, count * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    *dev = static_cast<const T*>(p);
    return NMC_OK;
}

int upload_f32(nmc_ctx* ctx, const double* host, size_t count, double scale, const float** dev) {
    std::vector<float> tmp(count);
    for (size_t i = 0; i < count; ++i) tmp[i] = (float)(host[i] * scale);
    return upload(ctx, tmp.data(), count, dev);
}

// The ln table [ns][nye][nt][nrho][ne] regrouped for opacity_interp_mixed: for every
// (rho, E) cell one float4 of its four corners, so that the 16 corner values of a
// point come in four 16-byte loads.
int upload_quads(nmc_ctx* ctx, const double* host, int ns, int nye, int nt, int nr, int ne, const float4** dev) {
    const size_t nrc = (size_t)(nr - 1), nec = (size_t)(ne - 1);
    std::vector<float4> q((size_t)ns * nye * nt * nrc * nec);
    size_t k = 0;
    for (size_t a = 0; a < (size_t)ns * nye * nt; ++a)
        for (size_t ir = 0; ir < nrc; ++ir)
            for (size_t e = 0; e < nec; ++e) {
                const double* r0 = host + (a * nr + ir) * ne + e;
                const double* r1 = r0 + ne;
                q[k++] = make_float4((float)r0[0], (float)r1[0], (float)r0[1], (float)r1[1]);
            }
    return upload(ctx, q.data(), q.size(), dev);
}

Axis make_axis(double lo, double hi, int n) {
    Axis a;
    a.lo = lo;
    a.inv_d = (n - 1) / (hi - lo);
    a.n = n;
    return a;
}

bool axis_ok(double lo, double hi, int n) { return n >= 2 && std::isfinite(lo) && std::isfinite(hi) && hi > lo; }

}  // namespace
}  // namespace nmc

using namespace nmc;

extern "C" {

void nmc_default_params(nmc_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tol_inner = 1e-10;
    p->tol_outer = 1e-10;
    p->m_inner = 3;
    p->m_outer = 3;
    p->max_inner = 500;
    p->max_outer = 100;
    p->precision = NMC_FP64;
    p->mode = NMC_MODE_FUSED;
    p->proc_mask = NMC_PROC_ALL;
    p->frozen_matter = 0;
    p->final_q = 1;
    p->semi_implicit = 0;
    p->d_min = 1e-30;
    p->d_max = 1.0 - 1e-6;
    p->norm_floor = 1e-30;
}

const char* nmc_last_error(const nmc_ctx* ctx) {
    if (!ctx) return "no context";
#ifdef NMC_DEBUG
    unsigned w = 0;
    if (ctx->g.dbg && cudaMemcpy(&w, ctx->g.dbg, sizeof(w), cudaMemcpyDeviceToHost) == cudaSuccess && w != 0)
        const_cast<nmc_ctx*>(ctx)->last_error = "NMC_DEBUG bounds check failed at site " + std::to_string(w);
#endif
    return ctx->last_error.c_str();
}

int nmc_trace_read(nmc_ctx* ctx, uint64_t* cycles, int32_t clear) {
    if (!ctx || !cycles) return NMC_EINVAL;
    for (int i = 0; i < kTraceWords; ++i) cycles[i] = 0;
#ifdef NMC_TRACE
    cudaError_t e = cudaMemcpy(cycles, ctx->g.trace, kTraceWords * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && clear) e = cudaMemset(ctx->g.trace, 0, kTraceWords * sizeof(uint64_t));
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("nmc_trace_read: ") + cudaGetErrorString(e));
    return NMC_OK;
#else
    (void)clear;
    return NMC_EUNSUPPORTED;
#endif
}

int nmc_debug_word(nmc_ctx* ctx, uint32_t* word, int32_t clear) {
    if (!ctx || !word) return NMC_EINVAL;
    *word = 0;
#ifdef NMC_DEBUG
    cudaError_t e = cudaMemcpy(word, ctx->g.dbg, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && clear) e = cudaMemset(ctx->g.dbg, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("nmc_debug_word: ") + cudaGetErrorString(e));
    return NMC_OK;
#else
    (void)clear;
    return NMC_EUNSUPPORTED;
#endif
}

int nmc_geometric_edges(int32_t n_elem, double de1, double emax, double* edges, double* alpha) {
    if (n_elem < 1 || !(de1 > 0.0) || !(emax > 0.0) || !edges || de1 * n_elem > emax) return NMC_EINVAL;
    auto total = [&](double a) { double s = 0.0, t = 1.0; for (int i = 0; i < n_elem; ++i) { s += t; t *= a; } return de1 * s; };
    double lo = 1.0, hi = 4.0;
    if (total(hi) < emax) return NMC_EINVAL;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (total(mid) < emax) lo = mid; else hi = mid;
    }
    const double a = 0.5 * (lo + hi);
    edges[0] = 0.0;
    double wdt = de1;
    for (int i = 0; i < n_elem; ++i) { edges[i + 1] = edges[i] + wdt; wdt *= a; }
    if (alpha) *alpha = a;
    return NMC_OK;
}

int nmc_grid_nodes(const nmc_grid* grid, double* eps, double* w2, double* w3) {
    if (!grid || !grid->edges || grid->n_elem < 1 || grid->n_q < 1 || grid->n_q > kMaxNq) return NMC_EINVAL;
    for (int i = 0; i < grid->n_elem; ++i)
        if (!(grid->edges[i + 1] > grid->edges[i])) return NMC_EINVAL;
    std::vector<double> xi, wq;
    lg_rule(grid->n_q, xi, wq);
    const double hc3 = kHC * kHC * kHC;
    for (int el = 0; el < grid->n_elem; ++el) {
        const double c = 0.5 * (grid->edges[el] + grid->edges[el + 1]);
        const double h = grid->edges[el + 1] - grid->edges[el];
        for (int k = 0; k < grid->n_q; ++k) {
            const int q = el * grid->n_q + k;
            const double ep = c + h * xi[k];
            const double v2 = 4.0 * kPi * wq[k] * ep * ep * h / hc3;
            if (eps) eps[q] = ep;
            if (w2) w2[q] = v2;
            if (w3) w3[q] = v2 * ep;
        }
    }
    return NMC_OK;
}

int nmc_create(const nmc_grid* grid, const nmc_tables* tb, nmc_ctx** out) {
    if (!out) return NMC_EINVAL;
    *out = nullptr;
    if (!grid || !tb || !grid->edges) return NMC_EINVAL;
    const int n_elem = grid->n_elem, nq = grid->n_q, ns = grid->n_species;
    if (n_elem < 1 || nq < 1 || nq > kMaxNq || ns < 2 || ns > kMaxSpecies || (ns & 1)) return NMC_EINVAL;
    const int ne = n_elem * nq;
    if (ne > kMaxNe || ne < 2) return NMC_EUNSUPPORTED;
    for (int i = 0; i < n_elem; ++i)
        if (!(grid->edges[i + 1] > grid->edges[i]) || !std::isfinite(grid->edges[i + 1])) return NMC_EINVAL;
    if (!(grid->edges[0] >= 0.0)) return NMC_EINVAL;
    if (!tb->emab || !tb->iso || !tb->nes || !tb->pair) return NMC_EINVAL;
    if ((tb->nes1 == nullptr) != (tb->pair1 == nullptr)) return NMC_EINVAL;
    if (!axis_ok(tb->lrho_min, tb->lrho_max, tb->n_rho) || !axis_ok(tb->lt_min, tb->lt_max, tb->n_t) ||
        !axis_ok(tb->ye_min, tb->ye_max, tb->n_ye) || !axis_ok(tb->klt_min, tb->klt_max, tb->n_kt) ||
        !axis_ok(tb->eta_min, tb->eta_max, tb->n_eta))
        return NMC_EINVAL;

    nmc_ctx* ctx = new (std::nothrow) nmc_ctx();
    if (!ctx) return NMC_ENOMEM;
    ctx->n_elem = n_elem;
    ctx->nq = nq;
    ctx->ns = ns;
    ctx->ne = ne;
    int nep = 1;
    if (ne <= 32) { while (nep < ne) nep <<= 1; } else { nep = ((ne + 31) / 32) * 32; }
    ctx->nep = nep;
    if (ns * nep > 1024) { delete ctx; return NMC_EUNSUPPORTED; }

    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if (e != cudaSuccess) { delete ctx; return NMC_ECUDA; }

    // ---- energy grid and weights (Eq. energy_integration_weights) ----
    std::vector<double> xi, wq, xg, wg;
    lg_rule(nq, xi, wq);
    lg_rule(kProjQuad, xg, wg);
    ctx->edges.assign(grid->edges, grid->edges + n_elem + 1);
    ctx->eps.resize(ne);
    ctx->w2.resize(ne);
    ctx->w3.resize(ne);
    std::vector<double> lneps(ne);
    double sum_w2 = 0.0;
    const double hc3 = kHC * kHC * kHC;
    for (int el = 0; el < n_elem; ++el) {
        const double c = 0.5 * (ctx->edges[el] + ctx->edges[el + 1]);
        const double h = ctx->edges[el + 1] - ctx->edges[el];
        for (int k = 0; k < nq; ++k) {
            const int q = el * nq + k;
            const double ep = c + h * xi[k];
            ctx->eps[q] = ep;
            ctx->w2[q] = 4.0 * kPi * wq[k] * ep * ep * h / hc3;
            ctx->w3[q] = ctx->w2[q] * ep;
            lneps[q] = std::log(ep);
            sum_w2 += ctx->w2[q];
        }
    }
    // ---- projection operators of Eq. fermiDiracProjection per element ----
    const int Q = kProjQuad;
    std::vector<double> pe(n_elem * Q), pc(n_elem * nq * Q), pa(n_elem * Q);
    for (int el = 0; el < n_elem; ++el) {
        const double c = 0.5 * (ctx->edges[el] + ctx->edges[el + 1]);
        const double h = ctx->edges[el + 1] - ctx->edges[el];
        std::vector<double> wt(Q), L(nq * Q);
        double swt = 0.0;
        for (int gq = 0; gq < Q; ++gq) {
            const double eg = c + h * xg[gq];
            pe[el * Q + gq] = eg;
            wt[gq] = wg[gq] * eg * eg * h;          // eps^2 d eps
            swt += wt[gq];
            for (int p = 0; p < nq; ++p) L[p * Q + gq] = lagrange(xi, p, xg[gq]);
        }
        std::vector<double> M(nq * nq, 0.0);
        for (int p = 0; p < nq; ++p)
            for (int r = 0; r < nq; ++r)
                for (int gq = 0; gq < Q; ++gq) M[p * nq + r] += wt[gq] * L[p * Q + gq] * L[r * Q + gq];
        if (!invert_small(M, nq)) { delete ctx; return NMC_EINVAL; }
        for (int p = 0; p < nq; ++p)
            for (int gq = 0; gq < Q; ++gq) {
                double v = 0.0;
                for (int r = 0; r < nq; ++r) v += M[p * nq + r] * wt[gq] * L[r * Q + gq];
                pc[(el * nq + p) * Q + gq] = v;
            }
        for (int gq = 0; gq < Q; ++gq) pa[el * Q + gq] = wt[gq] / swt;
    }
    DevGrid& g = ctx->g;
    g.ns = ns;
    g.ne = ne;
    g.nep = nep;
    g.n_elem = n_elem;
    g.nq = nq;
    g.ld = ne + 1;
    g.sum_w2 = sum_w2;
    for (int p = 0; p < kMaxNq; ++p) {
        g.ends[0][p] = p < nq ? lagrange(xi, p, -0.5) : 0.0;
        g.ends[1][p] = p < nq ? lagrange(xi, p, 0.5) : 0.0;
    }
    std::vector<double> wt(ne);
    double sum_wt = 0.0;
    for (int q = 0; q < ne; ++q) { wt[q] = ctx->w2[q] / kCW; sum_wt += wt[q]; }
    g.sum_wt = sum_wt;
    int rc = NMC_OK;
    if (rc == NMC_OK) rc = upload(ctx, ctx->eps.data(), ne, &g.eps);
    if (rc == NMC_OK) rc = upload(ctx, wt.data(), ne, &g.wt);
    if (rc == NMC_OK) rc = upload_f32(ctx, wt.data(), ne, 1.0, &g.wt_f);
    if (rc == NMC_OK) rc = upload_f32(ctx, pe.data(), pe.size(), 1.0, &g.proj_e_f);
    if (rc == NMC_OK) {
        std::vector<double> lo(pe.size());
        for (size_t i = 0; i < pe.size(); ++i) lo[i] = pe[i] - (double)(float)pe[i];
        rc = upload_f32(ctx, lo.data(), lo.size(), 1.0, &g.proj_e_fl);
    }
    if (rc == NMC_OK) rc = upload_f32(ctx, pc.data(), pc.size(), 1.0, &g.proj_c_f);
    if (rc == NMC_OK) rc = upload_f32(ctx, pa.data(), pa.size(), 1.0, &g.proj_a_f);
    if (rc == NMC_OK) rc = upload(ctx, ctx->w2.data(), ne, &g.w2);
    if (rc == NMC_OK) rc = upload(ctx, ctx->w3.data(), ne, &g.w3);
    if (rc == NMC_OK) rc = upload(ctx, lneps.data(), ne, &g.lneps);
    if (rc == NMC_OK) rc = upload(ctx, pe.data(), pe.size(), &g.proj_e);
    if (rc == NMC_OK) rc = upload(ctx, pc.data(), pc.size(), &g.proj_c);
    if (rc == NMC_OK) rc = upload(ctx, pa.data(), pa.size(), &g.proj_a);

    // ---- tables ----
    DevTables& t = ctx->tb;
    t.rho = make_axis(tb->lrho_min, tb->lrho_max, tb->n_rho);
    t.t = make_axis(tb->lt_min, tb->lt_max, tb->n_t);
    t.ye = make_axis(tb->ye_min, tb->ye_max, tb->n_ye);
    t.kt = make_axis(tb->klt_min, tb->klt_max, tb->n_kt);
    t.eta = make_axis(tb->eta_min, tb->eta_max, tb->n_eta);
    const size_t n_op = (size_t)ns * tb->n_ye * tb->n_t * tb->n_rho * ne;
    const size_t n_nes = (size_t)ns * tb->n_kt * tb->n_eta * ne * ne;
    const size_t n_pair = (size_t)(ns / 2) * tb->n_kt * tb->n_eta * ne * ne;
    t.n_op = (long long)n_op;
    t.n_nes = (long long)n_nes;
    t.n_pair = (long long)n_pair;
    if (rc == NMC_OK) rc = upload(ctx, tb->emab, n_op, &t.emab);
    if (rc == NMC_OK) rc = upload(ctx, tb->iso, n_op, &t.iso);
    if (rc == NMC_OK) rc = upload(ctx, tb->nes, n_nes, &t.nes);
    if (rc == NMC_OK) rc = upload(ctx, tb->pair, n_pair, &t.pair);
    // linear-order kernels (optional, both or neither; read by the O(v/c) solve)
    t.nes1 = nullptr;
    t.pair1 = nullptr;
    if (rc == NMC_OK && tb->nes1 && tb->pair1) {
        rc = upload(ctx, tb->nes1, n_nes, &t.nes1);
        if (rc == NMC_OK) rc = upload(ctx, tb->pair1, n_pair, &t.pair1);
    }
    // FP32 copies for the mixed path; kernel tables prescaled by 4 pi / (hc)^3
    if (rc == NMC_OK) rc = upload_f32(ctx, tb->emab, n_op, 1.0, &t.emab_f);
    if (rc == NMC_OK) rc = upload_f32(ctx, tb->iso, n_op, 1.0, &t.iso_f);
    if (rc == NMC_OK) rc = upload_quads(ctx, tb->emab, ns, tb->n_ye, tb->n_t, tb->n_rho, ne, &t.emab_q);
    if (rc == NMC_OK) rc = upload_quads(ctx, tb->iso, ns, tb->n_ye, tb->n_t, tb->n_rho, ne, &t.iso_q);
    t.n_quad = (long long)ns * tb->n_ye * tb->n_t * (tb->n_rho - 1) * (ne - 1);
    if (rc == NMC_OK) rc = upload_f32(ctx, tb->nes, n_nes, kCW, &t.nes_f);
    if (rc == NMC_OK) rc = upload_f32(ctx, tb->pair, n_pair, kCW, &t.pair_f);
    if (rc == NMC_OK) {
        void* p = nullptr;
        e = cudaMalloc(&p, 256);
        if (e != cudaSuccess) rc = NMC_ENOMEM;
        else { ctx->allocations.push_back(p); ctx->queue = static_cast<int*>(p); }
    }
#ifdef NMC_DEBUG
    if (rc == NMC_OK) {   // the bounds-check error word, cleared
        void* p = nullptr;
        e = cudaMalloc(&p, 256);
        if (e == cudaSuccess) e = cudaMemset(p, 0, 256);
        if (e != cudaSuccess) rc = NMC_ENOMEM;
        else { ctx->allocations.push_back(p); ctx->g.dbg = static_cast<unsigned*>(p); }
    }
#endif
#ifdef NMC_TRACE
    if (rc == NMC_OK) {   // the stage counters, cleared
        void* p = nullptr;
        e = cudaMalloc(&p, kTraceWords * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(p, 0, kTraceWords * sizeof(unsigned long long));
        if (e != cudaSuccess) rc = NMC_ENOMEM;
        else { ctx->allocations.push_back(p); ctx->g.trace = static_cast<unsigned long long*>(p); }
    }
#endif
    // Set-up of collision_solve_noalloc, done here because this call may allocate: load the fused
    // kernel's variants (lazy module loading would load them at their first launch) and look up the
    // device address of the no-allocation scratch array for this device.
    if (rc == NMC_OK) {
        e = preload_fused_f64_m3();
        if (e == cudaSuccess) e = preload_fused_f64_m5();
        if (e == cudaSuccess) e = preload_fused_f32_m3();
        if (e == cudaSuccess) e = preload_fused_f32_m5();
        if (e != cudaSuccess) rc = NMC_ECUDA;
    }
    if (rc == NMC_OK) {
        int* scratch = nullptr;
        rc = noalloc_scratch_address(ctx, &scratch);
    }
    if (rc != NMC_OK) { nmc_destroy(ctx); return rc; }
    *out = ctx;
    return NMC_OK;
}

void nmc_destroy(nmc_ctx* ctx) {
    if (!ctx) return;
    for (void* p : ctx->allocations) cudaFree(p);
    if (ctx->plain_scratch) cudaFree(ctx->plain_scratch);
    if (ctx->plain_counts_host) cudaFreeHost(ctx->plain_counts_host);
    host_pipe_release(ctx);
    delete ctx;
}

int nmc_energy_nodes(const nmc_ctx* ctx, double* eps, double* w2, double* w3, int32_t* ne) {
    if (!ctx) return NMC_EINVAL;
    if (ne) *ne = ctx->ne;
    for (int q = 0; q < ctx->ne; ++q) {
        if (eps) eps[q] = ctx->eps[q];
        if (w2) w2[q] = ctx->w2[q];
        if (w3) w3[q] = ctx->w3[q];
    }
    return NMC_OK;
}

int nmc_check_params_internal(nmc_ctx* ctx, const nmc_params* p) {
    if (!p) return set_error(ctx, NMC_EINVAL, "params is NULL");
    if (!(p->tol_inner > 0.0) || !(p->tol_outer > 0.0) || !std::isfinite(p->tol_inner) || !std::isfinite(p->tol_outer))
        return set_error(ctx, NMC_EINVAL, "tolerances must be positive and finite");
    if (p->m_inner < 1 || p->m_inner > 5 || p->m_outer < 1 || p->m_outer > kMaxOuterMem)
        return set_error(ctx, NMC_EINVAL, "Anderson memory must be in 1..5");
    if (p->max_inner < 1 || p->max_outer < 1) return set_error(ctx, NMC_EINVAL, "iteration caps must be >= 1");
    if (p->precision != NMC_FP64 && p->precision != NMC_MIXED) return set_error(ctx, NMC_EINVAL, "unknown precision");
    // the mixed path is validated for constant and linear elements; with quadratic ones it missed the
    // heavy flavours' fixed point at a profile node, so it is refused until that is understood
    if (p->precision == NMC_MIXED && ctx->nq > 2)
        return set_error(ctx, NMC_EUNSUPPORTED, "the mixed-precision path supports n_q <= 2 nodes per element");
    if (p->mode != NMC_MODE_FUSED && p->mode != NMC_MODE_PLAIN) return set_error(ctx, NMC_EINVAL, "unknown mode");
    if (p->proc_mask < 0 || p->proc_mask > NMC_PROC_ALL) return set_error(ctx, NMC_EINVAL, "bad process mask");
    if (!(p->d_min > 0.0) || !(p->d_max < 1.0) || !(p->d_min < p->d_max))
        return set_error(ctx, NMC_EINVAL, "need 0 < d_min < d_max < 1");
    if (!(p->norm_floor >= 0.0)) return set_error(ctx, NMC_EINVAL, "norm_floor must be >= 0");
    if (p->semi_implicit != 0 && p->semi_implicit != 1) return set_error(ctx, NMC_EINVAL, "semi_implicit must be 0 or 1");
    return NMC_OK;
}

int collision_solve(nmc_ctx* ctx, const nmc_params* params, int64_t n, const double* rho,
                    const double* T_in, const double* Ye_in, const double* J_in, const double* H_in,
                    const double* dt, const double* opac_scale, double* J_out, double* H_out,
                    double* Ye_out, double* eps_out, double* T_out, int32_t* n_outer,
                    int32_t* n_inner, uint32_t* status, void* stream) {
    if (!ctx) return NMC_EINVAL;
    int rc = nmc_check_params_internal(ctx, params);
    if (rc != NMC_OK) return rc;
    if (n < 0) return set_error(ctx, NMC_EINVAL, "n < 0");
    if (n > (int64_t(1) << 30)) return set_error(ctx, NMC_EUNSUPPORTED, "n > 2^30 nodes per call");
    if (n == 0) return NMC_OK;
    if (!rho || !T_in || !Ye_in || !J_in || !H_in || !dt || !J_out || !H_out || !Ye_out || !eps_out ||
        !T_out || !n_outer || !n_inner || !status)
        return set_error(ctx, NMC_EINVAL, "null array argument");
    SolveArgs a{};
    a.g = ctx->g;
    a.tb = ctx->tb;
    a.p = *params;
    a.n = n;
    a.rho = rho; a.T = T_in; a.Ye = Ye_in; a.J = J_in; a.H = H_in; a.dt = dt; a.scale = opac_scale;
    a.J_out = J_out; a.H_out = H_out; a.Ye_out = Ye_out; a.eps_out = eps_out; a.T_out = T_out;
    a.n_outer = n_outer; a.n_inner = n_inner; a.status = status;
    a.queue = ctx->queue;
    if (params->mode == NMC_MODE_PLAIN) return launch_plain(ctx, a, static_cast<cudaStream_t>(stream));
    return launch_fused(ctx, a, static_cast<cudaStream_t>(stream));
}

int collision_solve_v(nmc_ctx* ctx, const nmc_params* params, int64_t n, const double* rho,
                      const double* T_in, const double* Ye_in, const double* v_in, const double* J_in,
                      const double* H_in, const double* dt, const double* opac_scale, int32_t freeze_velocity,
                      double v_floor, double* J_out, double* H_out, double* v_out, double* Ye_out,
                      double* eps_out, double* T_out, int32_t* n_outer, int32_t* n_inner, uint32_t* status,
                      void* stream) {
    if (!ctx) return NMC_EINVAL;
    int rc = nmc_check_params_internal(ctx, params);
    if (rc != NMC_OK) return rc;
    if (n < 0) return set_error(ctx, NMC_EINVAL, "n < 0");
    if (n > (int64_t(1) << 30)) return set_error(ctx, NMC_EUNSUPPORTED, "n > 2^30 nodes per call");
    if (!(v_floor > 0.0) || !std::isfinite(v_floor)) return set_error(ctx, NMC_EINVAL, "v_floor must be > 0");
    if (params->mode != NMC_MODE_FUSED) return set_error(ctx, NMC_EUNSUPPORTED, "the O(v/c) solve runs fused");
    if (n == 0) return NMC_OK;
    if (!rho || !T_in || !Ye_in || !v_in || !J_in || !H_in || !dt || !J_out || !H_out || !v_out || !Ye_out ||
        !eps_out || !T_out || !n_outer || !n_inner || !status)
        return set_error(ctx, NMC_EINVAL, "null array argument");
    SolveArgs a{};
    a.g = ctx->g;
    a.tb = ctx->tb;
    a.p = *params;
    a.n = n;
    a.rho = rho; a.T = T_in; a.Ye = Ye_in; a.J = J_in; a.H = H_in; a.dt = dt; a.scale = opac_scale;
    a.J_out = J_out; a.H_out = H_out; a.Ye_out = Ye_out; a.eps_out = eps_out; a.T_out = T_out;
    a.n_outer = n_outer; a.n_inner = n_inner; a.status = status;
    a.queue = ctx->queue;
    return launch_velocity(ctx, a, v_in, v_out, freeze_velocity ? 1 : 0, v_floor, static_cast<cudaStream_t>(stream));
}

int conserved_to_primitive(nmc_ctx* ctx, int64_t n, const double* N_in, const double* G_in, const double* v,
                           double tol, int32_t memory, int32_t max_iter, double* D_out, double* I_out,
                           int32_t* iters, uint32_t* status, void* stream) {
    if (!ctx) return NMC_EINVAL;
    if (n < 0) return set_error(ctx, NMC_EINVAL, "n < 0");
    if (n > (int64_t(1) << 30)) return set_error(ctx, NMC_EUNSUPPORTED, "n > 2^30 nodes per call");
    if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(ctx, NMC_EINVAL, "tol must be > 0");
    if (memory < 1 || memory > 3) return set_error(ctx, NMC_EINVAL, "memory must be 1..3");
    if (max_iter < 1) return set_error(ctx, NMC_EINVAL, "max_iter must be >= 1");
    if (n == 0) return NMC_OK;
    if (!N_in || !G_in || !v || !D_out || !I_out || !status) return set_error(ctx, NMC_EINVAL, "null array argument");
    return launch_c2p(ctx, n, N_in, G_in, v, tol, memory, max_iter, D_out, I_out, iters, status,
                      static_cast<cudaStream_t>(stream));
}

int nmc_autotune(nmc_ctx* ctx, const nmc_params* params, int64_t n, const double* rho, const double* T_in,
                 const double* Ye_in, const double* J_in, const double* H_in, const double* dt,
                 const double* opac_scale, double* J_out, double* H_out, double* Ye_out, double* eps_out,
                 double* T_out, int32_t* n_outer, int32_t* n_inner, uint32_t* status, int32_t* chosen,
                 float* ms, void* stream) {
    if (!ctx) return NMC_EINVAL;
    int rc = nmc_check_params_internal(ctx, params);
    if (rc != NMC_OK) return rc;
    if (params->mode != NMC_MODE_FUSED) return set_error(ctx, NMC_EINVAL, "autotuning applies to the fused mode");
    if (n < 1 || n > (int64_t(1) << 30)) return set_error(ctx, NMC_EINVAL, "autotune needs 1 <= n <= 2^30 nodes");
    if (!rho || !T_in || !Ye_in || !J_in || !H_in || !dt || !J_out || !H_out || !Ye_out || !eps_out ||
        !T_out || !n_outer || !n_inner || !status)
        return set_error(ctx, NMC_EINVAL, "null array argument");
    SolveArgs a{};
    a.g = ctx->g;
    a.tb = ctx->tb;
    a.p = *params;
    a.n = n;
    a.rho = rho; a.T = T_in; a.Ye = Ye_in; a.J = J_in; a.H = H_in; a.dt = dt; a.scale = opac_scale;
    a.J_out = J_out; a.H_out = H_out; a.Ye_out = Ye_out; a.eps_out = eps_out; a.T_out = T_out;
    a.n_outer = n_outer; a.n_inner = n_inner; a.status = status;
    a.queue = ctx->queue;
    return autotune_fused(ctx, a, static_cast<cudaStream_t>(stream), chosen, ms);
}

int nmc_set_plain_chunk(nmc_ctx* ctx, int64_t nodes) {
    if (!ctx) return NMC_EINVAL;
    if (nodes < 1 || nodes > (int64_t(1) << 30)) return set_error(ctx, NMC_EINVAL, "plain chunk must be in 1..2^30");
    ctx->plain_chunk = nodes;
    return NMC_OK;
}

int opacity_interp(nmc_ctx* ctx, int32_t which, int32_t species, int64_t p, const double* rho,
                   const double* T, const double* Ye, const double* E, double* out, void* stream) {
    if (!ctx) return NMC_EINVAL;
    if (which != 0 && which != 1) return set_error(ctx, NMC_EINVAL, "which must be 0 (EmAb) or 1 (Iso)");
    if (species < 0 || species >= ctx->ns) return set_error(ctx, NMC_EINVAL, "species out of range");
    if (p < 0) return set_error(ctx, NMC_EINVAL, "p < 0");
    if (p == 0) return NMC_OK;
    if (!rho || !T || !Ye || !E || !out) return set_error(ctx, NMC_EINVAL, "null array argument");
    return launch_opacity_interp(ctx, which, species, p, rho, T, Ye, E, out, static_cast<cudaStream_t>(stream));
}

int opacity_interp_mixed(nmc_ctx* ctx, int32_t which, int32_t species, int64_t p, const double* rho,
                         const double* T, const double* Ye, const double* E, double* out, void* stream) {
    if (!ctx) return NMC_EINVAL;
    if (which != 0 && which != 1) return set_error(ctx, NMC_EINVAL, "which must be 0 (EmAb) or 1 (Iso)");
    if (species < 0 || species >= ctx->ns) return set_error(ctx, NMC_EINVAL, "species out of range");
    if (p < 0) return set_error(ctx, NMC_EINVAL, "p < 0");
    if (p == 0) return NMC_OK;
    if (!rho || !T || !Ye || !E || !out) return set_error(ctx, NMC_EINVAL, "null array argument");
    return launch_opacity_interp_mixed(ctx, which, species, p, rho, T, Ye, E, out, static_cast<cudaStream_t>(stream));
}

int collision_adjoint(nmc_ctx* ctx, const nmc_params* params, int64_t n, const double* rho,
                      const double* T_in, const double* Ye_in, const double* J_in, const double* H_in,
                      const double* dt, const double* opac_scale, const double* J_out, const double* T_out,
                      const double* gJ_out, const double* gH_out, const double* gYe_out,
                      const double* geps_out, const double* gT_out, double* gJ_in, double* gH_in,
                      double* gYe_in, double* gT_in, double* gscale, uint32_t* status, void* stream) {
    if (!ctx) return NMC_EINVAL;
    int rc = nmc_check_params_internal(ctx, params);
    if (rc != NMC_OK) return rc;
    if (params->semi_implicit)
        return set_error(ctx, NMC_EUNSUPPORTED, "collision_adjoint differentiates the fully implicit solve only");
    if (n < 0) return set_error(ctx, NMC_EINVAL, "n < 0");
    if (n == 0) return NMC_OK;
    if (!rho || !T_in || !Ye_in || !J_in || !dt || !J_out || !gJ_in || !gYe_in || !gT_in)
        return set_error(ctx, NMC_EINVAL, "null array argument");
    if (gH_out && !H_in) return set_error(ctx, NMC_EINVAL, "gH_out needs H_in");
    AdjointArgs a{};
    a.g = ctx->g;
    a.tb = ctx->tb;
    a.p = *params;
    a.n = n;
    a.rho = rho; a.T = T_in; a.Ye = Ye_in; a.J = J_in; a.H = H_in; a.dt = dt; a.scale = opac_scale;
    a.J_out = J_out; a.T_out = T_out;
    a.gJ = gJ_out; a.gH = gH_out; a.gYe = gYe_out; a.geps = geps_out; a.gT = gT_out;
    a.gJ_in = gJ_in; a.gH_in = gH_in; a.gYe_in = gYe_in; a.gT_in = gT_in; a.gscale = gscale;
    a.status = status;
    a.fd_rel = 1e-6;
    return launch_adjoint(ctx, a, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
