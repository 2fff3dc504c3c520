// collision_solve_host: collision_solve on HOST buffers, with the copies
// pipelined against the solve.
//
// The batch is cut into chunks.  Chunk i is staged through device slot i % 2:
// its inputs go up on an upload stream, it is solved on the caller's stream,
// and its outputs come down on a download stream, so that the upload of chunk
// i + 1 and the download of chunk i - 1 run while chunk i is solved.  Events
// order the three streams: an upload into a slot waits until the solve two
// chunks back has finished reading it, a solve waits for its upload and for
// the download two chunks back to have emptied its output slot, a download
// waits for its solve.  All solves run on the caller's stream, one after the
// other (the persistent kernel's work-queue counter is per context).  At the
// end the caller's stream waits for the last downloads, so the call is
// stream-ordered like collision_solve: the host outputs are complete once the
// caller's stream is.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "nmc_internal.h"

namespace nmc {
namespace {

// Device staging for two chunks of `chunk` nodes, the two side streams and the
// per-slot events; kept in the context and grown on demand.
int ensure_staging(nmc_ctx* ctx, long long chunk) {
    HostPipe& hp = ctx->host_pipe;
    if (!hp.up) {
        cudaError_t e = cudaStreamCreateWithFlags(&hp.up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp.down, cudaStreamNonBlocking);
        for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
            e = cudaEventCreateWithFlags(&hp.uploaded[s], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.solved[s], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.downloaded[s], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("collision_solve_host set-up: ") +
                                                                  cudaGetErrorString(e));
    }
    if (chunk <= hp.chunk) return NMC_OK;
    const size_t nsne = (size_t)ctx->ns * ctx->ne;
    // per node: rho, T, Ye, dt, scale[4] in; J, H in; J, H, Ye, eps, T out; n_outer, n_inner, status
    const size_t per_node = 8 * (4 + 4) + 2 * 8 * nsne * 4 + 8 * 3 + 4 * 3;
    // two slots of 15 arrays, each rounded up to 256 bytes
    const size_t bytes = 2 * (per_node * (size_t)chunk + 15 * 256);
    if (hp.buf) cudaFree(hp.buf);
    hp.buf = nullptr;
    hp.chunk = 0;
    cudaError_t e = cudaMalloc(&hp.buf, bytes);
    if (e != cudaSuccess) { hp.buf = nullptr; return set_error(ctx, NMC_ENOMEM, "collision_solve_host: staging buffers"); }
    hp.chunk = chunk;
    return NMC_OK;
}

// Device pointers of one slot's arrays inside the staging buffer (every array 256-byte aligned).
struct Slot {
    double *rho, *T, *Ye, *dt, *scale, *J, *H, *J_out, *H_out, *Ye_out, *eps_out, *T_out;
    int32_t *n_outer, *n_inner;
    uint32_t* status;
};

Slot slot_ptrs(const nmc_ctx* ctx, int s) {
    const HostPipe& hp = ctx->host_pipe;
    const size_t C = (size_t)hp.chunk, nsne = (size_t)ctx->ns * ctx->ne;
    char* p = static_cast<char*>(hp.buf);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* r = p + off;
        off += (bytes + 255) & ~size_t(255);
        return r;
    };
    Slot sl[2];
    for (int k = 0; k < 2; ++k) {
        Slot& x = sl[k];
        x.rho = (double*)take(8 * C); x.T = (double*)take(8 * C); x.Ye = (double*)take(8 * C);
        x.dt = (double*)take(8 * C); x.scale = (double*)take(32 * C);
        x.J = (double*)take(8 * C * nsne); x.H = (double*)take(24 * C * nsne);
        x.J_out = (double*)take(8 * C * nsne); x.H_out = (double*)take(24 * C * nsne);
        x.Ye_out = (double*)take(8 * C); x.eps_out = (double*)take(8 * C); x.T_out = (double*)take(8 * C);
        x.n_outer = (int32_t*)take(4 * C); x.n_inner = (int32_t*)take(4 * C); x.status = (uint32_t*)take(4 * C);
    }
    return sl[s];
}

}  // namespace

void host_pipe_release(nmc_ctx* ctx) {
    HostPipe& hp = ctx->host_pipe;
    if (hp.buf) cudaFree(hp.buf);
    for (int s = 0; s < 2; ++s) {
        if (hp.uploaded[s]) cudaEventDestroy(hp.uploaded[s]);
        if (hp.solved[s]) cudaEventDestroy(hp.solved[s]);
        if (hp.downloaded[s]) cudaEventDestroy(hp.downloaded[s]);
    }
    if (hp.up) cudaStreamDestroy(hp.up);
    if (hp.down) cudaStreamDestroy(hp.down);
    hp = HostPipe{};
}

}  // namespace nmc

using namespace nmc;

extern "C" int collision_solve_host(nmc_ctx* ctx, const nmc_params* params, int64_t n, const double* rho,
                                    const double* T_in, const double* Ye_in, const double* J_in,
                                    const double* H_in, const double* dt, const double* opac_scale,
                                    double* J_out, double* H_out, double* Ye_out, double* eps_out, double* T_out,
                                    int32_t* n_outer, int32_t* n_inner, uint32_t* status, int64_t chunk,
                                    void* stream) {
    if (!ctx) return NMC_EINVAL;
    int rc = nmc_check_params_internal(ctx, params);
    if (rc != NMC_OK) return rc;
    if (n < 0 || chunk < 0) return set_error(ctx, NMC_EINVAL, "n < 0 or chunk < 0");
    if (n > (int64_t(1) << 30)) return set_error(ctx, NMC_EUNSUPPORTED, "n > 2^30 nodes per call");
    if (n == 0) return NMC_OK;
    if (!rho || !T_in || !Ye_in || !J_in || !H_in || !dt || !J_out || !H_out || !Ye_out || !eps_out || !T_out ||
        !n_outer || !n_inner || !status)
        return set_error(ctx, NMC_EINVAL, "null array argument");
    long long C = chunk > 0 ? chunk : std::max<long long>(8192, (n + 7) / 8);
    C = std::min<long long>(C, n);
    rc = ensure_staging(ctx, C);
    if (rc != NMC_OK) return rc;
    HostPipe& hp = ctx->host_pipe;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const size_t nsne = (size_t)ctx->ns * ctx->ne;
    cudaError_t e = cudaSuccess;
    // the staging slots are free once earlier work on the caller's stream is done
    e = cudaEventRecord(hp.solved[0], cs);
    if (e == cudaSuccess) e = cudaEventRecord(hp.solved[1], cs);
    if (e == cudaSuccess) e = cudaEventRecord(hp.downloaded[0], cs);
    if (e == cudaSuccess) e = cudaEventRecord(hp.downloaded[1], cs);
    const long long nchunks = (n + C - 1) / C;
    for (long long i = 0; i < nchunks && e == cudaSuccess; ++i) {
        const int s = (int)(i & 1);
        const long long n0 = i * C, m = std::min<long long>(C, n - n0);
        const Slot d = slot_ptrs(ctx, s);
        // upload
        e = cudaStreamWaitEvent(hp.up, hp.solved[s], 0);
        auto up = [&](void* dst, const void* src, size_t bytes) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, hp.up);
        };
        up(d.rho, rho + n0, 8 * m);
        up(d.T, T_in + n0, 8 * m);
        up(d.Ye, Ye_in + n0, 8 * m);
        up(d.dt, dt + n0, 8 * m);
        if (opac_scale) up(d.scale, opac_scale + 4 * n0, 32 * m);
        up(d.J, J_in + n0 * nsne, 8 * m * nsne);
        up(d.H, H_in + 3 * n0 * nsne, 24 * m * nsne);
        if (e == cudaSuccess) e = cudaEventRecord(hp.uploaded[s], hp.up);
        // solve on the caller's stream
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, hp.uploaded[s], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, hp.downloaded[s], 0);
        if (e != cudaSuccess) break;
        rc = collision_solve(ctx, params, m, d.rho, d.T, d.Ye, d.J, d.H, d.dt, opac_scale ? d.scale : nullptr,
                             d.J_out, d.H_out, d.Ye_out, d.eps_out, d.T_out, d.n_outer, d.n_inner, d.status, cs);
        if (rc != NMC_OK) return rc;
        e = cudaEventRecord(hp.solved[s], cs);
        // download
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.down, hp.solved[s], 0);
        auto down = [&](void* dst, const void* src, size_t bytes) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, hp.down);
        };
        down(J_out + n0 * nsne, d.J_out, 8 * m * nsne);
        down(H_out + 3 * n0 * nsne, d.H_out, 24 * m * nsne);
        down(Ye_out + n0, d.Ye_out, 8 * m);
        down(eps_out + n0, d.eps_out, 8 * m);
        down(T_out + n0, d.T_out, 8 * m);
        down(n_outer + n0, d.n_outer, 4 * m);
        down(n_inner + n0, d.n_inner, 4 * m);
        down(status + n0, d.status, 4 * m);
        if (e == cudaSuccess) e = cudaEventRecord(hp.downloaded[s], hp.down);
    }
    // the caller's stream completes after the last downloads
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, hp.downloaded[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, hp.downloaded[1], 0);
    if (e != cudaSuccess) return set_error(ctx, NMC_ECUDA, std::string("collision_solve_host: ") + cudaGetErrorString(e));
    return NMC_OK;
}
