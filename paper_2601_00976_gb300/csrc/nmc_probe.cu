// nmc_fma_probe: the FMA-pipe peak that bounds the collision solve's kernels.
//
// The solve is per-node dense arithmetic (mat-vecs, Anderson sums), so its
// roofline denominator is the FP64 FMA rate (FP64 path) or the FP32 FMA rate
// (mixed path), not HBM bandwidth.  This kernel measures that rate on the
// device it runs on: every thread advances sixteen independent FMA chains
// x <- x * b + c (b, c chosen so that x stays O(1), never denormal), so the
// pipe sees sixteen independent instructions per dependency latency, and the
// grid fills every SM at full occupancy.  The caller times the launch with
// CUDA events on the stream and divides the returned flop count by it.
#include <cuda_runtime.h>

#include <string>

#include "nmc.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 512;

template <typename R>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, R b, R c, R* sink) {
    R x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (R)(threadIdx.x + k) * (R)1e-3;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = x[k] * b + c;
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    // never true for the values the chains reach (they tend to c / (1 - b)); keeps the work live
    if (s == (R)-1) sink[0] = s;
}

template <typename R>
int launch(int blocks_per_sm, int iters, void* sink, double* flops, void* stream) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return NMC_ECUDA;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<R>, kThreads, 0);
    if (e != cudaSuccess || per_sm < 1) return NMC_ECUDA;
    const int bps = blocks_per_sm > 0 && blocks_per_sm < per_sm ? blocks_per_sm : per_sm;
    const long long grid = (long long)bps * sms;
    fma_probe_kernel<R><<<(unsigned)grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        iters, (R)0.999, (R)0.001, static_cast<R*>(sink));
    if (cudaGetLastError() != cudaSuccess) return NMC_ECUDA;
    if (flops) *flops = 2.0 * kChains * (double)iters * (double)kThreads * (double)grid;
    return NMC_OK;
}

}  // namespace

extern "C" int nmc_fma_probe(int32_t precision, int32_t blocks_per_sm, int32_t iters, void* sink, double* flops,
                             void* stream) {
    if (iters < 1 || !sink || (precision != NMC_FP64 && precision != NMC_MIXED)) return NMC_EINVAL;
    return precision == NMC_FP64 ? launch<double>(blocks_per_sm, iters, sink, flops, stream)
                                 : launch<float>(blocks_per_sm, iters, sink, flops, stream);
}
