// nmc_fma_probe: the FMA-pipe peak that bounds the collision solve's kernels.
// nmc_smem_probe: the shared-memory load rate that bounds the mixed kernel's
// contraction loop.
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

constexpr int kSmemThreads = 1024;
constexpr int kSmemFloats = 4096;

// Every warp issues `iters` x 64 shared-memory loads of one kind (mode): 4-byte
// loads of consecutive words (one 128-byte wavefront per warp load: the pipe's
// peak), or warp-uniform broadcasts of 4, 8 or 16 bytes, or 16-byte loads of
// consecutive words.  The address changes with the loop counter so that no
// load can be hoisted; every index stays inside the 16 KB array.
template <int MODE>
__global__ void __launch_bounds__(kSmemThreads) smem_probe_kernel(int iters, float* sink) {
    __shared__ __align__(16) float buf[kSmemFloats];
    for (int i = threadIdx.x; i < kSmemFloats; i += blockDim.x) buf[i] = (float)(i & 7) * 1e-3f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int it = 0; it < iters; ++it) {
        const int par = it & 1;
#pragma unroll 16
        for (int j = 0; j < 64; ++j) {
            if (MODE == 0) {   // 4-byte, consecutive: j * 33 + lane <= 2110
                a0 += buf[j * 33 + lane + par];
            } else if (MODE == 1) {   // 4-byte broadcast: <= 253
                a0 += buf[j * 4 + par];
            } else if (MODE == 2) {   // 8-byte broadcast: float2 index <= 127
                const float2 v = reinterpret_cast<const float2*>(buf)[j * 2 + par];
                a0 += v.x; a1 += v.y;
            } else if (MODE == 3) {   // 16-byte broadcast: float4 index <= 64
                const float4 v = reinterpret_cast<const float4*>(buf)[j + par];
                a0 += v.x; a1 += v.y; a2 += v.z; a3 += v.w;
            } else {   // 16-byte, consecutive: float4 index < 1024
                const float4 v = reinterpret_cast<const float4*>(buf)[(j * 8 + lane + par) & 1023];
                a0 += v.x; a1 += v.y; a2 += v.z; a3 += v.w;
            }
        }
    }
    const float s = a0 + a1 + a2 + a3;
    if (s == -1.f) sink[0] = s;   // never true (all terms are non-negative); keeps the loads live
}

template <int MODE>
int launch_smem(int iters, void* sink, double* warp_loads, void* stream) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_probe_kernel<MODE>, kSmemThreads, 0);
    if (e != cudaSuccess || per_sm < 1) return NMC_ECUDA;
    const long long grid = (long long)per_sm * sms;
    smem_probe_kernel<MODE><<<(unsigned)grid, kSmemThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        iters, static_cast<float*>(sink));
    if (cudaGetLastError() != cudaSuccess) return NMC_ECUDA;
    if (warp_loads) *warp_loads = 64.0 * (double)iters * (kSmemThreads / 32) * (double)grid;
    return NMC_OK;
}

}  // namespace

extern "C" int nmc_smem_probe(int32_t mode, int32_t iters, void* sink, double* warp_loads, void* stream) {
    if (iters < 1 || !sink) return NMC_EINVAL;
    switch (mode) {
        case 0: return launch_smem<0>(iters, sink, warp_loads, stream);
        case 1: return launch_smem<1>(iters, sink, warp_loads, stream);
        case 2: return launch_smem<2>(iters, sink, warp_loads, stream);
        case 3: return launch_smem<3>(iters, sink, warp_loads, stream);
        case 4: return launch_smem<4>(iters, sink, warp_loads, stream);
        default: return NMC_EINVAL;
    }
}

extern "C" int nmc_fma_probe(int32_t precision, int32_t blocks_per_sm, int32_t iters, void* sink, double* flops,
                             void* stream) {
    if (iters < 1 || !sink || (precision != NMC_FP64 && precision != NMC_MIXED)) return NMC_EINVAL;
    return precision == NMC_FP64 ? launch<double>(blocks_per_sm, iters, sink, flops, stream)
                                 : launch<float>(blocks_per_sm, iters, sink, flops, stream);
}
