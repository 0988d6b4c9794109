// FP64 arithmetic rate of the device: the roof of the FP64 Dslash on GPUs whose
// FP64 units, not memory, bound that kernel (GB300 runs 2 FP64 FMAs per SM per
// clock, so 1320 flop per 960 bytes needs far less than the HBM bandwidth).
//
// Every thread runs kChains independent multiply-add chains acc = acc * m + c,
// so the FP64 pipe always has independent work; there are no memory accesses in
// the loop.  The result is stored only when it equals an impossible value, which
// keeps the compiler from removing the chains without adding traffic.
#include <cmath>
#include "wd_host.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ double g_probe_sink;

__global__ void __launch_bounds__(kThreads) k_fp64_fma_chains(double m, double c, double never) {
    double acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (double)(threadIdx.x + k);
#pragma unroll 4
    for (int i = 0; i < kIters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], m, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    if (s == never) g_probe_sink = s;
}

}  // namespace

extern "C" wd_status wd_measure_fp64_rate(double *gflops) {
    if (!gflops) return WD_ERR_ARG;
    *gflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WD_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return WD_ERR_CUDA;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return WD_ERR_CUDA;
    wd::EventPair ev;
    cudaError_t e = ev.create();
    const dim3 grid(sms * kBlocksPerSm), block(kThreads);
    const double flop = 2.0 * kChains * kIters * (double)grid.x * kThreads;
    float best = 0.f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(ev.e0, st);
        if (e == cudaSuccess) {
            k_fp64_fma_chains<<<grid, block, 0, st>>>(0.9999999, 1e-7, -1.0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev.e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev.e1);
        const float ms = ev.ms();
        if (e == cudaSuccess && rep > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
    }
    cudaStreamDestroy(st);
    if (e != cudaSuccess || best <= 0.f) return WD_ERR_CUDA;
    *gflops = flop / (best * 1e-3) / 1e9;
    return WD_OK;
}
