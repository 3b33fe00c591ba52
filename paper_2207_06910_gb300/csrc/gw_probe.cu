// gw_probe.cu -- gw_fma_rate: measured FMA throughput of the FP64 and FP32
// pipes, the denominators of the roofline fractions of the point kernels.
//
// Every thread runs NCHAIN independent FMA chains (x = x * a + b) for `iters`
// iterations, so the pipe, not the FMA latency, limits the rate; the FP32
// chains are packed FP32x2 FMAs (FFMA2, two FMAs per instruction), which on this
// GPU issue at up to twice the rate of scalar FFMA.  The grid is
// blocks_per_sm blocks of 256 threads per SM, all resident at once; thread 0 of
// every block reads the SM clock counter (clock64) before and after its loop.
// A block's FMAs times the blocks per SM over the block's cycles is the SM's
// rate per clock; the launch's CUDA-event time gives the rate per second and,
// with the cycle counts, the SM clock during the loop.
#include <cstdint>

#include "../../include/gwfish.h"
#include "gw_kernels.cuh"

namespace gw {
namespace {

constexpr int NCHAIN = 8;
constexpr int PROBE_THREADS = 256;

__global__ void __launch_bounds__(PROBE_THREADS) k_fma_rate64(int iters, double a, double b,
                                                              double *sink, long long *cycles)
{
    double x[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; c++) x[c] = (double)(threadIdx.x + c);
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < NCHAIN; c++) x[c] = fma(x[c], a, b);
    }
    __syncthreads();
    const long long t1 = clock64();
    double s = 0;
#pragma unroll
    for (int c = 0; c < NCHAIN; c++) s += x[c];
    if (s == 1.2345) sink[threadIdx.x] = s;   // keeps the loop; never true for these inputs
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// FP32: packed FP32x2 FMAs (two FMAs per instruction, the form the mixed
// kernels use); NCHAIN packed chains = 2 NCHAIN FMAs per iteration
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_rate32(int iters, float a, float b,
                                                              float *sink, long long *cycles)
{
    float2 x[NCHAIN];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < NCHAIN; c++) x[c] = make_float2((float)(threadIdx.x + c), (float)c);
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < NCHAIN; c++) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0;
#pragma unroll
    for (int c = 0; c < NCHAIN; c++) s += x[c].x + x[c].y;
    if (s == 1.2345f) sink[threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace gw

using namespace gw;

extern "C" gw_status gw_fma_rate(int fp64, int iters, double *fma_per_clk_sm, double *fma_per_s,
                                 double *sm_mhz, void *stream)
{
    if (iters < 1 || iters > (1 << 24) || !fma_per_clk_sm || !fma_per_s || !sm_mhz)
        return GW_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = device_sm_count();
    const int per_sm = fp64 ? 2 : 4;
    const int blocks = sms * per_sm;
    long long *cyc = nullptr;
    void *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gw_status st = GW_ECUDA;
    if (cudaMalloc((void **)&cyc, sizeof(long long) * blocks) != cudaSuccess ||
        cudaMalloc(&sink, sizeof(double) * PROBE_THREADS) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        goto done;
    for (int rep = 0; rep < 2; rep++) {   // the first launch warms the clocks up
        cudaEventRecord(e0, s);
        if (fp64)
            k_fma_rate64<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999999, 1e-7, (double *)sink, cyc);
        else
            k_fma_rate32<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999999f, 1e-7f, (float *)sink, cyc);
        cudaEventRecord(e1, s);
    }
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) goto done;
    {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        long long *h = new long long[blocks];
        cudaMemcpy(h, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
        double mean = 0.0;
        for (int i = 0; i < blocks; i++) mean += (double)h[i];
        mean /= blocks;
        delete[] h;
        const double fma_block = (double)PROBE_THREADS * iters * NCHAIN * (fp64 ? 1 : 2);
        *fma_per_clk_sm = fma_block * per_sm / mean;
        *fma_per_s = fma_block * blocks / (ms * 1e-3);
        *sm_mhz = mean / (ms * 1e-3) / 1e6;
        st = GW_OK;
    }
done:
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(cyc);
    cudaFree(sink);
    return st;
}
