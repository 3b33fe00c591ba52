// gw_points_fp64.cu -- FP64 point loop: the SNR, SNR-gradient and log-det passes,
// and the per-device launch facts (the Fisher pass is instantiated in
// gw_points_fp64_fisher.cu and, with its Gram on the tensor cores, in
// gw_points_fp64_tc.cu, so the three compile in parallel).
#include "gw_points_fp64.cuh"

namespace gw {

int device_sm_count()
{
    static std::atomic<int> cache[MAX_CACHED_DEV];   // 0 = not looked up yet
    const int dev = current_device();
    int sms = dev < MAX_CACHED_DEV ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (sms > 0) return sms;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0) {
        cudaGetLastError();
        sms = 1;
    }
    if (dev < MAX_CACHED_DEV) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

int points_grid_size(int blocks_per_sm) { return blocks_per_sm * device_sm_count(); }

cudaError_t launch_points_fp64_fisher(int np, int rot, const PointArgs &a, cudaStream_t s);

cudaError_t launch_points_fp64(int mode, int np, int rot, const PointArgs &a, cudaStream_t s)
{
    switch (mode) {
    case MODE_SNR: return launch_mode<MODE_SNR>(np, rot, a, s);
    case MODE_FISHER: return launch_points_fp64_fisher(np, rot, a, s);
    case MODE_SNRGRAD: return launch_mode<MODE_SNRGRAD>(np, rot, a, s);
    default: return launch_mode<MODE_LOGDET>(np, rot, a, s);
    }
}

}  // namespace gw
