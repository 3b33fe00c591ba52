// gw_points_mixed.cu -- mixed-precision point loop: the SNR and SNR-gradient
// passes (the Fisher pass is instantiated in gw_points_mixed_fisher.cu, so the
// two compile in parallel).
#include "gw_points_mixed.cuh"

namespace gw {

cudaError_t launch_points_mixed_fisher(int np, int rot, const PointArgs &a, cudaStream_t s);

cudaError_t launch_points_mixed(int mode, int np, int rot, const PointArgs &a, cudaStream_t s)
{
    switch (mode) {
    case MODE_SNR: return launch_mode_m<MODE_SNR>(np, rot, a, s);
    case MODE_FISHER: return launch_points_mixed_fisher(np, rot, a, s);
    default: return launch_mode_m<MODE_SNRGRAD>(np, rot, a, s);
    }
}

}  // namespace gw
