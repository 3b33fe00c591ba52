// gw_points_mixed_fisher.cu -- mixed-precision point loop: the Fisher pass
// (every tile of the autotuner), in a translation unit of its own.
#include "gw_points_mixed.cuh"

namespace gw {

cudaError_t launch_points_mixed_fisher(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    return launch_mode_m<MODE_FISHER>(np, rot, a, s);
}

}  // namespace gw
