// gw_points_fp64_fisher.cu -- FP64 point loop: the Fisher pass (every tile of
// the autotuner), in a translation unit of its own.
#include "gw_points_fp64.cuh"

namespace gw {

cudaError_t launch_points_fp64_fisher(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    return launch_mode<MODE_FISHER>(np, rot, a, s);
}

}  // namespace gw
