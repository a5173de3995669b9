// Build-kernel instantiations for the fp64 precision mode (state double, Kalman update double).
#include "build_kernel.cuh"

namespace tkf {
cudaError_t launch_build_fp64(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy)
{
    return launch_build_t<double, double>(a, nmax, grid, s, occupancy);
}
}  // namespace tkf
