// Build-kernel instantiations for the fp32 precision mode (state float, Kalman update float).
#include "build_kernel.cuh"

namespace tkf {
cudaError_t launch_build_fp32(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy)
{
    return launch_build_t<float, float>(a, nmax, grid, s, occupancy);
}
}  // namespace tkf
