// Build-kernel instantiations for the mixed precision mode (state float, Kalman update double).
#include "build_kernel.cuh"

namespace tkf {
cudaError_t launch_build_mixed(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy)
{
    return launch_build_t<float, double>(a, nmax, grid, s, occupancy);
}
}  // namespace tkf
