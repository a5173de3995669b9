// Build-kernel instantiations for hits off the layers' cylinders (the two-step propagation of
// Sec. 2.2), fp64 precision mode (state double, Kalman update double).
#include "build_kernel.cuh"

namespace tkf {
cudaError_t launch_build2_fp64(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy)
{
    return launch_build_t<double, double, true>(a, nmax, grid, s, occupancy);
}
}  // namespace tkf
