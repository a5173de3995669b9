// Build-kernel instantiations for trackers with endcap disks (the "endcap z" of Sec. 2.2),
// fp64 precision mode (state and update double).
#include "build_kernel.cuh"

namespace tkf {
cudaError_t launch_build3_fp64(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy)
{
    return launch_build_t<double, double, false, true>(a, nmax, grid, s, occupancy);
}
}  // namespace tkf
