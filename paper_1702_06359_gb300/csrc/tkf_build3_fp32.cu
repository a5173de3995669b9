// Build-kernel instantiations for trackers with endcap disks (the "endcap z" of Sec. 2.2),
// fp32 precision mode (state float, Kalman update float).
#include "build_kernel.cuh"

namespace tkf {
cudaError_t launch_build3_fp32(const BuildArgs &a, int nmax, int grid, cudaStream_t s, int *occupancy)
{
    return launch_build_t<float, float, false, true>(a, nmax, grid, s, occupancy);
}
}  // namespace tkf
