// Instantiations of the evolution kernels for __half voxels (see ac_evolve.cuh).
#include "ac_evolve.cuh"
#include "ac_host.h"

namespace ac {
cudaError_t launch_evolve_f16(const EvolveArgs &a, bool brick, int G, bool comp, bool acc, int warps, int64_t grid,
                             cudaStream_t st)
{
    return launch_evolve_t<__half>(a, brick, G, comp, acc, warps, grid, st);
}
}  // namespace ac
