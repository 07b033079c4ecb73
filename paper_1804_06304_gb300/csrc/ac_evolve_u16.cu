// Instantiations of the evolution kernels for uint16_t voxels (see ac_evolve.cuh).
#include "ac_evolve.cuh"
#include "ac_host.h"

namespace ac {
cudaError_t launch_evolve_u16(const EvolveArgs &a, bool brick, int G, bool comp, bool acc, int warps, int64_t grid,
                             cudaStream_t st)
{
    return launch_evolve_t<uint16_t>(a, brick, G, comp, acc, warps, grid, st);
}
}  // namespace ac
