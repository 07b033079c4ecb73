// Instantiations of the evolution kernels for uint8_t voxels (see ac_evolve.cuh).
#include "ac_evolve.cuh"
#include "ac_host.h"

namespace ac {
cudaError_t launch_evolve_u8(const EvolveArgs &a, bool brick, int G, bool comp, bool acc, int warps, int64_t grid,
                             cudaStream_t st)
{
    return launch_evolve_t<uint8_t>(a, brick, G, comp, acc, warps, grid, st);
}
}  // namespace ac
