// Host-side call into cuRAND's Philox4x32-10 (a header of the CUDA toolkit), used
// only as an independent library check of the oracle's generator.
#include <cstdint>
#include <curand_philox4x32_x.h>
extern "C" void curand_philox_batch(long n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    uint2 k = {key[0], key[1]};
    for (long i = 0; i < n; ++i) {
        uint4 c = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
        uint4 r = curand_Philox4x32_10(c, k);
        out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
    }
}
