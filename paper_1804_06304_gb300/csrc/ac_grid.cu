// ac_grid.cu -- the voxel-grid form of Eq. 5 (the paper's integration before it
// moved to Monte-Carlo sampling): the sums of Eqs. 5 and 7-10 run over every
// voxel centre inside the ball of radius R + dR/2, each weighted by one voxel
// volume, instead of over N random samples.  No interpolation and no random
// numbers; the image beyond the volume is clamp-to-edge, as for the samples.
//
// One group of G lanes per contour keeps the state in registers for every
// iteration of its window.  The group walks the rows of the ball's bounding box
// (y, z), skips rows that miss the ball, and its lanes take consecutive voxels of
// a row's chord, so a row is read with neighbouring addresses.  Gathers go
// through the read-only cache from global memory.
#include "ac_evolve.cuh"
#include "ac_host.h"

namespace ac {
namespace {

template <int DIM, typename T, int G, bool COMP>
__device__ __forceinline__ Step eval_grid(const VolDesc &V, const EvolveArgs &a, const float *c, float R, int lig,
                                          unsigned mask)
{
    const float Ro = R + 0.5f * a.dR;
    const float Ro2 = Ro * Ro;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        lo[d] = (int)ceilf((c[d] - Ro) * V.inv_sp[d]);
        hi[d] = (int)floorf((c[d] + Ro) * V.inv_sp[d]);
    }
    const float B1 = fmaf(-a.rho * R, a.inv_dr, 0.5f);   // inner band coordinate: r / dr + B1
    const float B2 = fmaf(-R, a.inv_dR, 0.5f);           // outer band coordinate: r / dR + B2
    const T *data = reinterpret_cast<const T *>(V.data);
    const int64_t nvox = V.pitch_z * V.n[2];   // extent for the checked build
    KSum acc[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int kz = lo[2]; kz <= hi[2]; ++kz) {
        const float dz = DIM == 3 ? fmaf((float)kz, V.sp[2], -c[2]) : 0.0f;
        const int zz = DIM == 3 ? min(max(kz, 0), V.n[2] - 1) : 0;
        for (int jy = lo[1]; jy <= hi[1]; ++jy) {
            const float dy = fmaf((float)jy, V.sp[1], -c[1]);
            const float rem = Ro2 - fmaf(dy, dy, dz * dz);
            if (rem < 0.0f) continue;   // the row misses the ball (same for the whole group)
            const float chord = sqrtf(rem);
            const int i0 = (int)ceilf((c[0] - chord) * V.inv_sp[0]);
            const int i1 = (int)floorf((c[0] + chord) * V.inv_sp[0]);
            const int yy = min(max(jy, 0), V.n[1] - 1);
            const int64_t row = (int64_t)zz * V.pitch_z + (int64_t)yy * V.pitch_y;
            // the terms of voxel ix of this row
            auto terms = [&](int ix, float *v) {
                const float dx = fmaf((float)ix, V.sp[0], -c[0]);
                const float I = ix <= i1 ? ldg_f<T>(data + checked(row + min(max(ix, 0), V.n[0] - 1), nvox, V.status))
                                         : 0.0f;
                const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                const float t1 = fmaf(r, a.inv_dr, B1), t2 = fmaf(r, a.inv_dR, B2);
                const float r1 = __saturatef(t1), r2 = __saturatef(t2);
                const float S = fmaf(2.0f, r1, -1.0f) - r2;
                const bool b1 = r1 == t1, b2 = r2 == t2;   // voxel inside the inner / outer band
                const float dSdR = (b1 ? a.kR1 : 0.0f) + (b2 ? a.kR2 : 0.0f);
                // -S'(r) I / r: the direction (x - c) / r without a division by zero at the centre
                const float g = r > 0.0f ? ((b1 ? a.kr1 : 0.0f) + (b2 ? a.kr2 : 0.0f)) * I / r : 0.0f;
                v[0] = S * I;
                v[1] = dSdR * I;
                v[2] = g * dx;
                v[3] = g * dy;
                v[4] = g * dz;
            };
            // two voxels per step (ix and ix + G), summed in one rounding before the
            // compensated addition: two independent chains of work per lane.  In 2D
            // every step takes a pair (a voxel beyond the chord adds zero: cheaper than
            // a divergent tail on these latency-bound rows); in 3D, whose rows are
            // shorter, pairs only while both voxels lie on the chord, then a single one
            int ix = i0 + lig;
            for (; DIM == 2 ? ix <= i1 : ix + G <= i1; ix += 2 * G) {
                float v[5], w[5];
                terms(ix, v);
                terms(ix + G, w);
#pragma unroll
                for (int m = 0; m < (DIM == 3 ? 5 : 4); ++m) {
                    if (COMP) kadd(acc[m], v[m] + w[m]);
                    else acc[m].s += v[m] + w[m];
                }
            }
            if (ix <= i1) {
                float v[5];
                terms(ix, v);
#pragma unroll
                for (int m = 0; m < (DIM == 3 ? 5 : 4); ++m) {
                    if (COMP) kadd(acc[m], v[m]);
                    else acc[m].s += v[m];
                }
            }
        }
    }
    float sums[5];
    sums[4] = 0.0f;
    group_reduce_all<G, COMP, DIM == 3 ? 5 : 4>(acc, sums, mask);
    // Eqs. 5-11 in centre/radius form with the voxel volume as the measure
    float vox = V.sp[0] * V.sp[1];
    if (DIM == 3) vox *= V.sp[2];
    const float w = vox * V.scale;
    const float inv2R = __frcp_rn(2.0f * R);
    const float inv = DIM == 3 ? inv2R * inv2R * inv2R : inv2R * inv2R;   // (2R)^-d
    Step s;
    const float J = sums[0] * w;
    s.E = J * inv;
    s.dEdR = (sums[1] * w - (float)DIM * 2.0f * J * inv2R) * inv;
    s.g[0] = sums[2] * w * inv;
    s.g[1] = sums[3] * w * inv;
    s.g[2] = DIM == 3 ? sums[4] * w * inv : 0.0f;
    return s;
}

template <int DIM, typename T, int G, bool COMP>
__global__ void __maxnreg__(80) evolve_grid_kernel(const __grid_constant__ EvolveArgs a)
{
    unsigned int evals = 0;
    const int lig = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    for (int64_t gi = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; gi < a.total_contours; gi += groups) {
        const int v = find_vol(a, gi, false);
        const VolDesc &V = a.vols[v];
        if (V.first_iter > V.last_iter) continue;   // no iterations for this set in this launch
        const int64_t k = gi - V.contour_base;
        const int64_t C = V.C;
        int32_t h = V.hold ? V.hold[k] : 0;
        if (h & HOLD_STOPPED) continue;
        float c[3] = {V.state[k], V.state[C + k], DIM == 3 ? V.state[2 * C + k] : 0.0f};
        float R = V.state[3 * C + k];
        Step s{0.0f, 0.0f, {0.0f, 0.0f, 0.0f}};
        for (int n = V.first_iter; n <= V.last_iter; ++n) {
            // bounded work per evaluation: a radius beyond the grid bound (possible
            // only through an explicitly set state) stops the contour with a status
            const float Ro = R + 0.5f * a.dR;
            bool wide = false;
#pragma unroll
            for (int d = 0; d < DIM; ++d) wide = wide || !(Ro * V.inv_sp[d] <= GRID_MAX_RADIUS_VOXELS);
            if (wide) {
                if (lig == 0) atomicOr(V.status, STATUS_GRID_RANGE);
                s.E = V.state[4 * C + k];
                break;
            }
            s = eval_grid<DIM, T, G, COMP>(V, a, c, R, lig, mask);
            ++evals;
            if (lig == 0) write_trace(a, v, k, n, c, R, s);
            if (!finite_step(s)) {
                if (lig == 0) atomicOr(V.status, STATUS_NONFINITE);
                break;
            }
            if (step_or_stop<DIM>(s, n, a, V, c, R, h)) break;
        }
        if (lig == 0) {
            V.state[k] = c[0];
            V.state[C + k] = c[1];
            if (DIM == 3) V.state[2 * C + k] = c[2];
            V.state[3 * C + k] = R;
            V.state[4 * C + k] = s.E;
            if (!(isfinite(s.E) && isfinite(R) && isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2])))
                atomicOr(V.status, STATUS_NONFINITE);
            if (V.hold && rules_on(a)) V.hold[k] = h;
        }
    }
    // contour-iterations, counted once per group, one atomic per warp
    const unsigned int tot = __reduce_add_sync(0xffffffffu, lig == 0 ? evals : 0u);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&a.path_counts[2], (unsigned long long)tot);
}

template <int DIM, typename T, int G, bool COMP>
cudaError_t launch_grid_t(const EvolveArgs &a, int warps, int64_t grid, cudaStream_t st)
{
    evolve_grid_kernel<DIM, T, G, COMP><<<(unsigned)grid, warps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

// 8 and 16 lanes, compensated and plain sums, 2D and 3D; 4 lanes in 2D (compensated).
template <typename T>
cudaError_t launch_grid_dtype(const EvolveArgs &a, int G, bool comp, int warps, int64_t grid, cudaStream_t st)
{
#define AC_GRID(DIM, GG, CC) \
    if (a.ndim == DIM && G == GG && comp == CC) return launch_grid_t<DIM, T, GG, CC>(a, warps, grid, st);
    AC_GRID(3, 8, true) AC_GRID(3, 16, true) AC_GRID(3, 8, false) AC_GRID(3, 16, false)
    AC_GRID(2, 8, true) AC_GRID(2, 16, true) AC_GRID(2, 8, false) AC_GRID(2, 16, false) AC_GRID(2, 4, true)
#undef AC_GRID
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_grid(ac_dtype t, const EvolveArgs &a, int G, bool comp, int warps, int64_t grid, cudaStream_t st)
{
    switch (t) {
    case AC_U8: return launch_grid_dtype<uint8_t>(a, G, comp, warps, grid, st);
    case AC_U16: return launch_grid_dtype<uint16_t>(a, G, comp, warps, grid, st);
    case AC_F16: return launch_grid_dtype<__half>(a, G, comp, warps, grid, st);
    default: return launch_grid_dtype<float>(a, G, comp, warps, grid, st);
    }
}

}  // namespace ac
