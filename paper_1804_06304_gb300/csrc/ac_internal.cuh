// ac_internal.cuh -- device routines and launch structures of libac (not part of
// the ABI).  Method: Lotfollahi et al., arXiv:1804.06304; see include/ac.h.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ac.h"

namespace ac {

// ----------------------------------------------------------------- status word
enum : int32_t {
    STATUS_TMA_TIMEOUT = 1,   // a brick's TMA load did not complete within the bound
    STATUS_NONFINITE = 2,     // a contour's state or energy became non-finite
    STATUS_LOCALIZE_LIMIT = 4 // localization rounds hit their bound
};

// ----------------------------------------------------------------- structures
// One volume (or one contour set on its volume) as a kernel sees it.
struct VolDesc {
    const void *data;    // row-pitched device copy, x fastest
    int64_t pitch_y;     // elements per row
    int64_t pitch_z;     // elements per plane
    int32_t n[3];        // voxels per axis (nz = 1 in 2D)
    float sp[3];         // spacing
    float inv_sp[3];     // 1 / spacing
    float box_hi[3];     // (n - 1) * spacing: upper bound of a centre
    float scale;         // intensity scale
    int32_t nb[3];       // bricks per axis (brick path)
    float *state;        // 5 x C float32, SoA: cx, cy, cz, R, E
    int64_t C;           // contours in this set
    int64_t brick_base;  // first global brick index of this set
    int64_t contour_base;// first global contour index of this set
    uint32_t key0, key1; // Philox key
};

struct EvolveArgs {
    const VolDesc *vols;
    int32_t n_vols;
    int32_t ndim;
    const CUtensorMap *tmaps;     // one per volume (brick path)
    const uint32_t *sorted_brick; // global brick index of each sorted contour
    const uint32_t *sorted_gidx;  // global contour index of each sorted contour
    int64_t total_contours;
    int64_t total_bricks;
    int32_t B[3];        // brick interior, voxels
    int32_t halo[3];     // halo, voxels (x a multiple of the TMA alignment)
    int32_t ext[3];      // staged region = B + 2 halo
    int32_t smem_bytes;  // staged region bytes
    int32_t N, T;
    int32_t iter0;       // plain path: the iteration this launch performs
    int32_t first_iter;  // n of the first iteration
    int32_t last_iter;   // n of the last iteration
    int32_t update_last; // update after the last iteration too
    uint32_t stream_id;
    float eps0, dR, Rmin, Rmax, max_step;
    float *trace;        // optional (volume 0 only)
    int64_t tk0, tk1;
    int32_t tt0, tt1;
    int32_t *status;
};

// ----------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): 10 rounds of the 4x32 bijection with
// multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 /
// 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// top 24 bits of a word as a uniform in [0, 1) (exact in FP32)
__device__ __forceinline__ float u24(uint32_t w)
{
    return __uint2float_rn(w >> 8) * 5.9604644775390625e-8f;
}

// ----------------------------------------------------------------- voxel loads
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<uint8_t>(uint8_t v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<uint16_t>(uint16_t v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }

template <typename T> __device__ __forceinline__ float ldg_f(const T *p) { return to_f<T>(__ldg(p)); }
template <> __device__ __forceinline__ float ldg_f<__half>(const __half *p)
{
    return __half2float(__ldg(reinterpret_cast<const __half *>(p)));
}

// ----------------------------------------------------------------- compensated sums
// Kahan accumulation per lane; value = s - c.
struct KSum {
    float s, c;
};
__device__ __forceinline__ void kadd(KSum &a, float x)
{
    const float y = x - a.c;
    const float t = a.s + y;
    a.c = (t - a.s) - y;
    a.s = t;
}

// Butterfly reduction over G lanes.  Compensated: (s, e) pairs combined with the
// exact TwoSum error; every lane of the group ends with the same bits.
template <int G, bool COMP>
__device__ __forceinline__ float group_reduce(KSum a, unsigned mask)
{
    if (!COMP) {
        float s = a.s;
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(mask, s, off);
        return s;
    }
    float s = a.s, e = -a.c;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const float os = __shfl_xor_sync(mask, s, off);
        const float oe = __shfl_xor_sync(mask, e, off);
        const float t = s + os;
        const float bp = t - s;
        const float err = (s - (t - bp)) + (os - bp);
        e = (e + oe) + err;
        s = t;
    }
    return s + e;
}

// ----------------------------------------------------------------- per-contour setup
// Centre in index units split into an integer voxel and a small remainder, so that
// sample positions keep full precision in large volumes.
struct AxisSplit {
    int ci;      // integer part (voxel index of the centre, floor)
    float cf;    // remainder in index units, about [0, 1)
    float lo;    // -ci: clamp of the remainder-relative coordinate at index 0
    float hi;    // (n - 1) - ci: clamp at the last index
    float top;   // (n - 2) - ci: largest base tap
};

__device__ __forceinline__ AxisSplit split_axis(float c, float sp, float inv_sp, int n)
{
    AxisSplit a;
    const float fi = floorf(c * inv_sp);
    a.ci = (int)fi;
    a.cf = fmaf(-fi, sp, c) * inv_sp;   // c - ci * sp is exact (fused), then scaled
    a.lo = (float)(-a.ci);
    a.hi = (float)(n - 1 - a.ci);
    a.top = (float)(n - 2 - a.ci);
    return a;
}

// Clamp-to-edge multilinear interpolation along one axis: the base tap (relative
// to the centre voxel) and the fraction.  Clamping the coordinate to [0, n-1] and
// the base tap to n-2 gives exactly the interpolant with clamped tap indices.
__device__ __forceinline__ void axis_tap(const AxisSplit &a, float off, int &base, float &fr)
{
    float x = a.cf + off;
    x = fminf(fmaxf(x, a.lo), a.hi);
    const float fl = fminf(floorf(x), a.top);
    fr = x - fl;
    base = (int)fl;
}

// ----------------------------------------------------------------- weight function
// S(r;R) = -1 + 2 ramp((r - rho R)/dr) - ramp((r - R)/dR), ramp(t) = clamp(t+1/2, 0, 1),
// dr = dR / 2^(1/d) (Eq. 5 and the relation below it); band membership t in [-1/2, 1/2).
struct WeightConsts {
    float a1, b1;  // t1 + 1/2 = r a1 + b1
    float a2, b2;  // t2 + 1/2 = r a2 + b2
    float kR1, kR2; // dS/dR on the inner / outer band
    float kr1, kr2; // -dS/dr on the inner / outer band
};

__device__ __forceinline__ WeightConsts weight_consts(float R, float dR, int ndim)
{
    const float rho = ndim == 3 ? 0.79370052598409973738f : 0.70710678118654752440f;
    const float dr = dR * rho;
    WeightConsts w;
    w.a1 = 1.0f / dr;
    w.b1 = 0.5f - rho * R / dr;
    w.a2 = 1.0f / dR;
    w.b2 = 0.5f - R / dR;
    w.kR1 = -2.0f * rho / dr;
    w.kR2 = 1.0f / dR;
    w.kr1 = -2.0f / dr;
    w.kr2 = 1.0f / dR;
    return w;
}

}  // namespace ac
