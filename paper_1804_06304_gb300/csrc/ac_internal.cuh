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
    STATUS_LOCALIZE_LIMIT = 4,// localization rounds hit their bound
    STATUS_GRID_RANGE = 8,    // grid path: a ball wider than the grid bound (contour stopped)
    STATUS_BOUNDS = 16        // checked build: a gather index outside its array (read as 0, reported)
};

// Checked build (compiled with AC_CHECKED): every gather index is tested against
// the extent of the array it reads; an index outside reads element 0 instead and
// sets STATUS_BOUNDS in the set's status word.  Otherwise the identity.
template <typename I> __device__ __forceinline__ I checked(I i, I n, int32_t *st)
{
#ifdef AC_CHECKED
    if (i < 0 || i >= n) {
        atomicOr(st, STATUS_BOUNDS);
        return 0;
    }
#else
    (void)n;
    (void)st;
#endif
    return i;
}

// Polls of the bounded mbarrier waits of the brick kernel: the first wait for a
// brick's TMA load (unless a test shortens it) and the drain wait after giving up.
constexpr uint32_t TMA_POLLS_DEFAULT = 1u << 22;
constexpr uint32_t TMA_DRAIN_POLLS = 1u << 22;

// Grid path: largest ball radius, in voxels along any axis, that an evaluation
// may cover (bounds the work of one evaluation).
constexpr float GRID_MAX_RADIUS_VOXELS = 256.0f;

// ----------------------------------------------------------------- stopping rules
// Per-contour hold word: the count of consecutive small steps (low 16 bits) and
// the rule that stopped the contour, if any.
enum : int32_t {
    HOLD_COUNT = 0xFFFF,
    HOLD_FROZEN = 1 << 30,    // stopped by the step rule
    HOLD_CULLED = 1 << 29,    // stopped by the energy rule
    HOLD_STOPPED = HOLD_FROZEN | HOLD_CULLED
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
    int32_t *status;     // this set's sticky status word
    int32_t *hold;       // per-contour hold words (nullptr: no stopping state)
    int64_t C;           // contours in this set
    int64_t brick_base;  // first global brick index of this set
    int64_t contour_base;// first global contour index of this set
    uint32_t stream;     // fourth Philox counter word of this set
    int32_t first_iter;  // iterations of this set: first_iter .. last_iter
    int32_t last_iter;
    int32_t update_last; // update after last_iter too
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
    int32_t halo[3];     // halo, voxels
    int32_t ext[3];      // staged region extents
    int32_t raw_bytes;   // staged region bytes (TMA box)
    int32_t quad_off;    // 2D: byte offset of the float4 quad array (0: raw gathers)
    int32_t smem_bytes;  // dynamic shared memory
    int32_t N, T;
    int32_t iter0;       // plain path: the iteration this launch performs
    int32_t first_iter;  // n of the first iteration
    int32_t last_iter;   // n of the last iteration
    int32_t update_last; // update after the last iteration too
    uint32_t rk0[10];    // Philox round keys: key + r * Weyl constant
    uint32_t rk1[10];
    float dR, Rmin, Rmax;
    float half_eps0;     // eps0 / 2: eta_n = half_eps0 / sqrt(n)
    float max_step, max_step2;
    float rho, inv_dr, inv_dR;   // weight bands (dr = rho dR)
    float kR1, kR2;      // dS/dR on the inner / outer band
    float kr1, kr2;      // -dS/dr on the inner / outer band
    float vol_coef;      // (4/3 pi or pi) / N: ball measure per sample, over Ro^d
    float freeze_tol;    // stopping rules (0: off)
    int32_t freeze_iters;
    int32_t cull_iter;
    float cull_E;
    float *trace;        // optional: rows of volume trace_vol only
    int64_t tk0, tk1;
    int32_t tt0, tt1;
    int32_t trace_vol;
    uint32_t tma_polls;  // polls of the first wait for a brick's TMA load (then it gives up)
    unsigned long long *path_counts;   // [3]: fast, clamped, global contour-iterations
    const uint32_t *active;            // plain path: contours to visit (nullptr: all)
    const unsigned long long *n_active;// device count of `active`
};

// ----------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): 10 rounds of the 4x32 bijection with
// multipliers 0xD2511F53 / 0xCD9E8D57; the round keys (key plus r times the Weyl
// constants 0x9E3779B9 / 0xBB67AE85) are launch constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t *rk0, const uint32_t *rk1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;   // one 32x32->64 multiply each
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk1[r],
                       (uint32_t)p0);
    }
    return c;
}

// Same generator with the key schedule computed in registers (test entry point).
__device__ __forceinline__ uint4 philox4x32_10_key(uint4 c, uint32_t k0, uint32_t k1)
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

// top 24 bits of a word as an exact float in [0, 2^24)
__device__ __forceinline__ float top24(uint32_t w) { return __uint2float_rn(w >> 8); }

// ----------------------------------------------------------------- fast functions
// Hardware approximations (MUFU): their errors (sqrt, lg2/ex2 ~2^-22 relative,
// sin/cos ~2^-20.5 absolute on [-pi, pi]) move a sample by well under 1e-5 voxel.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// x + y rounded toward minus infinity
__device__ __forceinline__ float add_rd(float x, float y) { return __fadd_rd(x, y); }

// Accurate (about 1 ulp) cosine and sine of the azimuth 2 pi m / 2^24 of a 24-bit
// integer m, both negated (the raw-direction convention of the kernels): m is split
// exactly into a quarter-turn index q and a remainder y in [-1/2, 1/2) quarter
// turns; sin(pi y/2) = y P(y^2), cos(pi y/2) = Q(y^2) with the fitted polynomials of
// gen_sincos_coeffs.py; the quarter turns rotate and flip the pair.
__device__ __forceinline__ void neg_sincos_turn(uint32_t m, float &nc, float &ns)
{
    const uint32_t q = (m + (1u << 21)) >> 22;                  // nearest quarter turn, 0..4
    const uint32_t f = m + (1u << 22) - (q << 22);              // remainder + 2^22, in [2^21, 3 2^21)
    // (2^23 + f) - (2^23 + 2^22) is exact: f stays inside the 23-bit mantissa
    const float y = (__uint_as_float(0x4B000000u + f) - 12582912.0f) * 2.384185791015625e-7f;
    const float y2 = y * y;
    const float s = y * fmaf(fmaf(fmaf(-0.004602177068591118f, y2, 0.07968022674322128f), y2,
                                  -0.6459634900093079f), y2, 1.5707963705062866f);
    const float c = fmaf(fmaf(fmaf(fmaf(0.0009036316769197583f, y2, -0.02086007222533226f), y2,
                                   0.25366920232772827f), y2, -1.2337005138397217f), y2, 1.0f);
    const bool odd = (q & 1u) != 0;
    const float cc = odd ? s : c, ss = odd ? c : s;
    nc = __int_as_float(__float_as_int(cc) ^ (int)(((q + 3u) & 2u) << 30));   // -cos: flip for q in {0, 3}
    ns = __int_as_float(__float_as_int(ss) ^ (int)((((q & 2u) ^ 2u)) << 30)); // -sin: flip for q in {0, 1}
}

// ----------------------------------------------------------------- voxel values
// Exact conversion of a stored voxel to float.  Integers below 2^23 go through the
// bit pattern of 2^23 + v (two integer/FMA-pipe instructions, no conversion unit).
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<uint8_t>(uint8_t v)
{
    return __uint_as_float(0x4B000000u | (uint32_t)v) - 8388608.0f;
}
template <> __device__ __forceinline__ float to_f<uint16_t>(uint16_t v)
{
    return __uint_as_float(0x4B000000u | (uint32_t)v) - 8388608.0f;
}
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }

// Integer taps as biased floats 2^23 + v (exact, one bitwise or): the difference of
// two biased taps is exact, so an interpolation converts only its base tap.
template <typename T> struct TapBias {
    static constexpr float value = 0.0f;
};
template <> struct TapBias<uint8_t> {
    static constexpr float value = 8388608.0f;
};
template <> struct TapBias<uint16_t> {
    static constexpr float value = 8388608.0f;
};
template <typename T> __device__ __forceinline__ float to_biased(T v) { return to_f<T>(v); }
template <> __device__ __forceinline__ float to_biased<uint8_t>(uint8_t v) { return __uint_as_float(0x4B000000u | v); }
template <> __device__ __forceinline__ float to_biased<uint16_t>(uint16_t v) { return __uint_as_float(0x4B000000u | v); }

template <typename T> __device__ __forceinline__ float ldg_f(const T *p) { return to_f<T>(__ldg(p)); }
template <> __device__ __forceinline__ float ldg_f<__half>(const __half *p)
{
    return __half2float(__ldg(reinterpret_cast<const __half *>(p)));
}
// biased load (integer voxels), plain load otherwise
template <typename T> __device__ __forceinline__ float ldg_biased(const T *p) { return ldg_f<T>(p); }
template <> __device__ __forceinline__ float ldg_biased<uint8_t>(const uint8_t *p) { return to_biased<uint8_t>(__ldg(p)); }
template <> __device__ __forceinline__ float ldg_biased<uint16_t>(const uint16_t *p) { return to_biased<uint16_t>(__ldg(p)); }

// ----------------------------------------------------------------- packed FP32 pairs
// Two independent single-precision operations in one instruction (sm_100 family).
// Each component rounds exactly as the scalar operation, so code written with these
// gives the bits of the same code written with scalars, in half the instructions.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ----------------------------------------------------------------- compensated sums
// Kahan accumulation per lane; value = s - c.  KSum2 holds two sums side by side.
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
struct KSum2 {
    float2 s, c;
};
__device__ __forceinline__ void kadd2(KSum2 &a, float2 x)
{
    const float2 y = sub2(x, a.c);
    const float2 t = add2(a.s, y);
    a.c = sub2(sub2(t, a.s), y);
    a.s = t;
}

// Reduction of K sums over G lanes by recursive halving: at each level (offset
// OFF) a lane keeps half of the partial sums it still holds -- the lower half
// where lane bit OFF is clear, the upper half where it is set -- and receives the
// partner's values of those, so each level exchanges about half as many values as
// the one before; once a lane holds one sum, each remaining level halves the lanes
// that hold it.  Compensated: (s, e) pairs combined with the exact TwoSum error.
// Sum i ends at a lane and position fixed at compile time and is broadcast from
// there, so every lane of the group ends with the same bits.
__device__ __forceinline__ void pair_add(float &s, float &e, float os, float oe)
{
    const float t = s + os;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (os - bp);
    e = (e + oe) + err;
    s = t;
}

template <int OFF, int N, bool COMP>
__device__ __forceinline__ void halve_level(float *s, float *e, unsigned lane, unsigned mask)
{
    if constexpr (OFF > 0) {
        constexpr int M = (N + 1) / 2;
        const bool up = (lane & OFF) != 0;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const float hs = (M + j < N) ? s[M + j] : 0.0f;
            const float he = (COMP && M + j < N) ? e[M + j] : 0.0f;
            const float ks = up ? hs : s[j], xs = up ? s[j] : hs;
            const float ke = up ? he : e[j], xe = up ? e[j] : he;
            const float rs = __shfl_xor_sync(mask, xs, OFF);
            if (COMP) {
                const float re = __shfl_xor_sync(mask, xe, OFF);
                s[j] = ks;
                e[j] = ke;
                pair_add(s[j], e[j], rs, re);
            } else {
                s[j] = ks + rs;
            }
        }
        halve_level<OFF / 2, M, COMP>(s, e, lane, mask);
    }
}

// Lane (within the group) and position where sum i ends.
template <int G, int K> __host__ __device__ constexpr int reduce_owner(int i)
{
    int n = K, p = i, lane = 0;
    for (int off = G / 2; off > 0; off >>= 1) {
        const int m = (n + 1) / 2;
        if (p >= m) {
            p -= m;
            lane |= off;
        }
        n = m;
    }
    return lane;
}
template <int G, int K> __host__ __device__ constexpr int reduce_pos(int i)
{
    int n = K, p = i;
    for (int off = G / 2; off > 0; off >>= 1) {
        const int m = (n + 1) / 2;
        if (p >= m) p -= m;
        n = m;
    }
    return p;
}

template <int G, bool COMP, int K>
__device__ __forceinline__ void group_reduce_all(const KSum *acc, float *out, unsigned mask)
{
    float s[K], e[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        s[i] = acc[i].s;
        e[i] = COMP ? -acc[i].c : 0.0f;
    }
    const unsigned lane = threadIdx.x & 31u;
    halve_level<G / 2, K, COMP>(s, e, lane, mask);
    const int base = (int)(lane & ~(unsigned)(G - 1));
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int pos = reduce_pos<G, K>(i);
        const float v = COMP ? s[pos] + e[pos] : s[pos];
        out[i] = __shfl_sync(mask, v, base + reduce_owner<G, K>(i));
    }
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
__device__ __forceinline__ void axis_tap(const AxisSplit &a, float x, int &base, float &fr)
{
    x = fminf(fmaxf(x, a.lo), a.hi);
    const float fl = fminf(floorf(x), a.top);
    fr = x - fl;
    base = (int)fl;
}

}  // namespace ac
