// ac_evolve.cuh -- Monte-Carlo snakuscule evolution kernels (stages a3-a8).
// Included once per voxel type by ac_evolve_<type>.cu so the instantiations
// compile in parallel.  Method: arXiv:1804.06304, Eqs. 5-15 and the
// "Monte-Carlo Integration" / "Parallel Contour Evaluation" sections.
//
// Every path (brick fast path, brick clamped path, global fallback, plain
// one-launch-per-iteration kernel) shares the sample generation, weights,
// accumulation, reduction and update below, and the gathers differ only in where
// the voxels come from; the paths therefore give bit-identical results.
#pragma once

#include "ac_internal.cuh"

namespace ac {

// ----------------------------------------------------------------- TMA + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return done != 0;
}

// Bounded wait: gives up after `limit` polls (each poll may itself suspend briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// ----------------------------------------------------------------- per contour-iteration
// Samples use a raw radius variable rv (2D: sqrt of a 24-bit integer, in [0, 2^12);
// 3D: cbrt of a uniform, in [0, 1)) and a raw direction (2D: (cos a, sin a) with
// a = 2 pi u - pi, i.e. minus the unit direction; 3D: (s cos a, s sin a, cos phi)
// with s = sin(phi)/2, i.e. (-dx/2, -dy/2, dz)).  The factors that turn them into
// physical distance and index offsets are folded into these constants.
template <int DIM> struct IterC {
    AxisSplit ax[3];
    float A1, B1;   // inner band coordinate t1 + 1/2 = rv A1 + B1
    float A2, B2;   // outer band coordinate t2 + 1/2 = rv A2 + B2
    float K[3];     // index offset along axis d = rv * K[d] * raw direction[d]
};

template <int DIM>
__device__ __forceinline__ void iter_consts(IterC<DIM> &ic, const float *c, float R, const VolDesc &V,
                                            const EvolveArgs &a)
{
    const float Ro = R + 0.5f * a.dR;                         // radius of K (Eq. 5)
    const float rs = DIM == 2 ? Ro * (1.0f / 4096.0f) : Ro;   // physical distance per unit rv
    ic.A1 = rs * a.inv_dr;
    ic.B1 = fmaf(-a.rho * R, a.inv_dr, 0.5f);
    ic.A2 = rs * a.inv_dR;
    ic.B2 = fmaf(-R, a.inv_dR, 0.5f);
    const float fxy = DIM == 3 ? -2.0f : -1.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d < DIM) ic.ax[d] = split_axis(c[d], V.sp[d], V.inv_sp[d], V.n[d]);
        ic.K[d] = (d < 2 ? fxy : 1.0f) * rs * V.inv_sp[d];
    }
}

// ----------------------------------------------------------------- gathers
// Coordinates x[d] arrive relative to the centre voxel ci (x = cf + offset).

// Fast path: every tap of the ball lies inside the volume and the staged region,
// so no clamping; floor and index come from one add rounded toward minus infinity
// onto 2^23 + (ci - region origin).
__device__ __forceinline__ void fast_axis(float x, float M, int &idx, float &fr)
{
    const float t = add_rd(x, M);
    fr = x - (t - M);
    idx = (int)__float_as_uint(t) - 0x4B000000;
}
// the same for the x and y axes in packed pairs
__device__ __forceinline__ void fast_axes2(float2 x, float2 M, int &i0, int &i1, float2 &fr)
{
    const float2 t = __fadd2_rd(x, M);
    fr = sub2(x, sub2(t, M));
    i0 = (int)__float_as_uint(t.x) - 0x4B000000;
    i1 = (int)__float_as_uint(t.y) - 0x4B000000;
}

// 2D region as quads: one shared-memory load feeds a bilinear sample.  With
// `diff`, a quad holds (v00, v01, v10 - v00, v11 - v01), the values of the two rows
// and the x-differences the interpolation needs (computed once per quad in FP32, as
// the sample would), so both rows are interpolated in one packed operation; else
// (v00, v01, v10, v11).  Four halves (8 bytes) for uint8 voxels (values and
// differences are integers below 2^9, exact in half precision) and binary16 voxels
// (values only: their differences need not be representable), float4 otherwise.
struct HQuad {
    __half2 lo, hi;
};
template <typename T> struct QuadOf {
    using type = float4;
    static constexpr bool diff = true;
};
template <> struct QuadOf<uint8_t> {
    using type = HQuad;
    static constexpr bool diff = true;
};
template <> struct QuadOf<__half> {
    using type = HQuad;
    static constexpr bool diff = false;
};

__device__ __forceinline__ float4 quad_f(const float4 &q) { return q; }
__device__ __forceinline__ float4 quad_f(const HQuad &q)
{
    const float2 a = __half22float2(q.lo), b = __half22float2(q.hi);
    return make_float4(a.x, a.y, b.x, b.y);
}
template <typename QT> __device__ __forceinline__ QT make_quad(float a, float b, float c, float d);
template <> __device__ __forceinline__ float4 make_quad<float4>(float a, float b, float c, float d)
{
    return make_float4(a, b, c, d);
}
template <> __device__ __forceinline__ HQuad make_quad<HQuad>(float a, float b, float c, float d)
{
    return HQuad{__floats2half2_rn(a, b), __floats2half2_rn(c, d)};
}

template <bool DIFF> __device__ __forceinline__ float quad_lerp(const float4 q, float f0, float f1)
{
    const float2 v0 = make_float2(q.x, q.y);                       // (v00, v01)
    const float2 d = DIFF ? make_float2(q.z, q.w) : sub2(make_float2(q.z, q.w), v0);
    const float2 a = fma2(dup2(f0), d, v0);                        // the two rows at x
    return fmaf(f1, a.y - a.x, a.x);
}

template <typename QT, bool DIFF> struct QuadFast {
    const QT *Q;
    int qp;          // quads per row
    float M[2];
    int nq;          // quads in the region (checked build)
    int32_t *st;     // status word (checked build)
    __device__ __forceinline__ float at(float x0, float x1, float) const
    {
        int i0, i1;
        float2 fr;
        fast_axes2(make_float2(x0, x1), make_float2(M[0], M[1]), i0, i1, fr);
        return quad_lerp<DIFF>(quad_f(Q[checked(i1 * qp + i0, nq, st)]), fr.x, fr.y);
    }
};

// Bilinear / trilinear from four / eight taps of a raw array at q.  The loader
// returns biased taps for integer voxels (TapBias); differences are exact either
// way and only the base of each x-interpolation is unbiased, which gives the same
// bits as converting every tap.
template <int DIM, typename T, typename LD>
__device__ __forceinline__ float interp(const T *q, int64_t py, int64_t pz, float f0, float f1, float f2, LD ld)
{
    constexpr float Z = LD::bias;
    if (DIM == 2) {
        const float2 lo = make_float2(ld(q), ld(q + py)), hi = make_float2(ld(q + 1), ld(q + py + 1));
        const float2 base = Z != 0.0f ? sub2(lo, dup2(Z)) : lo;
        const float2 a = fma2(dup2(f0), sub2(hi, lo), base);      // (row y0, row y1) at x
        return fmaf(f1, a.y - a.x, a.x);
    }
    // x-interpolation of rows (y0, z0) and (y0, z1) as one pair, (y1, z0) and
    // (y1, z1) as the other; then y for both planes at once, then z
    const T *r = q + pz;
    const float2 lo0 = make_float2(ld(q), ld(r)), hi0 = make_float2(ld(q + 1), ld(r + 1));
    const float2 lo1 = make_float2(ld(q + py), ld(r + py)), hi1 = make_float2(ld(q + py + 1), ld(r + py + 1));
    const float2 a0 = fma2(dup2(f0), sub2(hi0, lo0), Z != 0.0f ? sub2(lo0, dup2(Z)) : lo0);
    const float2 a1 = fma2(dup2(f0), sub2(hi1, lo1), Z != 0.0f ? sub2(lo1, dup2(Z)) : lo1);
    const float2 sz = fma2(dup2(f1), sub2(a1, a0), a0);           // (plane z0, plane z1)
    return fmaf(f2, sz.y - sz.x, sz.x);
}

// Tap loaders (biased taps for integer voxels, see interp); base, n and st serve
// the checked build only.
template <typename T> struct SmemLoad {
    static constexpr float bias = TapBias<T>::value;
    const T *base;
    int64_t n;
    int32_t *st;
    __device__ __forceinline__ float operator()(const T *p) const
    {
#ifdef AC_CHECKED
        return to_biased<T>(base[checked((int64_t)(p - base), n, st)]);
#else
        return to_biased<T>(*p);
#endif
    }
};
template <typename T> struct GlobalLoad {
    static constexpr float bias = 0.0f;
    const T *base;
    int64_t n;
    int32_t *st;
    __device__ __forceinline__ float operator()(const T *p) const
    {
#ifdef AC_CHECKED
        return ldg_f<T>(base + checked((int64_t)(p - base), n, st));
#else
        return ldg_f<T>(p);
#endif
    }
};

template <int DIM, typename T> struct RawFast {
    const T *p;
    int py, pz;
    float M[3];
    int64_t n;       // voxels in the region (checked build)
    int32_t *st;
    __device__ __forceinline__ float at(float x0, float x1, float x2) const
    {
        int i0, i1, i2 = 0;
        float2 fr;
        float f2 = 0.0f;
        fast_axes2(make_float2(x0, x1), make_float2(M[0], M[1]), i0, i1, fr);
        if (DIM == 3) fast_axis(x2, M[2], i2, f2);
        return interp<DIM, T>(p + i0 + i1 * py + i2 * pz, py, pz, fr.x, fr.y, f2, SmemLoad<T>{p, n, st});
    }
};

// Raw taps through 32-bit shared-memory addresses (3D fast path; the bounds-checked
// build keeps RawFast): the directed
// add leaves bits(t_d) = 2^23 + tap index d (as an integer 0x4B000000 + index), so the
// byte address of the base tap is C + es bits(t0) + es py bits(t1) + es pz bits(t2)
// with the biases folded into C (arithmetic modulo 2^32); the other taps are
// that address plus row / plane pitches, the x+1 taps an immediate offset.
template <typename T> __device__ __forceinline__ float lds_tap(uint32_t a);
template <typename T> __device__ __forceinline__ float lds_tap_next(uint32_t a);
template <> __device__ __forceinline__ float lds_tap<uint16_t>(uint32_t a)
{
    unsigned short v;
    asm("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return __uint_as_float(0x4B000000u | v);
}
template <> __device__ __forceinline__ float lds_tap_next<uint16_t>(uint32_t a)
{
    unsigned short v;
    asm("ld.shared.u16 %0, [%1+2];" : "=h"(v) : "r"(a));
    return __uint_as_float(0x4B000000u | v);
}
template <> __device__ __forceinline__ float lds_tap<uint8_t>(uint32_t a)
{
    unsigned short v;
    asm("ld.shared.u8 %0, [%1];" : "=h"(v) : "r"(a));
    return __uint_as_float(0x4B000000u | v);
}
template <> __device__ __forceinline__ float lds_tap_next<uint8_t>(uint32_t a)
{
    unsigned short v;
    asm("ld.shared.u8 %0, [%1+1];" : "=h"(v) : "r"(a));
    return __uint_as_float(0x4B000000u | v);
}
template <> __device__ __forceinline__ float lds_tap<__half>(uint32_t a)
{
    unsigned short v;
    asm("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"(a));
    return __half2float(__ushort_as_half(v));
}
template <> __device__ __forceinline__ float lds_tap_next<__half>(uint32_t a)
{
    unsigned short v;
    asm("ld.shared.b16 %0, [%1+2];" : "=h"(v) : "r"(a));
    return __half2float(__ushort_as_half(v));
}
template <> __device__ __forceinline__ float lds_tap<float>(uint32_t a)
{
    float v;
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
template <> __device__ __forceinline__ float lds_tap_next<float>(uint32_t a)
{
    float v;
    asm("ld.shared.f32 %0, [%1+4];" : "=f"(v) : "r"(a));
    return v;
}

template <typename T> struct RawFast3S {
    uint32_t C;      // folded base address (see above)
    uint32_t pyb, pzb;   // row and plane pitch, bytes
    float M[3];
    __device__ __forceinline__ float at(float x0, float x1, float x2) const
    {
        constexpr float Z = TapBias<T>::value;
        constexpr uint32_t es = sizeof(T);
        const float2 t = __fadd2_rd(make_float2(x0, x1), make_float2(M[0], M[1]));
        const float2 fr = sub2(make_float2(x0, x1), sub2(t, make_float2(M[0], M[1])));
        const float t2 = add_rd(x2, M[2]);
        const float f2 = x2 - (t2 - M[2]);
        const uint32_t a = C + es * __float_as_uint(t.x) + pyb * __float_as_uint(t.y) + pzb * __float_as_uint(t2);
        const uint32_t r = a + pzb, ay = a + pyb, ry = r + pyb;
        const float2 lo0 = make_float2(lds_tap<T>(a), lds_tap<T>(r)), hi0 = make_float2(lds_tap_next<T>(a), lds_tap_next<T>(r));
        const float2 lo1 = make_float2(lds_tap<T>(ay), lds_tap<T>(ry)), hi1 = make_float2(lds_tap_next<T>(ay), lds_tap_next<T>(ry));
        const float2 a0 = fma2(dup2(fr.x), sub2(hi0, lo0), Z != 0.0f ? sub2(lo0, dup2(Z)) : lo0);
        const float2 a1 = fma2(dup2(fr.x), sub2(hi1, lo1), Z != 0.0f ? sub2(lo1, dup2(Z)) : lo1);
        const float2 sz = fma2(dup2(fr.y), sub2(a1, a0), a0);           // (plane z0, plane z1)
        return fmaf(f2, sz.y - sz.x, sz.x);
    }
};

// Clamped path in shared memory (quads in 2D, raw voxels otherwise).
template <int DIM, typename T, bool QUAD> struct SmemClamp {
    const void *p;
    int py, pz;      // raw pitches, or quads per row in py
    AxisSplit ax[3];
    int o[3];        // centre voxel relative to the region origin
    int64_t n;       // quads or voxels in the region (checked build)
    int32_t *st;
    __device__ __forceinline__ float at(float x0, float x1, float x2) const
    {
        int b0, b1, b2 = 0;
        float f0, f1, f2 = 0.0f;
        axis_tap(ax[0], x0, b0, f0);
        axis_tap(ax[1], x1, b1, f1);
        if (DIM == 3) axis_tap(ax[2], x2, b2, f2);
        if (QUAD) {
            using QT = typename QuadOf<T>::type;
            const int64_t qi = checked((int64_t)(o[1] + b1) * py + (o[0] + b0), n, st);
            return quad_lerp<QuadOf<T>::diff>(quad_f(reinterpret_cast<const QT *>(p)[qi]), f0, f1);
        }
        const T *q = reinterpret_cast<const T *>(p) + (o[0] + b0) + (o[1] + b1) * py + (DIM == 3 ? (o[2] + b2) * pz : 0);
        return interp<DIM, T>(q, py, pz, f0, f1, f2, SmemLoad<T>{reinterpret_cast<const T *>(p), n, st});
    }
};

// Clamped path from the row-pitched volume in global memory.
template <int DIM, typename T> struct GlobalClamp {
    const T *p;
    int64_t py, pz;
    AxisSplit ax[3];
    int64_t n;       // elements of the row-pitched volume (checked build)
    int32_t *st;
    __device__ __forceinline__ float at(float x0, float x1, float x2) const
    {
        int b0, b1, b2 = 0;
        float f0, f1, f2 = 0.0f;
        axis_tap(ax[0], x0, b0, f0);
        axis_tap(ax[1], x1, b1, f1);
        if (DIM == 3) axis_tap(ax[2], x2, b2, f2);
        const T *q = p + (int64_t)(ax[0].ci + b0) + (int64_t)(ax[1].ci + b1) * py +
                     (DIM == 3 ? (int64_t)(ax[2].ci + b2) * pz : 0);
        return interp<DIM, T>(q, py, pz, f0, f1, f2, GlobalLoad<T>{p, n, st});
    }
};

// ----------------------------------------------------------------- one sample
// Weights of Eq. 5 (four regions; linear bands of widths dr and dR) and the terms
// of the five sums J = sum S I, J_R = sum dS/dR I, J_c = sum -S'(r) (raw
// direction) I for one sample.
struct Terms {
    float2 a;   // (S I, dS/dR I)
    float2 b;   // -S' I times raw direction (d0, d1)
    float c;    // -S' I d2 (3D)
};

template <int DIM>
__device__ __forceinline__ Terms sample_terms(const IterC<DIM> &ic, const EvolveArgs &a, float rv, float I, float d0,
                                              float d1, float d2)
{
    const float2 t = fma2(dup2(rv), make_float2(ic.A1, ic.A2), make_float2(ic.B1, ic.B2));   // band coordinates
    const float r1 = __saturatef(t.x), r2 = __saturatef(t.y);
    const float S = fmaf(2.0f, r1, -1.0f) - r2;
    // I where the sample lies inside the inner / outer band (slopes there), else 0
    const float m1 = r1 == t.x ? I : 0.0f, m2 = r2 == t.y ? I : 0.0f;
    // (-S' I, dS/dR I) = (kr1, kR1) m1 + (kr2, kR2) m2
    const float2 gk = fma2(make_float2(a.kr1, a.kR1), dup2(m1), mul2(make_float2(a.kr2, a.kR2), dup2(m2)));
    Terms o;
    o.a = make_float2(S * I, gk.y);
    o.b = mul2(dup2(gk.x), make_float2(d0, d1));
    o.c = DIM == 3 ? gk.x * d2 : 0.0f;
    return o;
}

// Per-lane accumulators of the five sums: (J, J_R) and (J_c0, J_c1) as packed
// pairs, J_c2 alone.
struct Acc {
    KSum2 a, b;
    KSum c;
};

// Adds the terms of one sample, or the sum of two in one rounding, with Kahan
// compensation (COMP) or plainly.
template <int DIM, bool COMP> __device__ __forceinline__ void add_terms(Acc &acc, const Terms &x)
{
    if (COMP) {
        kadd2(acc.a, x.a);
        kadd2(acc.b, x.b);
        if (DIM == 3) kadd(acc.c, x.c);
    } else {
        acc.a.s = add2(acc.a.s, x.a);
        acc.b.s = add2(acc.b.s, x.b);
        if (DIM == 3) acc.c.s += x.c;
    }
}
template <int DIM> __device__ __forceinline__ Terms sum2(const Terms &x, const Terms &y)
{
    Terms h;
    h.a = add2(x.a, y.a);
    h.b = add2(x.b, y.b);
    h.c = DIM == 3 ? x.c + y.c : 0.0f;
    return h;
}
template <int DIM, bool COMP> __device__ __forceinline__ void add_terms(Acc &acc, const Terms &x, const Terms &y)
{
    add_terms<DIM, COMP>(acc, sum2<DIM>(x, y));
}

// Pairwise sum of four samples in two roundings (kept to be joined with the next
// four, or added with one compensated step: fewer additions per sample).
template <int DIM> __device__ __forceinline__ Terms sum4(const Terms &x, const Terms &y, const Terms &z, const Terms &w)
{
    return sum2<DIM>(sum2<DIM>(x, y), sum2<DIM>(z, w));
}
template <int DIM, bool COMP>
__device__ __forceinline__ void add_terms4(Acc &acc, const Terms &x, const Terms &y, const Terms &z, const Terms &w)
{
    add_terms<DIM, COMP>(acc, sum4<DIM>(x, y, z, w));
}

// All samples of one contour-iteration handled by this lane (lane `lig` of G).
// The words of iteration n of contour k form the stream Philox(0, n, k, stream),
// Philox(1, n, k, stream), ... (four words per block) and sample j takes words 2j
// and 2j + 1, so block m gives samples 2m and 2m + 1.  3D: three 21-bit uniforms
// from the two words, radius cbrt(u0), cos(phi) = 1 - 2 u1, azimuth 2 pi u2; 2D:
// two 24-bit uniforms, radius sqrt(u0), azimuth 2 pi u1 ("Monte-Carlo
// Integration" section).  ACC selects
// correctly rounded sqrt / cbrt and the polynomial sine and cosine (used when few
// samples make per-sample accuracy visible); otherwise the hardware
// approximations.
// Raw direction (minus the unit direction) of the azimuth 2 pi m / 2^BITS of an
// integer m below 2^BITS.
template <bool ACC, int BITS>
__device__ __forceinline__ void raw_direction(uint32_t m, float &d0, float &d1)
{
    if (ACC) {
        neg_sincos_turn(m << (24 - BITS), d0, d1);
    } else {
        constexpr float ANG = 6.283185307179586f / (float)(1u << BITS);   // 2 pi / 2^BITS
        const float ang = fmaf(__uint2float_rn(m), ANG, -3.14159265358979323846f);
        d0 = cos_approx(ang);
        d1 = sin_approx(ang);
    }
}

// 3D: the two words of a sample give three 21-bit uniforms -- u0 = w0 bits 31..11,
// u1 = w1 bits 20..0, u2 = w0 bits 10..0 followed by w1 bits 31..22 -- each times
// 2^-21.  u0 and u1 are read as the biased floats 2^23 + u (exact, one logic
// operation each) and scaled and unbiased by one packed FMA (exact).
template <int DIM, bool ACC, typename Gather>
__device__ __forceinline__ Terms sample3(const Gather &gat, const IterC<DIM> &ic, const EvolveArgs &a, uint32_t w0,
                                         uint32_t w1)
{
    const float b0 = __uint_as_float((w0 >> 11) | 0x4B000000u);
    const float b1 = __uint_as_float((w1 & 0x1FFFFFu) | 0x4B000000u);
    const uint32_t u2 = __funnelshift_l(w1, w0, 10) & 0x1FFFFFu;
    const float2 ut = fma2(make_float2(b0, b1), dup2(4.76837158203125e-7f), dup2(-4.0f));   // (b - 2^23) 2^-21
    const float u0 = ut.x, t = ut.y;
    const float rv = ACC ? cbrtf(u0) : ex2_approx(lg2_approx(u0) * (1.0f / 3.0f));
    const float cphi = fmaf(-2.0f, t, 1.0f);
    const float sh = ACC ? sqrtf(t * (1.0f - t)) : sqrt_approx(t * (1.0f - t));
    float c0, s0;
    raw_direction<ACC, 21>(u2, c0, s0);
    const float2 d = mul2(dup2(sh), make_float2(c0, s0));
    const float2 x = fma2(mul2(dup2(rv), make_float2(ic.K[0], ic.K[1])), d, make_float2(ic.ax[0].cf, ic.ax[1].cf));
    const float x2 = fmaf(rv * ic.K[2], cphi, ic.ax[2].cf);
    return sample_terms<DIM>(ic, a, rv, gat.at(x.x, x.y, x2), d.x, d.y, cphi);
}

template <int DIM, bool ACC, typename Gather>
__device__ __forceinline__ Terms sample2(const Gather &gat, const IterC<DIM> &ic, const EvolveArgs &a, uint32_t wr,
                                         uint32_t wa)
{
    const float rv = ACC ? sqrtf(top24(wr)) : sqrt_approx(top24(wr));
    float d0, d1;
    raw_direction<ACC, 24>(wa >> 8, d0, d1);
    const float2 x = fma2(mul2(dup2(rv), make_float2(ic.K[0], ic.K[1])), make_float2(d0, d1),
                          make_float2(ic.ax[0].cf, ic.ax[1].cf));
    return sample_terms<DIM>(ic, a, rv, gat.at(x.x, x.y, 0.0f), d0, d1, 0.0f);
}

template <int DIM, int G, bool COMP, bool ACC, typename Gather>
__device__ __forceinline__ void sample_contour(const Gather &gat, const IterC<DIM> &ic, const EvolveArgs &a,
                                               uint32_t n, uint32_t k, uint32_t stream, int lig, Acc &acc)
{
    if constexpr (DIM == 3) {
        // block m gives samples 2m and 2m + 1; a lane takes blocks m and m + G (four
        // samples, summed in two roundings before one compensated addition), then a
        // leftover block, then an odd N's last sample
        const int pairs = a.N >> 1;
        int m = lig;
#pragma unroll 1
        for (; m + G < pairs; m += 2 * G) {
            const uint4 A = philox4x32_10(make_uint4((uint32_t)m, n, k, stream), a.rk0, a.rk1);
            const uint4 B = philox4x32_10(make_uint4((uint32_t)(m + G), n, k, stream), a.rk0, a.rk1);
            add_terms4<DIM, COMP>(acc, sample3<DIM, ACC>(gat, ic, a, A.x, A.y), sample3<DIM, ACC>(gat, ic, a, A.z, A.w),
                                  sample3<DIM, ACC>(gat, ic, a, B.x, B.y), sample3<DIM, ACC>(gat, ic, a, B.z, B.w));
        }
        if (m < pairs) {
            const uint4 A = philox4x32_10(make_uint4((uint32_t)m, n, k, stream), a.rk0, a.rk1);
            add_terms<DIM, COMP>(acc, sample3<DIM, ACC>(gat, ic, a, A.x, A.y), sample3<DIM, ACC>(gat, ic, a, A.z, A.w));
        }
        if ((a.N & 1) && lig == pairs % G) {
            const uint4 A = philox4x32_10(make_uint4((uint32_t)pairs, n, k, stream), a.rk0, a.rk1);
            add_terms<DIM, COMP>(acc, sample3<DIM, ACC>(gat, ic, a, A.x, A.y));
        }
    } else {
        // the two samples of a Philox block form a pair; four blocks of a lane (m,
        // m + G, m + 2G, m + 3G) are summed pairwise in three roundings before one
        // compensated addition, then two blocks, then a leftover block and an odd
        // N's last sample
        const int pairs = a.N >> 1;
        int m = lig;
#pragma unroll 1
        for (; m + 3 * G < pairs; m += 4 * G) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)m, n, k, stream), a.rk0, a.rk1);
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(m + G), n, k, stream), a.rk0, a.rk1);
            const Terms h = sum4<DIM>(sample2<DIM, ACC>(gat, ic, a, w.x, w.y), sample2<DIM, ACC>(gat, ic, a, w.z, w.w),
                                      sample2<DIM, ACC>(gat, ic, a, u.x, u.y), sample2<DIM, ACC>(gat, ic, a, u.z, u.w));
            const uint4 w2 = philox4x32_10(make_uint4((uint32_t)(m + 2 * G), n, k, stream), a.rk0, a.rk1);
            const uint4 u2 = philox4x32_10(make_uint4((uint32_t)(m + 3 * G), n, k, stream), a.rk0, a.rk1);
            const Terms q = sum4<DIM>(sample2<DIM, ACC>(gat, ic, a, w2.x, w2.y), sample2<DIM, ACC>(gat, ic, a, w2.z, w2.w),
                                      sample2<DIM, ACC>(gat, ic, a, u2.x, u2.y), sample2<DIM, ACC>(gat, ic, a, u2.z, u2.w));
            add_terms<DIM, COMP>(acc, h, q);
        }
#pragma unroll 1
        for (; m + G < pairs; m += 2 * G) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)m, n, k, stream), a.rk0, a.rk1);
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(m + G), n, k, stream), a.rk0, a.rk1);
            add_terms4<DIM, COMP>(acc, sample2<DIM, ACC>(gat, ic, a, w.x, w.y), sample2<DIM, ACC>(gat, ic, a, w.z, w.w),
                                  sample2<DIM, ACC>(gat, ic, a, u.x, u.y), sample2<DIM, ACC>(gat, ic, a, u.z, u.w));
        }
        if (m < pairs) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)m, n, k, stream), a.rk0, a.rk1);
            add_terms<DIM, COMP>(acc, sample2<DIM, ACC>(gat, ic, a, w.x, w.y), sample2<DIM, ACC>(gat, ic, a, w.z, w.w));
        }
        if ((a.N & 1) && lig == pairs % G) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)pairs, n, k, stream), a.rk0, a.rk1);
            add_terms<DIM, COMP>(acc, sample2<DIM, ACC>(gat, ic, a, w.x, w.y));
        }
    }
}

// ----------------------------------------------------------------- finish + step
struct Step {
    float E, dEdR, g[3];
};

// Sums to energy and gradient (Eqs. 5-11, centre/radius form).
template <int DIM>
__device__ __forceinline__ Step finish(const float *sums, float R, const EvolveArgs &a, float scale)
{
    const float Ro = R + 0.5f * a.dR;
    const float RoD = DIM == 3 ? Ro * Ro * Ro : Ro * Ro;
    const float wmc = a.vol_coef * RoD * scale;                 // (V / N) x intensity scale
    const float inv2R = __frcp_rn(2.0f * R);
    const float inv = DIM == 3 ? inv2R * inv2R * inv2R : inv2R * inv2R;   // (2R)^-d
    const float fxy = DIM == 3 ? -2.0f : -1.0f;                 // raw direction to unit direction
    Step s;
    const float J = sums[0] * wmc;
    s.E = J * inv;
    s.dEdR = (sums[1] * wmc - (float)DIM * 2.0f * J * inv2R) * inv;
    s.g[0] = fxy * sums[2] * wmc * inv;
    s.g[1] = fxy * sums[3] * wmc * inv;
    s.g[2] = DIM == 3 ? sums[4] * wmc * inv : 0.0f;
    return s;
}

// Eqs. 12-15 in centre/radius form: c -= eps_n/2 dE/dc, R -= eps_n/2 dE/dR, with
// the step, radius and box clamps.
template <int DIM>
__device__ __forceinline__ void update(const Step &s, int n, const EvolveArgs &a, const float *box_hi, float *c,
                                       float &R)
{
    const float eta = a.half_eps0 * rsqrt_approx((float)n);
    float d[3] = {-eta * s.g[0], -eta * s.g[1], DIM == 3 ? -eta * s.g[2] : 0.0f};
    const float nrm2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (nrm2 > a.max_step2) {
        const float f = a.max_step * rsqrt_approx(nrm2);
        d[0] *= f;
        d[1] *= f;
        d[2] *= f;
    }
    const float dRr = fminf(fmaxf(-eta * s.dEdR, -a.max_step), a.max_step);
    R = fminf(fmaxf(R + dRr, a.Rmin), a.Rmax);
#pragma unroll
    for (int i = 0; i < DIM; ++i) c[i] = fminf(fmaxf(c[i] + d[i], 0.0f), box_hi[i]);
}

// Stopping rules, then the update after evaluation n.  The energy rule stops a
// contour whose energy at iteration cull_iter is above cull_E; the step rule
// counts consecutive updates whose step (largest absolute change of a centre
// coordinate or R, after the clamps) is below freeze_tol and stops the contour,
// without that step, when the count reaches freeze_iters.  Every lane of a group
// holds the same sums, so the decision is uniform over the group.  Returns true
// when the contour stops.
template <int DIM>
__device__ __forceinline__ bool step_or_stop(const Step &s, int n, const EvolveArgs &a, const VolDesc &V, float *c,
                                             float &R, int32_t &h)
{
    if (a.cull_iter > 0 && n == a.cull_iter && s.E > a.cull_E) {
        h |= HOLD_CULLED;
        return true;
    }
    if (!(n < V.last_iter || V.update_last)) return false;
    if (a.freeze_iters <= 0) {
        update<DIM>(s, n, a, V.box_hi, c, R);
        return false;
    }
    float cn[3] = {c[0], c[1], c[2]}, Rn = R;
    update<DIM>(s, n, a, V.box_hi, cn, Rn);
    float step = fabsf(Rn - R);
#pragma unroll
    for (int d = 0; d < DIM; ++d) step = fmaxf(step, fabsf(cn[d] - c[d]));
    const int32_t cnt = step < a.freeze_tol ? min((h & HOLD_COUNT) + 1, (int32_t)HOLD_COUNT) : 0;
    h = (h & ~HOLD_COUNT) | cnt;
    if (cnt >= a.freeze_iters) {
        h |= HOLD_FROZEN;
        return true;
    }
    c[0] = cn[0];
    c[1] = cn[1];
    c[2] = cn[2];
    R = Rn;
    return false;
}

__device__ __forceinline__ bool rules_on(const EvolveArgs &a) { return a.freeze_iters > 0 || a.cull_iter > 0; }

// A non-finite evaluation (non-finite voxels) freezes the contour and is reported
// through the status word rather than pushed through the clamps.
__device__ __forceinline__ bool finite_step(const Step &s)
{
    return isfinite(s.E) && isfinite(s.dEdR) && isfinite(s.g[0]) && isfinite(s.g[1]) && isfinite(s.g[2]);
}

__device__ __forceinline__ void write_trace(const EvolveArgs &a, int vol, int64_t k, int n, const float *c, float R,
                                            const Step &s)
{
    if (a.trace == nullptr || vol != a.trace_vol || k < a.tk0 || k >= a.tk1 || n < a.tt0 || n >= a.tt1) return;
    float *t = a.trace + (((int64_t)(n - a.tt0) * (a.tk1 - a.tk0)) + (k - a.tk0)) * 9;
    t[0] = c[0]; t[1] = c[1]; t[2] = c[2]; t[3] = R;
    t[4] = s.E; t[5] = s.dEdR; t[6] = s.g[0]; t[7] = s.g[1]; t[8] = s.g[2];
}

template <int G> __device__ __forceinline__ unsigned group_mask()
{
    if (G == 32) return 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    return ((1u << (G & 31)) - 1u) << (lane & ~(unsigned)(G - 1));
}

// Votes over the whole warp.  With one contour per warp (G = 32) its lanes agree
// already, so the vote is the lane's own value.
template <int G> __device__ __forceinline__ bool warp_any(bool p)
{
    if constexpr (G == 32) return p;
    else return __any_sync(0xffffffffu, p);
}
template <int G> __device__ __forceinline__ bool warp_all(bool p)
{
    if constexpr (G == 32) return p;
    else return __all_sync(0xffffffffu, p);
}

// Evaluate one contour-iteration with the chosen gather, reduce over the group.
template <int DIM, int G, bool COMP, bool ACC, typename Gather>
__device__ __forceinline__ Step eval_contour(const Gather &gat, const IterC<DIM> &ic, float R, const EvolveArgs &a,
                                             int n, uint32_t k, uint32_t stream, float scale, int lig, unsigned mask)
{
    Acc acc;
    acc.a.s = acc.a.c = acc.b.s = acc.b.c = make_float2(0.0f, 0.0f);
    acc.c.s = acc.c.c = 0.0f;
    sample_contour<DIM, G, COMP, ACC>(gat, ic, a, (uint32_t)n, k, stream, lig, acc);
    const KSum k5[5] = {{acc.a.s.x, acc.a.c.x}, {acc.a.s.y, acc.a.c.y}, {acc.b.s.x, acc.b.c.x},
                        {acc.b.s.y, acc.b.c.y}, {acc.c.s, acc.c.c}};
    float sums[5];
    sums[4] = 0.0f;
    group_reduce_all<G, COMP, DIM == 3 ? 5 : 4>(k5, sums, mask);
    return finish<DIM>(sums, R, a, scale);
}

__device__ __forceinline__ int find_vol(const EvolveArgs &a, int64_t idx, bool by_brick)
{
    int v = 0;
    for (int i = 1; i < a.n_vols; ++i)
        if ((by_brick ? a.vols[i].brick_base : a.vols[i].contour_base) <= idx) v = i;
    return v;
}

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t *keys, int64_t n, uint32_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ----------------------------------------------------------------- brick kernel
// One CTA per brick: TMA stages the brick plus halo into shared memory once (2D:
// then rewritten as quads so one shared-memory load feeds a bilinear sample);
// each group of G lanes evolves one contour of the brick through all iterations
// with its state in registers ("Parallel Contour Evaluation": lanes share the
// samples of a contour).  Per iteration a group takes the fast path (ball inside
// the volume and the region), the clamped shared-memory path (ball crosses the
// volume border) or, when the ball has left the region, global-memory gathers.
template <int DIM, typename T, int G, bool COMP, bool ACC>
// Register caps: 96 in 2D lets two 10-warp CTAs share an SM; 128 in 3D, two
// 8-warp CTAs (or one of 16 warps).
__global__ void __maxnreg__(DIM == 2 ? 96 : 128) evolve_brick_kernel(const __grid_constant__ EvolveArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    using QT = typename QuadOf<T>::type;

    const int64_t b = blockIdx.x;
    const int64_t cb = lower_bound_u32(a.sorted_brick, a.total_contours, (uint32_t)b);
    const int64_t ce = lower_bound_u32(a.sorted_brick, a.total_contours, (uint32_t)(b + 1));
    if (cb == ce) return;   // empty brick (uniform over the CTA)

    const int v = find_vol(a, b, true);
    const VolDesc &V = a.vols[v];
    if (V.first_iter > V.last_iter) return;   // no iterations for this set in this launch
    const int64_t lb = b - V.brick_base;
    const int bxi = (int)(lb % V.nb[0]);
    const int byi = (int)((lb / V.nb[0]) % V.nb[1]);
    const int bzi = (int)(lb / ((int64_t)V.nb[0] * V.nb[1]));
    // region origin: max(0, brick - halo), x rounded down to the 16-byte TMA alignment
    constexpr int AL = 16 / (int)sizeof(T);
    const int r0[3] = {max(0, bxi * a.B[0] - a.halo[0]) / AL * AL, max(0, byi * a.B[1] - a.halo[1]),
                       DIM == 3 ? max(0, bzi * a.B[2] - a.halo[2]) : 0};

    // One thread issues the load and decides whether it landed within the bound, so
    // every thread of the CTA takes the same branch.  On giving up it records the
    // timeout and waits (again bounded) for the copy in flight, so that no copy is
    // still writing shared memory when the CTA exits.
    __shared__ int landed;
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&mbar, (uint32_t)a.raw_bytes);
        tma_load_3d(smem_raw, &a.tmaps[v], r0[0], r0[1], r0[2], &mbar);
        landed = mbar_wait_bounded(&mbar, 0, a.tma_polls) ? 1 : 0;
        if (!landed) {
            atomicOr(V.status, STATUS_TMA_TIMEOUT);
            mbar_wait_bounded(&mbar, 0, TMA_DRAIN_POLLS);
        }
    }
    __syncthreads();
    if (!landed) return;
    // each thread observes the completed phase itself (at once) before reading the region
    mbar_wait_bounded(&mbar, 0, TMA_DRAIN_POLLS);
    const T *reg = reinterpret_cast<const T *>(smem_raw);
    const bool quad = DIM == 2 && a.quad_off > 0;
    QT *Q = reinterpret_cast<QT *>(smem_raw + a.quad_off);
    const int qp = a.ext[0] - 1;
    if (quad) {
        const int nq = qp * (a.ext[1] - 1);
        for (int i = threadIdx.x; i < nq; i += blockDim.x) {
            const int y = i / qp, x = i - y * qp;
            const T *r = reg + y * a.ext[0] + x;
            const float v00 = to_f<T>(r[0]), v10 = to_f<T>(r[1]);
            const float v01 = to_f<T>(r[a.ext[0]]), v11 = to_f<T>(r[a.ext[0] + 1]);
            Q[i] = QuadOf<T>::diff ? make_quad<QT>(v00, v01, v10 - v00, v11 - v01) : make_quad<QT>(v00, v01, v10, v11);
        }
        __syncthreads();
    }

    const int py = a.ext[0], pz = a.ext[0] * a.ext[1];
    // base of the 32-bit tap addresses of the 3D fast path, biases folded (modulo 2^32)
    const uint32_t raw_C = smem_u32(smem_raw) - (uint32_t)sizeof(T) * 0x4B000000u * (uint32_t)(1 + py + pz);
    // the staged region's first and last usable tap per axis (within the volume)
    float fr_lo[3], fr_hi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        fr_lo[d] = (float)r0[d];
        fr_hi[d] = (float)min(V.n[d] - 1, r0[d] + a.ext[d] - 1);
    }
    const int nquads = qp * (a.ext[1] - 1);                       // extents for the checked build
    const int64_t nraw = (int64_t)a.ext[0] * a.ext[1] * a.ext[2];
    const int lig = threadIdx.x % G;
    const int grp = threadIdx.x / G;
    const int ngrp = blockDim.x / G;
    const int wsub = grp % (32 / G);   // this group's place among the groups of its warp
    const unsigned mask = group_mask<G>();
    const int64_t C = V.C;
    unsigned int n_fast = 0, n_clamped = 0, n_global = 0;   // this group's contour-iterations per gather path

    // The groups of a warp walk the brick's contours together (slots wi + wsub), so
    // that every lane of the warp reaches the per-iteration path votes below; a group
    // without a contour, or whose contour has stopped, idles through them.
    for (int64_t wi = cb + (grp - wsub); wi < ce; wi += ngrp) {
        const int64_t i = wi + wsub;
        bool live = i < ce;
        int64_t k = 0;
        int32_t h = 0;
        if (live) {
            k = (int64_t)a.sorted_gidx[i] - V.contour_base;
            h = V.hold ? V.hold[k] : 0;
            live = !(h & HOLD_STOPPED);   // stopped by a rule in an earlier call
        }
        const bool owned = live;          // this group writes the contour back
        float c[3] = {0.0f, 0.0f, 0.0f}, R = 0.0f;
        if (live) {
            c[0] = V.state[k];
            c[1] = V.state[C + k];
            if (DIM == 3) c[2] = V.state[2 * C + k];
            R = V.state[3 * C + k];
        }
        Step s = {0.0f, 0.0f, {0.0f, 0.0f, 0.0f}};
        for (int n = V.first_iter; n <= V.last_iter; ++n) {
            if (!warp_any<G>(live)) break;
            IterC<DIM> ic;
            bool inside = true, interior = true;
            int o[3] = {0, 0, 0};
            if (live) {
                iter_consts<DIM>(ic, c, R, V, a);
                // where do the taps of the whole ball fall (clamped like the samples)?
                const float Ro = R + 0.5f * a.dR;
                // fast path: every tap index ci + floor(cf - e) .. ci + floor(cf + e) + 1
                // inside the volume and the staged region, i.e. per axis
                // cf - e >= r0 - ci and cf + e < min(n - 1, r0 + ext - 1) - ci (lo = -ci)
                // (3D; in 2D the full test below is as cheap)
                bool fast = DIM == 3;
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const AxisSplit &x = ic.ax[d];
                    const float e = fmaf(Ro, V.inv_sp[d], 1e-3f);
                    fast = fast && (x.cf - e >= fr_lo[d] + x.lo) && (x.cf + e < fr_hi[d] + x.lo);
                }
                inside = fast;
                interior = fast;
                if (!fast) {
                    inside = true;
                    interior = true;
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        const AxisSplit &x = ic.ax[d];
                        const float e = fmaf(Ro, V.inv_sp[d], 1e-3f);
                        interior = interior && (x.cf - e >= x.lo) && (x.cf + e < x.hi);
                        const float lo = fminf(fmaxf(x.cf - e, x.lo), x.hi);
                        const float hi = fminf(fmaxf(x.cf + e, x.lo), x.hi);
                        const int tlo = x.ci + (int)fminf(floorf(lo), x.top);
                        const int thi = x.ci + (int)fminf(floorf(hi), x.top) + 1;
                        inside = inside && tlo >= r0[d] && thi < r0[d] + a.ext[d];
                    }
                }
                o[0] = ic.ax[0].ci - r0[0];
                o[1] = ic.ax[1].ci - r0[1];
                o[2] = DIM == 3 ? ic.ax[2].ci - r0[2] : 0;
            }
            // Several contours per warp take the slowest path any of them needs (every
            // path gives the same bits), so their lanes never run two paths in turn.
            const bool use_fast = warp_all<G>(inside && interior);
            const bool use_smem = warp_all<G>(inside);
            if (!live) continue;
            n_fast += use_fast ? 1u : 0u;
            n_clamped += (use_smem && !use_fast) ? 1u : 0u;
            n_global += use_smem ? 0u : 1u;
            if (use_fast) {
                const float M[3] = {8388608.0f + (float)o[0], 8388608.0f + (float)o[1], 8388608.0f + (float)o[2]};
                if (quad) {
                    QuadFast<QT, QuadOf<T>::diff> gat{Q, qp, {M[0], M[1]}, nquads, V.status};
                    s = eval_contour<DIM, G, COMP, ACC>(gat, ic, R, a, n, (uint32_t)k, V.stream, V.scale, lig, mask);
                } else {
#ifndef AC_CHECKED
                    if constexpr (DIM == 3) {   // 32-bit shared addresses, biases folded into raw_C
                        RawFast3S<T> gat{raw_C, (uint32_t)(sizeof(T) * py), (uint32_t)(sizeof(T) * pz),
                                         {M[0], M[1], M[2]}};
                        s = eval_contour<DIM, G, COMP, ACC>(gat, ic, R, a, n, (uint32_t)k, V.stream, V.scale, lig,
                                                            mask);
                    } else
#endif
                    {
                        RawFast<DIM, T> gat{reg, py, pz, {M[0], M[1], M[2]}, nraw, V.status};
                        s = eval_contour<DIM, G, COMP, ACC>(gat, ic, R, a, n, (uint32_t)k, V.stream, V.scale, lig,
                                                            mask);
                    }
                }
            } else if (use_smem) {
                if (quad) {
                    SmemClamp<DIM, T, true> gat{Q, qp, 0, {ic.ax[0], ic.ax[1], ic.ax[2]}, {o[0], o[1], o[2]},
                                                nquads, V.status};
                    s = eval_contour<DIM, G, COMP, ACC>(gat, ic, R, a, n, (uint32_t)k, V.stream, V.scale, lig, mask);
                } else {
                    SmemClamp<DIM, T, false> gat{reg, py, pz, {ic.ax[0], ic.ax[1], ic.ax[2]}, {o[0], o[1], o[2]},
                                                 nraw, V.status};
                    s = eval_contour<DIM, G, COMP, ACC>(gat, ic, R, a, n, (uint32_t)k, V.stream, V.scale, lig, mask);
                }
            } else {
                GlobalClamp<DIM, T> gat{reinterpret_cast<const T *>(V.data), V.pitch_y, V.pitch_z,
                                        {ic.ax[0], ic.ax[1], ic.ax[2]}, V.pitch_z * V.n[2], V.status};
                s = eval_contour<DIM, G, COMP, ACC>(gat, ic, R, a, n, (uint32_t)k, V.stream, V.scale, lig, mask);
            }
            if (lig == 0) write_trace(a, v, k, n, c, R, s);
            if (!finite_step(s)) {
                if (lig == 0) atomicOr(V.status, STATUS_NONFINITE);
                live = false;
            } else if (step_or_stop<DIM>(s, n, a, V, c, R, h)) {
                live = false;
            }
        }
        if (owned && lig == 0) {
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
    // one atomic per warp and path: sum the groups' counts over the warp
    const unsigned int cnt[3] = {n_fast, n_clamped, n_global};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const unsigned int tot = __reduce_add_sync(0xffffffffu, lig == 0 ? cnt[p] : 0u);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&a.path_counts[p], (unsigned long long)tot);
    }
}

// ----------------------------------------------------------------- plain kernel
// One iteration (a.iter0) for every contour: state read from and written back to
// global memory, samples gathered from the global volume.  Launched T times.
template <int DIM, typename T, int G, bool COMP, bool ACC>
__global__ void __launch_bounds__(256) evolve_plain_kernel(const __grid_constant__ EvolveArgs a)
{
    unsigned int glob = 0;
    const int lig = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    const int n = a.iter0;
    // every contour, or only those of a compacted list (contours still running after
    // a stopping rule)
    const int64_t items = a.active ? (int64_t)*a.n_active : a.total_contours;
    for (int64_t it = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; it < items; it += groups) {
        const int64_t gi = a.active ? (int64_t)a.active[it] : it;
        const int v = find_vol(a, gi, false);
        const VolDesc &V = a.vols[v];
        if (n < V.first_iter || n > V.last_iter) continue;   // outside this set's iterations
        const int64_t k = gi - V.contour_base;
        const int64_t C = V.C;
        int32_t h = V.hold ? V.hold[k] : 0;
        if (h & HOLD_STOPPED) continue;
        float c[3] = {V.state[k], V.state[C + k], DIM == 3 ? V.state[2 * C + k] : 0.0f};
        float R = V.state[3 * C + k];
        IterC<DIM> ic;
        iter_consts<DIM>(ic, c, R, V, a);
        GlobalClamp<DIM, T> gat{reinterpret_cast<const T *>(V.data), V.pitch_y, V.pitch_z,
                                {ic.ax[0], ic.ax[1], ic.ax[2]}, V.pitch_z * V.n[2], V.status};
        const Step s = eval_contour<DIM, G, COMP, ACC>(gat, ic, R, a, n, (uint32_t)k, V.stream, V.scale, lig, mask);
        if (lig == 0) {
            ++glob;
            write_trace(a, v, k, n, c, R, s);
            if (!finite_step(s)) atomicOr(V.status, STATUS_NONFINITE);
            else step_or_stop<DIM>(s, n, a, V, c, R, h);
            if (V.hold && rules_on(a)) V.hold[k] = h;
            V.state[k] = c[0];
            V.state[C + k] = c[1];
            if (DIM == 3) V.state[2 * C + k] = c[2];
            V.state[3 * C + k] = R;
            V.state[4 * C + k] = s.E;
            if (!(isfinite(s.E) && isfinite(R)))
                atomicOr(V.status, STATUS_NONFINITE);
        }
    }
    const unsigned int tot = __reduce_add_sync(0xffffffffu, glob);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&a.path_counts[2], (unsigned long long)tot);
}

// ----------------------------------------------------------------- launchers
template <int DIM, typename T, int G, bool COMP, bool ACC>
cudaError_t launch_brick_t(const EvolveArgs &a, int warps, cudaStream_t st)
{
    auto kern = evolve_brick_kernel<DIM, T, G, COMP, ACC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)a.total_bricks, warps * 32, a.smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <int DIM, typename T, int G, bool COMP, bool ACC>
cudaError_t launch_plain_t(const EvolveArgs &a, int warps, int64_t grid, cudaStream_t st)
{
    evolve_plain_kernel<DIM, T, G, COMP, ACC><<<(unsigned)grid, warps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

// Instantiated combinations: 8, 16 and 32 lanes with compensated sums in the fast
// and the accurate sampling mode and with plain FP32 sums in the fast mode, and 4
// lanes with compensated sums in the fast mode.
template <typename T>
cudaError_t launch_evolve_t(const EvolveArgs &a, bool brick, int G, bool comp, bool acc, int warps, int64_t grid,
                            cudaStream_t st)
{
#define AC_DISPATCH(DIM, GG, CC, AA)                                                                \
    if (a.ndim == DIM && G == GG && comp == CC && acc == AA)                                       \
        return brick ? launch_brick_t<DIM, T, GG, CC, AA>(a, warps, st)                            \
                     : launch_plain_t<DIM, T, GG, CC, AA>(a, warps, grid, st);
#define AC_DISPATCH_G(DIM, CC, AA) AC_DISPATCH(DIM, 32, CC, AA) AC_DISPATCH(DIM, 16, CC, AA) AC_DISPATCH(DIM, 8, CC, AA)
    AC_DISPATCH_G(3, true, false) AC_DISPATCH_G(3, false, false) AC_DISPATCH_G(3, true, true)
    AC_DISPATCH_G(2, true, false) AC_DISPATCH_G(2, false, false) AC_DISPATCH_G(2, true, true)
    AC_DISPATCH(2, 4, true, false) AC_DISPATCH(3, 4, true, false)
#undef AC_DISPATCH_G
#undef AC_DISPATCH
    return cudaErrorInvalidValue;
}

}  // namespace ac
