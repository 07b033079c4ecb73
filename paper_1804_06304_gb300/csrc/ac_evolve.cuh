// ac_evolve.cuh -- Monte-Carlo snakuscule evolution kernels (stages a3-a8).
// Included once per voxel type by ac_evolve_<type>.cu so the instantiations
// compile in parallel.  Method: arXiv:1804.06304, Eqs. 5-15 and the
// "Monte-Carlo Integration" / "Parallel Contour Evaluation" sections.
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

// ----------------------------------------------------------------- gathers
// Staged region in shared memory: dense [ez][ey][ex] elements.
template <typename T> struct SmemGather {
    const T *p;
    int py, pz;       // region pitches in elements
    int ox, oy, oz;   // centre voxel relative to the region origin

    template <int DIM>
    __device__ __forceinline__ float at(int bx, int by, int bz, float fx, float fy, float fz) const
    {
        const T *q = p + (ox + bx) + (oy + by) * py + (DIM == 3 ? (oz + bz) * pz : 0);
        const float v00 = to_f<T>(q[0]), v10 = to_f<T>(q[1]);
        const float v01 = to_f<T>(q[py]), v11 = to_f<T>(q[py + 1]);
        const float a0 = fmaf(fx, v10 - v00, v00), a1 = fmaf(fx, v11 - v01, v01);
        const float s0 = fmaf(fy, a1 - a0, a0);
        if (DIM == 2) return s0;
        const T *r = q + pz;
        const float w00 = to_f<T>(r[0]), w10 = to_f<T>(r[1]);
        const float w01 = to_f<T>(r[py]), w11 = to_f<T>(r[py + 1]);
        const float b0 = fmaf(fx, w10 - w00, w00), b1 = fmaf(fx, w11 - w01, w01);
        const float s1 = fmaf(fy, b1 - b0, b0);
        return fmaf(fz, s1 - s0, s0);
    }
};

// The row-pitched volume in global memory (read-only path).
template <typename T> struct GlobalGather {
    const T *p;
    int64_t py, pz;
    int ci, cj, ck;   // centre voxel

    template <int DIM>
    __device__ __forceinline__ float at(int bx, int by, int bz, float fx, float fy, float fz) const
    {
        const T *q = p + (int64_t)(ci + bx) + (int64_t)(cj + by) * py + (DIM == 3 ? (int64_t)(ck + bz) * pz : 0);
        const float v00 = ldg_f<T>(q), v10 = ldg_f<T>(q + 1);
        const float v01 = ldg_f<T>(q + py), v11 = ldg_f<T>(q + py + 1);
        const float a0 = fmaf(fx, v10 - v00, v00), a1 = fmaf(fx, v11 - v01, v01);
        const float s0 = fmaf(fy, a1 - a0, a0);
        if (DIM == 2) return s0;
        const T *r = q + pz;
        const float w00 = ldg_f<T>(r), w10 = ldg_f<T>(r + 1);
        const float w01 = ldg_f<T>(r + py), w11 = ldg_f<T>(r + py + 1);
        const float b0 = fmaf(fx, w10 - w00, w00), b1 = fmaf(fx, w11 - w01, w01);
        const float s1 = fmaf(fy, b1 - b0, b0);
        return fmaf(fz, s1 - s0, s0);
    }
};

// ----------------------------------------------------------------- one sample
// Adds the sample at distance r along unit direction dir to the five sums
// J = sum S I, J_R = sum dS/dR I, J_c = sum -S'(r) dir I (Eqs. 5, 7-10).
template <int DIM, bool COMP, typename Gather>
__device__ __forceinline__ void add_sample(const Gather &gat, const AxisSplit *ax, const float *inv_sp,
                                           const WeightConsts &W, float r, float dx, float dy, float dz,
                                           KSum *acc)
{
    int bx, by, bz = 0;
    float fx, fy, fz = 0.0f;
    axis_tap(ax[0], r * dx * inv_sp[0], bx, fx);
    axis_tap(ax[1], r * dy * inv_sp[1], by, fy);
    if (DIM == 3) axis_tap(ax[2], r * dz * inv_sp[2], bz, fz);
    const float I = gat.template at<DIM>(bx, by, bz, fx, fy, fz);

    const float t1 = fmaf(r, W.a1, W.b1), t2 = fmaf(r, W.a2, W.b2);
    const float S = fmaf(2.0f, __saturatef(t1), -1.0f) - __saturatef(t2);
    const float in1 = (t1 >= 0.0f && t1 < 1.0f) ? 1.0f : 0.0f;
    const float in2 = (t2 >= 0.0f && t2 < 1.0f) ? 1.0f : 0.0f;
    const float dSdR = fmaf(in1, W.kR1, in2 * W.kR2);
    const float g = fmaf(in1, W.kr1, in2 * W.kr2) * I;   // -S'(r) I
    if (COMP) {
        kadd(acc[0], S * I);
        kadd(acc[1], dSdR * I);
        kadd(acc[2], g * dx);
        kadd(acc[3], g * dy);
        if (DIM == 3) kadd(acc[4], g * dz);
    } else {
        acc[0].s = fmaf(S, I, acc[0].s);
        acc[1].s = fmaf(dSdR, I, acc[1].s);
        acc[2].s = fmaf(g, dx, acc[2].s);
        acc[3].s = fmaf(g, dy, acc[3].s);
        if (DIM == 3) acc[4].s = fmaf(g, dz, acc[4].s);
    }
}

// All samples of one contour-iteration handled by this lane (lane `lig` of G).
// 3D: sample j uses Philox block (j, n, k, stream): radius cbrt(u0), cos(phi) =
// 1 - 2 u1, azimuth 2 pi u2.  2D: block m gives samples 2m and 2m+1, radius
// sqrt(u), azimuth 2 pi u' ("Monte-Carlo Integration" section).
template <int DIM, int G, bool COMP, typename Gather>
__device__ __forceinline__ void sample_contour(const Gather &gat, const AxisSplit *ax, const float *inv_sp,
                                               const WeightConsts &W, float Ro, int N, uint32_t n, uint32_t k,
                                               uint32_t stream, uint32_t key0, uint32_t key1, int lig,
                                               KSum *acc)
{
    if (DIM == 3) {
#pragma unroll 2
        for (int j = lig; j < N; j += G) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)j, n, k, stream), key0, key1);
            const float u1 = u24(w.y);
            const float rad = cbrtf(u24(w.x));
            const float cphi = fmaf(-2.0f, u1, 1.0f);
            const float sphi = 2.0f * sqrtf(u1 * (1.0f - u1));
            float sn, cs;
            sincospif(2.0f * u24(w.z), &sn, &cs);
            add_sample<3, COMP>(gat, ax, inv_sp, W, Ro * rad, sphi * cs, sphi * sn, cphi, acc);
        }
    } else {
        const int blocks = (N + 1) >> 1;
        for (int m = lig; m < blocks; m += G) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)m, n, k, stream), key0, key1);
            {
                float sn, cs;
                sincospif(2.0f * u24(w.y), &sn, &cs);
                add_sample<2, COMP>(gat, ax, inv_sp, W, Ro * sqrtf(u24(w.x)), cs, sn, 0.0f, acc);
            }
            if (2 * m + 1 < N) {
                float sn, cs;
                sincospif(2.0f * u24(w.w), &sn, &cs);
                add_sample<2, COMP>(gat, ax, inv_sp, W, Ro * sqrtf(u24(w.z)), cs, sn, 0.0f, acc);
            }
        }
    }
}

// ----------------------------------------------------------------- finish + step
struct Step {
    float E, dEdR, g[3];
};

// Sums to energy and gradient (Eqs. 5-11, centre/radius form).
template <int DIM>
__device__ __forceinline__ Step finish(const float *sums, float R, float dR, int N, float scale)
{
    const float Ro = R + 0.5f * dR;
    const float V = DIM == 3 ? 4.18879020478639098461f * Ro * Ro * Ro : 3.14159265358979323846f * Ro * Ro;
    const float wmc = V / (float)N * scale;
    const float twoR = 2.0f * R;
    const float inv = DIM == 3 ? 1.0f / (twoR * twoR * twoR) : 1.0f / (twoR * twoR);
    Step s;
    const float J = sums[0] * wmc;
    s.E = J * inv;
    s.dEdR = (sums[1] * wmc - (float)DIM * J / R) * inv;
    s.g[0] = sums[2] * wmc * inv;
    s.g[1] = sums[3] * wmc * inv;
    s.g[2] = DIM == 3 ? sums[4] * wmc * inv : 0.0f;
    return s;
}

// Eqs. 12-15 in centre/radius form: c -= eps_n/2 dE/dc, R -= eps_n/2 dE/dR, with
// the step, radius and box clamps.
template <int DIM>
__device__ __forceinline__ void update(const Step &s, int n, const EvolveArgs &a, const float *box_hi, float *c,
                                       float &R)
{
    const float eta = 0.5f * a.eps0 / sqrtf((float)n);
    float d[3] = {-eta * s.g[0], -eta * s.g[1], DIM == 3 ? -eta * s.g[2] : 0.0f};
    const float nrm = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (nrm > a.max_step) {
        const float f = a.max_step / nrm;
        d[0] *= f;
        d[1] *= f;
        d[2] *= f;
    }
    const float dRr = fminf(fmaxf(-eta * s.dEdR, -a.max_step), a.max_step);
    R = fminf(fmaxf(R + dRr, a.Rmin), a.Rmax);
#pragma unroll
    for (int i = 0; i < DIM; ++i) c[i] = fminf(fmaxf(c[i] + d[i], 0.0f), box_hi[i]);
}

__device__ __forceinline__ void write_trace(const EvolveArgs &a, int vol, int64_t k, int n, const float *c, float R,
                                            const Step &s)
{
    if (a.trace == nullptr || vol != 0 || k < a.tk0 || k >= a.tk1 || n < a.tt0 || n >= a.tt1) return;
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

// Evaluate one contour-iteration with the chosen gather, reduce over the group.
template <int DIM, int G, bool COMP, typename Gather>
__device__ __forceinline__ Step eval_contour(const Gather &gat, const AxisSplit *ax, const float *inv_sp,
                                             float R, const EvolveArgs &a, int n, uint32_t k, uint32_t key0,
                                             uint32_t key1, float scale, int lig, unsigned mask)
{
    const float Ro = R + 0.5f * a.dR;
    const WeightConsts W = weight_consts(R, a.dR, DIM);
    KSum acc[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
    sample_contour<DIM, G, COMP>(gat, ax, inv_sp, W, Ro, a.N, (uint32_t)n, k, a.stream_id, key0, key1, lig, acc);
    float sums[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) sums[i] = (DIM == 2 && i == 4) ? 0.0f : group_reduce<G, COMP>(acc[i], mask);
    return finish<DIM>(sums, R, a.dR, a.N, scale);
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
// One CTA per brick: TMA stages the brick plus halo into shared memory once; each
// group of G lanes then evolves one contour of the brick through all T iterations
// with its state in registers ("Parallel Contour Evaluation": lanes share the
// samples of a contour).  A contour whose ball leaves the staged region gathers
// from global memory for that iteration (the branch is uniform per group).
template <int DIM, typename T, int G, bool COMP>
__global__ void __launch_bounds__(256) evolve_brick_kernel(const EvolveArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;

    const int64_t b = blockIdx.x;
    const int64_t cb = lower_bound_u32(a.sorted_brick, a.total_contours, (uint32_t)b);
    const int64_t ce = lower_bound_u32(a.sorted_brick, a.total_contours, (uint32_t)(b + 1));
    if (cb == ce) return;   // empty brick (uniform over the CTA)

    const int v = find_vol(a, b, true);
    const VolDesc &V = a.vols[v];
    const int64_t lb = b - V.brick_base;
    const int bxi = (int)(lb % V.nb[0]);
    const int byi = (int)((lb / V.nb[0]) % V.nb[1]);
    const int bzi = (int)(lb / ((int64_t)V.nb[0] * V.nb[1]));
    // region origin: max(0, brick - halo), x rounded down to the 16-byte TMA alignment
    constexpr int AL = 16 / (int)sizeof(T);
    const int r0x = max(0, bxi * a.B[0] - a.halo[0]) / AL * AL;
    const int r0y = max(0, byi * a.B[1] - a.halo[1]);
    const int r0z = DIM == 3 ? max(0, bzi * a.B[2] - a.halo[2]) : 0;

    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&mbar, (uint32_t)a.smem_bytes);
        tma_load_3d(smem_raw, &a.tmaps[v], r0x, r0y, r0z, &mbar);
    }
    if (!mbar_wait_bounded(&mbar, 0, 1u << 22)) {
        if (threadIdx.x == 0) atomicOr(a.status, STATUS_TMA_TIMEOUT);
        mbar_wait_bounded(&mbar, 0, 1u << 22);   // let an in-flight copy land before exit
        return;
    }

    const T *reg = reinterpret_cast<const T *>(smem_raw);
    const int py = a.ext[0], pz = a.ext[0] * a.ext[1];
    const float inv_sp[3] = {V.inv_sp[0], V.inv_sp[1], V.inv_sp[2]};
    const int lig = threadIdx.x % G;
    const int grp = threadIdx.x / G;
    const int ngrp = blockDim.x / G;
    const unsigned mask = group_mask<G>();
    const int64_t C = V.C;

    for (int64_t i = cb + grp; i < ce; i += ngrp) {
        const int64_t k = (int64_t)a.sorted_gidx[i] - V.contour_base;
        float c[3] = {V.state[k], V.state[C + k], DIM == 3 ? V.state[2 * C + k] : 0.0f};
        float R = V.state[3 * C + k];
        Step s;
        for (int n = a.first_iter; n <= a.last_iter; ++n) {
            AxisSplit ax[3];
#pragma unroll
            for (int d = 0; d < DIM; ++d) ax[d] = split_axis(c[d], V.sp[d], inv_sp[d], V.n[d]);
            // taps of the whole ball, clamped like the samples: inside the region?
            const float Ro = R + 0.5f * a.dR;
            bool inside = true;
            const int r0[3] = {r0x, r0y, r0z};
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const float e = fmaf(Ro, inv_sp[d], 1e-3f);
                const float lo = fminf(fmaxf(ax[d].cf - e, ax[d].lo), ax[d].hi);
                const float hi = fminf(fmaxf(ax[d].cf + e, ax[d].lo), ax[d].hi);
                const int tlo = ax[d].ci + (int)fminf(floorf(lo), ax[d].top);
                const int thi = ax[d].ci + (int)fminf(floorf(hi), ax[d].top) + 1;
                inside = inside && tlo >= r0[d] && thi < r0[d] + a.ext[d];
            }
            if (inside) {
                SmemGather<T> gat{reg, py, pz, ax[0].ci - r0x, ax[1].ci - r0y, DIM == 3 ? ax[2].ci - r0z : 0};
                s = eval_contour<DIM, G, COMP>(gat, ax, inv_sp, R, a, n, (uint32_t)k, V.key0, V.key1, V.scale,
                                               lig, mask);
            } else {
                GlobalGather<T> gat{reinterpret_cast<const T *>(V.data), V.pitch_y, V.pitch_z, ax[0].ci, ax[1].ci,
                                    DIM == 3 ? ax[2].ci : 0};
                s = eval_contour<DIM, G, COMP>(gat, ax, inv_sp, R, a, n, (uint32_t)k, V.key0, V.key1, V.scale,
                                               lig, mask);
            }
            if (lig == 0) write_trace(a, v, k, n, c, R, s);
            if (n < a.last_iter || a.update_last) update<DIM>(s, n, a, V.box_hi, c, R);
        }
        if (lig == 0) {
            V.state[k] = c[0];
            V.state[C + k] = c[1];
            if (DIM == 3) V.state[2 * C + k] = c[2];
            V.state[3 * C + k] = R;
            V.state[4 * C + k] = s.E;
            if (!(isfinite(s.E) && isfinite(R) && isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2])))
                atomicOr(a.status, STATUS_NONFINITE);
        }
    }
}

// ----------------------------------------------------------------- plain kernel
// One iteration (a.iter0) for every contour: state read from and written back to
// global memory, samples gathered from the global volume.  Launched T times.
template <int DIM, typename T, int G, bool COMP>
__global__ void __launch_bounds__(256) evolve_plain_kernel(const EvolveArgs a)
{
    const int lig = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    const int n = a.iter0;
    for (int64_t gi = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; gi < a.total_contours; gi += groups) {
        const int v = find_vol(a, gi, false);
        const VolDesc &V = a.vols[v];
        const int64_t k = gi - V.contour_base;
        const int64_t C = V.C;
        float c[3] = {V.state[k], V.state[C + k], DIM == 3 ? V.state[2 * C + k] : 0.0f};
        float R = V.state[3 * C + k];
        const float inv_sp[3] = {V.inv_sp[0], V.inv_sp[1], V.inv_sp[2]};
        AxisSplit ax[3];
#pragma unroll
        for (int d = 0; d < DIM; ++d) ax[d] = split_axis(c[d], V.sp[d], inv_sp[d], V.n[d]);
        GlobalGather<T> gat{reinterpret_cast<const T *>(V.data), V.pitch_y, V.pitch_z, ax[0].ci, ax[1].ci,
                            DIM == 3 ? ax[2].ci : 0};
        const Step s = eval_contour<DIM, G, COMP>(gat, ax, inv_sp, R, a, n, (uint32_t)k, V.key0, V.key1, V.scale,
                                                  lig, mask);
        if (lig == 0) {
            write_trace(a, v, k, n, c, R, s);
            if (n < a.last_iter || a.update_last) update<DIM>(s, n, a, V.box_hi, c, R);
            V.state[k] = c[0];
            V.state[C + k] = c[1];
            if (DIM == 3) V.state[2 * C + k] = c[2];
            V.state[3 * C + k] = R;
            V.state[4 * C + k] = s.E;
            if (!(isfinite(s.E) && isfinite(R)))
                atomicOr(a.status, STATUS_NONFINITE);
        }
    }
}

// ----------------------------------------------------------------- launchers
template <int DIM, typename T, int G, bool COMP>
cudaError_t launch_brick_t(const EvolveArgs &a, int warps, cudaStream_t st)
{
    auto kern = evolve_brick_kernel<DIM, T, G, COMP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)a.total_bricks, warps * 32, a.smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <int DIM, typename T, int G, bool COMP>
cudaError_t launch_plain_t(const EvolveArgs &a, int warps, int64_t grid, cudaStream_t st)
{
    evolve_plain_kernel<DIM, T, G, COMP><<<(unsigned)grid, warps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_evolve_t(const EvolveArgs &a, bool brick, int G, bool comp, int warps, int64_t grid,
                            cudaStream_t st)
{
#define AC_DISPATCH(DIM, GG, CC)                                                                    \
    if (a.ndim == DIM && G == GG && comp == CC)                                                     \
        return brick ? launch_brick_t<DIM, T, GG, CC>(a, warps, st) : launch_plain_t<DIM, T, GG, CC>(a, warps, grid, st);
    AC_DISPATCH(3, 32, true) AC_DISPATCH(3, 16, true) AC_DISPATCH(3, 8, true)
    AC_DISPATCH(3, 32, false) AC_DISPATCH(3, 16, false) AC_DISPATCH(3, 8, false)
    AC_DISPATCH(2, 32, true) AC_DISPATCH(2, 16, true) AC_DISPATCH(2, 8, true)
    AC_DISPATCH(2, 32, false) AC_DISPATCH(2, 16, false) AC_DISPATCH(2, 8, false)
#undef AC_DISPATCH
    return cudaErrorInvalidValue;
}

}  // namespace ac
