// ac_api.cu -- C ABI of libac: volumes, seeding, evolution orchestration, state.
// Method: Lotfollahi et al., arXiv:1804.06304 (see include/ac.h for the mapping of
// each entry point to the paper).
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <cub/cub.cuh>
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "ac_host.h"

namespace ac {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
static std::atomic<int64_t> g_launches{0};
void count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void Scratch::release_all()
{
    DevBuf *all[] = {&keys, &vals, &skeys, &svals, &cub, &desc, &tmaps, &active, &flags, &surv, &ekeys, &surv_sorted,
                     &pos, &cellk, &celli, &cellk_s, &celli_s, &cell_start, &stat, &acc, &cells, &counters};
    for (DevBuf *b : all) b->release();
    lsets.release();
    und.release();
    hcount.release();
    hcells.release();
    hsets.release();
}

}  // namespace ac

using namespace ac;

static int elem_size(ac_dtype t)
{
    switch (t) {
    case AC_U8: return 1;
    case AC_U16: return 2;
    case AC_F16: return 2;
    case AC_F32: return 4;
    }
    return 0;
}

extern "C" const char *ac_last_error(void) { return g_err.c_str(); }

// Wait bounds that tests may shorten (ac_set_wait_limits); negative = default.
static std::atomic<int64_t> g_tma_polls{-1};
static std::atomic<int64_t> g_localize_rounds{-1};
uint32_t ac::tma_poll_limit()
{
    const int64_t v = g_tma_polls.load();
    return v < 0 ? TMA_POLLS_DEFAULT : (uint32_t)std::min<int64_t>(v, TMA_POLLS_DEFAULT);
}
int64_t ac::localize_round_limit(int64_t n)
{
    const int64_t v = g_localize_rounds.load();
    return v < 0 ? n + 8 : v;
}
extern "C" ac_status ac_set_wait_limits(int64_t tma_polls, int64_t localize_rounds)
{
    g_tma_polls.store(tma_polls < 0 ? -1 : tma_polls);
    g_localize_rounds.store(localize_rounds < 0 ? -1 : localize_rounds);
    return AC_OK;
}

extern "C" int64_t ac_kernel_launches(void) { return g_launches.load(); }

// Clamp a centre coordinate into the box of voxel centres of one axis.
static float clamp_box(float c, const ac_volume *v, int d)
{
    const float hi = (float)((double)(v->n[d] - 1) * v->sp[d]);
    return c < 0.0f ? 0.0f : (c > hi ? hi : c);
}

namespace {
// The row-pitched copy of a device array with element strides (1, rs, ps):
// block row blockIdx.y is plane z0 + blockIdx.y, threads run over its elements.
template <typename E>
__global__ void repack_kernel(const E *src, int64_t rs, int64_t ps, E *dst, int64_t pitch_y, int64_t nx, int64_t ny,
                              int64_t z0)
{
    const int64_t z = z0 + blockIdx.y;
    const int64_t plane = nx * ny;
    const E *s = src + z * ps;
    E *d = dst + z * ny * pitch_y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = plane < ((int64_t)1 << 32) ? (int64_t)((uint32_t)i / (uint32_t)nx) : i / nx;
        const int64_t x = i - y * nx;
        d[y * pitch_y + x] = s[y * rs + x];
    }
}

template <typename E>
cudaError_t repack_t(const ac_volume *v, const void *src, int64_t rs, int64_t ps, cudaStream_t st)
{
    const int64_t plane = v->n[0] * v->n[1];
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((plane + 255) / 256, 2048));
    for (int64_t z0 = 0; z0 < v->n[2]; z0 += 65535) {
        const unsigned gy = (unsigned)std::min<int64_t>(65535, v->n[2] - z0);
        repack_kernel<E><<<dim3(gx, gy), 256, 0, st>>>(static_cast<const E *>(src), rs, ps, static_cast<E *>(v->data),
                                                       v->pitch_y, v->n[0], v->n[1], z0);
        count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t repack(const ac_volume *v, const void *src, int64_t rs, int64_t ps, cudaStream_t st)
{
    switch (v->es) {
    case 1: return repack_t<uint8_t>(v, src, rs, ps, st);
    case 2: return repack_t<uint16_t>(v, src, rs, ps, st);
    default: return repack_t<uint32_t>(v, src, rs, ps, st);
    }
}
}  // namespace

// Copy voxels with element strides (1, row_stride, plane_stride) into the
// row-pitched device copy of `v`.  Device voxels are repacked by a kernel.  Dense
// host voxels whose rows need padding go up in one contiguous copy and are
// repacked on the device (a 2D copy of short rows runs at a few GB/s): through a
// stream-ordered temporary when a volume is created, through a staging buffer
// that the volume keeps when voxels are loaded again (`keep_staging`); volumes of
// a request loop (allocated from its pool) copy row by row instead, so that they
// hold no memory beyond what the loop's budget charges.  Strided host voxels are
// copied row by row.
static cudaError_t copy_voxels(ac_volume *v, const void *data, int data_on_device, int64_t row_stride,
                               int64_t plane_stride, cudaStream_t st, bool keep_staging)
{
    const int64_t *n = v->n;
    const int es = v->es;
    const size_t row_bytes = (size_t)n[0] * es;
    const size_t pitch = (size_t)v->pitch_y * es;
    const cudaMemcpyKind kind = data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const char *src = (const char *)data;
    const bool dense = row_stride == n[0] && plane_stride == row_stride * n[1];
    if (pitch == row_bytes && dense) return cudaMemcpyAsync(v->data, src, v->bytes, kind, st);
    if (data_on_device) return repack(v, data, row_stride, plane_stride, st);
    if (dense && !v->pool) {
        const size_t dense_bytes = row_bytes * (size_t)n[1] * (size_t)n[2];
        cudaError_t e;
        if (keep_staging) {
            if (v->staging_bytes < dense_bytes) {
                if (v->staging) cudaFree(v->staging);
                v->staging = nullptr;
                v->staging_bytes = 0;
                if ((e = cudaMalloc(&v->staging, dense_bytes)) != cudaSuccess) return e;
                v->staging_bytes = dense_bytes;
            }
            if ((e = cudaMemcpyAsync(v->staging, src, dense_bytes, kind, st)) != cudaSuccess) return e;
            return repack(v, v->staging, n[0], n[0] * n[1], st);
        }
        void *tmp = nullptr;
        if ((e = cudaMallocAsync(&tmp, dense_bytes, st)) != cudaSuccess) return e;
        e = cudaMemcpyAsync(tmp, src, dense_bytes, kind, st);
        if (e == cudaSuccess) e = repack(v, tmp, n[0], n[0] * n[1], st);
        const cudaError_t f = cudaFreeAsync(tmp, st);
        return e != cudaSuccess ? e : f;
    }
    if (plane_stride == row_stride * n[1])
        return cudaMemcpy2DAsync(v->data, pitch, src, (size_t)row_stride * es, row_bytes, (size_t)(n[1] * n[2]), kind, st);
    cudaError_t e = cudaSuccess;
    for (int64_t z = 0; z < n[2] && e == cudaSuccess; ++z)
        e = cudaMemcpy2DAsync((char *)v->data + z * pitch * n[1], pitch, src + z * plane_stride * es,
                              (size_t)row_stride * es, row_bytes, (size_t)n[1], kind, st);
    return e;
}

// Device allocation: stream-ordered from `pool` on `st`, or plain cudaMalloc.
static cudaError_t dev_alloc(void **p, size_t bytes, cudaMemPool_t pool, cudaStream_t st)
{
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMalloc(p, bytes);
}
static void dev_free(void *p, cudaMemPool_t pool, cudaStream_t st)
{
    if (!p) return;
    if (pool) cudaFreeAsync(p, st);
    else cudaFree(p);
}

// ------------------------------------------------------------------ volume
static ac_status create_volume_impl(cudaMemPool_t pool, const void *data, int data_on_device, ac_dtype dtype,
                                    int ndim, const int64_t dims[3], int64_t row_stride, int64_t plane_stride,
                                    const float spacing[3], float intensity_scale, cudaStream_t st, ac_volume **out)
{
    if (!out) AC_FAIL(AC_ERR_ARG, "ac_create_volume: out is NULL");
    *out = nullptr;
    if (!data || !dims || !spacing) AC_FAIL(AC_ERR_ARG, "ac_create_volume: NULL data, dims or spacing");
    const int es = elem_size(dtype);
    if (es == 0) AC_FAIL(AC_ERR_ARG, "ac_create_volume: unknown dtype");
    if (ndim != 2 && ndim != 3) AC_FAIL(AC_ERR_ARG, "ac_create_volume: ndim must be 2 or 3");
    int64_t n[3] = {dims[0], dims[1], ndim == 3 ? dims[2] : 1};
    for (int d = 0; d < ndim; ++d) {
        if (n[d] < 2 || n[d] > (1 << 30)) AC_FAIL(AC_ERR_ARG, "ac_create_volume: every used dimension must be in [2, 2^30]");
        if (!(spacing[d] > 0.0f) || !std::isfinite(spacing[d]))
            AC_FAIL(AC_ERR_ARG, "ac_create_volume: spacing must be positive and finite");
    }
    if (!std::isfinite(intensity_scale)) AC_FAIL(AC_ERR_ARG, "ac_create_volume: intensity_scale not finite");
    if (row_stride == 0) row_stride = n[0];
    if (plane_stride == 0) plane_stride = row_stride * n[1];
    if (row_stride < n[0] || plane_stride < row_stride * n[1])
        AC_FAIL(AC_ERR_ARG, "ac_create_volume: strides smaller than the extents");
    if (n[0] * n[1] * n[2] > ((int64_t)1 << 36)) AC_FAIL(AC_ERR_ARG, "ac_create_volume: volume too large");

    ac_volume *v = new ac_volume();
    cudaGetDevice(&v->device);
    v->dtype = dtype;
    v->ndim = ndim;
    for (int d = 0; d < 3; ++d) {
        v->n[d] = n[d];
        v->sp[d] = d < ndim ? spacing[d] : 1.0f;
    }
    v->scale = intensity_scale;
    v->es = es;
    const size_t row_bytes = (size_t)n[0] * es;
    const size_t pitch = (row_bytes + 15) / 16 * 16;   // TMA: strides multiple of 16 bytes
    v->pitch_y = (int64_t)(pitch / es);
    v->pitch_z = v->pitch_y * n[1];
    v->bytes = pitch * (size_t)n[1] * (size_t)n[2];
    v->pool = pool;
    cudaError_t e = dev_alloc(&v->data, v->bytes, pool, st);
    if (e != cudaSuccess) {
        delete v;
        AC_FAIL(e == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA,
                std::string("ac_create_volume: allocation: ") + cudaGetErrorString(e));
    }
    e = copy_voxels(v, data, data_on_device, row_stride, plane_stride, st, false);
    if (e != cudaSuccess) {
        dev_free(v->data, pool, st);
        delete v;
        AC_FAIL(AC_ERR_CUDA, std::string("ac_create_volume: copy: ") + cudaGetErrorString(e));
    }
    *out = v;
    return AC_OK;
}

extern "C" ac_status ac_create_volume(const void *data, int data_on_device, ac_dtype dtype, int ndim,
                                      const int64_t dims[3], int64_t row_stride, int64_t plane_stride,
                                      const float spacing[3], float intensity_scale, void *cuda_stream,
                                      ac_volume **out)
{
    ac::Range nvtx_range("ac_create_volume");
    g_err.clear();
    return create_volume_impl(nullptr, data, data_on_device, dtype, ndim, dims, row_stride, plane_stride, spacing,
                              intensity_scale, (cudaStream_t)cuda_stream, out);
}

ac_status ac::create_volume_pooled(cudaMemPool_t pool, const void *data, int data_on_device, ac_dtype dtype,
                                   int ndim, const int64_t dims[3], int64_t row_stride, int64_t plane_stride,
                                   const float spacing[3], float intensity_scale, cudaStream_t st, ac_volume **out)
{
    return create_volume_impl(pool, data, data_on_device, dtype, ndim, dims, row_stride, plane_stride, spacing,
                              intensity_scale, st, out);
}

extern "C" ac_status ac_load_volume(ac_volume *vol, const void *data, int data_on_device, int64_t row_stride,
                                    int64_t plane_stride, void *cuda_stream)
{
    ac::Range nvtx_range("ac_load_volume");
    g_err.clear();
    if (!vol || !data) AC_FAIL(AC_ERR_ARG, "ac_load_volume: NULL argument");
    if (row_stride == 0) row_stride = vol->n[0];
    if (plane_stride == 0) plane_stride = row_stride * vol->n[1];
    if (row_stride < vol->n[0] || plane_stride < row_stride * vol->n[1])
        AC_FAIL(AC_ERR_ARG, "ac_load_volume: strides smaller than the extents");
    AC_CUDA(copy_voxels(vol, data, data_on_device, row_stride, plane_stride, (cudaStream_t)cuda_stream, true));
    return AC_OK;
}

void ac::destroy_volume_on(ac_volume *vol, cudaStream_t st)
{
    if (!vol) return;
    dev_free(vol->data, vol->pool, st);
    if (vol->staging) cudaFree(vol->staging);
    delete vol;
}

extern "C" void ac_destroy_volume(ac_volume *vol) { ac::destroy_volume_on(vol, nullptr); }

// ------------------------------------------------------------------ seeding
__global__ void seed_lattice_kernel(float *state, int64_t C, int Lx, int Ly, float fx, float fy, float fz,
                                    float stride, float R0, int ndim)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < C; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k % Lx, j = (k / Lx) % Ly, l = k / ((int64_t)Lx * Ly);
        state[k] = fmaf((float)i, stride, fx);
        state[C + k] = fmaf((float)j, stride, fy);
        state[2 * C + k] = ndim == 3 ? fmaf((float)l, stride, fz) : 0.0f;
        state[3 * C + k] = R0;
        state[4 * C + k] = 0.0f;
    }
}

// Contour set of C contours on `vol`: state, status word, hold words and path
// counters (zeroed), allocated plainly or, with a pool, in stream order on `st`.
static ac_status make_contours(ac_volume *vol, int64_t C, ac_contours **out, cudaMemPool_t pool = nullptr,
                               cudaStream_t st = nullptr)
{
    ac_contours *c = new ac_contours();
    c->vol = vol;
    c->C = C;
    c->pool = pool;
    auto zero = [&](void *p, size_t n) { return pool ? cudaMemsetAsync(p, 0, n, st) : cudaMemset(p, 0, n); };
    const size_t cn = (size_t)(C > 0 ? C : 1);
    cudaError_t e = dev_alloc((void **)&c->state, sizeof(float) * 5 * cn, pool, st);
    if (e == cudaSuccess) e = dev_alloc((void **)&c->status, sizeof(int32_t) * 4, pool, st);
    if (e == cudaSuccess) e = zero(c->status, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = dev_alloc((void **)&c->hold, sizeof(int32_t) * cn, pool, st);
    if (e == cudaSuccess) e = zero(c->hold, sizeof(int32_t) * cn);
    if (e == cudaSuccess) e = dev_alloc((void **)&c->path_counts, sizeof(unsigned long long) * 4, pool, st);
    if (e == cudaSuccess) e = zero(c->path_counts, sizeof(unsigned long long) * 4);
    if (e != cudaSuccess) {
        dev_free(c->state, pool, st);
        dev_free(c->status, pool, st);
        dev_free(c->hold, pool, st);
        dev_free(c->path_counts, pool, st);
        delete c;
        AC_FAIL(e == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA,
                std::string("ac_seed: allocation: ") + cudaGetErrorString(e));
    }
    *out = c;
    return AC_OK;
}

static ac_status seed_impl(ac_volume *vol, const ac_seed_params *params, const float *explicit_cR,
                           int64_t n_explicit, void *cuda_stream, ac_contours **out, cudaMemPool_t pool);

extern "C" ac_status ac_seed(ac_volume *vol, const ac_seed_params *params, const float *explicit_cR,
                             int64_t n_explicit, void *cuda_stream, ac_contours **out)
{
    ac::Range nvtx_range("ac_seed");
    g_err.clear();
    return seed_impl(vol, params, explicit_cR, n_explicit, cuda_stream, out, nullptr);
}

ac_status ac::seed_lattice_pooled(cudaMemPool_t pool, ac_volume *vol, const ac_seed_params *params, cudaStream_t st,
                                  ac_contours **out)
{
    return seed_impl(vol, params, nullptr, 0, st, out, pool);
}

static ac_status seed_impl(ac_volume *vol, const ac_seed_params *params, const float *explicit_cR,
                           int64_t n_explicit, void *cuda_stream, ac_contours **out, cudaMemPool_t pool)
{
    if (!out) AC_FAIL(AC_ERR_ARG, "ac_seed: out is NULL");
    *out = nullptr;
    if (!vol) AC_FAIL(AC_ERR_ARG, "ac_seed: vol is NULL");
    if (n_explicit < 0) AC_FAIL(AC_ERR_ARG, "ac_seed: n_explicit is negative");
    if (explicit_cR && n_explicit == 0) {   // an empty set
        ac_contours *c = nullptr;
        ac_status s = make_contours(vol, 0, &c);
        if (s != AC_OK) return s;
        *out = c;
        return AC_OK;
    }
    if (n_explicit > 0) {
        if (!explicit_cR) AC_FAIL(AC_ERR_ARG, "ac_seed: explicit_cR is NULL");
        if (n_explicit >= ((int64_t)1 << 31)) AC_FAIL(AC_ERR_ARG, "ac_seed: too many contours");
        std::vector<float> soa((size_t)n_explicit * 5, 0.0f);
        double rmax = 0.0;
        for (int64_t k = 0; k < n_explicit; ++k) {
            for (int m = 0; m < 4; ++m) {
                const float x = explicit_cR[4 * k + m];
                if (!std::isfinite(x)) AC_FAIL(AC_ERR_ARG, "ac_seed: non-finite explicit seed");
                soa[(size_t)m * n_explicit + k] = x;
            }
            if (!(explicit_cR[4 * k + 3] > 0.0f) || explicit_cR[4 * k + 3] > 1e6f)
                AC_FAIL(AC_ERR_ARG, "ac_seed: explicit radius must be in (0, 1e6]");
            for (int d = 0; d < vol->ndim; ++d)
                soa[(size_t)d * n_explicit + k] = clamp_box(soa[(size_t)d * n_explicit + k], vol, d);
            if (vol->ndim == 2) soa[(size_t)2 * n_explicit + k] = 0.0f;
            rmax = std::max(rmax, (double)explicit_cR[4 * k + 3]);
        }
        ac_contours *c = nullptr;
        ac_status s = make_contours(vol, n_explicit, &c);
        if (s != AC_OK) return s;
        cudaError_t e = cudaMemcpy(c->state, soa.data(), soa.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            ac_destroy_contours(c);
            AC_FAIL(AC_ERR_CUDA, std::string("ac_seed: copy: ") + cudaGetErrorString(e));
        }
        c->r_hint = rmax;
        c->stride_hint = std::sqrt(1.5) * rmax;
        *out = c;
        return AC_OK;
    }
    if (!params) AC_FAIL(AC_ERR_ARG, "ac_seed: params is NULL");
    const double s = params->stride;
    if (!(s > 0.0) || !std::isfinite(s)) AC_FAIL(AC_ERR_ARG, "ac_seed: stride must be positive");
    const double R0 = params->R0 > 0.0 ? params->R0 : s / std::sqrt(1.5);
    int64_t L[3] = {1, 1, 1};
    double first[3] = {0, 0, 0};
    for (int d = 0; d < vol->ndim; ++d) {
        const double ext = (double)vol->n[d] * vol->sp[d];
        L[d] = (int64_t)std::floor(ext / s);
        if (L[d] < 1) L[d] = 1;
        first[d] = -0.5 * vol->sp[d] + 0.5 * (ext - (double)L[d] * s) + 0.5 * s;
    }
    const int64_t C = L[0] * L[1] * L[2];
    if (C >= ((int64_t)1 << 31)) AC_FAIL(AC_ERR_ARG, "ac_seed: lattice too fine");
    ac_contours *c = nullptr;
    ac_status rs = make_contours(vol, C, &c, pool, (cudaStream_t)cuda_stream);
    if (rs != AC_OK) return rs;
    c->lattice = true;
    for (int d = 0; d < 3; ++d) {
        c->L[d] = L[d];
        c->first[d] = (float)first[d];
    }
    c->stride = (float)s;
    c->R0 = (float)R0;
    c->r_hint = R0;
    c->stride_hint = s;
    ac_status rs2 = ac_reseed(c, cuda_stream);
    if (rs2 != AC_OK) {
        ac::destroy_contours_on(c, (cudaStream_t)cuda_stream);
        return rs2;
    }
    *out = c;
    return AC_OK;
}

extern "C" ac_status ac_reseed(ac_contours *c, void *cuda_stream)
{
    ac::Range nvtx_range("ac_reseed");
    if (!c) AC_FAIL(AC_ERR_ARG, "ac_reseed: NULL handle");
    if (!c->lattice) AC_FAIL(AC_ERR_STATE, "ac_reseed: handle was seeded explicitly");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int threads = 256;
    const int64_t C = c->C;
    const int64_t blocks = std::min<int64_t>((C + threads - 1) / threads, 1 << 16);
    AC_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int32_t) * 4, st));
    AC_CUDA(cudaMemsetAsync(c->hold, 0, sizeof(int32_t) * (size_t)(C > 0 ? C : 1), st));
    seed_lattice_kernel<<<(unsigned)blocks, threads, 0, st>>>(c->state, C, (int)c->L[0], (int)c->L[1], c->first[0],
                                                              c->first[1], c->first[2], c->stride, c->R0,
                                                              c->vol->ndim);
    count_launch();
    AC_CUDA(cudaGetLastError());
    return AC_OK;
}

extern "C" int64_t ac_contour_count(const ac_contours *ctr) { return ctr ? ctr->C : -1; }

void ac::destroy_contours_on(ac_contours *ctr, cudaStream_t st)
{
    if (!ctr) return;
    ctr->scratch.release_all();
    if (ctr->ev0) cudaEventDestroy(ctr->ev0);
    if (ctr->ev1) cudaEventDestroy(ctr->ev1);
    dev_free(ctr->state, ctr->pool, st);
    dev_free(ctr->status, ctr->pool, st);
    dev_free(ctr->hold, ctr->pool, st);
    dev_free(ctr->path_counts, ctr->pool, st);
    delete ctr;
}

extern "C" void ac_destroy_contours(ac_contours *ctr) { ac::destroy_contours_on(ctr, nullptr); }

// ------------------------------------------------------------------ state
ac_status ac::status_error(int32_t w)
{
    if (w & STATUS_TMA_TIMEOUT) AC_FAIL(AC_ERR_TIMEOUT, "device status: a brick load did not complete in time");
    if (w & STATUS_LOCALIZE_LIMIT) AC_FAIL(AC_ERR_TIMEOUT, "device status: localization round bound reached");
    if (w & STATUS_NONFINITE) AC_FAIL(AC_ERR_NUMERIC, "device status: non-finite contour state");
    if (w & STATUS_BOUNDS)
        AC_FAIL(AC_ERR_STATE, "device status: a gather index left its array (bounds-checked build)");
    if (w & STATUS_GRID_RANGE)
        AC_FAIL(AC_ERR_ARG, "device status: a contour radius exceeded the grid path's bound (contour stopped)");
    return AC_OK;
}

static ac_status check_status(ac_contours *ctr, cudaStream_t st)
{
    int32_t s[4];
    AC_CUDA(cudaMemcpyAsync(s, ctr->status, sizeof(s), cudaMemcpyDeviceToHost, st));
    AC_CUDA(cudaStreamSynchronize(st));
    return status_error(s[0]);
}

extern "C" ac_status ac_get_state(ac_contours *ctr, float *out_host, void *cuda_stream)
{
    g_err.clear();
    if (!ctr || !out_host) AC_FAIL(AC_ERR_ARG, "ac_get_state: NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    AC_CUDA(cudaMemcpyAsync(out_host, ctr->state, sizeof(float) * 5 * ctr->C, cudaMemcpyDeviceToHost, st));
    return check_status(ctr, st);
}

extern "C" ac_status ac_set_state(ac_contours *ctr, const float *in_host, void *cuda_stream)
{
    g_err.clear();
    if (!ctr || !in_host) AC_FAIL(AC_ERR_ARG, "ac_set_state: NULL argument");
    const int64_t C = ctr->C;
    std::vector<float> st(in_host, in_host + 5 * C);
    for (int64_t i = 0; i < 4 * C; ++i)
        if (!std::isfinite(st[i])) AC_FAIL(AC_ERR_ARG, "ac_set_state: non-finite centre or radius");
    for (int64_t k = 0; k < C; ++k) {
        if (!(st[3 * C + k] > 0.0f) || st[3 * C + k] > 1e6f) AC_FAIL(AC_ERR_ARG, "ac_set_state: radius must be in (0, 1e6]");
        for (int d = 0; d < 3; ++d)
            st[d * C + k] = d < ctr->vol->ndim ? clamp_box(st[d * C + k], ctr->vol, d) : 0.0f;
    }
    AC_CUDA(cudaMemcpyAsync(ctr->state, st.data(), sizeof(float) * 5 * C, cudaMemcpyHostToDevice,
                            (cudaStream_t)cuda_stream));
    AC_CUDA(cudaMemsetAsync(ctr->hold, 0, sizeof(int32_t) * (size_t)(C > 0 ? C : 1), (cudaStream_t)cuda_stream));
    AC_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
    return AC_OK;
}

extern "C" ac_status ac_state_device_ptr(ac_contours *ctr, float **out)
{
    if (!ctr || !out) AC_FAIL(AC_ERR_ARG, "ac_state_device_ptr: NULL argument");
    *out = ctr->state;
    return AC_OK;
}

// ------------------------------------------------------------------ support
__global__ void philox_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        const uint4 w = philox4x32_10_key(c, k0, k1);
        out[4 * i] = w.x;
        out[4 * i + 1] = w.y;
        out[4 * i + 2] = w.z;
        out[4 * i + 3] = w.w;
    }
}

extern "C" ac_status ac_philox4x32_10(const uint32_t *ctr_dev, uint64_t key, uint32_t *out_dev, int64_t n,
                                      void *cuda_stream)
{
    g_err.clear();
    if (n < 0 || (n > 0 && (!ctr_dev || !out_dev))) AC_FAIL(AC_ERR_ARG, "ac_philox4x32_10: bad arguments");
    if (n == 0) return AC_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1 << 16);
    philox_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(ctr_dev, (uint32_t)key,
                                                                           (uint32_t)(key >> 32), out_dev, n);
    count_launch();
    AC_CUDA(cudaGetLastError());
    return AC_OK;
}

// ------------------------------------------------------------------ evolution
namespace {

struct Plan {
    int B[3], halo[3], ext[3];
    int raw;        // staged region bytes
    int quad_off;   // 2D: byte offset of the quads (0: none)
    int smem;       // dynamic shared memory bytes
    int G, warps;
    bool brick, grid, comp, acc;
};

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

ac_status check_params(const ac_evolve_params *p)
{
    if (!p) AC_FAIL(AC_ERR_ARG, "ac_evolve: params is NULL");
    if (p->N < 1 || p->N > (1 << 24)) AC_FAIL(AC_ERR_ARG, "ac_evolve: N must be in [1, 2^24]");
    if (p->T < 1 || p->T > (1 << 24)) AC_FAIL(AC_ERR_ARG, "ac_evolve: T must be in [1, 2^24]");
    if (!(p->dR > 0.0f) || !std::isfinite(p->dR)) AC_FAIL(AC_ERR_ARG, "ac_evolve: dR must be positive");
    if (!(p->Rmin > 0.0f) || !(p->Rmax >= p->Rmin) || !std::isfinite(p->Rmax))
        AC_FAIL(AC_ERR_ARG, "ac_evolve: need 0 < Rmin <= Rmax");
    if (!(p->max_step > 0.0f) || !std::isfinite(p->max_step)) AC_FAIL(AC_ERR_ARG, "ac_evolve: max_step must be positive");
    if (!(p->eps0 >= 0.0f) || !std::isfinite(p->eps0)) AC_FAIL(AC_ERR_ARG, "ac_evolve: eps0 must be >= 0");
    if (p->path != AC_PATH_BRICK && p->path != AC_PATH_PLAIN && p->path != AC_PATH_GRID)
        AC_FAIL(AC_ERR_ARG, "ac_evolve: unknown path");
    if (p->path == AC_PATH_GRID && p->lanes_per_contour != 0 && p->lanes_per_contour != 8 &&
        p->lanes_per_contour != 16 && p->lanes_per_contour != 4)
        AC_FAIL(AC_ERR_ARG, "ac_evolve: the grid path takes 4 (2D, compensated), 8 or 16 lanes per contour");
    if (!(p->freeze_tol >= 0.0f) || !std::isfinite(p->freeze_tol)) AC_FAIL(AC_ERR_ARG, "ac_evolve: freeze_tol must be >= 0");
    if (p->freeze_iters < 0 || p->freeze_iters > 0xFFFF) AC_FAIL(AC_ERR_ARG, "ac_evolve: freeze_iters in [0, 65535]");
    if (p->cull_iter < 0) AC_FAIL(AC_ERR_ARG, "ac_evolve: cull_iter must be >= 0");
    if (std::isnan(p->cull_E)) AC_FAIL(AC_ERR_ARG, "ac_evolve: cull_E is NaN");
    if (p->sampling < 0 || p->sampling > 2) AC_FAIL(AC_ERR_ARG, "ac_evolve: sampling must be 0, 1 or 2");
    if (!(p->halo_factor >= 0.0f) || p->halo_factor > 64.0f) AC_FAIL(AC_ERR_ARG, "ac_evolve: halo_factor in [0, 64]");
    if (p->first_iter < 0 || (int64_t)(p->first_iter ? p->first_iter : 1) + p->T > (1 << 30))
        AC_FAIL(AC_ERR_ARG, "ac_evolve: first_iter out of range");
    if (p->lanes_per_contour != 0 && p->lanes_per_contour != 4 && p->lanes_per_contour != 8 &&
        p->lanes_per_contour != 16 && p->lanes_per_contour != 32)
        AC_FAIL(AC_ERR_ARG, "ac_evolve: lanes_per_contour must be 0, 4, 8, 16 or 32");
    if (p->lanes_per_contour == 4 && (p->compensated == 0 || p->sampling == 1 || (p->sampling == 0 && p->N < 64)))
        AC_FAIL(AC_ERR_ARG, "ac_evolve: 4 lanes per contour are built for compensated sums and fast sampling");
    if (p->warps_per_block < 0 || p->warps_per_block > 16) AC_FAIL(AC_ERR_ARG, "ac_evolve: warps_per_block in [0, 16]");
    if (p->path != AC_PATH_BRICK && p->warps_per_block > 8)
        AC_FAIL(AC_ERR_ARG, "ac_evolve: the plain and grid paths take at most 8 warps per block");
    for (int d = 0; d < 3; ++d)
        if (p->brick[d] < 0 || p->brick[d] > 224) AC_FAIL(AC_ERR_ARG, "ac_evolve: brick sizes must be in [0, 224]");
    return AC_OK;
}

// Brick interior, halo and staged-region size.  The halo covers a ball of 2.5x
// (3D) or 3.5x (2D) the initial radius plus dR/2 and a margin (contours that
// outgrow it read from global memory for that iteration).  A region starts at max(0, brick - halo)
// (x rounded down to the 16-byte TMA alignment) and never extends past what the
// volume needs; when the region would exceed the shared-memory budget the halo,
// then the brick, shrinks.
ac_status plan_evolve(const ac_volume *vol, double stride_hint, double r_hint, const ac_evolve_params *p, Plan &pl)
{
    pl.brick = p->path == AC_PATH_BRICK;
    pl.grid = p->path == AC_PATH_GRID;
    pl.comp = p->compensated != 0;
    if (pl.grid) {   // no samples: no sampling mode; lanes walk the chords of the ball
        pl.acc = false;
        // measured best: 4 lanes in 2D (compensated sums), 8 in 3D
        pl.G = p->lanes_per_contour ? p->lanes_per_contour : (vol->ndim == 2 && pl.comp ? 4 : 8);
        if (pl.G == 4 && (vol->ndim != 2 || !pl.comp))
            AC_FAIL(AC_ERR_ARG, "ac_evolve: 4 lanes on the grid path are built for 2D with compensated sums");
        pl.warps = p->warps_per_block ? p->warps_per_block : 8;
        pl.quad_off = 0;
        return AC_OK;
    }
    pl.acc = p->sampling == 1 || (p->sampling == 0 && p->N < 64);
    if (pl.acc && !pl.comp) AC_FAIL(AC_ERR_ARG, "ac_evolve: accurate sampling is built with compensated sums only");
    // lanes per contour: 2D about 32 samples per lane (4 lanes only with compensated
    // sums and fast sampling, otherwise at least 8); 3D about 8 to 16, except that
    // 512 <= N < 1024 takes 8 lanes (64 samples per lane, four contours per warp:
    // measured best at N = 512); at most 32
    int G = p->lanes_per_contour;
    if (G == 0) {
        if (vol->ndim == 3) {
            G = 8;
            while (G < 32 && (int64_t)G * 8 < p->N) G *= 2;
            if (p->N >= 512 && p->N < 1024) G = 8;
        } else {
            G = (pl.comp && !pl.acc) ? 4 : 8;
            while (G < 32 && (int64_t)G * 32 < p->N) G *= 2;
        }
    }
    pl.G = G;
    pl.warps = p->warps_per_block ? p->warps_per_block : 8;
    pl.quad_off = 0;
    if (!pl.brick) return AC_OK;
    const int al = 16 / vol->es;
    int B[3] = {1, 1, 1}, h[3] = {0, 0, 0};
    // lattice cells per brick.  3D: 2x2x2 (8 contours of 32 lanes fill 8 warps, two
    // CTAs per SM), 2x4x2 with 16 lanes (the longer axis is y, because a row of 64
    // 16-bit voxels would put every row of the region on the same shared-memory
    // banks), and with 8 lanes at N >= 512, 4x4x4 (64 contours fill 16 warps, one CTA
    // per SM with a region of up to 215 KB).  2D: 10x8 (measured best for 128
    // samples: 80 contours of 4 lanes fill 10 warps, two CTAs per SM at 96 registers).
    int cells[3] = {10, 8, 2};
    if (vol->ndim == 3) {
        cells[0] = cells[1] = cells[2] = 2;
        if (G == 16) cells[1] = 4;
        if (G == 8 && p->N >= 512) cells[0] = cells[1] = cells[2] = 4;
    }
    // groups for the contours of a brick (lattice estimate), 1..16 warps
    auto warps_of = [&]() {
        if (p->warps_per_block) return p->warps_per_block;
        double per = 1.0;
        for (int d = 0; d < vol->ndim; ++d) per *= std::max(1.0, B[d] * (double)vol->sp[d] / stride_hint);
        return std::max(1, std::min(16, (int)std::ceil(per * G / 32.0)));
    };
    auto brick_of = [&](int d) {
        const int b = p->brick[d] ? p->brick[d] : (int)std::lround(cells[d] * stride_hint / vol->sp[d]);
        return std::max(1, std::min(b, (int)std::min<int64_t>(vol->n[d], 224)));
    };
    for (int d = 0; d < vol->ndim; ++d) {
        B[d] = brick_of(d);
        const double hf = p->halo_factor > 0.0f ? p->halo_factor : (vol->ndim == 3 ? 2.5 : 3.5);
        h[d] = (int)std::ceil((hf * r_hint + 0.5 * p->dR) / vol->sp[d]) + 2;
    }
    if (!p->brick[0] && !p->brick[1] && !p->brick[2]) {
        // a small volume gets more, smaller bricks (down to 2 cells per axis in 2D, 1 in
        // 3D), so that the grid holds about four CTAs per slot (152 SMs x 2) instead of
        // a tail wave
        auto n_bricks = [&]() {
            int64_t nb = 1;
            for (int d = 0; d < vol->ndim; ++d) nb *= (vol->n[d] + B[d] - 1) / B[d];
            return nb;
        };
        const int min_cells = vol->ndim == 3 ? 1 : 2;
        while (n_bricks() < 1216) {
            int dm = -1;
            for (int d = 0; d < vol->ndim; ++d)
                if (cells[d] > min_cells && (dm < 0 || cells[d] > cells[dm])) dm = d;
            if (dm < 0) break;
            cells[dm] = std::max(min_cells, cells[dm] / 2);
            B[dm] = brick_of(dm);
        }
    }
    // The staged region may take the shared memory its CTA's registers leave it: in 3D
    // (128 registers a thread) a CTA of more than 8 warps has its SM alone, smaller ones
    // share it with a second CTA.
    for (int iter = 0; iter < 4096; ++iter) {
        const int64_t budget = vol->ndim == 3 ? (warps_of() > 8 ? 215 * 1024 : 110 * 1024) : 200 * 1024;
        int64_t raw = vol->es;
        bool fits_box = true;
        for (int d = 0; d < 3; ++d) {
            int ext = 1;
            if (d < vol->ndim) {
                int64_t need = (int64_t)B[d] + 2 * (int64_t)h[d] + (d == 0 ? al - 1 : 0);
                const int64_t cap = vol->n[d] + (d == 0 ? al - 1 : 0);
                need = std::min(need, cap);
                if (d == 0) need = (need + al - 1) / al * al;
                // 3D taps are read from the raw region: a row of a multiple of 128 bytes
                // would put the same voxel column of every row on one shared-memory bank,
                // so such rows get 16 more bytes (unless the region spans the volume's rows)
                if (d == 0 && vol->ndim == 3 && need < vol->n[0] && need * vol->es % 128 == 0) need += al;
                if (need > 256) fits_box = false;
                ext = (int)need;
            }
            pl.ext[d] = ext;
            pl.B[d] = B[d];
            pl.halo[d] = h[d];
            raw *= ext;
        }
        int64_t quad_off = 0, total = raw;
        if (vol->ndim == 2) {   // quads after the raw region: 4 halves (uint8, binary16) or float4
            const int qbytes = (vol->dtype == AC_U8 || vol->dtype == AC_F16) ? 8 : 16;
            quad_off = (raw + 127) / 128 * 128;
            total = quad_off + (int64_t)(pl.ext[0] - 1) * (pl.ext[1] - 1) * qbytes;
        }
        if (fits_box && total <= budget) {
            pl.raw = (int)raw;
            pl.quad_off = (int)quad_off;
            pl.smem = (int)total;
            pl.warps = warps_of();
            return AC_OK;
        }
        int hmax = 0, bmax = 0;
        for (int d = 0; d < vol->ndim; ++d) {
            hmax = std::max(hmax, h[d]);
            bmax = std::max(bmax, B[d]);
        }
        if (hmax > 1) {
            for (int d = 0; d < vol->ndim; ++d) h[d] = std::max(1, h[d] - 1);
        } else if (bmax > 1 && p->brick[0] == 0 && p->brick[1] == 0 && p->brick[2] == 0) {
            for (int d = 0; d < vol->ndim; ++d) B[d] = std::max(1, B[d] - 1);
        } else {
            break;
        }
    }
    AC_FAIL(AC_ERR_ARG, "ac_evolve: staged region cannot fit the shared-memory budget; use smaller bricks");
}

__global__ void bin_kernel(const VolDesc *vols, int n_vols, int64_t total, int3 B, uint32_t *keys, uint32_t *vals)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        int v = 0;
        for (int i = 1; i < n_vols; ++i)
            if (vols[i].contour_base <= g) v = i;
        const VolDesc &V = vols[v];
        const int64_t k = g - V.contour_base;
        const int Bd[3] = {B.x, B.y, B.z};
        int bi[3];
        for (int d = 0; d < 3; ++d) {
            const float c = V.state[d * V.C + k];
            int idx = (int)floorf(c * V.inv_sp[d]);
            idx = idx < 0 ? 0 : (idx >= V.n[d] ? V.n[d] - 1 : idx);
            int b = idx / Bd[d];
            bi[d] = b >= V.nb[d] ? V.nb[d] - 1 : b;
        }
        keys[g] = (uint32_t)(V.brick_base + bi[0] + (int64_t)V.nb[0] * (bi[1] + (int64_t)V.nb[1] * bi[2]));
        vals[g] = (uint32_t)g;
    }
}

CUtensorMapDataType tma_type(ac_dtype t)
{
    switch (t) {
    case AC_U8: return CU_TENSOR_MAP_DATA_TYPE_UINT8;
    case AC_U16: return CU_TENSOR_MAP_DATA_TYPE_UINT16;
    case AC_F16: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    }
}

VolDesc make_desc(const ac_contours *c, uint32_t stream)
{
    const ac_volume *v = c->vol;
    VolDesc d;
    std::memset(&d, 0, sizeof(d));
    d.data = v->data;
    d.pitch_y = v->pitch_y;
    d.pitch_z = v->pitch_z;
    for (int i = 0; i < 3; ++i) {
        d.n[i] = (int32_t)v->n[i];
        d.sp[i] = v->sp[i];
        d.inv_sp[i] = 1.0f / v->sp[i];
        d.box_hi[i] = (float)((double)(v->n[i] - 1) * v->sp[i]);
    }
    d.scale = v->scale;
    d.state = c->state;
    d.status = c->status;
    d.hold = c->hold;
    d.C = c->C;
    d.stream = stream;
    return d;
}

cudaError_t launch_evolve(ac_dtype t, const EvolveArgs &a, const Plan &pl, int64_t grid, cudaStream_t st)
{
    switch (t) {
    case AC_U8: return launch_evolve_u8(a, pl.brick, pl.G, pl.comp, pl.acc, pl.warps, grid, st);
    case AC_U16: return launch_evolve_u16(a, pl.brick, pl.G, pl.comp, pl.acc, pl.warps, grid, st);
    case AC_F16: return launch_evolve_f16(a, pl.brick, pl.G, pl.comp, pl.acc, pl.warps, grid, st);
    default: return launch_evolve_f32(a, pl.brick, pl.G, pl.comp, pl.acc, pl.warps, grid, st);
    }
}

// A launch over one or more contour sets, planned on the host.
struct Prepared {
    Plan pl;
    EvolveArgs a;
    ac_dtype dtype = AC_U8;
    int n_sets = 0;
    int64_t total = 0, bricks = 0;
    int end_bit = 1;
    size_t cub_bytes = 0;
    std::vector<VolDesc> desc;
    std::vector<CUtensorMap> maps;
    ac_contours *owner = nullptr;   // status word, path counters, kernel-time events
    // brick launches with an energy rule inside the span run in two phases: the
    // brick kernel up to cull_iter, then the plain kernel over the contours still
    // running (compacted); desc2 holds the second phase's windows
    bool split = false;
    int32_t p2_first = 0, p2_last = -1;
    std::vector<VolDesc> desc2;
};

// Phase windows of a split launch (see Prepared::split) and the upload of the
// descriptors: [phase-1 or only descriptors | phase-2 descriptors].
ac_status upload_desc(Prepared &pr, Scratch &sc, cudaStream_t st)
{
    const EvolveArgs &a = pr.a;
    const int c = a.cull_iter;
    pr.split = pr.pl.brick && c > 0 && c >= a.first_iter && c < a.last_iter;
    std::vector<VolDesc> d1 = pr.desc;
    if (pr.split) {
        pr.desc2 = pr.desc;
        pr.p2_first = c + 1;
        pr.p2_last = a.last_iter;
        for (int i = 0; i < pr.n_sets; ++i) {
            const VolDesc &o = pr.desc[i];
            VolDesc &x = d1[i], &y = pr.desc2[i];
            if (o.first_iter > o.last_iter) continue;   // empty window stays empty in both
            if (o.first_iter > c) {                     // entirely after the energy test
                x.first_iter = 1;
                x.last_iter = 0;
            } else {
                x.last_iter = std::min(o.last_iter, c);
                x.update_last = o.last_iter > c ? 1 : o.update_last;
            }
            if (o.last_iter <= c) {                     // entirely up to the energy test
                y.first_iter = 1;
                y.last_iter = 0;
            } else {
                y.first_iter = std::max(o.first_iter, c + 1);
            }
        }
    }
    AC_CUDA(sc.desc.ensure(sizeof(VolDesc) * pr.n_sets * 2));
    AC_CUDA(cudaMemcpyAsync(sc.desc.p, d1.data(), sizeof(VolDesc) * pr.n_sets, cudaMemcpyHostToDevice, st));
    if (pr.split)
        AC_CUDA(cudaMemcpyAsync(sc.desc.as<VolDesc>() + pr.n_sets, pr.desc2.data(), sizeof(VolDesc) * pr.n_sets,
                                cudaMemcpyHostToDevice, st));
    return AC_OK;
}

// Applies per-set iteration windows and stream words to the descriptors and the
// launch's iteration span.
ac_status apply_items(Prepared &pr, const ac_batch_item *items, const ac_evolve_params *p)
{
    EvolveArgs &a = pr.a;
    a.first_iter = p->first_iter ? p->first_iter : 1;
    a.last_iter = a.first_iter + p->T - 1;
    a.update_last = p->update_last ? 1 : 0;
    if (items) {   // the launch spans every set's window (plain path: one launch per n)
        int lo = 1 << 30, hi = 0;
        for (int i = 0; i < pr.n_sets; ++i) {
            if (items[i].first_iter < 1 || items[i].n_iter < 0 ||
                (int64_t)items[i].first_iter + items[i].n_iter > (1 << 30))
                AC_FAIL(AC_ERR_ARG, "ac_evolve_batch: item iterations out of range");
            if (items[i].n_iter == 0) continue;
            lo = std::min(lo, items[i].first_iter);
            hi = std::max(hi, items[i].first_iter + items[i].n_iter - 1);
        }
        a.first_iter = lo;
        a.last_iter = hi;
    }
    for (int i = 0; i < pr.n_sets && i < (int)pr.desc.size(); ++i) {   // no descriptors: only empty sets
        VolDesc &d = pr.desc[i];
        d.stream = items ? items[i].stream_id : p->stream_id;
        d.first_iter = items ? items[i].first_iter : a.first_iter;
        d.last_iter = items ? items[i].first_iter + items[i].n_iter - 1 : a.last_iter;
        d.update_last = items ? (items[i].update_last ? 1 : 0) : a.update_last;
    }
    return AC_OK;
}

// Host work of a launch: checks, plan, descriptors, tensor maps, scratch sizes;
// uploads the descriptors and maps into `sc` on the stream.
ac_status prepare_sets(ac_contours *const *sets, const ac_batch_item *items, int n_sets, const ac_evolve_params *p,
                       const ac_trace *trace, Scratch &sc, Prepared &pr, cudaStream_t st)
{
    ac_status s = check_params(p);
    if (s != AC_OK) return s;
    const ac_volume *v0 = sets[0]->vol;
    double stride_hint = 0, r_hint = 0;
    int64_t total = 0;
    for (int i = 0; i < n_sets; ++i) {
        if (!sets[i] || !sets[i]->vol) AC_FAIL(AC_ERR_ARG, "ac_evolve: NULL contour set");
        if (sets[i]->vol->dtype != v0->dtype || sets[i]->vol->ndim != v0->ndim)
            AC_FAIL(AC_ERR_ARG, "ac_evolve_batch: every set must share dtype and ndim");
        stride_hint = std::max(stride_hint, sets[i]->stride_hint);
        r_hint = std::max(r_hint, sets[i]->r_hint);
        total += sets[i]->C;
    }
    if (total >= ((int64_t)1 << 31)) AC_FAIL(AC_ERR_ARG, "ac_evolve: too many contours in one launch");
    if (total == 0) {   // only empty sets: nothing to plan or launch
        pr = Prepared();
        pr.n_sets = n_sets;
        pr.owner = sets[0];
        return AC_OK;
    }
    Plan &pl = pr.pl;
    s = plan_evolve(v0, stride_hint, r_hint, p, pl);
    if (s != AC_OK) return s;
    pr.dtype = v0->dtype;
    pr.n_sets = n_sets;
    pr.total = total;
    pr.owner = sets[0];

    EvolveArgs &a = pr.a;
    std::memset(&a, 0, sizeof(a));
    a.n_vols = n_sets;
    a.ndim = v0->ndim;
    a.total_contours = total;
    a.N = p->N;
    a.T = p->T;
    {
        // Philox round keys and the weight-band constants of Eq. 5 (launch constants)
        uint32_t k0 = (uint32_t)p->seed, k1 = (uint32_t)(p->seed >> 32);
        for (int r = 0; r < 10; ++r) {
            a.rk0[r] = k0;
            a.rk1[r] = k1;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const int d = v0->ndim;
        const double rho = std::pow(2.0, -1.0 / d), dR = p->dR, dr = rho * dR;
        a.dR = p->dR;
        a.Rmin = p->Rmin;
        a.Rmax = p->Rmax;
        a.half_eps0 = (float)(0.5 * p->eps0);
        a.max_step = p->max_step;
        a.max_step2 = (float)((double)p->max_step * p->max_step);
        a.rho = (float)rho;
        a.inv_dr = (float)(1.0 / dr);
        a.inv_dR = (float)(1.0 / dR);
        a.kR1 = (float)(-2.0 * rho / dr);
        a.kR2 = (float)(1.0 / dR);
        a.kr1 = (float)(-2.0 / dr);
        a.kr2 = (float)(1.0 / dR);
        a.vol_coef = (float)((d == 3 ? 4.0 / 3.0 * M_PI : M_PI) / p->N);
        a.freeze_tol = p->freeze_tol;
        a.freeze_iters = p->freeze_iters;
        a.cull_iter = p->cull_iter;
        a.cull_E = p->cull_E;
    }
    a.path_counts = sets[0]->path_counts;
    a.tma_polls = tma_poll_limit();
    if (pl.grid)   // bounded work per evaluation
        for (int i = 0; i < n_sets; ++i)
            for (int d = 0; d < sets[i]->vol->ndim; ++d) {
                const double lim = (double)GRID_MAX_RADIUS_VOXELS * sets[i]->vol->sp[d];
                if ((double)p->Rmax + 0.5 * p->dR > lim || sets[i]->r_hint + 0.5 * p->dR > lim)
                    AC_FAIL(AC_ERR_ARG, "ac_evolve: the grid path takes balls of at most 256 voxels radius "
                                        "(Rmax + dR/2 and the seeded radii)");
            }

    pr.desc.assign(n_sets, VolDesc());
    int64_t bricks = 0, cbase = 0;
    for (int i = 0; i < n_sets; ++i) {
        pr.desc[i] = make_desc(sets[i], p->stream_id);
        pr.desc[i].contour_base = cbase;
        cbase += sets[i]->C;
        if (pl.brick) {
            int64_t nb = 1;
            for (int d = 0; d < 3; ++d) {
                pr.desc[i].nb[d] = (int32_t)((sets[i]->vol->n[d] + pl.B[d] - 1) / pl.B[d]);
                nb *= pr.desc[i].nb[d];
            }
            pr.desc[i].brick_base = bricks;
            bricks += nb;
        }
    }
    if (bricks >= ((int64_t)1 << 31)) AC_FAIL(AC_ERR_ARG, "ac_evolve: too many bricks");
    pr.bricks = bricks;
    s = apply_items(pr, items, p);
    if (s != AC_OK) return s;
    if (trace && trace->device_buf) {
        if (n_sets != 1) AC_FAIL(AC_ERR_ARG, "ac_evolve: trace is supported for a single set");
        if (trace->k_begin < 0 || trace->k_end > sets[0]->C || trace->k_begin > trace->k_end || trace->t_begin < 1 ||
            trace->t_begin < a.first_iter || trace->t_end > a.last_iter + 1 || trace->t_begin > trace->t_end)
            AC_FAIL(AC_ERR_ARG, "ac_evolve: trace range outside the contours or iterations");
        a.trace = trace->device_buf;
        a.tk0 = trace->k_begin;
        a.tk1 = trace->k_end;
        a.tt0 = trace->t_begin;
        a.tt1 = trace->t_end;
    }
    if (total == 0) return AC_OK;

    s = upload_desc(pr, sc, st);
    if (s != AC_OK) return s;
    a.vols = sc.desc.as<VolDesc>();
    // the compaction list exists whenever a split is possible, so its address is
    // fixed for every later item change of a plan
    if (pl.brick && a.cull_iter > 0) AC_CUDA(sc.active.ensure(sizeof(uint32_t) * total + 64));
    if (!sets[0]->ev0) {
        AC_CUDA(cudaEventCreate(&sets[0]->ev0));
        AC_CUDA(cudaEventCreate(&sets[0]->ev1));
    }
    if (!pl.brick) return AC_OK;

    // tensor maps: one box of the staged-region size per volume
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) AC_FAIL(AC_ERR_CUDA, "ac_evolve: cuTensorMapEncodeTiled is not available from the driver");
    pr.maps.assign(n_sets, CUtensorMap());
    for (int i = 0; i < n_sets; ++i) {
        const ac_volume *v = sets[i]->vol;
        cuuint64_t gdim[3] = {(cuuint64_t)v->n[0], (cuuint64_t)v->n[1], (cuuint64_t)v->n[2]};
        cuuint64_t gstride[2] = {(cuuint64_t)(v->pitch_y * v->es), (cuuint64_t)(v->pitch_z * v->es)};
        cuuint32_t box[3] = {(cuuint32_t)pl.ext[0], (cuuint32_t)pl.ext[1], (cuuint32_t)pl.ext[2]};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&pr.maps[i], tma_type(v->dtype), 3, v->data, gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) AC_FAIL(AC_ERR_CUDA, "ac_evolve: cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
    }
    AC_CUDA(sc.tmaps.ensure(sizeof(CUtensorMap) * n_sets + 128));
    CUtensorMap *dmaps = reinterpret_cast<CUtensorMap *>(((uintptr_t)sc.tmaps.p + 127) & ~(uintptr_t)127);
    AC_CUDA(cudaMemcpyAsync(dmaps, pr.maps.data(), sizeof(CUtensorMap) * n_sets, cudaMemcpyHostToDevice, st));

    // binning and sort space
    AC_CUDA(sc.keys.ensure(sizeof(uint32_t) * total));
    AC_CUDA(sc.vals.ensure(sizeof(uint32_t) * total));
    AC_CUDA(sc.skeys.ensure(sizeof(uint32_t) * total));
    AC_CUDA(sc.svals.ensure(sizeof(uint32_t) * total));
    pr.end_bit = 1;
    while (((int64_t)1 << pr.end_bit) < bricks + 1) ++pr.end_bit;
    AC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, pr.cub_bytes, sc.keys.as<uint32_t>(), sc.skeys.as<uint32_t>(),
                                            sc.vals.as<uint32_t>(), sc.svals.as<uint32_t>(), (int)total, 0, pr.end_bit, st));
    AC_CUDA(sc.cub.ensure(pr.cub_bytes));

    a.tmaps = dmaps;
    a.sorted_brick = sc.skeys.as<uint32_t>();
    a.sorted_gidx = sc.svals.as<uint32_t>();
    a.total_bricks = bricks;
    for (int d = 0; d < 3; ++d) {
        a.B[d] = pl.B[d];
        a.halo[d] = pl.halo[d];
        a.ext[d] = pl.ext[d];
    }
    a.raw_bytes = pl.raw;
    a.quad_off = pl.quad_off;
    a.smem_bytes = pl.smem;
    return AC_OK;
}

// Contours whose second-phase window is not empty and that no rule has stopped,
// appended (in any order: every contour evolves independently) to `list`.
__global__ void compact_active_kernel(const VolDesc *vols, int n_vols, int64_t total, uint32_t *list,
                                      unsigned long long *count)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += stride) {
        int v = 0;
        for (int i = 1; i < n_vols; ++i)
            if (vols[i].contour_base <= gi) v = i;
        const VolDesc &V = vols[v];
        const int64_t k = gi - V.contour_base;
        const bool run = V.first_iter <= V.last_iter && !(V.hold && (V.hold[k] & HOLD_STOPPED));
        // one atomic per warp: the lanes of this iteration share a block of the list
        const unsigned act = __activemask();
        const unsigned m = __ballot_sync(act, run);
        const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
        unsigned long long base = 0;
        if (lane == leader && m) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(act, base, leader);
        if (run) list[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)gi;
    }
}

// Device work of a prepared launch only (no host synchronisation, no allocation):
// counters, binning by brick, sort, evolution kernel(s), kernel-time events.
// While a stream is captured, the kernel-time events become event-record nodes of
// the graph (cudaEventRecordExternal), so that each replay records them.
ac_status enqueue_prepared(Prepared &pr, Scratch &sc, cudaStream_t st, int64_t *launches, bool count = true,
                           bool capturing = false)
{
    if (pr.total == 0) return AC_OK;
    const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    EvolveArgs a = pr.a;
    ac_contours *owner = pr.owner;
    int64_t nl = 0;
    AC_CUDA(cudaMemsetAsync(owner->path_counts, 0, sizeof(unsigned long long) * 3, st));
    if (pr.pl.grid) {
        const int64_t per_cta = (int64_t)pr.pl.warps * 32 / pr.pl.G;
        const int64_t grid = std::min<int64_t>((pr.total + per_cta - 1) / per_cta, (int64_t)1 << 30);
        AC_CUDA(cudaEventRecordWithFlags(owner->ev0, st, ev_flags));
        cudaError_t e = launch_grid(pr.dtype, a, pr.pl.G, pr.pl.comp, pr.pl.warps, grid, st);
        if (e != cudaSuccess) AC_FAIL(AC_ERR_CUDA, std::string("ac_evolve: grid launch: ") + cudaGetErrorString(e));
        ++nl;
        AC_CUDA(cudaEventRecordWithFlags(owner->ev1, st, ev_flags));
    } else if (!pr.pl.brick) {
        const int64_t per_cta = (int64_t)pr.pl.warps * 32 / pr.pl.G;
        const int64_t grid = std::min<int64_t>((pr.total + per_cta - 1) / per_cta, (int64_t)1 << 30);
        AC_CUDA(cudaEventRecordWithFlags(owner->ev0, st, ev_flags));
        for (int n = a.first_iter; n <= a.last_iter; ++n) {
            a.iter0 = n;
            cudaError_t e = launch_evolve(pr.dtype, a, pr.pl, grid, st);
            if (e != cudaSuccess) AC_FAIL(AC_ERR_CUDA, std::string("ac_evolve: plain launch: ") + cudaGetErrorString(e));
            ++nl;
        }
        AC_CUDA(cudaEventRecordWithFlags(owner->ev1, st, ev_flags));
    } else {
        const int64_t blocks = std::min<int64_t>((pr.total + 255) / 256, 1 << 16);
        bin_kernel<<<(unsigned)blocks, 256, 0, st>>>(a.vols, pr.n_sets, pr.total,
                                                     make_int3(pr.pl.B[0], pr.pl.B[1], pr.pl.B[2]),
                                                     sc.keys.as<uint32_t>(), sc.vals.as<uint32_t>());
        ++nl;
        AC_CUDA(cudaGetLastError());
        size_t tmp = pr.cub_bytes;
        AC_CUDA(cub::DeviceRadixSort::SortPairs(sc.cub.p, tmp, sc.keys.as<uint32_t>(), sc.skeys.as<uint32_t>(),
                                                sc.vals.as<uint32_t>(), sc.svals.as<uint32_t>(), (int)pr.total, 0,
                                                pr.end_bit, st));
        AC_CUDA(cudaEventRecordWithFlags(owner->ev0, st, ev_flags));
        cudaError_t e = launch_evolve(pr.dtype, a, pr.pl, pr.bricks, st);
        if (e != cudaSuccess) AC_FAIL(AC_ERR_CUDA, std::string("ac_evolve: brick launch: ") + cudaGetErrorString(e));
        ++nl;
        if (pr.split) {
            // second phase: the contours the energy rule left running, compacted,
            // one plain launch per remaining iteration over a fixed grid that reads
            // the list length on the device (no host synchronisation)
            EvolveArgs b = a;
            b.vols = sc.desc.as<VolDesc>() + pr.n_sets;
            uint32_t *list = sc.active.as<uint32_t>();
            unsigned long long *cnt = reinterpret_cast<unsigned long long *>(
                reinterpret_cast<unsigned char *>(sc.active.p) + ((sizeof(uint32_t) * pr.total + 7) / 8 * 8));
            AC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
            const int64_t cblocks = std::min<int64_t>((pr.total + 255) / 256, 1 << 16);
            compact_active_kernel<<<(unsigned)cblocks, 256, 0, st>>>(b.vols, pr.n_sets, pr.total, list, cnt);
            ++nl;
            AC_CUDA(cudaGetLastError());
            b.active = list;
            b.n_active = cnt;
            Plan p2 = pr.pl;
            p2.brick = false;
            p2.warps = std::min(p2.warps, 8);
            const int64_t per_cta = (int64_t)p2.warps * 32 / p2.G;
            const int64_t grid = std::min<int64_t>((pr.total + per_cta - 1) / per_cta, 152 * 16);
            for (int n = pr.p2_first; n <= pr.p2_last; ++n) {
                b.iter0 = n;
                e = launch_evolve(pr.dtype, b, p2, grid, st);
                if (e != cudaSuccess) AC_FAIL(AC_ERR_CUDA, std::string("ac_evolve: compacted launch: ") + cudaGetErrorString(e));
                ++nl;
            }
        }
        AC_CUDA(cudaEventRecordWithFlags(owner->ev1, st, ev_flags));
    }
    owner->timed = true;
    if (launches) *launches = nl;
    if (count) count_launch(nl);
    return AC_OK;
}

// ac_evolve and ac_evolve_batch: sets[0] owns the scratch buffers.
ac_status evolve_sets(ac_contours *const *sets, const ac_batch_item *items, int n_sets, const ac_evolve_params *p,
                      const ac_trace *trace, cudaStream_t st)
{
    Prepared pr;
    ac_status s = prepare_sets(sets, items, n_sets, p, trace, sets[0]->scratch, pr, st);
    if (s != AC_OK) return s;
    return enqueue_prepared(pr, sets[0]->scratch, st, nullptr);
}

}  // namespace

ac_status ac::check_evolve_params(const ac_evolve_params *p) { return check_params(p); }


// ------------------------------------------------------------------ allocation-free evolve
// One file-scope device array holds every temporary of ac_evolve_static.  Byte
// layout: [0, 16) status word, [64, 96) path counters, [256, ...) volume
// descriptor, [512, 640) TMA descriptor, [1024, ...) binning keys, contour indices
// and their sorted copies (4 x 4 bytes per contour), then the sort's temporary
// space up to the end of the array.
static __device__ __align__(256) unsigned char g_static_scratch[AC_STATIC_SCRATCH_BYTES];

namespace {

constexpr size_t kStaticDesc = 256, kStaticTmap = 512, kStaticArrays = 1024;
static_assert(sizeof(VolDesc) <= kStaticTmap - kStaticDesc, "descriptor slot too small");

// Device address of the array on `dev`, looked up once per device.  In host code
// the array's name is only a host-side stand-in, never a device address.
ac_status static_scratch_ptr(int dev, unsigned char **out)
{
    static std::mutex mu;
    static void *addr[128] = {nullptr};
    if (dev < 0 || dev >= 128) AC_FAIL(AC_ERR_ARG, "ac_evolve_static: device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            AC_FAIL(AC_ERR_CUDA, std::string("ac_evolve_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(addr[dev]);
    return AC_OK;
}

}  // namespace

extern "C" ac_status ac_plan_layout(int32_t ndim, ac_dtype dtype, const int64_t dims[3], const float spacing[3],
                                    double stride, double r0, const ac_evolve_params *p, ac_layout *out)
{
    g_err.clear();
    if (!dims || !spacing || !p || !out) AC_FAIL(AC_ERR_ARG, "ac_plan_layout: NULL argument");
    ac_status s = check_params(p);
    if (s != AC_OK) return s;
    const int es = elem_size(dtype);
    if (es == 0) AC_FAIL(AC_ERR_ARG, "ac_plan_layout: unknown dtype");
    if (ndim != 2 && ndim != 3) AC_FAIL(AC_ERR_ARG, "ac_plan_layout: ndim must be 2 or 3");
    if (!(stride > 0.0) || !(r0 > 0.0) || !std::isfinite(stride) || !std::isfinite(r0))
        AC_FAIL(AC_ERR_ARG, "ac_plan_layout: stride and r0 must be positive");
    ac_volume vol;   // geometry only: nothing on the device
    vol.device = -1;
    vol.dtype = dtype;
    vol.ndim = ndim;
    vol.es = es;
    vol.scale = 1.0f;
    vol.data = nullptr;
    vol.bytes = 0;
    vol.pool = nullptr;
    for (int d = 0; d < 3; ++d) {
        vol.n[d] = d < ndim ? dims[d] : 1;
        vol.sp[d] = d < ndim ? spacing[d] : 1.0f;
        if (d < ndim && (vol.n[d] < 2 || vol.n[d] > (1 << 30) || !(vol.sp[d] > 0.0f) || !std::isfinite(vol.sp[d])))
            AC_FAIL(AC_ERR_ARG, "ac_plan_layout: every used dimension must be in [2, 2^30] with positive spacing");
    }
    vol.pitch_y = vol.n[0];
    vol.pitch_z = vol.n[0] * vol.n[1];
    Plan pl;
    s = plan_evolve(&vol, stride, r0, p, pl);
    if (s != AC_OK) return s;
    std::memset(out, 0, sizeof(*out));
    out->lanes_per_contour = pl.G;
    out->warps_per_block = pl.warps;
    if (pl.brick) {
        for (int d = 0; d < 3; ++d) {
            out->brick[d] = d < ndim ? pl.B[d] : 1;
            out->halo[d] = d < ndim ? pl.halo[d] : 0;
            out->region[d] = pl.ext[d];
        }
        out->smem_bytes = pl.smem;
    }
    return AC_OK;
}

extern "C" ac_status ac_evolve_static(const void *volume_dev, ac_dtype dtype, int ndim, const int64_t dims[3],
                                      int64_t row_stride, int64_t plane_stride, const float spacing[3],
                                      float intensity_scale, float *state_dev, int64_t n_contours, float r0,
                                      float stride, const ac_evolve_params *p, void *cuda_stream)
{
    ac::Range nvtx_range("ac_evolve_static");
    g_err.clear();
    if (n_contours > AC_STATIC_MAX_CONTOURS)
        AC_FAIL(AC_ERR_BUDGET, "ac_evolve_static: n_contours exceeds AC_STATIC_MAX_CONTOURS (" +
                                   std::to_string(AC_STATIC_MAX_CONTOURS) + ")");
    if (n_contours < 1) AC_FAIL(AC_ERR_ARG, "ac_evolve_static: need at least one contour");
    if (!volume_dev || !state_dev || !dims || !spacing) AC_FAIL(AC_ERR_ARG, "ac_evolve_static: NULL argument");
    ac_status s = check_params(p);
    if (s != AC_OK) return s;
    if (p->path == AC_PATH_GRID || p->freeze_iters > 0 || p->cull_iter > 0)
        AC_FAIL(AC_ERR_ARG, "ac_evolve_static: takes the brick and plain paths without stopping rules");
    const int es = elem_size(dtype);
    if (es == 0) AC_FAIL(AC_ERR_ARG, "ac_evolve_static: unknown dtype");
    if (ndim != 2 && ndim != 3) AC_FAIL(AC_ERR_ARG, "ac_evolve_static: ndim must be 2 or 3");
    ac_volume vol;
    vol.dtype = dtype;
    vol.ndim = ndim;
    vol.es = es;
    vol.scale = intensity_scale;
    for (int d = 0; d < 3; ++d) {
        vol.n[d] = d < ndim ? dims[d] : 1;
        vol.sp[d] = d < ndim ? spacing[d] : 1.0f;
        if (d < ndim && (vol.n[d] < 2 || vol.n[d] > (1 << 30) || !(vol.sp[d] > 0.0f) || !std::isfinite(vol.sp[d])))
            AC_FAIL(AC_ERR_ARG, "ac_evolve_static: every used dimension must be in [2, 2^30] with positive spacing");
    }
    if (row_stride == 0) row_stride = vol.n[0];
    if (plane_stride == 0) plane_stride = row_stride * vol.n[1];
    if (row_stride < vol.n[0] || plane_stride < row_stride * vol.n[1])
        AC_FAIL(AC_ERR_ARG, "ac_evolve_static: strides smaller than the extents");
    if (!std::isfinite(intensity_scale)) AC_FAIL(AC_ERR_ARG, "ac_evolve_static: intensity_scale not finite");
    vol.data = const_cast<void *>(volume_dev);
    vol.pitch_y = row_stride;
    vol.pitch_z = plane_stride;
    vol.bytes = (size_t)plane_stride * vol.n[2] * es;
    const bool brick = p->path == AC_PATH_BRICK;
    if (brick && (((uintptr_t)volume_dev % 16) != 0 || (row_stride * es) % 16 != 0 || (plane_stride * es) % 16 != 0))
        AC_FAIL(AC_ERR_ARG, "ac_evolve_static: the brick path needs a 16-byte aligned volume with row and plane "
                            "strides that are multiples of 16 bytes (use AC_PATH_PLAIN otherwise)");
    if (brick && (!(r0 > 0.0f) || !(stride > 0.0f)))
        AC_FAIL(AC_ERR_ARG, "ac_evolve_static: r0 and stride must be positive");
    int dev = 0;
    AC_CUDA(cudaGetDevice(&dev));
    // both buffers must be memory this device's kernels may read: device memory of
    // this device (a peer's would be read with this device's scratch) or managed
    cudaPointerAttributes pa;
    for (const void *q : {volume_dev, (const void *)state_dev}) {
        if (cudaPointerGetAttributes(&pa, q) != cudaSuccess ||
            (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            AC_FAIL(AC_ERR_ARG, "ac_evolve_static: volume and state must be device memory");
        }
        if (pa.type == cudaMemoryTypeDevice && pa.device != dev)
            AC_FAIL(AC_ERR_ARG, "ac_evolve_static: volume and state must be memory of the current device (device " +
                                    std::to_string(dev) + "), not of device " + std::to_string(pa.device));
    }
    unsigned char *base = nullptr;
    s = static_scratch_ptr(dev, &base);
    if (s != AC_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    ac_contours ctr;   // host-side view of the caller's state (nothing allocated)
    ctr.vol = &vol;
    ctr.C = n_contours;
    ctr.state = state_dev;
    ctr.status = reinterpret_cast<int32_t *>(base);
    ctr.path_counts = reinterpret_cast<unsigned long long *>(base + 64);
    ctr.r_hint = r0;
    ctr.stride_hint = stride;
    Plan pl;
    s = plan_evolve(&vol, stride, r0, p, pl);
    if (s != AC_OK) return s;

    EvolveArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n_vols = 1;
    a.ndim = ndim;
    a.total_contours = n_contours;
    a.N = p->N;
    a.T = p->T;
    a.first_iter = p->first_iter ? p->first_iter : 1;
    a.last_iter = a.first_iter + p->T - 1;
    a.update_last = p->update_last ? 1 : 0;
    {
        uint32_t k0 = (uint32_t)p->seed, k1 = (uint32_t)(p->seed >> 32);
        for (int r = 0; r < 10; ++r) {
            a.rk0[r] = k0;
            a.rk1[r] = k1;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const double rho = std::pow(2.0, -1.0 / ndim), dR = p->dR, dr = rho * dR;
        a.dR = p->dR;
        a.Rmin = p->Rmin;
        a.Rmax = p->Rmax;
        a.half_eps0 = (float)(0.5 * p->eps0);
        a.max_step = p->max_step;
        a.max_step2 = (float)((double)p->max_step * p->max_step);
        a.rho = (float)rho;
        a.inv_dr = (float)(1.0 / dr);
        a.inv_dR = (float)(1.0 / dR);
        a.kR1 = (float)(-2.0 * rho / dr);
        a.kR2 = (float)(1.0 / dR);
        a.kr1 = (float)(-2.0 / dr);
        a.kr2 = (float)(1.0 / dR);
        a.vol_coef = (float)((ndim == 3 ? 4.0 / 3.0 * M_PI : M_PI) / p->N);
    }
    a.path_counts = ctr.path_counts;
    a.tma_polls = tma_poll_limit();

    VolDesc desc = make_desc(&ctr, p->stream_id);
    desc.first_iter = a.first_iter;
    desc.last_iter = a.last_iter;
    desc.update_last = a.update_last;
    int64_t bricks = 1;
    if (brick)
        for (int d = 0; d < 3; ++d) {
            desc.nb[d] = (int32_t)((vol.n[d] + pl.B[d] - 1) / pl.B[d]);
            bricks *= desc.nb[d];
        }
    VolDesc *ddesc = reinterpret_cast<VolDesc *>(base + kStaticDesc);
    a.vols = ddesc;
    // start from a clean status word and counters every call (the array keeps the last call's contents)
    AC_CUDA(cudaMemsetAsync(base, 0, 96, st));
    AC_CUDA(cudaMemcpyAsync(ddesc, &desc, sizeof(desc), cudaMemcpyHostToDevice, st));

    if (!brick) {
        const int64_t per_cta = (int64_t)pl.warps * 32 / pl.G;
        const int64_t grid = std::min<int64_t>((n_contours + per_cta - 1) / per_cta, (int64_t)1 << 30);
        for (int n = a.first_iter; n <= a.last_iter; ++n) {
            a.iter0 = n;
            cudaError_t e = launch_evolve(dtype, a, pl, grid, st);
            if (e != cudaSuccess) AC_FAIL(AC_ERR_CUDA, std::string("ac_evolve_static: launch: ") + cudaGetErrorString(e));
            count_launch();
        }
    } else {
        if (bricks >= ((int64_t)1 << 31)) AC_FAIL(AC_ERR_ARG, "ac_evolve_static: too many bricks");
        PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
        if (!enc) AC_FAIL(AC_ERR_CUDA, "ac_evolve_static: cuTensorMapEncodeTiled is not available from the driver");
        CUtensorMap map;
        cuuint64_t gdim[3] = {(cuuint64_t)vol.n[0], (cuuint64_t)vol.n[1], (cuuint64_t)vol.n[2]};
        cuuint64_t gstride[2] = {(cuuint64_t)(row_stride * es), (cuuint64_t)(plane_stride * es)};
        cuuint32_t box[3] = {(cuuint32_t)pl.ext[0], (cuuint32_t)pl.ext[1], (cuuint32_t)pl.ext[2]};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&map, tma_type(dtype), 3, vol.data, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            AC_FAIL(AC_ERR_CUDA, "ac_evolve_static: cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
        CUtensorMap *dmap = reinterpret_cast<CUtensorMap *>(base + kStaticTmap);
        AC_CUDA(cudaMemcpyAsync(dmap, &map, sizeof(map), cudaMemcpyHostToDevice, st));
        uint32_t *keys = reinterpret_cast<uint32_t *>(base + kStaticArrays);
        uint32_t *vals = keys + AC_STATIC_MAX_CONTOURS;
        uint32_t *skeys = vals + AC_STATIC_MAX_CONTOURS;
        uint32_t *svals = skeys + AC_STATIC_MAX_CONTOURS;
        unsigned char *tmp_space = reinterpret_cast<unsigned char *>(svals + AC_STATIC_MAX_CONTOURS);
        const size_t tmp_cap = (size_t)AC_STATIC_SCRATCH_BYTES - (size_t)(tmp_space - base);
        int end_bit = 1;
        while (((int64_t)1 << end_bit) < bricks + 1) ++end_bit;
        size_t tmp = 0;
        AC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, keys, skeys, vals, svals, (int)n_contours, 0, end_bit, st));
        if (tmp > tmp_cap)
            AC_FAIL(AC_ERR_BUDGET, "ac_evolve_static: the sort needs " + std::to_string(tmp) +
                                       " bytes of temporary space, more than the static array holds");
        const int64_t blocks = std::min<int64_t>((n_contours + 255) / 256, 1 << 16);
        bin_kernel<<<(unsigned)blocks, 256, 0, st>>>(ddesc, 1, n_contours, make_int3(pl.B[0], pl.B[1], pl.B[2]), keys,
                                                     vals);
        count_launch();
        AC_CUDA(cudaGetLastError());
        AC_CUDA(cub::DeviceRadixSort::SortPairs(tmp_space, tmp, keys, skeys, vals, svals, (int)n_contours, 0, end_bit, st));
        a.tmaps = dmap;
        a.sorted_brick = skeys;
        a.sorted_gidx = svals;
        a.total_bricks = bricks;
        for (int d = 0; d < 3; ++d) {
            a.B[d] = pl.B[d];
            a.halo[d] = pl.halo[d];
            a.ext[d] = pl.ext[d];
        }
        a.raw_bytes = pl.raw;
        a.quad_off = pl.quad_off;
        a.smem_bytes = pl.smem;
        cudaError_t e = launch_evolve(dtype, a, pl, bricks, st);
        if (e != cudaSuccess) AC_FAIL(AC_ERR_CUDA, std::string("ac_evolve_static: launch: ") + cudaGetErrorString(e));
        count_launch();
    }
    return check_status(&ctr, st);
}

// ------------------------------------------------------------------ plans, graphs, autotuning
struct ac_plan {
    std::vector<ac_contours *> sets;
    ac_evolve_params params;
    Prepared pr;
    Scratch sc;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_launches = 0;
    int32_t span0 = 0, span1 = 0;   // iteration span the graph was captured with
    bool valid = true;              // false after a failed rebind
    bool stale = false;             // the launch changed since the graph was captured
};

static void drop_graph(ac_plan *pl)
{
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    pl->exec = nullptr;
    pl->graph = nullptr;
}

extern "C" ac_status ac_plan_create(ac_contours *const *sets, const ac_batch_item *items, int32_t n_sets,
                                    const ac_evolve_params *params, ac_plan **out)
{
    ac::Range nvtx_range("ac_plan_create");
    g_err.clear();
    if (!out) AC_FAIL(AC_ERR_ARG, "ac_plan_create: out is NULL");
    *out = nullptr;
    if (!sets || n_sets < 1 || n_sets > 4096 || !params) AC_FAIL(AC_ERR_ARG, "ac_plan_create: need 1..4096 sets and params");
    ac_plan *pl = new ac_plan();
    pl->sets.assign(sets, sets + n_sets);
    pl->params = *params;
    ac_status s = prepare_sets(pl->sets.data(), items, n_sets, params, nullptr, pl->sc, pl->pr, 0);
    cudaError_t e = cudaStreamSynchronize(0);
    if (s == AC_OK && e != cudaSuccess) {
        ac::set_error(std::string("ac_plan_create: ") + cudaGetErrorString(e));
        s = AC_ERR_CUDA;
    }
    if (s != AC_OK) {
        pl->sc.release_all();
        delete pl;
        return s;
    }
    *out = pl;
    return AC_OK;
}

extern "C" ac_status ac_plan_rebind(ac_plan *pl, ac_contours *const *sets, const ac_batch_item *items,
                                    int32_t n_sets, void *cuda_stream)
{
    ac::Range nvtx_range("ac_plan_rebind");
    g_err.clear();
    if (!pl) AC_FAIL(AC_ERR_ARG, "ac_plan_rebind: NULL plan");
    if (!sets || n_sets < 1 || n_sets > 4096) AC_FAIL(AC_ERR_ARG, "ac_plan_rebind: need 1..4096 sets");
    pl->stale = true;   // the next graph launch recaptures and updates the executable graph
    pl->valid = false;
    std::vector<ac_contours *> keep(sets, sets + n_sets);
    Prepared pr;
    ac_status s = prepare_sets(keep.data(), items, n_sets, &pl->params, nullptr, pl->sc, pr, (cudaStream_t)cuda_stream);
    if (s != AC_OK) return s;
    pl->sets = std::move(keep);
    pl->pr = std::move(pr);
    pl->valid = true;
    return AC_OK;
}

extern "C" ac_status ac_plan_set_items(ac_plan *pl, const ac_batch_item *items, void *cuda_stream)
{
    g_err.clear();
    if (!pl) AC_FAIL(AC_ERR_ARG, "ac_plan_set_items: NULL plan");
    if (!pl->valid) AC_FAIL(AC_ERR_STATE, "ac_plan_set_items: the plan has no sets (a rebind failed)");
    ac_status s = apply_items(pl->pr, items, &pl->params);
    if (s != AC_OK) return s;
    if (pl->pr.total == 0) return AC_OK;
    Prepared &pr = pl->pr;
    const bool was_split = pr.split;
    const int32_t p2f = pr.p2_first, p2l = pr.p2_last;
    s = upload_desc(pr, pl->sc, (cudaStream_t)cuda_stream);
    if (s != AC_OK) return s;
    // a captured graph holds one plain launch per iteration of its span (plain path,
    // or the second phase of a split brick launch)
    if (!pr.pl.brick && !pr.pl.grid && (pr.a.first_iter != pl->span0 || pr.a.last_iter != pl->span1)) pl->stale = true;
    if (pr.pl.brick && (was_split != pr.split || p2f != pr.p2_first || p2l != pr.p2_last)) pl->stale = true;
    return AC_OK;
}

extern "C" ac_status ac_plan_launch(ac_plan *pl, int use_graph, void *cuda_stream)
{
    ac::Range nvtx_range("ac_plan_launch");
    g_err.clear();
    if (!pl) AC_FAIL(AC_ERR_ARG, "ac_plan_launch: NULL plan");
    if (!pl->valid) AC_FAIL(AC_ERR_STATE, "ac_plan_launch: the plan has no sets (a rebind failed)");
    if (pl->pr.total == 0) return AC_OK;   // only empty sets
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!use_graph) return enqueue_prepared(pl->pr, pl->sc, st, nullptr);
    if (!pl->exec || pl->stale) {
        // capture on a stream of the plan's own (the legacy stream cannot capture);
        // an executable graph from an earlier capture is updated in place when the
        // new capture has its topology (same launches, other sizes and arguments),
        // and instantiated afresh otherwise
        if (!pl->cap_stream) AC_CUDA(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
        AC_CUDA(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeRelaxed));
        int64_t n = 0;
        ac_status s = enqueue_prepared(pl->pr, pl->sc, pl->cap_stream, &n, false, true);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
        if (s != AC_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        AC_CUDA(e);
        bool updated = false;
        if (pl->exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(pl->exec, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(pl->exec);
                pl->exec = nullptr;
            }
        }
        if (pl->graph) cudaGraphDestroy(pl->graph);
        pl->graph = g;
        if (!updated) AC_CUDA(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
        pl->stale = false;
        pl->graph_launches = n;
        pl->span0 = pl->pr.a.first_iter;
        pl->span1 = pl->pr.a.last_iter;
    }
    AC_CUDA(cudaGraphLaunch(pl->exec, st));
    count_launch(pl->graph_launches);
    return AC_OK;
}

ac_status ac::plan_set_trace(ac_plan *pl, int set, const ac_trace *tr)
{
    if (!pl || set < 0 || set >= (int)pl->sets.size()) AC_FAIL(AC_ERR_ARG, "plan_set_trace: bad set");
    EvolveArgs &a = pl->pr.a;
    if (!tr || !tr->device_buf) {
        if (a.trace) pl->stale = true;
        a.trace = nullptr;
        return AC_OK;
    }
    const ac_contours *c = pl->sets[set];
    if (tr->k_begin < 0 || tr->k_end > c->C || tr->k_begin > tr->k_end || tr->t_begin < 1 || tr->t_begin > tr->t_end)
        AC_FAIL(AC_ERR_ARG, "plan_set_trace: trace range outside the contours or iterations");
    a.trace = tr->device_buf;
    a.tk0 = tr->k_begin;
    a.tk1 = tr->k_end;
    a.tt0 = tr->t_begin;
    a.tt1 = tr->t_end;
    a.trace_vol = set;
    pl->stale = true;
    return AC_OK;
}

extern "C" void ac_destroy_plan(ac_plan *pl)
{
    if (!pl) return;
    drop_graph(pl);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    pl->sc.release_all();
    delete pl;
}

namespace {

struct TuneKey {
    int ndim, dtype, N, G_in, comp, acc, halo_milli;
    int64_t stride_milli, r_milli;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(ndim, dtype, N, G_in, comp, acc, halo_milli, stride_milli, r_milli) <
               std::tie(o.ndim, o.dtype, o.N, o.G_in, o.comp, o.acc, o.halo_milli, o.stride_milli, o.r_milli);
    }
};
struct TuneVal {
    int G, warps, brick[3];
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

}  // namespace

extern "C" ac_status ac_autotune(ac_contours *const *sets, int32_t n_sets, ac_evolve_params *params, void *cuda_stream)
{
    ac::Range nvtx_range("ac_autotune");
    g_err.clear();
    if (!sets || n_sets < 1 || n_sets > 4096 || !params) AC_FAIL(AC_ERR_ARG, "ac_autotune: need 1..4096 sets and params");
    ac_status s = check_params(params);
    if (s != AC_OK) return s;
    if (params->path != AC_PATH_BRICK) return AC_OK;   // nothing to tune on the plain path
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const ac_volume *v0 = sets[0]->vol;
    double stride_hint = 0, r_hint = 0;
    int64_t total = 0;
    for (int i = 0; i < n_sets; ++i) {
        if (!sets[i] || !sets[i]->vol) AC_FAIL(AC_ERR_ARG, "ac_autotune: NULL contour set");
        stride_hint = std::max(stride_hint, sets[i]->stride_hint);
        r_hint = std::max(r_hint, sets[i]->r_hint);
        total += sets[i]->C;
    }
    if (total == 0) return AC_OK;   // only empty sets: nothing to time
    const bool comp = params->compensated != 0;
    const bool acc = params->sampling == 1 || (params->sampling == 0 && params->N < 64);
    const TuneKey key{v0->ndim, (int)v0->dtype, params->N, params->lanes_per_contour, comp, acc,
                      (int)std::lround(params->halo_factor * 1000), (int64_t)std::llround(stride_hint * 1000),
                      (int64_t)std::llround(r_hint * 1000)};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            params->lanes_per_contour = it->second.G;
            params->warps_per_block = it->second.warps;
            for (int d = 0; d < 3; ++d) params->brick[d] = it->second.brick[d];
            return AC_OK;
        }
    }
    // candidates: lanes per contour x lattice cells per brick
    std::vector<int> Gs;
    for (int G : {4, 8, 16, 32}) {
        if (params->lanes_per_contour && G != params->lanes_per_contour) continue;
        if (G == 4 && (!comp || acc)) continue;
        if (G > 4 && (int64_t)G > params->N) continue;
        Gs.push_back(G);
    }
    std::vector<std::array<int, 3>> cells;
    if (v0->ndim == 2) cells = {{8, 8, 1}, {10, 8, 1}, {12, 8, 1}, {16, 8, 1}};
    else cells = {{2, 2, 2}, {2, 4, 2}, {2, 2, 1}, {3, 3, 2}, {4, 4, 2}, {4, 4, 4}};

    // trial copies of the contour states (trials must not move the real contours)
    std::vector<ac_contours> tmp(n_sets);
    std::vector<ac_contours *> tsets(n_sets);
    std::vector<float *> copies(n_sets, nullptr);
    int32_t *tstatus = nullptr;
    unsigned long long *tcounts = nullptr;
    auto cleanup = [&]() {
        for (float *c : copies)
            if (c) cudaFree(c);
        if (tstatus) cudaFree(tstatus);
        if (tcounts) cudaFree(tcounts);
        for (auto &t : tmp) {
            t.scratch.release_all();
            if (t.ev0) cudaEventDestroy(t.ev0);
            if (t.ev1) cudaEventDestroy(t.ev1);
        }
    };
    cudaError_t e = cudaMalloc(&tstatus, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&tcounts, sizeof(unsigned long long) * 4);
    for (int i = 0; i < n_sets && e == cudaSuccess; ++i) {
        e = cudaMalloc(&copies[i], sizeof(float) * 5 * std::max<int64_t>(1, sets[i]->C));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(copies[i], sets[i]->state, sizeof(float) * 5 * sets[i]->C, cudaMemcpyDeviceToDevice, st);
        tmp[i].vol = sets[i]->vol;
        tmp[i].C = sets[i]->C;
        tmp[i].state = copies[i];
        tmp[i].status = tstatus;
        tmp[i].path_counts = tcounts;
        tmp[i].r_hint = sets[i]->r_hint;
        tmp[i].stride_hint = sets[i]->stride_hint;
        tsets[i] = &tmp[i];
    }
    if (e != cudaSuccess) {
        cleanup();
        AC_FAIL(e == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA,
                std::string("ac_autotune: trial state: ") + cudaGetErrorString(e));
    }
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best_ms = 1e30f;
    TuneVal best{0, 0, {0, 0, 0}};
    for (int G : Gs) {
        for (const auto &cl : cells) {
            ac_evolve_params tp = *params;
            tp.lanes_per_contour = G;
            tp.warps_per_block = 0;
            tp.T = std::min(params->T, 8);
            tp.first_iter = 1;
            tp.update_last = 0;
            tp.freeze_iters = 0;   // trials time the full work of every contour
            tp.cull_iter = 0;
            double per = 1.0;
            for (int d = 0; d < 3; ++d) {
                tp.brick[d] = d < v0->ndim ? std::max(1, (int)std::lround(cl[d] * stride_hint / v0->sp[d])) : 0;
                if (d < v0->ndim) per *= cl[d];
            }
            if (per * G / 32.0 > 16.0) continue;   // more groups than a CTA holds
            Prepared pr;
            if (prepare_sets(tsets.data(), nullptr, n_sets, &tp, nullptr, tmp[0].scratch, pr, st) != AC_OK) continue;
            if (enqueue_prepared(pr, tmp[0].scratch, st, nullptr, false) != AC_OK) continue;   // warm-up
            float ms = 1e30f;
            bool ok = true;
            for (int rep = 0; rep < 2 && ok; ++rep) {   // best of two timed trials
                cudaEventRecord(t0, st);
                ok = enqueue_prepared(pr, tmp[0].scratch, st, nullptr, false) == AC_OK;
                cudaEventRecord(t1, st);
                float t = 0;
                ok = ok && cudaEventSynchronize(t1) == cudaSuccess && cudaEventElapsedTime(&t, t0, t1) == cudaSuccess;
                if (ok) ms = std::min(ms, t);
            }
            if (!ok) continue;
            if (ms < best_ms) {
                best_ms = ms;
                best = TuneVal{G, pr.pl.warps, {tp.brick[0], tp.brick[1], tp.brick[2]}};
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaStreamSynchronize(st);
    cudaGetLastError();
    cleanup();
    if (best.G == 0) AC_FAIL(AC_ERR_ARG, "ac_autotune: no candidate configuration could run");
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    params->lanes_per_contour = best.G;
    params->warps_per_block = best.warps;
    for (int d = 0; d < 3; ++d) params->brick[d] = best.brick[d];
    return AC_OK;
}

extern "C" ac_status ac_evolve(ac_contours *ctr, const ac_evolve_params *params, const ac_trace *trace,
                               void *cuda_stream)
{
    ac::Range nvtx_range("ac_evolve");
    g_err.clear();
    if (!ctr) AC_FAIL(AC_ERR_ARG, "ac_evolve: ctr is NULL");
    return evolve_sets(&ctr, nullptr, 1, params, trace, (cudaStream_t)cuda_stream);
}

extern "C" ac_status ac_evolve_batch(ac_contours *const *sets, const ac_batch_item *items, int32_t n_sets,
                                     const ac_evolve_params *params, void *cuda_stream)
{
    ac::Range nvtx_range("ac_evolve_batch");
    g_err.clear();
    if (!sets || n_sets < 1 || n_sets > 4096) AC_FAIL(AC_ERR_ARG, "ac_evolve_batch: need 1..4096 sets");
    return evolve_sets(sets, items, n_sets, params, nullptr, (cudaStream_t)cuda_stream);
}

extern "C" ac_status ac_evolve_stats(ac_contours *ctr, int64_t counts[3], void *cuda_stream)
{
    g_err.clear();
    if (!ctr || !counts) AC_FAIL(AC_ERR_ARG, "ac_evolve_stats: NULL argument");
    unsigned long long c[3];
    AC_CUDA(cudaMemcpyAsync(c, ctr->path_counts, sizeof(c), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream));
    AC_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
    for (int i = 0; i < 3; ++i) counts[i] = (int64_t)c[i];
    return AC_OK;
}

namespace {
__global__ void count_stops_kernel(const int32_t *hold, int64_t C, unsigned long long *out)
{
    unsigned int f = 0, c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t h = hold[i];
        f += (h & HOLD_FROZEN) ? 1u : 0u;
        c += (h & HOLD_CULLED) ? 1u : 0u;
    }
    f = __reduce_add_sync(0xffffffffu, f);
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) {
        if (f) atomicAdd(&out[0], (unsigned long long)f);
        if (c) atomicAdd(&out[1], (unsigned long long)c);
    }
}
}  // namespace

extern "C" ac_status ac_evolve_stops(ac_contours *ctr, int64_t counts[2], void *cuda_stream)
{
    g_err.clear();
    if (!ctr || !counts) AC_FAIL(AC_ERR_ARG, "ac_evolve_stops: NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    AC_CUDA(ctr->scratch.counters.ensure(2 * sizeof(unsigned long long)));
    unsigned long long *d = ctr->scratch.counters.as<unsigned long long>();
    AC_CUDA(cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), st));
    const int64_t blocks = std::min<int64_t>((ctr->C + 255) / 256, 1024);
    if (ctr->C > 0) {
        count_stops_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(ctr->hold, ctr->C, d);
        count_launch();
        AC_CUDA(cudaGetLastError());
    }
    unsigned long long h[2] = {0, 0};
    AC_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    AC_CUDA(cudaStreamSynchronize(st));
    counts[0] = (int64_t)h[0];
    counts[1] = (int64_t)h[1];
    return AC_OK;
}

extern "C" ac_status ac_evolve_kernel_ms(ac_contours *ctr, float *ms)
{
    g_err.clear();
    if (!ctr || !ms) AC_FAIL(AC_ERR_ARG, "ac_evolve_kernel_ms: NULL argument");
    if (!ctr->timed) AC_FAIL(AC_ERR_STATE, "ac_evolve_kernel_ms: no evolution recorded on this handle");
    AC_CUDA(cudaEventSynchronize(ctr->ev1));
    AC_CUDA(cudaEventElapsedTime(ms, ctr->ev0, ctr->ev1));
    return AC_OK;
}

extern "C" ac_status ac_localize(ac_contours *ctr, const ac_localize_params *params, ac_cell *out_host, int64_t cap,
                                 int64_t *n_out, void *cuda_stream)
{
    ac::Range nvtx_range("ac_localize");
    g_err.clear();
    if (!ctr || !params || !n_out || cap < 0 || (cap > 0 && !out_host)) AC_FAIL(AC_ERR_ARG, "ac_localize: bad arguments");
    if (std::isnan(params->E0)) AC_FAIL(AC_ERR_ARG, "ac_localize: E0 is NaN");
    *n_out = 0;
    return localize_many(&ctr, &params->E0, &out_host, &cap, n_out, 1, (cudaStream_t)cuda_stream);
}

extern "C" ac_status ac_localize_batch(ac_contours *const *sets, int32_t n_sets, const ac_localize_params *params,
                                       ac_cell *const *out_host, const int64_t *caps, int64_t *n_out,
                                       void *cuda_stream)
{
    ac::Range nvtx_range("ac_localize_batch");
    g_err.clear();
    if (n_sets < 0 || (n_sets > 0 && (!sets || !params || !out_host || !caps || !n_out)))
        AC_FAIL(AC_ERR_ARG, "ac_localize_batch: bad arguments");
    std::vector<float> E0((size_t)n_sets);
    for (int32_t i = 0; i < n_sets; ++i) {
        if (!sets[i] || caps[i] < 0 || (caps[i] > 0 && !out_host[i]))
            AC_FAIL(AC_ERR_ARG, "ac_localize_batch: bad arguments for set " + std::to_string(i));
        if (std::isnan(params[i].E0)) AC_FAIL(AC_ERR_ARG, "ac_localize_batch: E0 is NaN for set " + std::to_string(i));
        for (int32_t j = 0; j < i; ++j)
            if (sets[j] == sets[i]) AC_FAIL(AC_ERR_ARG, "ac_localize_batch: a contour set appears twice");
        E0[(size_t)i] = params[i].E0;
        n_out[i] = 0;
    }
    if (n_sets == 0) return AC_OK;
    return localize_many(sets, E0.data(), out_host, caps, n_out, n_sets, (cudaStream_t)cuda_stream);
}
