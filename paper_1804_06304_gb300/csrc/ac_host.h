// ac_host.h -- host-side internals of libac shared by its translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <string>

#include "ac_internal.cuh"

struct ac_volume {
    int device;
    ac_dtype dtype;
    int ndim;
    int64_t n[3];
    float sp[3];
    float scale;
    int es;               // bytes per voxel
    void *data;           // row-pitched copy
    int64_t pitch_y;      // elements per row
    int64_t pitch_z;      // elements per plane
    size_t bytes;
    cudaMemPool_t pool;   // non-null: `data` is a stream-ordered allocation from this pool
    void *staging = nullptr;     // dense voxels uploaded by ac_load_volume, repacked on the device
    size_t staging_bytes = 0;
};

namespace ac {

// A device buffer that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = bytes + bytes / 4 + 256;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Grow-only page-locked host buffer (device-to-host copies that do not block the
// host until the stream reaches them).
struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t want = bytes + bytes / 4 + 256;
        cudaError_t e = cudaMallocHost(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

struct Scratch {
    DevBuf keys, vals, skeys, svals, cub, desc, tmaps, active;       // evolve
    DevBuf flags, surv, ekeys, surv_sorted, pos, cellk, celli, cellk_s, celli_s, cell_start, stat, acc,
        cells, counters;                                               // localize
    DevBuf lsets, und;                                                 // localize: set descriptors, open counts
    HostBuf hcount, hcells, hsets;                                     // localize: read back / uploaded
    void release_all();
};

}  // namespace ac

struct ac_contours {
    ac_volume *vol = nullptr;
    int64_t C = 0;
    float *state = nullptr;              // 5 x C
    int32_t *status = nullptr;           // device status word
    int32_t *hold = nullptr;             // device [C]: stopping-rule state per contour
    unsigned long long *path_counts = nullptr;   // device [3]: contour-iterations per gather path
    double stride_hint = 0;   // lattice stride (or mean spacing of explicit seeds)
    double r_hint = 0;        // largest initial radius
    ac::Scratch scratch;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the last evolution kernel(s)
    bool lattice = false;                       // lattice-seeded: parameters below
    int64_t L[3] = {1, 1, 1};
    float first[3] = {0, 0, 0};
    float stride = 0, R0 = 0;
    bool timed = false;
    cudaMemPool_t pool = nullptr;        // non-null: state, status, hold and counters come from this pool
};

namespace ac {

// thread-local error message
void set_error(const std::string &msg);

// NVTX range for the lifetime of a scope (visible in profilers' timelines; a no-op
// when no tool is attached)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
// count of the library's own kernel launches
void count_launch(int64_t n = 1);

cudaError_t launch_evolve_u8(const EvolveArgs &a, bool brick, int G, bool comp, bool acc, int warps, int64_t grid,
                             cudaStream_t st);
cudaError_t launch_evolve_u16(const EvolveArgs &a, bool brick, int G, bool comp, bool acc, int warps, int64_t grid,
                              cudaStream_t st);
cudaError_t launch_evolve_f16(const EvolveArgs &a, bool brick, int G, bool comp, bool acc, int warps, int64_t grid,
                              cudaStream_t st);
cudaError_t launch_evolve_f32(const EvolveArgs &a, bool brick, int G, bool comp, bool acc, int warps, int64_t grid,
                              cudaStream_t st);

// the voxel-grid form of Eq. 5 (ac_grid.cu)
cudaError_t launch_grid(ac_dtype t, const EvolveArgs &a, int G, bool comp, int warps, int64_t grid, cudaStream_t st);

// the argument checks of ac_evolve (ac_api.cu)
ac_status check_evolve_params(const ac_evolve_params *p);

// bounds of the device waits (ac_set_wait_limits): polls of the first wait for a
// brick's TMA load, and localization rounds for n survivors
uint32_t tma_poll_limit();
int64_t localize_round_limit(int64_t n);

// Volumes and lattice contour sets whose device memory is allocated from `pool`
// in stream order on `st` (no implicit device synchronisation, unlike cudaMalloc
// and cudaFree), released in stream order on the stream given to the destroy
// functions.  Used by the request loop so that admitting and retiring tiles does
// not stall the rounds running on other streams.
ac_status create_volume_pooled(cudaMemPool_t pool, const void *data, int data_on_device, ac_dtype dtype, int ndim,
                               const int64_t dims[3], int64_t row_stride, int64_t plane_stride,
                               const float spacing[3], float intensity_scale, cudaStream_t st, ac_volume **out);
ac_status seed_lattice_pooled(cudaMemPool_t pool, ac_volume *vol, const ac_seed_params *params, cudaStream_t st,
                              ac_contours **out);
void destroy_contours_on(ac_contours *ctr, cudaStream_t st);
void destroy_volume_on(ac_volume *vol, cudaStream_t st);

// Record the evaluations of set `set` of a plan into `trace` on its later launches
// (nullptr: no trace); drops the plan's captured graph.  Used by the request loop.
ac_status plan_set_trace(ac_plan *plan, int set, const ac_trace *trace);

// localization (ac_localize.cu) of n distinct sets in one pass on one stream,
// each with its own threshold, host output and cap; the first set's scratch holds
// the batch's buffers.  The whole batch synchronizes the stream four times (plus
// once per further eight competition rounds).  Returns an ac_status (the first
// failing set's) and sets the message.
ac_status localize_many(ac_contours *const *sets, const float *E0, ac_cell *const *out_host, const int64_t *cap,
                        int64_t *n_out, int n, cudaStream_t st);

// the error a device status word reports (AC_OK if none), message set (ac_api.cu)
ac_status status_error(int32_t word);

}  // namespace ac

// Error returns of the C ABI entry points: set the calling thread's message.
#define AC_FAIL(code, msg)        \
    do {                          \
        ac::set_error(msg);       \
        return code;              \
    } while (0)

#define AC_CUDA(call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            ac::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                          \
            return e_ == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA;                          \
        }                                                                                               \
    } while (0)
