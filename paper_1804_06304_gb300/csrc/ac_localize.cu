// ac_localize.cu -- energy cull and overlap competition (stage a9).
//
// Section "Results and Discussion" of arXiv:1804.06304: contours with energy above
// E0 are removed, and overlapping contours (|c' - c''| < max(R', R'') / 2^(1/3))
// compete, the lower energy surviving.  Visiting survivors by increasing (E, k)
// and keeping a contour unless a kept one overlaps it defines the result.  The
// GPU computes exactly that set in parallel rounds: a contour is accepted once
// every overlapping contour of higher priority is rejected, and rejected as soon
// as one of them is accepted (the lexicographically first maximal independent
// set).  Neighbours are found through a uniform grid of cell size
// rho max(R), built with a sort.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cub/cub.cuh>
#include <string>
#include <thrust/iterator/counting_iterator.h>

#include "ac_host.h"

#define LC_FAIL(code, msg)        \
    do {                          \
        ac::set_error(msg);       \
        return code;              \
    } while (0)

#define LC_CUDA(call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            ac::set_error(std::string("ac_localize: ") + #call + ": " + cudaGetErrorString(e_));         \
            return e_ == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA;                          \
        }                                                                                               \
    } while (0)

namespace ac {
namespace {

enum : uint8_t { UNDECIDED = 0, ACCEPTED = 1, REJECTED = 2 };

__global__ void flag_kernel(const float *E, int64_t C, float E0, uint8_t *flags)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < C; k += (int64_t)gridDim.x * blockDim.x) {
        const float e = E[k];
        flags[k] = (isfinite(e) && !(e > E0)) ? 1 : 0;
    }
}

__global__ void gather_energy_kernel(const float *E, const int32_t *surv, int64_t n, float *keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = E[surv[i]] + 0.0f;   // -0 and +0 compare equal: one key
}

// positions in priority order and the largest radius (float bits of R > 0 order like ints)
__global__ void positions_kernel(const float *state, int64_t C, const int32_t *order, int64_t n, float4 *pos,
                                 int32_t *maxR_bits)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = order[p];
        const float4 q = make_float4(state[k], state[C + k], state[2 * C + k], state[3 * C + k]);
        pos[p] = q;
        atomicMax(maxR_bits, __float_as_int(q.w));
    }
}

struct Grid {
    float inv_h;
    int nc[3];
};

__device__ __forceinline__ int cell_axis(float x, float inv_h, int nc)
{
    int i = (int)floorf(x * inv_h);
    return i < 0 ? 0 : (i >= nc ? nc - 1 : i);
}

__global__ void cell_kernel(const float4 *pos, int64_t n, Grid g, uint32_t *cellk, uint32_t *celli)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = pos[p];
        const int cx = cell_axis(q.x, g.inv_h, g.nc[0]);
        const int cy = cell_axis(q.y, g.inv_h, g.nc[1]);
        const int cz = cell_axis(q.z, g.inv_h, g.nc[2]);
        cellk[p] = (uint32_t)(cx + (int64_t)g.nc[0] * (cy + (int64_t)g.nc[1] * cz));
        celli[p] = (uint32_t)p;
    }
}

__global__ void cell_start_kernel(const uint32_t *cellk_sorted, int64_t n, int64_t ncells, int32_t *start)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= ncells; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cellk_sorted[mid] < (uint32_t)c) lo = mid + 1; else hi = mid;
        }
        start[c] = (int32_t)lo;
    }
}

// One round of the parallel greedy competition.
__global__ void round_kernel(const float4 *pos, int64_t n, Grid g, const int32_t *start, const uint32_t *celli_sorted,
                             float rho, uint8_t *status, int32_t *undecided)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        if (status[p] != UNDECIDED) continue;
        const float4 a = pos[p];
        const int cx = cell_axis(a.x, g.inv_h, g.nc[0]);
        const int cy = cell_axis(a.y, g.inv_h, g.nc[1]);
        const int cz = cell_axis(a.z, g.inv_h, g.nc[2]);
        bool rejected = false, pending = false;
        for (int dz = -1; dz <= 1 && !rejected; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= g.nc[2]) continue;
            for (int dy = -1; dy <= 1 && !rejected; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= g.nc[1]) continue;
                for (int dx = -1; dx <= 1 && !rejected; ++dx) {
                    const int x = cx + dx;
                    if (x < 0 || x >= g.nc[0]) continue;
                    const int64_t c = x + (int64_t)g.nc[0] * (y + (int64_t)g.nc[1] * z);
                    for (int32_t j = start[c]; j < start[c + 1]; ++j) {
                        const uint32_t q = celli_sorted[j];
                        if ((int64_t)q >= p) continue;   // only higher priority
                        const float4 b = pos[q];
                        const float ex = a.x - b.x, ey = a.y - b.y, ez = a.z - b.z;
                        const float dist = sqrtf(ex * ex + ey * ey + ez * ez);
                        if (!(dist < rho * fmaxf(a.w, b.w))) continue;
                        const uint8_t sq = *(volatile const uint8_t *)&status[q];
                        if (sq == ACCEPTED) {
                            rejected = true;
                            break;
                        }
                        if (sq == UNDECIDED) pending = true;
                    }
                }
            }
        }
        if (rejected) status[p] = REJECTED;
        else if (!pending) status[p] = ACCEPTED;
        else atomicAdd(undecided, 1);
    }
}

__global__ void accepted_flags_kernel(const uint8_t *status, int64_t n, uint8_t *flags)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        flags[p] = status[p] == ACCEPTED ? 1 : 0;
}

__global__ void cells_kernel(const float4 *pos, const int32_t *order, const int32_t *acc, int64_t m, const float *E,
                             float rho, ac_cell *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = acc[i];
        const float4 q = pos[p];
        const int32_t k = order[p];
        ac_cell c;
        c.c[0] = q.x;
        c.c[1] = q.y;
        c.c[2] = q.z;
        c.r = rho * q.w;
        c.E = E[k];
        c.id = k;
        out[i] = c;
    }
}

unsigned blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace

ac_status localize_impl(ac_contours *ctr, float E0, ac_cell *out_host, int64_t cap, int64_t *n_out, cudaStream_t st)
{
    Scratch &sc = ctr->scratch;
    const int64_t C = ctr->C;
    const int ndim = ctr->vol->ndim;
    const float rho = ndim == 3 ? 0.79370052598409973738f : 0.70710678118654752440f;
    *n_out = 0;
    if (C == 0) return AC_OK;
    const float *E = ctr->state + 4 * C;

    // 1. survivors of the energy cull, by contour index
    LC_CUDA(sc.flags.ensure(C));
    LC_CUDA(sc.surv.ensure(sizeof(int32_t) * C));
    LC_CUDA(sc.counters.ensure(sizeof(int32_t) * 8));
    int32_t *cnt = sc.counters.as<int32_t>();
    LC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 8, st));
    flag_kernel<<<blocks_for(C), 256, 0, st>>>(E, C, E0, sc.flags.as<uint8_t>());
    count_launch();
    LC_CUDA(cudaGetLastError());
    thrust::counting_iterator<int32_t> iota(0);
    size_t tmp = 0;
    LC_CUDA(cub::DeviceSelect::Flagged(nullptr, tmp, iota, sc.flags.as<uint8_t>(), sc.surv.as<int32_t>(), cnt, (int)C, st));
    LC_CUDA(sc.cub.ensure(tmp));
    LC_CUDA(cub::DeviceSelect::Flagged(sc.cub.p, tmp, iota, sc.flags.as<uint8_t>(), sc.surv.as<int32_t>(), cnt, (int)C, st));
    int32_t n_surv = 0;
    LC_CUDA(cudaMemcpyAsync(&n_surv, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LC_CUDA(cudaStreamSynchronize(st));
    if (n_surv == 0) return AC_OK;
    const int64_t n = n_surv;

    // 2. priority order: increasing (E, k) -- the radix sort is stable, input is by k
    LC_CUDA(sc.ekeys.ensure(sizeof(float) * 2 * n));
    LC_CUDA(sc.surv_sorted.ensure(sizeof(int32_t) * n));
    float *ek = sc.ekeys.as<float>();
    gather_energy_kernel<<<blocks_for(n), 256, 0, st>>>(E, sc.surv.as<int32_t>(), n, ek);
    count_launch();
    LC_CUDA(cudaGetLastError());
    tmp = 0;
    LC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, ek, ek + n, sc.surv.as<int32_t>(), sc.surv_sorted.as<int32_t>(),
                                            (int)n, 0, 32, st));
    LC_CUDA(sc.cub.ensure(tmp));
    LC_CUDA(cub::DeviceRadixSort::SortPairs(sc.cub.p, tmp, ek, ek + n, sc.surv.as<int32_t>(), sc.surv_sorted.as<int32_t>(),
                                            (int)n, 0, 32, st));
    const int32_t *order = sc.surv_sorted.as<int32_t>();

    // 3. positions in priority order and the neighbour grid
    LC_CUDA(sc.pos.ensure(sizeof(float4) * n));
    float4 *pos = sc.pos.as<float4>();
    positions_kernel<<<blocks_for(n), 256, 0, st>>>(ctr->state, C, order, n, pos, cnt + 1);
    count_launch();
    LC_CUDA(cudaGetLastError());
    int32_t maxR_bits = 0;
    LC_CUDA(cudaMemcpyAsync(&maxR_bits, cnt + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LC_CUDA(cudaStreamSynchronize(st));
    float maxR;
    std::memcpy(&maxR, &maxR_bits, sizeof(float));
    double h = (double)rho * (double)maxR * 1.0001;
    if (!(h > 0.0)) h = 1.0;
    Grid g;
    int64_t ncells = 1;
    for (int pass = 0; pass < 64; ++pass) {
        ncells = 1;
        for (int d = 0; d < 3; ++d) {
            const double top = d < ndim ? (double)(ctr->vol->n[d] - 1) * ctr->vol->sp[d] : 0.0;
            g.nc[d] = (int)std::floor(top / h) + 1;
            ncells *= g.nc[d];
        }
        if (ncells <= ((int64_t)1 << 26)) break;
        h *= 2.0;
    }
    g.inv_h = (float)(1.0 / h);
    LC_CUDA(sc.cellk.ensure(sizeof(uint32_t) * n));
    LC_CUDA(sc.celli.ensure(sizeof(uint32_t) * n));
    LC_CUDA(sc.cellk_s.ensure(sizeof(uint32_t) * n));
    LC_CUDA(sc.celli_s.ensure(sizeof(uint32_t) * n));
    LC_CUDA(sc.cell_start.ensure(sizeof(int32_t) * (ncells + 1)));
    cell_kernel<<<blocks_for(n), 256, 0, st>>>(pos, n, g, sc.cellk.as<uint32_t>(), sc.celli.as<uint32_t>());
    count_launch();
    LC_CUDA(cudaGetLastError());
    int end_bit = 1;
    while (((int64_t)1 << end_bit) < ncells + 1) ++end_bit;
    tmp = 0;
    LC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, sc.cellk.as<uint32_t>(), sc.cellk_s.as<uint32_t>(),
                                            sc.celli.as<uint32_t>(), sc.celli_s.as<uint32_t>(), (int)n, 0, end_bit, st));
    LC_CUDA(sc.cub.ensure(tmp));
    LC_CUDA(cub::DeviceRadixSort::SortPairs(sc.cub.p, tmp, sc.cellk.as<uint32_t>(), sc.cellk_s.as<uint32_t>(),
                                            sc.celli.as<uint32_t>(), sc.celli_s.as<uint32_t>(), (int)n, 0, end_bit, st));
    cell_start_kernel<<<blocks_for(ncells + 1), 256, 0, st>>>(sc.cellk_s.as<uint32_t>(), n, ncells,
                                                              sc.cell_start.as<int32_t>());
    count_launch();
    LC_CUDA(cudaGetLastError());

    // 4. rounds until every survivor is decided (bounded)
    LC_CUDA(sc.stat.ensure(n));
    uint8_t *status = sc.stat.as<uint8_t>();
    LC_CUDA(cudaMemsetAsync(status, UNDECIDED, n, st));
    // every round decides at least the undecided survivor of highest priority, so n
    // rounds always settle it; the bound (n + 8 unless a test lowers it) is checked
    // between batches of up to 8 rounds
    const int64_t max_rounds = localize_round_limit(n);
    int64_t rounds = 0;
    int32_t und = (int32_t)n;
    while (und > 0) {
        if (rounds >= max_rounds) {
            const int32_t bit = STATUS_LOCALIZE_LIMIT;
            LC_CUDA(cudaMemcpyAsync(ctr->status, &bit, sizeof(bit), cudaMemcpyHostToDevice, st));
            LC_CUDA(cudaStreamSynchronize(st));
            LC_FAIL(AC_ERR_TIMEOUT, "ac_localize: competition did not settle within its round bound");
        }
        const int64_t batch = std::min<int64_t>(8, max_rounds - rounds);
        for (int64_t r = 0; r < batch; ++r, ++rounds) {
            LC_CUDA(cudaMemsetAsync(cnt + 2, 0, sizeof(int32_t), st));
            round_kernel<<<blocks_for(n), 256, 0, st>>>(pos, n, g, sc.cell_start.as<int32_t>(), sc.celli_s.as<uint32_t>(),
                                                        rho, status, cnt + 2);
            count_launch();
            LC_CUDA(cudaGetLastError());
        }
        LC_CUDA(cudaMemcpyAsync(&und, cnt + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        LC_CUDA(cudaStreamSynchronize(st));
    }

    // 5. kept contours in priority (= acceptance) order
    LC_CUDA(sc.acc.ensure(sizeof(int32_t) * n));
    accepted_flags_kernel<<<blocks_for(n), 256, 0, st>>>(status, n, sc.flags.as<uint8_t>());
    count_launch();
    LC_CUDA(cudaGetLastError());
    tmp = 0;
    LC_CUDA(cub::DeviceSelect::Flagged(nullptr, tmp, iota, sc.flags.as<uint8_t>(), sc.acc.as<int32_t>(), cnt + 3, (int)n, st));
    LC_CUDA(sc.cub.ensure(tmp));
    LC_CUDA(cub::DeviceSelect::Flagged(sc.cub.p, tmp, iota, sc.flags.as<uint8_t>(), sc.acc.as<int32_t>(), cnt + 3, (int)n, st));
    int32_t m = 0;
    LC_CUDA(cudaMemcpyAsync(&m, cnt + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LC_CUDA(cudaStreamSynchronize(st));
    *n_out = m;
    const int64_t ncopy = m < cap ? m : cap;
    if (ncopy > 0) {
        LC_CUDA(sc.cells.ensure(sizeof(ac_cell) * ncopy));
        cells_kernel<<<blocks_for(ncopy), 256, 0, st>>>(pos, order, sc.acc.as<int32_t>(), ncopy, E, rho,
                                                        sc.cells.as<ac_cell>());
        count_launch();
        LC_CUDA(cudaGetLastError());
        LC_CUDA(cudaMemcpyAsync(out_host, sc.cells.p, sizeof(ac_cell) * ncopy, cudaMemcpyDeviceToHost, st));
        LC_CUDA(cudaStreamSynchronize(st));
    }
    return AC_OK;
}

}  // namespace ac
