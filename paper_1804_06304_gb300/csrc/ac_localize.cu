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
//
// Any number of contour sets is localized in one pass: their contours are
// indexed one after another (set-major), the cull and the selection of survivors
// run once over all of them, one sort by (set, E, k) gives every set's priority
// order, every set has its own grid, placed one after another in one cell index
// space sorted once, and each round decides survivors of all sets at once.  A
// batch costs the same few launches and four stream synchronisations whatever
// the number of sets.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cub/cub.cuh>
#include <string>
#include <thrust/iterator/counting_iterator.h>
#include <vector>

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

struct Grid {
    float inv_h;
    int nc[3];
};

// One contour set of a batch, as the kernels see it.
struct LocSet {
    const float *state;       // 5 x C
    const int32_t *status;    // the set's status word
    int64_t C;
    int64_t cbase;            // index of the set's first contour in the batch
    int64_t sbase;            // index of its first survivor (survivors in priority order)
    int64_t n;                // its survivors
    int64_t cellbase;         // index of its first grid cell
    Grid g;
    float E0, rho;
};

// Per-set counters, CNT_N int32 per set in one device array (and its page-locked
// copy); two batch totals follow them.
enum { CNT_SURV, CNT_MAXR, CNT_STATUS, CNT_ABASE, CNT_ACC, CNT_N };

// the set holding batch position `i` of the index whose set offsets are `base`
// (sets in increasing order of their offsets)
template <int64_t LocSet::*base>
__device__ __forceinline__ int set_of(const LocSet *sets, int nsets, int64_t i)
{
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sets[mid].*base <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void status_kernel(const LocSet *sets, int nsets, int32_t *cnt)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsets; s += gridDim.x * blockDim.x)
        cnt[s * CNT_N + CNT_STATUS] = *sets[s].status;
}

// Survivors of the energy cull (flags over the batch's contours), their count
// and largest radius per set (float bits of R > 0 order like ints; one atomic
// per warp).  Block row blockIdx.y is set blockIdx.y; launched with whole warps.
__global__ void flag_kernel(const LocSet *sets, uint8_t *flags, int32_t *cnt)
{
    const LocSet &S = sets[blockIdx.y];
    const float *E = S.state + 4 * S.C, *R = S.state + 3 * S.C;
    int32_t nk = 0, mx = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < S.C; k += (int64_t)gridDim.x * blockDim.x) {
        const float e = E[k];
        const bool keep = isfinite(e) && !(e > S.E0);
        flags[S.cbase + k] = keep ? 1 : 0;
        if (keep) {
            ++nk;
            mx = max(mx, __float_as_int(R[k]));
        }
    }
    nk = __reduce_add_sync(0xffffffffu, nk);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) {
        if (nk) atomicAdd(&cnt[blockIdx.y * CNT_N + CNT_SURV], nk);
        if (mx > 0) atomicMax(&cnt[blockIdx.y * CNT_N + CNT_MAXR], mx);
    }
}

// Sort keys of the survivors: set index above the energy's bits, mapped so that
// unsigned order is the order of the floats (-0 folded into +0).  The survivors
// arrive by batch index, so a stable sort leaves equal energies by k.
__global__ void key_kernel(const LocSet *sets, int nsets, const int32_t *surv, int64_t n, uint64_t *keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = surv[i];
        const int s = set_of<&LocSet::cbase>(sets, nsets, g);
        const LocSet &S = sets[s];
        const uint32_t b = __float_as_uint(S.state[4 * S.C + (g - S.cbase)] + 0.0f);
        const uint32_t u = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
        keys[i] = ((uint64_t)s << 32) | u;
    }
}

// positions in priority order
__global__ void positions_kernel(const LocSet *sets, int nsets, const int32_t *order, int64_t n, float4 *pos)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const LocSet &S = sets[set_of<&LocSet::sbase>(sets, nsets, p)];
        const int64_t k = order[p] - S.cbase;
        pos[p] = make_float4(S.state[k], S.state[S.C + k], S.state[2 * S.C + k], S.state[3 * S.C + k]);
    }
}

__device__ __forceinline__ int cell_axis(float x, float inv_h, int nc)
{
    int i = (int)floorf(x * inv_h);
    return i < 0 ? 0 : (i >= nc ? nc - 1 : i);
}

__global__ void cell_kernel(const LocSet *sets, int nsets, const float4 *pos, int64_t n, uint32_t *cellk,
                            uint32_t *celli)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const LocSet &S = sets[set_of<&LocSet::sbase>(sets, nsets, p)];
        const float4 q = pos[p];
        const int cx = cell_axis(q.x, S.g.inv_h, S.g.nc[0]);
        const int cy = cell_axis(q.y, S.g.inv_h, S.g.nc[1]);
        const int cz = cell_axis(q.z, S.g.inv_h, S.g.nc[2]);
        cellk[p] = (uint32_t)(S.cellbase + cx + (int64_t)S.g.nc[0] * (cy + (int64_t)S.g.nc[1] * cz));
        celli[p] = (uint32_t)p;
    }
}

__global__ void cell_start_kernel(const uint32_t *cellk_sorted, int64_t n, int64_t ncells, int32_t *start)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= ncells; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)cellk_sorted[mid] < c) lo = mid + 1; else hi = mid;
        }
        start[c] = (int32_t)lo;
    }
}

// One round of the parallel greedy competition over the survivors of every set.
// A set's cells hold only its own survivors, and within a set batch order is
// priority order.  `undecided` counts per set what is still open.
__global__ void round_kernel(const LocSet *sets, int nsets, const float4 *pos, int64_t n, const int32_t *start,
                             const uint32_t *celli_sorted, uint8_t *status, int32_t *undecided)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        if (status[p] != UNDECIDED) continue;
        const int s = set_of<&LocSet::sbase>(sets, nsets, p);
        const LocSet &S = sets[s];
        const Grid &g = S.g;
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
                    const int64_t c = S.cellbase + x + (int64_t)g.nc[0] * (y + (int64_t)g.nc[1] * z);
                    for (int32_t j = start[c]; j < start[c + 1]; ++j) {
                        const uint32_t q = celli_sorted[j];
                        if ((int64_t)q >= p) continue;   // only higher priority
                        const float4 b = pos[q];
                        const float ex = a.x - b.x, ey = a.y - b.y, ez = a.z - b.z;
                        const float dist = sqrtf(ex * ex + ey * ey + ez * ez);
                        if (!(dist < S.rho * fmaxf(a.w, b.w))) continue;
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
        else atomicAdd(&undecided[s], 1);
    }
}

__global__ void accepted_flags_kernel(const uint8_t *status, int64_t n, uint8_t *flags)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        flags[p] = status[p] == ACCEPTED ? 1 : 0;
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int64_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Where each set's accepted survivors start in the accepted list (which is in
// batch order) and how many there are; *m is the list's length.
__global__ void accepted_ranges_kernel(const LocSet *sets, int nsets, const int32_t *acc, const int32_t *m,
                                       int32_t *cnt)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsets; s += gridDim.x * blockDim.x) {
        const int64_t b = lower_bound_i32(acc, *m, sets[s].sbase);
        const int64_t e = lower_bound_i32(acc, *m, sets[s].sbase + sets[s].n);
        cnt[s * CNT_N + CNT_ABASE] = (int32_t)b;
        cnt[s * CNT_N + CNT_ACC] = (int32_t)(e - b);
    }
}

// the accepted contours as cells, in the order of the accepted list
__global__ void cells_kernel(const LocSet *sets, int nsets, const float4 *pos, const int32_t *order,
                             const int32_t *acc, const int32_t *m, ac_cell *out)
{
    const int64_t lim = *m;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < lim; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = acc[i];
        const LocSet &S = sets[set_of<&LocSet::sbase>(sets, nsets, p)];
        const float4 q = pos[p];
        const int64_t k = order[p] - S.cbase;
        ac_cell c;
        c.c[0] = q.x;
        c.c[1] = q.y;
        c.c[2] = q.z;
        c.r = S.rho * q.w;
        c.E = S.state[4 * S.C + k];
        c.id = (int32_t)k;
        out[i] = c;
    }
}

unsigned blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

int bits_for(uint64_t v)   // smallest b >= 1 with v < 2^b
{
    int b = 1;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

}  // namespace

ac_status localize_many(ac_contours *const *sets, const float *E0, ac_cell *const *out_host, const int64_t *cap,
                        int64_t *n_out, int nsets, cudaStream_t st)
{
    if (nsets <= 0) return AC_OK;
    if (nsets > 65535) LC_FAIL(AC_ERR_ARG, "ac_localize: at most 65535 sets per call");
    Scratch &sc = sets[0]->scratch;   // holds the batch's buffers
    std::vector<LocSet> L((size_t)nsets);
    int64_t total = 0, maxC = 0;
    for (int s = 0; s < nsets; ++s) {
        n_out[s] = 0;
        LocSet &S = L[(size_t)s];
        S.state = sets[s]->state;
        S.status = sets[s]->status;
        S.C = sets[s]->C;
        S.cbase = total;
        S.E0 = E0[s];
        S.rho = sets[s]->vol->ndim == 3 ? 0.79370052598409973738f : 0.70710678118654752440f;
        total += S.C;
        maxC = std::max(maxC, S.C);
    }
    if (total >= ((int64_t)1 << 31)) LC_FAIL(AC_ERR_ARG, "ac_localize: more than 2^31 - 1 contours in one call");
    const size_t cnt_ints = (size_t)nsets * CNT_N + 2;
    LC_CUDA(sc.lsets.ensure(sizeof(LocSet) * nsets));
    LC_CUDA(sc.hsets.ensure(sizeof(LocSet) * nsets));
    LC_CUDA(sc.counters.ensure(sizeof(int32_t) * cnt_ints));
    LC_CUDA(sc.hcount.ensure(sizeof(int32_t) * cnt_ints));
    LC_CUDA(sc.und.ensure(sizeof(int32_t) * nsets));
    LocSet *dsets = sc.lsets.as<LocSet>();
    int32_t *cnt = sc.counters.as<int32_t>();
    int32_t *h = sc.hcount.as<int32_t>();
    int32_t *tot = cnt + (size_t)nsets * CNT_N;   // [0] survivors, [1] accepted

    // 1. the cull over every set's contours: flags, per-set counts and largest
    //    radius, the survivors by batch index, and the status words
    std::memcpy(sc.hsets.p, L.data(), sizeof(LocSet) * nsets);
    LC_CUDA(cudaMemcpyAsync(dsets, sc.hsets.p, sizeof(LocSet) * nsets, cudaMemcpyHostToDevice, st));
    LC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * cnt_ints, st));
    status_kernel<<<blocks_for(nsets), 256, 0, st>>>(dsets, nsets, cnt);
    count_launch();
    LC_CUDA(cudaGetLastError());
    if (total > 0) {
        LC_CUDA(sc.flags.ensure(total));
        LC_CUDA(sc.surv.ensure(sizeof(int32_t) * total));
        const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((maxC + 255) / 256, 4096));
        flag_kernel<<<dim3(bx, (unsigned)nsets), 256, 0, st>>>(dsets, sc.flags.as<uint8_t>(), cnt);
        count_launch();
        LC_CUDA(cudaGetLastError());
        thrust::counting_iterator<int32_t> iota(0);
        size_t tmp = 0;
        LC_CUDA(cub::DeviceSelect::Flagged(nullptr, tmp, iota, sc.flags.as<uint8_t>(), sc.surv.as<int32_t>(), tot,
                                           (int)total, st));
        LC_CUDA(sc.cub.ensure(tmp));
        LC_CUDA(cub::DeviceSelect::Flagged(sc.cub.p, tmp, iota, sc.flags.as<uint8_t>(), sc.surv.as<int32_t>(), tot,
                                           (int)total, st));
    }
    LC_CUDA(cudaMemcpyAsync(h, cnt, sizeof(int32_t) * cnt_ints, cudaMemcpyDeviceToHost, st));
    LC_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < nsets; ++s) {
        const ac_status e = status_error(h[s * CNT_N + CNT_STATUS]);
        if (e != AC_OK) return e;
    }

    // 2. per set: survivors, the grid (cell size rho max R) and the offsets
    int64_t n = 0, ncells = 0, n_max = 0;
    for (int s = 0; s < nsets; ++s) {
        LocSet &S = L[(size_t)s];
        const ac_volume *v = sets[s]->vol;
        S.sbase = n;
        S.n = h[s * CNT_N + CNT_SURV];
        n += S.n;
        n_max = std::max(n_max, S.n);
        float maxR;
        std::memcpy(&maxR, &h[s * CNT_N + CNT_MAXR], sizeof(float));
        double hc = (double)S.rho * (double)maxR * 1.0001;
        if (!(hc > 0.0)) hc = 1.0;
        int64_t nc = 1;
        for (int pass = 0; pass < 64; ++pass) {
            nc = 1;
            for (int d = 0; d < 3; ++d) {
                const double top = d < v->ndim ? (double)(v->n[d] - 1) * v->sp[d] : 0.0;
                S.g.nc[d] = (int)std::floor(top / hc) + 1;
                nc *= S.g.nc[d];
            }
            if (nc <= ((int64_t)1 << 26)) break;
            hc *= 2.0;
        }
        S.g.inv_h = (float)(1.0 / hc);
        S.cellbase = ncells;
        ncells += S.n > 0 ? nc : 0;
    }
    if (total > 0 && n != h[(size_t)nsets * CNT_N]) LC_FAIL(AC_ERR_CUDA, "ac_localize: survivor counts disagree");
    if (n == 0) return AC_OK;
    if (ncells >= ((int64_t)1 << 31)) LC_FAIL(AC_ERR_OOM, "ac_localize: neighbour grids too large for one call");

    // 3. priority order by (set, E, k), positions, the grids' cells sorted
    std::memcpy(sc.hsets.p, L.data(), sizeof(LocSet) * nsets);
    LC_CUDA(cudaMemcpyAsync(dsets, sc.hsets.p, sizeof(LocSet) * nsets, cudaMemcpyHostToDevice, st));
    LC_CUDA(sc.ekeys.ensure(sizeof(uint64_t) * 2 * n));
    LC_CUDA(sc.surv_sorted.ensure(sizeof(int32_t) * n));
    uint64_t *ek = sc.ekeys.as<uint64_t>();
    int32_t *order = sc.surv_sorted.as<int32_t>();
    key_kernel<<<blocks_for(n), 256, 0, st>>>(dsets, nsets, sc.surv.as<int32_t>(), n, ek);
    count_launch();
    LC_CUDA(cudaGetLastError());
    const int key_bits = nsets > 1 ? 32 + bits_for((uint64_t)(nsets - 1)) : 32;   // one set: the energy bits only
    size_t tmp = 0;
    LC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, ek, ek + n, sc.surv.as<int32_t>(), order, (int)n, 0,
                                            key_bits, st));
    LC_CUDA(sc.cub.ensure(tmp));
    LC_CUDA(cub::DeviceRadixSort::SortPairs(sc.cub.p, tmp, ek, ek + n, sc.surv.as<int32_t>(), order, (int)n, 0,
                                            key_bits, st));
    LC_CUDA(sc.pos.ensure(sizeof(float4) * n));
    float4 *pos = sc.pos.as<float4>();
    positions_kernel<<<blocks_for(n), 256, 0, st>>>(dsets, nsets, order, n, pos);
    count_launch();
    LC_CUDA(cudaGetLastError());
    LC_CUDA(sc.cellk.ensure(sizeof(uint32_t) * n));
    LC_CUDA(sc.cellk_s.ensure(sizeof(uint32_t) * n));
    LC_CUDA(sc.celli.ensure(sizeof(uint32_t) * n));
    LC_CUDA(sc.celli_s.ensure(sizeof(uint32_t) * n));
    LC_CUDA(sc.cell_start.ensure(sizeof(int32_t) * (ncells + 1)));
    cell_kernel<<<blocks_for(n), 256, 0, st>>>(dsets, nsets, pos, n, sc.cellk.as<uint32_t>(), sc.celli.as<uint32_t>());
    count_launch();
    LC_CUDA(cudaGetLastError());
    const int cell_bits = bits_for((uint64_t)ncells);
    tmp = 0;
    LC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, sc.cellk.as<uint32_t>(), sc.cellk_s.as<uint32_t>(),
                                            sc.celli.as<uint32_t>(), sc.celli_s.as<uint32_t>(), (int)n, 0, cell_bits,
                                            st));
    LC_CUDA(sc.cub.ensure(tmp));
    LC_CUDA(cub::DeviceRadixSort::SortPairs(sc.cub.p, tmp, sc.cellk.as<uint32_t>(), sc.cellk_s.as<uint32_t>(),
                                            sc.celli.as<uint32_t>(), sc.celli_s.as<uint32_t>(), (int)n, 0, cell_bits,
                                            st));
    cell_start_kernel<<<blocks_for(ncells + 1), 256, 0, st>>>(sc.cellk_s.as<uint32_t>(), n, ncells,
                                                              sc.cell_start.as<int32_t>());
    count_launch();
    LC_CUDA(cudaGetLastError());

    // 4. rounds until every survivor is decided.  Each round decides at least the
    //    undecided survivor of highest priority of every set, so the largest set's
    //    n rounds settle all; the bound (that n + 8 unless a test lowers it) is
    //    checked between batches of up to eight rounds.
    LC_CUDA(sc.stat.ensure(n));
    uint8_t *status = sc.stat.as<uint8_t>();
    int32_t *und = sc.und.as<int32_t>();
    int32_t *hund = h;   // the page-locked counts are read: reused for the undecided counts
    LC_CUDA(cudaMemsetAsync(status, UNDECIDED, n, st));
    const int64_t max_rounds = localize_round_limit(n_max);
    int64_t rounds = 0;
    for (bool open = true; open;) {
        if (rounds >= max_rounds) {
            const int32_t bit = STATUS_LOCALIZE_LIMIT;
            for (int s = 0; s < nsets; ++s)
                if (L[(size_t)s].n > 0 && (rounds == 0 || hund[s] > 0))
                    LC_CUDA(cudaMemcpyAsync(sets[s]->status, &bit, sizeof(bit), cudaMemcpyHostToDevice, st));
            LC_CUDA(cudaStreamSynchronize(st));
            LC_FAIL(AC_ERR_TIMEOUT, "ac_localize: competition did not settle within its round bound");
        }
        const int64_t batch = std::min<int64_t>(8, max_rounds - rounds);
        for (int64_t r = 0; r < batch; ++r, ++rounds) {
            LC_CUDA(cudaMemsetAsync(und, 0, sizeof(int32_t) * nsets, st));
            round_kernel<<<blocks_for(n), 256, 0, st>>>(dsets, nsets, pos, n, sc.cell_start.as<int32_t>(),
                                                        sc.celli_s.as<uint32_t>(), status, und);
            count_launch();
            LC_CUDA(cudaGetLastError());
        }
        LC_CUDA(cudaMemcpyAsync(hund, und, sizeof(int32_t) * nsets, cudaMemcpyDeviceToHost, st));
        LC_CUDA(cudaStreamSynchronize(st));
        open = false;
        for (int s = 0; s < nsets; ++s) open = open || hund[s] > 0;
    }

    // 5. the kept survivors in batch (= per set, acceptance) order, each set's
    //    range of them, and the cells, copied back after the counts
    LC_CUDA(sc.acc.ensure(sizeof(int32_t) * n));
    accepted_flags_kernel<<<blocks_for(n), 256, 0, st>>>(status, n, sc.flags.as<uint8_t>());
    count_launch();
    LC_CUDA(cudaGetLastError());
    thrust::counting_iterator<int32_t> iota(0);
    tmp = 0;
    LC_CUDA(cub::DeviceSelect::Flagged(nullptr, tmp, iota, sc.flags.as<uint8_t>(), sc.acc.as<int32_t>(), tot + 1,
                                       (int)n, st));
    LC_CUDA(sc.cub.ensure(tmp));
    LC_CUDA(cub::DeviceSelect::Flagged(sc.cub.p, tmp, iota, sc.flags.as<uint8_t>(), sc.acc.as<int32_t>(), tot + 1,
                                       (int)n, st));
    accepted_ranges_kernel<<<blocks_for(nsets), 256, 0, st>>>(dsets, nsets, sc.acc.as<int32_t>(), tot + 1, cnt);
    count_launch();
    LC_CUDA(cudaGetLastError());
    LC_CUDA(sc.cells.ensure(sizeof(ac_cell) * n));
    LC_CUDA(sc.hcells.ensure(sizeof(ac_cell) * n));
    cells_kernel<<<blocks_for(n), 256, 0, st>>>(dsets, nsets, pos, order, sc.acc.as<int32_t>(), tot + 1,
                                                sc.cells.as<ac_cell>());
    count_launch();
    LC_CUDA(cudaGetLastError());
    LC_CUDA(cudaMemcpyAsync(h, cnt, sizeof(int32_t) * cnt_ints, cudaMemcpyDeviceToHost, st));
    LC_CUDA(cudaStreamSynchronize(st));
    const int64_t M = h[(size_t)nsets * CNT_N + 1];   // the cells, contiguous, set by set
    if (M > 0) {
        LC_CUDA(cudaMemcpyAsync(sc.hcells.p, sc.cells.p, sizeof(ac_cell) * M, cudaMemcpyDeviceToHost, st));
        LC_CUDA(cudaStreamSynchronize(st));
    }
    const ac_cell *cells = sc.hcells.as<ac_cell>();
    for (int s = 0; s < nsets; ++s) {
        const int64_t m = h[s * CNT_N + CNT_ACC];
        n_out[s] = m;
        const int64_t k = std::min(m, cap[s]);
        if (k > 0) std::memcpy(out_host[s], cells + h[s * CNT_N + CNT_ABASE], sizeof(ac_cell) * (size_t)k);
    }
    return AC_OK;
}

}  // namespace ac
