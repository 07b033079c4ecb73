// ac_serve.cu -- serving form: a request loop over image tiles on a native worker
// thread.  The loop is a client of the library's own entry points (volumes,
// lattice seeding, a plan over the resident tiles with per-tile iteration windows,
// and localization; volumes and contour sets allocated from the server's
// stream-ordered pool), so a tile evolves exactly as it would alone: the sample
// counters are (block, n, k, stream_id) under the server's single Philox key, and the
// lane grouping depends only on the evolve parameters, never on the mix.  Three
// streams overlap: uploads of admitted tiles, the rounds, and the localization of
// the tiles the previous round finished.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ac_host.h"
#include "ac_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Tile {
    int64_t ticket = 0;
    const void *data = nullptr;
    int64_t dims[3] = {1, 1, 1};
    int64_t row_stride = 0, plane_stride = 0;
    float spacing[3] = {1, 1, 1};
    float scale = 1.0f;
    uint32_t stream_id = 0;
    int64_t contours = 0, voxels = 0, est_bytes = 0, lattice = 0;
    Clock::time_point t_submit, t_admit, t_done;
    ac_volume *vol = nullptr;
    ac_contours *ctr = nullptr;
    int32_t progress = 0;   // iterations done
    int32_t rounds = 0;
    ac_status status = AC_OK;
    std::string error;
    std::vector<ac_cell> cells;
    int64_t n_cells = 0;
    bool done = false;
    bool traced = false;    // evaluations recorded into `trace` (one traced tile resident at a time)
    ac_trace trace{};
    cudaEvent_t ready = nullptr;   // recorded on the upload stream after upload and seeding
    bool joined = false;           // the round stream waits for `ready`
};

int elem_bytes(int dtype) { return dtype == AC_U8 ? 1 : dtype == AC_F32 ? 4 : 2; }

// Lattice size of ac_seed for this tile (cells of side `stride` per axis).
int64_t lattice_contours(const int64_t dims[3], const float sp[3], int ndim, double stride)
{
    int64_t C = 1;
    for (int d = 0; d < ndim; ++d) C *= std::max<int64_t>(1, (int64_t)std::floor((double)dims[d] * sp[d] / stride));
    return C;
}

}  // namespace

struct ac_server {
    ac_server_params p;
    int device = 0;
    cudaStream_t st = nullptr;             // rounds
    cudaStream_t up_st = nullptr;          // uploads and seeding of admitted tiles
    cudaStream_t loc_st = nullptr;         // localization and release of finished tiles
    cudaMemPool_t pool = nullptr;          // stream-ordered device memory of the tiles
    cudaEvent_t ev_round[2] = {nullptr, nullptr};   // end of the last two rounds
    int ev_i = 0;
    ac::Scratch loc_scratch;               // grow-only localization buffers, lent to each finished tile
    std::vector<Tile *> retiring;          // finished in the last round, not yet localized (worker only)
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Tile *> pending;
    std::vector<Tile *> resident;          // changed by the worker only, under mu
    std::map<int64_t, Tile *> tiles;       // every ticket not yet collected
    int64_t next_ticket = 1;
    bool stop = false;
    int64_t resident_bytes = 0, peak_bytes = 0, rounds = 0, completed = 0, failed = 0, finished = 0;
    int64_t resident_contours = 0;         // lattice sizes of the resident tiles
    bool traced_resident = false;          // a traced tile is resident
    ac_plan *plan = nullptr;               // worker only
};

namespace {

// Releases a tile's device memory in stream order on `st` (after the work already
// queued there).
void release_device(Tile *t, cudaStream_t st)
{
    if (t->ctr) ac::destroy_contours_on(t->ctr, st);
    if (t->vol) ac::destroy_volume_on(t->vol, st);
    if (t->ready) cudaEventDestroy(t->ready);
    t->ctr = nullptr;
    t->vol = nullptr;
    t->ready = nullptr;
}

// Marks a tile finished (caller holds mu).
void finish_locked(ac_server *S, Tile *t, ac_status s, const std::string &err)
{
    t->status = s;
    t->error = err;
    t->t_done = Clock::now();
    t->done = true;
    ++S->finished;
    if (s == AC_OK) ++S->completed;
    else ++S->failed;
}

std::string last_error(const char *what)
{
    std::string m = ac_last_error();
    return std::string(what) + (m.empty() ? "" : ": " + m);
}

// Localizes tiles whose last round ended at event `after`, all in one pass on the
// localization stream (so the round launched since keeps the GPU busy), keeps
// their cells and releases their memory in stream order behind the localization.
void retire(ac_server *S, std::vector<Tile *> &tiles, cudaEvent_t after)
{
    if (tiles.empty()) return;
    cudaStreamWaitEvent(S->loc_st, after, 0);
    const size_t nt = tiles.size();
    std::vector<std::pair<ac_status, std::string>> outcome(nt, {AC_OK, std::string()});
    std::vector<ac_contours *> sets(nt);
    std::vector<ac_cell *> outs(nt);
    std::vector<float> E0(nt, S->p.E0);
    std::vector<int64_t> caps(nt), n_out(nt, 0);
    for (size_t i = 0; i < nt; ++i) {
        tiles[i]->cells.resize((size_t)std::max<int64_t>(1, tiles[i]->contours));
        sets[i] = tiles[i]->ctr;
        outs[i] = tiles[i]->cells.data();
        caps[i] = (int64_t)tiles[i]->cells.size();
    }
    // every finished tile in one pass, the server's buffers lent to the first; if
    // that fails, each tile alone, so that a failure is reported for its own tile
    std::swap(sets[0]->scratch, S->loc_scratch);
    ac_status ls =
        ac::localize_many(sets.data(), E0.data(), outs.data(), caps.data(), n_out.data(), (int)nt, S->loc_st);
    std::swap(sets[0]->scratch, S->loc_scratch);
    if (ls != AC_OK)
        for (size_t i = 0; i < nt; ++i) {
            std::swap(sets[i]->scratch, S->loc_scratch);
            const ac_status li = ac::localize_many(&sets[i], &E0[i], &outs[i], &caps[i], &n_out[i], 1, S->loc_st);
            std::swap(sets[i]->scratch, S->loc_scratch);
            outcome[i] = {li, li == AC_OK ? std::string() : last_error("localize")};
        }
    for (size_t i = 0; i < nt; ++i) {
        Tile *t = tiles[i];
        t->n_cells = outcome[i].first == AC_OK ? n_out[i] : 0;
        t->cells.resize((size_t)std::min<int64_t>(t->n_cells, (int64_t)t->cells.size()));
        t->cells.shrink_to_fit();
        release_device(t, S->loc_st);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = 0; i < tiles.size(); ++i) {
        S->resident_bytes -= tiles[i]->est_bytes;
        S->resident_contours -= tiles[i]->lattice;
        if (tiles[i]->traced) S->traced_resident = false;
        finish_locked(S, tiles[i], outcome[i].first, outcome[i].second);
    }
    tiles.clear();
    S->cv_done.notify_all();
}

// The worker.  Each pass admits waiting tiles (uploaded and seeded on the upload
// stream, joined to the round stream by an event), launches one round over the
// resident tiles on the round stream, and then localizes the tiles that finished
// in the previous round on the localization stream while this round runs.  Tile
// memory comes from the server's pool in stream order, so neither admission nor
// release synchronizes the device.
void serve_loop(ac_server *S)
{
    cudaSetDevice(S->device);
    const int T = S->p.evolve.T;
    bool dirty = true;   // the resident set changed since the plan was bound
    for (;;) {
        std::vector<Tile *> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty() || !S->resident.empty(); });
            if (S->stop) return;
            // arrival order, within the budget and the resident cap
            while (!S->pending.empty()) {
                Tile *t = S->pending.front();
                const int64_t n_res = (int64_t)(S->resident.size() + S->retiring.size() + admit.size());
                if (n_res > 0 && S->resident_bytes + t->est_bytes > S->p.hbm_budget_bytes) break;
                if (S->p.max_resident > 0 && n_res >= S->p.max_resident) break;
                if (n_res > 0 && S->p.max_resident_contours > 0 &&
                    S->resident_contours + t->lattice > S->p.max_resident_contours)
                    break;
                if (t->traced && S->traced_resident) break;   // one traced tile at a time
                if (t->traced) S->traced_resident = true;
                S->pending.pop_front();
                S->resident_bytes += t->est_bytes;
                S->resident_contours += t->lattice;
                S->peak_bytes = std::max(S->peak_bytes, S->resident_bytes);
                admit.push_back(t);
            }
        }
        // upload and seed outside the lock, on the upload stream
        for (Tile *t : admit) {
            t->t_admit = Clock::now();
            ac_status s = ac::create_volume_pooled(S->pool, t->data, 0, (ac_dtype)S->p.dtype, S->p.ndim, t->dims,
                                                   t->row_stride, t->plane_stride, t->spacing, t->scale, S->up_st,
                                                   &t->vol);
            std::string err;
            if (s != AC_OK) err = last_error("upload");
            if (s == AC_OK) {
                ac_seed_params sp{S->p.stride, S->p.R0};
                s = ac::seed_lattice_pooled(S->pool, t->vol, &sp, S->up_st, &t->ctr);
                if (s != AC_OK) err = last_error("seed");
            }
            if (s == AC_OK) {
                t->contours = ac_contour_count(t->ctr);
                cudaError_t e = cudaEventCreateWithFlags(&t->ready, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventRecord(t->ready, S->up_st);
                if (e != cudaSuccess) {
                    s = AC_ERR_CUDA;
                    err = std::string("upload: ") + cudaGetErrorString(e);
                }
            }
            std::lock_guard<std::mutex> lk(S->mu);
            if (s != AC_OK) {
                cudaStreamSynchronize(S->up_st);
                release_device(t, S->up_st);
                S->resident_bytes -= t->est_bytes;
                S->resident_contours -= t->lattice;
                if (t->traced) S->traced_resident = false;
                finish_locked(S, t, s, err);
                S->cv_done.notify_all();
            } else {
                S->resident.push_back(t);
                dirty = true;
            }
        }
        std::vector<Tile *> finished;
        bool launched = false;
        if (!S->resident.empty()) {
            // one round: every resident tile advances up to iters_per_round iterations
            ac::Range nvtx_round("ac_server_round");
            const int n = (int)S->resident.size();
            std::vector<ac_contours *> sets(n);
            std::vector<ac_batch_item> items(n);
            int64_t largest = 1;
            for (Tile *t : S->resident) largest = std::max(largest, t->lattice);
            for (int i = 0; i < n; ++i) {
                Tile *t = S->resident[i];
                // a round lasts about as long as its largest tile's share: smaller tiles can
                // take more iterations in it without lengthening it much
                const int64_t f =
                    S->p.balance_rounds ? std::min<int64_t>(8, std::max<int64_t>(1, largest / t->lattice)) : 1;
                const int m = (int)std::min<int64_t>((int64_t)S->p.iters_per_round * f, T - t->progress);
                sets[i] = t->ctr;
                items[i].stream_id = t->stream_id;
                items[i].first_iter = t->progress + 1;
                items[i].n_iter = m;
                items[i].update_last = t->progress + m < T ? 1 : 0;
                if (!t->joined) {   // the round reads what the upload stream wrote
                    cudaStreamWaitEvent(S->st, t->ready, 0);
                    t->joined = true;
                }
            }
            ac_status s = AC_OK;
            int traced = -1;
            for (int i = 0; i < n; ++i)
                if (S->resident[i]->traced) traced = i;
            if (!S->plan) s = ac_plan_create(sets.data(), items.data(), n, &S->p.evolve, &S->plan);
            else if (dirty) s = ac_plan_rebind(S->plan, sets.data(), items.data(), n, S->st);
            else s = ac_plan_set_items(S->plan, items.data(), S->st);
            if (s == AC_OK && traced >= 0) s = ac::plan_set_trace(S->plan, traced, &S->resident[traced]->trace);
            // graph replay, updated in place after a rebind; rounds with a trace launch directly
            if (s == AC_OK) s = ac_plan_launch(S->plan, traced >= 0 ? 0 : 1, S->st);
            if (s == AC_OK && cudaEventRecord(S->ev_round[S->ev_i], S->st) != cudaSuccess) {
                ac::set_error("cudaEventRecord failed");
                s = AC_ERR_CUDA;
            }
            if (s != AC_OK) {
                // the launch failed for the whole mix: end every resident tile with it
                const std::string err = last_error("round");
                cudaStreamSynchronize(S->st);
                cudaStreamSynchronize(S->up_st);
                std::lock_guard<std::mutex> lk(S->mu);
                for (Tile *t : S->resident) {
                    release_device(t, S->st);
                    S->resident_bytes -= t->est_bytes;
                    S->resident_contours -= t->lattice;
                    finish_locked(S, t, s, err);
                }
                S->resident.clear();
                S->traced_resident = std::any_of(S->retiring.begin(), S->retiring.end(),
                                                 [](const Tile *t) { return t->traced; });
                if (S->plan) ac_destroy_plan(S->plan);
                S->plan = nullptr;
                dirty = true;
                S->cv_done.notify_all();
            } else {
                launched = true;
                dirty = false;
                std::vector<Tile *> keep;
                for (int i = 0; i < n; ++i) {
                    Tile *t = S->resident[i];
                    t->progress += items[i].n_iter;
                    t->rounds += 1;
                    (t->progress >= T ? finished : keep).push_back(t);
                }
                if (!finished.empty()) dirty = true;   // the plan still refers to them: rebind next round
                std::lock_guard<std::mutex> lk(S->mu);
                S->resident = keep;
                S->retiring.insert(S->retiring.end(), finished.begin(), finished.end());
                ++S->rounds;
            }
        }
        // tiles that finished in the previous round are localized while this one runs
        std::vector<Tile *> prev;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Tile *t : S->retiring)
                if (std::find(finished.begin(), finished.end(), t) == finished.end()) prev.push_back(t);
        }
        retire(S, prev, S->ev_round[S->ev_i ^ 1]);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->retiring = finished;
        }
        if (launched) S->ev_i ^= 1;
        // nothing left to overlap with: localize this round's finished tiles now
        bool idle;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            idle = S->resident.empty() && S->pending.empty();
        }
        if (idle && !finished.empty()) {
            std::vector<Tile *> now = finished;
            retire(S, now, S->ev_round[S->ev_i ^ 1]);
            std::lock_guard<std::mutex> lk(S->mu);
            S->retiring.clear();
        }
    }
}

}  // namespace

extern "C" ac_status ac_server_create(const ac_server_params *params, ac_server **out)
{
    if (!out) AC_FAIL(AC_ERR_ARG, "ac_server_create: out is NULL");
    *out = nullptr;
    if (!params) AC_FAIL(AC_ERR_ARG, "ac_server_create: params is NULL");
    const ac_server_params &p = *params;
    if (p.dtype < AC_U8 || p.dtype > AC_F32) AC_FAIL(AC_ERR_ARG, "ac_server_create: unknown dtype");
    if (p.ndim != 2 && p.ndim != 3) AC_FAIL(AC_ERR_ARG, "ac_server_create: ndim must be 2 or 3");
    if (!(p.stride > 0.0f) || !std::isfinite(p.stride)) AC_FAIL(AC_ERR_ARG, "ac_server_create: stride must be positive");
    if (!(p.R0 >= 0.0f) || !std::isfinite(p.R0)) AC_FAIL(AC_ERR_ARG, "ac_server_create: R0 must be >= 0");
    if (!std::isfinite(p.E0)) AC_FAIL(AC_ERR_ARG, "ac_server_create: E0 must be finite");
    if (p.iters_per_round < 1) AC_FAIL(AC_ERR_ARG, "ac_server_create: iters_per_round must be >= 1");
    if (p.max_resident < 0) AC_FAIL(AC_ERR_ARG, "ac_server_create: max_resident must be >= 0");
    if (p.hbm_budget_bytes <= 0) AC_FAIL(AC_ERR_ARG, "ac_server_create: hbm_budget_bytes must be positive");
    if (p.max_resident_contours < 0) AC_FAIL(AC_ERR_ARG, "ac_server_create: max_resident_contours must be >= 0");
    if (p.balance_rounds != 0 && p.balance_rounds != 1) AC_FAIL(AC_ERR_ARG, "ac_server_create: balance_rounds must be 0 or 1");
    ac_status s = ac::check_evolve_params(&p.evolve);
    if (s != AC_OK) return s;
    ac_server *S = new ac_server();
    S->p = p;
    S->p.evolve.first_iter = 0;
    S->p.evolve.update_last = 0;
    cudaError_t e = cudaGetDevice(&S->device);
    // The upload and localization streams run at the highest priority: a round's
    // evolution fills every SM, and their short kernels (seeding, localization)
    // then take SMs as the round's blocks retire instead of waiting for its end.
    int prio_low = 0, prio_high = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S->up_st, cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S->loc_st, cudaStreamNonBlocking, prio_high);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&S->ev_round[i], cudaEventDisableTiming);
    if (e == cudaSuccess) {
        // the tiles' memory pool keeps up to the budget cached between tiles
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = S->device;
        e = cudaMemPoolCreate(&S->pool, &props);
        uint64_t keep = (uint64_t)p.hbm_budget_bytes;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        const std::string msg = std::string("ac_server_create: ") + cudaGetErrorString(e);
        for (cudaStream_t q : {S->st, S->up_st, S->loc_st})
            if (q) cudaStreamDestroy(q);
        for (cudaEvent_t ev : S->ev_round)
            if (ev) cudaEventDestroy(ev);
        if (S->pool) cudaMemPoolDestroy(S->pool);
        delete S;
        AC_FAIL(AC_ERR_CUDA, msg);
    }
    S->worker = std::thread(serve_loop, S);
    *out = S;
    return AC_OK;
}

extern "C" ac_status ac_server_submit(ac_server *S, const void *data_host, const int64_t dims[3], int64_t row_stride,
                                      int64_t plane_stride, const float spacing[3], float intensity_scale,
                                      uint32_t stream_id, int64_t *ticket)
{
    return ac_server_submit_traced(S, data_host, dims, row_stride, plane_stride, spacing, intensity_scale, stream_id,
                                   nullptr, ticket);
}

extern "C" ac_status ac_server_submit_traced(ac_server *S, const void *data_host, const int64_t dims[3],
                                             int64_t row_stride, int64_t plane_stride, const float spacing[3],
                                             float intensity_scale, uint32_t stream_id, const ac_trace *trace,
                                             int64_t *ticket)
{
    if (!S || !data_host || !dims || !spacing || !ticket) AC_FAIL(AC_ERR_ARG, "ac_server_submit: NULL argument");
    *ticket = 0;
    const int nd = S->p.ndim;
    for (int d = 0; d < 3; ++d) {
        const int64_t want_min = d < nd ? 2 : 1;
        if (dims[d] < want_min || dims[d] > ((int64_t)1 << 24) || (d >= nd && dims[d] != 1))
            AC_FAIL(AC_ERR_ARG, "ac_server_submit: bad dims");
        if (d < nd && (!(spacing[d] > 0.0f) || !std::isfinite(spacing[d])))
            AC_FAIL(AC_ERR_ARG, "ac_server_submit: spacing must be positive");
    }
    Tile *t = new Tile();
    std::memcpy(t->dims, dims, sizeof(t->dims));
    std::memcpy(t->spacing, spacing, sizeof(t->spacing));
    for (int d = nd; d < 3; ++d) t->spacing[d] = 1.0f;
    t->data = data_host;
    t->row_stride = row_stride;
    t->plane_stride = plane_stride;
    t->scale = intensity_scale;
    t->stream_id = stream_id;
    t->voxels = dims[0] * dims[1] * dims[2];
    const int es = elem_bytes(S->p.dtype);
    const int64_t pitch = (dims[0] * es + 15) / 16 * 16;
    const int64_t C = lattice_contours(t->dims, t->spacing, nd, S->p.stride);
    t->lattice = C;
    t->est_bytes = pitch * dims[1] * dims[2] + 100 * C + (1 << 20);
    if (t->est_bytes > S->p.hbm_budget_bytes) {
        delete t;
        AC_FAIL(AC_ERR_BUDGET, "ac_server_submit: the tile alone exceeds the memory budget");
    }
    if (trace && trace->device_buf) {
        if (trace->k_begin < 0 || trace->k_end > C || trace->k_begin > trace->k_end || trace->t_begin < 1 ||
            trace->t_begin > trace->t_end || trace->t_end > S->p.evolve.T + 1) {
            delete t;
            AC_FAIL(AC_ERR_ARG, "ac_server_submit_traced: trace range outside the tile's contours or iterations");
        }
        t->traced = true;
        t->trace = *trace;
    }
    t->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete t;
            AC_FAIL(AC_ERR_STATE, "ac_server_submit: server is stopping");
        }
        t->ticket = S->next_ticket++;
        S->tiles[t->ticket] = t;
        S->pending.push_back(t);
    }
    S->cv_work.notify_one();
    *ticket = t->ticket;
    return AC_OK;
}

extern "C" ac_status ac_server_wait(ac_server *S, int64_t ticket, double timeout_s, ac_cell *cells_out, int64_t cap,
                                    ac_tile_result *result)
{
    if (!S || !result) AC_FAIL(AC_ERR_ARG, "ac_server_wait: NULL argument");
    if (cap > 0 && !cells_out) AC_FAIL(AC_ERR_ARG, "ac_server_wait: cells_out is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->tiles.find(ticket) == S->tiles.end()) AC_FAIL(AC_ERR_ARG, "ac_server_wait: unknown or collected ticket");
    // another thread may collect the ticket while this one waits: look it up again
    // on every wake-up instead of keeping a pointer to the tile
    auto ready = [&] {
        const auto f = S->tiles.find(ticket);
        return f == S->tiles.end() || f->second->done;
    };
    if (timeout_s < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
        AC_FAIL(AC_ERR_TIMEOUT, "ac_server_wait: tile not finished yet");
    const auto it = S->tiles.find(ticket);
    if (it == S->tiles.end()) AC_FAIL(AC_ERR_ARG, "ac_server_wait: ticket collected by another caller");
    Tile *t = it->second;
    std::memset(result, 0, sizeof(*result));
    result->ticket = t->ticket;
    result->status = t->status;
    result->rounds = t->rounds;
    result->n_cells = t->n_cells;
    result->contours = t->contours;
    result->voxels = t->voxels;
    result->est_bytes = t->est_bytes;
    const bool admitted = t->t_admit.time_since_epoch().count() != 0;
    result->queue_ms = ms_between(t->t_submit, admitted ? t->t_admit : t->t_done);
    result->run_ms = admitted ? ms_between(t->t_admit, t->t_done) : 0.0;
    result->total_ms = ms_between(t->t_submit, t->t_done);
    const int64_t n = std::min<int64_t>(cap, (int64_t)t->cells.size());
    if (n > 0) std::memcpy(cells_out, t->cells.data(), sizeof(ac_cell) * (size_t)n);
    const ac_status s = t->status;
    const std::string err = t->error;
    S->tiles.erase(it);
    --S->finished;
    delete t;
    lk.unlock();
    if (s != AC_OK) AC_FAIL(s, "tile " + std::to_string(ticket) + ": " + err);
    return AC_OK;
}

extern "C" ac_status ac_server_get_stats(ac_server *S, ac_server_stats *out)
{
    if (!S || !out) AC_FAIL(AC_ERR_ARG, "ac_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    out->pending = (int64_t)S->pending.size();
    out->resident = (int64_t)S->resident.size();
    out->finished = S->finished;
    out->completed = S->completed;
    out->failed = S->failed;
    out->rounds = S->rounds;
    out->resident_bytes = S->resident_bytes;
    out->peak_resident_bytes = S->peak_bytes;
    out->budget_bytes = S->p.hbm_budget_bytes;
    return AC_OK;
}

extern "C" void ac_server_destroy(ac_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (cudaStream_t q : {S->st, S->up_st, S->loc_st}) cudaStreamSynchronize(q);
    for (Tile *t : S->resident) release_device(t, S->st);
    for (Tile *t : S->retiring) release_device(t, S->st);
    if (S->plan) ac_destroy_plan(S->plan);
    S->loc_scratch.release_all();
    for (auto &kv : S->tiles) delete kv.second;
    cudaStreamSynchronize(S->st);
    for (cudaStream_t q : {S->st, S->up_st, S->loc_st}) cudaStreamDestroy(q);
    for (cudaEvent_t ev : S->ev_round) cudaEventDestroy(ev);
    cudaMemPoolDestroy(S->pool);
    delete S;
}
