/*
 * ac_serve.h -- serving form of libac: a request loop over image tiles.
 *
 * Tiles of different sizes arrive over time; each is uploaded, seeded on the
 * lattice, evolved for T iterations and localized exactly as ac_create_volume /
 * ac_seed / ac_evolve / ac_localize would do it alone (Eqs. 5-15 and the
 * localization rules of section "Results and Discussion"); the paper itself
 * processes one image at a time and has no serving counterpart.
 *
 * A native worker thread runs rounds.  In every round each resident tile advances
 * `iters_per_round` iterations (fewer in its last round) through one batched
 * launch over all resident tiles (an ac_plan, replayed as a CUDA graph that is
 * updated in place when the resident set changes; the per-tile iteration windows
 * of ac_batch_item).  Between rounds, waiting tiles are admitted in arrival order
 * while the estimated device bytes of the resident and not yet released tiles
 * stay within `hbm_budget_bytes` (a tile is admitted when it fits the byte
 * budget, the tile cap and the contour cap; the first tile in line is always
 * admitted when nothing is resident).  The work overlaps on three streams of the
 * server: admitted tiles are uploaded and seeded on an upload stream while the
 * current round runs (the round stream waits on an event before the tile's first
 * round); the tiles a round finishes are localized, their cells kept for the
 * caller, on a localization stream while the next round runs; tile memory comes
 * from a stream-ordered pool of the server (caching up to the budget), so
 * neither admission nor release synchronizes the device.  Because the Philox counters of a
 * sample are (block, n, k, stream_id) with one key for the server, a tile's cells and
 * energies do not depend on which tiles it shared rounds with: they equal those
 * of ac_evolve on that tile alone with the server's evolve parameters and the
 * tile's stream_id.
 *
 * Conventions are those of ac.h.  Every entry point may be called from any host
 * thread, except that no call may be in progress when ac_server_destroy starts.
 */
#ifndef AC_SERVE_H
#define AC_SERVE_H

#include "ac.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ac_server ac_server;

typedef struct {
    ac_evolve_params evolve;    /* N, T (iterations per tile), step sizes, seed (one
                                   Philox key for every tile), path, lanes, ... ;
                                   first_iter and update_last are ignored          */
    int32_t dtype;              /* ac_dtype of every tile                          */
    int32_t ndim;               /* 2 or 3                                          */
    float stride;               /* seeding lattice stride, physical (> 0)          */
    float R0;                   /* initial radius; 0: stride / sqrt(1.5)           */
    float E0;                   /* localization energy threshold                   */
    int32_t iters_per_round;    /* iterations per tile per round (>= 1)            */
    int32_t max_resident;       /* tiles resident at once; 0: budget only          */
    int64_t hbm_budget_bytes;   /* admission budget for resident tiles (> 0)       */
    int64_t max_resident_contours; /* contours resident at once (lattice sizes);
                                   0: no limit.  A few times what the GPU holds in
                                   flight keeps it busy while tiles finish in
                                   arrival order instead of together             */
    int32_t balance_rounds;     /* 1: a tile advances iters_per_round x
                                   min(8, largest resident lattice / its lattice)
                                   iterations per round, so small tiles finish in
                                   fewer rounds; 0: iters_per_round for every tile */
    int32_t reserved_;          /* 0 */
} ac_server_params;

/* Per-tile outcome, filled by ac_server_wait. */
typedef struct {
    int64_t ticket;
    int32_t status;             /* ac_status of the tile                           */
    int32_t rounds;             /* rounds the tile took part in                    */
    int64_t n_cells;            /* cells found (may exceed the caller's cap)       */
    int64_t contours;           /* contours seeded                                 */
    int64_t voxels;
    int64_t est_bytes;          /* device bytes charged against the budget        */
    double queue_ms;            /* submit -> admitted (host steady clock)          */
    double run_ms;              /* admitted -> cells ready                         */
    double total_ms;            /* submit -> cells ready: the tile latency         */
} ac_tile_result;

typedef struct {
    int64_t pending;            /* submitted, not yet admitted                     */
    int64_t resident;           /* admitted, not yet finished                      */
    int64_t finished;           /* finished (successfully or not), not collected   */
    int64_t completed;          /* finished successfully since creation            */
    int64_t failed;             /* finished with an error since creation           */
    int64_t rounds;             /* rounds launched since creation                  */
    int64_t resident_bytes;     /* estimated device bytes of the resident tiles    */
    int64_t peak_resident_bytes;
    int64_t budget_bytes;
} ac_server_stats;

/*
 * ac_server_create -- check the parameters, create the server's stream (on the
 * current device) and start its worker thread.  Errors: AC_ERR_ARG (bad
 * parameters, including every ac_evolve check), AC_ERR_CUDA.
 */
ac_status ac_server_create(const ac_server_params *params, ac_server **out);

/*
 * ac_server_submit -- queue one tile (host memory, `dims` = (nx, ny, nz), x
 * fastest, element strides (1, row_stride, plane_stride), 0 for dense; spacing
 * and intensity_scale as in ac_create_volume) with fourth Philox counter word
 * `stream_id`.  The tile's memory must stay valid and unchanged until
 * ac_server_wait has returned for its ticket (it is read when the tile is
 * admitted; pinned memory makes that copy faster).  The tile's device bytes are
 * estimated as its row-pitched voxel bytes plus 100 bytes per lattice contour plus
 * 1 MiB.  Writes a ticket (> 0).  Errors: AC_ERR_ARG (null pointers, bad sizes),
 * AC_ERR_BUDGET (the tile alone exceeds the budget), AC_ERR_STATE (server
 * stopping).  Never blocks on the device.
 */
ac_status ac_server_submit(ac_server *srv, const void *data_host, const int64_t dims[3], int64_t row_stride,
                           int64_t plane_stride, const float spacing[3], float intensity_scale, uint32_t stream_id,
                           int64_t *ticket);

/*
 * ac_server_submit_traced -- ac_server_submit that also records the tile's
 * evaluations in `trace` (as ac_evolve's trace: device buffer of (t_end - t_begin)
 * x (k_end - k_begin) x 9 floats for the tile's contours k in [k_begin, k_end) and
 * iterations n in [t_begin, t_end), 1 <= t_begin, t_end <= T + 1), so that a served
 * tile can be checked evaluation by evaluation like a tile evolved alone.  The
 * buffer must stay valid until ac_server_wait has returned for the ticket.  One
 * traced tile is resident at a time (a second one waits for the first to finish),
 * and rounds with a traced tile are launched without graph replay.  trace NULL:
 * ac_server_submit.  Errors: those of ac_server_submit; AC_ERR_ARG for a trace
 * range outside the tile's lattice or the server's iterations.
 */
ac_status ac_server_submit_traced(ac_server *srv, const void *data_host, const int64_t dims[3], int64_t row_stride,
                                  int64_t plane_stride, const float spacing[3], float intensity_scale,
                                  uint32_t stream_id, const ac_trace *trace, int64_t *ticket);

/*
 * ac_server_wait -- wait up to `timeout_s` seconds (< 0: forever, 0: poll) for a
 * tile to finish.  When it has: copies up to `cap` cells (acceptance order, as
 * ac_localize) to `cells_out`, fills *result, releases the ticket and returns the
 * tile's own status (AC_OK, or the error that ended it, with its message).  When
 * it has not: returns AC_ERR_TIMEOUT and the ticket stays valid.  Several threads may
 * wait on one ticket: the first to wake collects it, the others return AC_ERR_ARG.
 * Errors: AC_ERR_ARG (unknown or collected ticket, null result), AC_ERR_TIMEOUT, and
 * the tile's errors (AC_ERR_CUDA, AC_ERR_OOM, AC_ERR_NUMERIC, ...).
 */
ac_status ac_server_wait(ac_server *srv, int64_t ticket, double timeout_s, ac_cell *cells_out, int64_t cap,
                         ac_tile_result *result);

/* ac_server_get_stats -- counters of the request loop (host values, no device work). */
ac_status ac_server_get_stats(ac_server *srv, ac_server_stats *out);

/*
 * ac_server_destroy -- stop the worker after its current round, fail the tiles not
 * yet finished, release every device allocation and the stream.  Synchronous.
 */
void ac_server_destroy(ac_server *srv);

#ifdef __cplusplus
}
#endif

#endif
