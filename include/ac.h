/*
 * ac.h -- C ABI of the GB300 Monte-Carlo snakuscule library (libac.so).
 *
 * Method: Lotfollahi et al., "Three-Dimensional GPU-Accelerated Active Contours
 * for Automated Localization of Cells in Large Images" (arXiv:1804.06304).  Many
 * symmetric contours (spheres in 3D, disks in 2D) are seeded on a lattice over an
 * image, each evolves independently by gradient descent on its energy (Eqs. 5-15),
 * estimated by Monte-Carlo sampling of the ball of radius R + dR/2 (section
 * "Monte-Carlo Integration"), and the converged contours are culled by energy and
 * merged by overlap competition into cell locations (section "Results and
 * Discussion").
 *
 * Conventions shared by every entry point:
 *   - Every function returns an ac_status; nothing throws across the ABI.  On a
 *     failure ac_last_error() returns a message for the calling thread.
 *   - The library owns every device allocation it makes, through the opaque
 *     handles below.  The caller owns host buffers and the CUDA stream
 *     (`cuda_stream` is a cudaStream_t; NULL means the legacy default stream).
 *   - Calls are asynchronous on that stream unless documented as synchronizing.
 *   - Positions are physical: voxel (i, j, k) has its centre at
 *     (i * spacing[0], j * spacing[1], k * spacing[2]).
 *   - A contour handle keeps a reference to its volume; destroy contours before
 *     their volume.
 *   - A CUDA device (the current one) is required; there is no CPU path.
 */
#ifndef AC_H
#define AC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AC_OK = 0,
    AC_ERR_ARG = 1,      /* invalid argument (null pointer, bad size, bad enum)      */
    AC_ERR_OOM = 2,      /* a device or pinned allocation failed                      */
    AC_ERR_CUDA = 3,     /* a CUDA runtime/driver call or a kernel launch failed      */
    AC_ERR_STATE = 4,    /* handle in the wrong state (e.g. no contours evolved)     */
    AC_ERR_TIMEOUT = 5,  /* a bounded device wait gave up (status word set)           */
    AC_ERR_BUDGET = 6,   /* request larger than the configured memory budget          */
    AC_ERR_NUMERIC = 7   /* non-finite contour state detected (status word set)       */
} ac_status;

typedef enum { AC_U8 = 0, AC_U16 = 1, AC_F16 = 2, AC_F32 = 3 } ac_dtype;

typedef enum {
    AC_PATH_BRICK = 0,   /* bricks + halo staged in shared memory by 3D TMA, one
                            persistent pass over all T iterations (default)        */
    AC_PATH_PLAIN = 1,   /* one launch per iteration, gathers from global memory    */
    AC_PATH_GRID = 2     /* Eq. 5 on the voxel grid (the paper's integration before
                            Monte Carlo): the sums run over every voxel centre within
                            R + dR/2, each of measure one voxel volume, instead of N
                            samples (N is ignored); one pass over all iterations,
                            gathers from global memory                              */
} ac_path;

typedef struct ac_volume ac_volume;
typedef struct ac_contours ac_contours;

/* ------------------------------------------------------------------ volume ---- */
/*
 * ac_create_volume -- copy an image into device memory (stage a1).
 * The image I(x) of Eqs. 1-2 / 5: `dims` = (nx, ny, nz) voxels, x fastest; ndim 2
 * ignores nz (use 1).  Every used dimension must be >= 2.  `data` holds the voxels
 * with element strides (1, row_stride, plane_stride); pass row_stride = 0 /
 * plane_stride = 0 for a dense array.  `data_on_device` = 0: `data` is host memory
 * (pinned memory gives an asynchronous copy), 1: device memory of the current
 * device.  The library keeps its own copy in a row-pitched layout (row pitch a
 * multiple of 16 bytes, as TMA requires); `data` may be reused once the stream has
 * passed this call.  Intensity used by the method = intensity_scale * stored value
 * (AC_F16 stores IEEE binary16).  spacing: physical voxel size per axis (> 0).
 * Errors: AC_ERR_ARG on bad sizes/dtype/null, AC_ERR_OOM, AC_ERR_CUDA.
 */
ac_status ac_create_volume(const void *data, int data_on_device, ac_dtype dtype, int ndim,
                           const int64_t dims[3], int64_t row_stride, int64_t plane_stride,
                           const float spacing[3], float intensity_scale, void *cuda_stream,
                           ac_volume **out);
void ac_destroy_volume(ac_volume *vol);

/*
 * ac_load_volume -- copy new voxels of the same extents and type into an existing
 * volume (a new image tile replacing the old one; no allocation).  Arguments as
 * ac_create_volume.  Asynchronous.  Errors: AC_ERR_ARG, AC_ERR_CUDA.
 */
ac_status ac_load_volume(ac_volume *vol, const void *data, int data_on_device, int64_t row_stride,
                         int64_t plane_stride, void *cuda_stream);

/* ------------------------------------------------------------------ seeding --- */
/*
 * Seeding (stage a2).  Lattice: the volume box is tiled by cells of side `stride`
 * (physical units; figures 1b and 4b place neighbours sqrt(1.5) R apart, so
 * R0 = stride / sqrt(1.5) when R0 <= 0), one contour at each cell centre, the
 * leftover split evenly between both ends of each axis; contour index k runs x
 * fastest.  Explicit: `explicit_cR` (host, n_explicit rows of cx, cy, cz, R as
 * float32) places contour k at row k; centres are clamped into the box of voxel
 * centres and radii must lie in (0, 1e6]; a non-NULL `explicit_cR` with
 * n_explicit = 0 gives an empty set (evolution and localization do nothing on it).
 * The contour index k enters the Philox counter, so results do not depend on how
 * contours are scheduled.  Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA.
 */
typedef struct {
    double stride;   /* lattice stride, physical units; ignored when n_explicit > 0 */
    double R0;       /* initial radius; <= 0 selects stride / sqrt(1.5)            */
} ac_seed_params;

ac_status ac_seed(ac_volume *vol, const ac_seed_params *params, const float *explicit_cR,
                  int64_t n_explicit, void *cuda_stream, ac_contours **out);
int64_t ac_contour_count(const ac_contours *ctr);
void ac_destroy_contours(ac_contours *ctr);

/* ac_reseed -- write the lattice of a lattice-seeded handle again (same stride and
 * R0, energies zero) and clear its status word and the stopping-rule state of
 * every contour; no allocation.  Asynchronous.
 * Errors: AC_ERR_ARG, AC_ERR_STATE (handle seeded explicitly), AC_ERR_CUDA. */
ac_status ac_reseed(ac_contours *ctr, void *cuda_stream);

/* ------------------------------------------------------------------ evolution - */
/*
 * ac_evolve -- T iterations of Monte-Carlo gradient descent for every contour
 * (stages a3-a8).  Iteration n, for contour k at centre c and radius R:
 *   samples  x_j = c + (R + dR/2) u_j, j < N, u_j uniform in the unit ball (disk)
 *            from the words 2j and 2j + 1 of the stream Philox4x32-10(counter =
 *            (b, n, k, stream_id), key = (seed low 32 bits, seed high 32 bits)),
 *            b = 0, 1, ..., four words per block, one block per two samples (2D:
 *            one 24-bit uniform per word; 3D: three 21-bit uniforms from the two
 *            words) -- "Monte-Carlo Integration" section;
 *   sums     J = V/N sum S I, J_R = V/N sum dS/dR I, J_c = V/N sum S'(r)(-(x-c)/r) I
 *            with V the volume (area) of the ball and S the four-region weight of
 *            Eq. 5 (linear bands of widths dR and dR / 2^(1/d));
 *   energy   E = J / (2R)^d (Eqs. 5-6), dE/dR = (-d J / R + J_R) / (2R)^d,
 *            dE/dc = J_c / (2R)^d (Eqs. 7-11 in centre/radius form);
 *   update   c -= eps_n/2 dE/dc, R -= eps_n/2 dE/dR, eps_n = eps0/sqrt(n)
 *            (Eqs. 12-15), each step clamped to max_step, R to [Rmin, Rmax] and c
 *            to the box of voxel centres.
 * Iterations run from n = first_iter to first_iter + T - 1; the update after the
 * last one is applied only when update_last is set.  Afterwards each contour holds
 * its centre and radius and the energy of its last evaluation.
 * Stopping rules (convergence freeze and energy culling; 0 disables each): a
 * contour stops when the step an update proposes (the largest absolute change of
 * a centre coordinate or of R, after the clamps) is below freeze_tol for
 * freeze_iters consecutive updates -- that last step is not applied -- or when its
 * energy at iteration cull_iter is above cull_E (no update follows).  A stopped
 * contour keeps the state and energy of its last evaluation and is skipped by
 * later calls until ac_reseed or ac_set_state; the count of consecutive small
 * steps carries over between calls, so resumed runs equal uninterrupted ones.  Arithmetic is
 * FP32 with compensated sums; volumes are read as stored (uint8/uint16/FP16/FP32).  `trace` (optional) records the state
 * and results of every evaluation for contours k in [k_begin, k_end) and
 * iterations n in [t_begin, t_end).  Asynchronous on the stream.
 * Errors: AC_ERR_ARG (bad parameters, trace too small), AC_ERR_OOM, AC_ERR_CUDA.
 * Bounded device waits that give up set the handle's status word, reported as
 * AC_ERR_TIMEOUT by the next synchronizing call.
 */
typedef struct {
    int32_t N;                 /* MC samples per contour and iteration (>= 1)         */
    int32_t T;                 /* iterations (>= 1)                                  */
    float eps0;                /* learning-rate constant, eps_n = eps0 / sqrt(n)      */
    float dR;                  /* fixed band width dR (> 0), physical units           */
    float Rmin, Rmax;          /* radius clamp, 0 < Rmin <= Rmax                      */
    float max_step;            /* per-iteration step clamp (> 0)                      */
    uint64_t seed;             /* Philox key                                          */
    uint32_t stream_id;        /* fourth Philox counter word                          */
    int32_t path;              /* ac_path                                             */
    int32_t lanes_per_contour; /* 4, 8, 16 or 32 lanes cooperate on one contour; 0 =
                                  auto (4 needs compensated sums, fast sampling)      */
    int32_t compensated;       /* 1: compensated (Kahan + TwoSum) sums, 0: plain FP32 */
    int32_t brick[3];          /* brick interior in voxels per axis; 0 = auto          */
    int32_t warps_per_block;   /* 0 = auto                                            */
    int32_t first_iter;        /* iteration number n of the first iteration (0 -> 1)  */
    int32_t update_last;       /* 1: also update after the last evaluation (a run
                                  continued by a later call with first_iter =
                                  first_iter + T then equals one uninterrupted run)   */
    int32_t sampling;          /* sample-point arithmetic: 0 auto (accurate when N < 64),
                                  1 accurate (correctly rounded sqrt/cbrt, ~1 ulp
                                  sine/cosine), 2 fast (hardware approximations,
                                  ~2^-20 absolute direction error)                    */
    float halo_factor;         /* brick halo = halo_factor x the largest initial radius
                                  + dR/2 + 2 voxels (0 = auto); balls that outgrow it
                                  read the global volume for that iteration           */
    float freeze_tol;          /* step below which an update counts as small (>= 0)   */
    int32_t freeze_iters;      /* consecutive small steps that stop a contour (0: off) */
    int32_t cull_iter;         /* iteration whose energy is tested (0: off)           */
    float cull_E;              /* a contour with E > cull_E at cull_iter stops        */
} ac_evolve_params;

typedef struct {
    float *device_buf;  /* (t_end - t_begin) x (k_end - k_begin) x 9 floats, device:
                           cx, cy, cz, R, E, dE/dR, dE/dcx, dE/dcy, dE/dcz          */
    int64_t k_begin, k_end;
    int32_t t_begin, t_end; /* 1-based iterations, t_end exclusive                  */
} ac_trace;

ac_status ac_evolve(ac_contours *ctr, const ac_evolve_params *params, const ac_trace *trace,
                    void *cuda_stream);

/*
 * ac_evolve_batch -- one launch over several contour sets, each on its own volume
 * (the batching form: uneven volumes and contour counts in one pass over all
 * iterations).  params are shared, including the Philox key (params->seed); set i
 * runs iterations items[i].first_iter .. first_iter + n_iter - 1 (update after the
 * last one if items[i].update_last) with fourth counter word items[i].stream_id,
 * so it gives exactly what ac_evolve on that set alone gives with those values.
 * items NULL: every set uses params' stream_id, first_iter, T and update_last.
 * A set with n_iter = 0 is left untouched.  Every set must share dtype and ndim.
 * Each set keeps its own status word: a non-finite state or a wait that gave up is
 * reported by the calls on the set where it happened (ac_get_state, ac_localize).
 * Asynchronous.  Errors as ac_evolve.
 */
typedef struct {
    uint32_t stream_id;   /* fourth Philox counter word of the set             */
    int32_t first_iter;   /* first iteration n (>= 1)                          */
    int32_t n_iter;       /* iterations this call (>= 0)                       */
    int32_t update_last;  /* 1: update after the last one too                  */
} ac_batch_item;

ac_status ac_evolve_batch(ac_contours *const *sets, const ac_batch_item *items, int32_t n_sets,
                          const ac_evolve_params *params, void *cuda_stream);

/*
 * Plans: a launch over fixed contour sets, planned once and launched many times
 * (batching form).  ac_plan_create does the host work of ac_evolve_batch -- brick
 * plan, descriptors, TMA descriptors, scratch -- and uploads it (synchronous).
 * ac_plan_launch enqueues only device work: binning, sort, the evolution kernel;
 * with use_graph = 1 that sequence is captured once into a CUDA graph and replayed
 * on every later launch.  ac_plan_set_items changes the sets' iteration windows
 * and stream words for later launches (a plain-path graph is recaptured when the
 * iteration span changes).  ac_plan_rebind replaces the plan's sets (and their
 * items) for later launches, keeping the plan's parameters and reusing its device
 * buffers, which only grow; it uploads on the stream and does not synchronize.
 * After a rebind (or an item change that alters the launches) the next launch
 * with use_graph = 1 captures again and updates the executable graph in place
 * (cudaGraphExecUpdate) when the launches keep their topology, or instantiates a
 * new one.  After a failed rebind the plan has no sets and its
 * launches return AC_ERR_STATE until a rebind succeeds.  The sets, their volumes
 * and the plan's own buffers must stay alive and unmoved while the plan launches
 * on them; launches on one plan are serialised by the caller's stream.
 * Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA, AC_ERR_STATE.
 */
typedef struct ac_plan ac_plan;
ac_status ac_plan_create(ac_contours *const *sets, const ac_batch_item *items, int32_t n_sets,
                         const ac_evolve_params *params, ac_plan **out);
ac_status ac_plan_rebind(ac_plan *plan, ac_contours *const *sets, const ac_batch_item *items, int32_t n_sets,
                         void *cuda_stream);
ac_status ac_plan_set_items(ac_plan *plan, const ac_batch_item *items, void *cuda_stream);
ac_status ac_plan_launch(ac_plan *plan, int use_graph, void *cuda_stream);
void ac_destroy_plan(ac_plan *plan);

/*
 * ac_autotune -- choose lanes_per_contour, brick and warps_per_block for these sets
 * by timing short trial launches (up to 8 iterations, best of two) of candidate configurations on
 * copies of their state (the sets are not modified), and write them into
 * *params.  A fixed lanes_per_contour is kept; the plain path is left untouched.
 * Results are cached per workload shape (dimension, voxel type, N, summation and
 * sampling mode, lattice spacing, radius, halo factor) for the process.
 * Synchronizes the stream.  Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA.
 */
ac_status ac_autotune(ac_contours *const *sets, int32_t n_sets, ac_evolve_params *params, void *cuda_stream);

/*
 * ac_plan_layout -- the launch layout ac_evolve takes for one contour set of a
 * volume with these extents, voxel type and spacing, seeded with lattice stride
 * `stride` and largest initial radius `r0` (as ac_seed records them), under
 * *params.  The layout is how the brick path of the "Parallel Contour
 * Evaluation" section is laid out on this GPU: lanes per contour, warps per CTA,
 * the brick interior and its halo, and the region each CTA stages into shared
 * memory.  Host logic only (no device work, no allocation): it may be called
 * without a GPU.  dims: x, y, z (z ignored in 2D); spacing likewise.  The
 * plain and grid paths report their lanes and warps; their brick, halo,
 * region and smem_bytes are 0.  Errors: AC_ERR_ARG for the arguments
 * ac_evolve rejects, or a region that cannot fit shared memory.
 */
typedef struct {
    int32_t lanes_per_contour;   /* lanes of a warp that share one contour's samples   */
    int32_t warps_per_block;     /* warps per CTA                                       */
    int32_t brick[3];            /* brick interior, voxels per axis (x, y, z)           */
    int32_t halo[3];             /* halo beyond the brick, voxels per axis              */
    int32_t region[3];           /* staged region per CTA (the TMA box), voxels         */
    int32_t smem_bytes;          /* dynamic shared memory per CTA                       */
} ac_layout;
ac_status ac_plan_layout(int32_t ndim, ac_dtype dtype, const int64_t dims[3], const float spacing[3], double stride,
                         double r0, const ac_evolve_params *params, ac_layout *out);

/*
 * ac_evolve_static -- ac_evolve for callers that cannot allocate device memory.
 * Some callers must not call cudaMalloc: code whose device memory is owned by
 * its own allocator (a framework's caching allocator that has reserved the free
 * memory, or a pool sized once at start-up), and latency-critical loops where an
 * allocation could block or synchronize the device.  This entry point makes no
 * allocation: the caller passes the volume and the contour state in device memory
 * it owns, and every temporary (binning keys, sort space, volume descriptor,
 * TMA descriptor, status word) lives in one file-scope device array of
 * AC_STATIC_SCRATCH_BYTES that every GPU using the library holds until the
 * process exits.  The paper has no counterpart: it describes no memory
 * management.
 *   volume_dev   voxels in device memory of the current device (or managed
 *                memory), element strides (1, row_stride, plane_stride) (0 =
 *                dense); the brick path needs a 16-byte aligned base and
 *                row/plane strides that are multiples of 16 bytes (AC_PATH_PLAIN
 *                takes any layout)
 *   state_dev    5 x n_contours float32 (cx[], cy[], cz[], R[], E[]) in device
 *                memory of the current device (or managed memory), updated in
 *                place; 1 <= n_contours <= AC_STATIC_MAX_CONTOURS
 *   r0, stride   radius and lattice spacing the contours were seeded with (they
 *                size the bricks), > 0
 * Other arguments and the iteration semantics are those of ac_create_volume and
 * ac_evolve.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Every call shares the one array: calls that overlap on the GPU (several
 * streams or threads) race and must be serialised by the caller.  Synchronizes
 * the stream and reports the status word.  Errors: AC_ERR_BUDGET (n_contours or
 * the sort space beyond the array), AC_ERR_ARG, AC_ERR_CUDA, AC_ERR_TIMEOUT,
 * AC_ERR_NUMERIC.
 */
#define AC_STATIC_MAX_CONTOURS (1 << 20)
#define AC_STATIC_SCRATCH_BYTES (32u << 20)
ac_status ac_evolve_static(const void *volume_dev, ac_dtype dtype, int ndim, const int64_t dims[3],
                           int64_t row_stride, int64_t plane_stride, const float spacing[3],
                           float intensity_scale, float *state_dev, int64_t n_contours, float r0,
                           float stride, const ac_evolve_params *params, void *cuda_stream);

/* ------------------------------------------------------------------ localize -- */
/*
 * ac_localize -- energy cull and overlap competition (stage a9, section "Results
 * and Discussion"): contours with E > E0 or non-finite E are removed; the rest are
 * visited in order of increasing (E, k) and a contour is kept unless a kept one
 * overlaps it, overlap meaning |c' - c''| < rho_d max(R', R''), rho_3 = 2^(-1/3),
 * rho_2 = 2^(-1/2).  Writes up to `cap` cells (host memory) in acceptance order and
 * the total count to *n_out (which may exceed cap).  Cell radius = rho_d R.
 * Synchronizes the stream.  Errors: AC_ERR_ARG (also for 2^31 or more contours),
 * AC_ERR_OOM, AC_ERR_CUDA, AC_ERR_TIMEOUT / AC_ERR_NUMERIC when the status word is
 * set.
 */
typedef struct {
    float E0;           /* energy threshold */
} ac_localize_params;

typedef struct {
    float c[3];         /* centre, physical */
    float r;            /* rho_d * R        */
    float E;            /* energy           */
    int32_t id;         /* contour index k  */
} ac_cell;

ac_status ac_localize(ac_contours *ctr, const ac_localize_params *params, ac_cell *out_host,
                      int64_t cap, int64_t *n_out, void *cuda_stream);

/*
 * ac_localize_batch -- ac_localize of n_sets distinct contour sets in one call
 * (the batching form: many tiles evolved by one plan).  Set i uses params[i],
 * writes up to caps[i] cells to out_host[i] (host memory, caller-owned) and its
 * total count to n_out[i]; the cells of each set are those ac_localize gives for
 * it alone.  The sets' work is queued phase by phase on one stream, so the call
 * synchronizes the stream four times (plus once per further eight competition
 * rounds) whatever n_sets is, instead of several times per set.  The first set's
 * handle holds the call's temporary buffers (sized for the whole batch).  Errors:
 * AC_ERR_ARG (NULL arrays, a NULL or repeated set, a negative cap, a NaN E0, more
 * than 65535 sets or 2^31 - 1 contours in one call), and the first failing set's
 * AC_ERR_OOM / AC_ERR_CUDA / AC_ERR_TIMEOUT / AC_ERR_NUMERIC, after which the
 * counts are unspecified.
 */
ac_status ac_localize_batch(ac_contours *const *sets, int32_t n_sets, const ac_localize_params *params,
                            ac_cell *const *out_host, const int64_t *caps, int64_t *n_out, void *cuda_stream);

/* ------------------------------------------------------------------ state ----- */
/*
 * ac_get_state / ac_set_state -- copy the contour state to / from host memory as
 * 5 x C float32, structure of arrays: cx[C], cy[C], cz[C], R[C], E[C].  With the
 * counter-based generator, setting a saved state and evolving from iteration n
 * reproduces an uninterrupted run (see first_iter / update_last).  ac_set_state
 * clamps centres into the box of voxel centres, needs radii in (0, 1e6] and
 * clears the stopping-rule state (see ac_evolve); ac_get_state synchronizes the
 * stream and
 * reports the status word.  Errors: AC_ERR_ARG, AC_ERR_CUDA, AC_ERR_TIMEOUT,
 * AC_ERR_NUMERIC.
 */
ac_status ac_get_state(ac_contours *ctr, float *out_host, void *cuda_stream);
ac_status ac_set_state(ac_contours *ctr, const float *in_host, void *cuda_stream);
/* Device pointer to the same 5 x C float32 state (valid until the handle dies). */
ac_status ac_state_device_ptr(ac_contours *ctr, float **out);

/* ------------------------------------------------------------------ support --- */
/* Philox4x32-10 words for n counters (device buffers of 4 x n uint32, x fastest),
 * computed by the same device routine that draws the samples.  Asynchronous. */
ac_status ac_philox4x32_10(const uint32_t *ctr_dev, uint64_t key, uint32_t *out_dev, int64_t n,
                           void *cuda_stream);

/* Device time in milliseconds of the evolution kernel launch(es) of the last
 * ac_evolve / ac_evolve_batch / ac_plan_launch whose first set is this handle (CUDA
 * events recorded by the library on the launching stream, inside the graph for a
 * graph launch; binning and sorting excluded).  Synchronizes on the end event.  Errors: AC_ERR_ARG, AC_ERR_STATE (nothing evolved yet), AC_ERR_CUDA. */
ac_status ac_evolve_kernel_ms(ac_contours *ctr, float *ms);

/* Contours of this handle stopped by the step rule (counts[0]) and by the energy
 * rule (counts[1]) of ac_evolve_params so far.  Synchronizes the stream.
 * Errors: AC_ERR_ARG, AC_ERR_CUDA. */
ac_status ac_evolve_stops(ac_contours *ctr, int64_t counts[2], void *cuda_stream);

/* Contour-iterations of the last ac_evolve / ac_evolve_batch on this handle by
 * gather path: counts[0] fast (ball inside the staged region and the volume),
 * counts[1] clamped (inside the region, crossing the volume border), counts[2]
 * global fallback (ball outside the staged region; plain path: every one).
 * Synchronizes the stream.  Errors: AC_ERR_ARG, AC_ERR_CUDA. */
ac_status ac_evolve_stats(ac_contours *ctr, int64_t counts[3], void *cuda_stream);

/*
 * ac_set_wait_limits -- lower the bounds of the library's device waits, process
 * wide, so that a test can make a wait give up without faulting or hanging the
 * GPU (the paper has no counterpart).  tma_polls: polls of the first wait of the
 * brick kernel for a brick's TMA load before it gives up (0: give up at once); a
 * brick that gives up records AC_ERR_TIMEOUT in its set's status word, still waits
 * (with the default bound) for its copy in flight, and skips its contours.
 * localize_rounds: rounds of the overlap competition after which ac_localize
 * returns AC_ERR_TIMEOUT (0: before the first round).  A negative value restores
 * the default (2^22 polls; n + 8 rounds for n survivors, which always suffice).
 * Plans and launches prepared afterwards use the new bound.  Always AC_OK.
 */
ac_status ac_set_wait_limits(int64_t tma_polls, int64_t localize_rounds);

/* Number of the library's own kernel launches since it was loaded (all threads).
 * Sorting and selection steps run CUB library kernels, which are not counted. */
int64_t ac_kernel_launches(void);

/* Message for the last failure on this thread ("" if none). */
const char *ac_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AC_H */
