/*
 * cdc.h -- C ABI of the GB300 seed-scanning track finder for a cylindrical
 * drift chamber (arXiv:1908.01949, "GPU Tracking in the COMET Phase-I
 * Cylindrical Drift Chamber").
 *
 * Conventions (all entry points):
 *   - Units: mm, MeV/c, T, rad.  A seed is the float32 vector
 *     (theta0, z0, px0, py0, pz0) at the cylinder r = R0 (sec. 2.1: the seed
 *     is defined in front of the first layer, so only five of its six
 *     parameters are scanned).
 *   - "host" pointers are read during the call and not kept; "device" pointers
 *     must be cudaMalloc'ed memory of the context's device (e.g. torch CUDA
 *     tensors).  The caller owns every buffer it passes.
 *   - Compute calls are asynchronous on the given stream (cudaStream_t passed
 *     as void*, NULL = legacy default stream); they allocate nothing and do not
 *     synchronise (one exception: cdc_hough_seeds uploads its vote-offset table
 *     when its radii or angles change).  They return CDC_OK once the work is
 *     enqueued.
 *   - Errors: every call returns a cdc_status; cdc_last_error(ctx) gives a
 *     one-line reason.  Argument errors are detected before anything is
 *     enqueued.  Per-event conditions (step cap reached, full found-hit list,
 *     empty event) are warning bits in the per-event flags output, never
 *     aborts.
 *   - Hits are given per event in CSR form: hit_off[e] .. hit_off[e+1] index
 *     wire_id[] / drift[]; one hit per fired wire (sec. 2.2: the sum of Eq. 1
 *     runs over wires).
 */
#ifndef CDC_H
#define CDC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CDC_MAX_LAYERS 64
#define CDC_MAX_WIRES 8192
#define CDC_MAX_K 64
#define CDC_MAX_ZOOM 8
#define CDC_MAX_ROUNDS 16
#define CDC_MAX_FOUND 256 /* per-seed record: passes of fired wires closer than drift + sqrt(lambda) */

typedef struct cdc_ctx cdc_ctx;

typedef enum {
    CDC_OK = 0,
    CDC_ERR_ARG = -1,        /* null pointer, negative size, inconsistent parameter */
    CDC_ERR_RANGE = -2,      /* a size or value beyond a documented limit */
    CDC_ERR_CUDA = -3,       /* a CUDA runtime call failed (message in cdc_last_error) */
    CDC_ERR_NOT_LOADED = -4, /* geometry or field not loaded, or workspace too small */
    CDC_ERR_TIMEOUT = -5,    /* reserved: a bounded device wait gave up */
    CDC_ERR_NOMEM = -6       /* device allocation failed (only in create/load/reserve) */
} cdc_status;

/* Per-event warning flags (bitmask). */
#define CDC_FLAG_STEP_CAP 1u        /* some seed stopped at max_steps */
#define CDC_FLAG_FOUND_OVERFLOW 2u  /* a seed's record of passes (CDC_MAX_FOUND, compacted when full) or refined hits overflowed */
#define CDC_FLAG_EMPTY 4u           /* no hits, no seeds, no Hough candidate, or grids beyond the reservation */
#define CDC_FLAG_NOT_SPD 8u         /* refine: normal matrix regularised */
#define CDC_FLAG_DOCA_ZERO 16u      /* refine: a hit at zero distance was left out */
#define CDC_FLAG_LOST_HIT 32u       /* refine: an assigned hit had no minimum in its partition */
#define CDC_FLAG_BAD_HIT 64u        /* wire id out of range, duplicate wire, or drift outside [0, max_drift] */

/* One seed grid: the seeds are centre[a] + (i_a - (n[a]-1)/2) * step[a] for
 * i_a in [0, n[a]), enumerated row-major over (theta0, z0, px0, py0, pz0);
 * each value is the float32 nearest that exact number. */
typedef struct {
    float centre[5];
    float step[5];
    int32_t n[5];
} cdc_grid;

/* Parameters of the seed scan (sec. 2.2). */
typedef struct {
    float h;                /* RKN step length [mm], > 0 */
    int32_t max_steps;      /* propagation cap per seed, 1 .. 1<<20 */
    float lambda;           /* cutoff of Eq. 1 [mm^2], > 0 */
    int32_t max_partitions; /* turn partitions followed per seed, 1 .. 16 */
    int32_t direction;      /* +1 propagate along p, -1 against p (exit seeds) */
    float charge;           /* particle charge [e], -1 for the electron */
    int32_t k;              /* best seeds kept per event, 1 .. CDC_MAX_K */
    int32_t n_rounds;       /* scan rounds: 1 coarse + (n_rounds-1) zoom rounds, 1 .. CDC_MAX_ROUNDS */
    int32_t n_zoom;         /* candidates re-scanned per zoom round, 1 .. min(k, CDC_MAX_ZOOM) */
    float max_drift;        /* upper bound of every drift value [mm]; sizes the wire search window */
} cdc_scan_params;

/* Parameters of the circle Hough transform (sec. 2.1, Fig. 4). */
typedef struct {
    int32_t n_bins;         /* accumulator n_bins x n_bins over the circle centre (x0, y0), <= 4096 */
    int32_t bin_um;         /* bin width [um], even, > 0 */
    int32_t origin_um;      /* coordinate of the lower edge of bin 0 [um] (both axes) */
    int32_t n_r;            /* radii R_j = r_min_um + j r_step_um, j < n_r <= 256 */
    int32_t r_min_um;
    int32_t r_step_um;
    int32_t n_phi;          /* vote angles 2 pi k / n_phi, <= 8192 */
    int32_t target_um;      /* circle must pass within this distance of the axis */
    int32_t min_peak;       /* absolute peak threshold */
    int32_t max_cand;       /* candidates kept per event, 1 .. 64 */
    int32_t r_hist_half_um; /* half width of the radius histogram bins [um] */
    float b_nominal;        /* field used to turn the radius into pT [T] */
    float charge;           /* particle charge [e] (sets the sense of rotation) */
    cdc_grid grid_template; /* steps/counts of all axes and the z0, pz0 centres of the output grid */
} cdc_hough_params;

typedef struct {
    int32_t ix, iy, count, r_bin; /* peak bin, votes, radius bin (-1 if none) */
    float theta0, px0, py0;       /* seed centre where the circle meets r = R0 moving outward (NaN if never) */
} cdc_candidate;

/* Parameters of the Gauss-Newton refinement (not in the paper). */
typedef struct {
    int32_t n_iter;         /* Gauss-Newton iterations, 0 .. 32 */
    float sigma;            /* drift resolution in the chi^2 [mm], > 0 */
    float scale[5];         /* parameter scales of the normal equations */
    int32_t checkpoint;     /* adjoint checkpoint interval in steps, 8 .. 512 */
} cdc_refine_params;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  *out receives the handle.
 * Errors: CDC_ERR_ARG (out NULL), CDC_ERR_CUDA (device unusable). */
int cdc_create(cdc_ctx** out, int device);

/* Release the context and all device memory it owns.  NULL is ignored. */
void cdc_destroy(cdc_ctx* ctx);

/* Reason for the last failed call on ctx (static string, never NULL). */
const char* cdc_last_error(const cdc_ctx* ctx);

/* ---- loading (copy host data into the context; synchronous) ------------ */

/* Sense-layer geometry (sec. 1: eighteen stereo layers).  Host arrays of
 * n_layers entries, layers ordered by increasing R: waist radius R [mm] at
 * z = 0, stereo angle alpha [rad], wires N, azimuth phi_off [rad] of wire 0.
 * Wire i of layer l sits at azimuth phi_off + 2 pi i / N at z = 0, direction
 * (-sin a sin phi, sin a cos phi, cos a); global wire ids run layer by layer.
 * z_half: active half length; R0: seed cylinder (sec. 2.1); R_out: outer
 * stop radius.  Errors: CDC_ERR_ARG, CDC_ERR_RANGE (n_layers > 64, total
 * wires > 8192, N outside 32..65535, wire pitch below about 2.1 mm, R not
 * increasing or below 32 mm, |alpha| >= 0.19, R_out above 982 mm),
 * CDC_ERR_NOMEM. */
int cdc_load_geometry(cdc_ctx* ctx, int n_layers, const double* R, const double* alpha, const int32_t* N,
                      const double* phi_off, double z_half, double R0, double R_out);

/* Magnetic field (sec. 1: 1 T solenoid; sec. 2.2: the field is copied to the
 * device).  kind 0: uniform (0, 0, b0).  kind 1: axisymmetric map, host
 * arrays bz, br of nr x nz float32 samples (index ir*nz + iz) at r = r_min +
 * ir dr, z = z_min + iz dz; the field is their bilinear interpolation with
 * coordinates clamped to the grid, Bx = Br x/r, By = Br y/r.
 * Errors: CDC_ERR_ARG, CDC_ERR_RANGE (nr, nz < 2), CDC_ERR_NOMEM. */
int cdc_load_field(cdc_ctx* ctx, int kind, float b0, const float* bz, const float* br, int nr, int nz,
                   float r_min, float z_min, float dr, float dz);

/* Size the context's workspace for calls with up to max_events events,
 * max_seeds seeds in total per scan round, and max_hits hits (besides the
 * per-seed scores and top-K segments, about 190 KB per event: the hit tables,
 * the coarse grid's block order, 64 records of scored wires kept for the
 * classification and the Hough peak search's slice lists).  Compute calls never allocate; a call that exceeds the
 * reservation fails with CDC_ERR_NOT_LOADED.  Errors: CDC_ERR_ARG,
 * CDC_ERR_NOMEM. */
int cdc_reserve(cdc_ctx* ctx, int max_events, int64_t max_seeds, int64_t max_hits);

/* ---- compute ------------------------------------------------------------ */

/* Circle Hough transform and seed-grid centre (sec. 2.1, Fig. 4).  For each
 * event, every hit (its wire at z = 0, rounded to integer um) votes, for each
 * radius R_j and angle phi_k, for the centre X + round(R_j (cos, sin) phi_k)
 * if that circle passes within target_um of the axis; integer arithmetic, so
 * the accumulator is bit-exact in any vote order.  Peaks: count >=
 * max(min_peak, ceil(max/2)), strict 3x3 maxima (equal neighbours resolved to
 * the lower linear index), ordered by (count desc, index asc).  Radius of a
 * peak: the R_j whose [R_j - half, R_j + half) holds most hits.
 * Device inputs: hit_off [n_events+1], wire_id [hits].  Device outputs:
 * acc [n_events][n_bins][n_bins] int32 (row = y bin; overwritten),
 * cand [n_events][max_cand], n_cand [n_events], grid_out [n_events] (nullable:
 * the top candidate's theta0, px0, py0 with the template's other fields; a
 * grid of zero seeds if there is no candidate), flags [n_events].
 * The peak search uses the context's workspace (cdc_reserve with at least
 * n_events events), so calls on one context must not overlap on the GPU.
 * The first call with a new (n_r, r_min_um, r_step_um, n_phi) computes the
 * integer vote offsets on the host and uploads them (a device allocation when
 * the table grows, and a synchronous copy); later calls with those values
 * allocate nothing and are asynchronous.
 * Errors: CDC_ERR_ARG, CDC_ERR_RANGE, CDC_ERR_NOT_LOADED (geometry not loaded,
 * or n_events above the reservation), CDC_ERR_CUDA. */
int cdc_hough_seeds(cdc_ctx* ctx, int n_events, const int32_t* hit_off, const int32_t* wire_id,
                    const cdc_hough_params* params, int32_t* acc, cdc_candidate* cand, int32_t* n_cand,
                    cdc_grid* grid_out, uint32_t* flags, void* stream);

/* One seed grid per Hough candidate (sec. 2.1: each candidate circle gives a
 * seed's theta0 and transverse momentum), so that the scan can search around
 * every candidate instead of the top one only.  For event e and slot
 * c < params->max_cand, grids[e * max_cand + c] = params->grid_template with
 * (theta0, px0, py0) centred on candidate c, or the template with zero seeds
 * where c >= n_cand[e] or the candidate's circle never crosses r = R0 (NaN
 * centre); slot 0 equals the grid cdc_hough_seeds writes to grid_out.  To scan
 * all of them, give cdc_scan_seeds each event's hits once per slot (the CSR
 * with every event repeated max_cand times) and these grids.
 * Device inputs: cand [n_events][max_cand], n_cand [n_events] as
 * cdc_hough_seeds writes them.  Device output: grids [n_events * max_cand].
 * Asynchronous on stream; allocates nothing.
 * Errors: CDC_ERR_ARG (NULL, n_events < 0), CDC_ERR_RANGE (max_cand outside
 * 1..64, n_events > 65535), CDC_ERR_CUDA. */
int cdc_candidate_grids(cdc_ctx* ctx, int n_events, const cdc_hough_params* params, const cdc_candidate* cand,
                        const int32_t* n_cand, cdc_grid* grids, void* stream);

/* Seed scan (sec. 2.2, Eq. 1).  For every seed of grids[e] the track is
 * propagated by RKN steps of length h and scored
 *     E = sum over the event's hits of min( min_k (|DCA_k| - drift)^2, lambda ),
 * DCA_k the distance of closest approach of the continuous track to the wire
 * line within turn partition k (partition k+1 starts at the k-th inward
 * crossing of R0; propagation ends after max_partitions partitions, at
 * |z| > z_half, at r > R_out or after max_steps).  The k best seeds of the
 * coarse grid are kept (order: E, then index), the n_zoom best are re-scanned
 * on 3^5 grids with half the previous step, n_rounds-1 times (sec. 2.2: finer
 * seed sets around the candidates, repeated), and each event's hits are
 * classified for its overall best seed (d^2 < lambda -> partition, else -1).
 * Device inputs: hit_off [n_events+1], wire_id, drift [hits], grids
 * [n_events].  Device outputs: E [sum of grid sizes] (nullable; coarse-round
 * scores, events concatenated), topk0 [n_events][k] (nullable; coarse-round
 * keys (float bits of E << 32) | seed index), best_E [n_events][k],
 * best_seed [n_events][k][5] (best over all rounds), hit_part [hits]
 * (nullable), hit_res2 [hits] (nullable; best squared residual of the best
 * seed), zoom_grids [n_rounds][n_events][n_zoom] (nullable; the grids of each
 * round, round 0 in slot 0), flags [n_events], steps (nullable, [n_rounds]
 * counters: RKN steps executed in each round, added to the current values).
 * The order in which seeds are processed (coarse grids: blocks of equal
 * (z0, pz0), longest estimated track first) changes no output.
 * Errors: CDC_ERR_ARG, CDC_ERR_RANGE, CDC_ERR_NOT_LOADED, CDC_ERR_CUDA. */
int cdc_scan_seeds(cdc_ctx* ctx, int n_events, const int32_t* hit_off, const int32_t* wire_id,
                   const float* drift, const cdc_grid* grids, const cdc_scan_params* params, float* E,
                   uint64_t* topk0, float* best_E, float* best_seed, int8_t* hit_part, float* hit_res2,
                   cdc_grid* zoom_grids, uint32_t* flags, unsigned long long* steps, void* stream);

/* Gauss-Newton refinement of seeds (not in the paper; it refines the scan's
 * surviving seeds in place of the Kalman fit of sec. 2.2).  Each seed first
 * classifies its event's hits as the scan does (d^2 < lambda -> partition);
 * then n_iter iterations minimise chi^2 = sum over classified hits of
 * ((DCA_k - drift)/sigma)^2 with J from forward tangents of the RKN step
 * (theta0's column from the symmetry of the field about z) and an FP64
 * Cholesky solve of the 5x5 normal equations in units of scale.  At most 256
 * classified hits per seed enter chi^2 (more: CDC_FLAG_FOUND_OVERFLOW, the
 * hits beyond the first 256 in the scan's record order are left out).
 * Device inputs: seed_event [n_seeds] (event of each seed, in [0, n_events);
 * a seed with another value gets CDC_FLAG_BAD_HIT and NaN outputs), seeds
 * [n_seeds][5], hit_off [n_events+1], wire_id, drift.  Device outputs: seeds_out
 * [n_seeds][5], chi2 [n_seeds] (FP64, at the refined seed), grad [n_seeds][5]
 * (nullable; d chi^2 / d seed at the refined seed from the adjoint RKN with
 * checkpoints every `checkpoint` steps), n_used [n_seeds] (nullable), flags
 * [n_seeds].  scan supplies h, max_steps, lambda, max_partitions, direction,
 * charge, max_drift; max_steps must stay below 64 * checkpoint.  Uses the
 * context's drift-table workspace (n_events <= reserved events).
 * Errors: CDC_ERR_ARG, CDC_ERR_RANGE, CDC_ERR_NOT_LOADED, CDC_ERR_CUDA. */
int cdc_refine_seeds(cdc_ctx* ctx, int n_seeds, const int32_t* seed_event, const float* seeds, int n_events,
                     const int32_t* hit_off, const int32_t* wire_id, const float* drift,
                     const cdc_scan_params* scan, const cdc_refine_params* params, float* seeds_out,
                     double* chi2, float* grad, int32_t* n_used, uint32_t* flags, void* stream);

/* chi^2 of fixed seeds and its gradient by the adjoint RKN kernel (the
 * backward half of cdc_refine_seeds, exposed for autograd).  Hit
 * classification as in cdc_refine_seeds, at the given seed.  Device outputs:
 * chi2 [n_seeds] (FP64), grad [n_seeds][5] (nullable).  Errors as above. */
int cdc_chi2_grad(cdc_ctx* ctx, int n_seeds, const int32_t* seed_event, const float* seeds, int n_events,
                  const int32_t* hit_off, const int32_t* wire_id, const float* drift,
                  const cdc_scan_params* scan, const cdc_refine_params* params, double* chi2, float* grad,
                  int32_t* n_used, uint32_t* flags, void* stream);

/* Recorded propagation (the RKN of sec. 2.2, for checking propagated
 * positions and for the precision sweep).  Each seed is propagated with the
 * scan's stop rules; every `every` steps (starting at step `every`) the
 * position is written, up to n_rec records.  precision 0: FP32 with
 * compensated state (the scan's stepper); 1: FP64; 2: FP32 with compensated
 * state and a two-float q/p (the refine's stepper).  Device outputs: pos
 * [n_seeds][n_rec][3] float64 (NaN after the track ended), n_steps [n_seeds],
 * path [n_seeds] (FP64 path length).  Errors as above. */
int cdc_propagate(cdc_ctx* ctx, int n_seeds, const float* seeds, const cdc_scan_params* scan, int every,
                  int n_rec, int precision, double* pos, int32_t* n_steps, double* path, void* stream);

/* Kernel timer for measurement (no counterpart in the paper): while enabled,
 * CUDA events are recorded on the call's stream immediately before and after
 * every launch of the seed-scan kernel (the scan's dominant kernel), up to
 * 1024 launches.  cdc_kernel_time waits for the recorded events, returns the
 * summed device time [ms], the number of timed launches since the last read
 * and (per_launch_ms nullable, host, cap entries) each launch's time in launch
 * order, and clears them.  enable: 0 off; 1 on; 2 on for a scan captured into
 * a CUDA graph: the marks become event-record nodes of the graph, every
 * replay records them again, and reads do not clear them (read after each
 * replay; enabling again clears them).  Errors: CDC_ERR_ARG, CDC_ERR_CUDA. */
int cdc_kernel_timer(cdc_ctx* ctx, int enable);
int cdc_kernel_time(cdc_ctx* ctx, double* total_ms, int64_t* launches, float* per_launch_ms, int cap);

/* FP32 FMA throughput of the context's GPU (measurement aid, no counterpart
 * in the paper): the denominator of the scan kernel's FP32 roofline.  Launches
 * a kernel in which every thread runs eight independent FMA chains of
 * 16 * iters FMAs each, on every SM at full occupancy, once to warm up and
 * once timed with CUDA events on `stream`; synchronous.  Outputs (host):
 * tflops = 2 FMAs / time [TFLOP/s], ms = the timed launch.  iters 1 .. 2^20
 * (4096 runs ~4 ms on a GB300).  Errors: CDC_ERR_ARG, CDC_ERR_RANGE,
 * CDC_ERR_CUDA. */
int cdc_fp32_peak(cdc_ctx* ctx, int iters, double* tflops, double* ms, void* stream);

/* ---- launch shape of the seed scan and its autotuner -------------------- */

/* Launch shape of the seed scan (no counterpart in the paper, which launches
 * one block per seed, sec. 2.2).  block = threads, i.e. seeds in flight, per
 * block of the one-lane-per-seed kernel (128 or 256); chunk = RKN steps a lane
 * takes between seed refills (16 or 32); warp_seeds = zoom rounds with at most
 * this many seeds (n_events * n_zoom * 243) run one warp per seed instead,
 * which shortens rounds too small to fill the GPU (0: never).  128-thread
 * blocks keep 896 resident threads per SM, 256-thread blocks 768; the results
 * do not depend on block and chunk, and the warp kernel records the same
 * minima in the same order.  A new context uses {128, 32, 16 * number of
 * SMs}. */
typedef struct {
    int32_t block;
    int32_t chunk;
    int32_t warp_seeds;
} cdc_scan_config;

#define CDC_SCAN_CONFIGS 4 /* shapes tried by cdc_tune_scan, in this order: */
/* {256, 16}, {256, 32}, {128, 16}, {128, 32} */

/* Set / read the shape used by later cdc_scan_seeds calls on ctx.  Errors:
 * CDC_ERR_ARG (NULL), CDC_ERR_RANGE (block not 128/256, chunk not 16/32 or
 * warp_seeds < 0). */
int cdc_set_scan_config(cdc_ctx* ctx, const cdc_scan_config* cfg);
int cdc_get_scan_config(const cdc_ctx* ctx, cdc_scan_config* cfg);

/* Autotuner: runs the coarse round of the given events (arguments as in
 * cdc_scan_seeds, device pointers; params->n_rounds is taken as 1) once as a
 * warm-up and `reps` (1..20) more times under each of the CDC_SCAN_CONFIGS
 * (block, chunk) shapes, keeps the one with the lowest median time for later
 * scans on ctx (warp_seeds is left as set),
 * and returns it in best (host, nullable) and each shape's median time [ms]
 * in ms (host, CDC_SCAN_CONFIGS entries, nullable).  Synchronous setup call:
 * it allocates and frees temporary device buffers and waits for the GPU, so it
 * must not run during stream capture.  Errors as cdc_scan_seeds, plus
 * CDC_ERR_NOMEM. */
int cdc_tune_scan(cdc_ctx* ctx, int n_events, const int32_t* hit_off, const int32_t* wire_id, const float* drift,
                  const cdc_grid* grids, const cdc_scan_params* params, int reps, cdc_scan_config* best, float* ms,
                  void* stream);

/* ---- the paper's two-kernel scan (A/B reference) ------------------------ */

/* Workspace of cdc_scan_seeds_split: room for the recorded states of `chunk`
 * seeds with up to max_steps steps (2 x 16 B per step and seed).  Errors:
 * CDC_ERR_ARG, CDC_ERR_RANGE (chunk outside 1..2^20, max_steps outside
 * 1..6900), CDC_ERR_NOMEM. */
int cdc_reserve_split(cdc_ctx* ctx, int chunk, int max_steps);

/* The coarse scan organised as the paper's two separate kernels (sec. 4.2:
 * propagation, then the distance search): for `chunk` seeds at a time, kernel
 * A (one thread per seed) records the state after every RKN step to the end of
 * the track, then kernel B (one block per seed, threads over the event's hits: the block-per-seed,
 * thread-per-wire layout of sec. 2.2) finds every hit's distance of closest
 * approach from the recorded states and sums Eq. 1.  Same minima and scores as
 * cdc_scan_seeds (up to the order of the Eq. 1 sum), one round only, scores
 * only: E [n_seeds] (device, float32, by row-major seed index), flags
 * [n_events].  n_seeds must equal the grids' total seed count (seeds beyond
 * the true total are skipped, their E left unwritten); duplicate wires in an
 * event (flagged CDC_FLAG_BAD_HIT) are scored per hit here.  params->max_steps
 * must not exceed the reserved max_steps.  Errors as cdc_scan_seeds, plus
 * CDC_ERR_NOT_LOADED (no cdc_reserve_split). */
int cdc_scan_seeds_split(cdc_ctx* ctx, int n_events, int64_t n_seeds, const int32_t* hit_off,
                         const int32_t* wire_id, const float* drift, const cdc_grid* grids,
                         const cdc_scan_params* params, float* E, uint32_t* flags, void* stream);

/* ---- the event loop over turn partitions ------------------------------- */

/* Seed of the neighbouring turn partition (sec. 2.3: the seeds of the previous
 * partition are predicted by extrapolating the fitted track backwards; the
 * flowchart of Fig. 7 repeats this partition by partition).  For each seed (a
 * turn's state at its outward R0 crossing) the track is propagated with the
 * scan's step h (the FP32 refine stepper) in `direction` (-1: back to the
 * previous turn, +1: on to the next) to its second change of side of the R0
 * cylinder (starting inside for -1, outside for +1); the crossing point and
 * direction are interpolated linearly in rho between the two states around
 * it, the point projected onto the cylinder: seeds_out [n_seeds][5] (float32,
 * momentum along the forward motion, |p| kept; NaN where none).  status
 * [n_seeds]: 0 found, 1 the track left |z| <= z_half or rho <= R_out first, 2
 * max_steps reached.  scan supplies h, max_steps and charge.  Device arrays.
 * Errors: CDC_ERR_ARG, CDC_ERR_RANGE, CDC_ERR_NOT_LOADED, CDC_ERR_CUDA. */
int cdc_extrapolate_turn(cdc_ctx* ctx, int n_seeds, const float* seeds, const cdc_scan_params* scan, int direction,
                         float* seeds_out, int32_t* status, void* stream);

/* ---- classification quality --------------------------------------------- */

/* Counts for the classification efficiency and purity of sec. 3.1 (Eqs. 2-3):
 * for every event e, counts[e][i + 1][j + 1] = number of hits with truth
 * partition i classified as partition j (i, j in -1 .. n_part - 1; -1 is noise
 * for the truth and "not classified" for the scan; labels outside that range
 * count as -1).  With C_{i->j} = counts[e][i+1][j+1] and C_i its row sum over
 * all j, Eq. 2 is eps_j = C_{j->j} / C_j and Eq. 3 is pi_j = C_{j->j} /
 * sum_{i >= 0} C_{i->j}.  The caller aligns the truth labels with the scan's
 * partition numbering (partition 0 = the turn of the scanned seed).  Device
 * inputs: hit_off [n_events + 1], hit_part and truth_part [H] (int8); device
 * output counts [n_events][n_part + 1][n_part + 1] (int32, overwritten).
 * n_part 1..16.  Errors: CDC_ERR_ARG, CDC_ERR_RANGE, CDC_ERR_CUDA. */
int cdc_classification_counts(cdc_ctx* ctx, int n_events, const int32_t* hit_off, const int8_t* hit_part,
                              const int8_t* truth_part, int n_part, int32_t* counts, void* stream);

/* Eqs. 2-3 of sec. 3.1 from classification counts: with C the element-wise
 * sum of counts[0 .. n_sets - 1] (the layout cdc_classification_counts
 * writes, [n_sets][n_part + 1][n_part + 1] int32, device), eff[j] =
 * C_{j->j} / C_j (all hits of truth partition j, classified anywhere) and
 * pur[j] = C_{j->j} / sum_{i >= 0} C_{i->j} (the signal's hits classified j),
 * j = 0 .. n_part - 1, as float32 on the device (NaN where a denominator is 0).
 * n_part 1..16, n_sets >= 1.  Asynchronous on `stream`.  Errors: CDC_ERR_ARG,
 * CDC_ERR_RANGE, CDC_ERR_CUDA. */
int cdc_efficiency_purity(cdc_ctx* ctx, int n_sets, const int32_t* counts, int n_part, float* eff, float* pur,
                          void* stream);

/* Hits found by both directions of the bidirectional scan (sec. 2.2: the scan
 * runs independently on seeds at the entrance and at the exit of a partition,
 * direction +1 and -1, and a track needs N_c >= 20 common hits): n_common[e] =
 * number of hits h of event e with part_a[h] == pa and part_b[h] == pb, where
 * part_a, part_b are the hit_part outputs of the two scans (for the turn
 * scanned from both ends, pa = pb = 0).  Device inputs hit_off [n_events + 1],
 * part_a, part_b [H] (int8); device output n_common [n_events] (int32).
 * Errors: CDC_ERR_ARG, CDC_ERR_CUDA. */
int cdc_common_hits(cdc_ctx* ctx, int n_events, const int32_t* hit_off, const int8_t* part_a, const int8_t* part_b,
                    int pa, int pb, int32_t* n_common, void* stream);

/* ---- allocation-free scan ---------------------------------------------- */

#define CDC_NOALLOC_MAX_EVENTS 8
#define CDC_NOALLOC_MAX_SEEDS 65536

/* The paper has no counterpart to this call.  It exists for callers that
 * cannot allocate device memory at call time (an allocator callback that must
 * not re-enter cudaMalloc, a process whose device memory belongs to another
 * framework's caching allocator, a real-time loop that forbids allocation
 * after start-up).  It computes what cdc_scan_seeds computes for a
 * single-round scan (params->n_rounds must be 1; no zoom rounds), with the
 * same inputs and outputs, but takes its workspace from a fixed array of
 * about 0.6 MB that the library keeps in device memory on every device where
 * it is loaded (until the process exits) instead of from cdc_reserve; it
 * calls no cudaMalloc, cudaFree or allocating library routine.
 * Limits: n_events <= CDC_NOALLOC_MAX_EVENTS and n_seeds (the number of seeds
 * the grids hold, stated by the caller) <= CDC_NOALLOC_MAX_SEEDS, else
 * CDC_ERR_RANGE; if the grids hold more than n_seeds seeds on the device
 * (whether E is given or not), every event is flagged CDC_FLAG_EMPTY and
 * nothing is scanned or written to E.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), which can load the library's device code and back
 * the array with device memory at that moment (lazy module loading): make
 * that first call at start-up, before any stream capture and outside any
 * context that forbids allocation.  The address is kept for the life of the
 * process; resetting the device's primary context (cudaDeviceReset) is not
 * supported, as for every other call of the context.
 * All calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and corrupt each other's results, so
 * serialise them.  Errors as cdc_scan_seeds. */
int cdc_scan_seeds_noalloc(cdc_ctx* ctx, int n_events, int64_t n_seeds, const int32_t* hit_off,
                           const int32_t* wire_id, const float* drift, const cdc_grid* grids,
                           const cdc_scan_params* params, float* E, uint64_t* topk0, float* best_E, float* best_seed,
                           int8_t* hit_part, float* hit_res2, uint32_t* flags, unsigned long long* steps,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CDC_H */
