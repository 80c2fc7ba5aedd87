/*
 * nyxrt.h -- C ABI of the GB300 adaptive ray-march library (libnyxrt.so).
 *
 * The library computes one radiative-transfer step of the adaptive ray
 * tracer of "Nyx-RT: Adaptive Ray Tracing in the Nyx Hydrodynamical Code"
 * (arXiv 2512.12466, Sec. 2.2-2.8): point sources emit rays on HEALPix
 * directions, rays split 4-way where a cell would be covered by fewer than
 * N_min rays (Eq. 4), march cell by cell accumulating optical depth (Eq. 2),
 * and deposit a photon-conserving photoionization rate (Eq. 1, V_box = h^3)
 * with the geometric overlap correction and conservative thresholding
 * (Eqs. 5-8). Sources sharing a cell are merged, sorted, and optionally
 * merged by bubble overlap (Alg. 3). Optionally the step iterates Gamma and
 * the C2-Ray time-averaged ionization update (Eq. 3, Sec. 2.3-2.4).
 *
 * Conventions for every call:
 *   - Grids are cubic, n^3 cells, flat index (iz*n + iy)*n + ix (x fastest),
 *     float64. Cell size dx = box_cm / n; cell volume dx^3.
 *   - `where` says whether a pointer is host memory (RT_HOST) or device
 *     memory of the handle's GPU (RT_DEVICE).
 *   - All device work is enqueued on the CUDA stream given to rt_create.
 *   - Return values: RT_OK (0) or a negative RT_E* code; no exception or
 *     abort crosses the ABI. rt_last_error() describes the last failure.
 *     A device-side error (RT_EDEVICE, RT_ETIMEOUT, RT_ECUDA) is sticky:
 *     later calls on the handle return RT_ESTATE until rt_destroy.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - The library owns the device memory it allocates; inputs are copied.
 */
#ifndef NYXRT_H
#define NYXRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_MAX_LEVELS 16

enum {
    RT_OK = 0,
    RT_EINVAL = -1,    /* invalid argument or input value */
    RT_ENOMEM = -2,    /* device or host allocation failed */
    RT_ECUDA = -3,     /* a CUDA runtime call failed */
    RT_EDEVICE = -4,   /* a kernel reported an internal error (e.g. buffer overflow) */
    RT_ETIMEOUT = -5,  /* a bounded device wait gave up */
    RT_ESTATE = -6,    /* call not valid in the handle's state (missing fields, sticky error) */
    RT_EPENDING = -7   /* a served request has not finished yet */
};
enum { RT_FP64 = 0, RT_FP32 = 1 };
enum { RT_HOST = 0, RT_DEVICE = 1 };
enum {
    RT_OVERLAP_NONE = 0,          /* deposit the whole segment rate in the current cell */
    RT_OVERLAP_LINEAR = 1,        /* Eq. 5 only (f_c < 1 near faces; photons lost) */
    RT_OVERLAP_ARC = 2,           /* Eqs. 5-6: secondary deposit into the nearest neighbour */
    RT_OVERLAP_CONSERVATIVE = 3,  /* Eqs. 7-8: secondary only if n'_H >= n_th (default) */
    RT_OVERLAP_SQUARED = 4,       /* f_c = (1/2 + D_edge/L_pix)^2 (Sec. 2.6.1 alternative) */
    RT_OVERLAP_NAIVE = 5          /* Eq. 5 always, Eq. 6 deposit only if n'_H >= n_th: the naive
                                     threshold of Sec. 2.6 (loses photons; for comparison) */
};
enum { RT_MERGE_OFF = 0, RT_MERGE_FORCED = 1, RT_MERGE_AUTO = 2 };

/* Step configuration. Fill with rt_config_default() and override. */
typedef struct rt_config {
    int32_t n;                 /* grid cells per side, 1..1024 */
    int32_t precision;         /* RT_FP64: FP64 march physics; RT_FP32: FP32 march physics with
                                  Kahan-compensated photon and optical-depth budgets. Deposits and
                                  the photon ledger are FP64 in both. */
    double box_cm;             /* box side length, cm */
    double sigma_cm2;          /* gray HI cross-section, cm^2 (Eq. 2) */
    double n_min_ray;          /* N_min^ray >= 1, minimum rays per cell (Eq. 4) */
    int32_t level_max;         /* maximum HEALPix level (RAY_FLTR, Alg. 1); -1: smallest l with
                                  R_l >= sqrt(3) n plus one, which never binds */
    int32_t overlap_mode;      /* RT_OVERLAP_* */
    double tau_max;            /* optical depth at which a ray's remaining photons are dropped */
    double n_th_cm3;           /* Eq. 7-8 threshold on the neighbour's n_H; < 0: 0.01 x mean(n_H) */
    double e_heat_erg;         /* heating per photoionization: heat = e_heat * Gamma * n_HI */
    int32_t merge_mode;        /* RT_MERGE_*: Alg. 3 source merging off / every step / once mean x
                                  exceeds automerge_xbar (Sec. 2.8) */
    int32_t merge_samp_level;  /* HEALPix level of the shell samples (12 * 4^level samples) */
    double automerge_xbar;     /* automerge threshold on the mean ionized fraction */
    double merge_x_th;         /* a sample counts as ionized if x >= merge_x_th */
    double merge_f_req;        /* a shell passes if N_ion / N_tot >= merge_f_req */
    double merge_dr_cells;     /* shell radius increment, cells */
    double merge_rmax_cells;   /* hard cap on the bubble radius, cells */
    double merge_f_ov;         /* overlap factor f_ov */
    double merge_eps;          /* tolerance epsilon in d^2 <= (f_ov (r_a + r_b))^2 + epsilon */
    int32_t merge_n_min;       /* below this many samples every sample must be ionized */
    int32_t chem_iterate;      /* 1: iterate trace <-> C2-Ray update to convergence (Sec. 2.4) */
    double alpha_B;            /* case-B recombination coefficient, cm^3/s */
    double C_H;                /* collisional ionization coefficient, cm^3/s */
    double clumping;           /* clumping factor C */
    double chem_tol;           /* convergence: max |<x>_new - <x>_old| < chem_tol */
    int32_t chem_max_iter;     /* iteration cap */
    int32_t flags;             /* RT_FLAG_* bits */
    int32_t periodic;          /* 1: periodic boundaries (Sec. 2.5.1): rays wrap around the box and
                                  stop once they have travelled sqrt(3) box lengths (without
                                  splitting; their remaining photons count as escaped) */
    int32_t spectrum;          /* RT_SPECTRUM_*: gray sigma_cm2, or Eq. 1 integrated over a
                                  blackbody spectrum (Sec. 2.5) */
    double t_bb_K;             /* blackbody temperature for RT_SPECTRUM_BLACKBODY */
} rt_config;

enum {
    RT_SPECTRUM_GRAY = 0,      /* one cross-section sigma_cm2 for all photons (default) */
    RT_SPECTRUM_BLACKBODY = 1  /* Eq. 1 over frequency: blackbody photons above the threshold,
                                  sigma_nu = sigma_cm2 (nu_0 / nu)^3. A ray keeps its geometric
                                  budget and carries threshold optical depth tau; it absorbs
                                  Phi(tau) - Phi(tau + dtau) of it per segment, Phi(tau) being the
                                  fraction of its photons that survive tau (cubic pieces in tau
                                  per temperature, 32 per octave below tau = 1 and 128 above, indexed
                                  by the bits of tau). tau_max <= 1e4.
                                  rt_step, the batched form (its heavy path) and the server; not
                                  the allocation-free form. */
};

#define RT_FLAG_VISIT_HASH 1   /* accumulate the visit-list hash in rt_stats (bookkeeping check) */
#define RT_FLAG_NO_GEOMETRY_TABLE 2  /* walk every ray's cells instead of reading them from the
                                        per-device geometry tables (same results; for comparison) */

/* Step statistics, filled by rt_step (host memory, valid on return). */
typedef struct rt_stats {
    int64_t n_src_in;          /* sources added */
    int64_t n_src_dedup;       /* after merging sources that share a cell */
    int64_t n_src_emit;        /* after Alg. 3 merging (= n_src_dedup when merging is off) */
    int32_t merged;            /* 1 if Alg. 3 merging ran this step */
    int32_t chem_iters;        /* traces performed (1 without chemistry) */
    int32_t level_max;         /* level cap in effect */
    int32_t launches;          /* kernel launches of the last trace */
    /* per HEALPix level, for the last trace: */
    int64_t rays[RT_MAX_LEVELS];           /* rays marched */
    int64_t splits[RT_MAX_LEVELS];         /* rays that reached R_l and split into 4 */
    int64_t escaped[RT_MAX_LEVELS];        /* rays that left the grid */
    int64_t dropped_tau[RT_MAX_LEVELS];    /* rays stopped at tau >= tau_max */
    int64_t dropped_level[RT_MAX_LEVELS];  /* rays stopped at level_max */
    int64_t segments[RT_MAX_LEVELS];       /* ray-cell segments (primary deposits) */
    int64_t secondary[RT_MAX_LEVELS];      /* secondary (neighbour) deposits, Eqs. 6/8 */
    uint64_t visit_hash;       /* sum over segments of a hash of (ray id, segment index, cell);
                                  0 unless RT_FLAG_VISIT_HASH */
    double emitted_ph;         /* photons/s emitted */
    double absorbed_ph;        /* photons/s absorbed along rays */
    double escaped_ph;         /* photons/s leaving the grid */
    double dropped_ph;         /* photons/s dropped at tau_max or level_max */
    double deposited_ph;       /* sum over cells of Gamma n_HI dx^3 */
    double chem_residual;      /* last max |<x>_new - <x>_old| */
    double ms_trace;           /* device time of the last trace, first to last march launch */
    double ms_step;            /* device time of the whole step */
    double ms_march;           /* sum of the march kernels' own durations in the last trace
                                  (CUDA events around each launch, on the handle's stream) */
    int64_t march_launches;    /* march kernel launches in the last trace */
    int64_t table_levels;      /* bit l set: level l's march read its cells from the per-device
                                  geometry tables in the last trace; clear: it walked its rays
                                  (or did not run) */
} rt_stats;

typedef struct rt_handle rt_handle;

/* Fill `cfg` with the library defaults for an n^3 grid of side box_cm:
 * FP64, sigma = 6.3e-18, N_min = 4, level_max = -1, conservative overlap,
 * tau_max = 30, n_th = -1, e_heat = 1 eV, merging off (Alg. 3 parameters
 * x_th = 0.9, f_req = 0.9, dr = 2, R_max = 16, f_ov = 1, eps = 1e-6,
 * N_min = 8, samples at level 3), chemistry off (alpha_B = 2.59e-13,
 * C_H = 0, C = 1, tol = 1e-6, 100 iterations). */
void rt_config_default(rt_config* cfg, int32_t n, double box_cm);

/* Create a solver for one grid (Sec. 2.5 ray-tracing state). `cuda_stream`
 * is a cudaStream_t (NULL = legacy default stream) on the current device.
 * Allocates the field and ray buffers on that device. */
int rt_create(const rt_config* cfg, void* cuda_stream, rt_handle** out);

/* Copy the hydrogen density n_H (cm^-3, >= 0, finite) and the ionized
 * fraction x in [0, 1] (n^3 float64 each) into the handle. The absorber
 * density is n_HI = (1 - x) n_H (Sec. 2.6). Device pointers must stay valid
 * until the stream reaches this call's copies. Values are validated on the
 * device during rt_step (RT_EINVAL). */
int rt_set_fields(rt_handle* h, const double* n_H, const double* x_ion, int where);

/* Append n point sources: cell_ijk is n x 3 int32 (ix, iy, iz) integer
 * cell coordinates (the ray origin is the cell centre), ndot is n float64
 * photon rates in photons/s (> 0). Copied; validated here for host input
 * and during rt_step for device input. */
int rt_add_sources(rt_handle* h, const int32_t* cell_ijk, const double* ndot, int64_t n, int where);

/* Remove all sources. */
int rt_clear_sources(rt_handle* h);

/* Re-target a handle to another configuration with the same n, precision
 * and chem_iterate setting (box size, threshold, ray and merge parameters
 * may all change), keeping its device allocations so that a long-lived
 * caller that serves many grids of one size allocates nothing per grid.
 * Sources are cleared and the fields must be set again before rt_step.
 * Returns RT_EINVAL, leaving the handle as it was, for an invalid
 * configuration or a different n, precision or chemistry setting. */
int rt_reconfigure(rt_handle* h, const rt_config* cfg);

/* One radiative-transfer step (Alg. 2 with the Sec. 2.8 source handling):
 * dedup/sort (and merge) sources, trace all rays, write Gamma (s^-1 per H
 * atom, Eq. 1) and heating (erg s^-1 cm^-3) into caller buffers of n^3
 * float64 (either may be NULL). With chem_iterate the trace and the
 * C2-Ray update of Eq. 3 are iterated over a step of dt_s seconds and the
 * handle's x becomes x(t + dt) (read it with rt_get_x). `st` may be NULL.
 * Synchronises the stream before returning. */
int rt_step(rt_handle* h, double dt_s, double* gamma_out, double* heat_out, int where, rt_stats* st);

/* Copy the handle's current ionized fraction (n^3 float64) out. */
int rt_get_x(rt_handle* h, double* x_out, int where);

/* The source catalog that the handle's last step (rt_step or a batched run)
 * traced, i.e. the sources whose 12 level-0 rays were emitted (Sec. 2.8):
 * deduplicated by cell, sorted by (ix, iy, iz) and, where that step merged,
 * replaced by the Alg. 3 groups (a group sits at its snapped centroid and
 * carries the sum of its members' rates, added in catalog order). Writes
 * min(catalog size, capacity) entries: cells_out as int32 (ix, iy, iz) triples,
 * ndot_out as float64 photons/s, both host or device memory per `where`;
 * *count receives the catalog size. With capacity 0 the two pointers may be
 * NULL (a size query). RT_ESTATE if sources were added or cleared (or the
 * handle reconfigured) since the last step, or none has run. */
int rt_get_sources(rt_handle* h, int32_t* cells_out, double* ndot_out, int64_t capacity, int64_t* count,
                   int where);

/* Checkpoint, to resume a run later or elsewhere: write the handle's configuration, its fields
 * (n_H and the current ionized fraction x, which rt_step advances under chem_iterate) and the
 * sources added since the last rt_clear_sources to the file `path` (binary, read back by rt_load).
 * A handle loaded from it steps as this one would: the same bookkeeping bit for bit, and fields
 * that agree to the order of the FP64 deposit atomics (about 1e-14 relative); under chem_iterate
 * the iteration count may differ by one where the convergence test sits at its tolerance.
 * RT_ESTATE before rt_set_fields; RT_ENOMEM if the host buffers cannot be allocated; RT_EINVAL if
 * the file cannot be written. Synchronises the handle's stream. */
int rt_save(rt_handle* h, const char* path);

/* Create a handle on `cuda_stream` (as rt_create) from a file rt_save wrote, holding its
 * configuration, fields and sources. RT_EINVAL if the file is missing, truncated or longer than
 * its header's counts say, of another format version or holds an invalid configuration
 * (rt_last_error(NULL) says which): the counts are checked against the file's size before any
 * buffer is sized from them. RT_ENOMEM if the host buffers cannot be allocated; otherwise the
 * codes of rt_create, rt_set_fields and rt_add_sources. */
int rt_load(const char* path, void* cuda_stream, rt_handle** out);

/* Free the handle and its device memory. NULL is accepted. */
int rt_destroy(rt_handle* h);

/* Device memory held by the geometry tables of CUDA device `device`, in
 * bytes. A ray's cells, segment lengths and overlap-correction geometry
 * relative to its source depend only on its HEALPix level and pixel (every
 * source sits at a cell centre: Sec. 2.5 with the source convention of
 * Alg. 3), so the march reads them from tables built on first use for each
 * (split radius, level, grid size) and kept until the process exits: row
 * offsets shared by both precisions, 8-byte entries for the FP32 march and
 * 16-byte ones for the FP64 march (each built when that precision first
 * needs the level), within a budget of a quarter of the device's memory
 * (environment variable NYXRT_GEOMETRY_BUDGET_MB overrides it); levels over
 * budget walk their rays. The batched form reads them in both precisions. */
int64_t rt_geometry_table_bytes(int32_t device);

/* Phi(tau) and the thin rate Psi(tau) = -dPhi/dtau of RT_SPECTRUM_BLACKBODY at
 * t_bb_K, from the library's own cubic pieces (the functions the FP64 march runs,
 * evaluated on the host; the FP32 march reads the same pieces rounded to float; for
 * checking). Returns RT_EINVAL for tau outside [0, 1e4] or t_bb_K <= 0, and
 * RT_ENOMEM if host memory for the pieces ran out. */
int rt_spectrum_eval(double t_bb_K, double tau, double* phi, double* psi);

/* The fraction Phi(tau) - Phi(tau + dtau) of a ray's photons that a segment of
 * threshold optical depth dtau > 0 absorbs after tau, computed on the host by the
 * same function the FP64 march runs on the device (the mean slope of the cubic
 * piece within a piece, split at a node, node values across several pieces;
 * Eq. 1 over a blackbody spectrum, Sec. 2.5). *frac receives it. Returns
 * RT_EINVAL for tau outside [0, 1e4], dtau not in (0, 1e4], t_bb_K <= 0 or a
 * null pointer, and RT_ENOMEM if host memory for the pieces ran out. For
 * checking. */
int rt_spectrum_absorb(double t_bb_K, double tau, double dtau, double* frac);

/* Text of the handle's last error ("" if none); for h == NULL, the last
 * error of a failed rt_create on this thread. */
const char* rt_last_error(const rt_handle* h);

/* Library version string. */
const char* rt_version(void);

/* ---------------------------------------------------------------------------
 * Batched form: many independent solves traced together.
 *
 * A batch groups handles (each with its own grid size, fields, sources and
 * configuration; all with the same precision, on one device, chemistry off)
 * and traces all their rays in one run of the ray-tracing loop of Alg. 2.
 * Light solves share cooperative, persistent launches whose warps claim tiles
 * of work from a device queue, level by level and slice by slice, over all
 * their solves at once: this fills the GPU when single solves are small and
 * removes the per-level host round trips of rt_step (a launch holds solves of
 * one rate: gray, or the blackbody at one temperature). Heavy solves (see
 * heavy_shift) are cut into chunks of
 * sources, each traced by one march launch per level sized on the device from
 * the parents the previous level counted, on parallel streams whose launches
 * overlap. Results equal those of rt_step on each handle (bookkeeping bit for
 * bit; fields to the order of the FP64 atomic deposits, and for FP64 walked
 * solves to the FP64 bar of 1e-12 against the table march's double-float
 * arithmetic).
 */
typedef struct rt_batch rt_batch;

/* Launch shape of the batch kernel (see rt_batch_tune). */
typedef struct rt_batch_params {
    int32_t block;          /* threads per block: 128 or 256 */
    int32_t blocks_per_sm;  /* co-resident blocks per SM, 1 .. the occupancy limit; 0: as many as fit
                               (a batch whose solves share N_min reads the geometry tables of its
                               precision, with a limit of its own) */
    int32_t tile;           /* children a warp claims from the work queue at once (multiple of 32) */
    int32_t heavy_shift;    /* a solve that traced 2^heavy_shift segments or more in its last run
                               takes the heavy path (before any run every gray solve is light);
                               0: 26; -1: every solve; at most 62 */
    int64_t slice;          /* children per slice; also the record capacity of each level's buffer */
    int64_t group_bytes;    /* solves run in consecutive groups whose kappa + Gamma bytes stay within
                               this budget (one launch per group, keeping each group's fields in
                               L2); 0: all solves in one launch */
} rt_batch_params;

/* Create a batch over `count` handles (fields set, sources added). Runs each
 * handle's source stage now (dedup, sort, Alg. 3 merging, the n_th default):
 * later rt_add_sources calls do not affect the batch, later rt_set_fields
 * calls do (kappa is rebuilt on every run). `cuda_stream` is unused (the
 * batch runs on a private stream and waits for the handles' streams). The
 * handles must outlive the batch. */
int rt_batch_create(rt_handle* const* handles, int32_t count, void* cuda_stream, rt_batch** out);

/* Set / read the launch shape. Changing `slice` reallocates the ray buffers. */
int rt_batch_set_params(rt_batch* b, const rt_batch_params* p);
int rt_batch_get_params(const rt_batch* b, rt_batch_params* p);

/* Autotuner: time the batch under candidate launch shapes (block 128/256,
 * 1, 2 and as many blocks per SM as fit, tiles 64/256/1024, slices 2^21/2^23/2^25, group
 * budgets of 48 MB and unlimited), each `repeats` times, keep the fastest and
 * return it with its time in ms. */
int rt_batch_tune(rt_batch* b, int32_t repeats, rt_batch_params* best, double* best_ms);

/* Capture one run (kappa rebuild, trace, finalize, statistics copy) into a
 * CUDA graph; rt_batch_run then replays it. Solves are sorted into the light
 * and heavy paths by their work in the previous run (heavy_shift), so
 * capturing after one run captures that split; before any run, every solve is
 * light (unless heavy_shift is -1). */
int rt_batch_capture(rt_batch* b);

/* Run the batch: write solve i's Gamma and heating into gamma_out[i] and
 * heat_out[i] (n_i^3 float64, host or device by `where`; arrays or entries may
 * be NULL) and its statistics into stats[i] (host array of `count`, may be
 * NULL; timings are the whole batch's). Synchronous. */
int rt_batch_run(rt_batch* b, double* const* gamma_out, double* const* heat_out, int where, rt_stats* stats);

/* Free the batch (not its handles). NULL is accepted. */
int rt_batch_destroy(rt_batch* b);

/* Text of the batch's last error. */
const char* rt_batch_last_error(const rt_batch* b);

/* ---------------------------------------------------------------------------
 * Serving: a request loop with admission by device memory and continuous
 * batching. Requests (one solve each: configuration, fields, sources) are
 * submitted as they arrive. A loader thread admits them in arrival order while
 * their device bytes fit the budget and loads them (handle, fields, sources,
 * source stage) while the GPU traces the previous batch; a worker thread forms
 * a batch from every loaded request (up to max_batch) and traces it in one
 * persistent launch (the batched form above), so requests that arrive while
 * a batch runs join the next one. Results go to the caller's host buffers and
 * the request's device memory is released.
 */
typedef struct rt_server rt_server;

typedef struct rt_server_config {
    int32_t precision;      /* RT_FP32 or RT_FP64; every request must match */
    int32_t max_batch;      /* requests per batch launch */
    int64_t hbm_budget;     /* device bytes admitted requests may hold; 0: free memory at creation
                               minus the batch workspace and a 4 GB margin */
    int64_t slice;          /* batch kernel slice (rt_batch_params.slice) */
    int64_t group_bytes;    /* batch group budget (rt_batch_params.group_bytes) */
    int32_t loaders;        /* loader threads (admission + host-to-device copies + source stage) */
    int32_t max_n;          /* largest grid expected: its HEALPix directions are built at creation */
} rt_server_config;

typedef struct rt_server_stats {
    int64_t submitted, completed, failed, batches;
    int64_t queued;         /* submitted, not yet traced */
    int64_t mem_budget, mem_in_use, mem_peak;   /* admitted-request device bytes */
    int64_t segments;       /* ray-cell segments of completed requests */
    double busy_ms;         /* GPU time of all batches */
    double elapsed_ms;      /* since rt_server_create */
    double p50_ms, p99_ms, mean_ms, max_ms;     /* latency submit -> done, completed requests */
    double load_ms, bind_ms, run_ms, finish_ms; /* host time summed per phase: loading requests,
                                                   forming batches, running them, returning results */
    double src_ms;          /* host time of the batched source stage (part of bind_ms) */
    double wait_admit_ms, wait_batch_ms, wait_finish_ms;  /* summed over requests: submit -> admitted,
                                                   loaded -> taken into a batch, traced -> result copy */
} rt_server_stats;

/* Defaults: FP32, max_batch 64, hbm_budget 0, slice 2^23, group 48 MB, 4 loaders, max_n 256.
 * The server sets the device's default stream-ordered memory pool to keep up
 * to the budget cached between requests (process-local; the pool is shared
 * with other cudaMallocAsync users of the process). */
void rt_server_config_default(rt_server_config* cfg);

/* Start a server on the current device (loader, worker and finisher threads).
 * Solver handles are pooled by grid size and reused across requests; idle
 * ones count against the budget and are released, least recently used
 * first, when a request of another size needs the room. With the
 * environment variable NYXRT_SERVER_TRACE=<file>, every request's phase
 * times are appended to that file when the server is destroyed. */
int rt_server_create(const rt_server_config* cfg, rt_server** out);

/* Submit one solve: `cfg` as for rt_create (chem_iterate 0, the server's
 * precision); n_H and x_ion (n^3), cell_ijk (nsrc x 3) and ndot (nsrc) are
 * HOST arrays that must stay valid until the request finishes; gamma_out and
 * heat_out (n^3 float64 host buffers, either may be NULL) receive the result.
 * Returns RT_ENOMEM at once if the request alone exceeds the budget. */
int rt_server_submit(rt_server* s, const rt_config* cfg, const double* n_H, const double* x_ion,
                     const int32_t* cell_ijk, const double* ndot, int64_t nsrc, double* gamma_out,
                     double* heat_out, int64_t* id_out);

/* Wait up to wait_s seconds for request `id`. On completion returns its status
 * (RT_OK or the error), fills `st` and `latency_ms` (either may be NULL) and
 * forgets the request; returns RT_EPENDING if it has not finished. */
int rt_server_poll(rt_server* s, int64_t id, double wait_s, rt_stats* st, double* latency_ms);

/* Counters and latency percentiles so far. */
int rt_server_stats_get(rt_server* s, rt_server_stats* out);

/* Stop the threads and free everything (unfinished requests are dropped). */
int rt_server_destroy(rt_server* s);

/* Text of the server's last error. */
const char* rt_server_last_error(const rt_server* s);

/* rt_step without any memory allocation, for small grids. There is no
 * counterpart in the paper: it exists for callers that may not allocate
 * device memory when they need a step (code running inside a memory-capped
 * or externally managed pool, real-time loops that must stay out of the CUDA
 * allocator, hosts that budget every allocation up front). It computes the
 * same step as rt_create + rt_set_fields + rt_add_sources + rt_step + rt_destroy
 * with the same configuration, but every scratch buffer it needs lives in one
 * fixed array of about 8.5 MB inside the library, which each GPU that loads
 * the library keeps until the process exits; it calls no allocator.
 *
 * Limits (violations return RT_EINVAL with a message): n <= 32, at most 4096
 * sources, merge_mode == RT_MERGE_OFF, chem_iterate == 0, spectrum ==
 * RT_SPECTRUM_GRAY, and rays may not need HEALPix levels above 7 (true for
 * n <= 32 with n_min_ray <= 4).
 *
 * Arguments: `cfg` as for rt_create; `cuda_stream` a cudaStream_t on the
 * current device; n_H and x_ion (n^3 float64), cell_ijk (nsrc x 3 int32) and
 * ndot (nsrc float64) are DEVICE pointers owned by the caller; gamma_out and
 * heat_out (n^3 float64, heat_out may be NULL) are DEVICE pointers the step
 * overwrites; `st` (host, may be NULL) receives the counters and ledger
 * (timings are 0); `err` (host, may be NULL) receives up to err_len - 1
 * characters of error text. Synchronises the stream before returning.
 *
 * The first call on each device sets the array up (looks up its device
 * address and copies the direction table into it synchronously): make that
 * first call before any stream capture. All calls share the array and each
 * overwrites what the last one left; calls that overlap on the GPU race and
 * must be serialised by the caller. */
int rt_step_noalloc(const rt_config* cfg, void* cuda_stream, const double* n_H, const double* x_ion,
                    const int32_t* cell_ijk, const double* ndot, int64_t nsrc, double* gamma_out,
                    double* heat_out, rt_stats* st, char* err, int32_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* NYXRT_H */
