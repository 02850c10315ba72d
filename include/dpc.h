/*
 * libdpc: exact Density-Peaks Clustering on one NVIDIA GB300 (sm_103a).
 *
 * The problem is the one defined in Amagata & Hara, "Fast Density-Peaks
 * Clustering: Multicore-based Parallelization Approach" (arXiv 2207.04649),
 * Section 2.1. For a set P of n points, a cutoff d_cut and thresholds
 * rho_min, delta_min:
 *   - local density      rho_i   = #{ p_j in P : dist(p_i, p_j) < d_cut }
 *                        (Definition 1; p_i counts itself; strict <),
 *   - dependent point    q_i     = nearest point of higher density
 *                        (Definition 2),
 *   - dependent distance delta_i = dist(p_i, q_i); infinity for the
 *                        densest point (Definition 3),
 *   - noise              rho_i < rho_min (Definition 4),
 *   - cluster center     not noise and delta_i >= delta_min, with
 *                        delta_min > d_cut (Definition 5),
 *   - cluster label      the center reached through dependent points
 *                        (Definition 6).
 *
 * Conventions fixed by this library where the paper leaves a choice:
 *   - dist is Euclidean over int32 coordinates and is compared squared, in
 *     exact integer arithmetic. delta is reported squared (delta2, int64).
 *   - "Higher density" is the total order (rho desc, original index asc):
 *     the order Ex-DPC (Section 3) processes points in when its density sort
 *     is stable. It replaces the paper's random tie-breaker.
 *   - Ties in distance go to the smaller original index (Definition 2 says
 *     ties are broken arbitrarily).
 *   - The densest point has dep = -1 and delta2 = INT64_MAX.
 *   - label_i is the original index of point i's center; -1 for noise.
 *   - Every output is in the caller's original point order. The results are
 *     deterministic and bit-exact: they do not depend on the GPU's schedule.
 *
 * Errors are returned as dpc_status, never thrown; dpc_last_error() gives a
 * message for the calling thread's last failure. Calls that take a context
 * run on that context's CUDA stream; calls writing to host memory return
 * once the data is there.
 */
#ifndef DPC_H
#define DPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DPC_OK = 0,
    DPC_PENDING = 1,            /* dpc_poll: the job is not finished */
    DPC_ERR_INVALID_ARG = -1,   /* a pointer, size or parameter is out of range */
    DPC_ERR_OOM = -2,           /* device memory could not be allocated */
    DPC_ERR_CUDA = -3,          /* a CUDA call failed (message in dpc_last_error) */
    DPC_ERR_TIMEOUT = -4,       /* a bounded wait ran out */
    DPC_ERR_STATE = -5,         /* handle used in the wrong state (released, unknown ticket) */
    DPC_ERR_CAPACITY = -6       /* the job can never fit the context's memory cap */
} dpc_status;

typedef struct dpc_ctx dpc_ctx;   /* device, stream, memory pool, job queue */
typedef struct dpc_ds dpc_ds;     /* one clustered dataset kept on the device */

typedef struct {
    int device;              /* CUDA device ordinal */
    void* cuda_stream;       /* cudaStream_t to run on; NULL: the context creates its own */
    uint64_t hbm_cap_bytes;  /* device memory the served mode may hold at once; 0: 150 GB */
    const char* tune_cache;  /* autotuner cache file (text, see dpc_autotune) or NULL */
    int debug_checks;        /* nonzero: synchronize and check after every stage */
    int mode;                /* 0: batched (dpc_flush runs the submitted jobs);
                                1: served (a worker thread admits jobs continuously) */
    int max_inflight;        /* served mode: batches on the device at once; 0: 4 */
} dpc_options;

/* Create a context on options->device (options may be NULL: device 0, own
 * stream, batched mode). *out receives the handle. */
dpc_status dpc_create(const dpc_options* options, dpc_ctx** out);

/* Destroy a context: waits for its jobs, frees its device memory. Datasets
 * created from it must be released first. */
dpc_status dpc_destroy(dpc_ctx* ctx);

/* Message describing the calling thread's last error ("" if none). */
const char* dpc_last_error(void);

/* Local density of every point (Definition 1).
 *   points:  n x d int32, row-major, 0 <= x < 2^30. Host memory when
 *            is_device == 0, device memory of the context's device otherwise.
 *            Read during the call; the caller keeps ownership.
 *   n:       0 <= n < 2^31 (n == 0 gives an empty dataset).
 *   d:       1 <= d <= 8.
 *   d_cut:   1 <= d_cut < 2^31.
 *   out:     receives the dataset handle; it owns the device-resident sorted
 *            points, rho, rank and (after dpc_dependent) dep/delta2 until
 *            dpc_release.
 *   rho_out: NULL or n int32 (host or device per is_device).
 * Errors: DPC_ERR_INVALID_ARG for any argument out of range (coordinates are
 * checked on the device), DPC_ERR_OOM, DPC_ERR_CUDA. */
dpc_status dpc_density(dpc_ctx* ctx, const int32_t* points, int64_t n, int32_t d, int64_t d_cut,
                       int is_device, dpc_ds** out, int32_t* rho_out);

/* Dependent point and squared dependent distance (Definitions 2-3).
 *   dep_out:    NULL or n int32: original index of the dependent point, -1
 *               for the densest point.
 *   delta2_out: NULL or n int64: squared distance to it, INT64_MAX for the
 *               densest point.
 * Both host or device memory, as for dpc_density's is_device. Computed once
 * per dataset; later calls copy the kept result. */
dpc_status dpc_dependent(dpc_ds* ds, int32_t* dep_out, int64_t* delta2_out);

/* Approx-DPC's dependent points (Section 4.3) instead of the exact ones.
 * The grid G of Section 4.1 has cells of side d_cut / sqrt(d), here the
 * integer side max(1, floor(d_cut / sqrt(d))) anchored at the per-dimension
 * minimum; p*(c) is a cell's highest point in the order (rho desc, index
 * asc). A point other than its cell's p* depends on p*(c) at distance d_cut;
 * a p* depends, at distance d_cut, on the highest p*(c') among the cells c'
 * that hold a point strictly within d_cut of it and all of whose points rank
 * higher; every other point gets its exact dependent point (Definitions
 * 2-3). With delta_min > d_cut the centers are those of dpc_dependent
 * (Section 4.4).
 *   dep_out, delta2_out: as for dpc_dependent (delta2 = d_cut^2 for an
 *               approximated point).
 *   exact_out:  NULL or n uint8: 1 where the dependent point is exact.
 * Host or device memory, as for dpc_density's is_device. Later dpc_label
 * calls use these dependent points until dpc_dependent is called. */
dpc_status dpc_dependent_approx(dpc_ds* ds, int32_t* dep_out, int64_t* delta2_out, uint8_t* exact_out);

/* S-Approx-DPC (Section 5): local densities and dependent points of one
 * picked point per cell of a finer grid G', instead of every point's.
 * G' has cells of side eps * d_cut / sqrt(d), here the integer side
 * max(1, floor(eps * d_cut / sqrt(d))) with eps = eps_num / eps_den,
 * anchored at the per-dimension minimum. A cell's pick is its point with the
 * smallest original index. Picks get their exact local density (Definition
 * 1) and are ordered by (rho desc, index asc). A pick's dependent point is
 * the nearest higher pick among the picks of the cells (other than its own)
 * that hold a point strictly within d_cut of it (first phase); without one,
 * its nearest higher pick over all picks (second phase); the densest pick
 * has none (-1, INT64_MAX). Ties in distance go to the smaller index. Every
 * other point depends on its cell's pick, at its exact squared distance.
 * dpc_label on the returned dataset labels the picks by Definitions 4-6 and
 * gives every other point its pick's label; dpc_dependent copies the
 * dependent points above; dpc_dependent_approx returns DPC_ERR_STATE.
 *   points, n, d, d_cut, is_device, out: as for dpc_density.
 *   eps_num, eps_den: 1 .. 2^20 each.
 *   rho_out:    NULL or n int32: rho of the picks, -1 elsewhere.
 *   dep_out, delta2_out: NULL or n int32 / int64, as for dpc_dependent.
 *   pick_out:   NULL or n uint8: 1 for the picks.
 * Host or device memory, as for is_device.
 * Errors: those of dpc_density. */
dpc_status dpc_sapprox(dpc_ctx* ctx, const int32_t* points, int64_t n, int32_t d, int64_t d_cut, int64_t eps_num,
                       int64_t eps_den, int is_device, dpc_ds** out, int32_t* rho_out, int32_t* dep_out,
                       int64_t* delta2_out, uint8_t* pick_out);

/* Noise, centers and labels (Definitions 4-6) for one (rho_min, delta_min)
 * query. Re-queryable: only this step runs again (the decision-graph
 * workflow of Section 2.1). Uses the dependent points of the last
 * dpc_dependent or dpc_dependent_approx call; runs dpc_dependent first when
 * neither has run.
 *   delta_min: d_cut < delta_min <= 3037000499 (so delta_min^2 fits int64).
 *   label_out: NULL or n int32 (host or device per is_device): original index
 *              of the point's center, -1 for noise.
 *   n_centers: NULL or one int64 in host memory. */
dpc_status dpc_label(dpc_ds* ds, int64_t rho_min, int64_t delta_min, int32_t* label_out, int64_t* n_centers);

/* The whole path in one call (Definitions 1-6 for one (rho_min,
 * delta_min) query): dpc_density, dpc_dependent and dpc_label on a dataset
 * that is released before the call returns. The results leave the device as
 * soon as each is final, on a second stream of the context, while the later
 * stages run (rho during the dependent-point search, dep and delta2 during
 * the labels); copies into page-locked host memory overlap, others are
 * staged by the driver.
 *   points, n, d, d_cut, is_device: as for dpc_density.
 *   rho_min, delta_min: as for dpc_label.
 *   rho_out, dep_out, delta2_out, label_out: NULL or n elements each, host or
 *            device memory per is_device, as the separate calls write them.
 *   n_centers: NULL or one int64 in host memory.
 * Returns when every output is written. Errors: those of the three calls. */
dpc_status dpc_cluster(dpc_ctx* ctx, const int32_t* points, int64_t n, int32_t d, int64_t d_cut, int is_device,
                       int64_t rho_min, int64_t delta_min, int32_t* rho_out, int32_t* dep_out, int64_t* delta2_out,
                       int32_t* label_out, int64_t* n_centers);

/* Free a dataset's device state. The handle is invalid afterwards. */
dpc_status dpc_release(dpc_ds* ds);

/* Labels with no device allocation. The paper has no counterpart: this is a
 * variant of the labels step for callers that cannot allocate device memory
 * when they call, e.g. code running on a device budget reserved up front, in
 * a section that must not allocate, or under a memory pool that fails once
 * exhausted. Its scratch (the parent of every point) is a fixed array
 * compiled into the library: 2^22 points (16 MiB), held on every GPU that
 * loads the library until the process exits.
 *   rho, dep, delta2: device arrays of n points as dpc_density and
 *            dpc_dependent (or dpc_dependent_approx) produce them (dep = -1
 *            and delta2 = INT64_MAX for the densest point); read only. On
 *            these inputs the labels and the center count equal dpc_label's.
 *            S-Approx-DPC datasets are not covered (their points that are
 *            not picked take their pick's label, which this call does not
 *            model): use dpc_label for those.
 *   n:       0 <= n <= 4194304; larger n gives DPC_ERR_INVALID_ARG.
 *   rho_min, delta_min: as dpc_label; 1 <= delta_min <= 3037000499 (the
 *            caller keeps delta_min > d_cut), else DPC_ERR_INVALID_ARG.
 *   label_out: device array of n int32: the center's index, -1 for noise,
 *            -2 for a point whose chain of dependent points runs into a
 *            rejected link (below).
 *   n_centers_out: NULL or one device int64: the number of centers, or -1
 *            when a link was rejected.
 *   cuda_stream: the cudaStream_t the work is queued on (NULL: the legacy
 *            default stream). The call returns once the work is queued, so
 *            it returns DPC_OK before the links are checked: a caller that
 *            passes links it did not get from this library reads
 *            n_centers_out to learn whether they were accepted.
 * A link of a point that is neither noise nor a center is accepted when dep
 * lies in [0, n) and ranks strictly higher in (rho desc, index asc), as
 * Definitions 2-3 make it; such links always form a forest. An out-of-range
 * dep is never used to read memory.
 * The first call on a device looks up the scratch's device address for that
 * device (cudaGetSymbolAddress, with the device current); make that first
 * call before any stream capture. All calls share the scratch and it keeps
 * the last call's contents, so calls that overlap on the GPU race. It calls
 * no cudaMalloc, cudaFree or allocating library routine. */
dpc_status dpc_label_static(const int32_t* rho, const int32_t* dep, const int64_t* delta2, int64_t n,
                            int64_t rho_min, int64_t delta_min, int32_t* label_out, int64_t* n_centers_out,
                            void* cuda_stream);

/* Counters of the last run on a dataset (sizes of the work, for reporting). */
typedef struct {
    int64_t n;
    int64_t cells;            /* non-empty grid cells */
    int64_t dense_cells;      /* cells handled one warp per work item */
    int64_t work_items;       /* dense work items */
    int64_t cand_pairs;       /* (query, candidate) pairs the density filter evaluates */
    int64_t open_after_ring;  /* points left open by the ring search */
    int64_t brute_points;     /* of those, sent to the brute-force pass */
    int32_t grid_dims;        /* gridded dimensions */
    int32_t pair_bits;        /* 32 or 64: width of the pair arithmetic */
    float ms_grid, ms_rho, ms_rank, ms_ring, ms_rest, ms_label;  /* stage times when profiling is on */
    int64_t tree_visits;      /* tree nodes visited by the search for open points */
    int64_t tree_pairs;       /* point pairs it tested */
    int32_t pair_mode;        /* density pair test: 0 direct 32-bit, 1 direct 64-bit, 2 expanded 32-bit */
    int32_t grid_key_bits;    /* width of the grid's sort key (radix passes: bits / 8, rounded up) */
    int64_t dense_pairs;      /* of cand_pairs, those of dense cells (one warp per work item) */
    float ms_rho_dense;       /* of ms_rho, the dense cells' kernels (profiling on) */
    int32_t rank_key_bits;    /* width of the rank sort's key */
    int64_t picks;            /* S-Approx-DPC: cells of G' (picked points) */
    int64_t second_phase;     /* S-Approx-DPC: picks without a first-phase dependent point */
    int32_t density_path;     /* the density's path: 0 every point (exact, Approx-DPC, S-Approx-DPC's
                                 all-point path); S-Approx-DPC's pick path: 1 one warp per pick,
                                 2 one warp per grid cell, 3 the dense kernels over pick items */
    int64_t device_bytes_peak; /* the most device memory the run's batch held at once: its allocations and
                                  frees counted in the order of its stream (they are all on it) */
} dpc_info;

dpc_status dpc_ds_info(const dpc_ds* ds, dpc_info* out);

/* Enable per-stage CUDA-event timing on a context (0 off, 1 on). */
dpc_status dpc_set_profiling(dpc_ctx* ctx, int on);

/* Tuning knobs of a context (no counterpart in the paper; they change speed,
 * never results). Keys and ranges:
 *   "kch"     candidates per dense work item, 32 .. 2^20 (default 1024)
 *   "qch"     queries per dense work item, 32, 64 or 128 (default 128): a
 *             cell of m points is split into ceil(m / qch) query chunks, each
 *             its own warp's work, so smaller values put more warps on a cell
 *   "kmax"    gridded dimensions at most, 1 .. 4 (default 4)
 *   "bf_rank" points still open after the ring search whose rank is below
 *             this take the brute-force pass (default 1024)
 *   "tree_warp"  the tree search for the other open points: 1 the 32 lanes
 *             of a warp walk the tree together over 32 neighbouring open
 *             points, 0 one lane per point, 2 the first for d >= 5 and the
 *             second below (default 2: on 1M x 8 the warp form takes 22 ms
 *             against 29, on 5.8M x 3 6.0 ms against 2.5)
 *   "hd_cell_factor"  f for datasets with d >= hd_min_d: grid cells of
 *             side ceil(d_cut / f), neighbours searched f cells away (a finer
 *             grid, fewer candidate pairs, more neighbour cells), 1 .. 3
 *             (default 2)
 *   "hd_min_d"  smallest d that takes hd_cell_factor, 1 .. 9 (default 7)
 *   "sparse_cand"  a cell of at most 4 points takes one thread (the sparse
 *             kernels) only if it has at most this many candidates, else one
 *             warp per work item like the larger cells, 0 .. 2^31 (default
 *             512; high-dimensional sets have small cells facing thousands of
 *             candidates)
 *   "sapprox_path"  dpc_sapprox: 1 the all-point path (the density kernels
 *             for every point, the ring search over pick ranks, a
 *             first-phase scan for the picks it leaves), 2 the pick path
 *             (one warp per pick for the density and the first-phase scan),
 *             0 chosen by the candidate pairs (default 0)
 *   "sapprox_ratio"  with sapprox_path 0: the pick path when the points'
 *             candidate pairs exceed this many times the picks' (at most 4
 *             times when the points' pairs number 2e10 or more), 1 .. 1024
 *             (default 16)
 *   "sapprox_rho_cells"  the pick path's density: 1 one warp per grid cell
 *             over its picks (candidates staged once per cell), 0 one warp
 *             per pick, 3 the dense density kernels with each cell's picks
 *             as queries, 2 by cell when picks face fewer than 512
 *             candidates each on average, else 3 (default 2)
 *   "rho_bulk"  dense density kernels of d <= 4 in a 32-bit pair form: 1
 *             stages the candidates in shared memory by bulk copies
 *             (cp.async.bulk completed on an mbarrier, one copy per run
 *             piece), 0 by 128-bit loads through registers (default 0)
 *   "sapprox_near_threads"  the pick path's first-phase scan over the
 *             picks of a pick's neighbour blocks: 1 one thread per pick,
 *             0 one warp per pick, 2 one thread while the grid's cells hold
 *             fewer than 6 picks on average, else one warp (default 2)
 *   "max_batch_jobs"  served mode: jobs one batch admits at most, 1 .. 4096
 *   "max_batch_points" served mode: points one batch admits at most, 1 .. 2^31 - 1 (default
 *                     2^20; a larger job runs in a batch of its own, so that it does not hold
 *                     back small ones). With a backlog, a batch may take up to the waiting
 *                     points divided by the number of workers instead.
 *             (default 64; 1 runs the jobs one at a time)
 * DPC_ERR_INVALID_ARG for an unknown key or a value out of range. */
dpc_status dpc_set_tuning(dpc_ctx* ctx, const char* key, int64_t value);
dpc_status dpc_get_tuning(dpc_ctx* ctx, const char* key, int64_t* value);

/* Number of CUDA kernels this library has launched in this process so far
 * (all contexts and threads); a difference of two readings counts the
 * launches of the calls in between. */
int64_t dpc_kernel_launches(void);

/* Measurement helper (no counterpart in the paper): the throughput of the
 * density stage's pair test for d-dimensional points with operands in
 * registers on every SM of `device`, i.e. the integer-ALU ceiling that the
 * density kernel is compared against, in the form dpc_ds_info reports as
 * pair_mode: 0 the direct 32-bit form (sum of squared differences), 1 the
 * direct 64-bit form, 2 the expanded 32-bit form (d <= 4); and mode 3, the
 * dependent-point ring search's pair test in the expanded form (d <= 4: the
 * same sum, a rank compare and the least packed
 * (distance, index) key kept), the ceiling of the ring kernel. Other modes
 * give DPC_ERR_INVALID_ARG. Writes pairs per
 * second (and the kernel's time in ms when ms is not NULL). Allocates and
 * frees a few bytes of device memory; synchronizes the device. */
dpc_status dpc_probe_pair_rate(int device, int d, int mode, double* pairs_per_s, double* ms);

/* ---------------------------------------------------------------------
 * Jobs: many independent datasets, batched or served.
 *
 * A job is one dataset plus n_queries (rho_min, delta_min) queries. Its
 * points and per-point outputs are host memory, or device memory of the
 * context's device when is_device is 1; rho_min, delta_min and
 * n_centers_out are always host memory. All of them are owned by the caller
 * and must stay valid until dpc_poll reports the job finished. In batched mode (dpc_options.mode 0)
 * jobs run when dpc_flush is called, all of them in one batch: every stage
 * is one launch over all datasets. In served mode (mode 1) a worker thread
 * admits waiting jobs as device memory (hbm_cap_bytes) and batch slots
 * (max_inflight) free up and runs them while earlier batches are still on
 * the device. Results are the same bits as running each dataset alone.
 * A job's method picks the dependent points: exact (dpc_dependent),
 * Approx-DPC (dpc_dependent_approx) or S-Approx-DPC (dpc_sapprox, whose rho
 * is -1 where not picked); a batch holds jobs of one method, so dpc_flush
 * runs the queued jobs as consecutive batches of equal method and the
 * served mode starts a new batch where the method changes.
 * ------------------------------------------------------------------- */
typedef struct {
    const int32_t* points;     /* n x d int32 row-major */
    int64_t n;
    int32_t d;
    int64_t d_cut;
    int32_t n_queries;         /* >= 1 */
    const int64_t* rho_min;    /* [n_queries] */
    const int64_t* delta_min;  /* [n_queries], each > d_cut */
    int32_t* rho_out;          /* NULL or [n] */
    int32_t* dep_out;          /* NULL or [n] */
    int64_t* delta2_out;       /* NULL or [n] */
    int32_t* label_out;        /* NULL or [n_queries * n], query-major */
    int64_t* n_centers_out;    /* NULL or [n_queries] */
    int32_t is_device;         /* 0: points and outputs in host memory; 1: in device memory. In a batch of
                                  several jobs, host points and outputs in page-locked memory (pinned or
                                  registered) are read and written by the device directly, all such jobs
                                  in one pass; pageable ones take one copy per array */
    int32_t method;            /* 0 exact (Definitions 2-3), 1 Approx-DPC (Section 4.3), 2 S-Approx-DPC (Section 5) */
    int64_t eps_num, eps_den;  /* method 2: eps = eps_num / eps_den, 1 .. 2^20 each; ignored otherwise */
    uint8_t* aux_out;          /* NULL or [n]: method 1, 1 where the dependent point is exact; method 2, 1 for
                                  the picks; unused for method 0 */
    int32_t keep;              /* 1: keep the job's rho and dependent points on the device after it finishes,
                                  for decision-graph re-queries (dpc_result.dataset); 0: free them */
} dpc_job;

typedef struct {
    dpc_status status;         /* DPC_OK, DPC_PENDING or the job's error */
    double queue_ms;           /* submit -> admitted */
    double run_ms;             /* admitted -> this job's results written */
    dpc_ds* dataset;           /* a finished job submitted with keep = 1: a handle to its device state for
                                  dpc_label (new (rho_min, delta_min) queries, labels only) and dpc_ds_info;
                                  owned by the caller, freed with dpc_release. NULL otherwise. It is handed
                                  out once, by the dpc_poll or dpc_wait that reports the job finished; a call
                                  with out = NULL frees it. Until it is released, its device memory counts
                                  against the served mode's hbm_cap_bytes. */
} dpc_result;

/* Queue a job; thread-safe. *ticket identifies it for dpc_poll. */
dpc_status dpc_submit(dpc_ctx* ctx, const dpc_job* job, uint64_t* ticket);

/* Non-blocking: DPC_PENDING until the job is done, then its final status
 * (also in out->status). A finished ticket is forgotten after it is polled.
 * A job is done as soon as its own outputs are written: in a batch, a job
 * with fewer queries can finish before the others. */
dpc_status dpc_poll(dpc_ctx* ctx, uint64_t ticket, dpc_result* out);

/* Device bytes the served mode reserves for a job of n points in d dims
 * (1 .. 8) run with `method` (0 exact, 1 Approx-DPC, 2 S-Approx-DPC) under
 * ctx's tuning knobs (NULL: the defaults): the admission estimate by which
 * the jobs in flight share hbm_cap_bytes. It bounds the run's peak,
 * dpc_info.device_bytes_peak, with one run slot per neighbour cell of the
 * grid for every point. No counterpart in the paper. */
uint64_t dpc_job_footprint(dpc_ctx* ctx, int64_t n, int32_t d, int32_t method);

/* Batched mode: run every job submitted so far as one batch and wait for it. */
dpc_status dpc_flush(dpc_ctx* ctx);

/* Counters and stage times (stage times need dpc_set_profiling) of the most
 * recent batch of jobs that finished on this context: n is the batch's total
 * number of points, cells, work items, candidate pairs and open points are
 * the batch's totals, and the per-dataset fields (grid_dims, pair_bits,
 * pair_mode) are its first dataset's. No counterpart in the paper.
 * DPC_ERR_STATE before the first batch finishes. */
dpc_status dpc_last_batch_info(dpc_ctx* ctx, dpc_info* out);

/* Autotuner (no counterpart in the paper). Runs the n_jobs sample jobs as
 * one batch under candidate settings of the knobs that change speed only
 * (kch and qch, the candidates and queries per dense work item, i.e. the
 * warps per cell; bf_rank; hd_min_d with hd_cell_factor, the grid's
 * cell factor, tried for every dataset's d; kmax when some d >= 4):
 * coordinate descent from the context's current knobs, each
 * setting timed as the best of `repeats` (1 .. 100) synchronous runs, a
 * change kept only when it is at least 2% faster. The fastest setting
 * becomes the context's knobs and its entry for the sample's signature (the
 * largest d and the rounded log2 of the mean n): later batches with that
 * signature run with it. With a tune_cache path in dpc_options the entries
 * are written there (one text line per signature) and read back by
 * dpc_create. When report is not NULL it receives the chosen setting as
 * "key=value ..." text, NUL-terminated, at most report_len bytes. The jobs'
 * outputs are written by every run (same values each time). Errors: those
 * of dpc_submit's checks and of a run; DPC_ERR_STATE when the cache file
 * cannot be written. */
dpc_status dpc_autotune(dpc_ctx* ctx, const dpc_job* jobs, int32_t n_jobs, int32_t repeats, char* report,
                        size_t report_len);

/* Block until the job is done or timeout_ms passes (DPC_ERR_TIMEOUT). */
dpc_status dpc_wait(dpc_ctx* ctx, uint64_t ticket, int64_t timeout_ms, dpc_result* out);

#ifdef __cplusplus
}
#endif

#endif /* DPC_H */
