/*
 * fmm.h -- C ABI of the GB300 restarted narrow band fast marching library
 * (libfmm_gb300.so, CUDA for sm_103a).
 *
 * The library solves the Eikonal equation |grad psi| F = 1 (Eq. (1) of Yang &
 * Stern, "A highly scalable massively parallel fast marching method for the
 * Eikonal equation") on a cell-centred 3-D grid of cells dx * dy * dz (uniform
 * in each direction, Sec. 2.1) with the first-order
 * Godunov upwind scheme of Eq. (2)-(3), by the restarted narrow band method
 * of Algorithm 16: subdomains (here 8x8x8 bricks of the grid) march locally up
 * to a global bound that rises by a stride at every restart, exchange changed
 * overlap data, and a global reduction of the front minimum sets the next
 * bound and decides termination.  The restart loop runs on the GPU; by
 * default (fmm_config.schedule) one launch runs the whole solve and the bound
 * rises as soon as a restart runs out of parallel work.
 *
 * Conventions shared by every entry point
 *   - Grid arrays are nx*ny*nz elements, x fastest: idx = (k*ny + j)*nx + i,
 *     psi at cell centres of cells h * hy * hz (Sec. 2.1).  Cells outside
 *     the grid do not exist; stencils never leave it (Sec. 4.1).
 *   - Array arguments marked "device" are caller-owned memory, contiguous,
 *     16-byte aligned, of the handle's dtype (float for FMM_F32, double for
 *     FMM_F64) unless stated otherwise: device (or managed) memory of the
 *     current CUDA device, or -- for fmm_create / fmm_set_speed's speed,
 *     fmm_solve, fmm_reinit_signed_distance, fmm_resume and fmm_adjoint --
 *     host memory, page-locked or pageable.  Host arrays are copied through
 *     device buffers the handle owns (allocated on first use, freed by
 *     fmm_destroy) on cfg->stream, inputs before the solve and outputs after
 *     it, and the call returns once host outputs are written.  The library
 *     never frees caller arrays and keeps no reference after the call returns.
 *   - Work is enqueued on cfg->stream (NULL = the legacy default stream).
 *     Entry points that run a solve return after it has finished (the restart
 *     loop reads the device's termination flag), so outputs are ready when
 *     they return FMM_OK.
 *   - On any error the call returns a non-zero fmm_status, leaves the outputs
 *     unspecified and records a message for fmm_last_error().
 *   - A handle may be used by one host thread at a time.
 *
 * Output tags (uint8, when requested): 0 FAR (never reached, psi = +inf),
 * 1 BAND (tentative value beyond width_band), 2 KNOWN (accepted),
 * 3 FIX (an initial interface / source cell, KNOWN_FIX of Sec. 4.2).
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_ERR_INVALID = 1,   /* bad argument (sizes, pointers, speed < 0, NaN, inf) */
    FMM_ERR_OOM = 2,       /* device allocation failed                        */
    FMM_ERR_CUDA = 3,      /* a CUDA runtime call failed                      */
    FMM_ERR_TIMEOUT = 4,   /* a round, restart, device-wait (wait_limit_ms) or
                              wall-clock (timeout_s) limit was reached         */
    FMM_ERR_STATE = 5      /* call order violated (e.g. adjoint before solve) */
} fmm_status;

typedef enum { FMM_F32 = 0, FMM_F64 = 1 } fmm_dtype;

typedef enum { FMM_TAG_FAR = 0, FMM_TAG_BAND = 1, FMM_TAG_KNOWN = 2, FMM_TAG_FIX = 3 } fmm_tag;

/* Solver configuration.  Zero-initialise and set nx, ny, nz, h, dtype; every
 * other field has a default when left 0. */
typedef struct {
    int64_t nx, ny, nz;    /* grid size, each >= 1                              */
    double h;              /* cell size along x (> 0); also along y and z unless
                              hy / hz are set                                  */
    int32_t dtype;         /* fmm_dtype                                         */
    int32_t record_tape;   /* 1: keep the upwind sets for fmm_adjoint           */
    double width;          /* width_band (Algorithm 5/12); 0 -> +inf (full march) */
    double stride;         /* restart stride delta_s in units of h (Algorithm 16);
                              0 -> the GB300 default (2 for FMM_F32, 1 for
                              FMM_F64; the paper suggests 2 for its CPU
                              cluster and tuning per platform, Sec. 5.5);
                              +inf allowed                                     */
    double bucket;         /* accepted bucket width inside a brick, in units of
                              h * min(1/F) / sqrt(3); 0 -> 4 (0.6 for the
                              second-order march, whose accepted values must
                              be final when their neighbours read them: see
                              accuracy); +inf allowed                        */
    int32_t ctas;          /* CTAs of the march kernel; 0 -> as many as fit     */
    int32_t timeout_s;     /* host wall-clock limit of one solve in seconds;
                              0 -> 600; exceeding it returns FMM_ERR_TIMEOUT  */
    int64_t max_restarts;  /* 0 -> no limit (timeout_s still applies)           */
    void *stream;          /* cudaStream_t                                      */
    int32_t time_kernels;  /* 1: time every march launch with CUDA events on
                              the solve's stream (fmm_stats.march_ms)         */
    int32_t exchange_passes; /* phased schedule: exchange + march passes after
                              the first march of every restart (Algorithm 16
                              has 1); 0 -> 2 for FMM_F32, 1 for FMM_F64      */
    int32_t schedule;      /* 0 -> continuous (the default; cell-parallel when
                              accuracy is 2); 1 phased: every
                              restart is a select + march launch, then
                              exchange_passes select + march launches, as in
                              Algorithm 16; 2 persistent: one launch per
                              restart marches every brick to the bound,
                              re-queuing bricks whose halo changed until none
                              is left; 3 continuous: one launch for the whole
                              solve, the bound rises by the stride whenever
                              few bricks are left below it, so one restart's
                              last bricks overlap the next one's first; 4
                              cell-parallel: no bricks or restarts, every
                              bucket step accepts the BAND cells within the
                              bucket of each side's minimum over the whole
                              grid and re-solves their neighbours (Jacobi
                              within the step, corrections as in the brick
                              march), three grid-wide launches per step; no
                              tape, no resume (max_restarts limits the
                              steps); the schedule of the second-order march
                              and, in first order, the same solution as the
                              others (one discrete solution, Sec. 5.2)      */
    int32_t max_lead;      /* continuous schedule: while bricks are queued or
                              marching, the bound stays within max_lead
                              strides of the smallest BAND value the last scan
                              saw (a small front cannot run ahead); 0 -> no
                              limit                                          */
    int32_t wait_limit_ms; /* every device-side wait (brick queue, bound
                              raise) gives up after this long without any
                              progress, sets an error bit and the call returns
                              FMM_ERR_TIMEOUT; 0 -> 4000                      */
    int32_t hold_queue;    /* testing only: 1 counts one phantom brick as
                              queued, so the persistent and continuous
                              schedules' waits run into wait_limit_ms (the
                              error path without a fault); 0 normally       */
    double hy, hz;         /* cell sizes along y and z (Sec. 2.1: cells of
                              dx * dy * dz, uniform in each direction;
                              Algorithm 11 uses h_i = 1/dx, 1/dy, 1/dz);
                              0 -> h.  The stride and the speed term are in
                              units of h, the bucket width in units of the
                              smallest cell size.  Batches need 0.          */
    double ahead;          /* continuous schedule: a brick march accepts cells
                              up to the bound plus ahead (units of h; +inf:
                              the whole brick), and a brick whose only work
                              is changed halo data waits until the bound
                              reaches the smallest changed value; 0 -> +inf.
                              The result does not depend on it.             */
    int32_t deterministic; /* 1: bit-reproducible results: the phased schedule
                              (schedule must be 0 or 1) with every brick
                              reading its neighbours' boundary values as they
                              stood at the end of the previous march pass, so
                              the result depends on no timing, CTA count or
                              launch order (the paper's synchronous exchange
                              per restart, Sec. 4.3); about twice the time of
                              the default, and one more array of 6 x 64
                              values per brick; stride 0 -> 8 for FMM_F32, 4
                              for FMM_F64 in this mode.  Single grids only (not batches, the
                              fmm_dd_* entry points or the entry point
                              without allocation).  0 normally.             */
    int32_t accuracy;      /* 0 or 1: the first-order upwind scheme of Eq.
                              (2)-(3).  2: the higher-order fast marching of
                              Sec. 6 (future work there), in the textbook
                              second-order form: on an upwind axis whose
                              next cell beyond the neighbour psi1, in the
                              same direction, is known with psi2 <= psi1,
                              the one-sided difference (3 t - 4 psi1 +
                              psi2) / (2 h) replaces (t - psi1) / h.  Needs
                              schedule 0 or 4 (runs the cell-parallel
                              schedule), record_tape 0, deterministic 0;
                              single grids only.  The second-order update is
                              not monotone in its operands (a larger psi2
                              lowers the root), so the result depends on the
                              order of acceptances and in general differs,
                              within the discretisation error, from the
                              sequential heap march's; buckets above 2/3 let
                              a value that is still being lowered serve as a
                              second neighbour and cost accuracy.  Quadratic
                              solutions are reproduced to rounding, and runs
                              are reproducible.                             */
} fmm_config;

/* Statistics of the last solve on a handle. */
typedef struct {
    int64_t restarts;        /* passes of the Algorithm 16 loop, including the
                                final one that only tests for termination
                                (schedule 4: bucket steps that accepted
                                cells; its brick counters stay 0)             */
    int64_t brick_marches;   /* local marches of a brick (both phases)           */
    int64_t march_rounds;    /* bucket rounds summed over all brick marches      */
    int64_t exchanges;       /* brick faces that sent changed overlap data       */
    int64_t accepted;        /* cell acceptances (re-acceptances counted again)  */
    int64_t n_bricks;        /* bricks of the grid                               */
    int64_t kernel_launches; /* kernels this library launched for the solve      */
    int64_t march_launches;  /* launches of the brick-march kernel               */
    double march_ms;         /* summed device time of those launches (only with
                                time_kernels; else 0)                          */
    int64_t adjoint_iterations; /* brick passes of the last fmm_adjoint          */
    int32_t error_flags;     /* device-side error bits (0 = none)                */
    int32_t reserved0;
    int64_t cell_solves;     /* Algorithm 11 evaluations in the brick marches    */
} fmm_stats;

typedef struct fmm_handle fmm_handle;

/*
 * fmm_create -- allocate a solver for one grid and load its speed field.
 *   cfg          : host pointer, copied.
 *   speed        : device, nx*ny*nz values of F (dtype), all finite and >= 0;
 *                  F = 0 marks an obstacle cell (the obstacles of test case
 *                  6, Sec. 5.1): it is never reached and stays FAR with
 *                  psi = +inf, and no front passes through it; or NULL for
 *                  the constant speed_const (> 0).
 *   src_ijk      : host, n_src (i, j, k) int64 triples: the point sources used
 *                  by fmm_solve (psi = 0, KNOWN_FIX; Algorithm 8); may be NULL
 *                  when n_src == 0.
 *   out          : receives the handle (owned by the caller; fmm_destroy).
 * The handle owns all device workspace (brick-layout psi and tags, per-brick
 * front minima and exchange masks, work lists, the restart control block and,
 * when record_tape is set, the upwind tape).
 */
fmm_status fmm_create(const fmm_config *cfg, const void *speed, double speed_const,
                      const int64_t *src_ijk, int64_t n_src, fmm_handle **out);

/*
 * fmm_solve_fixed -- solve from given interface values (Algorithm 8 with the
 * values of the interface cells supplied by the caller instead of computed
 * from a level set or point sources; then Algorithms 9-12/16 as fmm_solve).
 *   T0       : nx*ny*nz values (dtype, x-fastest, device or host, 16-byte
 *              aligned).  A finite value makes the cell KNOWN_FIX with psi =
 *              T0 on the side of its sign (v < 0: side -1; +0 and -0 are
 *              side +1); +inf / -inf marks a FAR cell of side +1 / -1.  As in
 *              Algorithm 8, both cells of every sign change between
 *              6-neighbours must be finite.
 *   T_out    : as fmm_solve.   tags_out : as fmm_solve (may be NULL).
 * Returns FMM_ERR_INVALID for a NaN in T0 or a sign change between two
 * cells that are not both finite (nothing solved), else as fmm_solve.  The
 * call synchronises the stream once after the initialisation to read that
 * check.
 */
fmm_status fmm_solve_fixed(fmm_handle *hd, const void *T0, void *T_out, uint8_t *tags_out);

/*
 * fmm_set_speed -- replace the speed field of an existing handle (same rules
 * as fmm_create's speed/speed_const); invalidates any recorded tape.
 */
fmm_status fmm_set_speed(fmm_handle *hd, const void *speed, double speed_const);

/*
 * fmm_solve -- point-source solve (Algorithm 16 with the sources of
 * fmm_create).  T_out: device, nx*ny*nz values of psi (dtype); tags_out:
 * device uint8 tags (fmm_tag) or NULL.
 */
fmm_status fmm_solve(fmm_handle *hd, void *T_out, uint8_t *tags_out);

/*
 * fmm_reinit_signed_distance -- two-sided reinitialisation (Sec. 3 and
 * Algorithm 16) of the level set phi0 (device, dtype).  Cells with a
 * 6-neighbour of the opposite sign of phi0 (sign(0) = +1) are the interface
 * cells (Algorithm 8): psi = sign(phi0) * (sum_a d_a^-2)^(-1/2) over the axes
 * whose segment to a neighbour crosses the interface, d_a the smaller
 * linear-interpolation crossing distance on axis a.  Both signs march.
 * T_out (device, dtype) receives the signed solution; tags_out as fmm_solve.
 */
fmm_status fmm_reinit_signed_distance(fmm_handle *hd, const void *phi0, void *T_out,
                                      uint8_t *tags_out);

/*
 * fmm_adjoint -- reverse-mode derivative of a scalar loss L(psi) with respect
 * to the slowness 1/F of every cell, about the last solve on this handle
 * (which must have been run with record_tape = 1 and have finished;
 * otherwise FMM_ERR_STATE).  The discrete Eq. (2) at an accepted non-FIX
 * cell p with final upwind set U(p) reads sum_{i in U(p)} ((psi_p -
 * psi_i)/h_i)^2 = s_p^2 (h_i the cell size along the axis of neighbour i),
 * which gives dpsi_p/ds_p = s_p/D_p and dpsi_p/dpsi_i = (psi_p - psi_i) /
 * (h_i^2 D_p) with D_p = sum_i (psi_p - psi_i)/h_i^2; these are applied in
 * decreasing psi.
 * FIX cells get zero.  dL_dT: device (dtype), dL/dpsi; dL_dslowness: device
 * (dtype), written.  (This derivative is not part of the paper.)
 */
fmm_status fmm_adjoint(fmm_handle *hd, const void *dL_dT, void *dL_dslowness);

/*
 * fmm_resume -- continue a solve on hd that stopped at its restart limit
 * (max_restarts) or wall-clock limit (timeout_s), or one loaded with
 * fmm_checkpoint_load.  Such a solve ends on a restart boundary of
 * Algorithm 16 (every brick marched to the last bound, no brick queued), so
 * the loop simply goes on from that state, with its restart count,
 * statistics and tape; the result is the one a single uninterrupted solve
 * reaches.  more_restarts: restarts allowed from here (0 -> no limit; the
 * wall-clock limit applies afresh).  T_out, tags_out as fmm_solve.
 * FMM_ERR_STATE when the last solve finished, failed otherwise, or was
 * followed by fmm_adjoint or fmm_set_speed (they reuse the control block);
 * FMM_ERR_TIMEOUT again when a limit stops it once more.  (Resuming is not
 * part of the paper.)
 */
fmm_status fmm_resume(fmm_handle *hd, int64_t more_restarts, void *T_out, uint8_t *tags_out);

/*
 * Checkpoints of a solve state, in host memory: the brick-layout psi, tags,
 * tape (when recorded), per-brick BAND minima, halo change masks and dirty
 * flags, and the restart control block, after an 88-byte header that records
 * the grid, dtype, cell sizes, record_tape and the kind of speed.
 *   fmm_checkpoint_size -- bytes an image of hd takes (*bytes).
 *   fmm_checkpoint_save -- write the image of the last solve on hd to
 *     host_buf (host memory of at least that size, owned by the caller;
 *     capacity its size).  The solve must have finished or stopped at a
 *     limit (fmm_resume's condition); otherwise FMM_ERR_STATE.  Synchronises
 *     hd's stream.
 *   fmm_checkpoint_load -- load an image into hd, which must have been
 *     created with the same grid, dtype, cell sizes, record_tape and kind of speed
 *     (the speed values themselves, which the image does not hold, must be
 *     the same too); else FMM_ERR_INVALID.  Afterwards hd is as the saving
 *     handle was: fmm_resume continues a stopped solve, fmm_adjoint works on
 *     a finished one with a tape.
 * Batch handles have no checkpoints (FMM_ERR_STATE).  (Not part of the
 * paper.)
 */
fmm_status fmm_checkpoint_size(fmm_handle *hd, int64_t *bytes);
fmm_status fmm_checkpoint_save(fmm_handle *hd, void *host_buf, int64_t capacity);
fmm_status fmm_checkpoint_load(fmm_handle *hd, const void *host_buf, int64_t size);

/*
 * fmm_create_batch -- a solver for n_grids independent grids of uneven sizes
 * that are solved together (fmm_reinit_batch: level sets with speed F = 1;
 * fmm_solve_batch: level sets or point sources, each grid with its own speed
 * field or constant): the bricks of all grids are packed into one brick
 * array, and with the continuous schedule (the default) the whole solve is
 * one launch that marches bricks of all grids from one shared queue
 * (persistent: one launch per restart; phased: one launch per phase over one
 * shared work list); a neighbour table stops data at the border of a grid.
 * The restart bound is common to all grids (Algorithm 16 is correct for any
 * bound): a brick of any grid starts once the bound reaches its smallest
 * BAND value, and a grid whose front is done simply has no work.
 *   dims : host, 3 * n_grids int64 (nx, ny, nz of every grid)
 *   h    : host, n_grids spacings
 *   cfg  : dtype, width, stride (in units of the smallest h), bucket,
 *          exchange_passes, ctas, max_restarts, timeout_s, time_kernels,
 *          stream; nx, ny, nz, h and record_tape are ignored / must be 0.
 * The batch handle works with fmm_reinit_batch, fmm_get_stats,
 * fmm_last_error and fmm_destroy.  (Batching is not part of the paper.)
 */
fmm_status fmm_create_batch(int n_grids, const int64_t *dims, const double *h,
                            const fmm_config *cfg, fmm_handle **out);

/*
 * fmm_reinit_batch -- two-sided reinitialisation of every grid of a batch
 * handle (the per-grid rule of fmm_reinit_signed_distance).  phi0, T_out
 * (and tags_out, which may be NULL or hold NULL entries) are host arrays of
 * n_grids device pointers to each grid's x-fastest arrays of the dtype.
 */
fmm_status fmm_reinit_batch(fmm_handle *hd, const void *const *phi0, void *const *T_out,
                            uint8_t *const *tags_out);

/*
 * fmm_solve_batch -- solve every grid of a batch handle in one solve (the
 * marches of all grids share one brick queue and one launch): each grid is
 * either a two-sided reinitialisation of its level set (phi0[g] non-NULL,
 * the rule of fmm_reinit_signed_distance) or a point-source problem
 * (phi0[g] NULL: the n_src[g] cells (i, j, k) of src_ijk[g] get psi = 0,
 * KNOWN_FIX, Algorithm 8), with its own speed: the device field speed[g]
 * (x-fastest, dtype, finite, >= 0; 0 marks an obstacle cell as in
 * fmm_create) or, where speed or speed[g] is NULL, the constant
 * speed_const[g] (> 0; 1 when speed_const is NULL).
 *   phi0, speed      : host arrays of n_grids device pointers (entries may be
 *                      NULL), or NULL for all grids;
 *   src_ijk, n_src   : host arrays of n_grids host pointers / counts (read only
 *                      for grids without phi0; may be NULL when every grid has
 *                      a level set);
 *   speed_const      : host array of n_grids values, or NULL;
 *   T_out, tags_out  : as fmm_reinit_batch.
 * FMM_ERR_INVALID for a misaligned pointer, a source outside its grid, a
 * grid with neither phi0 nor a source list, or a bad speed value.  (Batching
 * is not part of the paper.)
 */
fmm_status fmm_solve_batch(fmm_handle *hd, const void *const *phi0, const int64_t *const *src_ijk,
                           const int64_t *n_src, const void *const *speed, const double *speed_const,
                           void *const *T_out, uint8_t *const *tags_out);

/* fmm_get_stats -- statistics of the last solve (synchronises the stream). */
fmm_status fmm_get_stats(const fmm_handle *hd, fmm_stats *out);

/* One march launch of the last solve (recorded when time_kernels is set). */
typedef struct {
    int32_t restart;   /* pass of the Algorithm 16 loop (1-based)          */
    int32_t phase;     /* 0 = first march, 1.. = exchange passes           */
    int32_t bricks;    /* bricks in the launch's work list                 */
    float ms;          /* device time of the launch (CUDA events)          */
} fmm_trace_entry;

/* fmm_get_trace -- per-launch trace of the last solve on hd: copies up to
 * capacity entries to out (host) and the number available to *n_out.
 * Needs time_kernels = 1 in the handle's config (else *n_out = 0). */
fmm_status fmm_get_trace(const fmm_handle *hd, fmm_trace_entry *out, int64_t capacity,
                         int64_t *n_out);

/* fmm_last_error -- message of the last failing call on hd, or of the last
 * failing fmm_create on this thread when hd is NULL.  Never NULL. */
const char *fmm_last_error(const fmm_handle *hd);

/* fmm_destroy -- free the handle and its workspace (NULL is allowed). */
void fmm_destroy(fmm_handle *hd);

/*
 * fmm_reinit_signed_distance_noalloc -- the same two-sided reinitialisation
 * as fmm_reinit_signed_distance with speed F = 1, for callers that cannot
 * allocate device memory when they solve: processes whose device memory
 * belongs to a pool or arena that forbids further driver allocations (a
 * framework allocator that has reserved the device, an application with a
 * fixed memory budget), and loops that cannot afford an allocation or an
 * out-of-memory failure mid-run.  The paper has no counterpart; this is a
 * packaging of the solve, not a different method.
 *   cfg      : host; nx, ny, nz, h, dtype, width, stride, bucket, ctas,
 *              schedule, exchange_passes, max_restarts, timeout_s and stream
 *              are used and checked as fmm_create checks them; record_tape
 *              must be 0 (no adjoint); no handle is created.
 *   phi0     : device (dtype), the level set; T_out: device (dtype), psi;
 *   tags_out : device uint8 tags or NULL.
 * No memory is allocated: the workspace is one file-scope device array of
 * about 2.4 MiB that every GPU loading the library holds until the process
 * exits.  Limit: at most 512 bricks of 8x8x8 cells (for example a 64^3 grid);
 * larger grids return FMM_ERR_INVALID.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and caches it.  Later
 * calls re-check the cached
 * address (cudaPointerGetAttributes) and look it up again after a
 * cudaDeviceReset.  The call synchronises cfg->stream: it reads the restart
 * control block back between batches of restarts.  All calls on a device share the
 * array and each call clears what it needs; calls whose GPU work overlaps on
 * the same device (e.g. on two streams) race and give undefined results.
 * Errors are reported through fmm_last_error(NULL).
 */
fmm_status fmm_reinit_signed_distance_noalloc(const fmm_config *cfg, const void *phi0, void *T_out,
                                              uint8_t *tags_out);

/*
 * Domain decomposition across processes (Sec. 4.1 and Algorithms 13-16): a
 * handle from fmm_create holds one rank's subdomain -- its slab of z layers
 * plus the ghost layer it shares with each neighbouring rank (the overlap
 * Xi_p of Sec. 4.1 is two layers wide: the rank's last layer and the
 * neighbour's first) -- and the caller runs the loop of Algorithm 16: the
 * global reductions (AllReduce MIN of the per-side minima, MAX of the
 * replaced-cell counts) and the exchange of overlap layers between ranks.
 *   fmm_dd_start     -- Algorithms 8 and 9 on the subdomain: the level set
 *                       phi0 (device, dtype, x-fastest) or, when phi0 is
 *                       NULL, the handle's point sources.  phi0 holds
 *                       extra_lo (0 or 1) layers below the subdomain and
 *                       extra_hi (0 or 1) above it, the neighbours' layers
 *                       beyond the ghost layers, so that the interface cells
 *                       of the ghost layers are those of the whole grid:
 *                       nx * ny * (nz + extra_lo + extra_hi) values.
 *   fmm_dd_minima    -- minval[2] (host): the smallest |psi| of a BAND cell
 *                       per side (-1, +1), width_band when there is none
 *                       (the local heap tops of Algorithm 16).
 *   fmm_dd_march     -- Algorithm 12 up to bound[2] (host; clipped to
 *                       width_band): every brick with a BAND cell at or below
 *                       the bound marches, and bricks whose halo changed march
 *                       again until none is left.
 *   fmm_dd_get_layers -- the nl layers z0 .. z0 + nl - 1 of signed psi
 *                       (x-fastest, nx * ny * nl values of the dtype, +inf
 *                       for FAR cells) into out (device): the outgoing buffer
 *                       of Algorithm 13 (every value; the receiver keeps only
 *                       the improvements).
 *   fmm_dd_integrate -- Algorithm 15 on the layers z0 .. z0 + nl - 1 from in
 *                       (device, as fmm_dd_get_layers writes them): a value
 *                       of smaller magnitude than the local one replaces it
 *                       as a BAND cell of its side (the next fmm_dd_march
 *                       accepts it if it is within the bound); FIX cells are
 *                       kept; *n_replaced (host, may be NULL) receives the
 *                       number of replaced cells (count_new of Algorithm 13,
 *                       counted where the data arrive).
 *   fmm_dd_finish    -- the subdomain's signed psi and tags (device arrays,
 *                       as fmm_solve).
 * All calls synchronise cfg->stream.  FMM_ERR_STATE before fmm_dd_start;
 * FMM_ERR_INVALID for layers outside the grid or non-device buffers.
 */
fmm_status fmm_dd_start(fmm_handle *hd, const void *phi0, int64_t extra_lo, int64_t extra_hi);
fmm_status fmm_dd_minima(fmm_handle *hd, double *minval);
fmm_status fmm_dd_march(fmm_handle *hd, const double *bound);
fmm_status fmm_dd_get_layers(fmm_handle *hd, int64_t z0, int64_t nl, void *out);
fmm_status fmm_dd_integrate(fmm_handle *hd, int64_t z0, int64_t nl, const void *in, int64_t *n_replaced);
fmm_status fmm_dd_finish(fmm_handle *hd, void *T_out, uint8_t *tags_out);

/*
 * fmm_selftest_fp64 -- diagnostics of the double-precision square root and
 * division the fp64 march (Algorithm 11's root) and the adjoint use: for
 * i < n, sqrt_out[i] = sqrt(a[i]) (a[i] >= 0) and div_out[i] = a[i] / b[i],
 * computed by the library's own routines (float seeds refined by Newton steps
 * in double; operands outside [1e-30, 1e30] in magnitude take CUDA's
 * correctly rounded operation).  a, b, sqrt_out, div_out: device, n doubles
 * each, caller-owned; enqueued on stream (cudaStream_t), asynchronous.
 * FMM_ERR_INVALID for n < 0 or a NULL array, FMM_ERR_CUDA if the launch
 * fails.  (Not part of the paper: it lets a test bound the routines' error.)
 */
fmm_status fmm_selftest_fp64(const double *a, const double *b, double *sqrt_out, double *div_out,
                             int64_t n, void *stream);

/*
 * fmm_selftest_root -- diagnostics of the double-grid root of Algorithm 11
 * (Sec. 2, Eq. (2) on the upwind set, solved in double-float arithmetic as
 * the fp64 march does): for i < n, sorted upwind values m[i] <= v1[i] <=
 * v2[i] of which the nd[i] (1..3) smallest take part, speed term q[i] =
 * (h/F)^2 in [1e-30, 1e30]; k_out[i] = the size of the causal set the
 * routine chose (dropping the largest value while the root does not exceed
 * it; 0: none) and t_out[i] = its root (+inf when k = 0).  All arrays device,
 * caller-owned, n elements; enqueued on stream (cudaStream_t), asynchronous.
 * FMM_ERR_INVALID for n < 0 or a NULL array, FMM_ERR_CUDA if the launch
 * fails.  (Not part of the paper: it lets a test check the causal set and
 * the root against exact arithmetic.)
 */
fmm_status fmm_selftest_root(const double *m, const double *v1, const double *v2, const int32_t *nd,
                             const double *q, double *t_out, int32_t *k_out, int64_t n, void *stream);

/*
 * fmm_probe_fma_rate -- diagnostics: the device's fused multiply-add
 * throughput in float (dtype FMM_F32) or double (FMM_F64), the arithmetic
 * ceiling the march kernels are held to beside HBM bandwidth (on GB300 the
 * double pipe, not memory, bounds the fp64 solve).  Runs iters steps of 8
 * independent multiply-add chains per thread on 8 CTAs of 256 threads per SM
 * of the current device (legacy default stream, a warm-up launch first),
 * times the second launch with CUDA events and writes 2 * FMAs / second to
 * *flops_per_s (host).  Synchronous.  FMM_ERR_INVALID for a NULL output,
 * iters < 1 or another dtype; FMM_ERR_CUDA if a launch or event fails.
 * (Not part of the paper.)
 */
fmm_status fmm_probe_fma_rate(int32_t dtype, int64_t iters, double *flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* FMM_GB300_H */
