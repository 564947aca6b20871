// fmm_internal.h -- declarations shared by the translation units of
// libfmm_gb300.so.  Not part of the public ABI (that is include/fmm.h).
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace fmmgb {

// ---------------------------------------------------------------------------
// Brick decomposition.  The grid is cut into 8x8x8 bricks; each brick plays
// the role of one subdomain Omega_p of Sec. 4.1 and its one-cell face halo the
// ghost layer Theta_p.  Brick-major layout: brick id = (bz*nby + by)*nbx + bx,
// the 512 cells of a brick contiguous, x fastest inside the brick.
// ---------------------------------------------------------------------------
constexpr int kB = 8;
constexpr int kB3 = 512;
constexpr int kTile = 10;          // brick plus one halo layer per side
constexpr int kTile3 = 1000;
constexpr int kFaces = 6;          // -x, +x, -y, +y, -z, +z
constexpr int kThreads = 512;      // threads of the per-brick helper kernels

// Cell tag (brick layout).  Bits 0-1: status; bit 2: side -1; bit 3: padding
// cell beyond the grid.  The status values equal the public fmm_tag values.
enum : uint8_t {
    ST_FAR = 0,
    ST_BAND = 1,
    ST_KNOWN = 2,
    ST_FIX = 3,
    ST_MASK = 3,
    TG_NEG = 4,
    TG_OUT = 8,
};

// Device-side error bits (Control::error).
enum : int {
    ERR_ROUNDS = 1,       // a brick march exceeded its round limit
    ERR_RESTARTS = 2,     // the restart limit was reached
    ERR_SPEED = 4,        // a speed value was not finite and > 0
    ERR_SPIN = 8,         // a bounded wait of the persistent march gave up
    ERR_INPUT = 16,       // given interface values: NaN, or a sign change
                          // without FIX cells at both ends
};

// Restart control block of Algorithm 16, in device memory.
struct Control {
    unsigned long long minbits[2];   // min |psi| over BAND cells per side
                                     // (bits of a non-negative double)
    unsigned long long marches;      // statistics
    unsigned long long rounds;
    unsigned long long exchanges;
    unsigned long long accepted;
    unsigned long long solves;       // Algorithm 11 evaluations
    double bound[2];                 // bound_band(-1), bound_band(+1)
    unsigned int dirty_count;        // count_global: bricks with pending
                                     // overlap changes
    unsigned int n_list[2];          // lengths of the two work lists
    unsigned int work[2];            // next unclaimed entry of each list
    int done;
    int error;
    int restart;                     // bound levels (restarts and raises)
    int host_restart;                // restarts the host enqueued (k_control)
    // persistent march: ring queue positions and the count of bricks pushed
    // and not yet marched, each on a line of its own (they are the only
    // words every warp touches)
    alignas(128) unsigned long long q_head;
    alignas(128) unsigned long long q_tail;
    alignas(128) int pending;
    int pad2[31];
    // continuous schedule: bound level (even = stable, odd = being raised),
    // chunk counters of the scan for the current level, minima it saw
    alignas(128) int epoch;
    int scan_next;
    int scan_done;
    int scan_clean;                  // the last scan started with nothing in flight
    int pad3;
    unsigned long long scan_min[2];
    unsigned long long wait_ns;      // limit of every device wait without progress
    int hold;                        // testing: one brick counted as pending forever
    int pad4[19];
};

struct Geom {
    int nx, ny, nz;
    int nbx, nby, nbz;
    long long nbricks;
};

// Parameters of one solve.
struct SolveParams {
    double h;           // cell size along x; the stride and the speed term
                        // (h/F)^2 are in its units
    double w;           // (1/h)^2
    double width;       // width_band
    double stride;      // delta_s (absolute units)
    double bucket;      // bucket width factor
    double spd_term;    // speed term (h/F)^2 of a constant speed
    long long max_restarts;
    int max_rounds;     // per brick march
    int passes;         // exchange + march passes after the first march
    int schedule;       // kSchedulePhased, kSchedulePersistent or kScheduleContinuous
    int raise_at;       // continuous schedule: raise the bound when fewer
                        // bricks than this are queued or marching
    double max_lead;    // continuous schedule: lead of the bound in strides
    double ahead;       // continuous schedule: a brick march accepts cells up
                        // to bound + ahead (absolute units; +inf: the whole
                        // brick), and a brick whose only work is halo changes
                        // starts once the bound reaches their smallest value
    unsigned long long wait_ns;   // limit of a device wait without progress
    int hold;           // testing: keep one phantom brick pending
    int aniso;          // hy or hz differs from h
    double hy, hz;      // cell sizes along y and z (h on a cubic-cell grid)
    double wy, wz;      // (h/hy)^2, (h/hz)^2: the h_i^2 of Algorithm 11
                        // relative to the x axis
    int accuracy;       // 1: Eq. (2)-(3); 2: second-order upwind differences
                        // (the cell-parallel schedule only)
};

// Cell sizes of Sec. 2.1 (hy, hz <= 0 mean h) and the per-axis weights of
// Algorithm 11 relative to the x axis.
inline void set_spacing(SolveParams &p, double h, double hy, double hz)
{
    p.h = h;
    p.hy = hy > 0.0 ? hy : h;
    p.hz = hz > 0.0 ? hz : h;
    p.wy = (h / p.hy) * (h / p.hy);
    p.wz = (h / p.hz) * (h / p.hz);
    p.aniso = p.hy != h || p.hz != h;
    p.w = (1.0 / h) * (1.0 / h);
}
inline double min_spacing(const SolveParams &p)
{
    const double m = p.h < p.hy ? p.h : p.hy;
    return m < p.hz ? m : p.hz;
}

constexpr int kSchedulePhased = 1;
constexpr int kSchedulePersistent = 2;
constexpr int kScheduleContinuous = 3;
constexpr int kScheduleCell = 4;     // cell-parallel bucketed march (fmm_cell.cu)
constexpr int kMarchWarps = 4;   // bricks in flight per CTA of the march kernels
#ifndef FMM_RAISE_DIV
#define FMM_RAISE_DIV 2
#endif
// Continuous schedule: the bound rises once fewer bricks than this are queued
// or marching (a fraction of the warps of the march launch).
inline int raise_threshold(int march_ctas) { return march_ctas * kMarchWarps / FMM_RAISE_DIV; }
// bricks one warp scans for the next bound (continuous schedule)
#ifndef FMM_SCAN_CHUNK
#define FMM_SCAN_CHUNK 1024
#endif
constexpr int kScanChunk = FMM_SCAN_CHUNK;
inline bool one_launch_schedule(int schedule)
{
    return schedule == kSchedulePersistent || schedule == kScheduleContinuous;
}

// Defaults of the restart parameters (units of h and of the bucket width),
// measured on GB300 for 8^3 bricks.
inline double default_stride(int dtype) { return dtype == 1 ? 1.0 : 2.0; }
// deterministic mode (phased schedule, pass-synchronous halos): information
// crosses one brick per pass, so wider strides pay (1024^3 sphere: fp64
// 722 / 493 / 529 ms at 1 / 4 / 8 h, fp32 374 / 278 / 238 ms at 2 / 4 / 8 h)
inline double default_stride_deterministic(int dtype) { return dtype == 1 ? 4.0 : 8.0; }
inline int default_passes(int dtype) { return dtype == 1 ? 1 : 2; }
// continuous schedule: look-ahead of a brick march beyond the bound (units of
// h; +inf: a brick marches to its end once the bound reaches its smallest
// BAND or changed halo value) and the lead limit of the bound (strides;
// +inf: none), measured on GB300 for 8^3 bricks
inline double default_ahead(int) { return INFINITY; }
inline double default_max_lead() { return INFINITY; }
constexpr double kDefaultBucket = 4.0;
// The second-order march's default bucket: a single-axis second-order root
// exceeds its upwind value by at least (2/3) h / F, so with buckets narrower
// than 2/3 (units of hmin min(1/F) / sqrt 3) a cell and the neighbour it
// mainly depends on are not accepted in the same step, and an accepted value
// is (up to corrections through axes of vanishing weight) final when the
// cells around it read it, as in the sequential march where every KNOWN
// value is final.  Wider buckets let a cell accepted with a value that the
// same step lowers serve as a stale second neighbour, whose too-large psi2
// lowers the root of another cell below its value; a cell keeps the
// smallest of its roots, so that error stays.
constexpr double kSecondOrderBucket = 0.6;

// Device buffers owned by a handle (typed by the launchers).
struct DeviceState {
    void *T;            // |psi| per cell, brick layout
    uint8_t *tag;       // tag per cell, brick layout
    void *spd;          // speed term per cell (brick layout) or null
    void *bdelta;       // per-brick bucket width (h * min slowness / sqrt 3)
    uint8_t *tape;      // upwind set per cell or null
    void *bmin;         // 2 per brick: min |psi| of BAND cells per side
    unsigned long long *fresh;   // 6 per brick: changed-halo masks (live)
    unsigned long long *inmin;   // 2 per brick (sides -1, +1): smallest value a
                                 // neighbour flagged in the masks since the
                                 // brick last took them (bits of a double;
                                 // all ones: none recorded)
    void *faces;        // deterministic mode, 6 x 64 per brick: its boundary
                        // layers (known value or +inf) as of the last pass
    unsigned long long *inbox;   // 6 per brick: masks taken by the last selection
    unsigned int *dirty;         // 1 per brick: has pending overlap changes
    int *list[2];       // work lists
    const int *nbr;     // 6 per brick: neighbour brick or -1 (batches only)
    unsigned long long *queue;   // persistent march: ring of (seq << 32 | brick + 1)
    unsigned *queued;            // per brick: in the queue or being marched
    Control *ctrl;
    int march_ctas;
};

// One grid of a batch (device table).
struct BatchGrid {
    int nx, ny, nz;
    int nbx, nby, nbz;
    long long brick0;      // first brick of the grid in the packed brick array
    double h;
    const void *phi0;      // caller's level set (x-fastest), or null: point sources
    void *T_out;           // caller's output psi (x-fastest)
    uint8_t *tags_out;     // caller's output tags or null
    const void *speed;     // caller's speed field (x-fastest) or null: speed_const
    double speed_const;
    long long src0, n_src; // the grid's sources in the batch's source array
};

// Launchers (fmm_march.cu).  All enqueue on `stream`; `dtype` is 0 for float
// and 1 for double.
cudaError_t launch_init_sources(int dtype, const Geom &g, const DeviceState &s,
                                const long long *src_ijk, long long n_src,
                                cudaStream_t stream);
// phi0 holds zlo extra layers below the grid and zhi above it (a subdomain
// of a decomposed grid); 0, 0 for a whole grid
cudaError_t launch_init_reinit(int dtype, const Geom &g, const DeviceState &s,
                               const SolveParams &p, const void *phi0,
                               cudaStream_t stream, int zlo = 0, int zhi = 0);
// h: the x cell size of the speed term (h/F)^2; hmin: the smallest cell size,
// the unit of the bucket width
cudaError_t launch_load_speed(int dtype, const Geom &g, const DeviceState &s,
                              double h, double hmin, const void *speed, double speed_const,
                              cudaStream_t stream);
cudaError_t launch_front_init(int dtype, const Geom &g, const DeviceState &s,
                              const SolveParams &p, cudaStream_t stream);
// One pass of the Algorithm 16 loop: reduce, control, the first select +
// march, then p.passes exchange passes (select + march, with a list reset
// before every pass but the first).  ev, when not null, holds one event pair
// per march launch (2 * (1 + passes) events).
inline int launches_per_restart(int passes, int schedule)
{
    return one_launch_schedule(schedule) ? 4 : 2 + 2 * (1 + passes) + (passes - 1);
}
// march launches (timed, traced) per restart
inline int marches_per_restart(int passes, int schedule)
{
    return one_launch_schedule(schedule) ? 1 : 1 + passes;
}
cudaError_t launch_restart(int dtype, const Geom &g, const DeviceState &s,
                           const SolveParams &p, cudaStream_t stream, cudaEvent_t *ev,
                           int *trace);
cudaError_t launch_reset_control(const DeviceState &s, cudaStream_t stream,
                                 unsigned long long wait_ns, int hold);
cudaError_t launch_output(int dtype, const Geom &g, const DeviceState &s,
                          void *T_out, uint8_t *tags_out, cudaStream_t stream);
int march_blocks_per_sm(int dtype, bool tape);
// Deterministic mode: rebuild the boundary layers of every brick from the state.
cudaError_t launch_faces_build(int dtype, const Geom &g, const DeviceState &s, cudaStream_t st);
cudaError_t launch_batch_init(int dtype, const BatchGrid *grids, const int *bgrid,
                              long long nbricks, const DeviceState &s, cudaStream_t stream);
cudaError_t launch_batch_speed(int dtype, const BatchGrid *grids, const int *bgrid,
                               long long nbricks, const DeviceState &s, cudaStream_t stream);
// src: 4 per source (grid, i, j, k)
cudaError_t launch_batch_sources(int dtype, const BatchGrid *grids, const long long *src,
                                 long long n_src, const DeviceState &s, cudaStream_t stream);
cudaError_t launch_batch_output(int dtype, const BatchGrid *grids, const int *bgrid,
                                long long nbricks, const DeviceState &s, cudaStream_t stream);
cudaError_t launch_select(int dtype, const Geom &g, const DeviceState &s, int which,
                          cudaStream_t stream);
// domain decomposition: overlap layers z0 .. z0 + nl - 1 (signed psi,
// x-fastest), their integration (count: replaced cells, added), one march to
// a given bound, and the per-side BAND minima (into Control::minbits)
cudaError_t launch_layer_export(int dtype, const Geom &g, const DeviceState &s, int z0, int nl,
                                void *out, cudaStream_t stream);
cudaError_t launch_layer_integrate(int dtype, const Geom &g, const DeviceState &s, int z0, int nl,
                                   const void *in, unsigned *count, cudaStream_t stream);
cudaError_t launch_march_to(int dtype, const Geom &g, const DeviceState &s, const SolveParams &p,
                            double b0, double b1, cudaStream_t stream);
cudaError_t launch_minima(int dtype, const Geom &g, const DeviceState &s, cudaStream_t stream);
cudaError_t launch_reset_list(const DeviceState &s, int which, cudaStream_t stream);

// Cell-parallel march and initialisation from given values (fmm_cell.cu).
// T0: the caller's x-fastest values (finite: FIX on the side of its sign;
// +-inf: FAR on that side); sets ERR_INPUT in the control block for NaN or a
// sign change between two cells that are not both FIX.
cudaError_t launch_init_fixed(int dtype, const Geom &g, const DeviceState &s, const void *T0,
                              cudaStream_t stream);
// next: one value per brick-layout cell (the step's new values); mins: 4
// words (two slots of the per-side BAND minima).  begin runs Algorithm 9 and
// fills slot 0; step k accepts from slot k & 1 and fills the other one.
cudaError_t launch_cell_begin(int dtype, const Geom &g, const DeviceState &s, const SolveParams &p,
                              void *next, unsigned long long *mins, cudaStream_t stream);
cudaError_t launch_cell_step(int dtype, const Geom &g, const DeviceState &s, const SolveParams &p,
                             void *next, unsigned long long *mins, long long step, cudaStream_t stream);

// Adjoint (fmm_adjoint.cu).  The reverse sweep can run by levels of |psi|
// of kAdjointLevelStep h each (at most kAdjointMaxLevels); 0 (the default)
// runs it as one level.  Measured on GB300 (512^3 heterogeneous speed):
// steps of 4-128 h cut brick passes from 7 to 3.7-6 per brick but were 2-60 %
// slower, so one level it is.
#ifndef FMM_ADJ_STEP_H
#define FMM_ADJ_STEP_H 0.0
#endif
constexpr double kAdjointLevelStep = FMM_ADJ_STEP_H;
constexpr long long kAdjointMaxLevels = 4096;
struct AdjointArgs {
    const void *dLdT;   // caller's dL/dpsi, x-fastest
    void *dlds;         // caller's dL/ds output, x-fastest
    void *mu;           // lambda / D per cell (brick layout), NaN until done
    void *top;          // per brick: largest |psi| of a cell still to do
                        // (bits of a non-negative value; 0: none left)
    Control *ctrl;      // the handle's control block (levels: Control::bound[0])
    double h;
    double spd_term;    // (h/F)^2 of a constant speed
    double wy, wz;      // (h/hy)^2, (h/hz)^2 (1 on a cubic-cell grid)
    int aniso;
};
cudaError_t launch_adjoint_init(int dtype, const Geom &g, const DeviceState &s,
                                const AdjointArgs &a, cudaStream_t stream);
// The reverse sweep by descending levels: level k starts the bricks whose
// largest unfinished |psi| is at or above top_max - (k + 1) step (the last
// level every brick), each level one persistent launch.
cudaError_t launch_adjoint_levels(int dtype, const Geom &g, const DeviceState &s,
                                  const AdjointArgs &a, double top_max, double step, int levels,
                                  cudaStream_t st);
// the largest per-brick top into *out (host, synchronous)
cudaError_t adjoint_top_max(int dtype, const Geom &g, const AdjointArgs &a, double *out,
                            cudaStream_t st);
cudaError_t launch_adjoint_pending(int dtype, const Geom &g, const AdjointArgs &a,
                                   unsigned *count, cudaStream_t stream);

}  // namespace fmmgb
