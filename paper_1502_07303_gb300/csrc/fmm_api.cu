// fmm_api.cu -- the C ABI of libfmm_gb300.so (declared in include/fmm.h):
// handle lifecycle, argument checking, device workspace and the host side of
// the restart loop of Algorithm 16.
#include "fmm.h"
#include "fmm_internal.h"

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace fmmgb;

struct fmm_handle {
    fmm_config cfg;
    Geom geom;
    SolveParams params;
    DeviceState st;
    cudaStream_t stream = nullptr;
    size_t rsize = 4;
    double speed_const = 1.0;
    long long *d_src = nullptr;
    long long n_src = 0;
    Control *h_ctrl = nullptr;   // pinned host mirror of the control block
    bool solved = false;
    bool tape_valid = false;
    bool resumable = false;           // stopped at the restart or time limit
    bool complete = false;            // the last forward solve finished
    Control fwd_ctrl;                 // its control block as it ended
    long long pre_launches = 0;       // init launches of the current solve
    fmm_stats stats;
    std::vector<cudaEvent_t> events;   // march timing pairs (time_kernels)
    int *d_trace = nullptr;            // 3 ints per march launch (time_kernels)
    size_t trace_cap = 0;              // launches the trace buffer holds
    std::vector<fmm_trace_entry> trace;
    void *adj_mu = nullptr;            // adjoint workspace (lambda / D per cell)
    unsigned *adj_count = nullptr;
    void *adj_top = nullptr;           // per brick: largest |psi| still to do
    unsigned *dd_count = nullptr;      // domain decomposition: replaced cells
    unsigned *h_dd_count = nullptr;    // pinned
    bool dd_started = false;
    // device copies of the caller's host arrays (x-fastest, allocated on
    // first use): inputs and psi / dL/ds, a second array, tags
    void *stage[2] = {nullptr, nullptr};
    uint8_t *stage_tags = nullptr;
    // batches (fmm_create_batch)
    int n_grids = 0;
    BatchGrid *d_grids = nullptr;
    BatchGrid *h_grids = nullptr;      // pinned
    int *d_bgrid = nullptr;
    int *d_nbr = nullptr;
    long long *d_bsrc = nullptr;       // batch sources, 4 per source (grid, i, j, k)
    size_t bsrc_cap = 0;               // sources d_bsrc holds
    bool batch_speed_const1 = true;    // the speed terms on the device are F = 1
    // cell-parallel march (schedule 4): the step's new values (brick
    // layout) and two slots of the per-side BAND minima
    void *cell_next = nullptr;
    unsigned long long *cell_min = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

fmm_status fail(fmm_handle *hd, fmm_status code, const std::string &msg)
{
    if (hd)
        hd->err = msg;
    else
        g_create_error = msg;
    return code;
}

fmm_status cuda_fail(fmm_handle *hd, cudaError_t e, const char *where)
{
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(hd, e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA, msg);
}

#define FMM_CUDA(hd, call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess)                              \
            return cuda_fail((hd), e_, #call);              \
    } while (0)

void free_state(fmm_handle *hd)
{
    DeviceState &s = hd->st;
    void *ptrs[] = {s.T,      s.tag,      s.spd,   s.bdelta,  s.tape,   s.bmin,   s.fresh, s.inmin, s.inbox,
                    s.dirty,  s.list[0],  s.list[1], s.ctrl,  hd->d_src, s.queue, s.queued, s.faces};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    if (hd->h_ctrl)
        cudaFreeHost(hd->h_ctrl);
    for (cudaEvent_t e : hd->events)
        cudaEventDestroy(e);
    hd->events.clear();
    if (hd->d_trace)
        cudaFree(hd->d_trace);
    hd->d_trace = nullptr;
    hd->trace_cap = 0;
    if (hd->d_grids)
        cudaFree(hd->d_grids);
    if (hd->d_bgrid)
        cudaFree(hd->d_bgrid);
    if (hd->d_nbr)
        cudaFree(hd->d_nbr);
    if (hd->d_bsrc)
        cudaFree(hd->d_bsrc);
    hd->d_bsrc = nullptr;
    hd->bsrc_cap = 0;
    if (hd->h_grids)
        cudaFreeHost(hd->h_grids);
    hd->d_grids = nullptr;
    hd->d_bgrid = nullptr;
    hd->d_nbr = nullptr;
    hd->h_grids = nullptr;
    if (hd->adj_mu)
        cudaFree(hd->adj_mu);
    if (hd->adj_count)
        cudaFree(hd->adj_count);
    if (hd->adj_top)
        cudaFree(hd->adj_top);
    hd->adj_top = nullptr;
    if (hd->dd_count)
        cudaFree(hd->dd_count);
    if (hd->h_dd_count)
        cudaFreeHost(hd->h_dd_count);
    hd->dd_count = nullptr;
    hd->h_dd_count = nullptr;
    hd->adj_mu = nullptr;
    hd->adj_count = nullptr;
    for (void *&p : hd->stage) {
        if (p)
            cudaFree(p);
        p = nullptr;
    }
    if (hd->stage_tags)
        cudaFree(hd->stage_tags);
    hd->stage_tags = nullptr;
    if (hd->cell_next)
        cudaFree(hd->cell_next);
    if (hd->cell_min)
        cudaFree(hd->cell_min);
    hd->cell_next = nullptr;
    hd->cell_min = nullptr;
    memset(&hd->st, 0, sizeof(hd->st));
    hd->d_src = nullptr;
    hd->h_ctrl = nullptr;
}

template <typename T>
cudaError_t alloc(T **p, size_t bytes)
{
    return cudaMalloc((void **)p, bytes < 16 ? 16 : bytes);
}

// A caller's array in host memory (page-locked or pageable) rather than in
// device memory (managed memory counts as device memory).
bool is_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error of an unknown pointer
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// The grid's cells in the caller's x-fastest layout.
size_t natural_cells(const fmm_handle *hd)
{
    return (size_t)hd->geom.nx * hd->geom.ny * hd->geom.nz;
}

// Device buffer k of the host staging (n values of the dtype), allocated on
// first use.
fmm_status stage_buffer(fmm_handle *hd, int k, void **out)
{
    if (!hd->stage[k])
        FMM_CUDA(hd, alloc(&hd->stage[k], natural_cells(hd) * hd->rsize));
    *out = hd->stage[k];
    return FMM_OK;
}

// An input array as the kernels read it: host arrays are copied (on the
// handle's stream) into staging buffer k.
fmm_status device_input(fmm_handle *hd, const void *arr, int k, const void **out)
{
    if (!is_host(arr)) {
        *out = arr;
        return FMM_OK;
    }
    void *buf = nullptr;
    const fmm_status r = stage_buffer(hd, k, &buf);
    if (r != FMM_OK)
        return r;
    FMM_CUDA(hd, cudaMemcpyAsync(buf, arr, natural_cells(hd) * hd->rsize, cudaMemcpyHostToDevice,
                                 hd->stream));
    *out = buf;
    return FMM_OK;
}

fmm_status load_speed(fmm_handle *hd, const void *speed, double speed_const)
{
    if (!speed && !(speed_const > 0.0 && std::isfinite(speed_const)))
        return fail(hd, FMM_ERR_INVALID, "speed_const must be finite and > 0 when speed is NULL");
    DeviceState &s = hd->st;
    const size_t cells = (size_t)hd->geom.nbricks * kB3;
    if (speed && !s.spd)
        FMM_CUDA(hd, alloc(&s.spd, cells * hd->rsize));
    if (!speed && s.spd) {
        cudaFree(s.spd);
        s.spd = nullptr;
    }
    hd->speed_const = speed ? 1.0 : speed_const;
    if (speed) {
        const fmm_status r = device_input(hd, speed, 0, &speed);
        if (r != FMM_OK)
            return r;
    }
    FMM_CUDA(hd, launch_reset_control(s, hd->stream, hd->params.wait_ns, hd->params.hold));
    FMM_CUDA(hd, launch_load_speed(hd->cfg.dtype, hd->geom, s, hd->params.h,
                                   min_spacing(hd->params), speed,
                                   hd->speed_const, hd->stream));
    FMM_CUDA(hd, cudaMemcpyAsync(hd->h_ctrl, s.ctrl, sizeof(Control), cudaMemcpyDeviceToHost,
                                 hd->stream));
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    if (hd->h_ctrl->error & ERR_SPEED)
        return fail(hd, FMM_ERR_INVALID, "speed values must be finite and > 0");
    // the constant-speed term of the shifted quadratic: (h/F)^2
    hd->params.spd_term = 0.0;
    if (!speed) {
        if (hd->cfg.dtype == FMM_F64) {
            hd->params.spd_term = (hd->params.h * hd->params.h) / (speed_const * speed_const);
        } else {
            const float hf = (float)hd->params.h;
            const float F = (float)speed_const;
            hd->params.spd_term = (double)((hf * hf) / (F * F));
        }
    }
    hd->tape_valid = false;
    hd->resumable = false;
    return FMM_OK;
}

fmm_status run_restarts(fmm_handle *hd, void *T_out, uint8_t *tags_out, long long launches);
fmm_status run_cell(fmm_handle *hd, void *T_out, uint8_t *tags_out);

// Algorithm 9, then the loop of Algorithm 16, then the output conversion.
fmm_status run_solve(fmm_handle *hd, void *T_out, uint8_t *tags_out)
{
    if (hd->params.schedule == kScheduleCell)
        return run_cell(hd, T_out, tags_out);
    DeviceState &s = hd->st;
    const Geom &g = hd->geom;
    const int dt = hd->cfg.dtype;
    cudaStream_t st = hd->stream;
    hd->solved = hd->tape_valid = hd->resumable = hd->complete = false;
    FMM_CUDA(hd, launch_reset_control(s, st, hd->params.wait_ns, hd->params.hold));
    FMM_CUDA(hd, cudaMemsetAsync(s.fresh, 0, (size_t)g.nbricks * kFaces * sizeof(unsigned long long), st));
    FMM_CUDA(hd, cudaMemsetAsync(s.inmin, 0xff, (size_t)g.nbricks * 2 * sizeof(unsigned long long), st));
    FMM_CUDA(hd, cudaMemsetAsync(s.dirty, 0, (size_t)g.nbricks * sizeof(unsigned), st));
    FMM_CUDA(hd, cudaMemsetAsync(s.queue, 0, (size_t)g.nbricks * sizeof(unsigned long long), st));
    FMM_CUDA(hd, cudaMemsetAsync(s.queued, 0, (size_t)g.nbricks * sizeof(unsigned), st));
    FMM_CUDA(hd, launch_front_init(dt, g, s, hd->params, st));
    return run_restarts(hd, T_out, tags_out, 2);   // control reset, front init
}

// The output conversion into the caller's arrays (device memory, or host
// memory through the staging buffers), then a synchronisation of the stream.
fmm_status write_outputs(fmm_handle *hd, void *T_out, uint8_t *tags_out, long long &launches)
{
    DeviceState &s = hd->st;
    const Geom &g = hd->geom;
    const int dt = hd->cfg.dtype;
    cudaStream_t st = hd->stream;
    if (T_out) {
        // host outputs go through the staging buffers (the input the first
        // one held was consumed by the initialisation, earlier on the stream)
        const bool host_T = is_host(T_out), host_G = tags_out && is_host(tags_out);
        void *Td = T_out;
        uint8_t *Gd = tags_out;
        if (host_T) {
            const fmm_status r = stage_buffer(hd, 0, &Td);
            if (r != FMM_OK)
                return r;
        }
        if (host_G) {
            if (!hd->stage_tags)
                FMM_CUDA(hd, alloc(&hd->stage_tags, natural_cells(hd)));
            Gd = hd->stage_tags;
        }
        FMM_CUDA(hd, launch_output(dt, g, s, Td, Gd, st));
        launches += 1;
        if (host_T)
            FMM_CUDA(hd, cudaMemcpyAsync(T_out, Td, natural_cells(hd) * hd->rsize,
                                         cudaMemcpyDeviceToHost, st));
        if (host_G)
            FMM_CUDA(hd, cudaMemcpyAsync(tags_out, Gd, natural_cells(hd), cudaMemcpyDeviceToHost, st));
    }
    FMM_CUDA(hd, cudaStreamSynchronize(st));
    return FMM_OK;
}

// The loop of Algorithm 16 from the current state (a fresh initialisation or
// the state after the last completed restart), then the output conversion.
fmm_status run_restarts(fmm_handle *hd, void *T_out, uint8_t *tags_out, long long launches)
{
    DeviceState &s = hd->st;
    const Geom &g = hd->geom;
    const int dt = hd->cfg.dtype;
    cudaStream_t st = hd->stream;
    const bool timing = hd->cfg.time_kernels != 0;
    size_t ev_used = 0;
    // The loop of Algorithm 16 runs on the device; the host enqueues restarts
    // in growing batches and reads the termination flag between batches
    // (restarts enqueued after termination return at once).
    const auto t0 = std::chrono::steady_clock::now();
    const double limit_s = hd->cfg.timeout_s > 0 ? (double)hd->cfg.timeout_s : 600.0;
    bool timed_out = false;
    long long batch = 1;
    for (;;) {
        const size_t ev_per = 2 * (size_t)marches_per_restart(hd->params.passes, hd->params.schedule);
        for (long long r = 0; r < batch; ++r) {
            cudaEvent_t *ev = nullptr;
            int *tr = nullptr;
            if (timing) {
                while (hd->events.size() < ev_used + ev_per) {
                    cudaEvent_t e;
                    FMM_CUDA(hd, cudaEventCreate(&e));
                    hd->events.push_back(e);
                }
                ev = &hd->events[ev_used];
                const size_t launch_idx = ev_used / 2;
                if (launch_idx + ev_per / 2 > hd->trace_cap) {
                    // grow the trace buffer (between batches nothing is in
                    // flight that writes to it)
                    FMM_CUDA(hd, cudaStreamSynchronize(st));
                    const size_t cap = 2 * (launch_idx + ev_per / 2) + 64;
                    int *nb = nullptr;
                    FMM_CUDA(hd, alloc(&nb, cap * 3 * sizeof(int)));
                    if (hd->d_trace) {
                        FMM_CUDA(hd, cudaMemcpy(nb, hd->d_trace, hd->trace_cap * 3 * sizeof(int),
                                                cudaMemcpyDeviceToDevice));
                        cudaFree(hd->d_trace);
                    }
                    hd->d_trace = nb;
                    hd->trace_cap = cap;
                }
                tr = hd->d_trace + 3 * launch_idx;
                ev_used += ev_per;
            }
            FMM_CUDA(hd, launch_restart(dt, g, s, hd->params, st, ev, tr));
            launches += launches_per_restart(hd->params.passes, hd->params.schedule) +
                        (timing ? marches_per_restart(hd->params.passes, hd->params.schedule) : 0);
        }
        FMM_CUDA(hd, cudaMemcpyAsync(hd->h_ctrl, s.ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
        FMM_CUDA(hd, cudaStreamSynchronize(st));
        if (hd->h_ctrl->done || (hd->h_ctrl->error & (ERR_SPIN | ERR_ROUNDS | ERR_RESTARTS)))
            break;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > limit_s) {
            timed_out = true;
            break;
        }
        if (batch < 16)
            batch *= 2;
    }
    const Control &c = *hd->h_ctrl;
    hd->stats.restarts = c.restart;
    hd->stats.brick_marches = (int64_t)c.marches;
    hd->stats.march_rounds = (int64_t)c.rounds;
    hd->stats.exchanges = (int64_t)c.exchanges;
    hd->stats.accepted = (int64_t)c.accepted;
    hd->stats.cell_solves = (int64_t)c.solves;
    hd->stats.n_bricks = g.nbricks;
    hd->stats.error_flags = c.error;
    {
        const fmm_status r = write_outputs(hd, T_out, tags_out, launches);
        if (r != FMM_OK)
            return r;
    }
    // restarts after the terminating pass only return; the march launches
    // that did work are those of every pass but the last
    const long long worked =
        c.host_restart > 0
            ? (long long)marches_per_restart(hd->params.passes, hd->params.schedule) * (c.host_restart - 1)
            : 0;
    hd->stats.march_launches = worked;
    hd->stats.kernel_launches = launches + hd->pre_launches;
    hd->pre_launches = 0;
    double ms = 0.0;
    if (timing) {
        for (long long k = 0; k < worked && (size_t)(2 * k + 1) < ev_used; ++k) {
            float e = 0.f;
            FMM_CUDA(hd, cudaEventElapsedTime(&e, hd->events[2 * k], hd->events[2 * k + 1]));
            ms += e;
        }
    }
    hd->stats.march_ms = ms;
    hd->trace.clear();
    if (timing && worked > 0) {
        std::vector<int> tr((size_t)worked * 3);
        FMM_CUDA(hd, cudaMemcpy(tr.data(), hd->d_trace, tr.size() * sizeof(int), cudaMemcpyDeviceToHost));
        for (long long k = 0; k < worked && (size_t)(2 * k + 1) < ev_used; ++k) {
            fmm_trace_entry e;
            e.restart = tr[3 * k];
            e.phase = tr[3 * k + 1];
            e.bricks = tr[3 * k + 2];
            float t = 0.f;
            FMM_CUDA(hd, cudaEventElapsedTime(&t, hd->events[2 * k], hd->events[2 * k + 1]));
            e.ms = t;
            hd->trace.push_back(e);
        }
    }
    hd->solved = true;
    hd->complete = c.done && c.error == 0 && !timed_out;
    hd->tape_valid = hd->complete && s.tape != nullptr;
    // a solve stopped by the restart or wall-clock limit ends on a restart
    // boundary: the state can be resumed (or saved and resumed elsewhere)
    hd->resumable = !hd->complete && (timed_out ? c.error == 0 : c.error == ERR_RESTARTS);
    hd->fwd_ctrl = c;
    if (timed_out)
        return fail(hd, FMM_ERR_TIMEOUT, "the solve exceeded its wall-clock limit (timeout_s)");
    if (c.error & ERR_ROUNDS)
        return fail(hd, FMM_ERR_TIMEOUT, "a brick march exceeded its round limit");
    if (c.error & ERR_SPIN)
        return fail(hd, FMM_ERR_TIMEOUT, "a bounded wait of the persistent march gave up");
    if (c.error & ERR_RESTARTS)
        return fail(hd, FMM_ERR_TIMEOUT, "the restart limit was reached before termination");
    return FMM_OK;
}

// The cell-parallel march (schedule 4): Algorithm 9, then bucket steps until
// the step that finds no BAND cell at or below width_band, enqueued in
// growing batches with the termination flag read between batches (steps
// enqueued after it return at once); then the output conversion.  The march
// has no restart boundary to stop on: a solve stopped by max_restarts (here
// a limit on the bucket steps) or timeout_s cannot be resumed.
fmm_status run_cell(fmm_handle *hd, void *T_out, uint8_t *tags_out)
{
    DeviceState &s = hd->st;
    const Geom &g = hd->geom;
    const int dt = hd->cfg.dtype;
    const SolveParams &p = hd->params;
    cudaStream_t st = hd->stream;
    hd->solved = hd->tape_valid = hd->resumable = hd->complete = false;
    if (g.nbricks > 0xffffffffll)
        return fail(hd, FMM_ERR_INVALID, "the cell-parallel schedule takes grids of fewer than 2^32 bricks");
    const size_t cells = (size_t)g.nbricks * kB3;
    if (!hd->cell_next)
        FMM_CUDA(hd, alloc(&hd->cell_next, cells * hd->rsize));
    if (!hd->cell_min)
        FMM_CUDA(hd, alloc(&hd->cell_min, 4 * sizeof(unsigned long long)));
    const bool timing = hd->cfg.time_kernels != 0;
    while (timing && hd->events.size() < 2) {
        cudaEvent_t e;
        FMM_CUDA(hd, cudaEventCreate(&e));
        hd->events.push_back(e);
    }
    FMM_CUDA(hd, launch_reset_control(s, st, p.wait_ns, p.hold));
    if (timing)
        FMM_CUDA(hd, cudaEventRecord(hd->events[0], st));
    FMM_CUDA(hd, launch_cell_begin(dt, g, s, p, hd->cell_next, hd->cell_min, st));
    long long launches = 4;   // control reset; seed, relax, apply
    const auto t0 = std::chrono::steady_clock::now();
    const double limit_s = hd->cfg.timeout_s > 0 ? (double)hd->cfg.timeout_s : 600.0;
    bool timed_out = false, limited = false;
    long long step = 0, batch = 1;
    for (;;) {
        long long n = batch;
        if (p.max_restarts > 0 && step + n > p.max_restarts)
            n = p.max_restarts - step;
        for (long long r = 0; r < n; ++r, ++step) {
            FMM_CUDA(hd, launch_cell_step(dt, g, s, p, hd->cell_next, hd->cell_min, step, st));
            launches += 3;
        }
        FMM_CUDA(hd, cudaMemcpyAsync(hd->h_ctrl, s.ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
        FMM_CUDA(hd, cudaStreamSynchronize(st));
        if (hd->h_ctrl->done)
            break;
        if (p.max_restarts > 0 && step >= p.max_restarts) {
            limited = true;
            break;
        }
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit_s) {
            timed_out = true;
            break;
        }
        if (batch < 64)
            batch *= 2;
    }
    if (timing)
        FMM_CUDA(hd, cudaEventRecord(hd->events[1], st));
    const Control c = *hd->h_ctrl;
    {
        const fmm_status r = write_outputs(hd, T_out, tags_out, launches);
        if (r != FMM_OK)
            return r;
    }
    memset(&hd->stats, 0, sizeof(hd->stats));
    hd->stats.restarts = c.restart;   // bucket steps that accepted cells
    hd->stats.accepted = (int64_t)c.accepted;
    hd->stats.cell_solves = (int64_t)c.solves;
    hd->stats.n_bricks = g.nbricks;
    hd->stats.error_flags = c.error;
    hd->stats.kernel_launches = launches + hd->pre_launches;
    hd->stats.march_launches = 3 * (step + 1);
    hd->pre_launches = 0;
    hd->trace.clear();
    if (timing) {
        float ms = 0.f;
        FMM_CUDA(hd, cudaEventElapsedTime(&ms, hd->events[0], hd->events[1]));
        hd->stats.march_ms = ms;
    }
    hd->solved = true;
    hd->complete = c.done && c.error == 0 && !timed_out && !limited;
    hd->fwd_ctrl = c;
    if (timed_out)
        return fail(hd, FMM_ERR_TIMEOUT, "the solve exceeded its wall-clock limit (timeout_s)");
    if (limited)
        return fail(hd, FMM_ERR_TIMEOUT, "the step limit (max_restarts) was reached before termination");
    return FMM_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Checkpoint image: this header, then T, tags, the tape (if recorded), the
// per-brick BAND minima, the change masks and the dirty flags (the brick
// layout of the device), then the control block the forward solve ended with.
struct CkptHeader {
    char magic[8];
    int32_t version;
    int32_t dtype;
    int64_t nx, ny, nz;
    double h, hy, hz;
    int32_t record_tape;
    int32_t hetero;
    int32_t resumable;
    int32_t complete;
    int64_t bytes;
};
constexpr char kCkptMagic[8] = {'F', 'M', 'M', 'C', 'K', 'P', 'T', '1'};
static_assert(sizeof(CkptHeader) == 88, "the header size fmm.h documents");

struct CkptSection {
    void *dev;
    size_t bytes;
};

std::vector<CkptSection> ckpt_sections(fmm_handle *hd)
{
    DeviceState &s = hd->st;
    const size_t nb = (size_t)hd->geom.nbricks, cells = nb * kB3;
    std::vector<CkptSection> v = {{s.T, cells * hd->rsize}, {s.tag, cells}};
    if (s.tape)
        v.push_back({s.tape, cells});
    v.push_back({s.bmin, 2 * nb * hd->rsize});
    v.push_back({s.fresh, nb * kFaces * sizeof(unsigned long long)});
    v.push_back({s.inmin, nb * 2 * sizeof(unsigned long long)});
    v.push_back({s.dirty, nb * sizeof(unsigned)});
    return v;
}

int64_t ckpt_bytes(fmm_handle *hd)
{
    size_t n = sizeof(CkptHeader) + sizeof(Control);
    for (const CkptSection &c : ckpt_sections(hd))
        n += c.bytes;
    return (int64_t)n;
}

void stats_from_control(fmm_handle *hd)
{
    const Control &c = hd->fwd_ctrl;
    hd->stats.restarts = c.restart;
    hd->stats.brick_marches = (int64_t)c.marches;
    hd->stats.march_rounds = (int64_t)c.rounds;
    hd->stats.exchanges = (int64_t)c.exchanges;
    hd->stats.accepted = (int64_t)c.accepted;
    hd->stats.cell_solves = (int64_t)c.solves;
    hd->stats.n_bricks = hd->geom.nbricks;
    hd->stats.error_flags = c.error;
}

}  // namespace

namespace fmmgb {
// The message fmm_last_error(NULL) returns on this thread (used by entry
// points that have no handle).
void set_create_error(const std::string &msg) { g_create_error = msg; }
}  // namespace fmmgb

extern "C" {

fmm_status fmm_create(const fmm_config *cfg, const void *speed, double speed_const,
                      const int64_t *src_ijk, int64_t n_src, fmm_handle **out)
{
    if (!out)
        return fail(nullptr, FMM_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    if (!cfg)
        return fail(nullptr, FMM_ERR_INVALID, "cfg must not be NULL");
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->nx > (1 << 20) || cfg->ny > (1 << 20) ||
        cfg->nz > (1 << 20))
        return fail(nullptr, FMM_ERR_INVALID, "grid sizes must be in [1, 2^20]");
    if (!(cfg->h > 0.0) || !std::isfinite(cfg->h))
        return fail(nullptr, FMM_ERR_INVALID, "h must be finite and > 0");
    if (!(cfg->hy >= 0.0) || !std::isfinite(cfg->hy) || !(cfg->hz >= 0.0) || !std::isfinite(cfg->hz))
        return fail(nullptr, FMM_ERR_INVALID, "hy and hz must be finite and >= 0 (0 -> h)");
    if (cfg->dtype != FMM_F32 && cfg->dtype != FMM_F64)
        return fail(nullptr, FMM_ERR_INVALID, "dtype must be FMM_F32 or FMM_F64");
    if (cfg->width < 0.0 || std::isnan(cfg->width) || cfg->stride < 0.0 || std::isnan(cfg->stride) ||
        cfg->bucket < 0.0 || std::isnan(cfg->bucket) || cfg->ahead < 0.0 || std::isnan(cfg->ahead))
        return fail(nullptr, FMM_ERR_INVALID, "width, stride, bucket and ahead must be >= 0");
    if (cfg->exchange_passes < 0 || cfg->exchange_passes > 64)
        return fail(nullptr, FMM_ERR_INVALID, "exchange_passes must be in [0, 64]");
    if (cfg->schedule < 0 || cfg->schedule > 4)
        return fail(nullptr, FMM_ERR_INVALID, "schedule must be 0, 1, 2, 3 or 4");
    if (cfg->deterministic != 0 && cfg->schedule != 0 && cfg->schedule != kSchedulePhased)
        return fail(nullptr, FMM_ERR_INVALID, "deterministic needs the phased schedule (schedule 0 or 1)");
    if (cfg->accuracy < 0 || cfg->accuracy > 2)
        return fail(nullptr, FMM_ERR_INVALID, "accuracy must be 0, 1 or 2");
    if (cfg->accuracy == 2 && cfg->schedule != 0 && cfg->schedule != kScheduleCell)
        return fail(nullptr, FMM_ERR_INVALID,
                    "the second-order march runs on the cell-parallel schedule (schedule 0 or 4)");
    if ((cfg->accuracy == 2 || cfg->schedule == kScheduleCell) && cfg->record_tape)
        return fail(nullptr, FMM_ERR_INVALID, "the cell-parallel schedule keeps no tape (record_tape must be 0)");
    if (cfg->accuracy == 2 && cfg->deterministic)
        return fail(nullptr, FMM_ERR_INVALID, "the second-order march has no deterministic mode (its "
                                              "results are reproducible without it)");
    if (n_src < 0 || (n_src > 0 && !src_ijk))
        return fail(nullptr, FMM_ERR_INVALID, "bad source list");
    if (speed && !aligned16(speed))
        return fail(nullptr, FMM_ERR_INVALID, "speed must be 16-byte aligned");
    for (int64_t i = 0; i < n_src; ++i) {
        const int64_t a = src_ijk[3 * i], b = src_ijk[3 * i + 1], c = src_ijk[3 * i + 2];
        if (a < 0 || a >= cfg->nx || b < 0 || b >= cfg->ny || c < 0 || c >= cfg->nz)
            return fail(nullptr, FMM_ERR_INVALID, "source cell outside the grid");
    }
    fmm_handle *hd = new (std::nothrow) fmm_handle();
    if (!hd)
        return fail(nullptr, FMM_ERR_OOM, "host allocation failed");
    hd->cfg = *cfg;
    hd->stream = (cudaStream_t)cfg->stream;
    hd->rsize = cfg->dtype == FMM_F64 ? 8 : 4;
    memset(&hd->stats, 0, sizeof(hd->stats));
    memset(&hd->st, 0, sizeof(hd->st));
    Geom &g = hd->geom;
    g.nx = (int)cfg->nx;
    g.ny = (int)cfg->ny;
    g.nz = (int)cfg->nz;
    g.nbx = (g.nx + kB - 1) / kB;
    g.nby = (g.ny + kB - 1) / kB;
    g.nbz = (g.nz + kB - 1) / kB;
    g.nbricks = (long long)g.nbx * g.nby * g.nbz;
    SolveParams &p = hd->params;
    set_spacing(p, cfg->h, cfg->hy, cfg->hz);
    p.width = cfg->width > 0.0 ? cfg->width : INFINITY;
    const double stride_h = cfg->stride > 0.0       ? cfg->stride
                            : cfg->deterministic ? default_stride_deterministic(cfg->dtype)
                                                 : default_stride(cfg->dtype);
    p.stride = stride_h * cfg->h;
    p.bucket = cfg->bucket > 0.0 ? cfg->bucket : cfg->accuracy == 2 ? kSecondOrderBucket : kDefaultBucket;
    p.passes = cfg->exchange_passes > 0 ? cfg->exchange_passes : default_passes(cfg->dtype);
    p.schedule = cfg->schedule == kSchedulePhased || cfg->deterministic ? kSchedulePhased
                 : cfg->schedule == kSchedulePersistent                 ? kSchedulePersistent
                 : cfg->schedule == kScheduleCell || cfg->accuracy == 2 ? kScheduleCell
                                                                        : kScheduleContinuous;
    p.accuracy = cfg->accuracy == 2 ? 2 : 1;
    p.max_restarts = cfg->max_restarts > 0 ? cfg->max_restarts : 0;
    p.max_rounds = 1 << 22;
    p.max_lead = cfg->max_lead > 0 ? (double)cfg->max_lead : default_max_lead();
    p.ahead = (cfg->ahead > 0.0 ? cfg->ahead : default_ahead(cfg->dtype)) * p.h;
    p.wait_ns = 1000000ull * (unsigned long long)(cfg->wait_limit_ms > 0 ? cfg->wait_limit_ms : 4000);
    p.hold = cfg->hold_queue != 0;

    auto bail = [&](fmm_status code) {
        g_create_error = hd->err;
        free_state(hd);
        delete hd;
        return code;
    };
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return bail(cuda_fail(hd, e, "cudaGetDevice"));
    DeviceState &s = hd->st;
    const size_t nb = (size_t)g.nbricks, cells = nb * kB3;
#define ALLOC(ptr, bytes)                                          \
    do {                                                           \
        cudaError_t e2 = alloc(&(ptr), (bytes));                   \
        if (e2 != cudaSuccess)                                     \
            return bail(cuda_fail(hd, e2, "cudaMalloc " #ptr));     \
    } while (0)
    ALLOC(s.T, cells * hd->rsize);
    ALLOC(s.tag, cells);
    ALLOC(s.bdelta, nb * hd->rsize);
    ALLOC(s.bmin, 2 * nb * hd->rsize);
    ALLOC(s.fresh, nb * kFaces * sizeof(unsigned long long));
    ALLOC(s.inmin, nb * 2 * sizeof(unsigned long long));
    ALLOC(s.inbox, nb * kFaces * sizeof(unsigned long long));
    ALLOC(s.dirty, nb * sizeof(unsigned));
    ALLOC(s.list[0], nb * sizeof(int));
    ALLOC(s.list[1], nb * sizeof(int));
    ALLOC(s.queue, nb * sizeof(unsigned long long));
    ALLOC(s.queued, nb * sizeof(unsigned));
    ALLOC(s.ctrl, sizeof(Control));
    if (cfg->record_tape)
        ALLOC(s.tape, cells);
    if (cfg->deterministic)
        ALLOC(s.faces, nb * kFaces * 64 * hd->rsize);
    if (n_src > 0) {
        ALLOC(hd->d_src, (size_t)n_src * 3 * sizeof(long long));
        e = cudaMemcpy(hd->d_src, src_ijk, (size_t)n_src * 3 * sizeof(long long), cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return bail(cuda_fail(hd, e, "cudaMemcpy sources"));
    }
#undef ALLOC
    hd->n_src = n_src;
    e = cudaMallocHost((void **)&hd->h_ctrl, sizeof(Control));
    if (e != cudaSuccess)
        return bail(cuda_fail(hd, e, "cudaMallocHost"));
    const int per_sm = march_blocks_per_sm(cfg->dtype, cfg->record_tape != 0);
    s.march_ctas = cfg->ctas > 0 ? cfg->ctas : sms * per_sm;
    hd->params.raise_at = raise_threshold(s.march_ctas);
    fmm_status rc = load_speed(hd, speed, speed_const);
    if (rc != FMM_OK)
        return bail(rc);
    *out = hd;
    return FMM_OK;
}

fmm_status fmm_set_speed(fmm_handle *hd, const void *speed, double speed_const)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (speed && !aligned16(speed))
        return fail(hd, FMM_ERR_INVALID, "speed must be 16-byte aligned");
    return load_speed(hd, speed, speed_const);
}

fmm_status fmm_solve(fmm_handle *hd, void *T_out, uint8_t *tags_out)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (!T_out || !aligned16(T_out))
        return fail(hd, FMM_ERR_INVALID, "T_out must be a 16-byte aligned pointer");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "a batch handle solves with fmm_reinit_batch");
    FMM_CUDA(hd, launch_init_sources(hd->cfg.dtype, hd->geom, hd->st, hd->d_src, hd->n_src, hd->stream));
    hd->pre_launches = hd->n_src > 0 ? 2 : 1;
    return run_solve(hd, T_out, tags_out);
}

fmm_status fmm_reinit_signed_distance(fmm_handle *hd, const void *phi0, void *T_out,
                                      uint8_t *tags_out)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (!phi0 || !aligned16(phi0))
        return fail(hd, FMM_ERR_INVALID, "phi0 must be a 16-byte aligned pointer");
    if (!T_out || !aligned16(T_out))
        return fail(hd, FMM_ERR_INVALID, "T_out must be a 16-byte aligned pointer");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "a batch handle solves with fmm_reinit_batch");
    const fmm_status r = device_input(hd, phi0, 0, &phi0);
    if (r != FMM_OK)
        return r;
    FMM_CUDA(hd, launch_init_reinit(hd->cfg.dtype, hd->geom, hd->st, hd->params, phi0, hd->stream));
    hd->pre_launches = 1;
    return run_solve(hd, T_out, tags_out);
}

fmm_status fmm_solve_fixed(fmm_handle *hd, const void *T0, void *T_out, uint8_t *tags_out)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (!T0 || !aligned16(T0))
        return fail(hd, FMM_ERR_INVALID, "T0 must be a 16-byte aligned pointer");
    if (!T_out || !aligned16(T_out))
        return fail(hd, FMM_ERR_INVALID, "T_out must be a 16-byte aligned pointer");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "a batch handle solves with fmm_solve_batch");
    const fmm_status r = device_input(hd, T0, 0, &T0);
    if (r != FMM_OK)
        return r;
    DeviceState &s = hd->st;
    FMM_CUDA(hd, launch_reset_control(s, hd->stream, hd->params.wait_ns, hd->params.hold));
    FMM_CUDA(hd, launch_init_fixed(hd->cfg.dtype, hd->geom, s, T0, hd->stream));
    FMM_CUDA(hd, cudaMemcpyAsync(hd->h_ctrl, s.ctrl, sizeof(Control), cudaMemcpyDeviceToHost, hd->stream));
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    if (hd->h_ctrl->error & ERR_INPUT) {
        hd->solved = hd->tape_valid = hd->resumable = hd->complete = false;
        return fail(hd, FMM_ERR_INVALID,
                    "T0 holds a NaN, or a sign change between two cells that are not both finite");
    }
    hd->pre_launches = 2;
    return run_solve(hd, T_out, tags_out);
}

fmm_status fmm_adjoint(fmm_handle *hd, const void *dL_dT, void *dL_dslowness)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (!dL_dT || !dL_dslowness)
        return fail(hd, FMM_ERR_INVALID, "dL_dT and dL_dslowness must not be NULL");
    if (!hd->solved || !hd->tape_valid)
        return fail(hd, FMM_ERR_STATE, "fmm_adjoint needs a solve with record_tape = 1 first");
    if (!aligned16(dL_dT) || !aligned16(dL_dslowness))
        return fail(hd, FMM_ERR_INVALID, "dL_dT and dL_dslowness must be 16-byte aligned");
    const Geom &g = hd->geom;
    DeviceState &s = hd->st;
    cudaStream_t st = hd->stream;
    const int dt = hd->cfg.dtype;
    if (!hd->adj_mu)
        FMM_CUDA(hd, alloc(&hd->adj_mu, (size_t)g.nbricks * kB3 * hd->rsize));
    if (!hd->adj_count)
        FMM_CUDA(hd, alloc(&hd->adj_count, sizeof(unsigned)));
    if (!hd->adj_top)
        FMM_CUDA(hd, alloc(&hd->adj_top, (size_t)g.nbricks * sizeof(unsigned long long)));
    const bool host_out = is_host(dL_dslowness);
    fmm_status r = device_input(hd, dL_dT, 0, &dL_dT);
    void *dlds = dL_dslowness;
    if (r == FMM_OK && host_out)
        r = stage_buffer(hd, 1, &dlds);
    if (r != FMM_OK)
        return r;
    AdjointArgs a;
    a.dLdT = dL_dT;
    a.dlds = dlds;
    a.mu = hd->adj_mu;
    a.h = hd->params.h;
    a.spd_term = hd->params.spd_term;
    a.wy = hd->params.wy;
    a.wz = hd->params.wz;
    a.aniso = hd->params.aniso;
    a.top = hd->adj_top;
    a.ctrl = s.ctrl;
    // every cell becomes ready once its downwind neighbours have published;
    // one persistent launch processes bricks until none is queued
    hd->resumable = false;   // the adjoint reuses the control block and the flags
    FMM_CUDA(hd, launch_reset_control(s, st, hd->params.wait_ns, hd->params.hold));
    FMM_CUDA(hd, cudaMemsetAsync(s.dirty, 0, (size_t)g.nbricks * sizeof(unsigned), st));
    FMM_CUDA(hd, launch_adjoint_init(dt, g, s, a, st));
    // levels of the reverse sweep, from the largest |psi| down (a brick
    // starts when the level reaches the largest |psi| it still has to do)
    double top_max = 0.0;
    FMM_CUDA(hd, adjoint_top_max(dt, g, a, &top_max, st));
    FMM_CUDA(hd, launch_reset_control(s, st, hd->params.wait_ns, hd->params.hold));
    const double step = kAdjointLevelStep * hd->params.h;
    long long levels = (top_max > 0.0 && step > 0.0) ? (long long)std::ceil(top_max / step) + 1 : 1;
    if (levels > kAdjointMaxLevels)
        levels = kAdjointMaxLevels;
    FMM_CUDA(hd, launch_adjoint_levels(dt, g, s, a, top_max, top_max / (double)(levels > 1 ? levels - 1 : 1),
                                       (int)levels, st));
    if (host_out)
        FMM_CUDA(hd, cudaMemcpyAsync(dL_dslowness, dlds, natural_cells(hd) * hd->rsize,
                                     cudaMemcpyDeviceToHost, st));
    FMM_CUDA(hd, cudaMemcpyAsync(hd->h_ctrl, s.ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    FMM_CUDA(hd, cudaMemsetAsync(hd->adj_count, 0, sizeof(unsigned), st));
    FMM_CUDA(hd, launch_adjoint_pending(dt, g, a, hd->adj_count, st));
    unsigned left = 0;
    FMM_CUDA(hd, cudaMemcpyAsync(&left, hd->adj_count, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    FMM_CUDA(hd, cudaStreamSynchronize(st));
    hd->stats.adjoint_iterations = (int64_t)hd->h_ctrl->marches;
    if (hd->h_ctrl->error & ERR_SPIN)
        return fail(hd, FMM_ERR_TIMEOUT, "adjoint: a device wait exceeded its time limit");
    if (left != 0)
        return fail(hd, FMM_ERR_STATE, "adjoint: some accepted cells could not be ordered");
    return FMM_OK;
}

fmm_status fmm_resume(fmm_handle *hd, int64_t more_restarts, void *T_out, uint8_t *tags_out)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (!T_out || !aligned16(T_out))
        return fail(hd, FMM_ERR_INVALID, "T_out must be a 16-byte aligned pointer");
    if (more_restarts < 0)
        return fail(hd, FMM_ERR_INVALID, "more_restarts must be >= 0");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "a batch handle cannot resume");
    if (!hd->resumable)
        return fail(hd, FMM_ERR_STATE,
                    "fmm_resume needs a solve stopped by its restart or time limit "
                    "(or a loaded checkpoint of one)");
    // the control block as the forward solve left it
    Control &c = *hd->h_ctrl;
    c = hd->fwd_ctrl;
    c.done = 0;
    c.error = 0;
    const long long keep = hd->params.max_restarts;
    hd->params.max_restarts = more_restarts > 0 ? (long long)c.restart + more_restarts : 0;
    hd->resumable = false;
    hd->pre_launches = 0;
    cudaError_t e = cudaMemcpyAsync(hd->st.ctrl, hd->h_ctrl, sizeof(Control), cudaMemcpyHostToDevice,
                                    hd->stream);
    if (e == cudaSuccess && hd->st.faces)
        e = launch_faces_build(hd->cfg.dtype, hd->geom, hd->st, hd->stream);   // from the stopped state
    if (e != cudaSuccess) {
        hd->params.max_restarts = keep;
        return cuda_fail(hd, e, "fmm_resume: control block");
    }
    const fmm_status r = run_restarts(hd, T_out, tags_out, 0);
    hd->params.max_restarts = keep;
    return r;
}

// ---------------------------------------------------------------------------
// Domain decomposition (Sec. 4.1, Algorithms 13-16 across processes): the
// handle's grid is one rank's subdomain with its ghost layers; the caller
// runs the loop of Algorithm 16 and the exchanges between ranks.
// ---------------------------------------------------------------------------

namespace {

fmm_status dd_layers_ok(fmm_handle *hd, int64_t z0, int64_t nl, const void *buf)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "batch handles have no domain decomposition");
    if (!hd->dd_started)
        return fail(hd, FMM_ERR_STATE, "fmm_dd_start first");
    if (nl < 1 || z0 < 0 || z0 + nl > hd->geom.nz)
        return fail(hd, FMM_ERR_INVALID, "layers outside the grid");
    if (!buf || !aligned16(buf) || is_host(buf))
        return fail(hd, FMM_ERR_INVALID, "layer buffers must be 16-byte aligned device memory");
    return FMM_OK;
}

}  // namespace

fmm_status fmm_dd_start(fmm_handle *hd, const void *phi0, int64_t extra_lo, int64_t extra_hi)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "batch handles have no domain decomposition");
    if (hd->st.faces)
        return fail(hd, FMM_ERR_STATE, "the fmm_dd_* entry points have no deterministic mode");
    if (hd->params.schedule == kScheduleCell)
        return fail(hd, FMM_ERR_STATE, "the fmm_dd_* entry points run the brick march (not schedule 4)");
    if (phi0 && (!aligned16(phi0) || is_host(phi0)))
        return fail(hd, FMM_ERR_INVALID, "phi0 must be 16-byte aligned device memory");
    if (extra_lo < 0 || extra_lo > 1 || extra_hi < 0 || extra_hi > 1)
        return fail(hd, FMM_ERR_INVALID, "extra_lo and extra_hi must be 0 or 1");
    DeviceState &s = hd->st;
    const Geom &g = hd->geom;
    const int dt = hd->cfg.dtype;
    cudaStream_t st = hd->stream;
    if (!hd->dd_count)
        FMM_CUDA(hd, alloc(&hd->dd_count, sizeof(unsigned)));
    if (!hd->h_dd_count)
        FMM_CUDA(hd, cudaMallocHost((void **)&hd->h_dd_count, sizeof(unsigned)));
    if (phi0) {
        FMM_CUDA(hd, launch_init_reinit(dt, g, s, hd->params, phi0, st, (int)extra_lo, (int)extra_hi));
    } else {
        FMM_CUDA(hd, launch_init_sources(dt, g, s, hd->d_src, hd->n_src, st));
    }
    hd->solved = hd->tape_valid = hd->resumable = hd->complete = false;
    FMM_CUDA(hd, launch_reset_control(s, st, hd->params.wait_ns, hd->params.hold));
    FMM_CUDA(hd, cudaMemsetAsync(s.fresh, 0, (size_t)g.nbricks * kFaces * sizeof(unsigned long long), st));
    FMM_CUDA(hd, cudaMemsetAsync(s.inmin, 0xff, (size_t)g.nbricks * 2 * sizeof(unsigned long long), st));
    FMM_CUDA(hd, cudaMemsetAsync(s.dirty, 0, (size_t)g.nbricks * sizeof(unsigned), st));
    FMM_CUDA(hd, cudaMemsetAsync(s.queue, 0, (size_t)g.nbricks * sizeof(unsigned long long), st));
    FMM_CUDA(hd, cudaMemsetAsync(s.queued, 0, (size_t)g.nbricks * sizeof(unsigned), st));
    FMM_CUDA(hd, launch_front_init(dt, g, s, hd->params, st));
    FMM_CUDA(hd, cudaStreamSynchronize(st));
    hd->dd_started = true;
    return FMM_OK;
}

fmm_status fmm_dd_minima(fmm_handle *hd, double *minval)
{
    if (!hd || !minval)
        return fail(hd, FMM_ERR_INVALID, "handle and minval must not be NULL");
    if (!hd->dd_started)
        return fail(hd, FMM_ERR_STATE, "fmm_dd_start first");
    FMM_CUDA(hd, launch_minima(hd->cfg.dtype, hd->geom, hd->st, hd->stream));
    FMM_CUDA(hd, cudaMemcpyAsync(hd->h_ctrl, hd->st.ctrl, sizeof(Control), cudaMemcpyDeviceToHost,
                                 hd->stream));
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    for (int sd = 0; sd < 2; ++sd) {
        double v;
        const unsigned long long b = hd->h_ctrl->minbits[sd];
        memcpy(&v, &b, sizeof(v));
        minval[sd] = v < hd->params.width ? v : hd->params.width;
    }
    return FMM_OK;
}

fmm_status fmm_dd_march(fmm_handle *hd, const double *bound)
{
    if (!hd || !bound)
        return fail(hd, FMM_ERR_INVALID, "handle and bound must not be NULL");
    if (!hd->dd_started)
        return fail(hd, FMM_ERR_STATE, "fmm_dd_start first");
    if (std::isnan(bound[0]) || std::isnan(bound[1]) || bound[0] < 0.0 || bound[1] < 0.0)
        return fail(hd, FMM_ERR_INVALID, "bounds must be >= 0");
    const double b0 = bound[0] < hd->params.width ? bound[0] : hd->params.width;
    const double b1 = bound[1] < hd->params.width ? bound[1] : hd->params.width;
    FMM_CUDA(hd, launch_march_to(hd->cfg.dtype, hd->geom, hd->st, hd->params, b0, b1, hd->stream));
    FMM_CUDA(hd, cudaMemcpyAsync(hd->h_ctrl, hd->st.ctrl, sizeof(Control), cudaMemcpyDeviceToHost,
                                 hd->stream));
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    if (hd->h_ctrl->error & (ERR_SPIN | ERR_ROUNDS))
        return fail(hd, FMM_ERR_TIMEOUT, "a march exceeded its round or wait limit");
    return FMM_OK;
}

fmm_status fmm_dd_get_layers(fmm_handle *hd, int64_t z0, int64_t nl, void *out)
{
    const fmm_status r = dd_layers_ok(hd, z0, nl, out);
    if (r != FMM_OK)
        return r;
    FMM_CUDA(hd, launch_layer_export(hd->cfg.dtype, hd->geom, hd->st, (int)z0, (int)nl, out, hd->stream));
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    return FMM_OK;
}

fmm_status fmm_dd_integrate(fmm_handle *hd, int64_t z0, int64_t nl, const void *in, int64_t *n_replaced)
{
    const fmm_status r = dd_layers_ok(hd, z0, nl, in);
    if (r != FMM_OK)
        return r;
    FMM_CUDA(hd, cudaMemsetAsync(hd->dd_count, 0, sizeof(unsigned), hd->stream));
    FMM_CUDA(hd, launch_layer_integrate(hd->cfg.dtype, hd->geom, hd->st, (int)z0, (int)nl, in,
                                        hd->dd_count, hd->stream));
    FMM_CUDA(hd, cudaMemcpyAsync(hd->h_dd_count, hd->dd_count, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                 hd->stream));
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    if (n_replaced)
        *n_replaced = (int64_t)*hd->h_dd_count;
    return FMM_OK;
}

fmm_status fmm_dd_finish(fmm_handle *hd, void *T_out, uint8_t *tags_out)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (!hd->dd_started)
        return fail(hd, FMM_ERR_STATE, "fmm_dd_start first");
    if (!T_out || !aligned16(T_out) || is_host(T_out) || (tags_out && is_host(tags_out)))
        return fail(hd, FMM_ERR_INVALID, "T_out (and tags_out) must be device memory, T_out 16-byte aligned");
    FMM_CUDA(hd, launch_output(hd->cfg.dtype, hd->geom, hd->st, T_out, tags_out, hd->stream));
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    return FMM_OK;
}

fmm_status fmm_checkpoint_size(fmm_handle *hd, int64_t *bytes)
{
    if (!hd || !bytes)
        return fail(hd, FMM_ERR_INVALID, "handle and bytes must not be NULL");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "batch handles have no checkpoint");
    *bytes = ckpt_bytes(hd);
    return FMM_OK;
}

fmm_status fmm_checkpoint_save(fmm_handle *hd, void *host_buf, int64_t capacity)
{
    if (!hd || !host_buf)
        return fail(hd, FMM_ERR_INVALID, "handle and host_buf must not be NULL");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "batch handles have no checkpoint");
    const int64_t need = ckpt_bytes(hd);
    if (capacity < need)
        return fail(hd, FMM_ERR_INVALID, "host_buf is smaller than fmm_checkpoint_size");
    const bool complete = hd->solved && hd->complete;
    if (!complete && !hd->resumable)
        return fail(hd, FMM_ERR_STATE,
                    "a checkpoint needs a finished solve or one stopped by its restart or time limit");
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    CkptHeader hdr;
    memset(&hdr, 0, sizeof(hdr));
    memcpy(hdr.magic, kCkptMagic, sizeof(hdr.magic));
    hdr.version = 2;
    hdr.dtype = hd->cfg.dtype;
    hdr.nx = hd->geom.nx;
    hdr.ny = hd->geom.ny;
    hdr.nz = hd->geom.nz;
    hdr.h = hd->params.h;
    hdr.hy = hd->params.hy;
    hdr.hz = hd->params.hz;
    hdr.record_tape = hd->st.tape != nullptr;
    hdr.hetero = hd->st.spd != nullptr;
    hdr.resumable = hd->resumable;
    hdr.complete = complete;
    hdr.bytes = need;
    unsigned char *p = (unsigned char *)host_buf;
    memcpy(p, &hdr, sizeof(hdr));
    p += sizeof(hdr);
    for (const CkptSection &c : ckpt_sections(hd)) {
        FMM_CUDA(hd, cudaMemcpy(p, c.dev, c.bytes, cudaMemcpyDeviceToHost));
        p += c.bytes;
    }
    memcpy(p, &hd->fwd_ctrl, sizeof(Control));
    return FMM_OK;
}

fmm_status fmm_checkpoint_load(fmm_handle *hd, const void *host_buf, int64_t size)
{
    if (!hd || !host_buf)
        return fail(hd, FMM_ERR_INVALID, "handle and host_buf must not be NULL");
    if (hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "batch handles have no checkpoint");
    CkptHeader hdr;
    if (size < (int64_t)sizeof(hdr))
        return fail(hd, FMM_ERR_INVALID, "checkpoint too short");
    memcpy(&hdr, host_buf, sizeof(hdr));
    if (memcmp(hdr.magic, kCkptMagic, sizeof(hdr.magic)) != 0 || hdr.version != 2)
        return fail(hd, FMM_ERR_INVALID, "not a checkpoint of this library");
    if (hdr.dtype != hd->cfg.dtype || hdr.nx != hd->geom.nx || hdr.ny != hd->geom.ny ||
        hdr.nz != hd->geom.nz || hdr.h != hd->params.h || hdr.hy != hd->params.hy ||
        hdr.hz != hd->params.hz)
        return fail(hd, FMM_ERR_INVALID, "checkpoint grid or dtype differs from the handle's");
    if ((hdr.record_tape != 0) != (hd->st.tape != nullptr) || (hdr.hetero != 0) != (hd->st.spd != nullptr))
        return fail(hd, FMM_ERR_INVALID, "checkpoint record_tape or speed kind differs from the handle's");
    if (hdr.bytes != ckpt_bytes(hd) || size < hdr.bytes)
        return fail(hd, FMM_ERR_INVALID, "checkpoint size does not match the handle");
    FMM_CUDA(hd, cudaStreamSynchronize(hd->stream));
    const unsigned char *p = (const unsigned char *)host_buf + sizeof(hdr);
    for (const CkptSection &c : ckpt_sections(hd)) {
        FMM_CUDA(hd, cudaMemcpy(c.dev, p, c.bytes, cudaMemcpyHostToDevice));
        p += c.bytes;
    }
    memcpy(&hd->fwd_ctrl, p, sizeof(Control));
    // this process's wait limit and testing flag, not the saver's
    hd->fwd_ctrl.wait_ns = hd->params.wait_ns;
    hd->fwd_ctrl.hold = hd->params.hold;
    *hd->h_ctrl = hd->fwd_ctrl;
    FMM_CUDA(hd, cudaMemcpy(hd->st.ctrl, hd->h_ctrl, sizeof(Control), cudaMemcpyHostToDevice));
    // the queue is empty between restarts
    const Geom &g = hd->geom;
    FMM_CUDA(hd, cudaMemset(hd->st.queue, 0, (size_t)g.nbricks * sizeof(unsigned long long)));
    FMM_CUDA(hd, cudaMemset(hd->st.queued, 0, (size_t)g.nbricks * sizeof(unsigned)));
    hd->complete = hdr.complete != 0;
    hd->resumable = hdr.resumable != 0;
    hd->solved = hd->complete || hd->resumable;
    hd->tape_valid = hd->complete && hd->st.tape != nullptr;
    stats_from_control(hd);
    return FMM_OK;
}

fmm_status fmm_create_batch(int n_grids, const int64_t *dims, const double *h,
                            const fmm_config *cfg, fmm_handle **out)
{
    if (!out)
        return fail(nullptr, FMM_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    if (!cfg || !dims || !h || n_grids < 1)
        return fail(nullptr, FMM_ERR_INVALID, "need n_grids >= 1, dims, h and cfg");
    if (cfg->dtype != FMM_F32 && cfg->dtype != FMM_F64)
        return fail(nullptr, FMM_ERR_INVALID, "dtype must be FMM_F32 or FMM_F64");
    if (cfg->width < 0.0 || std::isnan(cfg->width) || cfg->stride < 0.0 || std::isnan(cfg->stride) ||
        cfg->bucket < 0.0 || std::isnan(cfg->bucket) || cfg->ahead < 0.0 || std::isnan(cfg->ahead) ||
        cfg->exchange_passes < 0 || cfg->exchange_passes > 64)
        return fail(nullptr, FMM_ERR_INVALID, "bad width, stride, bucket, ahead or exchange_passes");
    if (cfg->record_tape)
        return fail(nullptr, FMM_ERR_INVALID, "batches keep no tape (record_tape must be 0)");
    if (cfg->deterministic)
        return fail(nullptr, FMM_ERR_INVALID, "batches have no deterministic mode (deterministic must be 0)");
    if (cfg->schedule == kScheduleCell || cfg->accuracy == 2)
        return fail(nullptr, FMM_ERR_INVALID,
                    "batches run the brick schedules (schedule 4 and accuracy 2 are single-grid only)");
    if (cfg->hy != 0.0 || cfg->hz != 0.0)
        return fail(nullptr, FMM_ERR_INVALID, "batches use cubic cells (hy and hz must be 0)");
    std::vector<BatchGrid> grids((size_t)n_grids);
    long long total = 0;
    double hmin = INFINITY;
    for (int gi = 0; gi < n_grids; ++gi) {
        const int64_t nx = dims[3 * gi], ny = dims[3 * gi + 1], nz = dims[3 * gi + 2];
        if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
            return fail(nullptr, FMM_ERR_INVALID, "grid sizes must be in [1, 2^20]");
        if (!(h[gi] > 0.0) || !std::isfinite(h[gi]))
            return fail(nullptr, FMM_ERR_INVALID, "every h must be finite and > 0");
        BatchGrid &G = grids[gi];
        memset(&G, 0, sizeof(G));
        G.nx = (int)nx;
        G.ny = (int)ny;
        G.nz = (int)nz;
        G.nbx = (G.nx + kB - 1) / kB;
        G.nby = (G.ny + kB - 1) / kB;
        G.nbz = (G.nz + kB - 1) / kB;
        G.brick0 = total;
        G.h = h[gi];
        G.speed_const = 1.0;
        total += (long long)G.nbx * G.nby * G.nbz;
        hmin = h[gi] < hmin ? h[gi] : hmin;
    }
    if (total >= (1LL << 31))
        return fail(nullptr, FMM_ERR_INVALID, "too many bricks in one batch");
    // grid of every brick and the neighbour table (no neighbour across grids)
    std::vector<int> bgrid((size_t)total), nbr((size_t)total * kFaces);
    for (int gi = 0; gi < n_grids; ++gi) {
        const BatchGrid &G = grids[gi];
        for (int bz = 0; bz < G.nbz; ++bz)
            for (int by = 0; by < G.nby; ++by)
                for (int bx = 0; bx < G.nbx; ++bx) {
                    const long long b = G.brick0 + ((long long)bz * G.nby + by) * G.nbx + bx;
                    bgrid[(size_t)b] = gi;
                    const int c[3] = {bx, by, bz}, e[3] = {G.nbx, G.nby, G.nbz};
                    for (int f = 0; f < kFaces; ++f) {
                        const int a = f >> 1, d = (f & 1) ? 1 : -1;
                        int q[3] = {bx, by, bz};
                        q[a] += d;
                        nbr[(size_t)b * kFaces + f] =
                            (q[a] < 0 || q[a] >= e[a])
                                ? -1
                                : (int)(G.brick0 + ((long long)q[2] * G.nby + q[1]) * G.nbx + q[0]);
                        (void)c;
                    }
                }
    }
    fmm_handle *hd = new (std::nothrow) fmm_handle();
    if (!hd)
        return fail(nullptr, FMM_ERR_OOM, "host allocation failed");
    hd->cfg = *cfg;
    hd->stream = (cudaStream_t)cfg->stream;
    hd->rsize = cfg->dtype == FMM_F64 ? 8 : 4;
    hd->n_grids = n_grids;
    memset(&hd->stats, 0, sizeof(hd->stats));
    memset(&hd->st, 0, sizeof(hd->st));
    Geom &g = hd->geom;
    memset(&g, 0, sizeof(g));
    g.nbricks = total;
    SolveParams &p = hd->params;
    set_spacing(p, hmin, 0.0, 0.0);
    p.accuracy = 1;
    p.width = cfg->width > 0.0 ? cfg->width : INFINITY;
    p.stride = (cfg->stride > 0.0 ? cfg->stride : default_stride(cfg->dtype)) * hmin;
    p.bucket = cfg->bucket > 0.0 ? cfg->bucket : kDefaultBucket;
    p.passes = cfg->exchange_passes > 0 ? cfg->exchange_passes : default_passes(cfg->dtype);
    p.schedule = cfg->schedule == kSchedulePhased      ? kSchedulePhased
                 : cfg->schedule == kSchedulePersistent ? kSchedulePersistent
                                                        : kScheduleContinuous;
    p.max_restarts = cfg->max_restarts > 0 ? cfg->max_restarts : 0;
    p.max_rounds = 1 << 22;
    p.max_lead = cfg->max_lead > 0 ? (double)cfg->max_lead : default_max_lead();
    p.ahead = (cfg->ahead > 0.0 ? cfg->ahead : default_ahead(cfg->dtype)) * p.h;
    p.wait_ns = 1000000ull * (unsigned long long)(cfg->wait_limit_ms > 0 ? cfg->wait_limit_ms : 4000);
    p.hold = cfg->hold_queue != 0;
    p.spd_term = 0.0;
    auto bail = [&](fmm_status code) {
        g_create_error = hd->err;
        free_state(hd);
        delete hd;
        return code;
    };
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return bail(cuda_fail(hd, e, "cudaGetDevice"));
    DeviceState &s = hd->st;
    const size_t nb = (size_t)total, cells = nb * kB3;
#define ALLOC(ptr, bytes)                                          \
    do {                                                           \
        cudaError_t e2 = alloc(&(ptr), (bytes));                   \
        if (e2 != cudaSuccess)                                     \
            return bail(cuda_fail(hd, e2, "cudaMalloc " #ptr));     \
    } while (0)
    ALLOC(s.T, cells * hd->rsize);
    ALLOC(s.tag, cells);
    ALLOC(s.spd, cells * hd->rsize);
    ALLOC(s.bdelta, nb * hd->rsize);
    ALLOC(s.bmin, 2 * nb * hd->rsize);
    ALLOC(s.fresh, nb * kFaces * sizeof(unsigned long long));
    ALLOC(s.inmin, nb * 2 * sizeof(unsigned long long));
    ALLOC(s.inbox, nb * kFaces * sizeof(unsigned long long));
    ALLOC(s.dirty, nb * sizeof(unsigned));
    ALLOC(s.list[0], nb * sizeof(int));
    ALLOC(s.list[1], nb * sizeof(int));
    ALLOC(s.queue, nb * sizeof(unsigned long long));
    ALLOC(s.queued, nb * sizeof(unsigned));
    ALLOC(s.ctrl, sizeof(Control));
    ALLOC(hd->d_nbr, nb * kFaces * sizeof(int));
    ALLOC(hd->d_bgrid, nb * sizeof(int));
    ALLOC(hd->d_grids, (size_t)n_grids * sizeof(BatchGrid));
#undef ALLOC
    e = cudaMallocHost((void **)&hd->h_ctrl, sizeof(Control));
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&hd->h_grids, (size_t)n_grids * sizeof(BatchGrid));
    if (e != cudaSuccess)
        return bail(cuda_fail(hd, e, "cudaMallocHost"));
    memcpy(hd->h_grids, grids.data(), (size_t)n_grids * sizeof(BatchGrid));
    s.nbr = hd->d_nbr;
    const int per_sm = march_blocks_per_sm(cfg->dtype, false);
    s.march_ctas = cfg->ctas > 0 ? cfg->ctas : sms * per_sm;
    hd->params.raise_at = raise_threshold(s.march_ctas);
    e = cudaMemcpy(hd->d_nbr, nbr.data(), nb * kFaces * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(hd->d_bgrid, bgrid.data(), nb * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(hd->d_grids, hd->h_grids, (size_t)n_grids * sizeof(BatchGrid),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_batch_speed(cfg->dtype, hd->d_grids, hd->d_bgrid, total, s, hd->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(hd->stream);
    if (e != cudaSuccess)
        return bail(cuda_fail(hd, e, "batch set-up"));
    *out = hd;
    return FMM_OK;
}

fmm_status fmm_solve_batch(fmm_handle *hd, const void *const *phi0, const int64_t *const *src_ijk,
                           const int64_t *n_src, const void *const *speed, const double *speed_const,
                           void *const *T_out, uint8_t *const *tags_out)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (!hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "fmm_solve_batch needs a handle from fmm_create_batch");
    if (!T_out)
        return fail(hd, FMM_ERR_INVALID, "T_out must be an array of device pointers");
    const int ng = hd->n_grids;
    // per-grid problem: a level set, or point sources
    long long total_src = 0;
    bool any_speed = false;
    for (int gi = 0; gi < ng; ++gi) {
        const BatchGrid &G = hd->h_grids[gi];
        const void *ph = phi0 ? phi0[gi] : nullptr;
        const long long ns = (!ph && n_src) ? (long long)n_src[gi] : 0;
        if (!T_out[gi] || !aligned16(T_out[gi]) || (ph && !aligned16(ph)))
            return fail(hd, FMM_ERR_INVALID, "every phi0 and T_out must be 16-byte aligned");
        if (!ph && (ns < 0 || (ns > 0 && (!src_ijk || !src_ijk[gi]))))
            return fail(hd, FMM_ERR_INVALID, "a grid without phi0 needs its source list");
        for (long long q = 0; q < ns; ++q) {
            const int64_t *c = src_ijk[gi] + 3 * q;
            if (c[0] < 0 || c[0] >= G.nx || c[1] < 0 || c[1] >= G.ny || c[2] < 0 || c[2] >= G.nz)
                return fail(hd, FMM_ERR_INVALID, "source cell outside its grid");
        }
        const void *sp = speed ? speed[gi] : nullptr;
        if (sp && !aligned16(sp))
            return fail(hd, FMM_ERR_INVALID, "every speed must be 16-byte aligned");
        const double sc = speed_const ? speed_const[gi] : 1.0;
        if (!sp && !(sc > 0.0 && std::isfinite(sc)))
            return fail(hd, FMM_ERR_INVALID, "speed_const must be finite and > 0 where speed is NULL");
        any_speed = any_speed || sp || sc != 1.0;
        total_src += ns;
    }
    cudaStream_t st = hd->stream;
    const long long nb = hd->geom.nbricks;
    // the source lists, flattened with their grid index
    if (total_src > 0) {
        std::vector<long long> flat((size_t)total_src * 4);
        long long k = 0;
        for (int gi = 0; gi < ng; ++gi) {
            const long long ns = (!(phi0 && phi0[gi]) && n_src) ? (long long)n_src[gi] : 0;
            hd->h_grids[gi].src0 = k;
            hd->h_grids[gi].n_src = ns;
            for (long long q = 0; q < ns; ++q, ++k) {
                flat[(size_t)(4 * k)] = gi;
                for (int a = 0; a < 3; ++a)
                    flat[(size_t)(4 * k + 1 + a)] = src_ijk[gi][3 * q + a];
            }
        }
        if ((size_t)total_src > hd->bsrc_cap) {
            FMM_CUDA(hd, cudaStreamSynchronize(st));
            if (hd->d_bsrc)
                cudaFree(hd->d_bsrc);
            hd->d_bsrc = nullptr;
            hd->bsrc_cap = 0;
            FMM_CUDA(hd, alloc(&hd->d_bsrc, (size_t)total_src * 4 * sizeof(long long)));
            hd->bsrc_cap = (size_t)total_src;
        }
        FMM_CUDA(hd, cudaMemcpyAsync(hd->d_bsrc, flat.data(), flat.size() * sizeof(long long),
                                     cudaMemcpyHostToDevice, st));
        FMM_CUDA(hd, cudaStreamSynchronize(st));   // flat is a host temporary
    }
    for (int gi = 0; gi < ng; ++gi) {
        BatchGrid &G = hd->h_grids[gi];
        G.phi0 = phi0 ? phi0[gi] : nullptr;
        G.T_out = T_out[gi];
        G.tags_out = tags_out ? tags_out[gi] : nullptr;
        G.speed = speed ? speed[gi] : nullptr;
        G.speed_const = speed_const ? speed_const[gi] : 1.0;
        if (total_src == 0)
            G.src0 = G.n_src = 0;
    }
    FMM_CUDA(hd, cudaMemcpyAsync(hd->d_grids, hd->h_grids, (size_t)ng * sizeof(BatchGrid),
                                 cudaMemcpyHostToDevice, st));
    long long pre = 1;
    if (any_speed || !hd->batch_speed_const1) {
        // speed terms and bucket widths of every grid; a bad speed value is
        // reported before the solve starts
        FMM_CUDA(hd, launch_reset_control(hd->st, st, hd->params.wait_ns, hd->params.hold));
        FMM_CUDA(hd, launch_batch_speed(hd->cfg.dtype, hd->d_grids, hd->d_bgrid, nb, hd->st, st));
        FMM_CUDA(hd, cudaMemcpyAsync(hd->h_ctrl, hd->st.ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
        FMM_CUDA(hd, cudaStreamSynchronize(st));
        hd->batch_speed_const1 = !any_speed;
        pre += 2;
        if (hd->h_ctrl->error & ERR_SPEED)
            return fail(hd, FMM_ERR_INVALID, "speed values must be finite and >= 0");
    }
    FMM_CUDA(hd, launch_batch_init(hd->cfg.dtype, hd->d_grids, hd->d_bgrid, nb, hd->st, st));
    if (total_src > 0) {
        FMM_CUDA(hd, launch_batch_sources(hd->cfg.dtype, hd->d_grids, hd->d_bsrc, total_src, hd->st, st));
        pre += 1;
    }
    hd->pre_launches = pre;
    fmm_status rc = run_solve(hd, nullptr, nullptr);
    if (rc != FMM_OK)
        return rc;
    FMM_CUDA(hd, launch_batch_output(hd->cfg.dtype, hd->d_grids, hd->d_bgrid, nb, hd->st, st));
    FMM_CUDA(hd, cudaStreamSynchronize(st));
    hd->stats.kernel_launches += 1;
    return FMM_OK;
}

fmm_status fmm_reinit_batch(fmm_handle *hd, const void *const *phi0, void *const *T_out,
                            uint8_t *const *tags_out)
{
    if (!hd)
        return fail(nullptr, FMM_ERR_INVALID, "handle is NULL");
    if (!hd->n_grids)
        return fail(hd, FMM_ERR_STATE, "fmm_reinit_batch needs a handle from fmm_create_batch");
    if (!phi0 || !T_out)
        return fail(hd, FMM_ERR_INVALID, "phi0 and T_out must be arrays of device pointers");
    for (int gi = 0; gi < hd->n_grids; ++gi)
        if (!phi0[gi])
            return fail(hd, FMM_ERR_INVALID, "every phi0 must be a 16-byte aligned device pointer");
    return fmm_solve_batch(hd, phi0, nullptr, nullptr, nullptr, nullptr, T_out, tags_out);
}

fmm_status fmm_get_trace(const fmm_handle *hd, fmm_trace_entry *out, int64_t capacity,
                         int64_t *n_out)
{
    if (!hd || !n_out || capacity < 0 || (capacity > 0 && !out))
        return FMM_ERR_INVALID;
    *n_out = (int64_t)hd->trace.size();
    const size_t n = hd->trace.size() < (size_t)capacity ? hd->trace.size() : (size_t)capacity;
    for (size_t i = 0; i < n; ++i)
        out[i] = hd->trace[i];
    return FMM_OK;
}

fmm_status fmm_get_stats(const fmm_handle *hd, fmm_stats *out)
{
    if (!hd || !out)
        return FMM_ERR_INVALID;
    *out = hd->stats;
    return FMM_OK;
}

const char *fmm_last_error(const fmm_handle *hd)
{
    if (!hd)
        return g_create_error.c_str();
    return hd->err.c_str();
}

void fmm_destroy(fmm_handle *hd)
{
    if (!hd)
        return;
    if (hd->stream)
        cudaStreamSynchronize(hd->stream);
    else
        cudaDeviceSynchronize();
    free_state(hd);
    delete hd;
}

}  // extern "C"
