// fmm_noalloc.cu -- fmm_reinit_signed_distance_noalloc: the two-sided
// reinitialisation without any memory allocation.
//
// Some callers cannot allocate device memory at solve time: processes whose
// device memory is owned by a pool or arena that forbids further driver
// allocations (a framework's caching allocator that has reserved the whole
// device, an embedding application with a fixed memory budget), and
// latency-bound loops that must not pay for an allocation or risk an
// out-of-memory failure in the middle of a run.  For them this entry point
// keeps all of its workspace in one file-scope __device__ array of fixed size,
// which the module loader reserves on every device that loads the library and
// which stays reserved until the process exits.  The caller still passes phi0
// and the outputs.
//
// The host cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so on the first call on each device, with that
// device current, the address is looked up with cudaGetSymbolAddress and
// cached.  Later calls check the cached address with cudaPointerGetAttributes (which allocates
// nothing) and look it up again if the device's context was reset since.
// Every call on a device shares the same array, and the array keeps the
// previous call's contents; everything the solve reads before writing
// (exchange masks, dirty flags, queue, the control block) is cleared at the
// start of each call.  Two calls whose GPU work overlaps on the same device
// (for example on two streams) race on the array.
#include "fmm.h"
#include "fmm_internal.h"

#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace fmmgb {
void set_create_error(const std::string &msg);
}

using namespace fmmgb;

namespace {

// Largest grid: 512 bricks of 8^3 cells (for example 64^3, or 128x64x32).
constexpr long long kNoAllocMaxBricks = 512;
constexpr size_t kCells = (size_t)kNoAllocMaxBricks * kB3;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// layout of the scratch, sized for double precision
constexpr size_t kOffT = 0;
constexpr size_t kOffTag = align256(kOffT + kCells * sizeof(double));
constexpr size_t kOffBdelta = align256(kOffTag + kCells);
constexpr size_t kOffBmin = align256(kOffBdelta + kNoAllocMaxBricks * sizeof(double));
constexpr size_t kOffFresh = align256(kOffBmin + 2 * kNoAllocMaxBricks * sizeof(double));
constexpr size_t kOffInmin = align256(kOffFresh + kFaces * kNoAllocMaxBricks * sizeof(unsigned long long));
constexpr size_t kOffInbox = align256(kOffInmin + 2 * kNoAllocMaxBricks * sizeof(unsigned long long));
constexpr size_t kOffDirty = align256(kOffInbox + kFaces * kNoAllocMaxBricks * sizeof(unsigned long long));
constexpr size_t kOffList0 = align256(kOffDirty + kNoAllocMaxBricks * sizeof(unsigned));
constexpr size_t kOffList1 = align256(kOffList0 + kNoAllocMaxBricks * sizeof(int));
constexpr size_t kOffQueue = align256(kOffList1 + kNoAllocMaxBricks * sizeof(int));
constexpr size_t kOffQueued = align256(kOffQueue + kNoAllocMaxBricks * sizeof(unsigned long long));
constexpr size_t kOffCtrl = align256(kOffQueued + kNoAllocMaxBricks * sizeof(unsigned));
constexpr size_t kScratchBytes = align256(kOffCtrl + sizeof(Control));   // about 2.4 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

fmm_status error(fmm_status code, const std::string &msg)
{
    set_create_error(msg);
    return code;
}

fmm_status cuda_error(cudaError_t e, const char *where)
{
    return error(FMM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device address of the scratch on the current device, looked up on the
// first call on a device and cached.  A cached address that no longer names device memory of this
// device (the context was reset with cudaDeviceReset, which unloads and
// reloads the module) is looked up again.
fmm_status scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return error(FMM_ERR_INVALID, "device ordinal out of range for the no-allocation entry point");
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[dev]) {
        cudaPointerAttributes a;
        const cudaError_t e = cudaPointerGetAttributes(&a, g_addr[dev]);
        if (e != cudaSuccess || a.type != cudaMemoryTypeDevice || a.device != dev ||
            a.devicePointer != g_addr[dev]) {
            cudaGetLastError();   // clear the error of an unknown pointer
            g_addr[dev] = nullptr;
        }
    }
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return FMM_OK;
}

}  // namespace

extern "C" fmm_status fmm_reinit_signed_distance_noalloc(const fmm_config *cfg, const void *phi0,
                                                         void *T_out, uint8_t *tags_out)
{
    if (!cfg)
        return error(FMM_ERR_INVALID, "cfg must not be NULL");
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->nx > (1 << 20) || cfg->ny > (1 << 20) ||
        cfg->nz > (1 << 20))
        return error(FMM_ERR_INVALID, "grid sizes must be in [1, 2^20]");
    if (!(cfg->h > 0.0) || !std::isfinite(cfg->h))
        return error(FMM_ERR_INVALID, "h must be finite and > 0");
    if (!(cfg->hy >= 0.0) || !std::isfinite(cfg->hy) || !(cfg->hz >= 0.0) || !std::isfinite(cfg->hz))
        return error(FMM_ERR_INVALID, "hy and hz must be finite and >= 0 (0 -> h)");
    if (cfg->dtype != FMM_F32 && cfg->dtype != FMM_F64)
        return error(FMM_ERR_INVALID, "dtype must be FMM_F32 or FMM_F64");
    if (cfg->width < 0.0 || std::isnan(cfg->width) || cfg->stride < 0.0 || std::isnan(cfg->stride) ||
        cfg->bucket < 0.0 || std::isnan(cfg->bucket) || cfg->ahead < 0.0 || std::isnan(cfg->ahead))
        return error(FMM_ERR_INVALID, "width, stride, bucket and ahead must be >= 0");
    if (cfg->exchange_passes < 0 || cfg->exchange_passes > 64)
        return error(FMM_ERR_INVALID, "exchange_passes must be in [0, 64]");
    if (cfg->schedule < 0 || cfg->schedule > 3)
        return error(FMM_ERR_INVALID, "schedule must be 0, 1, 2 or 3");
    if (cfg->record_tape)
        return error(FMM_ERR_INVALID, "the no-allocation entry point keeps no tape (record_tape must be 0)");
    if (cfg->deterministic)
        return error(FMM_ERR_INVALID, "the no-allocation entry point has no deterministic mode");
    if (cfg->accuracy != 0 && cfg->accuracy != 1)
        return error(FMM_ERR_INVALID, "the no-allocation entry point runs the first-order march (accuracy 0 or 1)");
    if (!phi0 || ((uintptr_t)phi0 & 15u) || !T_out || ((uintptr_t)T_out & 15u))
        return error(FMM_ERR_INVALID, "phi0 and T_out must be 16-byte aligned device pointers");
    Geom g;
    g.nx = (int)cfg->nx;
    g.ny = (int)cfg->ny;
    g.nz = (int)cfg->nz;
    g.nbx = (g.nx + kB - 1) / kB;
    g.nby = (g.ny + kB - 1) / kB;
    g.nbz = (g.nz + kB - 1) / kB;
    g.nbricks = (long long)g.nbx * g.nby * g.nbz;
    if (g.nbricks > kNoAllocMaxBricks)
        return error(FMM_ERR_INVALID,
                     "grid too large for fmm_reinit_signed_distance_noalloc: at most 512 bricks of "
                     "8x8x8 cells (for example 64^3); use fmm_create for larger grids");

    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_error(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return cuda_error(e, "cudaDeviceGetAttribute");
    unsigned char *base = nullptr;
    fmm_status rc = scratch_address(dev, &base);
    if (rc != FMM_OK)
        return rc;

    DeviceState s;
    memset(&s, 0, sizeof(s));
    s.T = base + kOffT;
    s.tag = base + kOffTag;
    s.bdelta = base + kOffBdelta;
    s.bmin = base + kOffBmin;
    s.fresh = (unsigned long long *)(base + kOffFresh);
    s.inmin = (unsigned long long *)(base + kOffInmin);
    s.inbox = (unsigned long long *)(base + kOffInbox);
    s.dirty = (unsigned *)(base + kOffDirty);
    s.list[0] = (int *)(base + kOffList0);
    s.list[1] = (int *)(base + kOffList1);
    s.queue = (unsigned long long *)(base + kOffQueue);
    s.queued = (unsigned *)(base + kOffQueued);
    s.ctrl = (Control *)(base + kOffCtrl);
    s.spd = nullptr;
    s.tape = nullptr;
    const int per_sm = march_blocks_per_sm(cfg->dtype, false);
    s.march_ctas = cfg->ctas > 0 ? cfg->ctas : sms * per_sm;

    SolveParams p;
    memset(&p, 0, sizeof(p));
    set_spacing(p, cfg->h, cfg->hy, cfg->hz);
    p.width = cfg->width > 0.0 ? cfg->width : INFINITY;
    p.stride = (cfg->stride > 0.0 ? cfg->stride : default_stride(cfg->dtype)) * cfg->h;
    p.bucket = cfg->bucket > 0.0 ? cfg->bucket : kDefaultBucket;
    p.passes = cfg->exchange_passes > 0 ? cfg->exchange_passes : default_passes(cfg->dtype);
    p.schedule = cfg->schedule == kSchedulePhased      ? kSchedulePhased
                 : cfg->schedule == kSchedulePersistent ? kSchedulePersistent
                                                        : kScheduleContinuous;
    p.accuracy = 1;
    p.max_restarts = cfg->max_restarts > 0 ? cfg->max_restarts : 0;
    p.max_rounds = 1 << 22;
    p.max_lead = cfg->max_lead > 0 ? (double)cfg->max_lead : default_max_lead();
    p.ahead = (cfg->ahead > 0.0 ? cfg->ahead : default_ahead(cfg->dtype)) * cfg->h;
    p.wait_ns = 1000000ull * (unsigned long long)(cfg->wait_limit_ms > 0 ? cfg->wait_limit_ms : 4000);
    p.hold = cfg->hold_queue != 0;
    p.raise_at = raise_threshold(s.march_ctas);
    if (cfg->dtype == FMM_F64) {
        p.spd_term = cfg->h * cfg->h;   // (h/F)^2 with F = 1
    } else {
        const float hf = (float)cfg->h;
        p.spd_term = (double)(hf * hf);   // (h/F)^2 with F = 1
    }

    cudaStream_t st = (cudaStream_t)cfg->stream;
    const int dt = cfg->dtype;
#define NA_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess)                          \
            return cuda_error(e_, #call);               \
    } while (0)
    // clear what the solve reads before it writes
    NA_CUDA(launch_reset_control(s, st, p.wait_ns, p.hold));
    NA_CUDA(cudaMemsetAsync(s.fresh, 0, (size_t)g.nbricks * kFaces * sizeof(unsigned long long), st));
    NA_CUDA(cudaMemsetAsync(s.inmin, 0xff, (size_t)g.nbricks * 2 * sizeof(unsigned long long), st));
    NA_CUDA(cudaMemsetAsync(s.dirty, 0, (size_t)g.nbricks * sizeof(unsigned), st));
    NA_CUDA(cudaMemsetAsync(s.queue, 0, (size_t)g.nbricks * sizeof(unsigned long long), st));
    NA_CUDA(cudaMemsetAsync(s.queued, 0, (size_t)g.nbricks * sizeof(unsigned), st));
    NA_CUDA(launch_load_speed(dt, g, s, p.h, min_spacing(p), nullptr, 1.0, st));
    NA_CUDA(launch_init_reinit(dt, g, s, p, phi0, st));
    NA_CUDA(launch_front_init(dt, g, s, p, st));
    // the loop of Algorithm 16; the control block is read back into a
    // stack variable between batches of restarts
    Control c;
    const double limit_s = cfg->timeout_s > 0 ? (double)cfg->timeout_s : 600.0;
    const auto t0 = std::chrono::steady_clock::now();
    long long batch = 1;
    for (;;) {
        for (long long r = 0; r < batch; ++r)
            NA_CUDA(launch_restart(dt, g, s, p, st, nullptr, nullptr));
        NA_CUDA(cudaMemcpyAsync(&c, s.ctrl, sizeof(Control), cudaMemcpyDeviceToHost, st));
        NA_CUDA(cudaStreamSynchronize(st));
        if (c.done)
            break;
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit_s)
            return error(FMM_ERR_TIMEOUT, "the solve exceeded its wall-clock limit (timeout_s)");
        if (batch < 16)
            batch *= 2;
    }
    NA_CUDA(launch_output(dt, g, s, T_out, tags_out, st));
    NA_CUDA(cudaStreamSynchronize(st));
#undef NA_CUDA
    if (c.error & ERR_ROUNDS)
        return error(FMM_ERR_TIMEOUT, "a brick march exceeded its round limit");
    if (c.error & ERR_RESTARTS)
        return error(FMM_ERR_TIMEOUT, "the restart limit was reached before termination");
    if (c.error & ERR_SPIN)
        return error(FMM_ERR_TIMEOUT, "a bounded wait of the persistent march gave up");
    return FMM_OK;
}
