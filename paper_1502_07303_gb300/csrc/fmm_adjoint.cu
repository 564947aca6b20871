// fmm_adjoint.cu -- reverse-mode derivative of a loss L(psi) with respect to
// the slowness s = 1/F, on the GPU, about a finished forward solve.
//
// The adjoint is not part of the paper; it is derived from the discrete
// Eq. (2).  At an accepted non-FIX cell p with final upwind set U(p) (the
// tape written by the forward march), sum_{i in U(p)} ((T_p - T_i)/h)^2 =
// s_p^2, so with D_p = sum_{i in U(p)} (T_p - T_i):
//     dT_p/ds_p = s_p h^2 / D_p,   dT_p/dT_i = (T_p - T_i) / D_p.
// The adjoint lambda_p = dL/dT_p + sum over the downwind cells q of p (the
// cells with p in U(q)) of lambda_q (T_q - T_p) / D_q, and dL/ds_p =
// lambda_p s_p h^2 / D_p.  FIX cells and cells that were not accepted get 0.
//
// GPU formulation (pull, no atomics on values): every cell publishes
// mu_p = lambda_p / D_p once it is done, with NaN meaning "not yet".  A cell
// is ready when all its downwind neighbours have published; then
// lambda_p = g_p + sum_q mu_q (T_q - T_p).  One persistent launch takes
// bricks from the device-side queue of the forward path; a warp processes a
// brick in rounds over its cells that are not done yet (per-lane 16-bit
// masks; the cells that become ready in one step of a round are computed
// together); downwind neighbours in other bricks are read from their
// published mu.  A brick that finished boundary cells flags and queues the
// bricks holding their upwind neighbours; a brick that ends its pass while a
// flag arrived queues itself again.  The launch ends when no brick is queued
// or being processed.  The order of the sums is fixed, so the result is
// deterministic.
#include "fmm_internal.h"
#include "fmm_queue.cuh"
#include "fmm_fp64.cuh"
#include "fmm_lanes.cuh"

#include <cmath>
#include <cstring>
#include <type_traits>

namespace fmmgb {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kAdjWarps = 4;

__device__ __forceinline__ unsigned long long vloadu(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

template <typename real>
__device__ __forceinline__ real nan_v();
template <>
__device__ __forceinline__ float nan_v<float>() { return __int_as_float(0x7fffffff); }
template <>
__device__ __forceinline__ double nan_v<double>() { return __longlong_as_double(0x7fffffffffffffffll); }

__device__ __forceinline__ bool accepted(uint8_t tg) { return (tg & ST_MASK) == ST_KNOWN && !(tg & TG_OUT); }

__device__ __forceinline__ void brick_xyz(const Geom &g, long long b, int &bx, int &by, int &bz)
{
    bx = (int)(b % g.nbx);
    const long long r = b / g.nbx;
    by = (int)(r % g.nby);
    bz = (int)(r / g.nby);
}

// mu = NaN (not done) on accepted cells, 0 elsewhere; dL/ds = 0; and per
// brick the largest |psi| of a cell to do (top, the bits of a double; the
// caller zeroes it first).  A warp's 32 cells lie in one brick.
template <typename real>
__global__ void k_adj_init(Geom g, const real *__restrict__ T, const uint8_t *__restrict__ tag, real *mu,
                           real *dlds, unsigned long long *top)
{
    const long long n = g.nbricks * kB3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int bx, by, bz;
        brick_xyz(g, e >> 9, bx, by, bz);
        const int c = (int)(e & 511);
        const int i = bx * kB + (c & 7), j = by * kB + ((c >> 3) & 7), k = bz * kB + (c >> 6);
        const bool acc = accepted(tag[e]);
        mu[e] = acc ? nan_v<real>() : (real)0;
        if (i < g.nx && j < g.ny && k < g.nz)
            dlds[((long long)k * g.ny + j) * g.nx + i] = (real)0;
        const unsigned long long tb =
            acc ? (unsigned long long)__double_as_longlong((double)T[e]) : 0ull;
        // the warp maximum of the 64-bit patterns: high words first
        const unsigned hi = __reduce_max_sync(FULL, (unsigned)(tb >> 32));
        const unsigned lo = __reduce_max_sync(FULL, (unsigned)(tb >> 32) == hi ? (unsigned)tb : 0u);
        if ((threadIdx.x & 31) == 0 && (hi | lo))
            atomicMax(&top[e >> 9], ((unsigned long long)hi << 32) | lo);
    }
}

// The largest top over all bricks into *out.
__global__ void k_adj_top_max(long long nbricks, const unsigned long long *__restrict__ top,
                              unsigned long long *out)
{
    unsigned long long m = 0;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nbricks;
         b += (long long)gridDim.x * blockDim.x)
        m = top[b] > m ? top[b] : m;
    const unsigned hi = __reduce_max_sync(FULL, (unsigned)(m >> 32));
    const unsigned lo = __reduce_max_sync(FULL, (unsigned)(m >> 32) == hi ? (unsigned)m : 0u);
    if ((threadIdx.x & 31) == 0 && (hi | lo))
        atomicMax(out, ((unsigned long long)hi << 32) | lo);
}

// Between levels: the previous launch ended with the queue empty, but warps
// that found it empty took tickets; restart the ring's positions.
__global__ void k_adj_level_reset(Control *c)
{
    c->q_head = 0ull;
    c->q_tail = 0ull;
    c->pending = 0;
}

// A level of the reverse sweep: push every brick whose top lies in
// [lo, hi) (bit patterns of non-negative doubles; top 0 = nothing to do).
__global__ void k_adj_seed_level(Geom g, const unsigned long long *__restrict__ top,
                                 unsigned long long lo, unsigned long long hi, Control *ctrl,
                                 unsigned *queued, unsigned long long *q)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long cap = (unsigned long long)g.nbricks;
    for (long long b0 = blockIdx.x * (long long)blockDim.x; b0 < g.nbricks;
         b0 += (long long)gridDim.x * blockDim.x) {
        const long long b = b0 + threadIdx.x;
        bool sel = false;
        if (b < g.nbricks) {
            const unsigned long long t = top[b];
            sel = t != 0ull && t >= lo && t < hi && atomicCAS(&queued[b], 0u, 1u) == 0u;
        }
        const unsigned ball = __ballot_sync(FULL, sel);
        if (ball == 0u)
            continue;
        unsigned long long basepos = 0;
        if (lane == 0) {
            atomicAdd(&ctrl->pending, __popc(ball));
            basepos = atomicAdd(&ctrl->q_tail, (unsigned long long)__popc(ball));
        }
        basepos = __shfl_sync(FULL, basepos, 0);
        if (sel) {
            const unsigned long long t = basepos + __popc(ball & ((1u << lane) - 1u));
            q[t % cap] = ((t & 0xffffffffull) << 32) | (unsigned long long)(b + 1);
        }
    }
}

template <typename real>
struct AdjTile {
    real T[kTile3];      // |psi| of the brick and its face halo
    real mu[kTile3];     // published mu (NaN = not done) of brick and halo
    uint8_t tp[kTile3];  // tape of brick and halo
    uint16_t list[kB3];  // the cells found ready in a round, compacted
};

// Tape code of axis a of cell tp: 0 none, 1 minus neighbour, 2 plus.
__device__ __forceinline__ int tape_axis(uint8_t tp, int a) { return (tp >> (2 * a)) & 3; }

// NaN test and "> 0" for values that are >= 0 or NaN, on the bit patterns
// (integer compares keep them off the FP64 pipe)
__device__ __forceinline__ bool is_nan_bits(float v) { return (__float_as_uint(v) & 0x7fffffffu) > 0x7f800000u; }
__device__ __forceinline__ bool is_nan_bits(double v)
{
    return (__double_as_longlong(v) & 0x7fffffffffffffffll) > 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool positive(float v) { return __float_as_int(v) > 0; }
__device__ __forceinline__ bool positive(double v) { return __double_as_longlong(v) > 0; }

// a / b and sqrt(v) for the adjoint; in double, float seeds refined by
// Newton steps without the FP64 pipe's slow conversions (fmm_fp64.cuh).
__device__ __forceinline__ float adj_div(float a, float b) { return a / b; }
__device__ __forceinline__ double adj_div(double a, double b) { return div_fp64(a, b); }
__device__ __forceinline__ float adj_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double adj_sqrt(double v) { return sqrt_fp64(v); }

template <typename real, bool kHetero, bool kAniso>
__global__ void __launch_bounds__(kAdjWarps * 32)
    k_adj_persistent(Geom g, DeviceState s, const real *__restrict__ dLdT, real *dlds, real *mu_g,
                     unsigned long long *top, unsigned long long level, double h,
                     double spd_const_term, double wy, double wz)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    AdjTile<real> &W = reinterpret_cast<AdjTile<real> *>(smem_raw)[warp];
    Control *ctrl = s.ctrl;
    const real *T = (const real *)s.T;
    const real *spd = (const real *)s.spd;
    const unsigned long long cap = (unsigned long long)g.nbricks;
    const int off[3] = {1, kTile, kTile * kTile};
    const int lx = lane & 7, lr = (lane >> 3) & 3;
    const real sh2_const = (real)(sqrt(spd_const_term) * h);
    unsigned long long rounds_total = 0, passes = 0;
    for (;;) {
        long long b = -1;
        if (lane == 0) {
            b = queue_pop(ctrl, s.queue, cap);
            if (b >= 0)
                atomicExch(&s.dirty[b], 0u);   // the flags this pass answers
            __threadfence();
        }
        b = __shfl_sync(FULL, b, 0);
        if (b < 0)
            break;
        int bx, by, bz;
        brick_xyz(g, b, bx, by, bz);
        const long long base = b * kB3;
        // ---- stage T, mu, tape of the brick; cells still to do -------------
        unsigned todo = 0;
#pragma unroll 4
        for (int k = 0; k < 16; ++k) {
            const int c = lane + 32 * k;
            const int ti = tile_of(c);
            const uint8_t tg = s.tag[base + c];
            const real m = __ldcg(mu_g + base + c);
            W.T[ti] = T[base + c];
            W.mu[ti] = m;
            // cells that were not accepted have no upwind set
            W.tp[ti] = accepted(tg) ? s.tape[base + c] : (uint8_t)0;
            todo |= (unsigned)(accepted(tg) && is_nan_bits(m)) << k;
        }
        // ---- halo: the face layers of the six neighbours ------------------
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const int hh = lane + 32 * k;
            const int f = hh >> 6, q = hh & 63, u = q & 7, v = q >> 3;
            const int axis = f >> 1, dir = (f & 1) ? 1 : -1;
            const int nbx = bx + (axis == 0 ? dir : 0);
            const int nby = by + (axis == 1 ? dir : 0);
            const int nbz = bz + (axis == 2 ? dir : 0);
            real tv = (real)0, mv = (real)0;
            uint8_t tpv = 0;
            if (nbx >= 0 && nbx < g.nbx && nby >= 0 && nby < g.nby && nbz >= 0 && nbz < g.nbz) {
                const int edge = dir < 0 ? kB - 1 : 0;
                const int cx = axis == 0 ? edge : u;
                const int cy = axis == 1 ? edge : (axis == 0 ? u : v);
                const int cz = axis == 2 ? edge : v;
                const long long nb = ((long long)nbz * g.nby + nby) * g.nbx + nbx;
                const long long ci = nb * kB3 + cx + kB * cy + kB * kB * cz;
                tv = T[ci];
                mv = __ldcg(mu_g + ci);
                tpv = accepted(s.tag[ci]) ? s.tape[ci] : (uint8_t)0;
            }
            const int hedge = dir < 0 ? 0 : kTile - 1;
            const int hx = axis == 0 ? hedge : u + 1;
            const int hy = axis == 1 ? hedge : (axis == 0 ? u + 1 : v + 1);
            const int hz = axis == 2 ? hedge : v + 1;
            const int hti = hx + kTile * hy + kTile * kTile * hz;
            W.T[hti] = tv;
            W.mu[hti] = mv;
            W.tp[hti] = tpv;
        }
        __syncwarp();

        // ---- rounds over the cells still to do ------------------------------
        // The first round tests every cell still to do; later rounds only the
        // neighbours of the cells done in the round before (a cell becomes
        // ready when its last downwind neighbour is done; halo values are
        // fixed for the pass).  Every candidate is tested before any cell of
        // the round publishes, then the ready cells are compacted and
        // computed 32 at a time.  Two cells ready in one round never depend
        // on each other (a cell is ready only after all cells downwind of
        // it), so their order does not matter.
        unsigned face_done = 0;   // bit f: a done cell has an upwind cell across face f
        unsigned done_any = 0;
        unsigned cand = todo;
        const real wax[3] = {(real)1, (real)wy, (real)wz};
        for (;;) {
            unsigned ready_mask = 0;
            for (unsigned rest = cand; rest; rest &= rest - 1u) {
                const int k = __ffs(rest) - 1;
                // ready when every downwind neighbour has published: on
                // axis a, q = p - e_a (its upwind code 2 points at p) and
                // q = p + e_a (code 1)
                const int ti = tb_of(lx, lr, k);
                bool ready = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int qm = ti - off[a], qp = ti + off[a];
                    if (tape_axis(W.tp[qm], a) == 2 && is_nan_bits(W.mu[qm]))
                        ready = false;
                    if (tape_axis(W.tp[qp], a) == 1 && is_nan_bits(W.mu[qp]))
                        ready = false;
                }
                ready_mask |= (unsigned)ready << k;
            }
            // compact the ready cells (warp prefix sum of the lane counts)
            const int cnt = __popc(ready_mask);
            int pre = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, pre, o);
                if (lane >= o)
                    pre += t;
            }
            const int n_ready = __shfl_sync(FULL, pre, 31);
            ++rounds_total;
            if (n_ready == 0)
                break;
            pre -= cnt;
            for (unsigned m = ready_mask; m; m &= m - 1u)
                W.list[pre++] = (uint16_t)(lane + 32 * (__ffs(m) - 1));
            __syncwarp();
            for (int i0 = 0; i0 < n_ready; i0 += 32) {
                const int i = i0 + lane;
                if (i < n_ready) {
                    const int c = W.list[i];
                    const int ti = tile_of(c);
                    real lam = (real)0, dsum = (real)0;
                    const real Tp = W.T[ti];
                    // unequal cells: the terms of axis a carry
                    // w_a = (h / h_a)^2 (Eq. (2) with h_i per axis)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int qm = ti - off[a], qp = ti + off[a];
                        const real wa = (kAniso && a > 0) ? wax[a] : (real)1;
                        if (tape_axis(W.tp[qm], a) == 2) {
                            if constexpr (kAniso)
                                lam += wa * (W.mu[qm] * (W.T[qm] - Tp));
                            else
                                lam += W.mu[qm] * (W.T[qm] - Tp);
                        }
                        if (tape_axis(W.tp[qp], a) == 1) {
                            if constexpr (kAniso)
                                lam += wa * (W.mu[qp] * (W.T[qp] - Tp));
                            else
                                lam += W.mu[qp] * (W.T[qp] - Tp);
                        }
                        const int code = tape_axis(W.tp[ti], a);
                        if (code) {
                            if constexpr (kAniso)
                                dsum += wa * (Tp - W.T[code == 1 ? qm : qp]);
                            else
                                dsum += Tp - W.T[code == 1 ? qm : qp];
                        }
                    }
                    const int cx = c & 7, cy = (c >> 3) & 7, cz = c >> 6;
                    const int gi = bx * kB + cx, gj = by * kB + cy, gk = bz * kB + cz;
                    const long long nat = ((long long)gk * g.ny + gj) * g.nx + gi;
                    lam += dLdT[nat];
                    const real m = positive(dsum) ? adj_div(lam, dsum) : (real)0;
                    // s_p h^2 = sqrt(q) h with q = (h/F)^2
                    const real sh2 = kHetero ? adj_sqrt(spd[base + c]) * (real)h : sh2_const;
                    dlds[nat] = m * sh2;
                    W.mu[ti] = m;
                    const uint8_t tpc = W.tp[ti];
                    if (cx == 0 && tape_axis(tpc, 0) == 1) face_done |= 1u;
                    if (cx == 7 && tape_axis(tpc, 0) == 2) face_done |= 2u;
                    if (cy == 0 && tape_axis(tpc, 1) == 1) face_done |= 4u;
                    if (cy == 7 && tape_axis(tpc, 1) == 2) face_done |= 8u;
                    if (cz == 0 && tape_axis(tpc, 2) == 1) face_done |= 16u;
                    if (cz == 7 && tape_axis(tpc, 2) == 2) face_done |= 32u;
                }
            }
            __syncwarp();
            todo &= ~ready_mask;
            done_any |= ready_mask;
            cand = neighbour_mask(ready_mask, lane) & todo;
        }
        // ---- publish mu, wake the bricks that hold upwind neighbours ------
        for (unsigned mm = done_any; mm; mm &= mm - 1u) {
            const int k = __ffs(mm) - 1;
            mu_g[base + lane + 32 * k] = W.mu[tb_of(lx, lr, k)];
        }
        // the brick's new top: the largest |psi| of a cell still to do
        {
            unsigned long long tmax = 0ull;
            for (unsigned mm = todo; mm; mm &= mm - 1u) {
                const int k = __ffs(mm) - 1;
                const unsigned long long tb =
                    (unsigned long long)__double_as_longlong((double)W.T[tb_of(lx, lr, k)]);
                tmax = tb > tmax ? tb : tmax;
            }
            const unsigned hi = __reduce_max_sync(FULL, (unsigned)(tmax >> 32));
            const unsigned lo = __reduce_max_sync(FULL, (unsigned)(tmax >> 32) == hi ? (unsigned)tmax : 0u);
            if (lane == 0)
                top[b] = ((unsigned long long)hi << 32) | lo;
        }
        __threadfence();
        face_done = __reduce_or_sync(FULL, face_done);
        if (lane < kFaces && ((face_done >> lane) & 1u)) {
            const int f = lane, axis = f >> 1, dir = (f & 1) ? 1 : -1;
            const int nbx = bx + (axis == 0 ? dir : 0);
            const int nby = by + (axis == 1 ? dir : 0);
            const int nbz = bz + (axis == 2 ? dir : 0);
            if (nbx >= 0 && nbx < g.nbx && nby >= 0 && nby < g.nby && nbz >= 0 && nbz < g.nbz) {
                const long long nb = ((long long)nbz * g.nby + nby) * g.nbx + nbx;
                atomicExch(&s.dirty[nb], 1u);
                __threadfence();
                // started only once the level reaches its top; a later level's
                // seed starts it otherwise
                if (vloadu(&top[nb]) >= level && atomicCAS(&s.queued[nb], 0u, 1u) == 0u) {
                    atomicAdd(&ctrl->pending, 1);
                    queue_push(ctrl, s.queue, cap, nb);
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            // end of the pass: queue the brick again if a flag arrived meanwhile
            atomicExch(&s.queued[b], 0u);
            __threadfence();
            if (vload((const int *)&s.dirty[b]) != 0 && vloadu(&top[b]) >= level &&
                atomicCAS(&s.queued[b], 0u, 1u) == 0u) {
                atomicAdd(&ctrl->pending, 1);
                queue_push(ctrl, s.queue, cap, b);
            }
            __threadfence();
            atomicAdd(&ctrl->pending, -1);
            ++passes;
        }
        __syncwarp();
    }
    if (lane == 0 && passes) {
        atomicAdd(&ctrl->marches, passes);
        atomicAdd(&ctrl->rounds, rounds_total);
    }
}

// Cells still waiting after the iteration (should be none).
template <typename real>
__global__ void k_adj_count_pending(long long n, const real *__restrict__ mu, unsigned *count)
{
    unsigned c = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        c += mu[e] != mu[e];
    c = __reduce_add_sync(FULL, c);
    if ((threadIdx.x & 31) == 0 && c)
        atomicAdd(count, c);
}

template <typename real>
size_t adj_smem() { return sizeof(AdjTile<real>) * kAdjWarps; }

template <typename real>
cudaError_t adj_persistent_launch(const Geom &g, const DeviceState &s, const AdjointArgs &a,
                                  unsigned long long level, cudaStream_t st)
{
    const size_t sm = adj_smem<real>();
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto go = [&](auto H, auto A) {
        constexpr bool het = decltype(H)::value, an = decltype(A)::value;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_persistent<real, het, an>,
                                                      kAdjWarps * 32, sm);
        const int ctas = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        k_adj_persistent<real, het, an><<<ctas, kAdjWarps * 32, sm, st>>>(
            g, s, (const real *)a.dLdT, (real *)a.dlds, (real *)a.mu, (unsigned long long *)a.top, level,
            a.h, a.spd_term, a.wy, a.wz);
    };
    using Y = std::true_type;
    using N = std::false_type;
    const bool het = s.spd != nullptr, an = a.aniso != 0;
    if (het)
        an ? go(Y{}, Y{}) : go(Y{}, N{});
    else
        an ? go(N{}, Y{}) : go(N{}, N{});
    return cudaGetLastError();
}

template <typename real>
void adj_configure()
{
    const int sm = (int)adj_smem<real>();
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaFuncSetAttribute(k_adj_persistent<real, true, false>, attr, sm);
    cudaFuncSetAttribute(k_adj_persistent<real, false, false>, attr, sm);
    cudaFuncSetAttribute(k_adj_persistent<real, true, true>, attr, sm);
    cudaFuncSetAttribute(k_adj_persistent<real, false, true>, attr, sm);
}

int grid_cap(long long n, int threads, int cap)
{
    long long b = (n + threads - 1) / threads;
    if (b < 1)
        b = 1;
    return (int)(b > cap ? cap : b);
}

}  // namespace

cudaError_t launch_adjoint_init(int dtype, const Geom &g, const DeviceState &s,
                                const AdjointArgs &a, cudaStream_t st)
{
    const int nb = grid_cap(g.nbricks * kB3, 256, 152 * 32);
    cudaMemsetAsync(a.top, 0, (size_t)g.nbricks * sizeof(unsigned long long), st);
    if (dtype == 1) {
        adj_configure<double>();
        k_adj_init<double><<<nb, 256, 0, st>>>(g, (const double *)s.T, s.tag, (double *)a.mu,
                                               (double *)a.dlds, (unsigned long long *)a.top);
    } else {
        adj_configure<float>();
        k_adj_init<float><<<nb, 256, 0, st>>>(g, (const float *)s.T, s.tag, (float *)a.mu,
                                              (float *)a.dlds, (unsigned long long *)a.top);
    }
    return cudaGetLastError();
}

cudaError_t adjoint_top_max(int, const Geom &g, const AdjointArgs &a, double *out, cudaStream_t st)
{
    // the control block's second minimum word serves as the scratch word
    unsigned long long *w = &a.ctrl->minbits[1];
    cudaMemsetAsync(w, 0, sizeof(unsigned long long), st);
    k_adj_top_max<<<grid_cap(g.nbricks, 256, 1024), 256, 0, st>>>(g.nbricks,
                                                                   (const unsigned long long *)a.top, w);
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, w, sizeof(v), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return e;
    memcpy(out, &v, sizeof(v));
    return cudaGetLastError();
}

cudaError_t launch_adjoint_levels(int dtype, const Geom &g, const DeviceState &s,
                                  const AdjointArgs &a, double top_max, double step, int levels,
                                  cudaStream_t st)
{
    const int nb = grid_cap(g.nbricks, 256, 152 * 32);
    auto bits = [](double v) {
        unsigned long long b;
        memcpy(&b, &v, sizeof(b));
        return b;
    };
    for (int k = 0; k < levels; ++k) {
        // level k: tops in [top_max - (k + 1) step, top_max - k step); the
        // first level is open above, the last one reaches down to 0
        const double lo_v = k == levels - 1 ? 0.0 : top_max - (double)(k + 1) * step;
        const unsigned long long lo = bits(lo_v > 0.0 ? lo_v : 0.0);
        const unsigned long long hi = k == 0 ? ~0ull : bits(top_max - (double)k * step);
        k_adj_level_reset<<<1, 1, 0, st>>>(s.ctrl);
        k_adj_seed_level<<<nb, 256, 0, st>>>(g, (const unsigned long long *)a.top, lo, hi, s.ctrl,
                                             s.queued, s.queue);
        const cudaError_t e = dtype == 1 ? adj_persistent_launch<double>(g, s, a, lo, st)
                                         : adj_persistent_launch<float>(g, s, a, lo, st);
        if (e != cudaSuccess)
            return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_pending(int dtype, const Geom &g, const AdjointArgs &a, unsigned *count,
                                   cudaStream_t st)
{
    const long long n = g.nbricks * kB3;
    const int nb = grid_cap(n, 256, 152 * 32);
    if (dtype == 1)
        k_adj_count_pending<double><<<nb, 256, 0, st>>>(n, (const double *)a.mu, count);
    else
        k_adj_count_pending<float><<<nb, 256, 0, st>>>(n, (const float *)a.mu, count);
    return cudaGetLastError();
}

}  // namespace fmmgb
