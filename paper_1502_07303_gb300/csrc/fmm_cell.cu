// fmm_cell.cu -- the cell-parallel march (schedule 4) and the interface
// initialisation from given values.
//
// The cell-parallel march runs Algorithms 9-12 over the whole grid without
// bricks, halos or queues: one bucket step accepts, on each side, every BAND
// cell at or below min(m + delta, width_band) (m the side's smallest BAND
// value, delta the bucket width of the cell's brick), then every cell next to
// a cell accepted in this step and above it is solved again (Algorithm 10:
// Algorithm 11 from the current values, Jacobi within the step: the solves
// read the state and write a second buffer), and the improvements are applied
// (an improved cell is BAND again, so an accepted value that drops is
// corrected, as in the label-correcting brick march).  The step that finds no
// BAND cell at or below width_band on either side ends the march.  For the
// first-order scheme of Eq. (2)-(3) the result is the unique discrete solution
// the heap march of Algorithm 12 reaches (Sec. 5.2).
//
// accuracy 2 is the higher-order fast marching that Sec. 6 names as future
// work, in the textbook second-order form: on an upwind axis whose next cell
// beyond the neighbour psi1, in the same direction, is known with
// psi2 <= psi1, the one-sided difference (3 t - 4 psi1 + psi2) / (2 h)
// replaces (t - psi1) / h, i.e. Algorithm 11 runs with psi_i = (4 psi1 -
// psi2) / 3 and the axis weight (3/2)^2.  That update is not monotone in its
// operands (a larger psi2 lowers the root, and a cell keeps the smallest of
// its roots), so a second neighbour must hold its final value when it is
// read: the second-order march runs with buckets narrower than the smallest
// single-axis increment (fmm_internal.h, kSecondOrderBucket), so that a cell
// and its upwind neighbour are not accepted in the same step, as in the
// sequential march where every KNOWN value is final.  The acceptance order
// still differs from the heap's, so this march and the sequential one reach
// different second-order solutions in general (both reproduce quadratic
// solutions to rounding).
//
// Every kernel is a grid-stride loop over the brick-layout cells with no
// device-side wait; the host enqueues steps in batches and reads the
// termination flag between batches.
#include "fmm_internal.h"

namespace fmmgb {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kCellThreads = 256;
constexpr uint8_t TG_ACC = 16;   // accepted in the current bucket step
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

template <typename real>
__device__ __forceinline__ real inf_r();
template <>
__device__ __forceinline__ float inf_r<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double inf_r<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

// the "no new value" mark of the second buffer (all bits set: a NaN)
template <typename real>
__device__ __forceinline__ real none_r();
template <>
__device__ __forceinline__ float none_r<float>() { return __int_as_float(-1); }
template <>
__device__ __forceinline__ double none_r<double>() { return __longlong_as_double(-1ll); }

__device__ __forceinline__ float vsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double vsqrt(double v) { return sqrt(v); }

__device__ __forceinline__ bool known(uint8_t t) { return (t & ST_MASK) >= ST_KNOWN; }

// a < b and a <= b for values >= 0 (+inf included) on their bit patterns:
// integer compares, off the FP64 pipe that runs at 1/64 of the float rate
__device__ __forceinline__ bool blt(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
__device__ __forceinline__ bool blt(float a, float b) { return __float_as_int(a) < __float_as_int(b); }
__device__ __forceinline__ bool ble(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }
__device__ __forceinline__ bool ble(float a, float b) { return __float_as_int(a) <= __float_as_int(b); }
// |v| with the sign bit cleared (-0 becomes +0, which the compares above
// need)
__device__ __forceinline__ double abs_bits(double v) { return __longlong_as_double(__double_as_longlong(v) & 0x7fffffffffffffffll); }
__device__ __forceinline__ float abs_bits(float v) { return __int_as_float(__float_as_int(v) & 0x7fffffff); }
// the "no new value" mark (all bits set)
__device__ __forceinline__ bool is_none(double v) { return __double_as_longlong(v) == -1ll; }
__device__ __forceinline__ bool is_none(float v) { return __float_as_int(v) == -1; }

// Natural coordinates of brick-layout cell e (32-bit divisions: the brick
// count of a grid of at most 2^20 cells per axis that fits in memory is far
// below 2^32).
__device__ __forceinline__ void cell_ijk(const Geom &g, long long e, int &i, int &j, int &k)
{
    const unsigned b = (unsigned)(e >> 9);
    const int c = (int)(e & 511);
    const unsigned nbx = (unsigned)g.nbx, nby = (unsigned)g.nby;
    const int bx = (int)(b % nbx);
    const unsigned r = b / nbx;
    const int by = (int)(r % nby);
    const int bz = (int)(r / nby);
    i = bx * kB + (c & 7);
    j = by * kB + ((c >> 3) & 7);
    k = bz * kB + (c >> 6);
}

// Brick-layout index of natural cell (i, j, k) (inside the grid).
__device__ __forceinline__ long long cell_at(const Geom &g, int i, int j, int k)
{
    const long long b = ((long long)(k >> 3) * g.nby + (j >> 3)) * g.nbx + (i >> 3);
    return b * kB3 + (i & 7) + 8 * (j & 7) + 64 * (k & 7);
}

// The cell `steps` cells from (i, j, k) along axis a (direction sign of
// steps), or -1 outside the grid.
__device__ __forceinline__ long long cell_along(const Geom &g, int i, int j, int k, int a, int steps)
{
    int c[3] = {i, j, k};
    const int ext[3] = {g.nx, g.ny, g.nz};
    c[a] += steps;
    if (c[a] < 0 || c[a] >= ext[a])
        return -1;
    return cell_at(g, c[0], c[1], c[2]);
}

// Algorithm 11 for the active axes (act bit a), values psi[a] and weights
// W[a] = (h / h_a)^2 (times (3/2)^2 on a second-order axis), speed term
// q = (h/F)^2: the quadratic sum_a W_a (t - psi_a)^2 = q for the unknown
// shifted by the smallest value, t = m + u, solved for the nested sets that
// drop the largest psi (ties: the higher axis) while non-empty; the smallest
// causal root (every psi_a < t), or +inf.
template <typename real>
__device__ real cell_root(const real psi[3], const real W[3], unsigned act, real q)
{
    real m = inf_r<real>();
    int nd = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if ((act >> a) & 1u) {
            ++nd;
            m = psi[a] < m ? psi[a] : m;
        }
    real best = inf_r<real>();
    for (; nd > 0; --nd) {
        real d[3], w[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const bool on = (act >> a) & 1u;
            d[a] = on ? psi[a] - m : (real)0;
            w[a] = on ? W[a] : (real)0;
        }
        const real qa = (w[0] + w[1]) + w[2];
        const real qb = (real)-2 * ((w[0] * d[0] + w[1] * d[1]) + w[2] * d[2]);
        const real qc = ((w[0] * d[0] * d[0] + w[1] * d[1] * d[1]) + w[2] * d[2] * d[2]) - q;
        const real disc = qb * qb - (real)4 * qa * qc;
        if (disc >= (real)0) {
            const real u = (-qb + vsqrt(disc)) / ((real)2 * qa);
            if (d[0] < u && d[1] < u && d[2] < u) {
                const real t = m + u;
                best = t < best ? t : best;
            }
        }
        int j = -1;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (((act >> a) & 1u) && (j < 0 || psi[a] >= psi[j]))
                j = a;
        act &= ~(1u << j);
    }
    return best;
}

// Interface initialisation from given values (Algorithm 8 with the values of
// the interface cells supplied): a finite T0 makes the cell FIX with |T0| on
// the side of its sign (-0 and +0 are side +1), +-inf a FAR cell of that
// side.  NaN, or a non-FIX cell next to a cell of the other side (Algorithm
// 8 puts FIX cells at both ends of every sign change), sets ERR_INPUT.
template <typename real>
__global__ void __launch_bounds__(kCellThreads) k_init_fixed(Geom g, const real *__restrict__ T0, real *T,
                                                            uint8_t *tag, Control *ctrl)
{
    const long long n = g.nbricks * kB3;
    bool bad = false;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(g, e, i, j, k);
        if (i >= g.nx || j >= g.ny || k >= g.nz) {
            T[e] = inf_r<real>();
            tag[e] = TG_OUT | ST_FAR;
            continue;
        }
        const long long p = ((long long)k * g.ny + j) * g.nx + i;
        const real v = T0[p];
        const bool neg = v < (real)0;
        if (v != v) {
            bad = true;
            T[e] = inf_r<real>();
            tag[e] = ST_FAR;
            continue;
        }
        const bool fixed = v > -inf_r<real>() && v < inf_r<real>();
        T[e] = fixed ? abs_bits(v) : inf_r<real>();
        tag[e] = (uint8_t)((fixed ? ST_FIX : ST_FAR) | (neg ? TG_NEG : 0));
        if (!fixed) {
            const int c[3] = {i, j, k};
            const int ext[3] = {g.nx, g.ny, g.nz};
            const long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (c[a] > 0 && (T0[p - st[a]] < (real)0) != neg)
                    bad = true;
                if (c[a] + 1 < ext[a] && (T0[p + st[a]] < (real)0) != neg)
                    bad = true;
            }
        }
    }
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0)
        atomicOr(&ctrl->error, ERR_INPUT);
}

// Start of the march: the FIX cells count as accepted (Algorithm 9 updates
// the neighbours of every FIX cell), the step minima are reset and the
// second buffer is marked empty.
template <typename real>
__global__ void __launch_bounds__(kCellThreads) k_cell_seed(Geom g, uint8_t *tag, real *next,
                                                           unsigned long long *mins)
{
    const long long n = g.nbricks * kB3;
    if (blockIdx.x == 0 && threadIdx.x < 4)
        mins[threadIdx.x] = kInfBits;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        next[e] = none_r<real>();
        const uint8_t t = tag[e];
        if ((t & ST_MASK) == ST_FIX && !(t & TG_OUT))
            tag[e] = t | TG_ACC;
    }
}

// Accept the bucket of each side: the BAND cells at or below
// min(m + bucket * bdelta, width) with m the side's smallest BAND value
// (slot `slot` of mins); ends the march when no side has a BAND cell at or
// below width.  Also resets the other slot, which the apply kernel of this
// step fills.
template <typename real>
__global__ void __launch_bounds__(kCellThreads) k_cell_accept(Geom g, const real *__restrict__ T, uint8_t *tag,
                                                             const real *__restrict__ bdelta, double bucket,
                                                             double width, unsigned long long *mins, int slot,
                                                             Control *ctrl)
{
    if (ctrl->done)
        return;
    const double m0 = __longlong_as_double((long long)mins[2 * slot]);
    const double m1 = __longlong_as_double((long long)mins[2 * slot + 1]);
    const double inf = __longlong_as_double((long long)kInfBits);
    const bool has0 = m0 < inf && m0 <= width, has1 = m1 < inf && m1 <= width;
    if (!has0 && !has1) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            ctrl->done = 1;
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        mins[2 * (slot ^ 1)] = kInfBits;
        mins[2 * (slot ^ 1) + 1] = kInfBits;
        ctrl->restart += 1;
    }
    const long long n = g.nbricks * kB3;
    unsigned acc = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const uint8_t t = tag[e];
        if ((t & ST_MASK) != ST_BAND || (t & TG_OUT))
            continue;
        const bool neg = (t & TG_NEG) != 0;
        if (!(neg ? has0 : has1))
            continue;
        const double lim = fmin((neg ? m0 : m1) + bucket * (double)bdelta[e >> 9], width);
        if ((double)T[e] <= lim) {
            tag[e] = (uint8_t)((t & ~ST_MASK) | ST_KNOWN | TG_ACC);
            ++acc;
        }
    }
    acc = __reduce_add_sync(FULL, acc);
    if ((threadIdx.x & 31) == 0 && acc)
        atomicAdd(&ctrl->accepted, (unsigned long long)acc);
}

// Algorithm 10 for the cells next to a cell accepted in this step: a non-FIX
// cell above an accepted neighbour is solved again from the current values
// (Algorithm 11: per axis the smaller known neighbour below the cell, the
// minus one on a tie; with kAcc = 2 the second-order difference where the
// cell beyond it is known and not above it); a smaller root goes to next.
template <typename real, int kAcc>
__global__ void __launch_bounds__(kCellThreads) k_cell_relax(Geom g, const real *__restrict__ T,
                                                            const uint8_t *__restrict__ tag,
                                                            const real *__restrict__ spd, double spd_const,
                                                            double wy, double wz, real *next, Control *ctrl)
{
    if (ctrl->done)
        return;
    const long long n = g.nbricks * kB3;
    const real wax[3] = {(real)1, (real)wy, (real)wz};
    unsigned solves = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const uint8_t t = tag[e];
        if ((t & TG_OUT) || (t & ST_MASK) == ST_FIX)
            continue;
        int i, j, k;
        cell_ijk(g, e, i, j, k);
        const real Tc = T[e];
        long long nb[6];
        bool trig = false;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            nb[q] = cell_along(g, i, j, k, q >> 1, (q & 1) ? 1 : -1);
            if (nb[q] >= 0 && (tag[nb[q]] & TG_ACC) && blt(T[nb[q]], Tc))
                trig = true;
        }
        if (!trig)
            continue;
        ++solves;
        real psi[3] = {(real)0, (real)0, (real)0}, W[3] = {(real)0, (real)0, (real)0};
        unsigned act = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const long long qm = nb[2 * a], qp = nb[2 * a + 1];
            const bool km = qm >= 0 && known(tag[qm]), kp = qp >= 0 && known(tag[qp]);
            const real vm = km ? T[qm] : inf_r<real>(), vp = kp ? T[qp] : inf_r<real>();
            int d = 0;
            if (km && blt(vm, Tc))
                d = -1;
            if (kp && blt(vp, Tc)) {
                if (d == 0)
                    d = 1;
                else if (blt(vp, vm))
                    d = 1;
            }
            if (d == 0)
                continue;
            act |= 1u << a;
            psi[a] = d < 0 ? vm : vp;
            W[a] = wax[a];
            if (kAcc == 2) {
                const long long q2 = cell_along(g, i, j, k, a, 2 * d);
                if (q2 >= 0 && known(tag[q2])) {
                    const real v2 = T[q2];
                    if (ble(v2, psi[a])) {
                        psi[a] = ((real)4 * psi[a] - v2) / (real)3;
                        W[a] = W[a] * (real)2.25;
                    }
                }
            }
        }
        const real q = spd ? spd[e] : (real)spd_const;
        const real r = cell_root<real>(psi, W, act, q);
        if (blt(r, Tc))
            next[e] = r;
    }
    solves = __reduce_add_sync(FULL, solves);
    if ((threadIdx.x & 31) == 0 && solves)
        atomicAdd(&ctrl->solves, (unsigned long long)solves);
}

// Apply the step's new values (the cell becomes BAND), clear the accepted
// marks, and reduce the smallest BAND value of each side into slot `slot`.
template <typename real>
__global__ void __launch_bounds__(kCellThreads) k_cell_apply(Geom g, real *T, uint8_t *tag, real *next,
                                                            unsigned long long *mins, int slot, Control *ctrl)
{
    if (ctrl->done)
        return;
    const long long n = g.nbricks * kB3;
    real l0 = inf_r<real>(), l1 = inf_r<real>();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const uint8_t t = tag[e];
        if (t & TG_OUT)
            continue;
        uint8_t nt = (uint8_t)(t & ~TG_ACC);
        real v = T[e];
        const real nv = next[e];
        if (!is_none(nv)) {
            v = nv;
            T[e] = nv;
            next[e] = none_r<real>();
            nt = (uint8_t)((nt & ~ST_MASK) | ST_BAND);
        }
        if (nt != t)
            tag[e] = nt;
        if ((nt & ST_MASK) == ST_BAND) {
            if (nt & TG_NEG)
                l0 = blt(v, l0) ? v : l0;
            else
                l1 = blt(v, l1) ? v : l1;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const real a = __shfl_xor_sync(FULL, l0, o), b = __shfl_xor_sync(FULL, l1, o);
        l0 = blt(a, l0) ? a : l0;
        l1 = blt(b, l1) ? b : l1;
    }
    if ((threadIdx.x & 31) == 0) {
        if (blt(l0, inf_r<real>()))
            atomicMin(&mins[2 * slot], (unsigned long long)__double_as_longlong((double)l0));
        if (blt(l1, inf_r<real>()))
            atomicMin(&mins[2 * slot + 1], (unsigned long long)__double_as_longlong((double)l1));
    }
}

int cell_grid(long long n)
{
    long long b = (n + kCellThreads - 1) / kCellThreads;
    const long long cap = 152LL * 16;
    if (b < 1)
        b = 1;
    return (int)(b > cap ? cap : b);
}

template <typename real>
void relax_launch(const Geom &g, const DeviceState &s, const SolveParams &p, void *next, int nb,
                  cudaStream_t st)
{
    const real *spd = (const real *)s.spd;
    if (p.accuracy == 2)
        k_cell_relax<real, 2><<<nb, kCellThreads, 0, st>>>(g, (const real *)s.T, s.tag, spd, p.spd_term,
                                                           p.wy, p.wz, (real *)next, s.ctrl);
    else
        k_cell_relax<real, 1><<<nb, kCellThreads, 0, st>>>(g, (const real *)s.T, s.tag, spd, p.spd_term,
                                                           p.wy, p.wz, (real *)next, s.ctrl);
}

template <typename real>
cudaError_t begin_t(const Geom &g, const DeviceState &s, const SolveParams &p, void *next,
                    unsigned long long *mins, cudaStream_t st)
{
    const int nb = cell_grid(g.nbricks * kB3);
    k_cell_seed<real><<<nb, kCellThreads, 0, st>>>(g, s.tag, (real *)next, mins);
    relax_launch<real>(g, s, p, next, nb, st);
    k_cell_apply<real><<<nb, kCellThreads, 0, st>>>(g, (real *)s.T, s.tag, (real *)next, mins, 0, s.ctrl);
    return cudaGetLastError();
}

template <typename real>
cudaError_t step_t(const Geom &g, const DeviceState &s, const SolveParams &p, void *next,
                   unsigned long long *mins, long long step, cudaStream_t st)
{
    const int nb = cell_grid(g.nbricks * kB3);
    const int slot = (int)(step & 1);
    k_cell_accept<real><<<nb, kCellThreads, 0, st>>>(g, (const real *)s.T, s.tag, (const real *)s.bdelta,
                                                     p.bucket, p.width, mins, slot, s.ctrl);
    relax_launch<real>(g, s, p, next, nb, st);
    k_cell_apply<real><<<nb, kCellThreads, 0, st>>>(g, (real *)s.T, s.tag, (real *)next, mins, slot ^ 1,
                                                    s.ctrl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init_fixed(int dtype, const Geom &g, const DeviceState &s, const void *T0,
                              cudaStream_t st)
{
    const int nb = cell_grid(g.nbricks * kB3);
    if (dtype == 1)
        k_init_fixed<double><<<nb, kCellThreads, 0, st>>>(g, (const double *)T0, (double *)s.T, s.tag, s.ctrl);
    else
        k_init_fixed<float><<<nb, kCellThreads, 0, st>>>(g, (const float *)T0, (float *)s.T, s.tag, s.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_cell_begin(int dtype, const Geom &g, const DeviceState &s, const SolveParams &p,
                              void *next, unsigned long long *mins, cudaStream_t st)
{
    return dtype == 1 ? begin_t<double>(g, s, p, next, mins, st) : begin_t<float>(g, s, p, next, mins, st);
}

cudaError_t launch_cell_step(int dtype, const Geom &g, const DeviceState &s, const SolveParams &p,
                             void *next, unsigned long long *mins, long long step, cudaStream_t st)
{
    return dtype == 1 ? step_t<double>(g, s, p, next, mins, step, st)
                      : step_t<float>(g, s, p, next, mins, step, st);
}

}  // namespace fmmgb
